"""Plain FP64 CPU oracle for the singles-and-doubles Quantum Flow sweep.

TEST INFRASTRUCTURE ONLY.  Nothing in the product path imports, links or runs this
package: only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may use it.  It shares no code with the CUDA library; the only module both
sides use is the seeded input generator ``paper_2606_04186_gb300.synth``.

Modules (each function cites the passage of the paper it follows):

* ``secondq``   second quantisation on bit-string determinants: spin-summed E_pq, H and T
                applied to vectors, exact e^{-T} H e^{T} (definition-level engine).
* ``hbar_brute`` the normal-ordered 0/1/2-body parts of e^{-T} H e^{T} read off exact
                Fock-space matrix elements (definition of the dressed Hamiltonian, tiny n).
* ``hbar``      closed-form spin-free H-bar (<= two-body) for a closed-shell reference:
                the dressing step of the flow at any size.
* ``ccsd``      closed-shell CCSD / MP2 reference energies.
* ``fci``       determinant full CI.
* ``cas``       active-space operator, its Phi-dominant root and the CI -> CC increment.
* ``flow``      Delta-epsilon ordering, owner map, Jacobi sweep, mean energy, DIIS.
* ``mlp``       FP64 reference of the warm-start network (forward, backward, Adam).

Parity-pin status of each function is stated in its docstring.
"""
