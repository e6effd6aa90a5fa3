"""GB300-native data-parallel hot path of the singles-and-doubles Quantum Flow sweep.

Importing the package is cheap: the CUDA library is loaded on first use of
``paper_2606_04186_gb300.qflow``.  ``synth`` holds the seeded input generators.
"""
