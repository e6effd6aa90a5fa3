"""CUDA path vs the FP64 oracle, element by element, through the C ABI.

Tolerances: plain FP64 path |dE| <= 1e-8 Eh per space and max |dt| <= 1e-7 (the flow's own
convergence thresholds); mixed path (FP32 sigma) |dE| <= 1e-6 Eh and |dt| <= 1e-5.
"""
import numpy as np
import pytest

from oracle import cas, ccsd, flow, hbar
from paper_2606_04186_gb300 import synth

from gpu_util import mixed_flow_w, dev, library

pytestmark = pytest.mark.gpu

TOL = {"fp64": (1e-8, 1e-7), "mixed": (1e-6, 1e-5)}


@pytest.fixture(scope="module")
def qf():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    return library()


def _pool(no, nv, seed=3, s1=0.01, s2=0.02):
    return synth.random_amplitudes(no, nv, seed, s1, s2)


@pytest.mark.parametrize("name", ["n10", "n24"])
def test_dress_matches_oracle(qf, name):
    import torch
    eps, h, g, _ = synth.system_inputs(name, with_spaces=False)
    s = synth.SYSTEMS[name]
    no, nv = s.nocc, s.n - s.nocc
    t1, t2 = _pool(no, nv)
    e0 = torch.zeros(1, dtype=torch.float64, device="cuda")
    F = torch.zeros((s.n, s.n), dtype=torch.float64, device="cuda")
    W = torch.zeros((s.n,) * 4, dtype=torch.float64, device="cuda")
    work = torch.zeros(qf.dress_workspace(s.n, no), dtype=torch.uint8, device="cuda")
    qf.dress_device(dev(h), dev(g), dev(t1), dev(t2), no, e0, F, W, work)
    torch.cuda.synchronize()
    e0r, Fr, Wr = hbar.hbar2(h, g, t1, t2, no)
    assert abs(e0.item() - e0r) < 1e-11
    assert np.abs(F.cpu().numpy() - Fr).max() < 1e-11
    assert np.abs(W.cpu().numpy() - Wr).max() < 1e-11


def _solve_on_gpu(qf, n, no, e0, F, W, k, spaces, own1, own2, t1, t2, precision):
    import torch
    ns = len(spaces)
    energy = torch.zeros(ns, dtype=torch.float64, device="cuda")
    status = torch.full((ns,), -1, dtype=torch.int32, device="cuda")
    iters = torch.zeros(ns, dtype=torch.int32, device="cuda")
    t1o, t2o = dev(t1), dev(t2)
    t1n, t2n = t1o.clone(), t2o.clone()
    qf.solve_device(n, no, dev(np.array([e0])), dev(F), dev(W), k, dev(spaces), energy, status, iters,
                    owner1=dev(own1.astype(np.int32)), owner2=dev(own2.astype(np.int32)), t1_old=t1o, t2_old=t2o,
                    t1_new=t1n, t2_new=t2n, precision=precision)
    torch.cuda.synchronize()
    return (energy.cpu().numpy(), status.cpu().numpy(), iters.cpu().numpy(), t1n.cpu().numpy(), t2n.cpu().numpy())


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
@pytest.mark.parametrize("k", [1, 2, 3])
def test_solver_on_oracle_hbar(qf, k, precision):
    eps, h, g, _ = synth.system_inputs("n10", with_spaces=False)
    n, no = 10, 3
    t1, t2 = _pool(no, n - no, 7)
    e0, F, W = hbar.hbar2(h, g, t1, t2, no)
    sp = synth.all_spaces(n, no, k, k)
    perm = flow.sort_spaces(sp, ccsd.fock_diagonal(h, g, no))
    sps = sp[perm]
    own1, own2 = flow.owner_maps(sps, no, n - no)
    E, st, it, t1n, t2n = _solve_on_gpu(qf, n, no, e0, F, W, k, sps, own1, own2, t1, t2, precision)
    ref = flow.solve_all(e0, F, W, sps)
    Er = np.array([r[0] for r in ref])
    t1r, t2r = flow.merge(t1, t2, sps, ref, own1, own2, no)
    te, tt = TOL[precision]
    assert (st == 0).all(), st
    assert np.abs(E - Er).max() < te
    assert np.abs(t1n - t1r).max() < tt and np.abs(t2n - t2r).max() < tt
    assert np.abs(t2n - t2n.transpose(1, 0, 3, 2)).max() < 1e-12
    assert it.max() < 60


def test_solver_skips_malformed_and_empty(qf):
    import torch
    eps, h, g, _ = synth.system_inputs("n10", with_spaces=False)
    e0, F, W = hbar.hbar2(h, g, np.zeros((3, 7)), np.zeros((3, 3, 7, 7)), 3)
    sp = synth.all_spaces(10, 3)[:4].copy()
    sp[1, 0] = 2           # wrong size class
    sp[2, 5] = 2           # virtual slot holding an occupied index
    E, st, it, _, _ = _solve_on_gpu(qf, 10, 3, e0, F, W, 3, sp, np.full((3, 7), -1), np.full((3, 3, 7, 7), -1),
                                    np.zeros((3, 7)), np.zeros((3, 3, 7, 7)), "fp64")
    assert list(st) == [0, 4, 4, 0]
    energy = torch.zeros(1, dtype=torch.float64, device="cuda")
    status = torch.zeros(1, dtype=torch.int32, device="cuda")
    qf.solve_device(10, 3, dev(np.array([e0])), dev(F), dev(W), 3, dev(sp[:0]), energy, status)


def test_flow_sweeps_match_oracle_fp64(qf):
    eps, h, g, sp = synth.system_inputs("n10")
    ref = flow.Flow(h, g, 3, sp)
    gpu = qf.Flow(h, g, 3, sp, precision="fp64")
    assert np.array_equal(gpu.order(), ref.perm)
    for sweep in range(4):
        er, der, dtr, _ = ref.sweep()
        de, dt, nf, code = gpu.sweep()
        e, per = gpu.energy(per_space=True)
        t1, t2 = gpu.amplitudes()
        assert nf == 0 and code == 0
        assert abs(e - er) < 1e-9
        assert np.abs(per - ref.energies).max() < 1e-9
        assert np.abs(t1 - ref.t1).max() < 1e-9 and np.abs(t2 - ref.t2).max() < 1e-9
        if sweep:
            assert abs(de - der) < 1e-9 and abs(dt - dtr) < 1e-9
    gpu.close()


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_flow_converges_to_ccsd(qf, precision):
    eps, h, g, sp = synth.system_inputs("n10")
    e_cc, t1c, t2c, _ = ccsd.ccsd(h, g, 3, tol=1e-13)
    gpu = qf.Flow(h, g, 3, sp, precision=precision)
    for _ in range(40):
        de, dt, nf, code = gpu.sweep()
        if abs(de) < 1e-10 and dt < 1e-9:
            break
    te, tt = TOL[precision]
    assert abs(gpu.energy() - e_cc) < (1e-9 if precision == "fp64" else te)
    t1, t2 = gpu.amplitudes()
    assert np.abs(t2 - t2c).max() < (1e-8 if precision == "fp64" else tt)
    gpu.close()


def test_ccsd_fixed_point_n24(qf):
    eps, h, g, sp = synth.system_inputs("n24")
    e_cc, t1c, t2c, _ = ccsd.ccsd(h, g, 5, tol=1e-12)
    gpu = qf.Flow(h, g, 5, sp, precision="fp64")
    gpu.set_amplitudes(t1c, t2c)
    de, dt, nf, code = gpu.sweep()
    e, per = gpu.energy(per_space=True)
    assert nf == 0 and dt < 1e-9
    assert np.abs(per - e_cc).max() < 1e-9
    gpu.close()


@pytest.mark.parametrize("name,precision", [("n24", "fp64"), ("n24", "mixed"), ("n40", "fp64"), ("n40", "mixed")])
def test_sampled_spaces_full_list(qf, name, precision):
    """Full space lists on the GPU; a seeded sample of spaces recomputed by the oracle."""
    eps, h, g, sp = synth.system_inputs(name)
    s = synth.SYSTEMS[name]
    no, nv = s.nocc, s.n - s.nocc
    t1, t2 = _pool(no, nv, 11, 0.01, 0.015)
    gpu = qf.Flow(h, g, no, sp, precision=precision)
    gpu.set_amplitudes(t1, t2)
    gpu.sweep()
    e, per = gpu.energy(per_space=True)
    t1n, t2n = gpu.amplitudes()
    perm = gpu.order()
    sps = sp[perm]
    e0, F, W = hbar.hbar2(h, g, t1, t2, no)
    own1, own2 = flow.owner_maps(sps, no, nv)
    rng = np.random.default_rng(5)
    te, tt = TOL[precision]
    for s_idx in rng.choice(len(sps), size=40, replace=False):
        occ, vir = flow.space_orbitals(sps[s_idx])
        er, x1, x2, st = cas.solve_space(e0, F, W, occ, vir)
        assert abs(per[s_idx] - er) < te
        va = [a - no for a in vir]
        for ii, i in enumerate(occ):
            for aa, a in enumerate(va):
                if own1[i, a] == s_idx:
                    assert abs(t1n[i, a] - (t1[i, a] + x1[ii, aa])) < tt
            for jj, j in enumerate(occ):
                for aa, a in enumerate(va):
                    for bb, b in enumerate(va):
                        if own2[i, j, a, b] == s_idx:
                            assert abs(t2n[i, j, a, b] - (t2[i, j, a, b] + x2[ii, jj, aa, bb])) < tt
    # amplitudes nobody owns keep their value; mean energy is the mean of the space energies
    assert abs(e - per.mean()) < 1e-12 * max(1.0, abs(e))
    unowned1 = own1 < 0
    assert np.array_equal(t1n[unowned1], t1[unowned1])
    gpu.close()


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_previous_root_guess_same_result(qf, precision):
    # Starting each space from its previous root gives the same flow.  (It is not a cheaper
    # start here: the pool absorbs each root's increment, so the next root is closer to Phi.)
    eps, h, g, sp = synth.system_inputs("n24")
    a = qf.Flow(h, g, 5, sp, precision=precision, guess="phi")
    b = qf.Flow(h, g, 5, sp, precision=precision, guess="previous")
    te, tt = TOL[precision]
    for sweep in range(3):
        a.sweep()
        b.sweep()
        ea, pa = a.energy(per_space=True)
        eb, pb = b.energy(per_space=True)
        assert np.abs(pa - pb).max() < te
    ta, tb = a.amplitudes(), b.amplitudes()
    assert np.abs(ta[1] - tb[1]).max() < tt
    a.close()
    b.close()


def test_diis_flow_matches_oracle(qf):
    eps, h, g, sp = synth.system_inputs("n10")
    ref = flow.Flow(h, g, 3, sp, diis=True)
    gpu = qf.Flow(h, g, 3, sp, precision="fp64", diis=8)
    for sweep in range(6):
        er, der, dtr, _ = ref.sweep()
        de, dt, nf, code = gpu.sweep()
        assert abs(gpu.energy() - er) < 1e-9
        t1, t2 = gpu.amplitudes()
        assert np.abs(t2 - ref.t2).max() < 1e-8 and np.abs(t1 - ref.t1).max() < 1e-8
    e_cc, *_ = ccsd.ccsd(h, g, 3, tol=1e-13)
    for _ in range(20):
        de, dt, nf, code = gpu.sweep()
        if abs(de) < 1e-11 and dt < 1e-10:
            break
    assert abs(gpu.energy() - e_cc) < 1e-9
    gpu.close()


def test_mixed_dressing_close_to_oracle(qf):
    """Mixed path: FP64 integrals with FP32 T1 correction sums (E0 and the Fock blocks follow
    them to ~1e-10), T2 contractions on the tensor cores onto FP64 bases."""
    eps, h, g, sp = synth.system_inputs("n24")
    s = synth.SYSTEMS["n24"]
    no, nv = s.nocc, s.n - s.nocc
    t1, t2 = _pool(no, nv, 13, 0.01, 0.02)
    gpu = qf.Flow(h, g, no, sp, precision="mixed")
    gpu.set_amplitudes(t1, t2)
    e0, F, W = gpu.dressed()
    e0r, Fr, Wr = hbar.hbar2(h, g, t1, t2, no)
    assert abs(e0 - e0r) < 1e-9
    assert np.abs(F - Fr).max() < 1e-9
    # vvvv: dressed where at most three virtual indices differ (what the flow's spaces read)
    assert np.abs(mixed_flow_w(W, Wr, no) - Wr).max() < 1e-6
    gpu.close()


def test_schedules_and_graph_replay_agree(qf):
    """Per-class launches, the persistent queue and CUDA-graph replay compute the same sweep."""
    eps, h, g, sp = synth.system_inputs("n40")
    runs = {}
    for name, kw in [("per_class", dict(schedule="per_class", graph=False)),
                     ("persistent", dict(schedule="persistent", graph=False)),
                     ("persistent_12_warps", dict(schedule="persistent", graph=False, warps=12)),
                     ("per_class_7_warps", dict(schedule="per_class", graph=False, warps=7)),
                     ("persistent_chunk_4", dict(schedule="persistent", graph=False, chunk=4)),
                     ("graph", dict(schedule="persistent", graph=True))]:
        f = qf.Flow(h, g, 6, sp, precision="mixed", **kw)
        per = []
        for _ in range(3):
            f.sweep()
            per.append(f.energy(per_space=True)[1])
            phases, launches = f.last_sweep_info()   # phase timers also work on a replayed sweep
            assert (np.asarray(phases) >= 0).all() and launches > 0
        runs[name] = (np.array(per), f.amplitudes(), f.schedule())
        f.close()
    ref = runs["per_class"]
    for name in ("persistent", "persistent_12_warps", "per_class_7_warps", "persistent_chunk_4", "graph"):
        assert np.array_equal(runs[name][0], ref[0]), name
        assert np.array_equal(runs[name][1][1], ref[1][1]), name
    assert runs["graph"][2]["graph"] and runs["graph"][2]["persistent"]
    assert runs["persistent_12_warps"][2]["warps_per_cta"] == 12 and runs["per_class_7_warps"][2]["warps_per_cta"] == 7
    assert runs["persistent_chunk_4"][2]["chunk"] == 4


def test_ladder_tile_widths_agree(qf):
    """The mixed dressing's ladder + oooo tensor-core product at 32, 64 and 128 columns per tile
    gives the same dressed operator and the same sweeps, bit for bit (each output element sums
    its K slabs in the same order whatever the tile width)."""
    eps, h, g, sp = synth.system_inputs("n40")
    runs = {}
    for bn in (32, 64, 128):
        f = qf.Flow(h, g, 6, sp, precision="mixed", schedule="persistent", graph=False, ladder_bn=bn)
        per = []
        for _ in range(2):
            f.sweep()
            per.append(f.energy(per_space=True)[1])
        e0, F, W = f.dressed()
        runs[bn] = (np.array(per), e0, F, W, f.dress_schedule())
        f.close()
    for bn in (32, 128):
        assert np.array_equal(runs[bn][0], runs[64][0]), bn
        assert runs[bn][1] == runs[64][1] and np.array_equal(runs[bn][2], runs[64][2]), bn
        assert np.array_equal(runs[bn][3], runs[64][3]), bn
    for bn in (32, 64, 128):
        assert runs[bn][4] == {"ladder_bn": bn, "candidate_ms": []}


def test_consecutive_spaces_reuse_the_gathered_block(qf):
    """A warp that takes consecutive spaces of the sorted list keeps the couplings of the five
    orbitals they share and gathers only those of the last virtual: every (3, 3) space of n24
    (consecutive spaces mostly differ in the last virtual) with 8 spaces per fetch gives the same
    sweeps, bit for bit, as the per-class schedule (no warp meets consecutive spaces there)."""
    eps, h, g, _ = synth.system_inputs("n24")
    sp = synth.all_spaces(24, 5, 3, 3)
    runs = []
    for kw in (dict(schedule="per_class"), dict(schedule="persistent", chunk=8)):
        f = qf.Flow(h, g, 5, sp, precision="mixed", graph=False, **kw)
        per = []
        for _ in range(3):
            f.sweep()
            per.append(f.energy(per_space=True)[1])
        runs.append((np.array(per), f.amplitudes()))
        f.close()
    assert np.array_equal(runs[0][0], runs[1][0])
    assert np.array_equal(runs[0][1][0], runs[1][1][0]) and np.array_equal(runs[0][1][1], runs[1][1][1])


def test_autotuner_times_candidates(qf):
    eps, h, g, sp = synth.system_inputs("n40")
    sp = sp[::3]   # a space list of its own, so the per-process cache is cold
    f = qf.Flow(h, g, 6, sp, precision="mixed", schedule="auto")
    f.sweep()
    assert f.schedule()["candidate_ms"] == []     # calibration happens at the second sweep
    f.sweep()
    sch = f.schedule()
    assert len(sch["candidate_ms"]) == 8 and min(sch["candidate_ms"]) > 0
    assert sch["persistent"] and sch["chunk"] in (1, 2, 4, 8) and sch["warps_per_cta"] in (12, 15)
    ds = f.dress_schedule()   # the dressing's ladder tile width is timed beside the solver's candidates
    assert len(ds["candidate_ms"]) == 3 and min(ds["candidate_ms"]) > 0 and ds["ladder_bn"] in (32, 64, 128)
    assert ds["ladder_bn"] == (32, 64, 128)[int(np.argmin(ds["candidate_ms"]))]
    f.close()
