#!/usr/bin/env python
"""Benchmark of the Quantum Flow sweep on one GB300: one step = one full sweep (dressing of the
pool, every active space gathered + folded + solved by the batched Davidson kernel, CI -> CC
increments merged by owner, mean energy and convergence reductions).

Default workload: the 82-orbital synthetic system (10 occupied, 72 virtual, xi = 5) with all
C(10,3) C(72,3) = 7,156,800 (3,3) active spaces per sweep, in the mixed form (the precision of
each step is listed in the output line under config.precision_steps).  Warm-up sweeps move the
pool from empty to a mid-flow state before the timed sweeps; the plain FP64 GPU form of the
same sweep is timed beside it, and the FP64 oracle is timed on the host cores on a bounded
sample (cpu_baseline).  The inputs (W: 362 MB) are larger than the 126 MB L2.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference] [--workload n82]

With N > 1 (torchrun, one process per GPU) the sweep is sharded: every rank holds the whole
problem, dresses the same pool, solves its block of every size class, and the ranks sum their
exchange vectors with one NCCL allreduce per sweep before the merge (strong scaling: the value is
the spaces of the one problem per second).  --sharded runs the same three-call path at N = 1.
"""
from __future__ import annotations

import argparse
import json
import math
import multiprocessing as mp
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_2606_04186_gb300 import synth  # noqa: E402

METRIC = "QFlow sweep time (s) + active spaces/s vs plain FP64 GPU form at |ΔE|≤1e-6 Eh"
UNIT = "active spaces/s"
# precision of each step of a sweep, per form (what the library computes in; see include/qflow.h)
PRECISION_STEPS = {
    "mixed": {
        "dressing_integrals_e0_fock": "f64 (T1 correction sums f32, added to f64)",
        "dressing_t2_contractions": "tcgen05 three-term tf32 products, f32 accumulation, added to f64 bases",
        "gather_fold_setup": "f32 (operator diagonal relative to <Phi|H|Phi>)",
        "sigma_vectors_davidson_vectors": "f32",
        "rayleigh_ritz_matrix_and_gram_schmidt_coefficients": "f64 (exact f32 products, compensated sums, "
                                                             "rounded to f64)",
        "projected_eigenproblem_ritz_value": "f64 (root chosen in f32 closed form, refined by f64 Newton steps)",
        "energy_amplitude_update_diis_reductions": "f64",
        "hard_spaces": "spaces the f32 warp pass leaves unconverged are re-solved in f64",
    },
    "fp64": {"every_step": "f64"},
    "ducc": {"every_step": "f64",
             "form": "DUCC: [H + [H, s] + 1/2 [[F, s], s]]_(<=2), s = T_ext - T_ext^+; common part from eight "
                     "FP64 dressings per sweep, each space's internal part subtracted in its solve"},
}


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--workload", default="n82", choices=sorted(synth.SYSTEMS))
    ap.add_argument("--precision", default="mixed", choices=["mixed", "fp64"])
    ap.add_argument("--form", default="ses", choices=["ses", "ducc"],
                    help="downfolding form: SES-CC (default) or the Hermitian DUCC form (FP64 only)")
    ap.add_argument("--fp64-steps", type=int, default=1, help="timed sweeps of the plain FP64 form (0 = skip)")
    ap.add_argument("--e2e-steps", type=int, default=2)
    ap.add_argument("--cpu-sample", type=int, default=3000, help="spaces solved by the oracle for cpu_baseline")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--schedule", default="auto", choices=["auto", "persistent", "per_class"])
    ap.add_argument("--ladder-bn", type=int, default=0, choices=[0, 32, 64, 128],
                    help="tile width of the dressing's ladder + oooo GEMM (0 = timed by the autotuner, else 64 "
                         "under a fixed schedule)")
    ap.add_argument("--sampler", type=int, default=-1,
                    help="space list from Algorithm 1 (greedy coverage cycle of (3,3) spaces) with this seed")
    ap.add_argument("--waves", type=int, default=0,
                    help="wave-ordered sweeps: the pool is updated after every K spaces (0 = Jacobi)")
    ap.add_argument("--sharded", action="store_true",
                    help="sharded sweep path (begin / exchange / end) also at N = 1")
    ap.add_argument("--launch-loop", action="store_true",
                    help="also time the solve as one launch per space (a per-space launch loop) against one "
                         "launch for every space, on the dressing of the timed pool (3,3 spaces only)")
    ap.add_argument("--no-mlp", action="store_true",
                    help="skip the warm-start network leg (mlp_vs_cold: flows to convergence from an empty pool "
                         "and from the network's pool, on a second system of the same recipe)")
    ap.add_argument("--spaces-limit", type=int, default=0,
                    help="keep an evenly strided subset of at most this many spaces (small profiling case)")
    return ap.parse_args()


# ---- per-space flop accounting of the solve kernel (6e6o, 400 determinants) ------------------

def solver_flops(iters: np.ndarray, ndet: int = 400, ns: int = 20, nsg: int = 12, k: int = 3, kmax: int = 3) -> float:
    """Algorithmic flops of the batched Davidson for 6e6o spaces that ran `iters` iterations.

    Every space: the Phi column of the operator from its coupling table (153 terms for the 117
    nonzero determinants) and its norm.  Spaces that iterate: the alpha-beta Coulomb row sums
    (NORB*NS*K), the first-order vector on the 117 nonzeros (diagonal, division, norm), and the
    same-spin string operator (1,980 merged terms).  Iteration m with subspace size j: the first
    (m = 1, from Phi) only scales the first-order vector; later ones form the residual
    400*(4j+4), precondition 400*8, orthogonalise in two passes 400*(4j)*2 and normalise 400*3.
    Each iteration applies sigma, 400 * (2*NSG^2 + 2*NS + 3) = 132,400 flop (alpha-beta, the
    alpha-alpha product whose transpose is the beta-beta part, the transpose added, the diagonal
    term); the first one, on the first-order vector (nonzero only on the 117 determinants of the
    Phi column), takes only the products against its nonzeros: 2 * 16,848 alpha-beta, 2 * 20 * 117
    alpha-alpha, 3 * 400 transpose and diagonal = 39,576 flop.  Each iteration forms the new
    row and column of the projected matrix 400*2*(2j+1); the subspace restarts at kmax.  The
    convergence test after the last iteration forms one more residual.
    """
    sig = ndet * (2 * nsg * nsg + 2 * ns + 3)
    sig1 = 2 * 16848 + 2 * ns * 117 + 3 * ndet  # sigma of the first-order vector
    nz = 117
    phi = 2 * 153 + 2 * nz
    first = 2 * 6 * ns * k + nz * 8 + 2 * 1980
    m_max = int(iters.max()) if iters.size else 0
    cum = np.zeros(m_max + 1)
    j, tot = 1, 0.0
    for m in range(1, m_max + 1):
        if j == kmax:
            tot += ndet * (4 * kmax + 6)          # restart: Ritz vector + its sigma combination + norms
            j = 1
        if m == 1:
            tot += ndet + sig1
        else:
            tot += ndet * (4 * j + 4) + ndet * 8 + ndet * 8 * j + ndet * 3 + sig
        tot += ndet * 2 * (2 * j + 1)
        j += 1
        cum[m] = tot + ndet * (4 * j + 4)         # + the residual of the convergence test
    it = np.clip(iters, 0, m_max)
    return float(phi * iters.size + first * np.count_nonzero(iters > 0) + cum[it].sum())


def dress_gemm_flops(o: int, v: int) -> float:
    """Algorithmic flops (2 M N K, one term) of the T2 contractions the mixed dressing runs as
    tensor-core GEMMs: Woooo, ring intermediates, ladder + oooo, the residual's rings, ovvo, oovv,
    the oovo v^2 term and its two O(ov) maps, the three vvvo maps (the restricted vvvv term runs
    on the SIMT pipes and is not counted)."""
    ov, vv, oo = o * v, v * v, o * o
    mnk = (oo * oo * vv + 4 * ov * ov * ov + oo * vv * (vv + oo) + ov * ov * (5 + 2 + 1 + 2) * ov
           + ov * ov * 2 * ov + ov * ov * ov + ov * oo * vv + oo * ov * 3 * ov
           + vv * (v * o) * (2 * ov + oo + ov))
    return 2.0 * mnk


# solve-kernel DRAM traffic per space, sweep 3 (ncu capture of the 477,120-space n82 subset)
TRAFFIC_PER_SPACE = {"n82": 151.1}


# ---- clocks ------------------------------------------------------------------------------------

class ClockSampler:
    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None
        return self

    def __exit__(self, *exc):
        self.lines = []
        if self.proc is not None:
            self.proc.terminate()
            try:
                out, _ = self.proc.communicate(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
                out, _ = self.proc.communicate()
            self.lines = [ln for ln in out.splitlines() if ln.strip()]
        return False

    def summary(self):
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            try:
                sm.append(float(f[0]))
                mx.append(float(f[1]))
            except (ValueError, IndexError):
                continue
            for nm, val in zip(names, f[4:8]):
                if val.lower() == "active":
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"], "samples": 0}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


# ---- CPU oracle leg -------------------------------------------------------------------------------

def _oracle_worker(args):
    from oracle import cas
    out = []
    for no, nv, c, h, w in args:
        out.append(cas.solve_problem(no, nv, c, h, w)[0])
    return out


def oracle_sweep_sample(name: str, sample: int, pool, seed: int = 7):
    """Time the oracle on a bounded sample of one sweep: full dressing + `sample` spaces."""
    from oracle import cas, flow, hbar
    eps, h, g, sp = synth.system_inputs(name)
    s = synth.SYSTEMS[name]
    no, nv = s.nocc, s.n - s.nocc
    t1, t2 = synth.random_amplitudes(no, nv, seed, 0.005, 0.01)
    t0 = time.perf_counter()
    e0, F, W = hbar.hbar2(h, g, t1, t2, no)
    t_dress = time.perf_counter() - t0
    rng = np.random.default_rng(seed)
    pick = rng.choice(len(sp), size=min(sample, len(sp)), replace=False)
    t0 = time.perf_counter()
    probs = [(int(sp[k][0]), int(sp[k][1]), *cas.space_problem(e0, F, W, *flow.space_orbitals(sp[k]))) for k in pick]
    nproc = getattr(pool, "_processes", 1)
    chunks = [probs[i::nproc] for i in range(nproc)]
    pool.map(_oracle_worker, chunks)
    t_solve = time.perf_counter() - t0
    per_space = t_solve / len(pick)
    sweep_s = t_dress + per_space * len(sp)
    return {"value": len(sp) / sweep_s, "sweep_s_extrapolated": sweep_s, "dress_s": t_dress,
            "solve_s_sample": t_solve, "sample": len(pick), "nspaces": len(sp)}


def workload_desc(name: str, s, sp: np.ndarray) -> str:
    """The workload as both arms name it: system, orbital counts, xi and the space list by class."""
    no, nv = s.nocc, s.n - s.nocc
    classes = ', '.join(f'{int((sp[:, 0] == k).sum())} ({k},{k})' for k in (3, 2, 1) if (sp[:, 0] == k).any())
    return f"{name}: {s.n} orbitals ({no} occ, {nv} virt), xi={s.xi}, {len(sp)} spaces ({classes})"


def log(msg: str):
    print(f"[bench {time.strftime('%H:%M:%S')}] {msg}", file=sys.stderr, flush=True)


def host_cores() -> int:
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count() or 1


def _warm_worker(_):
    from oracle import cas
    for k in (1, 2, 3):
        cas.coupling(k, k)  # build the determinant coupling maps once per worker
    return 0


def make_pool():
    n = host_cores()
    ctx = mp.get_context("spawn")
    saved = {k: os.environ.get(k) for k in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS")}
    for k in saved:
        os.environ[k] = "1"          # one BLAS thread per worker: the pool already uses every core
    pool = ctx.Pool(n)
    for k, v in saved.items():
        if v is None:
            os.environ.pop(k, None)
        else:
            os.environ[k] = v
    pool.map(_warm_worker, range(n))
    return pool, n


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    pool, cores = make_pool()
    s = synth.SYSTEMS[args.workload]
    sample = max(64, args.cpu_sample // 3)
    for _ in range(args.warmup):
        oracle_sweep_sample(args.workload, sample, pool)
    vals, secs, timed = [], [], []
    for k in range(args.steps):
        r = oracle_sweep_sample(args.workload, sample, pool, seed=11 + k)
        vals.append(r["value"])
        secs.append(r["sweep_s_extrapolated"])
        timed.append(r["dress_s"] + r["solve_s_sample"])
    pool.close()
    value = statistics.median(vals)
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * statistics.median(secs),
        "higher_is_better": True, "scaling": "strong", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": workload_desc(args.workload, s, synth.system_inputs(args.workload)[3]), "precision": "fp64",
                   "note": "each step: full oracle dressing + a seeded sample of spaces solved on all host cores; "
                           "sweep time extrapolated linearly in the number of spaces"},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                         "sample": f"{r['sample']} spaces per step of {r['nspaces']} + full dressing, extrapolated",
                         "timed_s_per_step": statistics.median(timed), "dress_s": r["dress_s"],
                         "solve_s_sample": r["solve_s_sample"], "extrapolated_sweep_s": statistics.median(secs)},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


# ---- GPU leg ---------------------------------------------------------------------------------------

def _converge(fl, stream, tol_e, tol_t, max_sweeps=40):
    """Sweeps until |dE| < tol_e and max|dt| < tol_t; returns (sweeps, CUDA-event seconds of the
    sweeps, energy after each sweep)."""
    import torch
    ms, es = 0.0, []
    for _ in range(max_sweeps):
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        de, dt, nf, code = fl.sweep(raise_on_fail=False)
        b.record(stream)
        torch.cuda.synchronize()
        ms += a.elapsed_time(b)
        es.append(fl.energy())
        if abs(de) < tol_e and dt < tol_t:
            break
    return len(es), ms / 1e3, es


def mlp_leg(qflow, name, s, h, g, sp, precision, sweep_ms, hidden=256, max_pairs=100000):
    """Warm-start network (not in the paper) at this workload: trained on the converged flow of
    the timed system (bare integrals of each space -> its converged internal amplitudes), then a
    second system of the same recipe (another seed) is run to convergence from an empty pool and
    from the network's pool; the warm start's inference (features, network, pool) is timed with
    CUDA events and counted in its time to convergence."""
    import torch
    no = s.nocc
    tol_e, tol_t = (1e-8, 1e-7) if precision == "fp64" else (1e-7, 1e-5)
    fa = qflow.Flow(h, g, no, sp, precision=precision)
    sa = torch.cuda.ExternalStream(fa.stream())
    _converge(fa, sa, tol_e, tol_t)
    stride = max(1, len(sp) // max_pairs)
    n = fa.mlp_collect(stride=stride, max_pairs=max_pairs, target="pool")
    fa.mlp_set_model(synth.mlp_init_model(hidden, 2), hidden, has_stats=False)
    t0 = time.perf_counter()
    loss = fa.mlp_train(epochs=60, batch=128, lr=2e-3, order=np.random.default_rng(4).permutation(n))
    t_train = time.perf_counter() - t0
    model = fa.mlp_get_model()
    fa.close()
    _, h2, g2 = synth.make_system(s.n, s.nocc, s.xi, s.seed + 100)
    cold = qflow.Flow(h2, g2, no, sp, precision=precision)
    k_cold, t_cold, e_cold = _converge(cold, torch.cuda.ExternalStream(cold.stream()), tol_e, tol_t)
    cold.close()
    warm = qflow.Flow(h2, g2, no, sp, precision=precision)
    sw = torch.cuda.ExternalStream(warm.stream())
    warm.mlp_set_model(model, hidden, has_stats=True)
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    a.record(sw)
    warm.mlp_warm_pool()
    b.record(sw)
    torch.cuda.synchronize()
    t_inf = a.elapsed_time(b) / 1e3
    k_warm, t_warm, e_warm = _converge(warm, sw, tol_e, tol_t)
    warm.close()
    e_fix = e_cold[-1]
    err_cold = [abs(e - e_fix) for e in e_cold[:3]]
    err_warm = [abs(e - e_fix) for e in e_warm[:3]]
    log(f"mlp: trained on {n} pairs in {t_train:.1f} s (loss {loss[0]:.3g} -> {loss[-1]:.3g}); cold {k_cold} sweeps "
        f"{t_cold:.3f} s, warm {k_warm} sweeps {t_warm:.3f} s + inference {1e3 * t_inf:.1f} ms; |E - E_fixed| after "
        f"sweeps 1-3: cold {err_cold}, warm {err_warm}")
    return {"train_pairs": n, "train_s": t_train, "loss_first_last": [float(loss[0]), float(loss[-1])],
            "system": f"{name} recipe, seed {s.seed + 100}", "tol": [tol_e, tol_t],
            "cold": {"sweeps": k_cold, "seconds": t_cold, "energy": e_cold[-1], "abs_error_sweeps_1_3": err_cold},
            "warm": {"sweeps": k_warm, "seconds_incl_inference": t_warm + t_inf, "energy": e_warm[-1],
                     "abs_error_sweeps_1_3": err_warm},
            "inference_ms": 1e3 * t_inf, "inference_over_timed_sweep": (1e3 * t_inf) / sweep_ms,
            "energy_difference": e_warm[-1] - e_cold[-1],
            "note": "network used to start the pool only; the plain flow is the judge (same fixed point)"}


def launch_loop_leg(qflow, fl, h, g, no, sp, precision):
    """The solve step of the timed pool's dressing (steps b + c for every (3,3) space) as one
    qflow_solve_device launch per space, against one launch for all spaces; CUDA events around
    each on the default stream.  Both use the warp pass alone (iteration cap 16)."""
    import torch
    e0, F, W = fl.dressed()
    t1, t2 = fl.amplitudes()
    perm = fl.order()
    sps = np.ascontiguousarray(sp[perm])
    keep = np.flatnonzero(sps[:, 0] == 3)
    _, o1, o2, _ = qflow.plan(h, g, no, sp)
    d = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()  # noqa: E731
    e0d, Fd, Wd = d(np.array([e0])), d(F), d(W)
    spd, o1d, o2d = d(sps[keep]), d(o1.astype(np.int32)), d(o2.astype(np.int32))
    t1o, t2o = d(t1), d(t2)
    n, ns = h.shape[0], len(keep)
    energy = torch.zeros(ns, dtype=torch.float64, device="cuda")
    status = torch.zeros(ns, dtype=torch.int32, device="cuda")

    def run(per_space: bool) -> float:
        t1n, t2n = t1o.clone(), t2o.clone()
        torch.cuda.synchronize()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        if per_space:
            for i in range(ns):
                qflow.solve_device(n, no, e0d, Fd, Wd, 3, spd[i:i + 1], energy[i:i + 1], status[i:i + 1],
                                   owner1=o1d, owner2=o2d, t1_old=t1o, t2_old=t2o, t1_new=t1n, t2_new=t2n,
                                   space_base=int(keep[i]), precision=precision, max_iter=16)
        else:
            qflow.solve_device(n, no, e0d, Fd, Wd, 3, spd, energy, status, owner1=o1d, owner2=o2d, t1_old=t1o,
                               t2_old=t2o, t1_new=t1n, t2_new=t2n, space_base=int(keep[0]), precision=precision,
                               max_iter=16)
        b.record()
        torch.cuda.synchronize()
        return a.elapsed_time(b)

    if not (np.diff(keep) == 1).all():
        return None  # the one-launch form needs the (3,3) spaces contiguous in the sorted list
    run(False)
    one = min(run(False) for _ in range(3))
    loop = run(True)
    log(f"launch loop: {ns} launches {loop:.1f} ms, one launch {one:.2f} ms")
    return {"spaces": ns, "per_space_launches_ms": loop, "one_launch_ms": one, "ratio": loop / one,
            "note": "qflow_solve_device per space (host launch loop) vs once over all spaces, same dressing"}


def run_ours(args):
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    pool = cores = None
    if rank == 0 and not args.no_cpu_baseline:
        pool, cores = make_pool()   # before the first GPU call
    import torch
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    from paper_2606_04186_gb300 import qflow
    qflow.lib()
    name = args.workload
    s = synth.SYSTEMS[name]
    eps, h, g, sp = synth.system_inputs(name)
    if args.sampler >= 0:   # one cycle of Algorithm 1 from the Fock diagonal of the system
        from paper_2606_04186_gb300 import qflow as _q
        _q.lib()
        fd = np.array([h[p, p] + sum(2 * g[p, p, k, k] - g[p, k, k, p] for k in range(s.nocc)) for p in range(s.n)])
        sp, _ = _q.sample_spaces(fd, s.nocc, 3, 3, args.sampler)
    if args.spaces_limit and len(sp) > args.spaces_limit:
        sp = np.ascontiguousarray(sp[::-(-len(sp) // args.spaces_limit)])
    no, nv = s.nocc, s.n - s.nocc
    log(f"inputs ready: {name}, {len(sp)} spaces")
    t_init = time.perf_counter()
    if args.form == "ducc":
        args.precision = "fp64"   # the DUCC form is FP64 throughout; its FP64 leg is the run itself
    fl = qflow.Flow(h, g, no, sp, precision=args.precision, schedule=args.schedule, form=args.form,
                    ladder_bn=args.ladder_bn if args.precision == "mixed" and args.form == "ses" else 0)
    t_init = time.perf_counter() - t_init
    stream = torch.cuda.ExternalStream(fl.stream())
    log(f"init {t_init:.1f} s")
    sharded = world > 1 or args.sharded
    if sharded and args.waves:
        raise SystemExit("--waves runs on one GPU (the waves follow each other)")
    if sharded:
        fl.set_shard(rank, world)
        xbuf = torch.empty(fl.exchange_size(), dtype=torch.float64, device="cuda")

    def sweep():
        if args.waves:
            return fl.sweep_waves(args.waves, raise_on_fail=False)
        if not sharded:
            return fl.sweep(raise_on_fail=False)
        if world > 1:
            return fl.sweep_sharded(xbuf, raise_on_fail=False)
        fl.sweep_shard_begin(xbuf)   # one rank: the exchange vector is already the sum
        return fl.sweep_shard_end(xbuf, raise_on_fail=False)
    # every timed step is the third sweep of the flow: the pool after two sweeps from empty is
    # restored before each step (outside the timed events)
    e_hist = []
    for _ in range(2):
        sweep()
        e_hist.append(fl.energy())
        log(f"sweep {len(e_hist)}: E = {e_hist[-1]:.10f}, phases {fl.last_sweep_info()[0]}")
    p2 = fl.amplitudes()
    for _ in range(max(3, args.warmup)):
        fl.set_amplitudes(*p2)
        sweep()
    e3 = fl.energy()
    log(f"warm-up done: sweep-3 E = {e3:.10f}, phases {fl.last_sweep_info()[0]}")

    def barrier():
        if dist is not None:
            dist.barrier()
        torch.cuda.synchronize()

    # the solver's roofline denominators, measured on this GPU (FMA chains on every SM)
    peaks = {"fp32_tflops": qflow.fma_peak("mixed"), "fp64_tflops": qflow.fma_peak("fp64"),
             "method": "qflow_fma_peak: 8 independent fma chains per thread, every SM full, "
                       "best of 3 CUDA-event-timed launches"}
    log(f"measured FMA peaks: {peaks['fp32_tflops']:.1f} FP32, {peaks['fp64_tflops']:.3f} FP64 TFLOP/s")

    phases, launches, codes = [], 0, []
    starts = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    ends = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    barrier()
    with ClockSampler(local) as clk:
        for k in range(args.steps):
            fl.set_amplitudes(*p2)
            starts[k].record(stream)
            de, dt, nf, code = sweep()
            ends[k].record(stream)
            codes.append(code)
            ph, nl = fl.last_sweep_info()
            phases.append(ph)
            launches += nl
        barrier()
    elapsed_ms = sum(a.elapsed_time(b) for a, b in zip(starts, ends))
    log(f"timed {args.steps} sweeps: {elapsed_ms:.1f} ms")
    it, st = fl.stats()
    e_mean = fl.energy()
    sched = fl.schedule()
    sched["dress_ladder"] = fl.dress_schedule()  # tile width of the ladder + oooo product
    if dist is not None:
        tt = torch.tensor([elapsed_ms], device="cuda")
        dist.all_reduce(tt, op=dist.ReduceOp.MAX)
        elapsed_ms = float(tt.item())
    sweep_ms = elapsed_ms / args.steps
    # sharded: the ranks share one problem (strong scaling); replicas are not run
    value = len(sp) / (sweep_ms / 1e3)
    ph = np.array(phases)
    solve_ms = float(ph[:, 1].mean())
    if world > 1:  # this rank's solve phase covers its own shard only
        own = qflow.shard_plan(h, g, no, sp, rank, world)[0].astype(bool)
        flops = solver_flops(it[own].astype(np.int64))
    else:
        flops = solver_flops(it.astype(np.int64))
    achieved = flops / (solve_ms / 1e3) / 1e12
    peak = peaks["fp32_tflops"] if args.precision == "mixed" else peaks["fp64_tflops"]

    # end-to-end through the public API with host buffers: pool H2D (pinned), sweep,
    # per-space energies + pool D2H, every step
    t1h = torch.empty((no, nv), dtype=torch.float64).pin_memory()
    t2h = torch.empty((no, no, nv, nv), dtype=torch.float64).pin_memory()
    t1h.numpy()[...] = p2[0]
    t2h.numpy()[...] = p2[1]
    ebuf = torch.empty(len(sp), dtype=torch.float64).pin_memory()
    barrier()
    t0 = time.perf_counter()
    for _ in range(args.e2e_steps):
        qflow.lib().qflow_set_amplitudes(fl._h, t1h.data_ptr(), t2h.data_ptr())
        sweep()
        ec = qflow.C.c_double()
        qflow.lib().qflow_energy(fl._h, qflow.C.byref(ec), ebuf.data_ptr())
        qflow.lib().qflow_amplitudes(fl._h, t1h.data_ptr(), t2h.data_ptr())
        t1h.numpy()[...] = p2[0]   # next step starts from the same pool again (host side, untimed work
        t2h.numpy()[...] = p2[1]   # of a few MB; part of the end-to-end wall time)
    barrier()
    e2e_s = (time.perf_counter() - t0) / max(1, args.e2e_steps)
    log(f"e2e {e2e_s:.3f} s per step")
    pool_bytes = 8 * (t1h.numel() + t2h.numel())
    fl_xsize = fl.exchange_size()
    # the dressing of the pool p2 (the last e2e step dressed it), kept to state the mixed form's
    # error per block against the plain FP64 form's dressing of the same pool
    dressed_mixed = fl.dressed() if (args.precision == "mixed" and args.fp64_steps > 0 and world == 1
                                     and s.n <= 82 and not args.waves) else None
    loop = launch_loop_leg(qflow, fl, h, g, no, sp, args.precision) if (args.launch_loop and world == 1) else None
    fl.close()

    mlp = None
    if not args.no_mlp and world == 1 and not args.waves and not sharded and args.form == "ses" and \
            args.sampler < 0 and not args.spaces_limit and (sp[:, 0] == 3).all():
        mlp = mlp_leg(qflow, name, s, h, g, sp, args.precision, sweep_ms)

    # plain FP64 GPU form of the same sweep (pool after the same number of sweeps as the first
    # warm-up of the mixed run: compare energies after sweep 2)
    fp64 = None
    if args.fp64_steps > 0 and args.precision == "mixed" and world == 1:
        f64 = qflow.Flow(h, g, no, sp, precision="fp64")
        s64 = torch.cuda.ExternalStream(f64.stream())
        ms = []
        for k in range(args.fp64_steps):
            f64.set_amplitudes(*p2)
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            barrier()
            a.record(s64)
            if args.waves:
                f64.sweep_waves(args.waves, raise_on_fail=False)
            else:
                f64.sweep(raise_on_fail=False)
            b.record(s64)
            barrier()
            ms.append(a.elapsed_time(b))
            log(f"fp64 sweep: {ms[-1]:.1f} ms, phases {f64.last_sweep_info()[0]}")
        ms64 = statistics.median(ms)
        e64 = f64.energy()
        dress_err = None
        if dressed_mixed is not None:
            e0d, Fd, Wd = f64.dressed()
            e0m, Fm, Wm = dressed_mixed
            o_, v_ = slice(0, no), slice(no, s.n)
            sl = {"o": o_, "v": v_}
            dress_err = {"e0": abs(e0m - e0d), "F": float(np.abs(Fm - Fd).max())}
            for blk in ("oooo", "ooov", "oovv", "ovov", "ovvo", "vovo", "vvoo", "vovv", "vvvo", "vvvv", "vooo",
                        "ovoo", "voov", "ovvv", "vvov", "oovo"):
                idx = tuple(sl[c] for c in blk)
                diff = np.abs(Wm[idx] - Wd[idx])
                if blk == "vvvv":  # the mixed flow dresses only elements with <= 3 distinct virtuals
                    nv_ = s.n - no
                    ar_ = np.arange(nv_)
                    a_, e_, b_, f_ = np.meshgrid(ar_, ar_, ar_, ar_, indexing="ij", sparse=True)
                    diff = np.where((a_ != e_) & (a_ != b_) & (a_ != f_) & (e_ != b_) & (e_ != f_) & (b_ != f_),
                                    0.0, diff)
                dress_err["W_" + blk] = float(diff.max())
            del Wm, Wd
            log(f"mixed - fp64 dressing, max |error| per block: {dress_err}")
        ph64, _ = f64.last_sweep_info()
        it64, _ = f64.stats()
        fp64 = {"sweep_s": ms64 / 1e3, "spaces_per_s": len(sp) / (ms64 / 1e3), "solve_ms": float(ph64[1]),
                "dress_ms": float(ph64[0]), "davidson_iters_mean": float(it64.mean()),
                "solve_tflops": solver_flops(it64.astype(np.int64)) / (ph64[1] / 1e3) / 1e12,
                "e_sweep3": e64, "mixed_minus_fp64_e_sweep3": e3 - e64,
                "mixed_minus_fp64_dressing_max_abs": dress_err}
        f64.close()

    if rank != 0:
        if dist is not None:
            dist.destroy_process_group()
        return
    cpu = None
    if pool is not None:
        log("oracle sample")
        r = oracle_sweep_sample(name, args.cpu_sample, pool)
        log(f"oracle: {r}")
        pool.close()
        cpu = {"value": r["value"], "unit": UNIT, "cores": cores, "kind": "oracle",
               "sample": (f"full dressing + {r['sample']} of {r['nspaces']} spaces on a spawn pool, sweep time "
                          f"extrapolated ({r['sweep_s_extrapolated']:.1f} s)") if r["sample"] < r["nspaces"]
               else f"full sweep: dressing + all {r['nspaces']} spaces on a spawn pool",
               "timed_s": r["dress_s"] + r["solve_s_sample"], "sweep_s": r["sweep_s_extrapolated"]}
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": max(3, args.warmup), "ms_per_step": sweep_ms, "higher_is_better": True,
        "scaling": "strong",   # every N sweeps the same list of spaces
        "vs_baseline": None, "dtype": "f32+f64" if args.precision == "mixed" else "f64", "data": "synthetic",
        "config": {"workload": workload_desc(name, s, sp),
                   "precision": args.precision, "sweep_s": sweep_ms / 1e3, "l2": (f"inputs larger than L2 (W = {8 * s.n ** 4 / 1e6:.0f} MB)" if 8 * s.n ** 4 > 126e6
                          else f"inputs smaller than L2 (W = {8 * s.n ** 4 / 1e6:.1f} MB), not flushed"), "e_sweep3": e_mean,
                   "space_list": (f"Algorithm 1 cycle, seed {args.sampler}" if args.sampler >= 0
                                  else "every (3,3) space" if len(sp) == math.comb(no, 3) * math.comb(nv, 3)
                                  else "list of the workload"),
                   "sweep_order": (f"waves of {args.waves} spaces in Delta-eps order, pool updated between "
                                f"waves ({-(-len(sp) // args.waves)} dressings per sweep)") if args.waves
                   else "Jacobi (all spaces read the pool of the last barrier)",
                   "parallelism": (f"sharded over {world} GPUs: per-class blocks, one allreduce of "
                                   f"{8 * fl_xsize / 1e6:.0f} MB per sweep") if sharded else "one GPU",
                   "step": "third sweep of the flow (pool after two sweeps restored before each step)",
                   "precision_steps": PRECISION_STEPS["ducc" if args.form == "ducc" else args.precision],
                   "form": "DUCC (Hermitian)" if args.form == "ducc" else "SES-CC",
                   "init_s": t_init},
        "roofline": {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                     "frac": achieved / peak,
                     "traffic": (TRAFFIC_PER_SPACE[name] * len(sp)
                                 if name in TRAFFIC_PER_SPACE and args.precision == "mixed" and not args.spaces_limit
                                 else None),
                     "kernel": ("solve_persistent_kernel" if sched["persistent"] else "solve_class_kernel<K>")
                     if args.precision == "mixed" else ("solve_kernel<K,double,DUCC>" if args.form == "ducc"
                                                        else "solve_kernel<K,double>"),
                     "flops_per_launch": flops, "launch_ms": solve_ms,
                     "flops_note": ("products the steps need (solver_flops): sigma of the first-order "
                                    "vector counts only its 117-determinant support, as the kernel "
                                    "computes it; the kernel is latency- and issue-bound (profiles/)"),
                     "peak_note": ("measured FP32 FMA peak of this GPU" if args.precision == "mixed"
                                   else "measured FP64 FMA peak of this GPU") + " (" + peaks["method"] + ")",
                     "peaks_measured": {k: v for k, v in peaks.items() if k != "method"}},
        "schedule": sched,
        "dress_tensor": ({"gemm_flops": dress_gemm_flops(no, nv), "phase_ms": float(ph[:, 0].mean()),
                          "tflops_over_phase": dress_gemm_flops(no, nv) / (float(ph[:, 0].mean()) / 1e3) / 1e12,
                          "note": "algorithmic one-term flops of the tcgen05 GEMMs / whole dressing phase"}
                         if args.precision == "mixed" else None),
        "phase_ms": {"dress": float(ph[:, 0].mean()), "solve": solve_ms, "merge": float(ph[:, 2].mean())},
        "davidson_iters_mean": float(it.mean()),
        "davidson_iters_hist": np.bincount(np.minimum(it.astype(np.int64), 12), minlength=13).tolist(),
        "failed_spaces": int((st != 0).sum()),
        "sweep_codes": sorted(set(int(c) for c in codes)),
        "fp64_form": fp64,
        "launch_loop": loop,
        "mlp_vs_cold": mlp,
        "speedup_vs_fp64": (fp64["sweep_s"] / (sweep_ms / 1e3)) if fp64 else None,
        "cpu_baseline": cpu,
        "e2e": {"value": len(sp) / e2e_s, "unit": UNIT, "h2d_bytes_per_step": pool_bytes,
                "d2h_bytes_per_step": pool_bytes + 8 * len(sp), "sweep_s": e2e_s},
        "clocks": clk.summary(),
        "gpu_launches": int(launches),
    }
    print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
