"""Thin ctypes binding of ``libqflow.so`` (argument marshalling only).

Every step of the sweep runs in the library's CUDA kernels; this module converts NumPy
arrays / torch device tensors to pointers and return codes to exceptions.  It never falls
back to any other implementation: if the library is missing it raises.

Space lists are int32 arrays of shape (nspaces, 8) laid out exactly like ``qflow_space``
(no, nv, orb[6]), as produced by ``paper_2606_04186_gb300.synth``.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libqflow.so")

PREC = {"fp64": 0, "mixed": 1}

OK, ERR_ARG, ERR_CUDA, ERR_OOM, ERR_NOCONV, ERR_ROOT, ERR_NONFINITE, ERR_STATE = 0, -1, -2, -3, -4, -5, -6, -7
ERR_TOO_LARGE = -8
WARN_UNCOVERED = 1


class QFlowError(RuntimeError):
    def __init__(self, code: int, where: str):
        super().__init__(f"{where}: {strerror(code)} ({code})")
        self.code = code


class Options(C.Structure):
    _fields_ = [("precision", C.c_int32), ("max_iter", C.c_int32), ("tol", C.c_double),
                ("diis", C.c_int32), ("guess", C.c_int32), ("schedule", C.c_int32), ("graph", C.c_int32),
                ("form", C.c_int32), ("warps", C.c_int32), ("chunk", C.c_int32),
                ("ladder_bn", C.c_int32), ("reserved", C.c_int32 * 2)]


_lib = None


def lib() -> C.CDLL:
    """The loaded library (raises if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError(f"{LIB_PATH} is missing: build it with paper_2606_04186_gb300.build.build()")
    L = C.CDLL(LIB_PATH)
    P, I32, I64, D, V = C.c_void_p, C.c_int32, C.c_int64, C.c_double, C.c_void_p
    sig = {
        "qflow_default_options": (None, [P, I32]),
        "qflow_plan": (I32, [P, P, I32, I32, P, I64, P, P, P, P]),
        "qflow_init": (I32, [P, P, P, I32, I32, P, I64, P]),
        "qflow_sweep": (I32, [P, P, P, P]),
        "qflow_energy": (I32, [P, P, P]),
        "qflow_amplitudes": (I32, [P, P, P]),
        "qflow_set_amplitudes": (I32, [P, P, P]),
        "qflow_space_order": (I32, [P, P]),
        "qflow_space_stats": (I32, [P, P, P]),
        "qflow_dressed": (I32, [P, P, P, P]),
        "qflow_stream": (V, [P]),
        "qflow_last_sweep_info": (I32, [P, P, P]),
        "qflow_schedule": (I32, [P, P, P, P, P, P, P]),
        "qflow_dress_schedule": (I32, [P, P, P, P]),
        "qflow_destroy": (None, [P]),
        "qflow_strerror": (C.c_char_p, [C.c_int]),
        "qflow_dress_workspace": (C.c_size_t, [I32, I32]),
        "qflow_dress_device_static": (I32, [P, P, P, P, I32, I32, P, P, P, P]),
        "qflow_static_scratch_bytes": (C.c_size_t, []),
        "qflow_fma_peak": (I32, [I32, P, P]),
        "qflow_dress_device": (I32, [P, P, P, P, I32, I32, P, P, P, P, C.c_size_t, P]),
        "qflow_solve_device": (I32, [I32, I32, P, P, P, I32, P, I64, I64, P, P, P, P, P, P, P, P, P, P, I32, I32,
                                     I32, D, P]),
        "qflow_mlp_param_count": (I64, [I32, I32, I32]),
        "qflow_mlp_model_size": (I64, [I32]),
        "qflow_mlp_set_model": (I32, [P, I32, P, I32]),
        "qflow_mlp_get_model": (I32, [P, P]),
        "qflow_mlp_collect": (I32, [P, I32, I64, I64, P]),
        "qflow_mlp_warm_pool": (I32, [P]),
        "qflow_mlp_train": (I32, [P, I32, I32, C.c_float, P, P]),
        "qflow_mlp_workspace": (C.c_size_t, [I32, I32, I32, I64]),
        "qflow_mlp_forward_device": (I32, [I32, I32, I32, P, P, I64, P, P, P]),
        "qflow_mlp_grad_device": (I32, [I32, I32, I32, P, P, P, P, I64, P, P, P, P]),
        "qflow_mlp_adam_device": (I32, [I64, P, P, P, P, I32, C.c_float, C.c_float, C.c_float, C.c_float, P]),
        "qflow_mlp_features_device": (I32, [I32, P, P, P, I64, P, P]),
        "qflow_mlp_targets_device": (I32, [P, I64, P, P]),
        "qflow_mlp_guess_device": (I32, [P, I64, P, P]),
        "qflow_gemm_tf32x3_device": (I32, [I32, I32, I32, P, I32, P, I32, P, I32, P, P]),
        "qflow_sweep_waves": (I32, [P, I64, P, P, P]),
        "qflow_sample_spaces": (I32, [I32, I32, I32, I32, P, C.c_uint64, P, I64, P, P]),
        "qflow_shard_plan": (I32, [P, P, I32, I32, P, I64, I32, I32, P, P]),
        "qflow_set_shard": (I32, [P, I32, I32]),
        "qflow_exchange_size": (I64, [P]),
        "qflow_sweep_shard_begin": (I32, [P, P]),
        "qflow_sweep_shard_end": (I32, [P, P, P, P, P]),
    }
    for name, (res, args) in sig.items():
        f = getattr(L, name)
        f.restype = res
        f.argtypes = args
    _lib = L
    return L


def strerror(code: int) -> str:
    return lib().qflow_strerror(int(code)).decode()


def _ptr(a: np.ndarray) -> int:
    return a.ctypes.data


def _f64(a) -> np.ndarray:
    return np.ascontiguousarray(a, dtype=np.float64)


def _spaces(sp) -> np.ndarray:
    sp = np.ascontiguousarray(sp, dtype=np.int32)
    if sp.ndim != 2 or sp.shape[1] != 8:
        raise ValueError("spaces must be an int32 array of shape (nspaces, 8)")
    return sp


def _check(code: int, where: str, allow=(OK, WARN_UNCOVERED)) -> int:
    if code not in allow:
        raise QFlowError(code, where)
    return code


def plan(h, eri, nocc: int, spaces):
    """(perm, owner1[o,v], owner2[o,o,v,v], n_uncovered) from the library's host planner."""
    h, eri, sp = _f64(h), _f64(eri), _spaces(spaces)
    n = h.shape[0]
    nv = n - nocc
    perm = np.empty(len(sp), dtype=np.int64)
    o1 = np.empty((nocc, nv), dtype=np.int32)
    o2 = np.empty((nocc, nocc, nv, nv), dtype=np.int32)
    unc = C.c_int64(0)
    _check(lib().qflow_plan(_ptr(h), _ptr(eri), n, nocc, _ptr(sp), len(sp), _ptr(perm), _ptr(o1), _ptr(o2),
                            C.byref(unc)), "qflow_plan")
    return perm, o1, o2, unc.value


def sample_spaces(eps, nocc: int, no: int, nv: int, seed: int):
    """Algorithm 1's cycle of (no, nv) spaces for orbital energies eps (host only):
    (spaces int32 (count, 8) sorted by Delta-eps, candidates drawn)."""
    eps = _f64(eps)
    nvir = len(eps) - nocc
    cap = max(1, (nocc * (nocc - 1) // 2) * (nvir * (nvir - 1) // 2))
    out = np.empty((cap, 8), dtype=np.int32)
    n, d = C.c_int64(), C.c_int64()
    _check(lib().qflow_sample_spaces(nocc, nvir, no, nv, _ptr(eps), seed, _ptr(out), cap, C.byref(n), C.byref(d)),
           "qflow_sample_spaces")
    return out[:n.value].copy(), d.value


def shard_plan(h, eri, nocc: int, spaces, rank: int, nranks: int):
    """(space_mask[nspaces] in sorted order, pool_mask[o*v + o^2 v^2]) of shard `rank` (host only)."""
    h, eri, sp = _f64(h), _f64(eri), _spaces(spaces)
    n = h.shape[0]
    nv = n - nocc
    smask = np.empty(len(sp), dtype=np.uint8)
    pmask = np.empty(nocc * nv + (nocc * nv) ** 2, dtype=np.uint8)
    _check(lib().qflow_shard_plan(_ptr(h), _ptr(eri), n, nocc, _ptr(sp), len(sp), rank, nranks, _ptr(smask),
                                  _ptr(pmask)), "qflow_shard_plan")
    return smask, pmask


def default_options(precision: str = "fp64") -> Options:
    o = Options()
    lib().qflow_default_options(C.byref(o), PREC[precision])
    return o


class Flow:
    """One flow on the current CUDA device (handle API of the library)."""

    def __init__(self, h, eri, nocc: int, spaces, precision: str = "fp64", max_iter: int | None = None,
                 tol: float | None = None, guess: str = "phi", diis: int = 0, schedule: str = "auto",
                 graph: bool = True, form: str = "ses", warps: int = 0, chunk: int = 0,
                 ladder_bn: int = 0):
        h, eri, sp = _f64(h), _f64(eri), _spaces(spaces)
        self.n, self.nocc = h.shape[0], nocc
        self.nvir = self.n - nocc
        self.nspaces = len(sp)
        opt = default_options(precision)
        if max_iter is not None:
            opt.max_iter = max_iter
        if tol is not None:
            opt.tol = tol
        opt.guess = {"phi": 0, "previous": 1, "network": 2}[guess]
        opt.diis = diis
        opt.schedule = {"auto": 0, "per_class": 1, "persistent": 2}[schedule]
        opt.graph = int(graph)
        opt.form = {"ses": 0, "ducc": 1}[form]
        opt.warps = warps
        opt.chunk = chunk
        opt.ladder_bn = ladder_bn
        self._h = C.c_void_p()
        code = lib().qflow_init(C.byref(self._h), _ptr(h), _ptr(eri), self.n, nocc, _ptr(sp), len(sp), C.byref(opt))
        self.init_status = _check(code, "qflow_init")

    def close(self):
        if self._h:
            lib().qflow_destroy(self._h)
            self._h = C.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def sweep(self, raise_on_fail: bool = True):
        de, dt, nf = C.c_double(), C.c_double(), C.c_int32()
        code = lib().qflow_sweep(self._h, C.byref(de), C.byref(dt), C.byref(nf))
        if raise_on_fail:
            _check(code, "qflow_sweep")
        return de.value, dt.value, nf.value, code

    def sweep_waves(self, wave: int, raise_on_fail: bool = True):
        """One sweep in waves of `wave` spaces in Delta-eps order (pool updated between waves)."""
        de, dt, nf = C.c_double(), C.c_double(), C.c_int32()
        code = lib().qflow_sweep_waves(self._h, int(wave), C.byref(de), C.byref(dt), C.byref(nf))
        if raise_on_fail:
            _check(code, "qflow_sweep_waves")
        return de.value, dt.value, nf.value, code

    # ---- sharded sweeps (one process per GPU, summed exchange vectors) ----
    def set_shard(self, rank: int, nranks: int):
        _check(lib().qflow_set_shard(self._h, rank, nranks), "qflow_set_shard")

    def exchange_size(self) -> int:
        return int(lib().qflow_exchange_size(self._h))

    def sweep_shard_begin(self, exchange):
        """Dressing + this shard's solves into `exchange` (float64 CUDA tensor of exchange_size())."""
        if exchange.dtype != _torch().float64 or exchange.numel() < self.exchange_size():
            raise ValueError("exchange must be a float64 CUDA tensor of exchange_size() elements")
        _check(lib().qflow_sweep_shard_begin(self._h, _dptr(exchange)), "qflow_sweep_shard_begin")

    def sweep_shard_end(self, exchange, raise_on_fail: bool = True):
        """Merge of the exchange vector summed over all ranks; returns what sweep() returns."""
        if exchange.dtype != _torch().float64 or exchange.numel() < self.exchange_size():
            raise ValueError("exchange must be a float64 CUDA tensor of exchange_size() elements")
        de, dt, nf = C.c_double(), C.c_double(), C.c_int32()
        code = lib().qflow_sweep_shard_end(self._h, _dptr(exchange), C.byref(de), C.byref(dt), C.byref(nf))
        if raise_on_fail:
            _check(code, "qflow_sweep_shard_end")
        return de.value, dt.value, nf.value, code

    def sweep_sharded(self, exchange, group=None, raise_on_fail: bool = True):
        """One sharded sweep with torch.distributed: begin, all_reduce(sum) of the exchange
        vector over `group`, end."""
        torch = _torch()
        self.sweep_shard_begin(exchange)
        torch.distributed.all_reduce(exchange, op=torch.distributed.ReduceOp.SUM, group=group)
        torch.cuda.current_stream(exchange.device).synchronize()
        return self.sweep_shard_end(exchange, raise_on_fail)

    def energy(self, per_space: bool = False):
        e = C.c_double()
        arr = np.empty(self.nspaces) if per_space else None
        _check(lib().qflow_energy(self._h, C.byref(e), _ptr(arr) if per_space else None), "qflow_energy")
        return (e.value, arr) if per_space else e.value

    def amplitudes(self):
        t1 = np.empty((self.nocc, self.nvir))
        t2 = np.empty((self.nocc, self.nocc, self.nvir, self.nvir))
        _check(lib().qflow_amplitudes(self._h, _ptr(t1), _ptr(t2)), "qflow_amplitudes")
        return t1, t2

    def set_amplitudes(self, t1, t2):
        t1, t2 = _f64(t1), _f64(t2)
        _check(lib().qflow_set_amplitudes(self._h, _ptr(t1), _ptr(t2)), "qflow_set_amplitudes")

    def order(self) -> np.ndarray:
        perm = np.empty(self.nspaces, dtype=np.int64)
        _check(lib().qflow_space_order(self._h, _ptr(perm)), "qflow_space_order")
        return perm

    def stats(self):
        it = np.empty(self.nspaces, dtype=np.int32)
        st = np.empty(self.nspaces, dtype=np.int32)
        _check(lib().qflow_space_stats(self._h, _ptr(it), _ptr(st)), "qflow_space_stats")
        return it, st

    def dressed(self):
        e0 = np.empty(1)
        F = np.empty((self.n, self.n))
        W = np.empty((self.n,) * 4)
        _check(lib().qflow_dressed(self._h, _ptr(e0), _ptr(F), _ptr(W)), "qflow_dressed")
        return float(e0[0]), F, W

    def last_sweep_info(self):
        ph = np.empty(3)
        nl = C.c_int64()
        _check(lib().qflow_last_sweep_info(self._h, _ptr(ph), C.byref(nl)), "qflow_last_sweep_info")
        return ph, nl.value

    def schedule(self) -> dict:
        p, ch, ct, gr, nc = C.c_int32(), C.c_int32(), C.c_int32(), C.c_int32(), C.c_int32()
        ms = (C.c_float * 8)()  # QFLOW_TUNE_MAX
        _check(lib().qflow_schedule(self._h, C.byref(p), C.byref(ch), C.byref(ct), C.byref(gr), ms, C.byref(nc)),
               "qflow_schedule")
        return {"persistent": bool(p.value), "chunk": ch.value, "warps_per_cta": ct.value, "graph": bool(gr.value),
                "candidate_ms": [float(ms[i]) for i in range(nc.value)]}

    def dress_schedule(self) -> dict:
        """Tile width of the mixed dressing's ladder + oooo product and the autotuner's times for
        32, 64 and 128 columns (empty when the width was fixed or cached)."""
        bn, nc = C.c_int32(), C.c_int32()
        ms = (C.c_float * 3)()  # QFLOW_LADDER_TUNE_MAX
        _check(lib().qflow_dress_schedule(self._h, C.byref(bn), ms, C.byref(nc)), "qflow_dress_schedule")
        return {"ladder_bn": bn.value, "candidate_ms": [float(ms[i]) for i in range(nc.value)]}

    def stream(self) -> int:
        return lib().qflow_stream(self._h) or 0

    # ---- warm-start network (guess="network") ----
    def mlp_set_model(self, model, hidden: int, has_stats: bool):
        model = np.ascontiguousarray(model, dtype=np.float32)
        if model.size != mlp_model_size(hidden):
            raise ValueError("model size does not match the hidden width")
        _check(lib().qflow_mlp_set_model(self._h, hidden, _ptr(model), int(has_stats)), "qflow_mlp_set_model")
        self._mlp_hidden = hidden

    def mlp_get_model(self) -> np.ndarray:
        out = np.empty(mlp_model_size(self._mlp_hidden), dtype=np.float32)
        _check(lib().qflow_mlp_get_model(self._h, _ptr(out)), "qflow_mlp_get_model")
        return out

    def mlp_collect(self, stride: int = 1, max_pairs: int = 1 << 20, target: str = "increment") -> int:
        """Store training pairs; target "increment" (Davidson guesses) or "pool" (flow warm start)."""
        n = C.c_int64()
        _check(lib().qflow_mlp_collect(self._h, {"increment": 0, "pool": 1}[target], stride, max_pairs,
                                       C.byref(n)), "qflow_mlp_collect")
        return n.value

    def mlp_warm_pool(self):
        """Set the pool to the model's prediction of every space's converged internal amplitudes."""
        _check(lib().qflow_mlp_warm_pool(self._h), "qflow_mlp_warm_pool")

    def mlp_train(self, epochs: int, batch: int, lr: float, order=None) -> np.ndarray:
        loss = np.empty(max(epochs, 0), dtype=np.float32)
        o = None if order is None else np.ascontiguousarray(order, dtype=np.int64)
        _check(lib().qflow_mlp_train(self._h, epochs, batch, lr, None if o is None else _ptr(o),
                                     _ptr(loss) if epochs > 0 else None), "qflow_mlp_train")
        return loss


# ---- device-level steps on torch CUDA tensors ------------------------------------------------

def _torch():
    import torch
    return torch


def _dptr(t) -> int:
    if not t.is_cuda or not t.is_contiguous():
        raise ValueError("device steps take contiguous CUDA tensors")
    return t.data_ptr()


def dress_device(h, eri, t1, t2, nocc: int, e0, F, W, work, stream: int = 0):
    """Step (a) on torch float64 CUDA tensors; `work` is a uint8 CUDA tensor of
    ``dress_workspace(n, nocc)`` bytes."""
    n = h.shape[0]
    _check(lib().qflow_dress_device(_dptr(h), _dptr(eri), _dptr(t1), _dptr(t2), n, nocc, _dptr(e0), _dptr(F),
                                    _dptr(W), _dptr(work), work.numel(), stream or None), "qflow_dress_device")


def dress_device_static(h, eri, t1, t2, nocc: int, e0, F, W, stream: int = 0):
    """Step (a) without any allocation: scratch comes from the library's static device array
    (see qflow_dress_device_static in include/qflow.h for the size limit and sharing rules)."""
    n = h.shape[0]
    _check(lib().qflow_dress_device_static(_dptr(h), _dptr(eri), _dptr(t1), _dptr(t2), n, nocc, _dptr(e0),
                                           _dptr(F), _dptr(W), stream or None), "qflow_dress_device_static")


def static_scratch_bytes() -> int:
    return int(lib().qflow_static_scratch_bytes())


def fma_peak(precision: str, stream: int = 0) -> float:
    """Measured FMA throughput of the current GPU in TFLOP/s (precision "fp64" or "mixed" = FP32)."""
    out = C.c_double(0.0)
    _check(lib().qflow_fma_peak(PREC[precision], C.byref(out), stream or None), "qflow_fma_peak")
    return float(out.value)


def dress_workspace(n: int, nocc: int) -> int:
    return int(lib().qflow_dress_workspace(n, nocc))


def solve_device(n: int, nocc: int, e0, F, W, size_class: int, spaces, energy, status, iters=None,
                 owner1=None, owner2=None, t1_old=None, t2_old=None, t1_new=None, t2_new=None,
                 guess=None, save_root: bool = False, space_base: int = 0, precision: str = "fp64",
                 max_iter: int = 60, tol: float | None = None, stream: int = 0):
    """Steps (b)+(c) for one size class on torch CUDA tensors (spaces: int32 [ns, 8])."""
    if tol is None:
        tol = 1e-6 if precision == "mixed" else 1e-9
    opt = lambda t: _dptr(t) if t is not None else None  # noqa: E731
    _check(lib().qflow_solve_device(n, nocc, _dptr(e0), _dptr(F), _dptr(W), size_class, _dptr(spaces),
                                    spaces.shape[0], space_base, opt(owner1), opt(owner2), opt(t1_old),
                                    opt(t2_old), opt(t1_new), opt(t2_new), _dptr(energy), _dptr(status),
                                    opt(iters), opt(guess), int(save_root), PREC[precision], max_iter, tol,
                                    stream or None), "qflow_solve_device")


# ---- warm-start network: sizes and device-level steps -----------------------------------------

MLP_NIN, MLP_NOUT = 708, 54


def mlp_param_count(n_in: int, hidden: int, n_out: int) -> int:
    return int(lib().qflow_mlp_param_count(n_in, hidden, n_out))


def mlp_model_size(hidden: int) -> int:
    return int(lib().qflow_mlp_model_size(hidden))


def mlp_workspace(n_in: int, hidden: int, n_out: int, rows: int) -> int:
    return int(lib().qflow_mlp_workspace(n_in, hidden, n_out, rows))


def mlp_forward_device(n_in, hidden, n_out, params, x, y, work, stream: int = 0):
    _check(lib().qflow_mlp_forward_device(n_in, hidden, n_out, _dptr(params), _dptr(x), x.shape[0], _dptr(y),
                                          _dptr(work), stream or None), "qflow_mlp_forward_device")


def mlp_grad_device(n_in, hidden, n_out, params, x, target, grad, loss, work, mask=None, stream: int = 0):
    _check(lib().qflow_mlp_grad_device(n_in, hidden, n_out, _dptr(params), _dptr(x), _dptr(target),
                                       None if mask is None else _dptr(mask), x.shape[0], _dptr(grad), _dptr(loss),
                                       _dptr(work), stream or None), "qflow_mlp_grad_device")


def mlp_adam_device(params, grad, m, v, step: int, lr: float, beta1: float = 0.9, beta2: float = 0.999,
                    eps: float = 1e-8, stream: int = 0):
    _check(lib().qflow_mlp_adam_device(params.numel(), _dptr(params), _dptr(grad), _dptr(m), _dptr(v), step, lr,
                                       beta1, beta2, eps, stream or None), "qflow_mlp_adam_device")


def mlp_features_device(n: int, F, W, spaces, features, stream: int = 0):
    _check(lib().qflow_mlp_features_device(n, _dptr(F), _dptr(W), _dptr(spaces), spaces.shape[0],
                                           _dptr(features), stream or None), "qflow_mlp_features_device")


def mlp_targets_device(roots, targets, stream: int = 0):
    _check(lib().qflow_mlp_targets_device(_dptr(roots), roots.shape[0], _dptr(targets), stream or None),
           "qflow_mlp_targets_device")


def mlp_guess_device(y, guess, stream: int = 0):
    _check(lib().qflow_mlp_guess_device(_dptr(y), y.shape[0], _dptr(guess), stream or None),
           "qflow_mlp_guess_device")


def gemm_tf32x3_device(A, B, C, err, stream: int = 0):
    """C = A @ B.T on the tensor cores (row-major float32 CUDA tensors; err: int32[1])."""
    M, K = A.shape
    N = B.shape[0]
    _check(lib().qflow_gemm_tf32x3_device(M, N, K, _dptr(A), A.stride(0), _dptr(B), B.stride(0), _dptr(C),
                                          C.stride(0), _dptr(err), stream or None), "qflow_gemm_tf32x3_device")
