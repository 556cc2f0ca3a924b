"""Thin Python binding of the C ABI in include/kt.h (argument marshalling only).

Every function here has the name of the C entry point it wraps and does no
arithmetic of its own: all work runs in libkt.so's CUDA kernels. PyTorch is
used for device memory (tensors) and streams. If the shared library is
missing and cannot be built, importing the engine raises; there is no CPU
fallback.
"""
from __future__ import annotations

import ctypes
import math
import os

import numpy as np

from . import build as _build

KT_OK, KT_EINVAL, KT_ENOMEM, KT_ECUDA, KT_ENOCONV, KT_ENUMERIC, KT_EZEROWEIGHT, KT_ETIMEOUT, KT_EUNSUPPORTED = range(9)
STATUS_NAMES = ["KT_OK", "KT_EINVAL", "KT_ENOMEM", "KT_ECUDA", "KT_ENOCONV", "KT_ENUMERIC", "KT_EZEROWEIGHT",
                "KT_ETIMEOUT", "KT_EUNSUPPORTED"]


def status_name(code: int) -> str:
    return STATUS_NAMES[code] if 0 <= code < len(STATUS_NAMES) else f"status {code}"


KT_FP64, KT_FP32_KRYLOV = 0, 1
KT_DENSITY_ONLY, KT_SECTOR_BLOCKS, KT_FP32_TRIDIAG64, KT_HOST_ONLY = 1, 2, 4, 256


class kt_model_params(ctypes.Structure):
    _fields_ = [("n_orb", ctypes.c_int32), ("U", ctypes.c_double), ("J", ctypes.c_double), ("Up", ctypes.c_double),
                ("mu", ctypes.c_double), ("delta", ctypes.POINTER(ctypes.c_double)), ("beta", ctypes.c_double),
                ("trunc_eps", ctypes.c_double), ("deg_tol", ctypes.c_double), ("krylov_tol", ctypes.c_double),
                ("krylov_pmax", ctypes.c_int32), ("precision", ctypes.c_int32), ("flags", ctypes.c_uint32)]


class kt_model_info(ctypes.Structure):
    _fields_ = [("n_orb", ctypes.c_int32), ("n_flavors", ctypes.c_int32), ("n_states", ctypes.c_int32),
                ("n_blocks", ctypes.c_int32), ("d_max", ctypes.c_int32), ("nnz_max", ctypes.c_int32),
                ("n_kept", ctypes.c_int32), ("precision", ctypes.c_int32), ("krylov_pmax", ctypes.c_int32),
                ("kernel_dmax", ctypes.c_int32), ("group_lanes", ctypes.c_int32), ("E0", ctypes.c_double),
                ("e_kept_max", ctypes.c_double),
                ("device_bytes", ctypes.c_size_t)]


STATS_FIELDS = ["walkers", "items", "items_alive", "items_vanished", "ops_applied", "intervals", "krylov_iters",
                "p_max", "noconv", "flops_vec", "flops_tri", "bytes_apply", "flops_alg", "flops_reorth"]


KT_P_HIST = 32
STATS_WORDS = len(STATS_FIELDS) + KT_P_HIST


class kt_stats(ctypes.Structure):
    _fields_ = [(f, ctypes.c_ulonglong) for f in STATS_FIELDS] + [("p_hist", ctypes.c_ulonglong * KT_P_HIST)]


class kt_sweep_params(ctypes.Structure):
    _fields_ = [("n_walkers", ctypes.c_int32), ("k_cap", ctypes.c_int32), ("n_tau", ctypes.c_int32),
                ("hyb", ctypes.c_void_p), ("n_bins", ctypes.c_int32), ("measure_obs", ctypes.c_int32),
                ("cache_ops", ctypes.c_int32)]


class kt_sweep_state(ctypes.Structure):
    _fields_ = [(f, ctypes.c_void_p) for f in ("lens", "tau", "flavor", "dagger", "sign", "trace_sign",
                                                "trace_logabs", "det_logabs", "order")]


class kt_sweep_accum(ctypes.Structure):
    _fields_ = [(f, ctypes.c_void_p) for f in ("g_tau", "sign_sum", "order_sum", "obs_sum")]


class kt_seq_batch(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int32), ("offsets", ctypes.c_void_p), ("tau", ctypes.c_void_p),
                ("flavor", ctypes.c_void_p), ("dagger", ctypes.c_void_p)]


class kt_move_batch(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_void_p), ("flavor", ctypes.c_void_p), ("t_dag", ctypes.c_void_p),
                ("t_ann", ctypes.c_void_p), ("rem_idx", ctypes.c_void_p)]


# Every function the header declares (checked by the CPU test suite).
ABI_FUNCTIONS = ["kt_status_string", "kt_model_create", "kt_model_query", "kt_model_kept", "kt_model_spectrum",
                 "kt_model_destroy", "kt_workspace_size", "kt_trace", "kt_trace_ratio", "kt_timing_begin",
                 "kt_timing_end", "kt_model_set_tiling", "kt_autotune", "kt_trace_ratio_static",
                 "kt_measure_workspace_size", "kt_measure",
                 "kt_sweep_create", "kt_sweep_run", "kt_sweep_get_state", "kt_sweep_get_accumulators",
                 "kt_sweep_counters", "kt_sweep_reset_accumulators", "kt_sweep_destroy",
                 "kt_sweep_set_configs", "kt_gemm_bf16", "kt_mlp_create", "kt_mlp_num_params",
                 "kt_mlp_set_params", "kt_mlp_get_params", "kt_mlp_forward", "kt_mlp_backward", "kt_mlp_get_grads",
                 "kt_mlp_adam", "kt_mlp_error", "kt_mlp_destroy", "kt_mlp_get_tape", "kt_sweep_feature_size",
                 "kt_sweep_collect",
                 "kt_sweep_set_surrogate", "kt_sweep_run_da", "kt_sweep_set_stats", "kt_ratio_cache_create",
                 "kt_ratio_cache_build", "kt_trace_ratio_cached", "kt_ratio_cache_destroy", "kt_ratio_cache_propose",
                 "kt_ratio_cache_commit", "kt_sweep_refresh", "kt_sweep_run_da_multi", "kt_sweep_memory_bytes"]

KT_SWEEP_NCOUNTERS = 10
KT_DA_MAX_TRIES = 16
KT_MLP_HIDDEN = 256
SWEEP_COUNTERS = ["insert_proposed", "insert_accepted", "remove_proposed", "remove_accepted", "null_moves",
                  "refused_at_k_cap", "trace_errors", "measurements", "stage1_rejected", "trace_evaluations"]

_lib = None


def library_path() -> str:
    return _build.LIB


def load():
    """Load libkt.so (building it in-tree first if it is missing or stale)."""
    global _lib
    if _lib is not None:
        return _lib
    path = _build.build()
    if not os.path.exists(path):
        raise RuntimeError("libkt.so is missing: build it with paper_0908_0681_gb300.build")
    lib = ctypes.CDLL(path)
    vp, i32 = ctypes.c_void_p, ctypes.c_int32
    lib.kt_status_string.argtypes = [ctypes.c_int]
    lib.kt_status_string.restype = ctypes.c_char_p
    lib.kt_model_create.argtypes = [ctypes.POINTER(kt_model_params), ctypes.POINTER(vp)]
    lib.kt_model_query.argtypes = [vp, ctypes.POINTER(kt_model_info)]
    lib.kt_model_kept.argtypes = [vp, vp, vp, vp, vp]
    lib.kt_model_spectrum.argtypes = [vp, vp]
    lib.kt_model_destroy.argtypes = [vp]
    lib.kt_model_destroy.restype = None
    lib.kt_workspace_size.argtypes = [vp, i32, ctypes.POINTER(ctypes.c_size_t)]
    lib.kt_trace.argtypes = [vp, ctypes.POINTER(kt_seq_batch), vp, vp, vp, vp, vp, ctypes.c_size_t, vp]
    lib.kt_trace_ratio.argtypes = [vp, ctypes.POINTER(kt_seq_batch), vp, vp, ctypes.POINTER(kt_move_batch),
                                   vp, vp, vp, vp, vp, ctypes.c_size_t, vp]
    lib.kt_measure_workspace_size.argtypes = [vp, i32, ctypes.POINTER(ctypes.c_size_t)]
    lib.kt_measure.argtypes = [vp, ctypes.POINTER(kt_seq_batch), vp, vp, vp, vp, vp, vp, ctypes.c_size_t, vp]
    lib.kt_sweep_create.argtypes = [vp, ctypes.POINTER(kt_sweep_params), ctypes.POINTER(vp)]
    lib.kt_sweep_memory_bytes.argtypes = [vp, ctypes.POINTER(kt_sweep_params), i32, ctypes.POINTER(ctypes.c_size_t)]
    lib.kt_sweep_run.argtypes = [vp, i32, vp, i32, vp]
    lib.kt_sweep_set_configs.argtypes = [vp, ctypes.POINTER(kt_seq_batch)]
    lib.kt_gemm_bf16.argtypes = [vp, i32, vp, i32, vp, i32, i32, i32, i32, vp, vp]
    lib.kt_mlp_create.argtypes = [i32, i32, ctypes.POINTER(vp)]
    lib.kt_mlp_num_params.argtypes = [vp, ctypes.POINTER(ctypes.c_int64)]
    lib.kt_mlp_set_params.argtypes = [vp, vp]
    lib.kt_mlp_get_params.argtypes = [vp, vp]
    lib.kt_mlp_forward.argtypes = [vp, vp, i32, vp, vp]
    lib.kt_mlp_backward.argtypes = [vp, vp, vp, i32, vp, vp]
    lib.kt_mlp_get_grads.argtypes = [vp, vp]
    lib.kt_mlp_get_tape.argtypes = [vp, i32, vp, vp, vp, vp, vp, vp, vp]
    lib.kt_mlp_adam.argtypes = [vp, ctypes.c_float, vp]
    lib.kt_mlp_error.argtypes = [vp, ctypes.POINTER(ctypes.c_int32)]
    lib.kt_mlp_destroy.argtypes = [vp]
    lib.kt_mlp_destroy.restype = None
    lib.kt_sweep_feature_size.argtypes = [vp, ctypes.POINTER(ctypes.c_int32)]
    lib.kt_sweep_collect.argtypes = [vp, i32, vp, vp, vp, vp, i32, vp]
    lib.kt_sweep_set_surrogate.argtypes = [vp, vp]
    lib.kt_sweep_run_da.argtypes = [vp, i32, vp, i32, vp]
    lib.kt_sweep_run_da_multi.argtypes = [vp, i32, i32, vp, i32, vp]
    lib.kt_sweep_set_stats.argtypes = [vp, vp]
    lib.kt_ratio_cache_create.argtypes = [vp, i32, i32, ctypes.POINTER(vp)]
    lib.kt_ratio_cache_build.argtypes = [vp, ctypes.POINTER(kt_seq_batch), vp]
    lib.kt_trace_ratio_cached.argtypes = [vp, ctypes.POINTER(kt_seq_batch), vp, vp, ctypes.POINTER(kt_move_batch),
                                          vp, vp, vp, vp, vp]
    lib.kt_ratio_cache_propose.argtypes = [vp, ctypes.POINTER(kt_seq_batch), vp, vp, ctypes.POINTER(kt_move_batch),
                                           vp, vp, vp, vp, vp]
    lib.kt_ratio_cache_commit.argtypes = [vp, vp, vp, vp]
    lib.kt_ratio_cache_destroy.argtypes = [vp]
    lib.kt_ratio_cache_destroy.restype = None
    lib.kt_sweep_get_state.argtypes = [vp, ctypes.POINTER(kt_sweep_state), vp]
    lib.kt_sweep_get_accumulators.argtypes = [vp, ctypes.POINTER(kt_sweep_accum), vp]
    lib.kt_sweep_counters.argtypes = [vp, vp]
    lib.kt_sweep_reset_accumulators.argtypes = [vp, vp]
    lib.kt_sweep_refresh.argtypes = [vp, vp, vp]
    lib.kt_sweep_destroy.argtypes = [vp]
    lib.kt_sweep_destroy.restype = None
    lib.kt_timing_begin.argtypes = [vp, i32]
    lib.kt_model_set_tiling.argtypes = [vp, i32]
    lib.kt_trace_ratio_static.argtypes = [vp, ctypes.POINTER(kt_seq_batch), vp, vp, ctypes.POINTER(kt_move_batch),
                                          vp, vp, vp, vp, vp]
    lib.kt_autotune.argtypes = [vp, ctypes.POINTER(kt_seq_batch), vp, vp, vp, vp, ctypes.c_size_t, vp,
                                ctypes.POINTER(ctypes.c_int32)]
    lib.kt_timing_end.argtypes = [vp, vp, ctypes.POINTER(ctypes.c_int32)]
    for f in ABI_FUNCTIONS:
        if f not in ("kt_status_string", "kt_model_destroy", "kt_sweep_destroy", "kt_mlp_destroy",
                     "kt_ratio_cache_destroy"):
            getattr(lib, f).restype = ctypes.c_int
    _lib = lib
    return lib


class KtError(RuntimeError):
    def __init__(self, code: int, what: str):
        super().__init__(f"{what}: {kt_status_string(code)} ({code})")
        self.code = code


def _check(code: int, what: str):
    if code != KT_OK:
        raise KtError(code, what)


def kt_status_string(code: int) -> str:
    return load().kt_status_string(int(code)).decode()


class KtModel:
    """Owning handle of a kt_model* (kt_model_destroy on close/garbage collection)."""

    def __init__(self, handle, params: dict):
        self.handle = handle
        self.params = params

    def close(self):
        if self.handle:
            load().kt_model_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def kt_model_create(n_orb: int, U: float, J: float, mu: float, beta: float, delta=None, Up: float = math.nan,
                    trunc_eps: float = 1e-10, deg_tol: float = 1e-9, krylov_tol: float = 1e-12,
                    krylov_pmax: int = 0, precision: int = KT_FP32_KRYLOV, flags: int = 0) -> KtModel:
    lib = load()
    d = np.zeros(n_orb, dtype=np.float64)
    if delta is not None:
        d[:] = np.asarray(delta, dtype=np.float64)
    p = kt_model_params(int(n_orb), float(U), float(J), float(Up), float(mu),
                        d.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), float(beta), float(trunc_eps),
                        float(deg_tol), float(krylov_tol), int(krylov_pmax), int(precision), int(flags))
    h = ctypes.c_void_p()
    _check(lib.kt_model_create(ctypes.byref(p), ctypes.byref(h)), "kt_model_create")
    return KtModel(h, dict(n_orb=n_orb, U=U, J=J, mu=mu, beta=beta, delta=d.tolist(), Up=Up, trunc_eps=trunc_eps,
                           deg_tol=deg_tol, krylov_tol=krylov_tol, krylov_pmax=krylov_pmax, precision=precision,
                           flags=flags))


def kt_model_query(m: KtModel) -> dict:
    info = kt_model_info()
    _check(load().kt_model_query(m.handle, ctypes.byref(info)), "kt_model_query")
    return {f: getattr(info, f) for f, _ in kt_model_info._fields_}


def kt_model_kept(m: KtModel) -> dict:
    nk = kt_model_query(m)["n_kept"]
    e = np.zeros(nk, np.float64); nu = np.zeros(nk, np.int32); nd = np.zeros(nk, np.int32); mk = np.zeros(nk, np.int32)
    _check(load().kt_model_kept(m.handle, e.ctypes.data, nu.ctypes.data, nd.ctypes.data, mk.ctypes.data), "kt_model_kept")
    return {"e_minus_e0": e, "n_up": nu, "n_dn": nd, "single_mask": mk}


def kt_model_spectrum(m: KtModel) -> np.ndarray:
    ns = kt_model_query(m)["n_states"]
    e = np.zeros(ns, np.float64)
    _check(load().kt_model_spectrum(m.handle, e.ctypes.data), "kt_model_spectrum")
    return e


def kt_workspace_size(m: KtModel, n: int) -> int:
    b = ctypes.c_size_t()
    _check(load().kt_workspace_size(m.handle, int(n), ctypes.byref(b)), "kt_workspace_size")
    return int(b.value)


def _ptr(t) -> int | None:
    return None if t is None else int(t.data_ptr())


def _stream_handle(stream) -> int | None:
    if stream is None:
        import torch
        return int(torch.cuda.current_stream().cuda_stream)
    return int(getattr(stream, "cuda_stream", stream))


def seq_batch(offsets, tau, flavor, dagger) -> kt_seq_batch:
    """kt_seq_batch over device tensors (int32 offsets, float64 tau, uint8 flavor/dagger)."""
    return kt_seq_batch(int(offsets.numel() - 1), _ptr(offsets), _ptr(tau), _ptr(flavor), _ptr(dagger))


def move_batch(kind, flavor, t_dag, t_ann, rem_idx) -> kt_move_batch:
    return kt_move_batch(_ptr(kind), _ptr(flavor), _ptr(t_dag), _ptr(t_ann), _ptr(rem_idx))


def kt_trace(m: KtModel, batch: kt_seq_batch, sign, logabs, status, stats=None, workspace=None, stream=None) -> None:
    ws_bytes = 0 if workspace is None else workspace.numel() * workspace.element_size()
    _check(load().kt_trace(m.handle, ctypes.byref(batch), _ptr(sign), _ptr(logabs), _ptr(status), _ptr(stats),
                           _ptr(workspace), ws_bytes, _stream_handle(stream)), "kt_trace")


def kt_trace_ratio(m: KtModel, cur: kt_seq_batch, cur_sign, cur_logabs, moves: kt_move_batch, sign, logratio, status,
                   stats=None, workspace=None, stream=None) -> None:
    ws_bytes = 0 if workspace is None else workspace.numel() * workspace.element_size()
    _check(load().kt_trace_ratio(m.handle, ctypes.byref(cur), _ptr(cur_sign), _ptr(cur_logabs), ctypes.byref(moves),
                                 _ptr(sign), _ptr(logratio), _ptr(status), _ptr(stats), _ptr(workspace), ws_bytes,
                                 _stream_handle(stream)), "kt_trace_ratio")


def kt_measure_workspace_size(m: KtModel, n: int) -> int:
    b = ctypes.c_size_t()
    _check(load().kt_measure_workspace_size(m.handle, int(n), ctypes.byref(b)), "kt_measure_workspace_size")
    return int(b.value)


def measure_nobs(n_orb: int) -> int:
    """KT_MEASURE_NOBS: observables per walker returned by kt_measure."""
    return 3 * n_orb + 1 + (n_orb + 1) ** 2


def kt_measure(m: KtModel, batch: kt_seq_batch, sign, logabs, obs, status, stats=None, workspace=None,
               stream=None) -> None:
    ws_bytes = 0 if workspace is None else workspace.numel() * workspace.element_size()
    _check(load().kt_measure(m.handle, ctypes.byref(batch), _ptr(sign), _ptr(logabs), _ptr(obs), _ptr(status),
                             _ptr(stats), _ptr(workspace), ws_bytes, _stream_handle(stream)), "kt_measure")


class KtSweep:
    """Owning handle of a kt_sweep (destroyed with the object); keeps its model alive."""

    def __init__(self, model: KtModel, hyb: np.ndarray, n_walkers: int, k_cap: int = 64, n_bins: int = 100,
                 measure_obs: bool = False, cache_ops: int = 0):
        self.model = model
        self._hyb = np.ascontiguousarray(hyb, dtype=np.float64)
        p = kt_sweep_params(int(n_walkers), int(k_cap), int(self._hyb.shape[1] - 1),
                            self._hyb.ctypes.data_as(ctypes.c_void_p), int(n_bins), 1 if measure_obs else 0,
                            int(cache_ops))
        h = ctypes.c_void_p()
        _check(load().kt_sweep_create(model.handle, ctypes.byref(p), ctypes.byref(h)), "kt_sweep_create")
        self.handle = h
        self.n_walkers, self.k_cap, self.n_bins = int(n_walkers), int(k_cap), int(n_bins)

    def __del__(self):
        h = getattr(self, "handle", None)
        if h is not None and _lib is not None:
            _lib.kt_sweep_destroy(h)
            self.handle = None


def kt_sweep_memory_bytes(model: KtModel, n_walkers: int, k_cap: int = 64, n_tau: int = 2000, n_bins: int = 100,
                          measure_obs: bool = False, cache_ops: int = 0, tries: int = 0) -> int:
    """Device bytes of a sweep with these parameters (kt_sweep_memory_bytes), plus the multi-try
    proposal slots of `tries` tries."""
    p = kt_sweep_params(int(n_walkers), int(k_cap), int(n_tau), None, int(n_bins), 1 if measure_obs else 0,
                        int(cache_ops))
    out = ctypes.c_size_t()
    _check(load().kt_sweep_memory_bytes(model.handle, ctypes.byref(p), int(tries), ctypes.byref(out)),
           "kt_sweep_memory_bytes")
    return int(out.value)


class KtRatioCache:
    """Owning handle of a kt_ratio_cache (destroyed with the object); keeps its model alive."""

    def __init__(self, model: KtModel, n_walkers: int, max_ops: int):
        self.model = model
        h = ctypes.c_void_p()
        _check(load().kt_ratio_cache_create(model.handle, int(n_walkers), int(max_ops), ctypes.byref(h)),
               "kt_ratio_cache_create")
        self.handle = h
        self.n_walkers, self.max_ops = int(n_walkers), int(max_ops)

    def __del__(self):
        h = getattr(self, "handle", None)
        if h is not None and _lib is not None:
            _lib.kt_ratio_cache_destroy(h)
            self.handle = None


def kt_ratio_cache_build(c: KtRatioCache, batch: kt_seq_batch, stream=None) -> None:
    _check(load().kt_ratio_cache_build(c.handle, ctypes.byref(batch), _stream_handle(stream)), "kt_ratio_cache_build")


def kt_trace_ratio_cached(c: KtRatioCache, cur: kt_seq_batch, cur_sign, cur_logabs, moves: kt_move_batch, sign,
                          logratio, status, stats=None, stream=None) -> None:
    _check(load().kt_trace_ratio_cached(c.handle, ctypes.byref(cur), _ptr(cur_sign), _ptr(cur_logabs),
                                        ctypes.byref(moves), _ptr(sign), _ptr(logratio), _ptr(status), _ptr(stats),
                                        _stream_handle(stream)), "kt_trace_ratio_cached")


def kt_ratio_cache_propose(c: KtRatioCache, cur: kt_seq_batch, cur_sign, cur_logabs, moves: kt_move_batch, sign,
                           logratio, status, stats=None, stream=None) -> None:
    _check(load().kt_ratio_cache_propose(c.handle, ctypes.byref(cur), _ptr(cur_sign), _ptr(cur_logabs),
                                         ctypes.byref(moves), _ptr(sign), _ptr(logratio), _ptr(status), _ptr(stats),
                                         _stream_handle(stream)), "kt_ratio_cache_propose")


def kt_ratio_cache_commit(c: KtRatioCache, accepted, status, stream=None) -> None:
    _check(load().kt_ratio_cache_commit(c.handle, _ptr(accepted), _ptr(status), _stream_handle(stream)),
           "kt_ratio_cache_commit")


def kt_sweep_set_stats(s: KtSweep, stats) -> None:
    """Count the trace pipeline's work of the following steps into a device kt_stats
    tensor (engine.new_stats); None stops counting."""
    _check(load().kt_sweep_set_stats(s.handle, _ptr(stats)), "kt_sweep_set_stats")


def kt_sweep_run(s: KtSweep, n_steps: int, uniforms, meas_every: int = 0, stream=None) -> None:
    _check(load().kt_sweep_run(s.handle, int(n_steps), _ptr(uniforms), int(meas_every), _stream_handle(stream)),
           "kt_sweep_run")


def kt_sweep_set_configs(s: KtSweep, offsets: np.ndarray, tau: np.ndarray, flavor: np.ndarray,
                         dagger: np.ndarray) -> None:
    """HOST CSR arrays (int32 offsets, float64 tau, uint8 flavor / dagger)."""
    arrs = [np.ascontiguousarray(a, dtype=t) for a, t in ((offsets, np.int32), (tau, np.float64),
                                                         (flavor, np.uint8), (dagger, np.uint8))]
    b = kt_seq_batch(len(arrs[0]) - 1, *[a.ctypes.data_as(ctypes.c_void_p) for a in arrs])
    _check(load().kt_sweep_set_configs(s.handle, ctypes.byref(b)), "kt_sweep_set_configs")


def kt_sweep_get_state(s: KtSweep, stream=None, **dst) -> None:
    st = kt_sweep_state(**{k: _ptr(v) for k, v in dst.items()})
    _check(load().kt_sweep_get_state(s.handle, ctypes.byref(st), _stream_handle(stream)), "kt_sweep_get_state")


def kt_sweep_get_accumulators(s: KtSweep, stream=None, **dst) -> None:
    ac = kt_sweep_accum(**{k: _ptr(v) for k, v in dst.items()})
    _check(load().kt_sweep_get_accumulators(s.handle, ctypes.byref(ac), _stream_handle(stream)),
           "kt_sweep_get_accumulators")


def kt_sweep_counters(s: KtSweep) -> dict:
    out = (ctypes.c_ulonglong * KT_SWEEP_NCOUNTERS)()
    _check(load().kt_sweep_counters(s.handle, out), "kt_sweep_counters")
    return dict(zip(SWEEP_COUNTERS, [int(x) for x in out]))


def kt_sweep_refresh(s: KtSweep, stream=None) -> dict:
    """Recompute M, log|det|, the permutation sign and the trace of every walker from scratch
    (synchronises); returns the deviations of the tracked values."""
    out = np.zeros(4, dtype=np.float64)
    _check(load().kt_sweep_refresh(s.handle, out.ctypes.data_as(ctypes.c_void_p), _stream_handle(stream)),
           "kt_sweep_refresh")
    return {"trace_log": float(out[0]), "det_log": float(out[1]), "sign_mismatches": int(out[2]),
            "unchanged": int(out[3])}


def kt_sweep_reset_accumulators(s: KtSweep, stream=None) -> None:
    _check(load().kt_sweep_reset_accumulators(s.handle, _stream_handle(stream)), "kt_sweep_reset_accumulators")


def kt_gemm_bf16(A, B, C, err, stream=None) -> None:
    """C = A . B^T on the tensor cores (A [M, K], B [N, K] bfloat16; C [M, N] float32; err int32[1])."""
    M, K = A.shape
    N = B.shape[0]
    _check(load().kt_gemm_bf16(_ptr(A), A.stride(0), _ptr(B), B.stride(0), _ptr(C), C.stride(0), M, N, K, _ptr(err),
                               _stream_handle(stream)), "kt_gemm_bf16")


class KtMlp:
    """Owning handle of a kt_mlp (the delayed-acceptance surrogate network)."""

    def __init__(self, n_in: int, max_batch: int):
        h = ctypes.c_void_p()
        _check(load().kt_mlp_create(int(n_in), int(max_batch), ctypes.byref(h)), "kt_mlp_create")
        self.handle = h
        self.n_in, self.max_batch = int(n_in), int(max_batch)
        c = ctypes.c_int64()
        _check(_lib.kt_mlp_num_params(h, ctypes.byref(c)), "kt_mlp_num_params")
        self.n_params = int(c.value)

    def __del__(self):
        h = getattr(self, "handle", None)
        if h is not None and _lib is not None:
            _lib.kt_mlp_destroy(h)
            self.handle = None


def kt_mlp_set_params(n: KtMlp, params: np.ndarray) -> None:
    a = np.ascontiguousarray(params, dtype=np.float32)
    assert a.size == n.n_params
    _check(load().kt_mlp_set_params(n.handle, a.ctypes.data_as(ctypes.c_void_p)), "kt_mlp_set_params")


def kt_mlp_get_params(n: KtMlp) -> np.ndarray:
    a = np.zeros(n.n_params, dtype=np.float32)
    _check(load().kt_mlp_get_params(n.handle, a.ctypes.data_as(ctypes.c_void_p)), "kt_mlp_get_params")
    return a


def kt_mlp_get_grads(n: KtMlp) -> np.ndarray:
    a = np.zeros(n.n_params, dtype=np.float32)
    _check(load().kt_mlp_get_grads(n.handle, a.ctypes.data_as(ctypes.c_void_p)), "kt_mlp_get_grads")
    return a


def kt_mlp_get_tape(n: KtMlp, B: int) -> dict:
    """Intermediate values of the last kt_mlp_backward on B rows (host numpy arrays; BF16
    entries as uint16 bit patterns, dz1 transposed [256][B])."""
    H = KT_MLP_HIDDEN
    t = {"z1": np.zeros((B, H), np.float32), "h1": np.zeros((B, H), np.uint16), "z2": np.zeros((B, H), np.float32),
         "dy": np.zeros(B, np.float32), "dz2": np.zeros((B, H), np.uint16), "dh1": np.zeros((B, H), np.float32),
         "dz1": np.zeros((H, B), np.uint16)}
    vp = ctypes.c_void_p
    _check(load().kt_mlp_get_tape(n.handle, B, *(t[k].ctypes.data_as(vp) for k in
                                                ("z1", "h1", "z2", "dy", "dz2", "dh1", "dz1"))), "kt_mlp_get_tape")
    return t


def kt_mlp_forward(n: KtMlp, X, y, stream=None) -> None:
    _check(load().kt_mlp_forward(n.handle, _ptr(X), X.shape[0], _ptr(y), _stream_handle(stream)), "kt_mlp_forward")


def kt_mlp_backward(n: KtMlp, X, t, loss=None, stream=None) -> None:
    _check(load().kt_mlp_backward(n.handle, _ptr(X), _ptr(t), X.shape[0], _ptr(loss), _stream_handle(stream)),
           "kt_mlp_backward")


def kt_mlp_adam(n: KtMlp, lr: float, stream=None) -> None:
    _check(load().kt_mlp_adam(n.handle, ctypes.c_float(lr), _stream_handle(stream)), "kt_mlp_adam")


def kt_mlp_error(n: KtMlp) -> int:
    e = ctypes.c_int32()
    _check(load().kt_mlp_error(n.handle, ctypes.byref(e)), "kt_mlp_error")
    return int(e.value)


def kt_sweep_feature_size(s: KtSweep) -> int:
    n = ctypes.c_int32()
    _check(load().kt_sweep_feature_size(s.handle, ctypes.byref(n)), "kt_sweep_feature_size")
    return int(n.value)


def kt_sweep_collect(s: KtSweep, n_steps: int, uniforms, features, targets, count, stream=None) -> None:
    _check(load().kt_sweep_collect(s.handle, int(n_steps), _ptr(uniforms), _ptr(features), _ptr(targets), _ptr(count),
                                   features.shape[0], _stream_handle(stream)), "kt_sweep_collect")


def kt_sweep_set_surrogate(s: KtSweep, net) -> None:
    _check(load().kt_sweep_set_surrogate(s.handle, None if net is None else net.handle), "kt_sweep_set_surrogate")
    s.surrogate = net   # keep the network alive while attached


def kt_sweep_run_da(s: KtSweep, n_steps: int, uniforms, meas_every: int = 0, stream=None) -> None:
    _check(load().kt_sweep_run_da(s.handle, int(n_steps), _ptr(uniforms), int(meas_every), _stream_handle(stream)),
           "kt_sweep_run_da")


def kt_sweep_run_da_multi(s: KtSweep, n_steps: int, tries: int, uniforms, meas_every: int = 0, stream=None) -> None:
    _check(load().kt_sweep_run_da_multi(s.handle, int(n_steps), int(tries), _ptr(uniforms), int(meas_every),
                                        _stream_handle(stream)), "kt_sweep_run_da_multi")


def kt_model_set_tiling(m: KtModel, group_lanes: int) -> None:
    _check(load().kt_model_set_tiling(m.handle, int(group_lanes)), "kt_model_set_tiling")


def kt_autotune(m: KtModel, batch: kt_seq_batch, sign, logabs, status, workspace, stream=None) -> int:
    g = ctypes.c_int32()
    ws_bytes = workspace.numel() * workspace.element_size()
    _check(load().kt_autotune(m.handle, ctypes.byref(batch), _ptr(sign), _ptr(logabs), _ptr(status), _ptr(workspace),
                              ws_bytes, _stream_handle(stream), ctypes.byref(g)), "kt_autotune")
    return int(g.value)


def kt_timing_begin(m: KtModel, max_launches: int) -> None:
    _check(load().kt_timing_begin(m.handle, int(max_launches)), "kt_timing_begin")


STAGES = ["prep", "prune", "items", "reduce"]


def kt_timing_end(m: KtModel):
    """(dict stage -> summed ms, number of timed calls)."""
    ms = np.zeros(4, np.float64)
    n = ctypes.c_int32()
    _check(load().kt_timing_end(m.handle, ms.ctypes.data, ctypes.byref(n)), "kt_timing_end")
    return dict(zip(STAGES, ms.tolist())), int(n.value)


KT_STATIC_SCRATCH_BYTES = 8 << 20


def kt_trace_ratio_static(m: KtModel, cur: kt_seq_batch, cur_sign, cur_logabs, moves: kt_move_batch, sign, logratio,
                          status, stats=None, stream=None) -> None:
    """kt_trace_ratio without a workspace (scratch in the library's fixed device array)."""
    _check(load().kt_trace_ratio_static(m.handle, ctypes.byref(cur), _ptr(cur_sign), _ptr(cur_logabs),
                                        ctypes.byref(moves), _ptr(sign), _ptr(logratio), _ptr(status), _ptr(stats),
                                        _stream_handle(stream)), "kt_trace_ratio_static")


def stats_from_tensor(t) -> dict:
    """Decode a kt_stats held in a uint64 tensor of STATS_WORDS words. `p_hist` is the list of
    propagations by stopping Krylov dimension p (index p; the last entry counts p >= KT_P_HIST - 1)."""
    v = t.cpu().numpy().astype(np.uint64)
    d = {f: int(v[i]) for i, f in enumerate(STATS_FIELDS)}
    d["p_hist"] = [int(x) for x in v[len(STATS_FIELDS):STATS_WORDS]]
    return d
