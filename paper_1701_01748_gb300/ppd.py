"""Python binding of libppd (argument marshalling only).

Every function here has the name of the C entry point it calls (see
``include/ppd.h``); all computation happens in the CUDA library.  Loading
fails loudly when ``libppd.so`` has not been built: there is no fallback.
"""
from __future__ import annotations

import ctypes as ct
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libppd.so")

PPD_OK = 0
PPD_ERR_INVALID_ARG = -1
PPD_ERR_OOM = -2
PPD_ERR_CUDA = -3
PPD_ERR_NONFINITE = -4
PPD_ERR_TIMEOUT = -5
PPD_ERR_NOT_READY = -6
PPD_ERR_UNSUPPORTED = -7
PPD_FP64_PLAIN = 0
PPD_FP32_FP64NORMS = 1
PPD_INNER_WARM = 0
PPD_INNER_CURRENT = 1
PPD_INNER_FB = 0
PPD_INNER_FISTA = 1
PPD_NORM_LANCZOS = 0
PPD_NORM_POWER = 1


class ppd_config(ct.Structure):
    _fields_ = [("n0", ct.c_int32), ("n1", ct.c_int32), ("oversample", ct.c_int32),
                ("kernel_width", ct.c_int32), ("kb_beta", ct.c_double), ("n_blocks", ct.c_int32),
                ("wavelet_levels", ct.c_int32), ("n_itr", ct.c_int32), ("tau", ct.c_double),
                ("lambda_", ct.c_double), ("kappa", ct.c_double), ("eta", ct.c_double),
                ("zeta", ct.c_double), ("precision", ct.c_int32), ("precond", ct.c_int32),
                ("inner_init", ct.c_int32), ("use_graph", ct.c_int32), ("tile", ct.c_int32),
                ("chunk", ct.c_int32), ("power_iters", ct.c_int32), ("power_tol", ct.c_double),
                ("stream", ct.c_void_p), ("inner_solver", ct.c_int32), ("inner_tol", ct.c_double),
                ("stop_tol", ct.c_double), ("stop_eps_factor", ct.c_double), ("stop_every", ct.c_int32),
                ("grid_warps", ct.c_int32), ("seed", ct.c_uint64), ("norm_method", ct.c_int32), ("launch_overlap", ct.c_int32),
                ("degrid_threads", ct.c_int32), ("pad1", ct.c_int32)]


class ppd_stats(ct.Structure):
    _fields_ = [("iters_done", ct.c_int32), ("status", ct.c_int32), ("rel_var", ct.c_double),
                ("snr_db", ct.c_double), ("max_res_over_eps", ct.c_double),
                ("block_residual", ct.POINTER(ct.c_double)), ("inner_steps", ct.POINTER(ct.c_int32)),
                ("stopped", ct.c_int32), ("iters_run", ct.c_int32)]


class ppd_params(ct.Structure):
    _fields_ = [("eta", ct.c_double), ("zeta", ct.c_double), ("tau", ct.c_double),
                ("kappa", ct.c_double), ("op_norm_sq", ct.c_double), ("power_iters_done", ct.c_int32),
                ("K0", ct.c_int32), ("K1", ct.c_int32), ("tile", ct.c_int32), ("chunk", ct.c_int32),
                ("n_chunks", ct.c_int64),
                ("M", ct.c_int64), ("convergence_lhs", ct.c_double),
                ("psiw_norm_sq", ct.c_double), ("alpha", ct.c_double), ("grid_warps", ct.c_int32),
                ("degrid_threads", ct.c_int32)]


class PPDError(RuntimeError):
    def __init__(self, status: int, where: str):
        self.status = status
        msg = _lib().ppd_last_error().decode()
        super().__init__(f"{where}: {_lib().ppd_status_string(status).decode()} ({status}): {msg}")


_LIB = None


def _lib():
    global _LIB
    if _LIB is None:
        if not os.path.exists(LIB_PATH):
            raise ImportError(f"libppd.so is not built ({LIB_PATH}); run __graft_entry__.build()")
        L = ct.CDLL(LIB_PATH)
        P, I, I32, I64, D, V = ct.c_void_p, ct.c_int, ct.c_int32, ct.c_int64, ct.POINTER(ct.c_double), None
        sig = {
            "ppd_config_default": (V, [ct.POINTER(ppd_config)]),
            "ppd_create": (I, [ct.POINTER(P), ct.POINTER(ppd_config)]),
            "ppd_destroy": (V, [P]),
            "ppd_set_visibilities": (I, [P, I64, D, D, ct.POINTER(ct.c_int32)]),
            "ppd_set_weights": (I, [P, D, D, D]),
            "ppd_set_ground_truth": (I, [P, D, I64]),
            "ppd_iterate": (I, [P, I32, ct.POINTER(ppd_stats)]),
            "ppd_get_image": (I, [P, D, I64]),
            "ppd_get_params": (I, [P, ct.POINTER(ppd_params)]),
            "ppd_get_bins": (I, [P, ct.POINTER(ct.c_int64), ct.POINTER(ct.c_int32),
                                 ct.POINTER(ct.c_int32), ct.POINTER(ct.c_int32)]),
            "ppd_autotune": (I, [P, I32, ct.POINTER(ct.c_int32), ct.POINTER(ct.c_int32)]),
            "ppd_get_state": (I, [P, P, ct.POINTER(ct.c_int64)]),
            "ppd_group_create": (I, [ct.POINTER(P), ct.POINTER(P), I32]),
            "ppd_group_iterate": (I, [P, I32]),
            "ppd_group_destroy": (V, [P]),
            "ppd_set_state": (I, [P, P, I64]),
            "ppd_set_prior_weights": (I, [P, D, I64]),
            "ppd_reweight": (I, [P, ct.c_double]),
            "ppd_get_prior_weights": (I, [P, D, I64]),
            "ppd_set_active_sets": (I, [P, I32, ct.POINTER(ct.c_uint8), ct.POINTER(ct.c_uint8)]),
            "ppd_op_forward": (I, [P, P, P, P]),
            "ppd_op_adjoint": (I, [P, P, P, P]),
            "ppd_op_adjoint_noalloc": (I, [P, P, P, P]),
            "ppd_psi_analysis": (I, [P, P, P, P]),
            "ppd_psi_synthesis": (I, [P, P, P, P]),
            "ppd_timing_enable": (I, [P, I32]),
            "ppd_timing_collect": (I, [P]),
            "ppd_timing_read": (I, [P, I32, ct.POINTER(ct.c_char_p), D, ct.POINTER(ct.c_int64),
                                    ct.POINTER(ct.c_int32)]),
            "ppd_launch_count": (I64, [P]),
            "ppd_set_wait_limit": (I, [P, I64]),
            "ppd_status_string": (ct.c_char_p, [I]),
            "ppd_last_error": (ct.c_char_p, []),
        }
        for name, (res, args) in sig.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _LIB = L
    return _LIB


def _check(status: int, where: str):
    if status != PPD_OK:
        raise PPDError(status, where)


# cudaStreamLegacy: the handle CUDA uses for the legacy default stream
_STREAM_LEGACY = 1


def _stream(s):
    """None -> NULL (the context's own stream); 0 (PyTorch's default stream) -> cudaStreamLegacy."""
    if s is None:
        return None
    return _STREAM_LEGACY if int(s) == 0 else int(s)


def _dptr(a: np.ndarray):
    return a.ctypes.data_as(ct.POINTER(ct.c_double)) if a is not None else None


# --------------------------------------------------------------- entry points
def ppd_config_default(**overrides) -> ppd_config:
    cfg = ppd_config()
    _lib().ppd_config_default(ct.byref(cfg))
    for k, v in overrides.items():
        setattr(cfg, "lambda_" if k == "lambda" else k, v)
    return cfg


def ppd_create(cfg: ppd_config) -> int:
    h = ct.c_void_p()
    _check(_lib().ppd_create(ct.byref(h), ct.byref(cfg)), "ppd_create")
    return h.value


def ppd_destroy(ctx: int) -> None:
    _lib().ppd_destroy(ctx)


def ppd_set_visibilities(ctx: int, omega: np.ndarray, y: np.ndarray, block: np.ndarray) -> None:
    om = np.ascontiguousarray(omega, dtype=np.float64)
    yy = np.ascontiguousarray(np.stack([np.real(y), np.imag(y)], axis=1), dtype=np.float64)
    bb = np.ascontiguousarray(block, dtype=np.int32)
    _check(_lib().ppd_set_visibilities(ctx, om.shape[0], _dptr(om), _dptr(yy),
                                       bb.ctypes.data_as(ct.POINTER(ct.c_int32))),
           "ppd_set_visibilities")


def ppd_set_weights(ctx: int, theta=None, U=None, eps=None) -> None:
    th = None if theta is None else np.ascontiguousarray(theta, dtype=np.float64)
    uu = None if U is None else np.ascontiguousarray(U, dtype=np.float64)
    ep = None if eps is None else np.ascontiguousarray(eps, dtype=np.float64)
    _check(_lib().ppd_set_weights(ctx, _dptr(th), _dptr(uu), _dptr(ep)), "ppd_set_weights")


def ppd_set_ground_truth(ctx: int, x_true) -> None:
    if x_true is None:
        _check(_lib().ppd_set_ground_truth(ctx, None, 0), "ppd_set_ground_truth")
        return
    xt = np.ascontiguousarray(x_true, dtype=np.float64).ravel()
    _check(_lib().ppd_set_ground_truth(ctx, _dptr(xt), xt.size), "ppd_set_ground_truth")


def ppd_iterate(ctx: int, n_iters: int, n_blocks: int | None = None, stats: bool = True):
    if not stats:
        _check(_lib().ppd_iterate(ctx, n_iters, None), "ppd_iterate")
        return None
    st = ppd_stats()
    res = steps = None
    if n_blocks:
        res = np.zeros(n_blocks)
        steps = np.zeros(n_blocks, np.int32)
        st.block_residual = _dptr(res)
        st.inner_steps = steps.ctypes.data_as(ct.POINTER(ct.c_int32))
    _check(_lib().ppd_iterate(ctx, n_iters, ct.byref(st)), "ppd_iterate")
    return dict(iters_done=st.iters_done, rel_var=st.rel_var, snr_db=st.snr_db,
                max_res_over_eps=st.max_res_over_eps, block_residual=res, inner_steps=steps,
                stopped=bool(st.stopped), iters_run=st.iters_run)


def ppd_get_image(ctx: int, n0: int, n1: int) -> np.ndarray:
    x = np.empty(n0 * n1)
    _check(_lib().ppd_get_image(ctx, _dptr(x), x.size), "ppd_get_image")
    return x.reshape(n0, n1)


def ppd_get_params(ctx: int) -> dict:
    p = ppd_params()
    _check(_lib().ppd_get_params(ctx, ct.byref(p)), "ppd_get_params")
    return {f: getattr(p, f) for f, _ in ppd_params._fields_}


def ppd_get_bins(ctx: int, M: int):
    perm = np.empty(M, np.int64)
    b0 = np.empty(M, np.int32)
    b1 = np.empty(M, np.int32)
    cnt = np.empty(M, np.int32)
    _check(_lib().ppd_get_bins(ctx, perm.ctypes.data_as(ct.POINTER(ct.c_int64)),
                               b0.ctypes.data_as(ct.POINTER(ct.c_int32)),
                               b1.ctypes.data_as(ct.POINTER(ct.c_int32)),
                               cnt.ctypes.data_as(ct.POINTER(ct.c_int32))), "ppd_get_bins")
    return perm, b0, b1, cnt


def ppd_autotune(ctx: int, iters: int = 10):
    t = ct.c_int32(0)
    c = ct.c_int32(0)
    _check(_lib().ppd_autotune(ctx, iters, ct.byref(t), ct.byref(c)), "ppd_autotune")
    return int(t.value), int(c.value)


def ppd_group_create(ctxs) -> int:
    arr = (ct.c_void_p * len(ctxs))(*ctxs)
    h = ct.c_void_p()
    _check(_lib().ppd_group_create(ct.byref(h), arr, len(ctxs)), "ppd_group_create")
    return h.value


def ppd_group_iterate(group: int, n_iters: int) -> None:
    _check(_lib().ppd_group_iterate(group, n_iters), "ppd_group_iterate")


def ppd_group_destroy(group: int) -> None:
    _lib().ppd_group_destroy(group)


def ppd_get_state(ctx: int) -> bytes:
    n = ct.c_int64(0)
    _check(_lib().ppd_get_state(ctx, None, ct.byref(n)), "ppd_get_state")
    buf = ct.create_string_buffer(n.value)
    _check(_lib().ppd_get_state(ctx, ct.cast(buf, ct.c_void_p), ct.byref(n)), "ppd_get_state")
    return buf.raw[: n.value]


def ppd_set_state(ctx: int, blob: bytes) -> None:
    buf = ct.create_string_buffer(blob, len(blob))
    _check(_lib().ppd_set_state(ctx, ct.cast(buf, ct.c_void_p), len(blob)), "ppd_set_state")


def ppd_set_prior_weights(ctx: int, w) -> None:
    """W of the re-weighted scheme (9 x n0 x n1, basis-major), or None for W = I."""
    if w is None:
        _check(_lib().ppd_set_prior_weights(ctx, None, 0), "ppd_set_prior_weights")
        return
    a = np.ascontiguousarray(w, dtype=np.float64).reshape(-1)
    _check(_lib().ppd_set_prior_weights(ctx, _dptr(a), a.size), "ppd_set_prior_weights")


def ppd_reweight(ctx: int, omega: float) -> None:
    _check(_lib().ppd_reweight(ctx, float(omega)), "ppd_reweight")


def ppd_get_prior_weights(ctx: int, n0: int, n1: int) -> np.ndarray:
    out = np.empty(9 * n0 * n1)
    _check(_lib().ppd_get_prior_weights(ctx, _dptr(out), out.size), "ppd_get_prior_weights")
    return out.reshape(9, n0, n1)


def ppd_set_active_sets(ctx: int, blocks=None, bases=None, n_iters: int | None = None) -> None:
    """Queue the sets D (n_iters x n_blocks) and P (n_iters x 9) of the next
    iterations; None = full sets; n_iters = 0 returns to the plain iteration."""
    b = None if blocks is None else np.ascontiguousarray(blocks, dtype=np.uint8)
    p = None if bases is None else np.ascontiguousarray(bases, dtype=np.uint8)
    if n_iters is None:
        n_iters = b.shape[0] if b is not None else (p.shape[0] if p is not None else 0)
    u8 = ct.POINTER(ct.c_uint8)
    _check(_lib().ppd_set_active_sets(ctx, int(n_iters), None if b is None else b.ctypes.data_as(u8),
                                      None if p is None else p.ctypes.data_as(u8)), "ppd_set_active_sets")


def ppd_op_forward(ctx: int, x_dev: int, y_dev: int, stream=None) -> None:
    _check(_lib().ppd_op_forward(ctx, x_dev, y_dev, _stream(stream)), "ppd_op_forward")


def ppd_op_adjoint(ctx: int, y_dev: int, x_dev: int, stream=None) -> None:
    _check(_lib().ppd_op_adjoint(ctx, y_dev, x_dev, _stream(stream)), "ppd_op_adjoint")


def ppd_op_adjoint_noalloc(ctx: int, y_dev: int, x_dev: int, stream=None) -> None:
    _check(_lib().ppd_op_adjoint_noalloc(ctx, y_dev, x_dev, _stream(stream)), "ppd_op_adjoint_noalloc")


def ppd_psi_analysis(ctx: int, x_dev: int, c_dev: int, stream=None) -> None:
    _check(_lib().ppd_psi_analysis(ctx, x_dev, c_dev, _stream(stream)), "ppd_psi_analysis")


def ppd_psi_synthesis(ctx: int, c_dev: int, x_dev: int, stream=None) -> None:
    _check(_lib().ppd_psi_synthesis(ctx, c_dev, x_dev, _stream(stream)), "ppd_psi_synthesis")


def ppd_timing_enable(ctx: int, enable: bool) -> None:
    _check(_lib().ppd_timing_enable(ctx, 1 if enable else 0), "ppd_timing_enable")


def ppd_timing_collect(ctx: int) -> None:
    _check(_lib().ppd_timing_collect(ctx), "ppd_timing_collect")


def ppd_timing_read(ctx: int) -> dict:
    n = ct.c_int32(0)
    _check(_lib().ppd_timing_read(ctx, 0, None, None, None, ct.byref(n)), "ppd_timing_read")
    k = n.value
    names = (ct.c_char_p * max(k, 1))()
    ms = np.zeros(max(k, 1))
    cnt = np.zeros(max(k, 1), np.int64)
    _check(_lib().ppd_timing_read(ctx, k, names, _dptr(ms), cnt.ctypes.data_as(ct.POINTER(ct.c_int64)),
                                  ct.byref(n)), "ppd_timing_read")
    return {names[i].decode(): (float(ms[i]), int(cnt[i])) for i in range(k)}


PPD_WAIT_LIMIT_DEFAULT = 1 << 21


def ppd_set_wait_limit(ctx: int, polls: int) -> None:
    _check(_lib().ppd_set_wait_limit(ctx, int(polls)), "ppd_set_wait_limit")


def ppd_launch_count(ctx: int) -> int:
    return int(_lib().ppd_launch_count(ctx))


def ppd_status_string(status: int) -> str:
    return _lib().ppd_status_string(status).decode()


def ppd_last_error() -> str:
    return _lib().ppd_last_error().decode()


# --------------------------------------------------------------- convenience
class Solver:
    """One library context for one imaging problem (owns the handle): an
    L x L1 image (L1 = L by default)."""

    def __init__(self, L: int, n_blocks: int = 1, precision: int = PPD_FP32_FP64NORMS, L1: int | None = None,
                 **cfg):
        self.L = L
        self.L1 = L if L1 is None else L1
        self.n_blocks = n_blocks
        if "stream" in cfg:
            cfg["stream"] = _stream(cfg["stream"])
        self.cfg = ppd_config_default(n0=L, n1=self.L1, n_blocks=n_blocks, precision=precision, **cfg)
        self.ctx = ppd_create(self.cfg)
        self.M = 0

    def set_problem(self, omega, y, block, theta=None, U=None, eps=None, x_true=None):
        ppd_set_visibilities(self.ctx, omega, y, block)
        self.M = int(np.asarray(omega).shape[0])
        ppd_set_weights(self.ctx, theta, U, eps)
        if x_true is not None:
            ppd_set_ground_truth(self.ctx, x_true)
        return self

    def iterate(self, n: int, stats: bool = True):
        return ppd_iterate(self.ctx, n, self.n_blocks, stats)

    def image(self) -> np.ndarray:
        return ppd_get_image(self.ctx, self.L, self.L1)

    def reweighted(self, n_reweights: int, iters: int, omega0: float = 1e-2, factor: float = 0.25,
                   stats_every: int = 0):
        """Algorithm 1: n_reweights + 1 warm-started PPD runs of `iters` iterations,
        re-weighting with omega^(k) = factor^k omega0 between consecutive runs."""
        hist = []
        for k in range(n_reweights + 1):
            if k > 0:
                ppd_reweight(self.ctx, omega0 * factor ** k)
            if stats_every > 0:
                for _ in range(iters // stats_every):
                    hist.append(self.iterate(stats_every))
                if iters % stats_every:
                    hist.append(self.iterate(iters % stats_every))
            else:
                self.iterate(iters, stats=False)
        return hist

    def params(self) -> dict:
        return ppd_get_params(self.ctx)

    def close(self):
        if self.ctx:
            ppd_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
