"""Python binding of libqdtrace (C ABI in include/qdtrace.h).

Argument marshalling only: every computation runs in the library's CUDA
kernels.  PyTorch supplies device memory and the stream.  Importing this
module loads ``libqdtrace.so`` from the package directory and raises
:class:`QDError` if it is missing (build it with
``python -m paper_1909_12234_gb300.build``); there is no fallback.

Device fields are ``torch.complex128`` CUDA tensors in the library's "qd
layout": fine level shape ``(V, 12, nrhs)`` with sites in even-odd order,
coarse level ``(Vc, dc, nrhs)`` with lexicographic coarse sites.
"""

import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libqdtrace.so")

QD_OK = 0
QD_ERR_INVALID = -1
QD_ERR_CUDA = -2
QD_ERR_OOM = -3
QD_ERR_NOT_CONVERGED = -4
QD_ERR_NONFINITE = -5
QD_ERR_TIMEOUT = -6
QD_ERR_INTERNAL = -7
QD_MAX_LEVELS = 4
QD_DEFL_EIG_ORTHO = 1
QD_DEFL_MG_OBLIQUE = 2
QD_PREC_F64 = 0
QD_PREC_MIXED = 1

_STATUS = {0: "QD_OK", -1: "QD_ERR_INVALID", -2: "QD_ERR_CUDA", -3: "QD_ERR_OOM",
           -4: "QD_ERR_NOT_CONVERGED", -5: "QD_ERR_NONFINITE", -6: "QD_ERR_TIMEOUT",
           -7: "QD_ERR_INTERNAL"}


class QDError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"{_STATUS.get(code, code)}: {msg}")
        self.code = code


class MGParams(ctypes.Structure):
    _fields_ = [("nlevels", ctypes.c_int),
                ("block", (ctypes.c_int * 4) * QD_MAX_LEVELS),
                ("nv", ctypes.c_int * QD_MAX_LEVELS),
                ("null_tol", ctypes.c_double),
                ("null_maxit", ctypes.c_int),
                ("seed", ctypes.c_uint64),
                ("smoother_steps", ctypes.c_int),
                ("coarse_tol", ctypes.c_double),
                ("coarse_maxit", ctypes.c_int),
                ("coarse_restart", ctypes.c_int),
                ("coarsest_direct", ctypes.c_int),
                ("coarsest_bf16", ctypes.c_int),
                ("use_graphs", ctypes.c_int),
                ("coarse_tc", ctypes.c_int),
                ("coarse_smoother_steps", ctypes.c_int),
                ("null_f32", ctypes.c_int)]


class SolverParams(ctypes.Structure):
    _fields_ = [("tol", ctypes.c_double),
                ("maxit", ctypes.c_int),
                ("restart", ctypes.c_int),
                ("precision", ctypes.c_int),
                ("inner_tol", ctypes.c_double),
                ("max_refine", ctypes.c_int),
                ("stag_window", ctypes.c_int),
                ("schur", ctypes.c_int)]


class SolveStats(ctypes.Structure):
    _fields_ = [("iterations", ctypes.c_int),
                ("converged", ctypes.c_int),
                ("max_true_rel_residual", ctypes.c_double),
                ("iters_per_rhs", ctypes.POINTER(ctypes.c_int)),
                ("true_rel_residual", ctypes.POINTER(ctypes.c_double)),
                ("stagnated", ctypes.c_int)]


class DeflParams(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int),
                ("k", ctypes.c_int),
                ("guard", ctypes.c_int),
                ("eig_tol", ctypes.c_double),
                ("solve_tol", ctypes.c_double),
                ("maxit", ctypes.c_int),
                ("seed", ctypes.c_uint64),
                ("tau_restart", ctypes.c_double),
                ("max_restarts", ctypes.c_int),
                ("stag_window", ctypes.c_int),
                ("solve_restart", ctypes.c_int),
                ("fail_first", ctypes.c_int)]


class TraceParams(ctypes.Structure):
    _fields_ = [("seed", ctypes.c_uint64),
                ("sample_offset", ctypes.c_int64),
                ("nsamples", ctypes.c_int),
                ("solver", SolverParams),
                ("dilution", ctypes.c_int)]


class TraceResult(ctypes.Structure):
    _fields_ = [("t0", ctypes.c_double * 2),
                ("mean", ctypes.c_double * 2),
                ("estimate", ctypes.c_double * 2),
                ("var", ctypes.c_double),
                ("var_re", ctypes.c_double),
                ("stderr_mean", ctypes.c_double),
                ("var_jackknife_err", ctypes.c_double),
                ("nsamples", ctypes.c_int),
                ("iterations", ctypes.c_int),
                ("max_true_rel_residual", ctypes.c_double),
                ("t_samples", ctypes.POINTER(ctypes.c_double)),
                ("ZhV", ctypes.POINTER(ctypes.c_double)),
                ("UhKZ", ctypes.POINTER(ctypes.c_double))]


class SmootherParams(ctypes.Structure):
    _fields_ = [("nsamples", ctypes.c_int), ("solve_tol", ctypes.c_double), ("seed", ctypes.c_uint64),
                ("mr_steps", ctypes.c_int), ("layers", ctypes.c_int)]


class SmootherInfo(ctypes.Structure):
    _fields_ = [("err_learned", ctypes.c_double), ("err_plain", ctypes.c_double), ("enabled", ctypes.c_int)]


class BatchItem(ctypes.Structure):
    _fields_ = [("gauge", ctypes.c_void_p), ("mg", ctypes.c_void_p), ("defl", ctypes.c_void_p),
                ("m0", ctypes.c_double), ("tau", ctypes.c_double), ("params", TraceParams),
                ("result", ctypes.POINTER(TraceResult)), ("status", ctypes.c_int)]


_P = ctypes.c_void_p
_I = ctypes.c_int
_D = ctypes.c_double
_PP = ctypes.POINTER(ctypes.c_void_p)
_IPTR = ctypes.POINTER(ctypes.c_int)
_DPTR = ctypes.POINTER(ctypes.c_double)
_I64PTR = ctypes.POINTER(ctypes.c_int64)

# name -> (restype, argtypes); the ABI's exported symbols
SIGNATURES = {
    "qd_abi_version": (_I, []),
    "qd_last_error": (ctypes.c_char_p, []),
    "qd_ctx_create": (_I, [_PP, _I, _P]),
    "qd_ctx_destroy": (_I, [_P]),
    "qd_eo_index": (_I, [_IPTR, _I64PTR]),
    "qd_gauge_create": (_I, [_P, _IPTR, _P, _PP]),
    "qd_gauge_destroy": (_I, [_P]),
    "qd_field_reorder": (_I, [_P, _P, _I, _I, _P, _P]),
    "qd_rademacher": (_I, [_P, _P, ctypes.c_uint64, ctypes.c_int64, _I, _P]),
    "qd_dirac_apply": (_I, [_P, _P, _D, _D, _I, _I, _P, _P]),
    "qd_dirac_apply_f32": (_I, [_P, _P, _D, _D, _I, _I, _P, _P]),
    "qd_dirac_residual_f32": (_I, [_P, _P, _D, _D, _I, _I, _P, _P, _P]),
    "qd_dirac_schur_apply": (_I, [_P, _P, _D, _D, _I, _P, _P]),
    "qd_dirac_schur_apply_f32": (_I, [_P, _P, _D, _D, _I, _P, _P]),
    "qd_mg_params_default": (None, [ctypes.POINTER(MGParams)]),
    "qd_mg_setup": (_I, [_P, _P, _D, _D, ctypes.POINTER(MGParams), _P, _PP]),
    "qd_mg_destroy": (_I, [_P]),
    "qd_mg_level_info": (_I, [_P, _I, _IPTR, _IPTR, _I64PTR, _IPTR]),
    "qd_prolongate": (_I, [_P, _I, _I, _P, _P]),
    "qd_restrict": (_I, [_P, _I, _I, _P, _P]),
    "qd_coarse_apply": (_I, [_P, _I, _I, _P, _P]),
    "qd_coarse_apply_f32": (_I, [_P, _I, _I, _P, _P]),
    "qd_coarse_apply_tc": (_I, [_P, _I, _I, _P, _P]),
    "qd_restrict_tc": (_I, [_P, _I, _I, _P, _P]),
    "qd_prolongate_f32": (_I, [_P, _I, _I, _P, _P]),
    "qd_coarse_residual_tc": (_I, [_P, _I, _I, _P, _P, _P]),
    "qd_coarse_solve": (_I, [_P, _I, _I, _P, _P]),
    "qd_coarse_solve_f32": (_I, [_P, _I, _I, _P, _P]),
    "qd_solver_params_default": (None, [ctypes.POINTER(SolverParams)]),
    "qd_solve": (_I, [_P, _P, _P, _D, _D, _I, _P, _P, ctypes.POINTER(SolverParams), ctypes.POINTER(SolveStats)]),
    "qd_defl_params_default": (None, [ctypes.POINTER(DeflParams)]),
    "qd_defl_create": (_I, [_P, _P, _P, _D, _D, ctypes.POINTER(DeflParams), _P, _PP]),
    "qd_defl_destroy": (_I, [_P]),
    "qd_defl_set_rank": (_I, [_P, _I, _DPTR]),
    "qd_defl_info": (_I, [_P, _DPTR, _DPTR, _IPTR]),
    "qd_defl_shift_info": (_I, [_P, _DPTR, _IPTR]),
    "qd_defl_gram": (_I, [_P, _DPTR]),
    "qd_defl_basis": (_I, [_P, _P]),
    "qd_deflate_project": (_I, [_P, _I, _P, _P]),
    "qd_deflate_project_static": (_I, [_P, _I, _P, _P]),
    "qd_deflate_coeffs": (_I, [_P, _I, _P, _DPTR, _DPTR]),
    "qd_smoother_params_default": (None, [ctypes.POINTER(SmootherParams)]),
    "qd_smoother_train": (_I, [_P, ctypes.POINTER(SmootherParams), ctypes.POINTER(SmootherInfo)]),
    "qd_smoother_fit": (_I, [_P, _I, _P, _P]),
    "qd_smoother_set_weights": (_I, [_P, _DPTR]),
    "qd_smoother_get_weights": (_I, [_P, _DPTR]),
    "qd_smoother_set_layer_weights": (_I, [_P, _I, _DPTR]),
    "qd_smoother_layers": (_I, [_P]),
    "qd_smoother_get_layer_weights": (_I, [_P, _DPTR]),
    "qd_smoother_enable": (_I, [_P, _I, _I]),
    "qd_smoother_apply": (_I, [_P, _I, _P, _P]),
    "qd_smoother_apply_f32": (_I, [_P, _I, _P, _P]),
    "qd_autotune_set": (None, [_I]),
    "qd_autotune_clear": (None, []),
    "qd_autotune_force": (None, [_I]),
    "qd_autotune_report": (_I, [ctypes.c_char_p, _I]),
    "qd_hutchinson_batch": (_I, [_P, _I, ctypes.POINTER(BatchItem), _I]),
    "qd_mg_subspace_sines": (_I, [_P, _I, _I, _P, _DPTR]),
    "qd_hutchinson_trace": (_I, [_P, _P, _P, _P, _D, _D, ctypes.POINTER(TraceParams),
                                 ctypes.POINTER(TraceResult)]),
    "qd_trace_stats": (_I, [_P, _I, _P, _DPTR, ctypes.POINTER(TraceResult)]),
    "qd_launch_count": (ctypes.c_longlong, []),
    "qd_alloc_count": (ctypes.c_longlong, []),
    "qd_prof_enable": (_I, [_P, _I]),
    "qd_prof_read": (_I, [_P, _I, _I64PTR, _DPTR, _DPTR, _DPTR, _I]),
}

PROF_KINDS = {"wilson_f64": 0, "wilson_f32": 1, "coarse_f64": 2, "coarse_f32": 3, "prolong_f64": 4,
              "prolong_f32": 5, "restrict_f64": 6, "restrict_f32": 7, "direct_f64": 8, "direct_f32": 9, "direct_bf16": 10,
              "blas_f64": 11, "dots_f32": 12, "axpy_f32": 13, "update_f32": 14, "smoother_f64": 15,
              "smoother_f32": 16, "coarse_tc": 17, "restrict_tc": 18}

_lib = None


def load(path=LIB_PATH):
    """Load libqdtrace.so (once) and declare every entry point."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise QDError(QD_ERR_INTERNAL, f"{path} not found: build it with "
                      "`python -m paper_1909_12234_gb300.build` (no CPU fallback exists)")
    lib = ctypes.CDLL(path)
    for name, (res, args) in SIGNATURES.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


def _check(rc, allow=()):
    if rc != QD_OK and rc not in allow:
        raise QDError(rc, load().qd_last_error().decode())
    return rc


def _ptr(t):
    """Device pointer of a contiguous complex128 CUDA tensor."""
    import torch
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise QDError(QD_ERR_INVALID, "expected a CUDA tensor")
    if t.dtype != torch.complex128 or not t.is_contiguous():
        raise QDError(QD_ERR_INVALID, "expected a contiguous torch.complex128 tensor")
    return ctypes.c_void_p(t.data_ptr())


def _dims(dims):
    return (ctypes.c_int * 4)(*[int(d) for d in dims])


def eo_index(dims):
    """eo_index(dims)[lex] from the library (host-side index arithmetic)."""
    V = int(np.prod(dims))
    out = np.empty(V, dtype=np.int64)
    _check(load().qd_eo_index(_dims(dims), out.ctypes.data_as(_I64PTR)))
    return out


class Context:
    """qd_ctx on one device, issuing work on a torch CUDA stream."""

    def __init__(self, device=0, stream=None):
        import torch
        self.device = int(device)
        self.stream = stream if stream is not None else torch.cuda.current_stream(self.device)
        h = ctypes.c_void_p()
        _check(load().qd_ctx_create(ctypes.byref(h), self.device, ctypes.c_void_p(self.stream.cuda_stream)))
        self.h = h

    def close(self):
        if getattr(self, "h", None):
            load().qd_ctx_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Gauge:
    """qd_gauge: links (4, V, 3, 3) complex128 numpy array (U[mu, lex])."""

    def __init__(self, ctx, dims, links):
        self.ctx = ctx
        self.dims = tuple(int(d) for d in dims)
        self.V = int(np.prod(self.dims))
        canon = np.ascontiguousarray(np.transpose(np.asarray(links, dtype=np.complex128), (1, 0, 2, 3)))
        if canon.shape != (self.V, 4, 3, 3):
            raise QDError(QD_ERR_INVALID, "links must have shape (4, V, 3, 3)")
        h = ctypes.c_void_p()
        _check(load().qd_gauge_create(ctx.h, _dims(self.dims), canon.ctypes.data_as(ctypes.c_void_p),
                                      ctypes.byref(h)))
        self.h = h

    @classmethod
    def from_host_buffer(cls, ctx, dims, host_tensor):
        """Links already in the C ABI's host order [V][4][3][3] complex, given
        as a contiguous (pinned) CPU torch tensor of float64 or complex128."""
        self = cls.__new__(cls)
        self.ctx = ctx
        self.dims = tuple(int(d) for d in dims)
        self.V = int(np.prod(self.dims))
        if host_tensor.is_cuda or not host_tensor.is_contiguous() or host_tensor.numel() * host_tensor.element_size() != self.V * 4 * 9 * 16:
            raise QDError(QD_ERR_INVALID, "host link buffer must be contiguous CPU memory of V*36 complex numbers")
        h = ctypes.c_void_p()
        _check(load().qd_gauge_create(ctx.h, _dims(self.dims), ctypes.c_void_p(host_tensor.data_ptr()),
                                      ctypes.byref(h)))
        self.h = h
        return self

    def close(self):
        if getattr(self, "h", None):
            load().qd_gauge_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def field_reorder(ctx, gauge, nrhs, to_qd, inp, out):
    _check(load().qd_field_reorder(ctx.h, gauge.h, int(nrhs), 1 if to_qd else 0, _ptr(inp), _ptr(out)))


def to_qd(ctx, gauge, x):
    """Host field (V, 4, 3, s) numpy, lexicographic -> device qd layout (V, 12, s)."""
    import torch
    x = np.asarray(x, dtype=np.complex128)
    s = x.shape[3]
    canon = torch.from_numpy(np.ascontiguousarray(np.transpose(x.reshape(gauge.V, 12, s), (2, 0, 1))))
    canon = canon.to(f"cuda:{ctx.device}")
    out = torch.empty((gauge.V, 12, s), dtype=torch.complex128, device=f"cuda:{ctx.device}")
    field_reorder(ctx, gauge, s, True, canon, out)
    return out


def from_qd(ctx, gauge, y):
    """Device qd-layout field (V, 12, s) -> host (V, 4, 3, s) numpy, lexicographic."""
    import torch
    s = y.shape[2]
    canon = torch.empty((s, gauge.V, 12), dtype=torch.complex128, device=y.device)
    field_reorder(ctx, gauge, s, False, y, canon)
    torch.cuda.synchronize(y.device)
    return np.transpose(canon.cpu().numpy(), (1, 2, 0)).reshape(gauge.V, 4, 3, s)


def rademacher(ctx, gauge, seed, sample_offset, nrhs, out):
    _check(load().qd_rademacher(ctx.h, gauge.h, int(seed), int(sample_offset), int(nrhs), _ptr(out)))


def dirac_apply(ctx, gauge, m0, tau, dagger, nrhs, inp, out):
    _check(load().qd_dirac_apply(ctx.h, gauge.h, float(m0), float(tau), 1 if dagger else 0, int(nrhs),
                                 _ptr(inp), _ptr(out)))


def dirac_apply_f32(ctx, gauge, m0, tau, dagger, nrhs, inp, out):
    """FP32 operator on torch.complex64 fields in qd layout."""
    _check(load().qd_dirac_apply_f32(ctx.h, gauge.h, float(m0), float(tau), 1 if dagger else 0, int(nrhs),
                                     _ptr64(inp), _ptr64(out)))


def dirac_residual_f32(ctx, gauge, m0, tau, dagger, nrhs, b, x, r):
    """r = b - A x (A^H with dagger) in FP32, torch.complex64 fields in qd layout."""
    _check(load().qd_dirac_residual_f32(ctx.h, gauge.h, float(m0), float(tau), 1 if dagger else 0, int(nrhs),
                                        _ptr64(b), _ptr64(x), _ptr64(r)))


def dirac_schur_apply(ctx, gauge, m0, tau, nrhs, inp, out):
    """Odd-site Schur complement S on half fields (odd half of the qd layout), FP64."""
    _check(load().qd_dirac_schur_apply(ctx.h, gauge.h, float(m0), float(tau), int(nrhs), _ptr(inp), _ptr(out)))


def dirac_schur_apply_f32(ctx, gauge, m0, tau, nrhs, inp, out):
    """The same in FP32 (torch.complex64)."""
    _check(load().qd_dirac_schur_apply_f32(ctx.h, gauge.h, float(m0), float(tau), int(nrhs), _ptr64(inp),
                                           _ptr64(out)))


def mg_params(nlevels=1, blocks=((2, 2, 2, 2),), nvs=(12,), **kw):
    p = MGParams()
    load().qd_mg_params_default(ctypes.byref(p))
    p.nlevels = int(nlevels)
    for l in range(nlevels):
        for m in range(4):
            p.block[l][m] = int(blocks[l][m])
        p.nv[l] = int(nvs[l])
    for k, v in kw.items():
        setattr(p, k, v)
    return p


class Multigrid:
    """qd_mg handle (adaptive setup)."""

    def __init__(self, ctx, gauge, m0, tau, params, injected_null=None):
        self.ctx, self.gauge, self.m0, self.tau = ctx, gauge, float(m0), float(tau)
        self.params = params
        h = ctypes.c_void_p()
        inj = _ptr(injected_null) if injected_null is not None else None
        _check(load().qd_mg_setup(ctx.h, gauge.h, self.m0, self.tau, ctypes.byref(params), inj, ctypes.byref(h)))
        self.h = h

    def level_info(self, level):
        dims = (ctypes.c_int * 4)()
        dof = ctypes.c_int()
        ns = ctypes.c_int64()
        nv = self.params.nv[level] if level < self.params.nlevels else 0
        steps = (ctypes.c_int * max(nv, 1))()
        _check(load().qd_mg_level_info(self.h, int(level), dims, ctypes.byref(dof), ctypes.byref(ns), steps))
        return tuple(dims), dof.value, ns.value, list(steps)[:nv]

    def close(self):
        if getattr(self, "h", None):
            load().qd_mg_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def prolongate(mg, level, nrhs, coarse, fine):
    _check(load().qd_prolongate(mg.h, int(level), int(nrhs), _ptr(coarse), _ptr(fine)))


def restrict(mg, level, nrhs, fine, coarse):
    _check(load().qd_restrict(mg.h, int(level), int(nrhs), _ptr(fine), _ptr(coarse)))


def mg_subspace_sines(mg, depth, V):
    """sin of the angle between each column of V (fine qd layout, complex128
    CUDA tensor (V, 12, k)) and the range of W_0 ... W_{depth-1}."""
    k = int(V.shape[-1])
    out = np.zeros(k)
    _check(load().qd_mg_subspace_sines(mg.h, int(depth), k, _ptr(V), out.ctypes.data_as(_DPTR)))
    return out


def coarse_apply(mg, level, nrhs, inp, out):
    _check(load().qd_coarse_apply(mg.h, int(level), int(nrhs), _ptr(inp), _ptr(out)))


def coarse_solve(mg, level, nrhs, inp, out):
    _check(load().qd_coarse_solve(mg.h, int(level), int(nrhs), _ptr(inp), _ptr(out)))


def _ptr64(t):
    """Device pointer of a contiguous complex64 CUDA tensor."""
    import torch
    if not isinstance(t, torch.Tensor) or not t.is_cuda or t.dtype != torch.complex64 or not t.is_contiguous():
        raise QDError(QD_ERR_INVALID, "expected a contiguous torch.complex64 CUDA tensor")
    return ctypes.c_void_p(t.data_ptr())


def coarse_apply_f32(mg, level, nrhs, inp, out):
    _check(load().qd_coarse_apply_f32(mg.h, int(level), int(nrhs), _ptr64(inp), _ptr64(out)))


def coarse_apply_tc(mg, level, nrhs, inp, out):
    _check(load().qd_coarse_apply_tc(mg.h, int(level), int(nrhs), _ptr64(inp), _ptr64(out)))


def coarse_residual_tc(mg, level, nrhs, b, x, r):
    _check(load().qd_coarse_residual_tc(mg.h, int(level), int(nrhs), _ptr64(b), _ptr64(x), _ptr64(r)))


def prolongate_f32(mg, level, nrhs, coarse, fine):
    _check(load().qd_prolongate_f32(mg.h, int(level), int(nrhs), _ptr64(coarse), _ptr64(fine)))


def restrict_tc(mg, level, nrhs, fine, coarse):
    _check(load().qd_restrict_tc(mg.h, int(level), int(nrhs), _ptr64(fine), _ptr64(coarse)))


def coarse_solve_f32(mg, level, nrhs, inp, out):
    _check(load().qd_coarse_solve_f32(mg.h, int(level), int(nrhs), _ptr64(inp), _ptr64(out)))


def solver_params(tol=1e-8, maxit=500, restart=16, precision=QD_PREC_F64, **kw):
    p = SolverParams()
    load().qd_solver_params_default(ctypes.byref(p))
    p.tol, p.maxit, p.restart, p.precision = float(tol), int(maxit), int(restart), int(precision)
    for k, v in kw.items():
        setattr(p, k, v)
    return p


def solve(ctx, gauge, mg, m0, tau, nrhs, b, x, tol, maxit=10000, restart=16, allow_not_converged=False,
          precision=QD_PREC_F64, **kw):
    """Returns (status, iterations, per-column iterations, per-column true residual)."""
    it = (ctypes.c_int * nrhs)()
    rel = (ctypes.c_double * nrhs)()
    st = SolveStats(0, 0, 0.0, it, rel, 0)
    p = solver_params(tol, maxit, restart, precision, **kw)
    rc = load().qd_solve(ctx.h, gauge.h, mg.h if mg is not None else None, float(m0), float(tau), int(nrhs),
                         _ptr(b), _ptr(x), ctypes.byref(p), ctypes.byref(st))
    _check(rc, allow=(QD_ERR_NOT_CONVERGED,) if allow_not_converged else ())
    solve.last_stagnated = bool(st.stagnated)
    return rc, st.iterations, list(it), list(rel)


def defl_params(kind=QD_DEFL_MG_OBLIQUE, k=24, **kw):
    p = DeflParams()
    load().qd_defl_params_default(ctypes.byref(p))
    p.kind = int(kind)
    p.k = int(k)
    for key, v in kw.items():
        setattr(p, key, v)
    return p


class Deflation:
    """qd_defl handle (Algorithm 1 or 2 deflation space)."""

    def __init__(self, ctx, gauge, mg, m0, tau, params, injected_basis=None):
        self.ctx, self.gauge, self.mg, self.params = ctx, gauge, mg, params
        h = ctypes.c_void_p()
        inj = _ptr(injected_basis) if injected_basis is not None else None
        _check(load().qd_defl_create(ctx.h, gauge.h, mg.h if mg is not None else None, float(m0), float(tau),
                                     ctypes.byref(params), inj, ctypes.byref(h)))
        self.h = h
        self.rank = params.k

    def set_rank(self, r):
        t0 = (ctypes.c_double * 2)()
        _check(load().qd_defl_set_rank(self.h, int(r), t0))
        self.rank = int(r)
        return complex(t0[0], t0[1])

    def info(self):
        k = self.params.k
        mu = (ctypes.c_double * k)()
        lam = (ctypes.c_double * k)()
        its = ctypes.c_int()
        _check(load().qd_defl_info(self.h, mu, lam, ctypes.byref(its)))
        return np.array(mu[:]), np.array(lam[:self.rank]), its.value

    def shift_info(self):
        """(eigensolver shift tau_eig after its restarts, number of restarts)."""
        tau = ctypes.c_double()
        n = ctypes.c_int()
        _check(load().qd_defl_shift_info(self.h, ctypes.byref(tau), ctypes.byref(n)))
        return tau.value, n.value

    def gram(self):
        """Algorithm 2: G = U_bar^H gamma5^W C U_bar (k x k)."""
        k = self.params.k
        G = np.zeros((k, k, 2))
        _check(load().qd_defl_gram(self.h, G.ctypes.data_as(_DPTR)))
        return G[..., 0] + 1j * G[..., 1]

    def basis(self, out):
        """Copy the k basis vectors into the complex128 CUDA tensor `out`."""
        _check(load().qd_defl_basis(self.h, _ptr(out)))

    def project(self, nrhs, z, out):
        _check(load().qd_deflate_project(self.h, int(nrhs), _ptr(z), _ptr(out)))

    def project_static(self, nrhs, z, out):
        """out = (I - U U^H) z for an orthonormal-eigenvector space, with the
        library's fixed device scratch (no device allocation during the
        call); see qdtrace.h."""
        _check(load().qd_deflate_project_static(self.h, int(nrhs), _ptr(z), _ptr(out)))

    def coeffs(self, nrhs, z):
        k = self.params.k
        zhv = np.zeros((nrhs, k, 2))
        uhkz = np.zeros((k, nrhs, 2))
        _check(load().qd_deflate_coeffs(self.h, int(nrhs), _ptr(z), zhv.ctypes.data_as(_DPTR),
                                        uhkz.ctypes.data_as(_DPTR)))
        return zhv[..., 0] + 1j * zhv[..., 1], uhkz[..., 0] + 1j * uhkz[..., 1]

    def close(self):
        if getattr(self, "h", None):
            load().qd_defl_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def trace_stats(ctx, t, t0=0j):
    """Device statistics of per-sample values t (1-D complex array, any host
    or device origin) with deterministic compensated sums; returns a dict."""
    import torch
    tt = torch.as_tensor(np.asarray(t, dtype=np.complex128)).to(f"cuda:{ctx.device}")
    r = TraceResult()
    t0a = (ctypes.c_double * 2)(complex(t0).real, complex(t0).imag)
    _check(load().qd_trace_stats(ctx.h, int(tt.numel()), _ptr(tt), t0a, ctypes.byref(r)))
    return {"t0": complex(r.t0[0], r.t0[1]), "mean": complex(r.mean[0], r.mean[1]),
            "estimate": complex(r.estimate[0], r.estimate[1]), "var": r.var, "var_re": r.var_re,
            "stderr": r.stderr_mean, "var_jackknife_err": r.var_jackknife_err, "s": r.nsamples}


def launch_count():
    """Kernels launched by libqdtrace since it was loaded."""
    return int(load().qd_launch_count())


def alloc_count():
    """Device allocations (cudaMalloc) libqdtrace has made since it was loaded."""
    return int(load().qd_alloc_count())


def prof_enable(ctx, on):
    _check(load().qd_prof_enable(ctx.h, 1 if on else 0))


def prof_read(ctx, kind, reset=False):
    """Totals of one kernel kind: dict(launches, ms, flops, bytes)."""
    n = ctypes.c_int64()
    ms, fl, by = ctypes.c_double(), ctypes.c_double(), ctypes.c_double()
    k = PROF_KINDS[kind] if isinstance(kind, str) else int(kind)
    _check(load().qd_prof_read(ctx.h, k, ctypes.byref(n), ctypes.byref(ms), ctypes.byref(fl), ctypes.byref(by),
                               1 if reset else 0))
    return {"launches": n.value, "ms": ms.value, "flops": fl.value, "bytes": by.value}


class _TraceOut:
    """Host buffers of one qd_trace_result and their conversion to a dict."""

    def __init__(self, defl, nsamples, want_samples, want_coeffs):
        self.r = TraceResult()
        self.ts = np.zeros((nsamples, 2)) if want_samples else None
        k = defl.params.k if defl is not None else 0
        self.zhv = np.zeros((nsamples, k, 2)) if want_coeffs and k else None
        self.uhkz = np.zeros((k, nsamples, 2)) if want_coeffs and k else None
        self.r.t_samples = self.ts.ctypes.data_as(_DPTR) if self.ts is not None else None
        self.r.ZhV = self.zhv.ctypes.data_as(_DPTR) if self.zhv is not None else None
        self.r.UhKZ = self.uhkz.ctypes.data_as(_DPTR) if self.uhkz is not None else None

    def as_dict(self, rc):
        r = self.r
        out = {
            "status": rc,
            "t0": complex(r.t0[0], r.t0[1]),
            "mean": complex(r.mean[0], r.mean[1]),
            "estimate": complex(r.estimate[0], r.estimate[1]),
            "var": r.var, "var_re": r.var_re, "stderr": r.stderr_mean,
            "var_jackknife_err": r.var_jackknife_err, "iterations": r.iterations,
            "max_true_rel_residual": r.max_true_rel_residual, "s": r.nsamples,
        }
        if self.ts is not None:
            out["t"] = self.ts[:, 0] + 1j * self.ts[:, 1]
        if self.zhv is not None:
            out["ZhV"] = self.zhv[..., 0] + 1j * self.zhv[..., 1]
            out["UhKZ"] = self.uhkz[..., 0] + 1j * self.uhkz[..., 1]
        return out


def hutchinson_trace(ctx, gauge, mg, defl, m0, tau, seed, sample_offset, nsamples, tol, maxit=10000,
                     restart=16, want_samples=True, want_coeffs=False, allow_not_converged=False,
                     precision=QD_PREC_F64, dilution=0, **kw):
    """One multi-RHS batch of the deflated estimator; returns a dict.
    dilution=12: spin-colour dilution (12 solves per sample)."""
    p = TraceParams(int(seed), int(sample_offset), int(nsamples), solver_params(tol, maxit, restart, precision, **kw),
                    int(dilution))
    o = _TraceOut(defl, nsamples, want_samples, want_coeffs)
    rc = load().qd_hutchinson_trace(ctx.h, gauge.h, mg.h if mg is not None else None,
                                    defl.h if defl is not None else None, float(m0), float(tau),
                                    ctypes.byref(p), ctypes.byref(o.r))
    _check(rc, allow=(QD_ERR_NOT_CONVERGED,) if allow_not_converged else ())
    return o.as_dict(rc)


_BATCH_KEYS = ("gauge", "mg", "defl", "m0", "tau", "seed", "sample_offset", "nsamples", "tol", "maxit", "restart",
               "precision", "want_samples")


def hutchinson_batch(ctx, problems, nstreams=4, allow_not_converged=False):
    """Independent estimators solved concurrently (qd_hutchinson_batch).

    ``problems``: dicts with gauge, mg, defl, m0, tau, seed, sample_offset,
    nsamples, tol and optional maxit, restart, precision, want_samples and
    solver keywords.  Returns one result dict per problem, in order."""
    n = len(problems)
    items = (BatchItem * max(n, 1))()
    outs = []
    for i, pr in enumerate(problems):
        kw = {k: v for k, v in pr.items() if k not in _BATCH_KEYS}
        sp = solver_params(pr["tol"], pr.get("maxit", 10000), pr.get("restart", 16),
                           pr.get("precision", QD_PREC_F64), **kw)
        o = _TraceOut(pr.get("defl"), pr["nsamples"], pr.get("want_samples", True), False)
        outs.append(o)
        items[i].gauge = pr["gauge"].h.value
        items[i].mg = pr["mg"].h.value if pr.get("mg") is not None else None
        items[i].defl = pr["defl"].h.value if pr.get("defl") is not None else None
        items[i].m0 = float(pr["m0"])
        items[i].tau = float(pr.get("tau", 0.0))
        items[i].params = TraceParams(int(pr["seed"]), int(pr.get("sample_offset", 0)), int(pr["nsamples"]), sp)
        items[i].result = ctypes.pointer(o.r)
    rc = load().qd_hutchinson_batch(ctx.h, n, items, int(nstreams))
    _check(rc, allow=(QD_ERR_NOT_CONVERGED,) if allow_not_converged else ())
    return [outs[i].as_dict(items[i].status) for i in range(n)]


def autotune_set(mode):
    load().qd_autotune_set(int(mode))


def autotune_clear():
    load().qd_autotune_clear()


def autotune_force(candidate):
    """Candidate k of every tunable kernel where it applies; -1: normal."""
    load().qd_autotune_force(int(candidate))


def autotune_report():
    """{key: (choice, [ms per candidate])} of the launch-shape autotuner."""
    n = load().qd_autotune_report(None, 0)
    buf = ctypes.create_string_buffer(n)
    load().qd_autotune_report(buf, n)
    out = {}
    for line in buf.value.decode().splitlines():
        parts = line.split(" ")
        # key words, then the choice and the times
        nums = []
        while parts and _isnum(parts[-1]):
            nums.insert(0, parts.pop())
        out[" ".join(parts)] = (int(nums[0]), [float(x) for x in nums[1:]])
    return out


def _isnum(w):
    try:
        float(w)
        return True
    except ValueError:
        return False


def smoother_params(**kw):
    p = SmootherParams()
    load().qd_smoother_params_default(ctypes.byref(p))
    for k, v in kw.items():
        setattr(p, k, v)
    return p


def smoother_train(mg, **kw):
    """Train the learned smoother on solver-generated pairs; returns the
    held-out errors and whether the V-cycle now uses it."""
    info = SmootherInfo()
    _check(load().qd_smoother_train(mg.h, ctypes.byref(smoother_params(**kw)), ctypes.byref(info)))
    return {"err_learned": info.err_learned, "err_plain": info.err_plain, "enabled": bool(info.enabled)}


def smoother_fit(mg, nrhs, e, r):
    _check(load().qd_smoother_fit(mg.h, int(nrhs), _ptr(e), _ptr(r)))


def smoother_set_weights(mg, w):
    w = np.ascontiguousarray(np.asarray(w, dtype=np.complex128).reshape(9, 4, 4))
    _check(load().qd_smoother_set_weights(mg.h, w.view(np.float64).ctypes.data_as(_DPTR)))


def smoother_get_weights(mg):
    w = np.zeros((9, 4, 4), dtype=np.complex128)
    _check(load().qd_smoother_get_weights(mg.h, w.view(np.float64).ctypes.data_as(_DPTR)))
    return w


def smoother_set_layer_weights(mg, w):
    """w: (layers, 9, 4, 4) complex, the layer applied first to r first."""
    w = np.ascontiguousarray(np.asarray(w, dtype=np.complex128))
    layers = w.size // 144
    _check(load().qd_smoother_set_layer_weights(mg.h, int(layers), w.view(np.float64).ctypes.data_as(_DPTR)))


def smoother_layers(mg):
    return int(load().qd_smoother_layers(mg.h))


def smoother_get_layer_weights(mg):
    L = smoother_layers(mg)
    w = np.zeros((L, 9, 4, 4), dtype=np.complex128)
    _check(load().qd_smoother_get_layer_weights(mg.h, w.view(np.float64).ctypes.data_as(_DPTR)))
    return w


def smoother_enable(mg, enabled=True, mr_steps=2):
    _check(load().qd_smoother_enable(mg.h, 1 if enabled else 0, int(mr_steps)))


def smoother_apply(mg, nrhs, inp, out):
    _check(load().qd_smoother_apply(mg.h, int(nrhs), _ptr(inp), _ptr(out)))


def smoother_apply_f32(mg, nrhs, inp, out):
    """FP32 S in (FP16-rounded weights) on torch.complex64 fields in qd layout."""
    _check(load().qd_smoother_apply_f32(mg.h, int(nrhs), _ptr64(inp), _ptr64(out)))
