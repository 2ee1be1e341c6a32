"""Python binding of the C ABI in include/of.h (ctypes; argument marshalling
only: every step of the solve runs in libof.so).

The functions carry the C names (of_create, of_setup_grid, ...); arrays are
torch tensors (CUDA or CPU) or numpy arrays, contiguous, float32/float64.
Work is ordered on the stream given to of_create (default: torch's current
stream of the device).  A missing library raises at import: there is no
fallback path.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
# OFSOLVE_LIB selects another build of the same library (the bounds-check build)
LIB_PATH = os.environ.get("OFSOLVE_LIB") or os.path.join(_HERE, "libof.so")

if not os.path.exists(LIB_PATH):
    raise ImportError(f"{LIB_PATH} is missing: build it first (python -c 'import __graft_entry__ as g; g.build()')")

_lib = ctypes.CDLL(LIB_PATH)

OF_OK, OF_ERR_ARG, OF_ERR_CUDA, OF_ERR_OOM, OF_ERR_STATE, OF_ERR_NOT_CONVERGED, OF_ERR_BREAKDOWN, OF_ERR_TIMEOUT = range(8)
STATUS_NAMES = {0: "OK", 1: "ERR_ARG", 2: "ERR_CUDA", 3: "ERR_OOM", 4: "ERR_STATE", 5: "ERR_NOT_CONVERGED",
                6: "ERR_BREAKDOWN", 7: "ERR_TIMEOUT"}
OF_F32, OF_F64 = 0, 1
OF_PREC_FP64, OF_PREC_MIXED = 0, 1
OF_PC_SCHWARZ, OF_PC_JACOBI = 0, 1
OF_MODEL_ILLUMINATION, OF_MODEL_CONSTANT = 0, 1


class GridOpts(ctypes.Structure):
    _fields_ = [("tile_x", ctypes.c_int), ("tile_y", ctypes.c_int), ("overlap", ctypes.c_int),
                ("sweeps", ctypes.c_int), ("precision", ctypes.c_int), ("lam", ctypes.c_double),
                ("preconditioner", ctypes.c_int), ("omega", ctypes.c_double), ("sigma", ctypes.c_double),
                ("model", ctypes.c_int), ("coarse", ctypes.c_int), ("rho", ctypes.c_double),
                ("schwarz", ctypes.c_int), ("lambda_min", ctypes.c_double), ("half_sweeps", ctypes.c_int)]


class SolveOpts(ctypes.Structure):
    _fields_ = [("rtol", ctypes.c_double), ("max_outer", ctypes.c_int), ("max_inner", ctypes.c_int),
                ("warm_start", ctypes.c_int), ("inner_rtol", ctypes.c_double), ("host_loop", ctypes.c_int),
                ("pass_frac", ctypes.c_double)]


class SolveInfo(ctypes.Structure):
    _fields_ = [("status", ctypes.c_int), ("outer_iters", ctypes.c_int), ("inner_iters", ctypes.c_int),
                ("rel_residual", ctypes.c_double), ("ms", ctypes.c_float)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class Profile(ctypes.Structure):
    _fields_ = [("launches", ctypes.c_int * 4), ("ms", ctypes.c_double * 4)]

    KINDS = ("pcg_apply", "schwarz", "residual", "other")

    def as_dict(self):
        return {k: {"launches": int(self.launches[i]), "ms": float(self.ms[i])} for i, k in enumerate(self.KINDS)}


_vp = ctypes.c_void_p
_h = ctypes.c_void_p
_lib.of_create.argtypes = [ctypes.POINTER(_h), ctypes.c_int, _vp]
_lib.of_setup_grid.argtypes = [_h, ctypes.c_int, ctypes.POINTER(ctypes.c_int32), ctypes.POINTER(ctypes.c_int32),
                               ctypes.POINTER(GridOpts)]
_lib.of_set_frames.argtypes = [_h, ctypes.c_int, _vp, _vp, ctypes.c_int, ctypes.c_int64]
_lib.of_set_alpha.argtypes = [_h, ctypes.c_int, _vp, ctypes.c_double, ctypes.c_int]
_lib.of_get_alpha.argtypes = [_h, ctypes.c_int, _vp, ctypes.c_int]
_lib.of_set_lambda.argtypes = [_h, ctypes.c_int, _vp, ctypes.c_double, ctypes.c_int]
_lib.of_get_lambda.argtypes = [_h, ctypes.c_int, _vp, ctypes.c_int]
_lib.of_get_frames.argtypes = [_h, ctypes.c_int, _vp, _vp, ctypes.c_int]
_lib.of_get_element_data.argtypes = [_h, ctypes.c_int, _vp, ctypes.c_int]
_lib.of_set_wait_limit.argtypes = [_h, ctypes.c_int64]
_lib.of_set_alloc_limit.argtypes = [_h, ctypes.c_int64]
_lib.of_debug_starve_staging.argtypes = [_h, ctypes.c_int]
_lib.of_solve.argtypes = [_h, ctypes.POINTER(SolveOpts), ctypes.POINTER(_vp), ctypes.c_int, ctypes.POINTER(SolveInfo)]
_lib.of_adapt_alpha.argtypes = [_h, ctypes.c_double, ctypes.c_double, ctypes.c_double, ctypes.POINTER(_vp), ctypes.c_int]
_lib.of_adjoint.argtypes = [_h, ctypes.POINTER(_vp), ctypes.POINTER(_vp), ctypes.POINTER(_vp), ctypes.POINTER(_vp),
                            ctypes.c_int, ctypes.POINTER(SolveInfo)]
_lib.of_adapt_alpha_vjp.argtypes = [_h, ctypes.c_double, ctypes.c_double, ctypes.c_double, ctypes.POINTER(_vp),
                                    ctypes.POINTER(_vp), ctypes.POINTER(_vp), ctypes.POINTER(_vp), ctypes.POINTER(_vp),
                                    ctypes.c_int]
_lib.of_apply.argtypes = [_h, ctypes.c_int, _vp, _vp, _vp, ctypes.c_int]
_lib.of_precondition.argtypes = [_h, ctypes.c_int, _vp, _vp, ctypes.c_int]
_lib.of_residual.argtypes = [_h, ctypes.c_int, _vp, ctypes.c_int, ctypes.POINTER(ctypes.c_double)]
_lib.of_set_profiling.argtypes = [_h, ctypes.c_int]
_lib.of_get_profile.argtypes = [_h, ctypes.POINTER(Profile)]
_lib.of_get_schwarz_history.argtypes = [_h, ctypes.c_int, ctypes.POINTER(ctypes.c_double), ctypes.c_int,
                                        ctypes.POINTER(ctypes.c_int)]
_lib.of_residual_noalloc.argtypes = [ctypes.c_int, ctypes.c_int, _vp, _vp, _vp, ctypes.c_double, _vp, _vp, _vp, _vp]
_lib.of_destroy.argtypes = [_h]
_lib.of_last_error.argtypes = [_h]
_lib.of_last_error.restype = ctypes.c_char_p
for _f in ("of_create", "of_setup_grid", "of_set_frames", "of_get_element_data", "of_set_alpha", "of_get_alpha", "of_solve",
           "of_adapt_alpha", "of_adapt_alpha_vjp", "of_adjoint", "of_apply", "of_precondition", "of_residual",
           "of_set_profiling", "of_get_profile", "of_residual_noalloc", "of_get_schwarz_history", "of_set_lambda",
           "of_get_lambda", "of_destroy"):
    getattr(_lib, _f).restype = ctypes.c_int

EXPORTS = ("of_create", "of_setup_grid", "of_set_frames", "of_get_frames", "of_get_element_data", "of_set_alpha",
           "of_get_alpha", "of_solve",
           "of_adapt_alpha", "of_adapt_alpha_vjp", "of_adjoint", "of_apply", "of_precondition", "of_residual",
           "of_set_profiling", "of_get_profile", "of_residual_noalloc", "of_set_wait_limit", "of_debug_starve_staging",
           "of_set_alloc_limit", "of_get_schwarz_history", "of_set_lambda", "of_get_lambda",
           "of_destroy", "of_last_error")


class OFError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {msg}")
        self.status = status


def _ptr_dtype(a):
    """(pointer, of_dtype) of a contiguous torch tensor or numpy array."""
    if a is None:
        return None, OF_F32
    try:
        import torch
        if isinstance(a, torch.Tensor):
            if not a.is_contiguous():
                raise ValueError("arrays must be contiguous")
            if a.dtype not in (torch.float32, torch.float64):
                raise TypeError("arrays must be float32 or float64")
            return a.data_ptr(), OF_F64 if a.dtype == torch.float64 else OF_F32
    except ImportError:
        pass
    if isinstance(a, np.ndarray):
        if not a.flags.c_contiguous:
            raise ValueError("arrays must be C-contiguous")
        if a.dtype not in (np.float32, np.float64):
            raise TypeError("arrays must be float32 or float64")
        return a.ctypes.data, OF_F64 if a.dtype == np.float64 else OF_F32
    raise TypeError(f"unsupported array type {type(a)}")


def _check(h, status, allow=()):
    if status != OF_OK and status not in allow:
        raise OFError(status, of_last_error(h))
    return status


def of_last_error(h) -> str:
    return _lib.of_last_error(h).decode()


def of_create(device: int = 0, stream=None):
    """Creates a handle on `device`, ordered on `stream` (a torch.cuda.Stream,
    an integer cudaStream_t, or None for torch's current stream)."""
    if stream is None:
        import torch
        stream = torch.cuda.current_stream(device).cuda_stream
    elif not isinstance(stream, int):
        stream = stream.cuda_stream
    h = _h()
    st = _lib.of_create(ctypes.byref(h), int(device), _vp(stream))
    if st != OF_OK:
        raise OFError(st, of_last_error(None))
    return h


def of_setup_grid(h, sizes, tile=(32, 32), overlap=0, sweeps=1, precision=OF_PREC_MIXED, lam=1.0,
                  preconditioner=OF_PC_SCHWARZ, omega=1.0, sigma=0.0, model=0, coarse=0, rho=0.0, schwarz=0,
                  half_sweeps=0, lambda_min=0.0):
    """sizes: list of (W, H); omega: relaxation factor of the local block SOR
    sweeps, in (0, 2); sigma: K_sigma pre-smoothing of the frames (0: none);
    model: OF_MODEL_ILLUMINATION or OF_MODEL_CONSTANT; coarse: spacing of the
    two-level preconditioner's coarse grid in nodes (0: one level); rho: K_rho
    integration scale of the data term (0: none); schwarz: 1 makes of_solve
    run the stationary Schwarz iteration instead of the PCG; half_sweeps:
    FP16 paired local sweeps on the mixed path (0: where the tile allows, 1:
    required, -1: off); lambda_min > 0: a per-element lambda, adapted by
    of_adapt_alpha with this threshold."""
    n = len(sizes)
    Wa = (ctypes.c_int32 * n)(*[int(w) for w, _ in sizes])
    Ha = (ctypes.c_int32 * n)(*[int(hh) for _, hh in sizes])
    o = GridOpts(int(tile[0]), int(tile[1]), int(overlap), int(sweeps), int(precision), float(lam), int(preconditioner),
                 float(omega), float(sigma), int(model), int(coarse), float(rho), int(schwarz), float(lambda_min),
                 int(half_sweeps))
    return _check(h, _lib.of_setup_grid(h, n, Wa, Ha, ctypes.byref(o)))


def of_set_frames(h, pair, f1, f2):
    p1, dt = _ptr_dtype(f1)
    p2, dt2 = _ptr_dtype(f2)
    if dt != dt2:
        raise TypeError("frames must share a dtype")
    return _check(h, _lib.of_set_frames(h, int(pair), _vp(p1), _vp(p2), dt, int(f1.shape[-1])))


def of_set_alpha(h, pair, alpha=None, alpha_const=0.0):
    p, dt = _ptr_dtype(alpha)
    return _check(h, _lib.of_set_alpha(h, int(pair), _vp(p) if p else None, float(alpha_const), dt))


def of_get_element_data(h, pair, out):
    """The K_rho element data of a pair into an [18][H-1][W-1] array (plane
    t * 9 + k: A_rho entries 00, 01, 02, 11, 12, 22, then F)."""
    p, dt = _ptr_dtype(out)
    return _check(h, _lib.of_get_element_data(h, int(pair), _vp(p), dt))


def of_get_frames(h, pair, f1, f2):
    """The stored (K_sigma-smoothed) frames into two [H][W] arrays."""
    p1, dt = _ptr_dtype(f1)
    p2, dt2 = _ptr_dtype(f2)
    if dt != dt2:
        raise TypeError("frames must share a dtype")
    return _check(h, _lib.of_get_frames(h, int(pair), _vp(p1), _vp(p2), dt))


def of_set_lambda(h, pair, lam=None, lam_const=0.0):
    """Per-element lambda of a pair ([H-1][W-1][2]) or a constant (grids with lambda_min > 0)."""
    p, dt = _ptr_dtype(lam)
    return _check(h, _lib.of_set_lambda(h, int(pair), _vp(p) if p else None, float(lam_const), dt))


def of_get_lambda(h, pair, out):
    p, dt = _ptr_dtype(out)
    return _check(h, _lib.of_get_lambda(h, int(pair), _vp(p), dt))


def of_get_alpha(h, pair, out):
    p, dt = _ptr_dtype(out)
    return _check(h, _lib.of_get_alpha(h, int(pair), _vp(p), dt))


def of_solve(h, U, rtol=1e-6, max_outer=20, max_inner=2000, warm_start=False, inner_rtol=0.0, raise_on=True,
             host_loop=False, pass_frac=0.0):
    """U: list of [3][H][W] arrays (one per pair, same dtype).  Returns
    (status, [info dict per pair])."""
    ptrs = [_ptr_dtype(u) for u in U]
    dt = ptrs[0][1]
    arr = (_vp * len(U))(*[p for p, _ in ptrs])
    info = (SolveInfo * len(U))()
    o = SolveOpts(float(rtol), int(max_outer), int(max_inner), int(bool(warm_start)), float(inner_rtol),
                  int(bool(host_loop)), float(pass_frac))
    st = _lib.of_solve(h, ctypes.byref(o), arr, dt, info)
    if raise_on:
        _check(h, st)
    return st, [i.as_dict() for i in info]


def of_get_schwarz_history(h, pair):
    """||U^k - U^{k-1}||_2 of each iteration of the last stationary Schwarz
    solve of a pair (numpy array)."""
    n = ctypes.c_int(0)
    _check(h, _lib.of_get_schwarz_history(h, int(pair), None, 0, ctypes.byref(n)))
    out = np.zeros(max(n.value, 1))
    _check(h, _lib.of_get_schwarz_history(h, int(pair), out.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                                          n.value, ctypes.byref(n)))
    return out[:n.value]


def of_adapt_alpha(h, kappa, eta_thr, alpha_th, eta=None):
    if eta is not None:
        ptrs = [_ptr_dtype(e) for e in eta]
        arr = (_vp * len(eta))(*[p for p, _ in ptrs])
        dt = ptrs[0][1]
    else:
        arr, dt = None, OF_F32
    return _check(h, _lib.of_adapt_alpha(h, float(kappa), float(eta_thr), float(alpha_th), arr, dt))


def of_adjoint(h, dLdU, dLdalpha=None, dLdf2=None, dLdf1=None, raise_on=True):
    n = len(dLdU)

    def lst(xs):
        if xs is None:
            return None, None
        ps = [_ptr_dtype(x) for x in xs]
        return (_vp * n)(*[p for p, _ in ps]), ps[0][1]

    a_u, dt = lst(dLdU)
    a_a, _ = lst(dLdalpha)
    a_2, _ = lst(dLdf2)
    a_1, _ = lst(dLdf1)
    info = (SolveInfo * n)()
    st = _lib.of_adjoint(h, a_u, a_a, a_2, a_1, dt, info)
    if raise_on:
        _check(h, st)
    return st, [i.as_dict() for i in info]


def of_adapt_alpha_vjp(h, kappa, eta_thr, alpha_th, dLdalpha_new, dLdalpha, dLdU, dLdf2=None, dLdf1=None):
    """VJP of one adaptation pass at the current alpha and solution (device
    tensors, one per pair)."""
    n = len(dLdalpha_new)

    def lst(xs):
        if xs is None:
            return None, None
        ps = [_ptr_dtype(x) for x in xs]
        return (_vp * n)(*[p for p, _ in ps]), ps[0][1]

    a_v, dt = lst(dLdalpha_new)
    a_a, _ = lst(dLdalpha)
    a_u, _ = lst(dLdU)
    a_2, _ = lst(dLdf2)
    a_1, _ = lst(dLdf1)
    return _check(h, _lib.of_adapt_alpha_vjp(h, float(kappa), float(eta_thr), float(alpha_th), a_v, a_a, a_u, a_2,
                                             a_1, dt))


def of_apply(h, pair, p, q, b=None):
    pp, dt = _ptr_dtype(p)
    pq, _ = _ptr_dtype(q)
    pb, _ = _ptr_dtype(b)
    return _check(h, _lib.of_apply(h, int(pair), _vp(pp), _vp(pq), _vp(pb) if pb else None, dt))


def of_precondition(h, pair, r, z):
    pr, dt = _ptr_dtype(r)
    pz, _ = _ptr_dtype(z)
    return _check(h, _lib.of_precondition(h, int(pair), _vp(pr), _vp(pz), dt))


def of_residual(h, pair, U) -> float:
    pu, dt = _ptr_dtype(U)
    rel = ctypes.c_double(0.0)
    _check(h, _lib.of_residual(h, int(pair), _vp(pu), dt, ctypes.byref(rel)))
    return float(rel.value)


def of_set_alloc_limit(h, nbytes):
    """Test hook: the handle's device allocations fail as out of memory past
    nbytes in all (0: no limit)."""
    return _check(h, _lib.of_set_alloc_limit(h, int(nbytes)))


def of_set_wait_limit(h, cycles):
    """Bound of every device wait in SM clock cycles (<= 0: the default)."""
    return _check(h, _lib.of_set_wait_limit(h, int(cycles)))


def of_debug_starve_staging(h, extra_bytes):
    """Test hook: staging barriers expect extra_bytes more than delivered, so
    their bounded waits run out (0: off)."""
    return _check(h, _lib.of_debug_starve_staging(h, int(extra_bytes)))


def of_set_profiling(h, on=True):
    return _check(h, _lib.of_set_profiling(h, int(bool(on))))


def of_get_profile(h) -> dict:
    p = Profile()
    _check(h, _lib.of_get_profile(h, ctypes.byref(p)))
    return p.as_dict()


def of_residual_noalloc(f1, f2, alpha, lam, U, r, norms, stream=None) -> int:
    """Handle-free FP64 residual for callers that cannot allocate device
    memory: all arrays are float64 CUDA tensors supplied by the caller
    (r may be None); norms (3 values) receives the relative residual and the
    two squared norms.  Returns the of_status code."""
    H, W = int(f1.shape[0]), int(f1.shape[1])
    if stream is None:
        import torch
        stream = torch.cuda.current_stream(f1.device).cuda_stream
    ptr = lambda t: None if t is None else _vp(_ptr_dtype(t)[0])
    return int(_lib.of_residual_noalloc(W, H, ptr(f1), ptr(f2), ptr(alpha), float(lam), ptr(U), ptr(r), ptr(norms),
                                        _vp(stream)))


def of_destroy(h):
    return _lib.of_destroy(h)
