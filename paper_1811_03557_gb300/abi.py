"""ctypes binding of libdpm (include/dpm.h), same names as the C ABI.

Argument marshalling only: every step of the method runs in the CUDA library.
Array arguments are torch tensors on the GPU (their data_ptr() is passed) or
None; ``stream`` is a torch.cuda.Stream, a raw cudaStream_t integer, or None
for torch's current stream.  A nonzero status raises DPMError with the
library's message.  There is no fallback: if libdpm.so is missing or a call
fails, the error propagates.
"""
from __future__ import annotations

import ctypes as C
import os
import re

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libdpm.so")
HEADER = os.path.join(os.path.dirname(_HERE), "include", "dpm.h")

DPM_OK, DPM_EINVAL, DPM_ENOMEM, DPM_ETIMEOUT, DPM_ENUMERIC, DPM_EUNSUPPORTED, DPM_ECUDA = (
    0, -1, -2, -3, -4, -5, -6)
DPM_PREC_FP32, DPM_PREC_FP64, DPM_PREC_TC32, DPM_PREC_FFT32 = 0, 1, 2, 3
DPM_LBL_MPLUS, DPM_LBL_GIN, DPM_LBL_GEX, DPM_LBL_SHELL = 1, 2, 4, 8


class DPMError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"libdpm error {code}: {msg}")
        self.code = code


class dpm_geom(C.Structure):
    _fields_ = [("kind", C.c_int), ("center", C.c_double * 3), ("axes", C.c_double * 3)]


class dpm_gaussian(C.Structure):
    _fields_ = [("amp", C.c_double), ("alpha", C.c_double), ("center", C.c_double * 3),
                ("zscale", C.c_double)]


class dpm_bep_info(C.Structure):
    _fields_ = [("N", C.c_int), ("lo", C.c_double), ("hi", C.c_double), ("h", C.c_double),
                ("sigma", C.c_double), ("K", C.c_int), ("beta", C.c_int), ("ncol", C.c_int),
                ("precision", C.c_int), ("n_mplus", C.c_int64), ("n_gin", C.c_int64),
                ("n_gex", C.c_int64), ("n_gamma", C.c_int64), ("n_shell", C.c_int64)]


class dpm_pks_params(C.Structure):
    _fields_ = [("geom", dpm_geom), ("N", C.c_int), ("lo", C.c_double), ("hi", C.c_double),
                ("chi", C.c_double), ("dt_max", C.c_double), ("K", C.c_int), ("beta", C.c_int),
                ("precision", C.c_int), ("dt_mode", C.c_int), ("rebuild", C.c_int),
                ("clamp", C.c_int)]


class dpm_pks_stats(C.Structure):
    _fields_ = [("t", C.c_double), ("dt", C.c_double), ("step", C.c_int64), ("rebuilt", C.c_int),
                ("mass", C.c_double), ("max_rho", C.c_double), ("min_rho", C.c_double),
                ("min_c", C.c_double), ("m2", C.c_double), ("free_energy", C.c_double)]


class dpm_dd_params(C.Structure):
    _fields_ = [("center", C.c_double * 3), ("r1", C.c_double), ("r2", C.c_double),
                ("N1", C.c_int), ("lo1", C.c_double), ("hi1", C.c_double),
                ("N2", C.c_int), ("lo2", C.c_double), ("hi2", C.c_double),
                ("KZ", C.c_int), ("KG", C.c_int), ("precision", C.c_int)]


class dpm_dd_info(C.Structure):
    _fields_ = [("N", C.c_int * 2), ("h", C.c_double * 2), ("precision", C.c_int * 2),
                ("n_mplus", C.c_int64 * 2), ("n_gin", C.c_int64 * 2), ("n_gamma", C.c_int64 * 2),
                ("nz", C.c_int), ("ng", C.c_int), ("ncol", C.c_int), ("sigma", C.c_double)]


class dpm_dd2_params(C.Structure):
    _fields_ = [("center", C.c_double * 3), ("R", C.c_double), ("rz", C.c_double), ("zoff", C.c_double),
                ("N1", C.c_int), ("lo1", C.c_double), ("hi1", C.c_double), ("origin1", C.c_double * 3),
                ("N2", C.c_int), ("lo2", C.c_double), ("hi2", C.c_double), ("origin2", C.c_double * 3),
                ("MZ", C.c_int), ("MG", C.c_int), ("precision", C.c_int), ("gamma_series", C.c_int)]


class dpm_dd2_info(C.Structure):
    _fields_ = [("N", C.c_int * 2), ("h", C.c_double * 2), ("precision", C.c_int * 2),
                ("n_mplus", C.c_int64 * 2), ("n_gin", C.c_int64 * 2), ("n_gamma", C.c_int64 * 2),
                ("n_rows", C.c_int64 * 2), ("n_wedge", C.c_int64 * 2), ("ncol", C.c_int),
                ("sigma", C.c_double)]


DPM_ML_MAX = 16


class dpm_ml_params(C.Structure):
    _fields_ = [("center", C.c_double * 3), ("L", C.c_int), ("radii", C.c_double * DPM_ML_MAX),
                ("N", C.c_int * DPM_ML_MAX), ("lo", C.c_double * DPM_ML_MAX), ("hi", C.c_double * DPM_ML_MAX),
                ("K", C.c_int * DPM_ML_MAX), ("KG", C.c_int), ("precision", C.c_int)]


class dpm_ml_info(C.Structure):
    _fields_ = [("L", C.c_int), ("N", C.c_int * DPM_ML_MAX), ("h", C.c_double * DPM_ML_MAX),
                ("precision", C.c_int * DPM_ML_MAX), ("n_mplus", C.c_int64 * DPM_ML_MAX),
                ("n_gin", C.c_int64 * DPM_ML_MAX), ("n_gamma", C.c_int64 * DPM_ML_MAX), ("ncol", C.c_int),
                ("sigma", C.c_double)]


_P = C.c_void_p
_SIGS = {
    "dpm_last_error": (C.c_char_p, []),
    "dpm_ctx_create": (C.c_int, [C.c_int, C.POINTER(C.c_void_p)]),
    "dpm_ctx_destroy": (C.c_int, [_P]),
    "dpm_classify": (C.c_int, [_P, C.POINTER(dpm_geom), C.c_int, C.c_double, C.c_double, _P, _P,
                               C.c_int64, _P, C.c_int64, C.POINTER(C.c_int64),
                               C.POINTER(C.c_int64), _P]),
    "dpm_aux_solve_batched": (C.c_int, [_P, C.c_int, C.c_double, C.c_double, C.c_int, _P, _P,
                                        C.c_int, _P]),
    "dpm_bep_build": (C.c_int, [_P, C.POINTER(dpm_geom), C.c_int, C.c_double, C.c_double,
                                C.c_double, C.c_int, C.c_int, C.c_int, C.POINTER(C.c_void_p), _P]),
    "dpm_bep_get_info": (C.c_int, [_P, C.POINTER(dpm_bep_info)]),
    "dpm_bep_matrix": (C.c_int, [_P, _P, _P]),
    "dpm_bep_gamma_geometry": (C.c_int, [_P, _P, _P, _P, _P, _P]),
    "dpm_bep_destroy": (C.c_int, [_P]),
    "dpm_solve": (C.c_int, [_P, _P, _P, _P, _P, _P]),
    "dpm_solve_batched": (C.c_int, [_P, C.c_int, _P, _P, _P, _P, _P]),
    "dpm_bep_device_bytes": (C.c_int, [_P, C.POINTER(C.c_int64)]),
    "dpm_bep_reserve": (C.c_int, [_P, C.c_int]),
    "dpm_pks_device_bytes": (C.c_int, [_P, C.POINTER(C.c_int64)]),
    "dpm_pks_create": (C.c_int, [_P, C.POINTER(dpm_pks_params), C.POINTER(dpm_gaussian),
                                 C.POINTER(dpm_gaussian), C.POINTER(C.c_void_p), _P]),
    "dpm_pks_set_state": (C.c_int, [_P, _P, _P, _P]),
    "dpm_pks_step": (C.c_int, [_P, C.c_int, C.POINTER(dpm_pks_stats), _P]),
    "dpm_pks_set_graph": (C.c_int, [_P, C.c_int, _P]),
    "dpm_pks_get_state": (C.c_int, [_P, _P, _P, _P]),
    "dpm_pks_destroy": (C.c_int, [_P]),
    "dpm_aux_solve_batched_noalloc": (C.c_int, [C.c_int, C.c_double, C.c_double, C.c_int, _P,
                                                _P, _P]),
    "dpm_simt_tile": (C.c_int, [C.c_int, C.c_int, C.c_int, C.POINTER(C.c_int)]),
    "dpm_dd_build": (C.c_int, [_P, C.POINTER(dpm_dd_params), C.c_double, C.POINTER(C.c_void_p), _P]),
    "dpm_dd_get_info": (C.c_int, [_P, C.POINTER(dpm_dd_info)]),
    "dpm_dd_matrix": (C.c_int, [_P, _P, _P]),
    "dpm_dd_solve": (C.c_int, [_P, _P, _P, _P, _P, _P, _P, _P]),
    "dpm_dd_destroy": (C.c_int, [_P]),
    "dpm_dd_pks_create": (C.c_int, [_P, C.POINTER(dpm_dd_params), C.c_double, C.c_double, C.c_int,
                                    C.c_int, C.c_int, C.POINTER(dpm_gaussian), C.POINTER(dpm_gaussian),
                                    C.POINTER(C.c_void_p), _P]),
    "dpm_dd_pks_step": (C.c_int, [_P, C.c_int, C.POINTER(dpm_pks_stats), _P]),
    "dpm_dd_pks_set_graph": (C.c_int, [_P, C.c_int, _P]),
    "dpm_dd_pks_get_state": (C.c_int, [_P, C.c_int, _P, _P, _P]),
    "dpm_dd_pks_destroy": (C.c_int, [_P]),
    "dpm_dd2_build": (C.c_int, [_P, C.POINTER(dpm_dd2_params), C.c_double, C.POINTER(C.c_void_p), _P]),
    "dpm_dd2_get_info": (C.c_int, [_P, C.POINTER(dpm_dd2_info)]),
    "dpm_dd2_matrix": (C.c_int, [_P, _P, _P]),
    "dpm_dd2_gamma": (C.c_int, [_P, C.c_int, _P, _P, _P, _P]),
    "dpm_dd2_solve": (C.c_int, [_P, _P, _P, _P, _P, _P, _P, _P, _P]),
    "dpm_dd2_destroy": (C.c_int, [_P]),
    "dpm_dd2_pks_create": (C.c_int, [_P, C.POINTER(dpm_dd2_params), C.c_double, C.c_double, C.c_int,
                                     C.c_int, C.c_int, C.POINTER(dpm_gaussian), C.POINTER(dpm_gaussian),
                                     C.POINTER(C.c_void_p), _P]),
    "dpm_dd2_pks_step": (C.c_int, [_P, C.c_int, C.POINTER(dpm_pks_stats), _P]),
    "dpm_dd2_pks_set_graph": (C.c_int, [_P, C.c_int, _P]),
    "dpm_dd2_pks_get_state": (C.c_int, [_P, C.c_int, _P, _P, _P]),
    "dpm_dd2_pks_destroy": (C.c_int, [_P]),
    "dpm_ml_build": (C.c_int, [_P, C.POINTER(dpm_ml_params), C.c_double, C.POINTER(C.c_void_p), _P]),
    "dpm_ml_get_info": (C.c_int, [_P, C.POINTER(dpm_ml_info)]),
    "dpm_ml_matrix": (C.c_int, [_P, _P, _P]),
    "dpm_ml_solve": (C.c_int, [_P, C.POINTER(C.c_void_p), _P, C.POINTER(C.c_void_p), _P, _P]),
    "dpm_ml_destroy": (C.c_int, [_P]),
    "dpm_ml_pks_create": (C.c_int, [_P, C.POINTER(dpm_ml_params), C.c_double, C.c_double, C.c_int, C.c_int,
                                    C.c_int, C.POINTER(dpm_gaussian), C.POINTER(dpm_gaussian),
                                    C.POINTER(C.c_void_p), _P]),
    "dpm_ml_pks_step": (C.c_int, [_P, C.c_int, C.POINTER(dpm_pks_stats), _P]),
    "dpm_ml_pks_set_graph": (C.c_int, [_P, C.c_int, _P]),
    "dpm_ml_pks_get_state": (C.c_int, [_P, C.c_int, _P, _P, _P]),
    "dpm_ml_pks_destroy": (C.c_int, [_P]),
    "dpm_launch_count": (C.c_int64, []),
    "dpm_profile_enable": (C.c_int, [C.c_int]),
    "dpm_profile_read": (C.c_int, [C.c_char_p, C.POINTER(C.c_double), C.POINTER(C.c_int64)]),
    "dpm_profile_reset": (C.c_int, []),
}

_lib = None


def lib() -> C.CDLL:
    """Load libdpm.so (raises if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"{LIB_PATH} is missing: build it with "
                               "`python -m paper_1811_03557_gb300.build`")
        L = C.CDLL(LIB_PATH)
        for name, (res, args) in _SIGS.items():
            fn = getattr(L, name)
            fn.restype = res
            fn.argtypes = args
        _lib = L
    return _lib


def header_functions() -> list[str]:
    """Names of the functions declared in include/dpm.h."""
    txt = open(HEADER).read()
    return sorted(set(re.findall(r"\b(dpm_[a-z_0-9]+)\s*\(", txt)))


def _check(rc: int):
    if rc != DPM_OK:
        raise DPMError(rc, lib().dpm_last_error().decode(errors="replace"))


def _ptr(t):
    if t is None:
        return None
    if isinstance(t, int):
        return t
    return t.data_ptr()


def _stream(stream):
    if stream is None:
        import torch
        return torch.cuda.current_stream().cuda_stream
    if isinstance(stream, int):
        return stream
    return stream.cuda_stream


def make_geom(geom) -> dpm_geom:
    """From an object with kind/center/axes (e.g. workloads.Geometry)."""
    g = dpm_geom()
    g.kind = int(geom.kind)
    for i in range(3):
        g.center[i] = float(geom.center[i])
        g.axes[i] = float(geom.axes[i])
    return g


def make_gaussian(gs) -> dpm_gaussian:
    g = dpm_gaussian()
    g.amp, g.alpha, g.zscale = float(gs.amp), float(gs.alpha), float(gs.zscale)
    for i in range(3):
        g.center[i] = float(gs.center[i])
    return g


# ---- entry points ------------------------------------------------------------
def dpm_last_error() -> str:
    return lib().dpm_last_error().decode(errors="replace")


def dpm_ctx_create(device: int = 0):
    h = C.c_void_p()
    _check(lib().dpm_ctx_create(device, C.byref(h)))
    return h


def dpm_ctx_destroy(ctx):
    _check(lib().dpm_ctx_destroy(ctx))


def dpm_classify(ctx, geom, N, lo, hi, labels=None, gin_idx=None, gex_idx=None, stream=None):
    """Returns (n_gin, n_gex).  labels: uint8 tensor [N^3]; gin_idx/gex_idx: int32 tensors."""
    ng, ne = C.c_int64(), C.c_int64()
    g = make_geom(geom) if not isinstance(geom, dpm_geom) else geom
    _check(lib().dpm_classify(ctx, C.byref(g), N, lo, hi, _ptr(labels), _ptr(gin_idx),
                              0 if gin_idx is None else gin_idx.numel(), _ptr(gex_idx),
                              0 if gex_idx is None else gex_idx.numel(), C.byref(ng),
                              C.byref(ne), _stream(stream)))
    return ng.value, ne.value


def dpm_aux_solve_batched(ctx, N, h, sigma, B, q, u, precision=DPM_PREC_FP32, stream=None):
    _check(lib().dpm_aux_solve_batched(ctx, N, h, sigma, B, _ptr(q), _ptr(u), precision,
                                       _stream(stream)))


def dpm_aux_solve_batched_noalloc(N, h, sigma, B, q, u, stream=None):
    """FP32 AP solve whose scratch is a fixed device array inside the library
    (no allocation); q, u float32 device tensors [B][N][N][N]."""
    _check(lib().dpm_aux_solve_batched_noalloc(N, h, sigma, B, _ptr(q), _ptr(u), _stream(stream)))


def dpm_simt_tile(N, precision=DPM_PREC_FP32, B=1):
    """Tile width the SIMT solver tuned for (N, precision, B) on the current
    device, 0 if none yet."""
    t = C.c_int(0)
    _check(lib().dpm_simt_tile(N, precision, B, C.byref(t)))
    return t.value


def dpm_bep_build(ctx, geom, N, lo, hi, sigma, K, beta=1, precision=DPM_PREC_FP32, stream=None):
    h = C.c_void_p()
    g = make_geom(geom) if not isinstance(geom, dpm_geom) else geom
    _check(lib().dpm_bep_build(ctx, C.byref(g), N, lo, hi, sigma, K, beta, precision,
                               C.byref(h), _stream(stream)))
    return h


def dpm_bep_get_info(bep) -> dpm_bep_info:
    info = dpm_bep_info()
    _check(lib().dpm_bep_get_info(bep, C.byref(info)))
    return info


def dpm_bep_matrix(bep, A, stream=None):
    _check(lib().dpm_bep_matrix(bep, _ptr(A), _stream(stream)))


def dpm_bep_gamma_geometry(bep, gamma_idx=None, foot=None, normal=None, dist=None, stream=None):
    _check(lib().dpm_bep_gamma_geometry(bep, _ptr(gamma_idx), _ptr(foot), _ptr(normal),
                                        _ptr(dist), _stream(stream)))


def dpm_bep_destroy(bep):
    _check(lib().dpm_bep_destroy(bep))


def dpm_solve(bep, f, u, neumann=None, coeffs=None, stream=None):
    _check(lib().dpm_solve(bep, _ptr(f), _ptr(neumann), _ptr(u), _ptr(coeffs), _stream(stream)))


def dpm_solve_batched(bep, fs, us, neumanns=None, coeffs=None, stream=None):
    """Solve len(fs) requests against one BEP in one batch (lists of device tensors)."""
    n = len(fs)
    arr = C.c_void_p * n
    fa = arr(*[_ptr(x) for x in fs])
    ua = arr(*[_ptr(x) for x in us])
    na = arr(*[_ptr(x) for x in neumanns]) if neumanns is not None else None
    ca = arr(*[_ptr(x) for x in coeffs]) if coeffs is not None else None
    _check(lib().dpm_solve_batched(bep, n, fa, na, ua, ca, _stream(stream)))


def dpm_bep_device_bytes(bep) -> int:
    v = C.c_int64(0)
    _check(lib().dpm_bep_device_bytes(bep, C.byref(v)))
    return int(v.value)


def dpm_bep_reserve(bep, max_nreq: int):
    _check(lib().dpm_bep_reserve(bep, int(max_nreq)))


def dpm_pks_device_bytes(pks) -> int:
    v = C.c_int64(0)
    _check(lib().dpm_pks_device_bytes(pks, C.byref(v)))
    return int(v.value)


def dpm_pks_create(ctx, params: dpm_pks_params, rho0, c0, stream=None):
    h = C.c_void_p()
    g0 = make_gaussian(rho0) if not isinstance(rho0, dpm_gaussian) else rho0
    g1 = make_gaussian(c0) if not isinstance(c0, dpm_gaussian) else c0
    _check(lib().dpm_pks_create(ctx, C.byref(params), C.byref(g0), C.byref(g1), C.byref(h),
                                _stream(stream)))
    return h


def dpm_pks_set_state(pks, rho, c, stream=None):
    _check(lib().dpm_pks_set_state(pks, _ptr(rho), _ptr(c), _stream(stream)))


def dpm_pks_step(pks, nsteps=1, want_stats=True, stream=None):
    st = dpm_pks_stats()
    _check(lib().dpm_pks_step(pks, nsteps, C.byref(st) if want_stats else None, _stream(stream)))
    return st if want_stats else None


def dpm_pks_set_graph(pks, on=True, stream=None):
    _check(lib().dpm_pks_set_graph(pks, 1 if on else 0, _stream(stream)))


def dpm_pks_get_state(pks, rho, c, stream=None):
    _check(lib().dpm_pks_get_state(pks, _ptr(rho), _ptr(c), _stream(stream)))


def dpm_pks_destroy(pks):
    _check(lib().dpm_pks_destroy(pks))


def pks_params(geom, N, lo, hi, chi, dt_max, K, beta=1, precision=DPM_PREC_FP32, dt_mode=0,
               rebuild=0, clamp=1) -> dpm_pks_params:
    p = dpm_pks_params()
    p.geom = make_geom(geom)
    p.N, p.lo, p.hi, p.chi, p.dt_max = N, lo, hi, chi, dt_max
    p.K, p.beta, p.precision, p.dt_mode, p.rebuild, p.clamp = K, beta, precision, dt_mode, rebuild, clamp
    return p


def dd_params(center, r1, r2, N1, lo1, hi1, N2, lo2, hi2, KZ, KG, precision=DPM_PREC_FP32) -> dpm_dd_params:
    p = dpm_dd_params()
    for t in range(3):
        p.center[t] = center[t]
    p.r1, p.r2, p.N1, p.lo1, p.hi1, p.N2, p.lo2, p.hi2 = r1, r2, N1, lo1, hi1, N2, lo2, hi2
    p.KZ, p.KG, p.precision = KZ, KG, precision
    return p


def dpm_dd_build(ctx, params: dpm_dd_params, sigma, stream=None):
    h = C.c_void_p()
    _check(lib().dpm_dd_build(ctx, C.byref(params), sigma, C.byref(h), _stream(stream)))
    return h


def dpm_dd_get_info(dd) -> dpm_dd_info:
    info = dpm_dd_info()
    _check(lib().dpm_dd_get_info(dd, C.byref(info)))
    return info


def dpm_dd_matrix(dd, A, stream=None):
    _check(lib().dpm_dd_matrix(dd, _ptr(A), _stream(stream)))


def dpm_dd_solve(dd, f1, f2, u1, u2, neumann2=None, coeffs=None, stream=None):
    _check(lib().dpm_dd_solve(dd, _ptr(f1), _ptr(f2), _ptr(neumann2), _ptr(u1), _ptr(u2), _ptr(coeffs),
                              _stream(stream)))


def dpm_dd_destroy(dd):
    _check(lib().dpm_dd_destroy(dd))


def dpm_dd_pks_create(ctx, params: dpm_dd_params, chi, dt_max, dt_mode, rebuild, clamp, rho0, c0,
                      stream=None):
    h = C.c_void_p()
    g0, g1 = make_gaussian(rho0), make_gaussian(c0)
    _check(lib().dpm_dd_pks_create(ctx, C.byref(params), chi, dt_max, dt_mode, rebuild, clamp, C.byref(g0),
                                   C.byref(g1), C.byref(h), _stream(stream)))
    return h


def dpm_dd_pks_step(pks, nsteps=1, want_stats=True, stream=None):
    st = dpm_pks_stats()
    _check(lib().dpm_dd_pks_step(pks, nsteps, C.byref(st) if want_stats else None, _stream(stream)))
    return st if want_stats else None


def dpm_dd_pks_set_graph(pks, on=True, stream=None):
    _check(lib().dpm_dd_pks_set_graph(pks, 1 if on else 0, _stream(stream)))


def dpm_dd_pks_get_state(pks, l, rho, c, stream=None):
    _check(lib().dpm_dd_pks_get_state(pks, l, _ptr(rho), _ptr(c), _stream(stream)))


def dpm_dd_pks_destroy(pks):
    _check(lib().dpm_dd_pks_destroy(pks))


def dpm_launch_count() -> int:
    return int(lib().dpm_launch_count())


def dpm_profile_enable(on: bool = True):
    _check(lib().dpm_profile_enable(1 if on else 0))


def dpm_profile_read(name: str | None = None):
    """(total device ms, launches) of the recorded kernels whose name contains `name`."""
    ms, n = C.c_double(), C.c_int64()
    _check(lib().dpm_profile_read(name.encode() if name else None, C.byref(ms), C.byref(n)))
    return ms.value, n.value


def dpm_profile_reset():
    _check(lib().dpm_profile_reset())


# ---- domain decomposition, Case 2 (interface meeting Gamma) -------------------------
def dd2_params(center, R, rz, zoff, N1, lo1, hi1, origin1, N2, lo2, hi2, origin2, MZ, MG,
               precision=DPM_PREC_FP32, gamma_series=2) -> dpm_dd2_params:
    p = dpm_dd2_params()
    for t in range(3):
        p.center[t], p.origin1[t], p.origin2[t] = center[t], origin1[t], origin2[t]
    p.R, p.rz, p.zoff = R, rz, zoff
    p.N1, p.lo1, p.hi1, p.N2, p.lo2, p.hi2 = N1, lo1, hi1, N2, lo2, hi2
    p.MZ, p.MG, p.precision, p.gamma_series = MZ, MG, precision, gamma_series
    return p


def dpm_dd2_build(ctx, params: dpm_dd2_params, sigma, stream=None):
    h = C.c_void_p()
    _check(lib().dpm_dd2_build(ctx, C.byref(params), sigma, C.byref(h), _stream(stream)))
    return h


def dpm_dd2_get_info(dd) -> dpm_dd2_info:
    info = dpm_dd2_info()
    _check(lib().dpm_dd2_get_info(dd, C.byref(info)))
    return info


def dpm_dd2_matrix(dd, A, stream=None):
    _check(lib().dpm_dd2_matrix(dd, _ptr(A), _stream(stream)))


def dpm_dd2_gamma(dd, l, gamma_idx=None, flags=None, foot_gamma=None, stream=None):
    _check(lib().dpm_dd2_gamma(dd, l, _ptr(gamma_idx), _ptr(flags), _ptr(foot_gamma), _stream(stream)))


def dpm_dd2_solve(dd, f1, f2, u1, u2, neumann1=None, neumann2=None, coeffs=None, stream=None):
    _check(lib().dpm_dd2_solve(dd, _ptr(f1), _ptr(f2), _ptr(neumann1), _ptr(neumann2), _ptr(u1), _ptr(u2),
                               _ptr(coeffs), _stream(stream)))


def dpm_dd2_destroy(dd):
    _check(lib().dpm_dd2_destroy(dd))


def dpm_dd2_pks_create(ctx, params: dpm_dd2_params, chi, dt_max, dt_mode, rebuild, clamp, rho0, c0,
                       stream=None):
    h = C.c_void_p()
    g0, g1 = make_gaussian(rho0), make_gaussian(c0)
    _check(lib().dpm_dd2_pks_create(ctx, C.byref(params), chi, dt_max, dt_mode, rebuild, clamp, C.byref(g0),
                                    C.byref(g1), C.byref(h), _stream(stream)))
    return h


def dpm_dd2_pks_step(pks, nsteps=1, want_stats=True, stream=None):
    st = dpm_pks_stats()
    _check(lib().dpm_dd2_pks_step(pks, nsteps, C.byref(st) if want_stats else None, _stream(stream)))
    return st if want_stats else None


def dpm_dd2_pks_set_graph(pks, on=True, stream=None):
    _check(lib().dpm_dd2_pks_set_graph(pks, 1 if on else 0, _stream(stream)))


def dpm_dd2_pks_get_state(pks, l, rho, c, stream=None):
    _check(lib().dpm_dd2_pks_get_state(pks, l, _ptr(rho), _ptr(c), _stream(stream)))


def dpm_dd2_pks_destroy(pks):
    _check(lib().dpm_dd2_pks_destroy(pks))


# ---- layered domain decomposition (ball + concentric shells) ------------------------
def ml_params(center, radii, grids, K, KG, precision=DPM_PREC_FP32) -> dpm_ml_params:
    """radii: rho_1 .. rho_{L-1}, R; grids: (N, lo, hi) per sub-domain; K: degree per interface."""
    p = dpm_ml_params()
    L = len(radii)
    if not 2 <= L <= DPM_ML_MAX or len(grids) != L or len(K) != L - 1:
        raise ValueError("need 2 <= L <= 16 radii, L grids and L - 1 interface degrees")
    for t in range(3):
        p.center[t] = center[t]
    p.L = L
    for l in range(L):
        p.radii[l] = radii[l]
        p.N[l], p.lo[l], p.hi[l] = grids[l]
    for m, k in enumerate(K):
        p.K[m] = k
    p.KG, p.precision = KG, precision
    return p


def dpm_ml_build(ctx, params: dpm_ml_params, sigma, stream=None):
    h = C.c_void_p()
    _check(lib().dpm_ml_build(ctx, C.byref(params), sigma, C.byref(h), _stream(stream)))
    return h


def dpm_ml_get_info(ml) -> dpm_ml_info:
    info = dpm_ml_info()
    _check(lib().dpm_ml_get_info(ml, C.byref(info)))
    return info


def dpm_ml_matrix(ml, A, stream=None):
    _check(lib().dpm_ml_matrix(ml, _ptr(A), _stream(stream)))


def dpm_ml_solve(ml, fs, us, neumann=None, coeffs=None, stream=None):
    """fs, us: lists of device tensors, one per sub-domain."""
    fa = (C.c_void_p * len(fs))(*[_ptr(f) for f in fs])
    ua = (C.c_void_p * len(us))(*[_ptr(u) for u in us])
    _check(lib().dpm_ml_solve(ml, fa, _ptr(neumann), ua, _ptr(coeffs), _stream(stream)))


def dpm_ml_destroy(ml):
    _check(lib().dpm_ml_destroy(ml))


def dpm_ml_pks_create(ctx, params: dpm_ml_params, chi, dt_max, dt_mode, rebuild, clamp, rho0, c0, stream=None):
    h = C.c_void_p()
    g0, g1 = make_gaussian(rho0), make_gaussian(c0)
    _check(lib().dpm_ml_pks_create(ctx, C.byref(params), chi, dt_max, dt_mode, rebuild, clamp, C.byref(g0),
                                   C.byref(g1), C.byref(h), _stream(stream)))
    return h


def dpm_ml_pks_step(pks, nsteps=1, want_stats=True, stream=None):
    st = dpm_pks_stats()
    _check(lib().dpm_ml_pks_step(pks, nsteps, C.byref(st) if want_stats else None, _stream(stream)))
    return st if want_stats else None


def dpm_ml_pks_set_graph(pks, on=True, stream=None):
    _check(lib().dpm_ml_pks_set_graph(pks, 1 if on else 0, _stream(stream)))


def dpm_ml_pks_get_state(pks, l, rho, c, stream=None):
    _check(lib().dpm_ml_pks_get_state(pks, l, _ptr(rho), _ptr(c), _stream(stream)))


def dpm_ml_pks_destroy(pks):
    _check(lib().dpm_ml_pks_destroy(pks))
