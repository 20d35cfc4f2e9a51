"""ctypes binding of include/hm.h: argument marshalling only.

Loads paper_2606_02169_gb300/_build/libhm.so (built by build.py). There is no
fallback: if the library is missing or fails to load, every call raises.
"""
from __future__ import annotations

import ctypes
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "_build", "libhm.so")

HM_SPIN, HM_BOSON = 0, 1
OPS = {"I": 0, "Sz": 1, "Sx": 2, "Sy": 3, "Sp": 4, "Sm": 5, "Sz2": 6, "Sp2": 7, "Sm2": 8,
       "N": 9, "a": 10, "adag": 11}
HM_F64, HM_F32, HM_C128, HM_C64 = 0, 1, 2, 3

HM_OK = 0
HM_ERR_INVALID_ARG = -1
HM_ERR_OVERFLOW = -2
HM_ERR_ALIAS = -3
HM_ERR_COMPLEX_REQUIRED = -4
HM_ERR_NOT_HERMITIAN = -5
HM_ERR_CUDA = -6
HM_ERR_OOM = -7
HM_ERR_TIMEOUT = -8
HM_ERR_UNSUPPORTED = -9
HM_ERR_TOO_LARGE = -10
HM_LANCZOS_BREAKDOWN = 1

# Every exported entry point and its signature; tests check that the library
# exports exactly these names.
EXPORTS = [
    "hm_create", "hm_create_sector", "hm_set_coefficients", "hm_dim", "hm_num_terms", "hm_apply", "hm_apply_ex",
    "hm_apply_adjoint", "hm_lanczos", "hm_batch_create", "hm_batch_apply", "hm_tune",
    "hm_tuned_config", "hm_destroy", "hm_strerror", "hm_last_error", "hm_plan_export", "hm_coupling_gradients_static",
    "hm_evolve", "hm_krylov_coefficients", "hm_device_status",
]


class hm_site(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int32), ("dim", ctypes.c_int32)]


class hm_term(ctypes.Structure):
    _fields_ = [("site_i", ctypes.c_int32), ("op_i", ctypes.c_int32), ("site_j", ctypes.c_int32),
                ("op_j", ctypes.c_int32), ("coef", ctypes.c_double)]


class HmError(RuntimeError):
    def __init__(self, code, where, detail=""):
        self.code = code
        super().__init__(f"{where}: {_strerror(code)} ({code}){': ' + detail if detail else ''}")


_lib = None


def _strerror(code):
    if _lib is None:
        return "hm library not loaded"
    return _lib.hm_strerror(code).decode()


def load(path: str = LIB_PATH):
    """Load libhm.so once; raise if it is missing (no CPU fallback exists)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise ImportError(f"CUDA library not built: {path} is missing "
                          "(run `python -c \"import __graft_entry__ as g; g.build()\"`)")
    lib = ctypes.CDLL(path)
    vp, i32, i64, dp = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.POINTER(ctypes.c_double)
    H = ctypes.c_void_p
    lib.hm_create.argtypes = [ctypes.POINTER(hm_site), i32, ctypes.POINTER(hm_term), i32,
                              ctypes.POINTER(H)]
    lib.hm_create_sector.argtypes = [ctypes.POINTER(hm_site), i32, ctypes.POINTER(hm_term), i32, i64,
                                     ctypes.POINTER(H)]
    lib.hm_set_coefficients.argtypes = [H, dp]
    lib.hm_dim.argtypes = [H]
    lib.hm_dim.restype = i64
    lib.hm_num_terms.argtypes = [H]
    lib.hm_num_terms.restype = i32
    lib.hm_apply.argtypes = [H, vp, vp, i64, ctypes.c_int, vp]
    lib.hm_apply_ex.argtypes = [H, vp, vp, i64, ctypes.c_int, i32, i32, vp]
    lib.hm_apply_adjoint.argtypes = [H, vp, vp, vp, vp, i64, ctypes.c_int, vp]
    lib.hm_lanczos.argtypes = [H, vp, i32, ctypes.c_int, i32, dp, dp, ctypes.POINTER(i32), vp, dp, vp]
    lib.hm_batch_create.argtypes = [ctypes.POINTER(H), i32, ctypes.POINTER(H)]
    lib.hm_batch_apply.argtypes = [H, ctypes.POINTER(vp), ctypes.POINTER(vp), i64, ctypes.c_int, vp]
    lib.hm_tune.argtypes = [H, i64, ctypes.c_int, vp]
    lib.hm_tuned_config.argtypes = [H, i64, ctypes.c_int, ctypes.POINTER(i32)]
    lib.hm_evolve.argtypes = [H, vp, vp, ctypes.c_double, i32, i32, i32, ctypes.c_int, dp, vp]
    lib.hm_krylov_coefficients.argtypes = [dp, dp, i32, ctypes.c_double, ctypes.c_double, dp]
    lib.hm_destroy.argtypes = [H]
    lib.hm_device_status.argtypes = [ctypes.POINTER(i32), i32]
    lib.hm_plan_export.argtypes = [ctypes.POINTER(hm_site), i32, ctypes.POINTER(hm_term), i32, i32,
                                   ctypes.c_char_p, i64, ctypes.POINTER(i64)]
    lib.hm_plan_export.restype = ctypes.c_int
    lib.hm_strerror.argtypes = [ctypes.c_int]
    lib.hm_strerror.restype = ctypes.c_char_p
    lib.hm_last_error.restype = ctypes.c_char_p
    for name in ("hm_create", "hm_create_sector", "hm_set_coefficients", "hm_apply", "hm_apply_ex", "hm_apply_adjoint",
                 "hm_lanczos", "hm_batch_create", "hm_batch_apply", "hm_tune", "hm_tuned_config",
                 "hm_destroy", "hm_evolve", "hm_krylov_coefficients", "hm_device_status"):
        getattr(lib, name).restype = ctypes.c_int
    _lib = lib
    return lib


def krylov_coefficients(alpha, beta, tau, nu=1.0):
    """Host-only: c = nu exp(-i tau T) e_1 for T = tridiag(beta, alpha, beta)
    (the combination hm_evolve applies to its Krylov basis), complex array."""
    import numpy as np
    lib = load()
    m = len(alpha)
    a = (ctypes.c_double * m)(*[float(v) for v in alpha])
    b = (ctypes.c_double * max(1, m - 1))(*[float(v) for v in beta[: m - 1]])
    c = (ctypes.c_double * (2 * m))()
    check(lib.hm_krylov_coefficients(a, b if m > 1 else None, m, float(tau), float(nu), c), "hm_krylov_coefficients")
    v = np.frombuffer(c, dtype=np.float64).copy()
    return v[0::2] + 1j * v[1::2]


def plan_export(sites, terms, which=0):
    """Host-only: the plan tables hm_create would upload, as a dict."""
    import json
    lib = load()
    ss = [(HM_SPIN if k in ("spin", HM_SPIN) else HM_BOSON, int(d)) for k, d in sites]
    ts = [(int(i), OPS[oi] if isinstance(oi, str) else int(oi), int(j),
           OPS[oj] if isinstance(oj, str) else int(oj), float(c)) for i, oi, j, oj, c in terms]
    cs = (hm_site * len(ss))(*[hm_site(k, d) for k, d in ss])
    ct = (hm_term * max(1, len(ts)))(*[hm_term(*t) for t in ts])
    n = ctypes.c_int64(0)
    check(lib.hm_plan_export(cs, len(ss), ct, len(ts), which, None, 0, ctypes.byref(n)), "hm_plan_export")
    buf = ctypes.create_string_buffer(n.value)
    check(lib.hm_plan_export(cs, len(ss), ct, len(ts), which, buf, n.value, ctypes.byref(n)), "hm_plan_export")
    return json.loads(buf.value.decode())


def device_status(clear=True):
    """Status bits of the current device's kernels since the last clear
    (bit 0: a bounded wait of the staged apply kernel gave up). Synchronises."""
    lib = load()
    v = ctypes.c_int32(0)
    check(lib.hm_device_status(ctypes.byref(v), 1 if clear else 0), "hm_device_status")
    return v.value


def check(rc, where):
    if rc < 0:
        raise HmError(rc, where, _lib.hm_last_error().decode())
    return rc
