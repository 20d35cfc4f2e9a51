"""CPU-only checks of the C ABI: the library builds for sm_103a, loads, exports
every function include/hm.h declares, and rejects bad plans on the host (no
kernel is launched; no GPU is needed)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    from paper_2606_02169_gb300 import build as B
    B.build()
    from paper_2606_02169_gb300 import _capi
    return _capi.load()


def declared_functions():
    src = open(os.path.join(ROOT, "include", "hm.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"^\s*(?:const\s+)?[A-Za-z_][A-Za-z0-9_]*\s*\*?\s*(hm_[a-z_0-9]+)\s*\(",
                                 src, flags=re.M)))


def test_header_declares_the_boundary():
    names = declared_functions()
    for must in ["hm_create", "hm_set_coefficients", "hm_dim", "hm_apply", "hm_apply_adjoint",
                 "hm_lanczos", "hm_batch_create", "hm_batch_apply", "hm_tune", "hm_destroy",
                 "hm_strerror"]:
        assert must in names, must


def test_library_exports_every_declared_symbol(lib):
    from paper_2606_02169_gb300 import _capi
    names = declared_functions()
    assert sorted(names) == sorted(_capi.EXPORTS)
    for n in names:
        assert hasattr(lib, n), n


def test_strerror_names_every_code(lib):
    from paper_2606_02169_gb300 import _capi as C
    for code in [C.HM_OK, C.HM_ERR_INVALID_ARG, C.HM_ERR_OVERFLOW, C.HM_ERR_ALIAS,
                 C.HM_ERR_COMPLEX_REQUIRED, C.HM_ERR_NOT_HERMITIAN, C.HM_ERR_CUDA, C.HM_ERR_OOM,
                 C.HM_ERR_TIMEOUT, C.HM_ERR_UNSUPPORTED, C.HM_ERR_TOO_LARGE, C.HM_LANCZOS_BREAKDOWN]:
        assert lib.hm_strerror(code).decode() != "unknown error"


def _create(lib, sites, terms):
    from paper_2606_02169_gb300 import _capi as C
    cs = (C.hm_site * len(sites))(*[C.hm_site(k, d) for k, d in sites])
    ts = (C.hm_term * max(1, len(terms)))(*[C.hm_term(*t) for t in terms])
    h = ctypes.c_void_p()
    rc = lib.hm_create(cs, len(sites), ts, len(terms), ctypes.byref(h))
    return rc, h


@pytest.mark.parametrize("sites,terms,code_name", [
    ([(0, 2), (0, 2)], [(0, 1, 0, 1, 1.0)], "HM_ERR_INVALID_ARG"),        # i == j
    ([(0, 2), (0, 2)], [(0, 9, -1, 0, 1.0)], "HM_ERR_INVALID_ARG"),       # boson op on a spin
    ([(1, 4), (0, 2)], [(0, 1, -1, 0, 1.0)], "HM_ERR_INVALID_ARG"),       # spin op on a boson
    ([(0, 1)], [], "HM_ERR_INVALID_ARG"),                                  # dim < 2
    ([(2, 2)], [], "HM_ERR_INVALID_ARG"),                                  # unknown kind
    ([(0, 2)], [(3, 1, -1, 0, 1.0)], "HM_ERR_INVALID_ARG"),               # site out of range
    ([(0, 2)], [(0, 1, -1, 0, float("nan"))], "HM_ERR_INVALID_ARG"),      # non-finite coef
    ([(0, 70000)], [], "HM_ERR_UNSUPPORTED"),                              # dim too large
])
def test_invalid_plans_are_rejected_on_host(lib, sites, terms, code_name):
    from paper_2606_02169_gb300 import _capi as C
    rc, h = _create(lib, sites, terms)
    assert rc == getattr(C, code_name)
    assert not h.value
    assert len(lib.hm_last_error().decode()) > 0


def test_dimension_overflow_rejected(lib):
    from paper_2606_02169_gb300 import _capi as C
    rc, _ = _create(lib, [(0, 2)] * 62 + [(0, 3)], [])
    assert rc == C.HM_ERR_OVERFLOW


def test_null_arguments(lib):
    from paper_2606_02169_gb300 import _capi as C
    assert lib.hm_create(None, 1, None, 0, None) == C.HM_ERR_INVALID_ARG
    assert lib.hm_apply(None, None, None, 1, 0, None) == C.HM_ERR_INVALID_ARG
    assert lib.hm_destroy(None) == C.HM_ERR_INVALID_ARG
    assert lib.hm_dim(None) < 0
    # complex dtypes map onto the same checks; hm_evolve validates before any device call
    assert lib.hm_apply(None, None, None, 1, C.HM_C128, None) == C.HM_ERR_INVALID_ARG
    assert lib.hm_evolve(None, None, None, 0.1, 10, 1, 0, C.HM_C128, None, None) == C.HM_ERR_INVALID_ARG
    assert lib.hm_evolve(None, None, None, 0.1, 10, 1, 0, C.HM_F64, None, None) == C.HM_ERR_INVALID_ARG
    assert lib.hm_evolve(None, None, None, float("nan"), 10, 1, 0, C.HM_C64, None, None) == C.HM_ERR_INVALID_ARG
    assert lib.hm_evolve(None, None, None, 0.1, 0, 1, 0, C.HM_C64, None, None) == C.HM_ERR_INVALID_ARG


def test_product_path_has_no_fallback(tmp_path):
    """Without the built library the binding raises instead of computing."""
    from paper_2606_02169_gb300 import _capi
    with pytest.raises(ImportError):
        saved = _capi._lib
        _capi._lib = None
        try:
            _capi.load(str(tmp_path / "missing.so"))
        finally:
            _capi._lib = saved
