"""Host logic of hm_evolve, on the CPU: the Krylov propagator coefficients
c = nu exp(-i tau T) e_1 of a real symmetric tridiagonal T (what the device
combines its Krylov basis with) against scipy.linalg.expm of the same T, for
Krylov sizes from 1 to the 128 limit, a split T (beta = 0), large tau |T|,
and the argument checks."""
import numpy as np
import pytest


@pytest.fixture(scope="module")
def capi():
    from paper_2606_02169_gb300 import build as B
    B.build()
    from paper_2606_02169_gb300 import _capi
    _capi.load()
    return _capi


def _ref(a, b, tau, nu):
    from scipy.linalg import expm
    m = len(a)
    T = np.diag(a) + np.diag(b[: m - 1], 1) + np.diag(b[: m - 1], -1)
    e1 = np.zeros(m)
    e1[0] = 1.0
    return nu * (expm(-1j * tau * T) @ e1)


@pytest.mark.parametrize("m", [1, 2, 5, 17, 40, 128])
@pytest.mark.parametrize("tau", [0.05, 0.7, -1.3])
def test_coefficients_match_the_matrix_exponential(capi, m, tau):
    rng = np.random.default_rng(m)
    a = rng.normal(size=m) * 3.0
    b = np.abs(rng.normal(size=max(m - 1, 0))) + 0.1
    nu = 2.5
    c = capi.krylov_coefficients(a, b, tau, nu)
    ref = _ref(a, b, tau, nu)
    assert np.allclose(c, ref, rtol=0, atol=1e-12 * nu)
    assert abs(np.linalg.norm(c) - nu) < 1e-12 * nu           # exp(-i tau T) is unitary


def test_split_tridiagonal_keeps_the_first_block(capi):
    # beta_1 = 0: e_1 never leaves the leading 2x2 block
    a = np.array([0.3, -1.1, 2.0, 0.5])
    b = np.array([0.8, 0.0, 1.5])
    c = capi.krylov_coefficients(a, b, 0.9)
    assert np.allclose(c, _ref(a, b, 0.9, 1.0), atol=1e-13)
    assert np.abs(c[2:]).max() == 0.0


def test_large_phase(capi):
    rng = np.random.default_rng(3)
    a = rng.normal(size=30) * 50
    b = np.abs(rng.normal(size=29)) * 20
    assert np.allclose(capi.krylov_coefficients(a, b, 3.0), _ref(a, b, 3.0, 1.0), atol=1e-10)


def test_invalid_arguments(capi):
    with pytest.raises(capi.HmError):
        capi.krylov_coefficients([], [], 0.1)
    with pytest.raises(capi.HmError):
        capi.krylov_coefficients([0.0] * 129, [1.0] * 128, 0.1)
    with pytest.raises(capi.HmError):
        capi.krylov_coefficients([np.nan, 1.0], [1.0], 0.1)
