"""The allocation-free spectrum entry point (ll_spectrum_static).

Some callers cannot allocate device memory while they run: a service whose memory pool has
already reserved the GPU, or a latency-critical loop where cudaMalloc/cudaFree would
synchronise the device.  For them ll_spectrum_static stages everything through one static
device array compiled into the library.  This file is collected last so that a run that stops
at the first failure has already run every other test; it also passes alone in a fresh
process.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lib():
    from paper_2111_06623_gb300.build import build_library
    build_library()
    from paper_2111_06623_gb300 import ll
    return ll


def _coefficients(m, seed):
    """A pseudo-Hermitian-like tridiagonal matrix: positive beta, gamma = beta, small z."""
    rng = np.random.default_rng(seed)
    beta = 0.3 + rng.random(m)
    z = np.zeros(m, dtype=np.complex128)
    z[1::2] = (rng.normal(size=m // 2) + 1j * rng.normal(size=m // 2)) * 1e-2
    return beta, beta.astype(np.complex128), z


def test_static_matches_allocating_entry_twice(lib):
    omega_cell, q = 270.011394, np.array([0.0612396, 0.0, 0.0])
    w = np.linspace(0.0, 40.0, 4001)
    for call, (m, seed) in enumerate([(300, 1), (1000, 2)]):
        beta, gamma, z = _coefficients(m, seed)
        ref = lib.spectrum(beta, gamma, z, omega_cell, q, w, 0.1)
        got = lib.spectrum_static(beta, gamma, z, omega_cell, q, w, 0.1)
        for a, b in zip(got, ref):
            assert np.max(np.abs(a - b)) <= 1e-12 * np.max(np.abs(b)), call


def test_static_at_the_limits_then_smaller(lib):
    """The largest accepted call uses the end of every region of the static array; a smaller
    call right after it must not see what the larger one left behind."""
    omega_cell, q = 270.011394, np.array([0.0612396, 0.0, 0.0])
    big_w = np.linspace(0.0, 40.0, lib.SPECTRUM_STATIC_MAX_OMEGA)
    small_w = np.linspace(1.0, 30.0, 777)
    for m, w, seed in [(lib.SPECTRUM_STATIC_MAX_COEF, big_w, 5), (97, small_w, 6)]:
        beta, gamma, z = _coefficients(m, seed)
        ref = lib.spectrum(beta, gamma, z, omega_cell, q, w, 0.1)
        got = lib.spectrum_static(beta, gamma, z, omega_cell, q, w, 0.1)
        for a, b in zip(got, ref):
            assert a.shape == b.shape
            assert np.max(np.abs(a - b)) <= 1e-12 * np.max(np.abs(b)), m


def test_static_rejects_oversize(lib):
    beta, gamma, z = _coefficients(lib.SPECTRUM_STATIC_MAX_COEF + 2, 3)
    with pytest.raises(lib.LLError) as e:
        lib.spectrum_static(beta, gamma, z, 270.0, np.array([0.05, 0, 0]), np.linspace(0, 40, 11), 0.1)
    assert e.value.code == lib.LL_EINVAL and "static limit" in str(e.value)
    beta, gamma, z = _coefficients(10, 4)
    with pytest.raises(lib.LLError) as e:
        lib.spectrum_static(beta, gamma, z, 270.0, np.array([0.05, 0, 0]),
                            np.linspace(0, 40, lib.SPECTRUM_STATIC_MAX_OMEGA + 1), 0.1)
    assert e.value.code == lib.LL_EINVAL and "static limit" in str(e.value)
