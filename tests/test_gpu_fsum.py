"""The f-sum printout (Sec. 2.1, the check of the post-processing in Sec. 3.3) on the GPU:
ll_fsum's trapezoid first moment of -Im eps^-1 against the oracle's on the same loss function,
and the rule itself on the free-electron gas (V = 0, a local potential: the moment is
(pi/2) omega_p^2 up to the O(eta/Omega) broadening error)."""
import numpy as np
import pytest

import workloads as w
from oracle import spectrum

from .helpers import chain_from_bundle
from .test_oracle_free_electron import K_SET, _gas

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lib():
    from paper_2111_06623_gb300.build import build_library
    build_library()
    from paper_2111_06623_gb300 import ll
    return ll


@pytest.mark.parametrize("approx", ["rpa", "tddft"])
def test_fsum_rule_free_electron_gas(lib, approx):
    b = _gas(K_SET, approx)
    ch = chain_from_bundle(b, approx=approx, flavour="ph", precision="fp64", max_steps=8)
    ch.lanczos(8)
    wev = np.linspace(0.0, 60.0, 30001)
    _, ei, _ = ch.spectrum(wev, 0.02)
    moment, expected = lib.fsum(wev, ei, b.spec.nelec, b.spec.omega)
    assert moment == pytest.approx(spectrum.fsum_moment(wev, ei), rel=1e-12)
    assert expected == pytest.approx(spectrum.fsum_expected(b.spec.nelec, b.spec.omega), rel=1e-14)
    assert abs(moment / expected - 1.0) < 5e-3


def test_fsum_printout_small_cell(lib):
    """With the non-local s channel the rule holds only approximately (Sec. 5 reports < 1 %
    for diamond); the printout matches the oracle's trapezoid on the same loss function."""
    b = w.get_bundle(w.config_small())
    ch = chain_from_bundle(b, max_steps=300)
    ch.lanczos(300)
    wev = np.linspace(0.0, 40.0, 4001)
    _, ei, _ = ch.spectrum(wev, 0.1)
    moment, expected = lib.fsum(wev, ei, b.spec.nelec, b.spec.omega)
    assert moment == pytest.approx(spectrum.fsum_moment(wev, ei), rel=1e-12)
    assert 0.5 < moment / expected < 1.5
    with pytest.raises(lib.LLError):
        lib.fsum(wev[:1], ei[:1], b.spec.nelec, b.spec.omega)
