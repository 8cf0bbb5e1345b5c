"""Coefficient files (the recursion-to-spectrum hand-off of Secs. 3.2-3.3): exact round trip
of oracle coefficients, and the spectrum from the file equal to the spectrum from memory."""
import numpy as np
import pytest

import workloads as w
from oracle import lanczos, spectrum
from oracle.liouvillian import System
from paper_2111_06623_gb300 import coefficients


@pytest.mark.parametrize("flavour", ["ph", "nh"])
def test_round_trip_is_exact(tmp_path, flavour):
    b = w.get_bundle(w.config_tiny())
    co = lanczos.run(System(b, "rpa"), 30, flavour)
    p = tmp_path / "chain.coef"
    coefficients.save(p, co.beta, co.gamma, co.z, b.spec.omega, b.spec.q_cart, flavour=flavour, approx="rpa")
    got = coefficients.load(p)
    assert np.array_equal(got["beta"], co.beta)
    assert np.array_equal(got["gamma"], co.gamma) and np.array_equal(got["z"], co.z)
    assert got["omega_cell"] == b.spec.omega and np.array_equal(got["q_cart"], b.spec.q_cart)
    assert (got["flavour"], got["approx"]) == (flavour, "rpa")
    wev = np.linspace(0.0, 40.0, 81)
    a = spectrum.spectrum(co.beta, co.gamma, co.z, b.spec.omega, b.spec.q_cart, wev, 0.1)
    c = spectrum.spectrum(got["beta"], got["gamma"], got["z"], got["omega_cell"], got["q_cart"], wev, 0.1)
    for x, y in zip(a, c):
        assert np.array_equal(x, y)


def test_rejects_malformed(tmp_path):
    with pytest.raises(ValueError):
        coefficients.save(tmp_path / "a", [1.0, 2.0], [1.0], [0.0, 1.0], 1.0, [0.1, 0, 0])
    with pytest.raises(ValueError):
        coefficients.save(tmp_path / "b", [1.0], [1.0], [0.0], 1.0, [0.1, 0, 0], flavour="p h")
    (tmp_path / "c").write_text("# something else\n0 1 1 0 0 0\n")
    with pytest.raises(ValueError):
        coefficients.load(tmp_path / "c")
