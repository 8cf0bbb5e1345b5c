"""The bundle cache: projectors are rebuilt on load bit for bit; the SCF potential is shared
by every momentum transfer of one crystal."""
import os
import tempfile

import numpy as np

import workloads as w
from workloads import groundstate as gs


def test_bundle_round_trip_rebuilds_projectors():
    b = w.get_bundle(w.config_tiny(kb=True))
    with tempfile.TemporaryDirectory() as d:
        path = os.path.join(d, "b.npz")
        gs.save_bundle(b, path)
        assert "beta_kq" not in np.load(path).files
        r = gs.load_bundle(b.spec, path)
    for a, c in zip(b.beta_kq, r.beta_kq):
        assert np.array_equal(a, c)
    for f in ("u_k", "u_kq", "miller_kq"):
        for a, c in zip(getattr(b, f), getattr(r, f)):
            assert np.array_equal(a, c)
    assert np.array_equal(b.vloc_r, r.vloc_r) and np.array_equal(b.eps_k, r.eps_k)


def test_scf_shared_across_q():
    s1 = w.config_tiny()
    s2 = w.config_tiny()
    s2.q_cart = s2.q_cart * 1.7
    b1, b2 = w.get_bundle(s1), w.get_bundle(s2)
    assert np.array_equal(b1.vloc_r, b2.vloc_r)
    assert not np.array_equal(b1.miller_kq[0], b2.miller_kq[0]) or not np.allclose(b1.u_kq[0], b2.u_kq[0])
