"""Pins of the plane-wave/FFT conventions and the index maps."""
import itertools

import numpy as np

import workloads as w
from oracle import basis


def test_sphere_brute_force():
    s = w.config_small()
    k = np.array([0.25, 0.5, 0.75]) @ s.bvec + s.q_cart
    m = w.sphere(k, s.bvec, s.ecut_ry)
    ref = []
    for t in itertools.product(range(-8, 9), repeat=3):
        g = k + np.array(t) @ s.bvec
        if g @ g <= s.ecut_ry:
            ref.append(t)
    assert np.array_equal(m, np.array(sorted(ref), dtype=np.int32))


def test_grid_round_trip_and_parseval():
    rng = np.random.default_rng(1)
    s = w.config_small()
    m = w.sphere(np.zeros(3), s.bvec, s.ecut_ry)
    c = rng.normal(size=(3, len(m))) + 1j * rng.normal(size=(3, len(m)))
    psi = basis.to_grid(c, m, s.nfft)
    assert np.allclose(basis.to_sphere(psi, m, s.nfft), c, atol=1e-13)
    # (1/N^3) sum_r |psi|^2 = sum_G |c|^2
    assert np.allclose(np.mean(np.abs(psi) ** 2, axis=(1, 2, 3)), np.sum(np.abs(c) ** 2, axis=1), rtol=1e-13)


def test_grid_plane_wave_definition():
    # a single coefficient at Miller m gives exp(2 pi i m.j / N) at grid point j
    n = 6
    m = np.array([[1, -2, 3]], dtype=np.int32)
    psi = basis.to_grid(np.array([1.0 + 0j]), m, n)
    j = (2, 4, 5)
    assert np.isclose(psi[j], np.exp(2j * np.pi * (1 * 2 - 2 * 4 + 3 * 5) / n), atol=1e-14)


def test_intersection_map_brute_force():
    s = w.config_small()
    kc = np.array([0.5, 0.25, 0.0]) @ s.bvec
    mk = w.sphere(kc, s.bvec, s.ecut_ry)
    mq = w.sphere(kc + s.q_cart, s.bvec, s.ecut_ry)
    mp = basis.intersection_map(mk, mq)
    for i, g in enumerate(mq):
        hits = np.where((mk == g).all(axis=1))[0]
        assert mp[i] == (hits[0] if len(hits) else -1)
    assert (mp >= 0).sum() > 0.8 * len(mq)


def test_columns_cover_sphere():
    s = w.config_small()
    m = w.sphere(np.zeros(3), s.bvec, s.ecut_ry)
    cols = basis.columns(m)
    assert sum(c[3] for c in cols) == len(m)
    for m1, m2, st, cnt in cols:
        seg = m[st:st + cnt]
        assert (seg[:, 0] == m1).all() and (seg[:, 1] == m2).all()
        assert (np.diff(seg[:, 2]) == 1).all()       # contiguous m3 runs
