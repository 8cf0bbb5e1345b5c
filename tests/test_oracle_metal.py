"""Pins of the oracle's metallic form (Sec. 2.6: the projector on empty states redefined,
fractional occupations as weights in the band sums).

The closed form is the Lindhard transition sum of a free-electron gas with smeared
occupations, written from its definition over every pair of plane waves,
    chi0(z) = (2/Omega)(1/N_k) sum_k sum_G (f(k+G) - f(k+Q+G)) / (z - (|k+Q+G|^2 - |k+G|^2)/2),
which uses none of the oracle's operator code (no projector, no metric, no split of the pairs
into directions).  Every orbital is one plane wave, the density is uniform and the response
diagonal in G, so the head obeys the scalar Dyson equation with the Hartree (+ ALDA) kernel.
The mesh is Gamma-centred with Q on it, so that k -> -k-Q maps it onto itself and the
anti-resonant half of the recursion's response is the sum's own de-excitation terms.

With occupations between 0 and 1 on several levels at k and at k+Q, a transition between two
partially occupied levels enters with weight f_v - f_m; a dropped metric, a dropped band
weight or a wrong projector weight all move the spectral weight at some transition energy.
"""
import numpy as np
import pytest

import workloads as w
from workloads.groundstate import build_bundle, smeared
from oracle import lanczos, spectrum, xc
from oracle.liouvillian import System, metal_weights


def _metal_gas(approx):
    """Simple-cubic gas, 2 electrons per cell, 8 plane-wave bands, Gaussian smearing 0.04 Ry,
    4x4x4 mesh, Q = b_1/4: 206 of the 296 open transitions join two partially occupied levels."""
    spec = w.config_free_electron(nk=4, qfrac=0.25)
    spec.nbnd, spec.electrons, spec.smearing_ry, spec.approx = 8, 2.0, 0.04, approx
    return build_bundle(spec)


def _lindhard_pairs(b):
    """(f_a - f_b, Delta) of every plane-wave pair k+G -> k+Q+G with different occupations."""
    spec = b.spec
    sig, q = spec.smearing_ry / 2, spec.q_cart
    out = []
    for k in b.kcart:
        at_kq = set(map(tuple, w.sphere(k + q, spec.bvec, spec.ecut_ry)))
        for m in w.sphere(k, spec.bvec, spec.ecut_ry):
            if tuple(m) not in at_kq:
                continue
            g = m @ spec.bvec
            ea, eb = 0.5 * np.dot(k + g, k + g), 0.5 * np.dot(k + q + g, k + q + g)
            fa, fb = smeared(np.array([ea, eb]), b.fermi, sig)
            if fa != fb:
                out.append((fa - fb, eb - ea))
    return np.array(out)


def _frequencies():
    wev = np.linspace(0.0, 12.0, 241)
    eta = 0.15
    return wev, eta, (wev + 1j * eta) / w.HA_EV


def test_metal_gas_occupations():
    """The smearing counts the electrons, and the gas has the partially occupied levels the
    other pins need at k and at k+Q."""
    b = _metal_gas("ipa")
    assert np.sum(b.occ_k) * 2 / b.nks == pytest.approx(2.0, rel=1e-12)
    part = (b.occ_k > 0) & (b.occ_k < 1)
    assert part.sum() >= 100 and ((b.occ_kq > 0) & (b.occ_kq < 1)).sum() >= 100
    assert b.gap_min > 0
    pairs = _lindhard_pairs(b)
    assert len(pairs) == 296


@pytest.mark.parametrize("flavour", ["ph", "nh"])
@pytest.mark.parametrize("approx", ["ipa", "rpa", "tddft"])
def test_lindhard_sum_of_metallic_gas(approx, flavour):
    """eps^-1 from the recursion over its whole Krylov space (four distinct transition
    energies: eight steps) equals the Dyson form on the Lindhard sum."""
    b = _metal_gas(approx)
    spec = b.spec
    pairs = _lindhard_pairs(b)
    assert len(np.unique(np.round(np.abs(pairs[:, 1]), 9))) == 4
    co = lanczos.run(System(b, approx), 8, flavour)
    wev, eta, z = _frequencies()
    chi0 = 2.0 / spec.omega / b.nks * np.sum(pairs[None, :, 0] / (z[:, None] - pairs[None, :, 1]), axis=1)
    q2 = float(spec.q_cart @ spec.q_cart)
    n = spec.nelec / spec.omega
    kern = {"ipa": 0.0, "rpa": 4 * np.pi / q2, "tddft": 4 * np.pi / q2 + float(xc.fxc(np.array(n)))}[approx]
    want = 1.0 + 4 * np.pi / q2 * chi0 / (1.0 - kern * chi0)
    _, eps_inv, _ = spectrum.spectrum(co.beta, co.gamma, co.z, spec.omega, spec.q_cart, wev, eta)
    assert np.max(np.abs(eps_inv - want)) < 1e-11 * np.max(np.abs(want - 1.0))


def test_kept_transitions_have_positive_metric_energy():
    """Each kept transition v -> m (c_mv > 0) is an eigenvector of D with a positive value of
    (x, D x) / (x, x) in the metric: the pseudo-Hermitian recursion's metric is positive.
    (Giving every pair both directions, weights f_v (1 - f_m), would keep some with a
    negative energy.)"""
    b = _metal_gas("ipa")
    sysm = System(b, "ipa")
    seen = 0
    for k in range(b.nks):
        c = sysm.c[k]
        for v in range(b.spec.nbnd):
            for m in range(b.spec.nbnd):
                if c[m, v] <= 0:
                    continue
                x = [np.zeros((b.spec.nbnd, len(b.miller_kq[k])), dtype=np.complex128)]
                x[0][v] = b.u_kq[k][m]
                dx = sysm.apply_d(x, [k])
                num, den = sysm.inner_part(x, dx, [k]).real, sysm.inner_part(x, x, [k]).real
                delta = b.eps_kq[k][m] - b.eps_k[k][v]
                assert den > 0 and num / den == pytest.approx(delta, rel=1e-10, abs=1e-12)
                assert delta > 0
                seen += 1
    assert seen > 100


def test_projector_weights_by_hand():
    """c_mv = max(1 - f_m/f_v, 0): a full band m gives 0 for every v, an empty one 1, a band
    v with f_v = 0 gives 0, and tiny weights are dropped."""
    f_v = np.array([1.0, 0.5, 0.0, 0.25])
    f_m = np.array([1.0, 0.0, 0.5, 0.25 * (1 - 1e-8)])
    c = metal_weights(f_v, f_m)
    assert np.array_equal(c[0], [0.0, 0.0, 0.0, 0.0])
    assert np.array_equal(c[1], [1.0, 1.0, 0.0, 1.0])
    assert np.array_equal(c[2], [0.5, 0.0, 0.0, 0.0])
    assert c[3, 3] == 0.0 and c[3, 1] == pytest.approx(0.5 + 0.5e-8, rel=1e-12)


def test_full_occupations_reduce_to_the_insulator():
    """A bundle with every occupation 1 run through the metallic form gives the insulator's
    coefficients (c = 0 everywhere: P_{c,v} = P'_v = P_c, the metric the plain product)."""
    b = w.get_bundle(w.config_tiny())
    ins = lanczos.run(System(b, "tddft"), 20, "ph")
    b.occ_k = np.ones_like(b.eps_k)
    b.occ_kq = np.ones_like(b.eps_kq)
    sysm = System(b, "tddft")
    assert sysm.metal
    met = lanczos.run(sysm, 20, "ph")
    assert np.max(np.abs(met.beta - ins.beta)) < 1e-12 * np.max(ins.beta)
    assert np.max(np.abs(met.z - ins.z)) < 1e-12 * np.max(np.abs(ins.z))


@pytest.mark.parametrize("flavour", ["ph", "nh"])
def test_fsum_of_metallic_gas(flavour):
    """The f-sum rule (Sec. 2.1) holds for any occupations of a local Hamiltonian: the
    integral of omega (-Im eps^-1) is (pi/2) omega_p^2, omega_p^2 = 4 pi n, n = 2/Omega."""
    b = _metal_gas("rpa")
    spec = b.spec
    co = lanczos.run(System(b, "rpa"), 8, flavour)
    wev = np.linspace(0.0, 60.0, 30001)
    _, eps_inv, _ = spectrum.spectrum(co.beta, co.gamma, co.z, spec.omega, spec.q_cart, wev, 0.02)
    moment = spectrum.fsum_moment(wev, eps_inv)
    assert abs(moment / spectrum.fsum_expected(spec.nelec, spec.omega) - 1.0) < 5e-3
