"""Free-electron pins of the oracle (V = 0): the plasmon pole of a uniform gas and the
Lindhard transition sum, both closed forms that use none of the oracle's operator code.

With V = 0 every orbital is a single plane wave, so the ground-state density is uniform and
a transition from k+G_v to k+Q+G_c carries density only at wave vector Q + (G_c - G_v): the
response is diagonal in G.  Its head therefore obeys the scalar Dyson equation of a uniform
system (Eq. 5 with the kernel of Eqs. 13 and 27, f_xc(n) constant under ALDA)
    chi = chi0 / (1 - (4 pi/|Q|^2 + f_xc) chi0),      eps^-1 = 1 + (4 pi/|Q|^2) chi,
with chi0 the Lindhard sum over the occupied plane waves (spin 2, weights 1/N_k)
    chi0(z) = (4/Omega)(1/N_k) sum_k Delta_k / (z^2 - Delta_k^2),
    Delta_k = |k+Q|^2/2 - |k|^2/2.
With the single k-point Gamma this is a plasmon pole,
    eps^-1(z) = 1 + omega_p^2 / (z^2 - Omega_pl^2),
    Omega_pl^2 = (Q^2/2)^2 + omega_p^2 + Q^2 n f_xc,   omega_p^2 = 4 pi n.

Occupations: one plane wave (G = 0) per k-point, k near Gamma, and Q = 0.75 b_1 past the
zone boundary, so that the lowest plane wave at k+Q is k+Q-b_1 and every head transition
k -> k+Q is open with a positive energy (D > 0, as the pseudo-Hermitian recursion needs).
The metallic gas (smeared occupations, Sec. 2.6) is pinned in test_oracle_metal.py.
"""
import numpy as np
import pytest

import workloads as w
from oracle import lanczos, spectrum, xc
from oracle.liouvillian import System

QFRAC = 0.75
# k-points in units of the reciprocal vectors, in +/- pairs (a current-free ground state);
# distinct k.Q, so the head transitions have distinct energies
K_SET = np.array([[0.02, 0.04, -0.03], [0.05, -0.01, 0.02], [0.08, 0.03, 0.05]])
K_SET = np.concatenate([K_SET, -K_SET])


def _gas(kfrac, approx, qfrac=QFRAC):
    """A ground-state bundle of plane waves: at k the plane wave G = 0, at k+Q the lowest one."""
    spec = w.config_free_electron(nk=1, qfrac=qfrac)
    spec.approx = approx
    spec.kmesh = (len(kfrac), 1, 1)
    bvec = spec.bvec
    kcart = np.asarray(kfrac, dtype=np.float64) @ bvec

    def lowest(k):
        mil = w.sphere(k, bvec, spec.ecut_ry)
        kg = k + mil @ bvec
        e = 0.5 * np.einsum("ij,ij->i", kg, kg)
        order = np.argsort(e)
        assert e[order[1]] - e[order[0]] > 1e-3          # the occupied level is not degenerate
        c = np.zeros((1, len(mil)), dtype=np.complex128)
        c[0, order[0]] = 1.0
        return mil, e, order[0], c

    mk, mkq, uk, ukq, ek, ekq = [], [], [], [], [], []
    for k in kcart:
        m0, e0, i0, c0 = lowest(k)
        m1, e1, i1, c1 = lowest(k + spec.q_cart)
        assert tuple(m0[i0]) == (0, 0, 0) and tuple(m1[i1]) == (-1, 0, 0)
        assert np.min(np.delete(e1, i1)) - e0[i0] > 0.05    # every transition energy positive
        mk.append(m0), mkq.append(m1), uk.append(c0), ukq.append(c1)
        ek.append([e0[i0]]), ekq.append([e1[i1]])
    n = spec.nfft
    return w.Bundle(spec=spec, kfrac=np.asarray(kfrac, dtype=np.float64), kcart=kcart,
                    miller_k=mk, miller_kq=mkq, u_k=uk, u_kq=ukq,
                    eps_k=np.array(ek), eps_kq=np.array(ekq),
                    vloc_r=np.zeros((n, n, n)), rho_r=np.full((n, n, n), spec.nelec / spec.omega),
                    beta_kq=[np.zeros((0, len(m)), dtype=np.complex128) for m in mkq], dij=np.zeros(0))


def _frequencies():
    wev = np.linspace(0.0, 12.0, 241)
    eta = 0.15
    return wev, eta, (wev + 1j * eta) / w.HA_EV


@pytest.mark.parametrize("flavour", ["ph", "nh"])
@pytest.mark.parametrize("approx", ["rpa", "tddft"])
def test_plasmon_pole_of_uniform_gas(approx, flavour):
    """Gamma only: the loss function is one pole at Omega_pl^2 = (Q^2/2)^2 + 4 pi n (+ Q^2 n f_xc
    under ALDA), with strength omega_p^2 = 4 pi n; two steps span the whole Krylov space."""
    b = _gas(np.zeros((1, 3)), approx)
    spec = b.spec
    sys = System(b, approx)
    co = lanczos.run(sys, 2, flavour)
    q2 = float(spec.q_cart @ spec.q_cart)
    n = spec.nelec / spec.omega
    fxc = float(xc.fxc(np.array(n))) if approx == "tddft" else 0.0
    wp2 = 4 * np.pi * n
    pole2 = (q2 / 2) ** 2 + wp2 + q2 * n * fxc
    # the 2x2 tridiagonal's eigenvalues are +-sqrt(beta_2 gamma_2)
    assert abs((co.beta[1] * co.gamma[1]).real / pole2 - 1.0) < 1e-12
    wev, eta, z = _frequencies()
    _, eps_inv, _ = spectrum.spectrum(co.beta, co.gamma, co.z, spec.omega, spec.q_cart, wev, eta)
    want = 1.0 + wp2 / (z ** 2 - pole2)
    assert np.max(np.abs(eps_inv - want)) < 1e-11 * np.max(np.abs(want - 1.0))
    # the loss peak sits on the pole (within the 0.05 eV grid step)
    assert abs(wev[np.argmax(spectrum.loss(eps_inv))] - np.sqrt(pole2) * w.HA_EV) <= 0.05


@pytest.mark.parametrize("flavour", ["ph", "nh"])
@pytest.mark.parametrize("approx", ["ipa", "rpa", "tddft"])
def test_lindhard_head_of_plane_wave_gas(approx, flavour):
    """Six k-points: eps^-1 from the recursion (run over the whole 2 N_k-dimensional Krylov
    space) equals the scalar Dyson form built on the Lindhard transition sum."""
    b = _gas(K_SET, approx)
    spec = b.spec
    sys = System(b, approx)
    co = lanczos.run(sys, 2 * len(K_SET), flavour)
    q = spec.q_cart
    q2 = float(q @ q)
    kc = K_SET @ spec.bvec
    delta = 0.5 * np.einsum("ij,ij->i", kc + q, kc + q) - 0.5 * np.einsum("ij,ij->i", kc, kc)
    wev, eta, z = _frequencies()
    chi0 = 4.0 / spec.omega * np.mean(delta[None, :] / (z[:, None] ** 2 - delta[None, :] ** 2), axis=1)
    n = spec.nelec / spec.omega
    kern = {"ipa": 0.0, "rpa": 4 * np.pi / q2, "tddft": 4 * np.pi / q2 + float(xc.fxc(np.array(n)))}[approx]
    chi = chi0 / (1.0 - kern * chi0)
    want = 1.0 + 4 * np.pi / q2 * chi
    _, eps_inv, _ = spectrum.spectrum(co.beta, co.gamma, co.z, spec.omega, q, wev, eta)
    assert np.max(np.abs(eps_inv - want)) < 1e-10 * np.max(np.abs(want - 1.0))


def test_plasma_frequency_from_first_moment():
    """Thomas-Reiche-Kuhn in the free-electron limit: (4 pi/Q^2)(4/Omega)(y, D y) is the
    squared plasma frequency 4 pi n, exactly, for a current-free set of plane waves."""
    b = _gas(K_SET, "rpa")
    spec = b.spec
    sys = System(b, "rpa")
    y = sys.starting_vector()
    m1 = 4.0 / spec.omega * sys.inner(y, sys.apply_d(y)).real
    wp2 = 4 * np.pi / float(spec.q_cart @ spec.q_cart) * m1
    assert abs(wp2 / (4 * np.pi * spec.nelec / spec.omega) - 1.0) < 1e-12


@pytest.mark.parametrize("flavour", ["ph", "nh"])
@pytest.mark.parametrize("approx", ["rpa", "tddft"])
def test_fsum_integral_of_loss_function(approx, flavour):
    """The f-sum rule on the broadened loss function (Sec. 2.1): the integral of
    omega (-Im eps^-1) over 0..60 eV is (pi/2) omega_p^2.  Each pole pair +-Omega adds two
    Lorentzians whose logarithmic tails cancel, leaving an O(eta/Omega) error (~0.1 %)."""
    b = _gas(K_SET, approx)
    spec = b.spec
    sys = System(b, approx)
    co = lanczos.run(sys, 2 * len(K_SET), flavour)
    wev = np.linspace(0.0, 60.0, 30001)
    _, eps_inv, _ = spectrum.spectrum(co.beta, co.gamma, co.z, spec.omega, spec.q_cart, wev, 0.02)
    wha = wev / w.HA_EV
    f = wha * spectrum.loss(eps_inv)
    moment = float(np.sum(0.5 * (f[1:] + f[:-1]) * np.diff(wha)))
    wp2 = 4 * np.pi * spec.nelec / spec.omega
    assert abs(moment / (0.5 * np.pi * wp2) - 1.0) < 5e-3
    # the oracle's f-sum printout is this trapezoid and this closed form
    assert spectrum.fsum_moment(wev, eps_inv) == pytest.approx(moment, rel=1e-14)
    assert spectrum.fsum_expected(spec.nelec, spec.omega) == pytest.approx(0.5 * np.pi * wp2, rel=1e-15)
