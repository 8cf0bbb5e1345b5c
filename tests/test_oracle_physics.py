"""Pins of the oracle's Liouvillian, recursions and spectrum against results the
mathematics fixes independently of the oracle's own code path."""
import numpy as np
import pytest

import workloads as w
from oracle import casida, lanczos, spectrum
from oracle.liouvillian import System


@pytest.fixture(scope="module")
def tiny():
    return w.get_bundle(w.config_tiny())


def _rand_batch(sys, seed):
    rng = np.random.default_rng(seed)
    x = [rng.normal(size=(sys.nbnd, len(m))) + 1j * rng.normal(size=(sys.nbnd, len(m))) for m in sys.mkq]
    return sys.project_c(x)


@pytest.mark.parametrize("approx,flavour", [("ipa", "ph"), ("rpa", "nh"), ("tddft", "ph"), ("tddft", "nh")])
def test_lanczos_matches_casida(tiny, approx, flavour):
    """Full-Liouvillian diagonalisation in the explicit transition basis (dense H_{k+Q}
    eigenvectors, pair densities) against the recursion run past the space dimension."""
    sys = System(tiny, approx)
    ref = casida.Casida(sys)
    wgrid = np.linspace(0.0, 40.0, 201) / w.HA_EV
    eta = 0.1 / w.HA_EV
    co = lanczos.run(sys, 2 * ref.dim, flavour)
    got = spectrum.chi_lanczos(co.beta, co.gamma, co.z, wgrid, eta)
    want = ref.chi_ll(wgrid + 1j * eta)
    assert np.max(np.abs(got - want)) / np.max(np.abs(want)) < 1e-9


def test_independent_particle_transition_sum(tiny):
    """IPA: chi = (4/Omega) sum_{vck} w_k |<c_{k+Q}|e^{iQr}|v_k>|^2 2 Delta/((w+i eta)^2 - Delta^2) / 2,
    written from dense eigenvectors without the Casida matrix."""
    sys = System(tiny, "ipa")
    ref = casida.Casida(sys)
    wv = np.array([5.0, 12.0, 20.0]) / w.HA_EV + 1j * 0.1 / w.HA_EV
    direct = np.array([np.sum(np.abs(ref.y) ** 2 * ref.delta / (x ** 2 - ref.delta ** 2)) for x in wv])
    co = lanczos.pseudo_hermitian(sys, 2 * ref.dim)
    got = spectrum.chi_lanczos(co.beta, co.gamma, co.z, wv.real, 0.1 / w.HA_EV)
    assert np.allclose(got, direct, rtol=1e-9)


@pytest.mark.parametrize("approx", ["ipa", "tddft"])
def test_operators_hermitian_and_positive(tiny, approx):
    sys = System(tiny, approx)
    a, b = _rand_batch(sys, 3), _rand_batch(sys, 4)
    for op in (sys.apply_d, sys.apply_k):
        ab = sys.inner(a, op(b))
        ba = sys.inner(b, op(a))
        assert abs(ab - np.conj(ba)) < 1e-12 * abs(ab) + 1e-14
    assert sys.inner(a, sys.apply_d(a)).real > 0
    assert sys.inner(a, sys.apply_op(a, upper=True)).real > 0


@pytest.mark.parametrize("flavour", ["ph", "nh"])
def test_moments_match_direct_liouvillian_powers(tiny, flavour):
    """((y,0), L^k (0,y)) from repeated direct applications of L equals b_1 (z, T^k e_1)
    for k < M: the Krylov relation the recursion must satisfy."""
    sys = System(tiny, "tddft")
    m = 8
    co = lanczos.run(sys, m, flavour)
    t = np.diag(co.beta[1:].astype(complex), -1) + np.diag(co.gamma[1:], 1)
    y = sys.starting_vector()
    up, lo = None, y
    e1 = np.zeros(m, dtype=complex)
    e1[0] = 1.0
    tk = e1
    for k in range(m):
        direct = sys.inner(y, up) if up is not None else 0.0
        via_t = co.beta[0] * np.dot(co.z, tk)
        assert abs(direct - via_t) <= 1e-10 * max(1.0, abs(direct)), (k, direct, via_t)
        up, lo = sys.apply_l(up, lo)
        tk = t @ tk


def test_pseudo_hermitian_half_the_applies(tiny):
    sys = System(tiny, "rpa")
    ph = lanczos.pseudo_hermitian(sys, 40)
    nh = lanczos.non_hermitian(sys, 40)
    assert ph.applies == 40 and nh.applies == 78


def test_zgtsv_against_dense_solve():
    rng = np.random.default_rng(5)
    m = 12
    beta = np.abs(rng.normal(size=m)) + 0.5
    gamma = beta * np.exp(1j * rng.normal(size=m) * 0.1)
    wv = 0.7 + 0.05j
    t = np.diag(beta[1:].astype(complex), -1) + np.diag(gamma[1:], 1)
    e1 = np.eye(m)[0]
    assert np.allclose(spectrum.tridiag_x(beta, gamma, wv), np.linalg.solve(wv * np.eye(m) - t, e1), rtol=1e-12)


def test_single_transition_spectrum():
    """One transition of weight W at Delta: T = [[0, Delta],[Delta, 0]] with z = (0, W/(b1 Delta))
    gives chi = W / ((w + i eta)^2 - Delta^2) exactly."""
    delta, weight, b1 = 0.3, 0.02, 0.5
    beta = np.array([b1, delta])
    z = np.array([0.0, weight / (b1 * delta)], dtype=complex)
    wv = np.array([0.1, 0.29, 0.5])
    got = spectrum.chi_lanczos(beta, beta.astype(complex), z, wv, 0.01)
    assert np.allclose(got, weight / ((wv + 0.01j) ** 2 - delta ** 2), rtol=1e-13)


def test_fsum_exact_moment_local_potential():
    """With a local potential and Q on the k-mesh, the first frequency moment of chi is
    n |Q|^2 (Eq. 6, Thomas-Reiche-Kuhn): (4/Omega)(y, D y) = n Q^2, up to the plane-wave
    truncation of e^{iQr} u (1e-7 of the norm at 30 Ry)."""
    spec = w.config_local_insulator()
    spec.ecut_ry, spec.nfft = 30.0, 20
    spec.q_cart = 0.5 * spec.bvec[0]
    b = w.get_bundle(spec)
    sys = System(b, "rpa")
    y = sys.starting_vector()
    m1 = 4.0 / spec.omega * sys.inner(y, sys.apply_d(y)).real
    n = spec.nelec / spec.omega
    assert abs(m1 / (n * spec.q_cart @ spec.q_cart) - 1.0) < 5e-5


def test_nh_and_ph_spectra_converge_together(tiny):
    """Below the space dimension the two recursions build different Krylov spaces; their
    broadened spectra still converge to each other as M grows (1 eV broadening)."""
    sys = System(tiny, "tddft")
    wgrid = np.linspace(0.0, 40.0, 401) / w.HA_EV
    errs = []
    for m in (150, 300):
        ph = lanczos.pseudo_hermitian(sys, m)
        nh = lanczos.non_hermitian(sys, m)
        a = spectrum.chi_lanczos(ph.beta, ph.gamma, ph.z, wgrid, 1.0 / w.HA_EV)
        b = spectrum.chi_lanczos(nh.beta, nh.gamma, nh.z, wgrid, 1.0 / w.HA_EV)
        errs.append(np.max(np.abs(a - b)) / np.max(np.abs(a)))
    assert errs[1] < 1e-4 and errs[1] < 0.1 * errs[0]


def test_hartree_kernel_and_fxc_tables(tiny):
    """The response kernel's ingredients against their definitions (Eq. 13, ALDA)."""
    from oracle import xc
    sys = System(tiny, "tddft")
    n = sys.n
    for idx in [(0, 0, 0), (1, 0, 0), (n - 1, 2, 5), (n // 2, n // 2, n // 2)]:
        m = np.array([i if i < n // 2 else i - n for i in idx])
        qg = sys.q + m @ sys.bvec
        assert np.isclose(sys.whart[idx], 4 * np.pi / (qg @ qg), rtol=1e-14)
    assert np.allclose(sys.fxc, xc.fxc(tiny.rho_r), rtol=0, atol=0)
    assert np.all(System(tiny, "rpa").fxc == 0)
    # Eq. 27 normalisation: int_cell n'[y] dr = 4 (1/N_k) sum <u_vk|y_vk> = 4 (y, y)
    # because y = P_c u and P_c is a projector
    y = sys.starting_vector()
    nr = sys.response_density(y)
    assert abs(nr.mean() * sys.omega - 4.0 * sys.inner(y, y)) < 1e-12
