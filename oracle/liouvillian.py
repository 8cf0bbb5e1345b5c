"""The Liouvillian in the standard batch representation (Sec. 2.4), FP64, written out.

A batch vector x = {x_{vk}} holds one lattice-periodic orbital per occupied band v and
k-point k, expanded on the sphere of k+Q; here it is a list over k of (nbnd, npw_kq[k])
complex arrays.  Scalar product of batches (the one the Lanczos recursions use):
    (a, b) = (1/N_k) sum_k sum_v sum_G conj(a_{vk}(G)) b_{vk}(G).

Operators (Eqs. 24-28, Hartree units):
    D x = { P_c^{k+Q} (H_{k+Q} - eps_{vk}) x_{vk} }                      (Eq. 25)
    K x = { P_c^{k+Q} v'_HXC[n'](r) u_{vk}(r) }                          (Eq. 26)
    n'(r) = 4 sum_{vk} w_k u*_{vk}(r) x_{vk}(r),  w_k = 1/N_k            (Eq. 27)
    v'_H(G) = 4 pi n'(G) / |Q+G|^2  on every grid frequency               (Eq. 13)
    v'_XC(r) = f_xc(n0(r)) n'(r)  (ALDA; RPA drops it; IPA drops K)      (Sec. 3.2)
    y = { P_c^{k+Q} u_{vk} }  (perturbation e^{iQ.r} with Q kept unfolded)  (Eq. 28)
    P_c^{k} = 1 - sum_v |u_{vk}><u_{vk}|                                  (Eq. 16)
    L (q, p) = (D p, (D + K) q)                                           (Eq. 24)

Readings: P_c is applied to the whole output of D and K (projecting H x as well keeps
every Lanczos vector in the conduction manifold); H_{k+Q} = kinetic + V_KS(r) + KB
projectors; the Hartree kernel runs over every frequency of the FFT box.

k-point symmetry (Sec. 2.6): when the bundle holds only the k-points of the irreducible
wedge of the small group G_Q of Q, each with its star size m_k (sum_k m_k = N_k of the full
mesh), every sum over the mesh becomes a weighted sum over the wedge,
    (a, b) = (1/N_k) sum_k m_k sum_v sum_G conj(a_{vk}(G)) b_{vk}(G),
    n~(r)  = 4 (1/N_k) sum_k m_k sum_v u*_{vk}(r) x_{vk}(r),
and the response density is the average of n~ over the group, n'(r) = (1/|G_Q|) sum_S
n~(S r) (the terms of the k-points of a star are the rotated terms of its representative).
Without symmetry m_k = 1 and G_Q = {E}: the plain sums above.

Metals (Sec. 2.6: the projector on empty states redefined, fractional occupations as weights
in the band sums; the smearing approach of the static theory the paper cites).  Reading:
with occupations f_{vk} and f_{m,k+Q} in [0, 1] (the bundle's, from Gaussian smearing), the
independent-particle response is the transition sum over (f_v - f_m) |M|^2/(w - Delta_mv);
each pair of levels is given to the one direction with a positive transition energy (a sharp
step theta(eps_m - eps_v) in the projector of the static theory), which leaves every kept
transition a weight w_vm = f_v - f_m > 0 and a positive energy, so the pseudo-Hermitian
recursion's metric stays positive.  Per band v of k, with c_mv = max(1 - f_m/f_v, 0)
(0 for f_v = 0; below C_MIN counted as 0) for the bands m of k+Q:
    P_{c,v} x = x - sum_m (1 - c_mv) |u_{m,k+Q}><u_{m,k+Q}|x>           (the redefined P_c)
    K x = { P_{c,v} v'_HXC[n'](r) u_{vk}(r) },  y = { P_{c,v} u_{vk} } (perturbation as above)
    n'(r) = 4 (1/N_k) sum_k m_k sum_v f_{vk} u*_{vk}(r) x_{vk}(r)        (band-sum weights)
    D x = { P'_v (H_{k+Q} - eps_{vk}) x_{vk} },  P'_v: removes the m with c_mv = 0
and the scalar product is the metric that makes D and K Hermitian,
    (a, b) = (1/N_k) sum_k m_k sum_v f_{vk} [ a_v^H b_v + sum_{m: c_mv > 0} (1/c_mv - 1)
             conj(<u_m|a_v>) <u_m|b_v> ].
Every new Lanczos vector is projected with P'_v.  Fully occupied bands (f = 1 everywhere)
give c = 0 and f_v = 1: the insulator's P_c, D, K and product.  The response is for Q + G
!= 0 only, so the Fermi level does not move (no shift term).
"""
from __future__ import annotations

import numpy as np
import scipy.fft as sfft

from . import basis, xc

# weights c_mv of the metallic projector below this count as 0 (the transition is dropped)
C_MIN = 1e-6


def metal_weights(f_v: np.ndarray, f_m: np.ndarray) -> np.ndarray:
    """c[m, v] = max(1 - f_m/f_v, 0) for f_v > 0, else 0; entries below C_MIN set to 0."""
    f_v = np.asarray(f_v, dtype=np.float64)
    f_m = np.asarray(f_m, dtype=np.float64)
    c = np.zeros((len(f_m), len(f_v)))
    for v in range(len(f_v)):
        if f_v[v] > 0.0:
            c[:, v] = np.maximum(1.0 - f_m / f_v[v], 0.0)
    c[c < C_MIN] = 0.0
    return c


class System:
    """Everything the operators need, derived from a ground-state bundle."""

    def __init__(self, bundle, approx: str | None = None):
        spec = bundle.spec
        self.spec = spec
        self.n = spec.nfft
        self.omega = spec.omega
        self.nks = bundle.nks
        self.kw = (np.ones(self.nks) if getattr(bundle, "kweight", None) is None
                   else np.asarray(bundle.kweight, dtype=np.float64))
        self.nfull = float(np.sum(self.kw))       # N_k of the full mesh
        self.sym = (np.eye(3, dtype=np.int64)[None] if getattr(bundle, "sym", None) is None
                    else np.asarray(bundle.sym, dtype=np.int64))
        self.nbnd = spec.nbnd
        self.approx = approx or spec.approx
        assert self.approx in ("ipa", "rpa", "tddft")
        self.q = np.asarray(spec.q_cart, dtype=np.float64)
        self.bvec = spec.bvec
        self.kcart = bundle.kcart
        self.mk = bundle.miller_k
        self.mkq = bundle.miller_kq
        self.uk = bundle.u_k
        self.ukq = bundle.u_kq
        self.eps = bundle.eps_k
        self.vloc = bundle.vloc_r
        self.rho = bundle.rho_r
        self.beta = bundle.beta_kq
        self.dij = bundle.dij
        n = self.n
        # kinetic energy 1/2 |k+Q+G|^2 on each sphere of k+Q
        self.kin = []
        for k in range(self.nks):
            kg = self.kcart[k] + self.q + self.mkq[k] @ self.bvec
            self.kin.append(0.5 * np.einsum("ij,ij->i", kg, kg))
        # Hartree weights 4 pi / |Q+G|^2 over the FFT box (frequencies in fftfreq order)
        f = np.fft.fftfreq(n, 1.0 / n)
        m = np.stack(np.meshgrid(f, f, f, indexing="ij"), axis=-1)
        qg = self.q + m @ self.bvec
        qg2 = np.einsum("...i,...i->...", qg, qg)
        if np.min(qg2) <= 0:
            raise ValueError("Q + G = 0 on the grid: Q must not be a reciprocal lattice vector")
        self.whart = 4 * np.pi / qg2
        self.fxc = xc.fxc(self.rho) if self.approx == "tddft" else np.zeros_like(self.rho)
        # ground-state orbitals u_{vk}(r) (times sqrt(Omega)) on the grid, each k-point's
        # transformed when first used (a rank of the k-point split touches only its own block)
        self.ur = _LazyGrids(self.uk, self.mk, n)
        self.map_k_kq = [basis.intersection_map(self.mk[k], self.mkq[k]) for k in range(self.nks)]
        self.metal = getattr(bundle, "occ_k", None) is not None
        if self.metal:
            self.f = np.asarray(bundle.occ_k, dtype=np.float64)
            fq = np.asarray(bundle.occ_kq, dtype=np.float64)
            self.c = [metal_weights(self.f[k], fq[k]) for k in range(self.nks)]

    # ----- batches -------------------------------------------------------------------
    def zeros(self):
        return [np.zeros((self.nbnd, len(m)), dtype=np.complex128) for m in self.mkq]

    def inner(self, a, b) -> complex:
        return self.inner_part(a, b) / self.nfull

    def inner_part(self, a, b, ks=None) -> complex:
        """N_k (a, b) restricted to the k-points ks (default all): the weighted sum over k."""
        ks = self._ks(a, ks)
        if not self.metal:
            return sum(self.kw[k] * np.vdot(ak, bk) for k, ak, bk in zip(ks, a, b))
        tot = 0.0
        for k, ak, bk in zip(ks, a, b):
            u, c = self.ukq[k], self.c[k]
            sa, sb = u.conj() @ ak.T, u.conj() @ bk.T             # <u_m|a_v>, (nbnd_m, nbnd_v)
            corr = np.where(c > 0, 1.0 / np.where(c > 0, c, 1.0) - 1.0, 0.0)
            per_v = np.einsum("vg,vg->v", ak.conj(), bk) + np.einsum("mv,mv,mv->v", corr, sa.conj(), sb)
            tot += self.kw[k] * np.dot(self.f[k], per_v)
        return tot

    # Every per-k method takes the k index of each entry of its batch in `ks` (default: all
    # k-points in order), so that a rank holding a block of k-points can apply it to its block.
    def _ks(self, x, ks):
        return range(len(x)) if ks is None else ks

    def project_c(self, x, ks=None):
        """P_c^{k+Q} x = x - U (U^H x) with U the occupied states at k+Q (Eq. 16).  A metal:
        P'_v, which removes only the states m with c_mv = 0."""
        out = []
        for k, xk in zip(self._ks(x, ks), x):
            u = self.ukq[k]
            s = u.conj() @ xk.T
            if self.metal:
                s = s * (self.c[k] == 0.0)
            out.append(xk - (u.T @ s).T)
        return out

    def project_weighted(self, x, ks=None):
        """The projector of K and y: P_c^{k+Q} (an insulator), P_{c,v} (a metal)."""
        if not self.metal:
            return self.project_c(x, ks)
        out = []
        for k, xk in zip(self._ks(x, ks), x):
            u = self.ukq[k]
            s = (u.conj() @ xk.T) * (1.0 - self.c[k])
            out.append(xk - (u.T @ s).T)
        return out

    def starting_vector(self):
        """y_{vk} = P_c^{k+Q} u_{vk}: u_{vk}'s coefficient at each Miller of sphere(k+Q), or 0."""
        y = []
        for k in range(self.nks):
            mp = self.map_k_kq[k]
            yk = np.zeros((self.nbnd, len(mp)), dtype=np.complex128)
            hit = mp >= 0
            yk[:, hit] = self.uk[k][:, mp[hit]]
            y.append(yk)
        return self.project_weighted(y)

    # ----- operators -----------------------------------------------------------------
    def apply_h_minus_eps(self, x, ks=None):
        """(H_{k+Q} - eps_{vk}) x_{vk}, unprojected: kinetic, V_KS(r), KB projectors."""
        n = self.n
        out = []
        for k, xk in zip(self._ks(x, ks), x):
            mil = self.mkq[k]
            psi = basis.to_grid(xk, mil, n)
            t = basis.to_sphere(self.vloc[None] * psi, mil, n)
            t += (self.kin[k][None, :] - self.eps[k][:, None]) * xk
            b = self.beta[k]
            if b.shape[0]:
                c = b.conj() @ xk.T                        # <beta_p|x_v>   (nproj, nbnd)
                t += ((b.T * self.dij) @ c).T
            out.append(t)
        return out

    def apply_d(self, x, ks=None):
        return self.project_c(self.apply_h_minus_eps(x, ks), ks)

    def response_density(self, x, ks=None):
        """n~(r) = 4 (1/N_k) sum_{vk} m_k u*_{vk}(r) x_{vk}(r), u = psi/sqrt(Omega) (times f_vk for
        a metal); with `ks`, the part of the sum over those k-points.  (Without symmetry, n'
        itself.)"""
        n = self.n
        nr = np.zeros((n, n, n), dtype=np.complex128)
        for k, xk in zip(self._ks(x, ks), x):
            psi = basis.to_grid(xk, self.mkq[k], n)
            if self.metal:
                nr += self.kw[k] * np.einsum("v,v...->...", self.f[k], self.ur[k].conj() * psi)
            else:
                nr += self.kw[k] * np.sum(self.ur[k].conj() * psi, axis=0)
        return 4.0 * nr / (self.omega * self.nfull)

    def symmetrize(self, nr):
        """n'(r_j) = (1/|G_Q|) sum_S n~(r_{M_S j}) over the small group of Q (M_S: the integer
        matrices of its operations on the grid indices, taken mod N)."""
        if len(self.sym) == 1:
            return nr
        n = self.n
        j = np.stack(np.meshgrid(np.arange(n), np.arange(n), np.arange(n), indexing="ij"), axis=-1)
        out = np.zeros_like(nr)
        for m in self.sym:
            jm = (j @ m.T) % n
            out += nr[jm[..., 0], jm[..., 1], jm[..., 2]]
        return out / len(self.sym)

    def hxc_potential(self, nr):
        """v'(r) = sum_G 4 pi n'(G)/|Q+G|^2 e^{iG.r} + f_xc(n0(r)) n'(r), n' the average of
        the density over the small group of Q."""
        nr = self.symmetrize(nr)
        vh = sfft.ifftn(self.whart * sfft.fftn(nr))
        return vh + self.fxc * nr

    def apply_k(self, x):
        if self.approx == "ipa":
            return self.zeros()
        return self.apply_v(self.hxc_potential(self.response_density(x)))

    def apply_v(self, v, ks=None):
        """K's last step: P_c^{k+Q} v'(r) u_{vk}(r) (P_{c,v} for a metal) for the k-points ks
        (default all)."""
        ks = range(self.nks) if ks is None else ks
        out = [basis.to_sphere(v[None] * self.ur[k], self.mkq[k], self.n) for k in ks]
        return self.project_weighted(out, ks)

    def apply_op(self, x, upper: bool):
        """The operator the recursions apply to one half of a batch: D + K on the upper
        (q) component, D on the lower (p) component (Eq. 24)."""
        d = self.apply_d(x)
        if not upper or self.approx == "ipa":
            return d
        kx = self.apply_k(x)
        return [a + b for a, b in zip(d, kx)]

    def apply_l(self, up, lo):
        """L (q, p) = (D p, (D + K) q) on a full batch pair (either half may be None = 0)."""
        new_up = self.apply_op(lo, upper=False) if lo is not None else None
        new_lo = self.apply_op(up, upper=True) if up is not None else None
        return new_up, new_lo


class _LazyGrids:
    """ur[k] = u_{vk}(r) sqrt(Omega) on the grid (basis.to_grid), computed once on first access."""

    def __init__(self, coefs, millers, n):
        self.coefs, self.millers, self.n = coefs, millers, n
        self.cache = {}

    def __len__(self):
        return len(self.coefs)

    def __getitem__(self, k):
        g = self.cache.get(k)
        if g is None:
            g = basis.to_grid(self.coefs[k], self.millers[k], self.n)
            self.cache[k] = g
        return g


def axpy(a, x, y):
    """a x + y on batches."""
    return [a * xk + yk for xk, yk in zip(x, y)]


def scale(a, x):
    return [a * xk for xk in x]
