"""Brute-force diagonalisation of the Liouvillian on a tiny system (a pin, not the method).

The conduction manifold at each k+Q is spanned explicitly by the eigenvectors of a
dense plane-wave Hamiltonian H_{GG'} = 1/2 |k+Q+G|^2 delta_{GG'} + V(G - G') +
sum_p beta_p(G) D_p beta_p(G')^*, with V(G - G') the cyclic convolution of the grid
potential.  In the orthonormal transition basis I = (v, c, k):
    D_IJ = (eps_{c,k+Q} - eps_{vk}) delta_IJ
    K_IJ = 4 / (Omega N_k N^3) sum_r conj(rho_I(r)) (kappa rho_J)(r),
           rho_I(r) = conj(psi_{vk}(r)) psi_{c,k+Q}(r),  kappa = Hartree + f_xc (Eqs. 12-13)
    y_I  = <c_{k+Q} | u_{vk}> / sqrt(N_k)
and the resolvent element of Eq. 10 in the SBR is
    ((y, 0), (w - L)^-1 (0, y)) = y^H D^1/2 (w^2 - M)^-1 D^1/2 y,  M = D^1/2 (D + K) D^1/2
(from w q = D p, w p = (D + K) q + y).  Diagonalising M gives the exact finite-basis
spectrum the Lanczos recursions converge to.
"""
from __future__ import annotations

import numpy as np

from . import basis
from .liouvillian import System


def dense_h(sys: System, k: int) -> np.ndarray:
    n = sys.n
    mil = sys.mkq[k]
    vbox = np.fft.fftn(sys.vloc) / n ** 3
    dm = (mil[:, None, :] - mil[None, :, :]) % n
    h = vbox[dm[..., 0], dm[..., 1], dm[..., 2]].astype(np.complex128)
    h[np.diag_indices_from(h)] += sys.kin[k]
    b = sys.beta[k]
    if b.shape[0]:
        h += (b.T * sys.dij) @ b.conj()
    return h


class Casida:
    def __init__(self, sys: System):
        self.sys = sys
        n, nb = sys.n, sys.nbnd
        delta, yv, rho = [], [], []
        for k in range(sys.nks):
            e, c = np.linalg.eigh(dense_h(sys, k))
            cond_e, cond = e[nb:], c[:, nb:].T                 # (nc, npw)
            u_on_kq = np.zeros((nb, len(sys.mkq[k])), dtype=np.complex128)
            mp = sys.map_k_kq[k]
            u_on_kq[:, mp >= 0] = sys.uk[k][:, mp[mp >= 0]]
            psi_c = basis.to_grid(cond, sys.mkq[k], n)         # (nc, N, N, N)
            for v in range(nb):
                delta.append(cond_e - sys.eps[k, v])
                yv.append(cond.conj() @ u_on_kq[v] / np.sqrt(sys.nks))
                rho.append((sys.ur[k][v].conj()[None] * psi_c).reshape(len(cond_e), -1))
        self.delta = np.concatenate(delta)
        self.y = np.concatenate(yv)
        self.rho = np.concatenate(rho)                          # (dim, N^3)
        self.dim = len(self.delta)
        if sys.approx == "ipa":
            kmat = np.zeros((self.dim, self.dim), dtype=np.complex128)
        else:
            r3 = self.rho.reshape(self.dim, n, n, n)
            krho = np.fft.ifftn(sys.whart[None] * np.fft.fftn(r3, axes=(1, 2, 3)), axes=(1, 2, 3))
            krho = krho + sys.fxc[None] * r3
            kmat = 4.0 / (sys.omega * sys.nks * n ** 3) * (self.rho.conj() @ krho.reshape(self.dim, -1).T)
        self.kmat = 0.5 * (kmat + kmat.conj().T)
        sd = np.sqrt(self.delta)
        m = sd[:, None] * (np.diag(self.delta) + self.kmat) * sd[None, :]
        self.omega2, self.vec = np.linalg.eigh(m)
        self.weight = np.abs(self.vec.conj().T @ (sd * self.y)) ** 2

    def chi_ll(self, w: np.ndarray) -> np.ndarray:
        """((y,0), (w - L)^-1 (0,y)) at complex frequencies w."""
        w = np.asarray(w, dtype=np.complex128)
        return (self.weight[None, :] / (w[:, None] ** 2 - self.omega2[None, :])).sum(axis=1)

    @property
    def excitation_energies(self) -> np.ndarray:
        return np.sqrt(self.omega2)
