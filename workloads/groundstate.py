"""Seeded LDA ground state of a synthetic cell: the stand-in for pw.x (Sec. 3.1).

The linear-response method takes as input the Kohn-Sham orbitals u_{vk} and u_{v,k+Q},
their energies, the self-consistent local potential and the ground-state density
(Sec. 3.1).  This module produces them by a plain plane-wave SCF with dense
Hamiltonian matrices: H_{GG'} = 1/2|k+G|^2 delta + V(G-G') + sum_p beta_p(k+G) D_p
beta_p(k+G')^*, where V(G-G') is the cyclic convolution on the FFT grid, i.e. exactly
the operator a grid-based apply of V(r) produces.  It contains no response arithmetic.

LDA: Slater exchange + Perdew-Zunger 1981 correlation (Sec. 5), unpolarised.
"""
from __future__ import annotations

import hashlib
import json
import os
from dataclasses import dataclass

import numpy as np
import scipy.linalg as sla
from scipy.special import dawsn, erfc

from .cells import (SystemSpec, fft_miller, grid_operations, irreducible_kpoints, kmesh_frac, small_group,
                    sphere)

PZ_GAMMA, PZ_B1, PZ_B2 = -0.1423, 1.0529, 0.3334
PZ_A, PZ_B, PZ_C, PZ_D = 0.0311, -0.048, 0.0020, -0.0116


def lda_vxc(n: np.ndarray) -> np.ndarray:
    """Slater + PZ81 exchange-correlation potential (Ha) of a density (bohr^-3)."""
    n = np.asarray(n, dtype=np.float64)
    out = np.zeros_like(n)
    m = n > 1e-10
    rs = (3.0 / (4.0 * np.pi * n[m])) ** (1.0 / 3.0)
    # Slater exchange energy per electron: -(3/4)(3/pi)^(1/3) n^(1/3)
    ex = -0.75 * (3.0 / np.pi) ** (1.0 / 3.0) * n[m] ** (1.0 / 3.0)
    vx = 4.0 / 3.0 * ex
    hi = rs >= 1.0
    vc = np.empty_like(rs)
    s = np.sqrt(rs[hi])
    den = 1.0 + PZ_B1 * s + PZ_B2 * rs[hi]
    ec = PZ_GAMMA / den
    vc[hi] = ec * (1.0 + 7.0 / 6.0 * PZ_B1 * s + 4.0 / 3.0 * PZ_B2 * rs[hi]) / den
    r = rs[~hi]
    lr = np.log(r)
    vc[~hi] = PZ_A * lr + (PZ_B - PZ_A / 3.0) + 2.0 / 3.0 * PZ_C * r * lr + (2.0 * PZ_D - PZ_C) / 3.0 * r
    out[m] = vx + vc
    return out


def grid_gvectors(spec: SystemSpec) -> tuple[np.ndarray, np.ndarray]:
    """Cartesian G of every FFT-grid frequency (N,N,N,3) and the integer Millers."""
    n = spec.nfft
    f = fft_miller(n)
    m = np.stack(np.meshgrid(f, f, f, indexing="ij"), axis=-1)
    return m @ spec.bvec, m


def vion_r(spec: SystemSpec) -> np.ndarray:
    """Ionic local potential on the grid: per atom -(4 pi Z/(Omega |G|^2)) exp(-|G|^2 rc^2/4)
    times the structure factor, G = 0 dropped, restricted to |G|^2 <= 4 ecut."""
    n = spec.nfft
    if spec.free_electron or len(spec.tau) == 0:
        return np.zeros((n, n, n))
    g, _ = grid_gvectors(spec)
    g2 = np.einsum("...i,...i->...", g, g)
    keep = (g2 > 0) & (g2 <= 4.0 * spec.ecut_ry)
    vg = np.zeros((n, n, n), dtype=np.complex128)
    form = np.zeros_like(g2)
    form[keep] = -4 * np.pi * spec.zval / (spec.omega * g2[keep]) * np.exp(-g2[keep] * spec.rc ** 2 / 4)
    for t in spec.tau:
        vg += np.exp(-1j * (g @ t)) * form
    return np.real(np.fft.ifftn(vg) * n ** 3)


def hartree_r(spec: SystemSpec, rho: np.ndarray) -> np.ndarray:
    n = spec.nfft
    g, _ = grid_gvectors(spec)
    g2 = np.einsum("...i,...i->...", g, g)
    keep = (g2 > 0) & (g2 <= 4.0 * spec.ecut_ry)
    rg = np.fft.fftn(rho) / n ** 3
    vg = np.zeros_like(rg)
    vg[keep] = 4 * np.pi * rg[keep] / g2[keep]
    return np.real(np.fft.ifftn(vg) * n ** 3)


def _ylm_real(kg: np.ndarray) -> np.ndarray:
    """Real spherical harmonics s, p_x, p_y, p_z of directions kg (npw,3); 0 at kg = 0."""
    k = np.linalg.norm(kg, axis=1)
    out = np.zeros((4, len(kg)))
    out[0] = 1.0 / np.sqrt(4 * np.pi)
    nz = k > 1e-12
    c = np.sqrt(3.0 / (4 * np.pi))
    for i in range(3):
        out[1 + i, nz] = c * kg[nz, i] / k[nz]
    return out


def kb_radial(g: np.ndarray, b: float) -> tuple[np.ndarray, np.ndarray]:
    """F_l(g) = 4 pi int r^2 j_l(g r) exp(-r^2/b^2) dr for l = 0, 1 (the (-i)^l kept apart).

    l = 0: pi^(3/2) b^3 exp(-g^2 b^2/4).  l = 1: with J(g) = int r j_0(g r) e^{-r^2/b^2} dr
    = b F(gb/2)/g (F the Dawson integral) and r j_1(g r) = -d j_0(g r)/dg, the integral is
    -J'(g) = b F(x)/g^2 - (b^2/2)(1 - 2 x F(x))/g with x = g b/2; g b^4/6 as g -> 0."""
    g = np.asarray(g, dtype=np.float64)
    f0 = np.pi ** 1.5 * b ** 3 * np.exp(-(g * b) ** 2 / 4.0)
    x = 0.5 * g * b
    small = g < 1e-4
    gs = np.where(small, 1.0, g)
    fx = dawsn(np.where(small, 0.0, x))
    i1 = b * fx / gs ** 2 - 0.5 * b * b * (1.0 - 2.0 * x * fx) / gs
    i1 = np.where(small, g * b ** 4 / 6.0, i1)
    return f0, 4 * np.pi * i1


def kb_projectors(spec: SystemSpec, kcart: np.ndarray, miller: np.ndarray) -> tuple[np.ndarray, np.ndarray]:
    """beta_p(k+G), (nproj, npw) complex, and D_p (Ha) for every atom: an s channel of
    strength s_core + D_s, then (when spec.kb) p_x, p_y, p_z of strength D_p."""
    kg = kcart[None, :] + miller @ spec.bvec
    if spec.nproj == 0:
        return np.zeros((0, len(miller)), dtype=np.complex128), np.zeros(0)
    g = np.linalg.norm(kg, axis=1)
    f0, f1 = kb_radial(g, spec.kb_b)
    y = _ylm_real(kg)
    ds = spec.s_core_ry + (spec.kb_d_ry[0] if spec.kb else 0.0)
    rows, d = [], []
    for t in spec.tau:
        ph = np.exp(-1j * (kg @ t)) / np.sqrt(spec.omega)
        rows.append(ph * f0 * y[0])
        d.append(0.5 * ds)
        if spec.kb:
            for i in range(3):
                rows.append(ph * (-1j) * f1 * y[1 + i])
                d.append(0.5 * spec.kb_d_ry[1])
    return np.array(rows), np.array(d)


def _hamiltonian(spec, kcart, miller, vbox):
    n = spec.nfft
    kg = kcart[None, :] + miller @ spec.bvec
    dm = (miller[:, None, :] - miller[None, :, :]) % n
    h = vbox[dm[..., 0], dm[..., 1], dm[..., 2]].astype(np.complex128)
    h[np.diag_indices_from(h)] += 0.5 * np.einsum("ij,ij->i", kg, kg)
    if spec.nproj:
        b, d = kb_projectors(spec, kcart, miller)
        h += (b.T * d) @ b.conj()
    return h


def _lowest(spec, kcart, vbox, nbnd):
    mil = sphere(kcart, spec.bvec, spec.ecut_ry)
    h = _hamiltonian(spec, kcart, mil, vbox)
    e, v = sla.eigh(h, subset_by_index=[0, nbnd - 1], driver="evr")
    return mil, e, v.T.copy()


# Occupations below F_MIN (or within F_MIN of one) are set to 0 (or 1): the response then
# counts a band as partially occupied only where its weight is significant.
F_MIN = 1e-12


def occupations(eps: np.ndarray, kw: np.ndarray, nelec: float, sigma_ha: float) -> tuple[float, np.ndarray]:
    """Gaussian smearing: f_vk = erfc((eps_vk - mu)/sigma)/2, with the Fermi level mu found by
    bisection so that 2 sum_k w_k sum_v f_vk = nelec (sum_k w_k = 1).  eps: (nks, nbnd) Ha.
    Returns (mu, f) with f clamped to exactly 0 or 1 within F_MIN of either."""
    eps = np.asarray(eps, dtype=np.float64)
    w = np.asarray(kw, dtype=np.float64)[:, None]

    def count(mu):
        return 2.0 * float(np.sum(w * 0.5 * erfc((eps - mu) / sigma_ha)))

    lo, hi = float(eps.min()) - 20 * sigma_ha, float(eps.max()) + 20 * sigma_ha
    if not count(lo) < nelec < count(hi):
        raise ValueError("too few bands for the electron count")
    for _ in range(200):
        mid = 0.5 * (lo + hi)
        if count(mid) < nelec:
            lo = mid
        else:
            hi = mid
    mu = 0.5 * (lo + hi)
    return mu, smeared(eps, mu, sigma_ha)


def smeared(eps: np.ndarray, mu: float, sigma_ha: float) -> np.ndarray:
    """erfc((eps - mu)/sigma)/2, clamped to exactly 0 or 1 within F_MIN of either."""
    f = 0.5 * erfc((np.asarray(eps, dtype=np.float64) - mu) / sigma_ha)
    f[f < F_MIN] = 0.0
    f[f > 1.0 - F_MIN] = 1.0
    return f


def _density(spec, pts, kw, occ=None):
    """2 sum_k w_k sum_v f_vk |psi_vk(r)|^2 / Omega (f = 1 without occupations)."""
    n = spec.nfft
    rho = np.zeros((n, n, n))
    for i, ((mil, e, c), w) in enumerate(zip(pts, kw)):
        grid = np.zeros((c.shape[0], n, n, n), dtype=np.complex128)
        idx = mil % n
        grid[:, idx[:, 0], idx[:, 1], idx[:, 2]] = c
        psi = np.fft.ifftn(grid, axes=(1, 2, 3)) * n ** 3
        a2 = np.abs(psi) ** 2
        if occ is None:
            rho += 2.0 * w * np.sum(a2, axis=0)
        else:
            rho += 2.0 * w * np.einsum("v,v...->...", occ[i], a2)
    return rho / spec.omega


def _feg_states(spec, kcart, nb):
    """Free-electron orbitals: the nb lowest plane waves of sphere(k)."""
    mil = sphere(kcart, spec.bvec, spec.ecut_ry)
    kg = kcart[None, :] + mil @ spec.bvec
    e = 0.5 * np.einsum("ij,ij->i", kg, kg)
    order = np.argsort(e, kind="stable")[:nb]
    c = np.zeros((nb, len(mil)), dtype=np.complex128)
    c[np.arange(nb), order] = 1.0
    return mil, e[order], c


@dataclass
class Bundle:
    """Everything the response calculation consumes (arrays in Hartree atomic units)."""
    spec: SystemSpec
    kfrac: np.ndarray          # (nks,3)
    kcart: np.ndarray          # (nks,3)
    miller_k: list             # nks x (npw_k,3) int32
    miller_kq: list            # nks x (npw_kq,3) int32
    u_k: list                  # nks x (nbnd,npw_k) complex128
    u_kq: list                 # nks x (nbnd,npw_kq) complex128, occupied states at k+Q
    eps_k: np.ndarray          # (nks,nbnd)
    eps_kq: np.ndarray         # (nks,nbnd)
    vloc_r: np.ndarray         # (N,N,N) total KS local potential, index [j1,j2,j3]
    rho_r: np.ndarray          # (N,N,N) ground-state density
    beta_kq: list              # nks x (nproj,npw_kq) complex128 (empty when no KB)
    dij: np.ndarray            # (nproj,) Ha
    scf_iters: int = 0
    gap_min: float = 0.0       # min_k (eps_{nbnd+1,k+Q} - eps_{nbnd,k}) (Ha), positivity of D
    kweight: np.ndarray | None = None   # (nks,) star sizes of irreducible k-points (None: every k once)
    sym: np.ndarray | None = None       # (nsym,3,3) int: the small group of Q on the FFT grid (None: identity)
    occ_k: np.ndarray | None = None     # (nks,nbnd) occupations f_vk in [0,1] of a metal (None: all 1)
    occ_kq: np.ndarray | None = None    # (nks,nbnd) occupations of the states at k+Q
    fermi: float = 0.0                  # Fermi level of a metal (Ha)

    @property
    def nks(self):
        return len(self.kfrac)

    @property
    def npw_k(self):
        return np.array([len(m) for m in self.miller_k], dtype=np.int32)

    @property
    def npw_kq(self):
        return np.array([len(m) for m in self.miller_kq], dtype=np.int32)


class _Runner:
    """Maps the per-k eigenproblems serially, or over a spawn pool of single-threaded
    workers when the work is large enough to pay for the start-up."""

    def __init__(self, work: float):
        self.pool = None
        ncpu = os.cpu_count() or 1
        if work > 1e11 and ncpu > 1:
            import multiprocessing as mp
            keys = ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS")
            saved = {k: os.environ.get(k) for k in keys}
            for k in keys:
                os.environ[k] = "1"
            try:
                self.pool = mp.get_context("spawn").Pool(min(ncpu, 32))
            finally:
                for k, v in saved.items():
                    if v is None:
                        os.environ.pop(k, None)
                    else:
                        os.environ[k] = v

    def map(self, fn, jobs):
        if self.pool is None:
            return [fn(j) for j in jobs]
        return self.pool.map(fn, jobs, chunksize=max(1, len(jobs) // (8 * self.pool._processes)))

    def close(self):
        if self.pool is not None:
            self.pool.close()
            self.pool.join()


def _lowest_job(args):
    spec, kc, vbox, nb = args
    return _lowest(spec, kc, vbox, nb)


def scf(spec: SystemSpec, tol: float = 1e-11, maxiter: int = 80, verbose: bool = False,
        runner: _Runner | None = None):
    """Self-consistent LDA potential on spec.scf_kmesh (or spec.kmesh), Pulay mixing of the
    density.  Returns (V_KS(r), rho(r), iterations)."""
    n = spec.nfft
    vion = vion_r(spec)
    mesh = spec.scf_kmesh or spec.kmesh
    kf = kmesh_frac(mesh)
    kc = kf @ spec.bvec
    kw = np.full(len(kf), 1.0 / len(kf))
    rho = np.full((n, n, n), spec.nelec / spec.omega)
    if spec.free_electron:
        # V = 0: the free-electron limit; the uniform gas's constant v_xc would shift every
        # level alike, and the plane-wave levels below are the bare kinetic energies
        return vion, rho, 0
    tol = spec.extra.get("scf_tol", tol)
    # a pool of single-threaded workers only pays with several k-points; one or two large
    # eigenproblems run here with threaded LAPACK
    runner = runner if (runner is not None and len(kc) >= 4) else _Runner(0)
    hist_in, hist_res = [], []
    err = np.inf
    for it in range(1, maxiter + 1):
        v = vion + hartree_r(spec, rho) + lda_vxc(rho)
        vbox = np.fft.fftn(v) / n ** 3
        pts = runner.map(_lowest_job, [(spec, k, vbox, spec.nbnd) for k in kc])
        occ = None
        if spec.metal:
            occ = occupations(np.array([p[1] for p in pts]), kw, spec.nelec, spec.smearing_ry / 2)[1]
        rout = _density(spec, pts, kw, occ)
        res = rout - rho
        err = np.sum(np.abs(res)) * spec.omega / n ** 3
        if verbose:
            print(f"scf {it:3d}  |drho| = {err:.3e}", flush=True)
        if err < tol:
            rho = rout
            break
        hist_in.append(rho.ravel().copy())
        hist_res.append(res.ravel().copy())
        hist_in, hist_res = hist_in[-8:], hist_res[-8:]
        m = len(hist_res)
        a = np.array([[np.dot(hist_res[i], hist_res[j]) for j in range(m)] for i in range(m)])
        a = np.pad(a, ((0, 1), (0, 1)), constant_values=1.0)
        a[-1, -1] = 0.0
        rhs = np.zeros(m + 1)
        rhs[-1] = 1.0
        try:
            c = np.linalg.solve(a, rhs)[:m]
        except np.linalg.LinAlgError:
            c = np.zeros(m)
            c[-1] = 1.0
        rin = sum(ci * h for ci, h in zip(c, hist_in))
        rr = sum(ci * h for ci, h in zip(c, hist_res))
        rho = np.maximum((rin + 0.4 * rr).reshape(n, n, n), 1e-12)
    else:
        raise RuntimeError(f"SCF did not converge in {maxiter} iterations ({err:.2e})")
    v = vion + hartree_r(spec, rho) + lda_vxc(rho)
    return v, rho, it


def build_bundle(spec: SystemSpec, verbose: bool = False) -> Bundle:
    """SCF, then the occupied states (and one more band, for the gap check) at every k and k+Q."""
    n = spec.nfft
    kweight = sym = None
    if spec.symmetry:
        ops = small_group(spec)
        kf, kweight = irreducible_kpoints(spec, ops)
        sym = grid_operations(spec, ops)
    else:
        kf = kmesh_frac(spec.kmesh)
    kc = kf @ spec.bvec
    kq = kc + spec.q_cart[None, :]
    npw_est = 4.0 / 3.0 * np.pi * spec.ecut_ry ** 1.5 * spec.omega / (2 * np.pi) ** 3
    runner = _Runner(2 * len(kc) * npw_est ** 3 * 10)
    try:
        v, rho, iters = _scf_cached(spec, verbose, runner)
        vbox = np.fft.fftn(v) / n ** 3
        if spec.free_electron:
            res_k = [_feg_states(spec, k, spec.nbnd + 1) for k in kc]
            res_q = [_feg_states(spec, k, spec.nbnd + 1) for k in kq]
            gap = 0.0
        else:
            out = runner.map(_lowest_job, [(spec, k, vbox, spec.nbnd + 1) for k in np.concatenate([kc, kq])])
            res_k, res_q = out[: len(kc)], out[len(kc):]
            gap = min(float(rq[1][spec.nbnd] - rk[1][spec.nbnd - 1]) for rk, rq in zip(res_k, res_q))
    finally:
        runner.close()
    nb = spec.nbnd
    occ_k = occ_kq = None
    fermi = 0.0
    if spec.metal:
        # occupations on the response mesh from its own levels (the wedge's with star weights)
        ek = np.array([r[1][:nb + 1] for r in res_k])
        eq = np.array([r[1][:nb + 1] for r in res_q])
        wk = np.ones(len(kc)) if kweight is None else np.asarray(kweight, dtype=np.float64)
        fermi, _ = occupations(ek[:, :nb], wk / wk.sum(), spec.nelec, spec.smearing_ry / 2)
        sig = spec.smearing_ry / 2
        if np.any(smeared(ek[:, nb], fermi, sig) > 0) or np.any(smeared(eq[:, nb], fermi, sig) > 0):
            raise ValueError("band nbnd+1 is occupied: more bands needed")
        occ_k, occ_kq = smeared(ek[:, :nb], fermi, sig), smeared(eq[:, :nb], fermi, sig)
        # every state left out at k+Q must lie above every occupied level at k (the
        # transitions into them then have positive energies)
        gap = float(eq[:, nb].min() - ek[:, :nb][occ_k > 0].max())
        if gap <= 0:
            raise ValueError("a state left out at k+Q lies below an occupied level")
    beta, dij = [], np.zeros(0)
    for k, r in zip(kq, res_q):
        b, dij = kb_projectors(spec, k, r[0])
        beta.append(b)
    return Bundle(spec=spec, kfrac=kf, kcart=kc,
                  miller_k=[r[0] for r in res_k], miller_kq=[r[0] for r in res_q],
                  u_k=[np.ascontiguousarray(r[2][:nb]) for r in res_k],
                  u_kq=[np.ascontiguousarray(r[2][:nb]) for r in res_q],
                  eps_k=np.array([r[1][:nb] for r in res_k]),
                  eps_kq=np.array([r[1][:nb] for r in res_q]),
                  vloc_r=v, rho_r=rho, beta_kq=beta, dij=dij, scf_iters=iters, gap_min=gap, kweight=kweight, sym=sym,
                  occ_k=occ_k, occ_kq=occ_kq, fermi=fermi)


def _scf_cached(spec: SystemSpec, verbose: bool, runner) -> tuple:
    """scf() once per crystal: the self-consistent potential does not depend on Q, so every
    momentum transfer of one system reuses it (npz under .ll_cache/)."""
    d = {k: (np.asarray(v).round(12).tolist() if isinstance(v, np.ndarray) else v)
         for k, v in spec.__dict__.items()
         if k not in ("steps", "flavour", "approx", "extra", "q_cart", "kmesh", "name", "scf_kmesh", "symmetry")}
    d["scf_mesh"] = list(spec.scf_kmesh or spec.kmesh)
    _drop_defaults(d)
    key = hashlib.sha1(json.dumps(d, sort_keys=True, default=str).encode()).hexdigest()[:16]
    path = os.path.join(cache_dir(), f"scf_{key}.npz")
    if os.path.exists(path):
        z = np.load(path)
        return z["v"], z["rho"], int(z["iters"])
    v, rho, iters = scf(spec, verbose=verbose, runner=runner)
    tmp = path + f".{os.getpid()}.tmp.npz"
    np.savez(tmp, v=v, rho=rho, iters=iters)
    os.replace(tmp, path)
    return v, rho, iters


def _drop_defaults(d: dict) -> None:
    """Insulators keep the cache keys they had before the metal options existed."""
    if not d.get("smearing_ry"):
        d.pop("smearing_ry", None)
    if d.get("electrons") is None:
        d.pop("electrons", None)


def _spec_key(spec: SystemSpec) -> str:
    d = {k: (np.asarray(v).round(12).tolist() if isinstance(v, np.ndarray) else v)
         for k, v in spec.__dict__.items() if k not in ("steps", "flavour", "approx", "extra")}
    if not d.get("symmetry"):      # keys of full-mesh bundles as before the option existed
        d.pop("symmetry", None)
    _drop_defaults(d)
    return hashlib.sha1(json.dumps(d, sort_keys=True, default=str).encode()).hexdigest()[:16]


def cache_dir() -> str:
    root = os.environ.get("LL_CACHE_DIR") or os.path.join(os.path.dirname(os.path.dirname(
        os.path.abspath(__file__))), ".ll_cache")
    os.makedirs(root, exist_ok=True)
    return root


def save_bundle(b: Bundle, path: str) -> None:
    """The projectors beta_kq are not stored: they are a closed form of the spec and the
    spheres, rebuilt on load (half the file for the cells with many projectors)."""
    arrs = dict(kfrac=b.kfrac, kcart=b.kcart, eps_k=b.eps_k, eps_kq=b.eps_kq, vloc_r=b.vloc_r,
                rho_r=b.rho_r, dij=b.dij, scf_iters=b.scf_iters, gap_min=b.gap_min,
                npw_k=b.npw_k, npw_kq=b.npw_kq,
                miller_k=np.concatenate(b.miller_k), miller_kq=np.concatenate(b.miller_kq),
                u_k=np.concatenate([u.T for u in b.u_k]), u_kq=np.concatenate([u.T for u in b.u_kq]))
    if b.kweight is not None:
        arrs.update(kweight=b.kweight, sym=b.sym)
    if b.occ_k is not None:
        arrs.update(occ_k=b.occ_k, occ_kq=b.occ_kq, fermi=b.fermi)
    np.savez(path, **arrs)


def load_bundle(spec: SystemSpec, path: str) -> Bundle:
    z = np.load(path)
    npk, npq = z["npw_k"], z["npw_kq"]
    sk, sq = np.concatenate([[0], np.cumsum(npk)]), np.concatenate([[0], np.cumsum(npq)])
    sl = lambda a, s, i: a[s[i]:s[i + 1]]
    nks = len(npk)
    if "beta_kq" in z.files:          # files written before the projectors were rebuilt on load
        beta = [np.ascontiguousarray(sl(z["beta_kq"], sq, i).T) for i in range(nks)]
    else:
        kq = z["kcart"] + spec.q_cart[None, :]
        beta = [kb_projectors(spec, kq[i], sl(z["miller_kq"], sq, i))[0] for i in range(nks)]
    return Bundle(spec=spec, kfrac=z["kfrac"], kcart=z["kcart"],
                  miller_k=[sl(z["miller_k"], sk, i) for i in range(nks)],
                  miller_kq=[sl(z["miller_kq"], sq, i) for i in range(nks)],
                  u_k=[np.ascontiguousarray(sl(z["u_k"], sk, i).T) for i in range(nks)],
                  u_kq=[np.ascontiguousarray(sl(z["u_kq"], sq, i).T) for i in range(nks)],
                  eps_k=z["eps_k"], eps_kq=z["eps_kq"], vloc_r=z["vloc_r"], rho_r=z["rho_r"],
                  beta_kq=beta, dij=z["dij"], scf_iters=int(z["scf_iters"]), gap_min=float(z["gap_min"]),
                  kweight=z["kweight"] if "kweight" in z.files else None, sym=z["sym"] if "sym" in z.files else None,
                  occ_k=z["occ_k"] if "occ_k" in z.files else None,
                  occ_kq=z["occ_kq"] if "occ_kq" in z.files else None,
                  fermi=float(z["fermi"]) if "fermi" in z.files else 0.0)


def bundle_digest(b: Bundle) -> str:
    """sha256 (16 hex digits) of every stored array a chain consumes, in a fixed order: two
    bundles with the same digest hold the same ground state to the last bit.  (A bundle rebuilt
    by another machine's LAPACK differs in the last bits of the orbitals, and so in its digest.)
    The KB projectors are left out: they are a closed form of the cell and the spheres (both
    covered), rebuilt on every load with the machine's own exp and Dawson function, so they
    may differ in the last bit between machines reading the same file."""
    h = hashlib.sha256()
    arrays = [b.kcart, b.eps_k, b.vloc_r, b.rho_r, b.dij] + list(b.miller_k) + list(b.miller_kq) + \
        list(b.u_k) + list(b.u_kq)
    if b.kweight is not None:
        arrays += [b.kweight, b.sym]
    if b.occ_k is not None:
        arrays += [b.eps_kq, b.occ_k, b.occ_kq]
    for a in arrays:
        a = np.ascontiguousarray(a)
        h.update(str(a.dtype).encode() + str(a.shape).encode())
        h.update(a.tobytes())
    return h.hexdigest()[:16]


def cached_bundle(spec: SystemSpec) -> Bundle | None:
    """The cached bundle of spec, or None when it has not been built here."""
    path = os.path.join(cache_dir(), f"{spec.name}_{_spec_key(spec)}.npz")
    return load_bundle(spec, path) if os.path.exists(path) else None


def get_bundle(spec: SystemSpec, verbose: bool = False) -> Bundle:
    """Cached build_bundle (npz under .ll_cache/, keyed by the ground-state parameters)."""
    path = os.path.join(cache_dir(), f"{spec.name}_{_spec_key(spec)}.npz")
    if os.path.exists(path):
        return load_bundle(spec, path)
    b = build_bundle(spec, verbose=verbose)
    tmp = path + f".{os.getpid()}.tmp.npz"
    save_bundle(b, tmp)
    os.replace(tmp, path)
    return b
