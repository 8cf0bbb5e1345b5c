"""Seeded synthetic systems: cells, k-meshes, momentum transfers and plane-wave spheres.

This module is an input generator shared by the FP64 oracle and the CUDA path.  It
holds none of the Liouville-Lanczos arithmetic (no response density, no Liouvillian,
no Lanczos step, no spectrum): it only describes the crystal and enumerates the
integer Miller indices of the plane-wave basis, i.e. what the ground-state program
(pw.x in the paper, Sec. 3.1) hands to the linear-response code.

Units are Hartree atomic units (Sec. 2.2); cut-offs are given in Rydberg as in the
paper's input tables and used as |k+G|^2 <= ecut_Ry (bohr^-2).
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

HA_EV = 27.211386245988          # CODATA 2018 Hartree in eV
A_LAT = 10.26                    # bohr: the lattice parameter of every synthetic cell


def fcc_primitive(a: float) -> np.ndarray:
    """Rows are the primitive vectors of the face-centred cubic lattice (ibrav=2 axes)."""
    return 0.5 * a * np.array([[-1.0, 0.0, 1.0], [0.0, 1.0, 1.0], [-1.0, 1.0, 0.0]])


def reciprocal(lattice: np.ndarray) -> np.ndarray:
    """Rows b_i with a_i . b_j = 2 pi delta_ij."""
    return 2.0 * np.pi * np.linalg.inv(lattice).T


def kmesh_frac(n: tuple[int, int, int]) -> np.ndarray:
    """Gamma-centred mesh in fractions of the reciprocal vectors, each in [0, 1), C order."""
    i, j, k = np.meshgrid(np.arange(n[0]), np.arange(n[1]), np.arange(n[2]), indexing="ij")
    return np.stack([i.ravel() / n[0], j.ravel() / n[1], k.ravel() / n[2]], axis=1)


@dataclass
class SystemSpec:
    """One synthetic crystal plus the response calculation run on it."""
    name: str
    lattice: np.ndarray            # (3,3) rows a_i, bohr
    tau: np.ndarray                # (nat,3) Cartesian atomic positions, bohr
    zval: float                    # ionic charge per atom of the local potential
    rc: float                      # Gaussian smearing radius of the local potential, bohr
    ecut_ry: float                 # wavefunction cut-off, Ry
    nfft: int                      # FFT grid side N (cubic N^3 grid along a_i)
    kmesh: tuple                   # response k-mesh (Gamma-centred)
    nbnd: int                      # occupied bands
    q_cart: np.ndarray             # momentum transfer Q, Cartesian bohr^-1
    approx: str = "tddft"          # 'ipa' | 'rpa' | 'tddft'
    kb: bool = False               # extra Kleinman-Bylander s+p channels on every atom
    kb_b: float = 0.8              # radial width of beta(r) = exp(-r^2/b^2), bohr
    kb_d_ry: tuple = (2.0, -1.0)   # (D_s, D_p) of the extra channels, Ry
    s_core_ry: float = 40.0        # repulsive s channel of every atom's pseudopotential, Ry
    scf_kmesh: tuple | None = None # mesh of the self-consistent density (None: kmesh)
    steps: int = 300
    flavour: str = "ph"            # 'ph' pseudo-Hermitian | 'nh' non-Hermitian
    free_electron: bool = False    # V_ion = 0 and plane-wave occupations (Lindhard pins)
    symmetry: bool = False         # response k-points in the irreducible wedge of the small group of Q
    smearing_ry: float = 0.0       # Gaussian smearing width of a metal's occupations, Ry (0: insulator)
    electrons: float | None = None # valence electrons per cell of a metal (None: 2 nbnd, every band full)
    extra: dict = field(default_factory=dict)

    @property
    def omega(self) -> float:
        return float(abs(np.linalg.det(self.lattice)))

    @property
    def bvec(self) -> np.ndarray:
        return reciprocal(self.lattice)

    @property
    def nks(self) -> int:
        return int(np.prod(self.kmesh))

    @property
    def nelec(self) -> float:
        return 2.0 * self.nbnd if self.electrons is None else float(self.electrons)

    @property
    def metal(self) -> bool:
        return self.smearing_ry > 0.0

    @property
    def nproj(self) -> int:
        """Projectors per cell: s on every atom, plus p_x, p_y, p_z when kb is set."""
        if len(self.tau) == 0 or (not self.kb and self.s_core_ry == 0.0):
            return 0
        return len(self.tau) * (4 if self.kb else 1)


def _diamond(a: float) -> tuple[np.ndarray, np.ndarray]:
    lat = fcc_primitive(a)
    tau = np.array([[0.0, 0.0, 0.0], [0.25 * a, 0.25 * a, 0.25 * a]])
    return lat, tau


def config_small(symmetry: bool = False) -> SystemSpec:
    """Two-atom diamond-structure cell, 10 Ry, 18^3 grid, 4x4x4 mesh, Q = 0.1 (2pi/a) x,
    RPA+ALDA kernel, 300 pseudo-Hermitian steps, FP64.  symmetry: the irreducible k-points of
    the small group of Q."""
    lat, tau = _diamond(A_LAT)
    q = 0.1 * (2 * np.pi / A_LAT) * np.array([1.0, 0.0, 0.0])
    return SystemSpec("fcc2_10ry_18" + ("_ibz" if symmetry else ""), lat, tau, 4.0, 1.0, 10.0, 18, (4, 4, 4), 4, q,
                      approx="tddft", steps=300, flavour="ph", symmetry=symmetry)


def config_kb(symmetry: bool = False) -> SystemSpec:
    """Same cell and Q as config_small plus KB s/p projectors, 25 Ry, 32^3 grid,
    8x8x8 mesh, 1000 steps of either recursion.  symmetry: the k-points of the irreducible
    wedge of the small group of Q, with their weights (Sec. 2.6)."""
    lat, tau = _diamond(A_LAT)
    q = 0.1 * (2 * np.pi / A_LAT) * np.array([1.0, 0.0, 0.0])
    return SystemSpec("fcc2kb_25ry_32" + ("_ibz" if symmetry else ""), lat, tau, 4.0, 1.0, 25.0, 32, (8, 8, 8), 4, q,
                      approx="tddft", kb=True, scf_kmesh=(4, 4, 4), steps=1000, flavour="ph", symmetry=symmetry)


def _diamond_cubic(a: float) -> tuple[np.ndarray, np.ndarray]:
    """Conventional cubic cell of the diamond structure: 8 atoms."""
    fcc = np.array([[0.0, 0.0, 0.0], [0.0, 0.5, 0.5], [0.5, 0.0, 0.5], [0.5, 0.5, 0.0]])
    frac = np.concatenate([fcc, fcc + 0.25])
    return a * np.eye(3), frac * a


def config_cubic8(q_cart: np.ndarray | None = None) -> SystemSpec:
    """Eight-atom conventional cubic cell (Omega = 1080 bohr^3), 20 Ry, 32^3 grid, 4x4x4 mesh,
    16 bands (8 x 4 electrons / 2), no extra KB channels (the repulsive s channel of every
    atom still makes 8 projectors), Q = 0.1 (2 pi/a) x unless given.  The self-consistent
    density is converged on a 2x2x2 mesh."""
    lat, tau = _diamond_cubic(A_LAT)
    q = 0.1 * (2 * np.pi / A_LAT) * np.array([1.0, 0.0, 0.0]) if q_cart is None else np.asarray(q_cart, float)
    return SystemSpec("cubic8_20ry_32", lat, tau, 4.0, 1.0, 20.0, 32, (4, 4, 4), 16, q,
                      approx="tddft", scf_kmesh=(2, 2, 2), steps=1500, flavour="ph")


def config_sc16(q_cart: np.ndarray | None = None) -> SystemSpec:
    """Sixteen-atom cell: the 2x2x2 supercell of the two-atom primitive cell (Omega = 2160
    bohr^3, all sides 14.51 bohr), atoms displaced by N(0, 0.05 bohr) from default_rng(20211112)
    (shape (16, 3), atom-major), KB s/p projectors on every atom (64), 30 Ry, 48^3 grid,
    4x4x4 mesh, 32 bands, Q = 0.15 (2 pi/a)(1,1,0)/sqrt(2) unless given.  The self-consistent
    density is converged at Gamma (the supercell's Gamma folds the primitive 2x2x2 mesh), to
    1e-8 in the L1 density residual."""
    lat0, tau0 = _diamond(A_LAT)
    lat = 2.0 * lat0
    shifts = [i * lat0[0] + j * lat0[1] + k * lat0[2] for i in range(2) for j in range(2) for k in range(2)]
    tau = np.array([t + sh for sh in shifts for t in tau0])
    tau = tau + np.random.default_rng(20211112).normal(0.0, 0.05, size=(16, 3))
    q = (0.15 * (2 * np.pi / A_LAT) * np.array([1.0, 1.0, 0.0]) / np.sqrt(2.0) if q_cart is None
         else np.asarray(q_cart, float))
    return SystemSpec("sc16kb_30ry_48", lat, tau, 4.0, 1.0, 30.0, 48, (4, 4, 4), 32, q,
                      approx="tddft", kb=True, scf_kmesh=(1, 1, 1), steps=2000, flavour="ph",
                      extra={"scf_tol": 1e-8})


def config_metal(kmesh: tuple = (4, 4, 4)) -> SystemSpec:
    """The two-atom cell of config_small with its bare local potential only (no repulsive s
    channel: a semimetal), 8 valence electrons in 6 bands, Gaussian smearing 0.04 Ry, 10 Ry,
    18^3 grid, Q = 0.1 (2pi/a) x, RPA+ALDA kernel, 300 pseudo-Hermitian steps."""
    lat, tau = _diamond(A_LAT)
    q = 0.1 * (2 * np.pi / A_LAT) * np.array([1.0, 0.0, 0.0])
    return SystemSpec("fcc2metal_10ry_18", lat, tau, 4.0, 1.0, 10.0, 18, kmesh, 6, q,
                      approx="tddft", steps=300, flavour="ph", s_core_ry=0.0,
                      smearing_ry=0.04, electrons=8.0)


def config_tiny(kb: bool = False, approx: str = "tddft") -> SystemSpec:
    """A cell small enough for brute-force Casida diagonalisation: 4 Ry, 12^3, 2x2x2 k."""
    lat, tau = _diamond(A_LAT)
    q = 0.1 * (2 * np.pi / A_LAT) * np.array([1.0, 0.0, 0.0])
    return SystemSpec("fcc2_4ry_12" + ("kb" if kb else ""), lat, tau, 4.0, 1.0, 4.0, 12,
                      (2, 2, 2), 4, q, approx=approx, kb=kb, steps=60, flavour="ph")


def config_local_insulator() -> SystemSpec:
    """Local-potential-only insulator for the f-sum rule (exact only for local potentials):
    the tiny cell without projectors, its two deep s-like bands occupied."""
    s = config_tiny()
    s.name, s.s_core_ry, s.nbnd = "fcc2_4ry_12_local2", 0.0, 2
    return s


def config_free_electron(nk: int = 6, ecut: float = 3.0, nfft: int = 12,
                         qfrac: float = 1.0 / 6.0) -> SystemSpec:
    """Simple-cubic free-electron gas (V_ion = 0); Q = qfrac * b_1 commensurate with the mesh."""
    a = A_LAT
    lat = a * np.eye(3)
    q = qfrac * (2 * np.pi / a) * np.array([1.0, 0.0, 0.0])
    s = SystemSpec("feg", lat, np.zeros((0, 3)), 0.0, 1.0, ecut, nfft, (nk, nk, nk), 1, q,
                   approx="rpa", steps=200, flavour="ph", free_electron=True, s_core_ry=0.0)
    return s


CONFIGS = {"small": config_small, "kb": config_kb, "tiny": config_tiny, "cubic8": config_cubic8, "sc16": config_sc16,
           "metal": config_metal}


def sphere(kcart: np.ndarray, bvec: np.ndarray, ecut_ry: float, guard: float = 1e-9) -> np.ndarray:
    """Miller indices m (int32, shape (npw,3)) with |k + m.B|^2 <= ecut, lexicographic order.

    Raises if a point sits within `guard` (relative) of the cut-off, so that the
    membership decision cannot depend on rounding order."""
    kmax = np.sqrt(ecut_ry) + np.linalg.norm(kcart)
    lat = 2 * np.pi * np.linalg.inv(bvec).T          # rows a_i
    mmax = [int(np.ceil(kmax * np.linalg.norm(lat[i]) / (2 * np.pi))) + 1 for i in range(3)]
    r = [np.arange(-mm, mm + 1) for mm in mmax]
    m1, m2, m3 = np.meshgrid(*r, indexing="ij")
    m = np.stack([m1.ravel(), m2.ravel(), m3.ravel()], axis=1)
    kg = kcart[None, :] + m @ bvec
    g2 = np.einsum("ij,ij->i", kg, kg)
    near = np.abs(g2 - ecut_ry) <= guard * ecut_ry
    if np.any(near):
        raise ValueError(f"plane wave within {guard} of the cut-off at k={kcart}")
    sel = m[g2 <= ecut_ry]
    order = np.lexsort((sel[:, 2], sel[:, 1], sel[:, 0]))
    return np.ascontiguousarray(sel[order].astype(np.int32))


def point_operations() -> list[np.ndarray]:
    """The 48 orthogonal operations of the cube (signed permutation matrices), Cartesian."""
    import itertools
    ops = []
    for perm in itertools.permutations(range(3)):
        for signs in itertools.product((1, -1), repeat=3):
            r = np.zeros((3, 3))
            for i, j in enumerate(perm):
                r[i, j] = signs[i]
            ops.append(r)
    return ops


def small_group(spec: SystemSpec, tol: float = 1e-9) -> list[np.ndarray]:
    """The point operations R (Cartesian) of the crystal that need no fractional translation
    (R maps every atom onto an atom of the same kind, up to a lattice vector, so the local
    potential and the s/p projectors are invariant) and leave Q invariant (R Q = Q): the small
    group of Q used to reduce the k-points (Sec. 2.6).  Identity first."""
    lat = spec.lattice
    inv_lat = np.linalg.inv(lat)
    out = []
    for r in point_operations():
        if np.linalg.norm(r @ spec.q_cart - spec.q_cart) > tol * max(1.0, np.linalg.norm(spec.q_cart)):
            continue
        m = inv_lat.T @ r @ lat.T                 # the operation on fractional coordinates
        if np.max(np.abs(m - np.round(m))) > tol:
            continue
        ok = True
        for t in spec.tau:
            f = (r @ t) @ inv_lat                 # fractional coordinates of R tau
            if not any(np.max(np.abs((f - u @ inv_lat) - np.round(f - u @ inv_lat))) < tol for u in spec.tau):
                ok = False
                break
        if ok:
            out.append(r)
    out.sort(key=lambda r: 0 if np.allclose(r, np.eye(3)) else 1)
    return out


def grid_operations(spec: SystemSpec, ops: list[np.ndarray]) -> np.ndarray:
    """Integer matrices M (nsym, 3, 3) with R r_j = r_{M j} for the grid points r_j = sum_i
    (j_i / N) a_i: M = A^-T R A^T (A rows a_i), indices taken mod N."""
    lat = spec.lattice
    return np.array([np.round(np.linalg.inv(lat.T) @ r @ lat.T).astype(np.int32) for r in ops], dtype=np.int32)


def irreducible_kpoints(spec: SystemSpec, ops: list[np.ndarray]) -> tuple[np.ndarray, np.ndarray]:
    """The k-points of the Gamma-centred mesh reduced by the operations (each star R k of the
    mesh represented by its first member in mesh order) and their multiplicities (star sizes,
    summing to the mesh size).  Returns (kfrac (nirr, 3), multiplicity (nirr,))."""
    n = np.array(spec.kmesh)
    kf = kmesh_frac(tuple(n))
    bvec = spec.bvec
    inv_b = np.linalg.inv(bvec)
    index = {tuple(np.round(f * n).astype(int) % n): i for i, f in enumerate(kf)}
    seen = np.full(len(kf), -1)
    reps, mult = [], []
    for i, f in enumerate(kf):
        if seen[i] >= 0:
            continue
        star = set()
        for r in ops:
            g = ((r @ (f @ bvec)) @ inv_b) * n
            gi = np.round(g).astype(int)
            if np.max(np.abs(g - gi)) > 1e-6:
                raise ValueError("an operation does not map the k-mesh onto itself")
            star.add(index[tuple(gi % n)])
        for j in star:
            seen[j] = len(reps)
        reps.append(f)
        mult.append(len(star))
    return np.array(reps), np.array(mult, dtype=np.float64)


def fft_miller(n: int) -> np.ndarray:
    """Integer frequency of each grid index, numpy fftfreq order: 0..N/2-1, -N/2..-1."""
    return np.fft.fftfreq(n, 1.0 / n).astype(np.int64)
