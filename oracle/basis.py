"""Plane-wave spheres on the FFT grid (Sec. 2.3: lattice-periodic parts expanded in e^{iG.r}).

Conventions (fixed for the whole oracle):
  grid point r_j = sum_i (j_i/N) a_i,  array index [j1, j2, j3]
  psi(r_j) = sum_G c_G e^{i G.r_j}                  (no 1/N^3; u(r) = psi(r)/sqrt(Omega))
  f_G = (1/N^3) sum_j f(r_j) e^{-i G.r_j}
A Miller index m maps to the grid frequency index m mod N.
The 3D transforms are scipy.fft's (pocketfft, the same plain DFT definitions as numpy.fft).
"""
from __future__ import annotations

import numpy as np
import scipy.fft as sfft


def grid_index(miller: np.ndarray, n: int) -> np.ndarray:
    """Flat index of each Miller triplet in a C-ordered N^3 array."""
    m = np.asarray(miller, dtype=np.int64) % n
    return (m[:, 0] * n + m[:, 1]) * n + m[:, 2]


def to_grid(coef: np.ndarray, miller: np.ndarray, n: int) -> np.ndarray:
    """psi(r) = sum_G c_G e^{iG.r} for a batch coef (..., npw) -> (..., N, N, N)."""
    coef = np.asarray(coef)
    lead = coef.shape[:-1]
    g = np.zeros(lead + (n ** 3,), dtype=np.complex128)
    g[..., grid_index(miller, n)] = coef
    g = g.reshape(lead + (n, n, n))
    return sfft.ifftn(g, axes=(-3, -2, -1)) * n ** 3


def to_sphere(f: np.ndarray, miller: np.ndarray, n: int) -> np.ndarray:
    """f_G = (1/N^3) sum_j f(r_j) e^{-iG.r_j} at the sphere's G: (..., N, N, N) -> (..., npw)."""
    fg = sfft.fftn(f, axes=(-3, -2, -1)) / n ** 3
    lead = fg.shape[:-3]
    return fg.reshape(lead + (n ** 3,))[..., grid_index(miller, n)]


def intersection_map(miller_from: np.ndarray, miller_to: np.ndarray) -> np.ndarray:
    """For each Miller of `miller_to`, its position in `miller_from`, or -1 (int32)."""
    pos = {tuple(int(v) for v in m): i for i, m in enumerate(miller_from)}
    return np.array([pos.get(tuple(int(v) for v in m), -1) for m in miller_to], dtype=np.int32)


def columns(miller: np.ndarray) -> list[tuple[int, int, int, int]]:
    """Runs of equal (m1, m2) in a lexicographically ordered sphere: (m1, m2, start, count)."""
    out = []
    i = 0
    while i < len(miller):
        j = i
        while j < len(miller) and miller[j, 0] == miller[i, 0] and miller[j, 1] == miller[i, 1]:
            j += 1
        out.append((int(miller[i, 0]), int(miller[i, 1]), i, j - i))
        i = j
    return out
