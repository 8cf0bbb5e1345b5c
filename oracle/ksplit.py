"""The operator and its scalar product split over ranks by blocks of k-points, FP64.

Test infrastructure, like the rest of `oracle/`: it pins the decomposition a multi-GPU
chain would use (the paper's k-point pools, Sec. 4).  Rank r of W holds the contiguous
block of k-points [k0, k1) of every batch vector.  D and P_c act on each k-point alone
(Eqs. 16, 25); the only sums over k are

  - the response density n'(r) = 4 (1/N_k) sum_{vk} u*_{vk}(r) x_{vk}(r) (Eq. 27), summed
    over ranks before v'_HXC is formed (one N^3 grid per D + K application), and
  - the scalar products (a, b) = (1/N_k) sum_{vk} a_{vk}^H b_{vk} of the recursions.

`allreduce(a)` returns the element-wise sum of the ndarray `a` over all ranks (for example
torch.distributed.all_reduce over gloo).  An object of this class has the methods the
recursions of `oracle.lanczos` call (starting_vector, apply_op, inner, project_c), so
those recursions run unchanged on the k-block of every rank.
"""
from __future__ import annotations

import numpy as np


def k_block(nks: int, rank: int, world: int) -> tuple[int, int]:
    """Contiguous block of k-points of `rank`: the first nks % world ranks take one more."""
    base, extra = divmod(nks, world)
    k0 = rank * base + min(rank, extra)
    return k0, k0 + base + (1 if rank < extra else 0)


class KSplit:
    def __init__(self, system, rank: int, world: int, allreduce):
        self.sys = system
        self.k0, self.k1 = k_block(system.nks, rank, world)
        self.ks = range(self.k0, self.k1)
        self.allreduce = allreduce
        self.nks = system.nks
        self.approx = system.approx

    def starting_vector(self):
        return self.sys.starting_vector()[self.k0:self.k1]

    def project_c(self, x):
        return self.sys.project_c(x, self.ks)

    def inner(self, a, b) -> complex:
        local = self.sys.inner_part(a, b, self.ks)
        tot = self.allreduce(np.array([complex(local).real, complex(local).imag]))
        return complex(tot[0], tot[1]) / self.sys.nfull

    def apply_op(self, x, upper: bool):
        d = self.sys.apply_d(x, self.ks)
        if not upper or self.approx == "ipa":
            return d
        part = self.sys.response_density(x, self.ks)
        nr = self.allreduce(np.stack([part.real, part.imag]))
        v = self.sys.hxc_potential(nr[0] + 1j * nr[1])
        kx = self.sys.apply_v(v, self.ks)
        return [a + b for a, b in zip(d, kx)]
