"""Test helpers: a chain on the device built from a ground-state bundle."""
import numpy as np


def chain_from_bundle(b, approx=None, flavour="ph", precision="fp64", max_steps=400, stream=None):
    from paper_2111_06623_gb300 import ll
    s = b.spec
    return ll.Chain(lattice=s.lattice, nfft=s.nfft, kcart=b.kcart, miller_k=b.miller_k, miller_kq=b.miller_kq,
                    u_k=b.u_k, u_kq=b.u_kq, eps_k=b.eps_k, vloc_r=b.vloc_r, rho_r=b.rho_r, beta_kq=b.beta_kq,
                    dij=b.dij, q_cart=s.q_cart, approx=approx or s.approx, flavour=flavour,
                    precision=precision, max_steps=max_steps, stream=stream,
                    kweight=getattr(b, "kweight", None), sym=getattr(b, "sym", None),
                    **metal_args(b))


def metal_args(b):
    """The occupations of a metal's bundle for the descriptor (nothing for an insulator)."""
    if getattr(b, "occ_k", None) is None:
        return {}
    return dict(occ_k=b.occ_k, occ_kq=b.occ_kq, eps_kq=b.eps_kq)


def rel_batch(a, b):
    """max |a - b| / max |b| over a batch (list of arrays)."""
    num = max(np.max(np.abs(x - y)) for x, y in zip(a, b))
    den = max(np.max(np.abs(y)) for y in b)
    return num / den
