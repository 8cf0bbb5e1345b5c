"""The two Lanczos recursions of Sec. 2.5, FP64, one operator application at a time.

Both start from the right-hand side of Eq. 23, (0, y), and produce a tridiagonal matrix
T_M with zero diagonal (each Lanczos vector has only one non-zero SBR half, and L maps an
upper-only vector to a lower-only one and back, so every alpha_j vanishes), plus
z_j = ((y, 0), v_j) (Eq. 31), accumulated on the fly.

Output convention (shared with the C ABI): after n steps
    beta[0]  = b_1 = the norm of the starting vector, beta[i] = T_{i+1,i}  (i >= 1)
    gamma[0] = b_1,                                    gamma[i] = T_{i,i+1}
    z[i] = z_{i+1}
so that chi ~ b_1 sum_j z_j [(omega - T)^-1]_{j1} (Eqs. 30, 32-33).

Non-Hermitian biorthogonal recursion (Sec. 2.5): right vectors v_j with L, left vectors
w_j with L^dagger = [[0, D+K], [D, 0]]; with s = (w_hat, v_hat):
    v_hat = L v_j - gamma_j v_{j-1},  w_hat = L^dag w_j - conj(beta_j) w_{j-1}
    beta_{j+1} = sqrt|s|,  gamma_{j+1} = s / beta_{j+1}
    v_{j+1} = v_hat / beta_{j+1},  w_{j+1} = w_hat / conj(gamma_{j+1}).
Two operator applications per step: D on one chain, D + K on the other.

Pseudo-Hermitian recursion (Sec. 2.5; the metric redefinition of the scalar product):
with eta = diag(D + K, D), eta L = L^dagger eta, so L is Hermitian in <a, b> = a^H eta b
(positive when D > 0 and D + K > 0, an insulator).  For a one-half vector, L v is the
half-swap of eta v, so a single application Op(r) = eta r per step gives both the norm
and the next L v:
    r_1 = (0, y), X_1 = D y, beta_1 = sqrt(Re y^H X_1)
    v_j = r_j / beta_j,  L v_j = swap(X_j) / beta_j
    r_{j+1} = L v_j - beta_j v_{j-1},  X_{j+1} = Op(r_{j+1})
    beta_{j+1} = sqrt(Re r_{j+1}^H X_{j+1})
T_M is symmetric (gamma = beta).  One operator application per step: twice as cheap.

Reading (both recursions): every new Lanczos vector is projected with P_c, like every
operator output.  In exact arithmetic this changes nothing; in floating point the
occupied-manifold components that rounding leaves in v_{j-1} lie in the null space of
D and of the metric, are never seen by the normalisation, and grow geometrically
(r_{j+1} inherits -beta_j/beta_{j-1} times them), breaking the pseudo-Hermitian recursion
after a few hundred steps.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np

from .liouvillian import System, axpy, scale


class Breakdown(RuntimeError):
    pass


@dataclass
class Coefficients:
    beta: np.ndarray     # (n,) float64 (non-Hermitian: complex beta is real by construction)
    gamma: np.ndarray    # (n,) complex128
    z: np.ndarray        # (n,) complex128
    applies: int         # operator applications used
    flavour: str

    @property
    def b1(self) -> float:
        return float(self.beta[0])


def pseudo_hermitian(sys: System, nsteps: int, breakdown_tol: float = 1e-28, on_step=None) -> Coefficients:
    """on_step(j), when given, is called once step j's coefficients are known (timing hook)."""
    y = sys.starting_vector()
    r, r_upper = y, False                        # r_1 = (0, y): lower half
    x = sys.apply_op(r, upper=False)             # X_1 = D y
    applies = 1
    if on_step:
        on_step(1)
    b2 = sys.inner(r, x).real
    if b2 <= 0:
        raise Breakdown("metric not positive at step 1")
    beta = [np.sqrt(b2)]
    z = []
    v_prev = None                                # v_{j-1}, same half as L v_j
    for j in range(1, nsteps + 1):
        bj = beta[-1]
        v = scale(1.0 / bj, r)                   # v_j (half r_upper)
        z.append(sys.inner(y, v) if r_upper else 0.0)
        if j == nsteps:
            break
        lv = scale(1.0 / bj, x)                  # L v_j, in the other half
        r_next = lv if v_prev is None else sys.project_c(axpy(-bj, v_prev, lv))
        v_prev, r, r_upper = v, r_next, not r_upper
        x = sys.apply_op(r, upper=r_upper)
        applies += 1
        b2 = sys.inner(r, x).real
        if b2 <= breakdown_tol * beta[0] ** 2:
            raise Breakdown(f"non-positive metric or breakdown at step {j + 1}: {b2:.3e}")
        beta.append(np.sqrt(b2))
        if on_step:
            on_step(j + 1)
    beta = np.array(beta)
    return Coefficients(beta=beta, gamma=beta.astype(np.complex128), z=np.array(z, dtype=np.complex128),
                        applies=applies, flavour="ph")


def non_hermitian(sys: System, nsteps: int, breakdown_tol: float = 1e-28, on_step=None) -> Coefficients:
    """on_step(j), when given, is called once step j's coefficients are known (timing hook)."""
    y = sys.starting_vector()
    b1 = np.sqrt(sys.inner(y, y).real)
    v = scale(1.0 / b1, y)                       # v_1 = w_1 = (0, y)/|y|: lower halves
    w = v
    upper = False                                # half of v_j and w_j
    v_prev = w_prev = None
    beta, gamma, z = [b1], [complex(b1)], []
    applies = 0
    for j in range(1, nsteps + 1):
        z.append(sys.inner(y, v) if upper else 0.0)
        if j == nsteps:
            break
        # L v_j and L^dag w_j land in the other half; L = [[0, D], [D+K, 0]],
        # L^dag = [[0, D+K], [D, 0]]: a lower v gets D, a lower w gets D+K, and vice versa.
        lv = sys.apply_op(v, upper=upper)
        lw = sys.apply_op(w, upper=not upper)
        applies += 2
        if v_prev is not None:
            lv = sys.project_c(axpy(-gamma[-1], v_prev, lv))
            lw = sys.project_c(axpy(-np.conj(beta[-1]), w_prev, lw))
        s = sys.inner(lw, lv)
        if abs(s) <= breakdown_tol * b1 ** 2:
            raise Breakdown(f"breakdown at step {j + 1}: |s| = {abs(s):.3e}")
        bn = np.sqrt(abs(s))
        gn = s / bn
        v_prev, w_prev = v, w
        v = scale(1.0 / bn, lv)
        w = scale(1.0 / np.conj(gn), lw)
        upper = not upper
        beta.append(bn)
        gamma.append(gn)
        if on_step:
            on_step(j + 1)
    return Coefficients(beta=np.array(beta, dtype=np.float64), gamma=np.array(gamma, dtype=np.complex128),
                        z=np.array(z, dtype=np.complex128), applies=applies, flavour="nh")


def run(sys: System, nsteps: int, flavour: str, on_step=None) -> Coefficients:
    return (pseudo_hermitian(sys, nsteps, on_step=on_step) if flavour == "ph"
            else non_hermitian(sys, nsteps, on_step=on_step))
