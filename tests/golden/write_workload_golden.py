"""Writes the oracle's Lanczos coefficients on the benchmark workloads under tests/golden/
(run from the repository root: `python tests/golden/write_workload_golden.py [case ...]`).

Cases (the FP64 oracle, RPA + ALDA kernel, Sec. 2.5 recursions on the operators of Eqs.
24-28):
  kb_ph    two-atom cell + KB s/p projectors, 25 Ry, 32^3, 8x8x8 k, 4 bands: pseudo-Hermitian
  kb_nh    the same cell: non-Hermitian
  sc16_ph  sixteen-atom 2x2x2 supercell + KB, 30 Ry, 48^3, 4x4x4 k, 32 bands: pseudo-Hermitian
  metal_ph the two-atom semimetal (bare local potential), smeared occupations (Sec. 2.6),
           10 Ry, 18^3, 4x4x4 k, 6 bands: pseudo-Hermitian
  metal_nh the same cell: non-Hermitian

Each file holds b_1 and T_{j+1,j}, T_{j,j+1}, z_j per row and, in its header, the digest of
the ground-state bundle it was computed on (workloads.bundle_digest): the GPU parity tests
compare against the file only when their bundle has the same digest, and run the oracle
themselves otherwise.  The recursions run on every core of this machine through the k-point
split of oracle.pool (the k sums regrouped; the same coefficients to rounding).  Only
oracle/ and the seeded input generator are called.
"""
import argparse
import os
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import workloads as w          # noqa: E402
from oracle import pool        # noqa: E402

HERE = os.path.dirname(os.path.abspath(__file__))
CASES = {
    "kb_ph": (w.config_kb, "ph", 1000),
    "kb_nh": (w.config_kb, "nh", 1000),
    "sc16_ph": (w.config_sc16, "ph", 100),
    "metal_ph": (w.config_metal, "ph", 300),
    "metal_nh": (w.config_metal, "nh", 120),
}


def path(case: str) -> str:
    return os.path.join(HERE, f"oracle_{case}.txt")


def load(case: str):
    """(digest, steps, beta, gamma, z) of a stored case, or None when the file is absent."""
    p = path(case)
    if not os.path.exists(p):
        return None
    digest = None
    with open(p) as fh:
        for line in fh:
            if not line.startswith("#"):
                break
            if "bundle_digest:" in line:
                digest = line.split("bundle_digest:")[1].split()[0]
    a = np.loadtxt(p, ndmin=2)
    return digest, len(a), a[:, 1], a[:, 2] + 1j * a[:, 3], a[:, 4] + 1j * a[:, 5]


def write(case: str, steps: int | None = None, world: int | None = None) -> None:
    mk, flavour, default_steps = CASES[case]
    spec = mk()
    steps = steps or default_steps
    b = w.get_bundle(spec, verbose=True)
    digest = w.bundle_digest(b)
    del b
    t0 = time.perf_counter()
    co, _, used = pool.run(spec, steps, flavour, world=world)
    dt = time.perf_counter() - t0
    rows = np.column_stack([np.arange(steps), co.beta, co.gamma.real, co.gamma.imag, co.z.real, co.z.imag])
    head = (f"oracle coefficients: {spec.name}, {spec.approx}, {flavour}, {steps} steps, FP64 "
            f"(written by tests/golden/write_workload_golden.py)\n"
            f"bundle_digest: {digest}\n"
            f"oracle processes: {used} (k-point split), {dt:.0f} s\n"
            "columns: i, beta[i], Re gamma[i], Im gamma[i], Re z[i], Im z[i]  (index 0: b_1; Sec. 2.5)")
    np.savetxt(path(case), rows, fmt=["%d"] + ["%.17e"] * 5, header=head)
    print(f"{case}: {steps} steps in {dt:.0f} s on {used} processes -> {path(case)}", flush=True)


def redigest(case: str) -> None:
    """Rewrite only the bundle_digest line of a stored case (after a change of the digest's
    definition), from the cached bundle; the coefficients are left as they are."""
    mk, _, _ = CASES[case]
    digest = w.bundle_digest(w.get_bundle(mk()))
    with open(path(case)) as fh:
        lines = fh.readlines()
    lines = [f"# bundle_digest: {digest}\n" if ln.startswith("# bundle_digest:") else ln for ln in lines]
    with open(path(case), "w") as fh:
        fh.writelines(lines)
    print(f"{case}: digest {digest}")


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("cases", nargs="*", default=list(CASES))
    ap.add_argument("--steps", type=int, default=None)
    ap.add_argument("--world", type=int, default=None)
    ap.add_argument("--redigest", action="store_true", help="rewrite the digest lines only")
    args = ap.parse_args()
    for c in args.cases:
        if args.redigest:
            redigest(c)
        else:
            write(c, args.steps, args.world)


if __name__ == "__main__":
    main()
