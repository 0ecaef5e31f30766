"""Writes tests/golden/bench_refs.npz: FP64 reference values that bench.py
compares the GPU results against, computed by the oracle alone (this script
calls only oracle/ and the seeded input generators).

  python tests/golden/make_bench_refs.py

Contents
  matvec_rows, matvec_Y, matvec_L: 100 sampled rows (rng 11) of Kh V and
      dKh/dl V on the fused matvec problem (n = 1e5, d = 3, Matern-3/2,
      V = [y | 31 Rademacher], seed 0);
  precision_rows, precision_Y: 200 sampled rows (rng 3) of Kh V on the
      precision problem (n = 1e6, d = 2, Gaussian, V = [y | 63 Rademacher]);
  diff_loss, diff_grad: the same-probe SLQ / Hutchinson estimate of L and
      dL/d(s, f, l) on the n = 4000 differentiation subsample (32 probes from
      seed 77, 40 Lanczos steps).
"""
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)

import oracle as O  # noqa: E402
from paper_2503_02259_gb300 import inputs  # noqa: E402

OUT = os.path.join(HERE, "bench_refs.npz")


def matvec_refs():
    prob = inputs.matvec_problem(seed=0)
    V = inputs.multivector(prob.y, 32, seed=0)
    rows = np.sort(np.random.default_rng(11).choice(prob.n, 100, replace=False))
    Y, _, Lr = O.kmv_rows(prob.X, V, prob.kind, prob.theta, rows=rows, block=50)
    return rows, Y, Lr


def precision_refs():
    prob = inputs.precision_problem(seed=0)
    V = inputs.multivector(prob.y, 64, seed=0)
    rows = np.sort(np.random.default_rng(3).choice(prob.n, 200, replace=False))
    Y, _, _ = O.kmv_rows(prob.X, V, prob.kind, prob.theta, rows=rows, block=20)
    return rows, Y


def diff_refs():
    sub = inputs.diff_problem(seed=0, n=4000)
    est = O.est_nll(sub.X, sub.y, sub.kind, sub.theta, O.rademacher_probes(sub.n, 32, 77), 40)
    return float(est["loss"]), np.asarray(est["grad"], dtype=np.float64)


def main():
    mr, mY, mL = matvec_refs()
    pr, pY = precision_refs()
    dl, dg = diff_refs()
    np.savez_compressed(OUT, matvec_rows=mr, matvec_Y=mY, matvec_L=mL, precision_rows=pr,
                        precision_Y=pY, diff_loss=np.float64(dl), diff_grad=dg)
    print("wrote", OUT)


if __name__ == "__main__":
    main()
