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
      seed 77, 40 Lanczos steps);
  serving_idx, serving_loss, serving_grad, serving_mu: for the first
      SERVING_COUNT requests with n <= SERVING_NMAX of the 512-request serving
      stream (seed 0), the same-probe estimate of L and dL/d(s, f, l) (16
      probes from seed 0, 20 Lanczos steps, exact solves) of the loss+grad
      requests and the posterior mean at the first 200 test points (exact
      solve) of the predictions; NaN where a field does not apply;
      serving_kappa: the condition number of each request's Kh (eigvalsh);
  preck_loss, preck_grad: the exact L and dL/d(s, f, l) (Cholesky) on the
      n = 4000 subsample of the precision problem (d = 2, Gaussian l = 0.05,
      s = 0.01), for the preconditioned-loss leg;
  diffx_loss, diffx_grad: the exact L and dL/d(s, f, l) (Cholesky) on the
      n = 4000 differentiation subsample, for its preconditioned arm.
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


def preck_refs():
    sub = inputs.precision_problem(seed=0, n=4000)
    ex = O.exact_nll(sub.X, sub.y, sub.kind, sub.theta)
    return float(ex["loss"]), np.asarray(ex["grad"], dtype=np.float64)


def diffx_refs():
    sub = inputs.diff_problem(seed=0, n=4000)
    ex = O.exact_nll(sub.X, sub.y, sub.kind, sub.theta)
    return float(ex["loss"]), np.asarray(ex["grad"], dtype=np.float64)


SERVING_NMAX = 3000
SERVING_COUNT = 24
SERVING_MU_POINTS = 200


def serving_selection():
    reqs = inputs.serving_stream(seed=0, count=512)
    idx = [i for i, r in enumerate(reqs) if r.problem.n <= SERVING_NMAX][:SERVING_COUNT]
    return reqs, np.asarray(idx, dtype=np.int64)


def serving_refs():
    reqs, idx = serving_selection()
    loss = np.full(len(idx), np.nan)
    grad = np.full((len(idx), 3), np.nan)
    mu = np.full((len(idx), SERVING_MU_POINTS), np.nan)
    kappa = np.empty(len(idx))
    for k, i in enumerate(idx):
        rq = reqs[i]
        p = rq.problem
        ev = np.linalg.eigvalsh(O.khat_dense(p.X, p.kind, p.theta))
        kappa[k] = ev[-1] / ev[0]
        if rq.kind == 0:
            est = O.est_nll(p.X, p.y, p.kind, p.theta, O.rademacher_probes(p.n, rq.nprobe, 0), 20)
            loss[k] = est["loss"]
            grad[k] = est["grad"]
        else:
            alpha = O.exact_nll(p.X, p.y, p.kind, p.theta)["alpha"]
            mu[k] = O.predict_mean(p.X, rq.Xstar[:SERVING_MU_POINTS], alpha, p.kind, p.theta)
    return idx, loss, grad, mu, kappa


def main():
    mr, mY, mL = matvec_refs()
    pr, pY = precision_refs()
    dl, dg = diff_refs()
    si, sl, sg, smu, sk = serving_refs()
    pl, pg = preck_refs()
    xl, xg = diffx_refs()
    np.savez_compressed(OUT, matvec_rows=mr, matvec_Y=mY, matvec_L=mL, precision_rows=pr,
                        precision_Y=pY, diff_loss=np.float64(dl), diff_grad=dg, serving_idx=si,
                        serving_loss=sl, serving_grad=sg, serving_mu=smu,
                        serving_kappa=sk, preck_loss=np.float64(pl), preck_grad=pg,
                        diffx_loss=np.float64(xl), diffx_grad=xg)
    print("wrote", OUT)


if __name__ == "__main__":
    main()
