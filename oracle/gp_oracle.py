"""FP64 CPU oracle for the HiGP training-loop hot path.

TEST INFRASTRUCTURE ONLY.  Nothing on the product path may import, call or
execute this module: only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` use it.  It
shares no code, constant table or helper with the CUDA library and never
imports it.

Everything is plain NumPy/SciPy in float64.  Inputs arrive as float32 arrays
(the same bytes the GPU sees) and are upcast, so input rounding is not
counted as error.

Paper passages followed (HiGP, arXiv 2503.02259):
  * §Gaussian Processes: parameters Theta = (s, f, l), training points X,
    observations y, test points X*.
  * §Gaussian Processes, the NLL equation: L = 1/2 (y^T Kh^-1 y + log|Kh| +
    n log 2pi).
  * §Gaussian Processes, the gradient equation: dL/dtheta = 1/2 (-y^T Kh^-1
    dKh Kh^-1 y + tr(Kh^-1 dKh)).
  * §Gaussian Processes, PCG (Saad 2003) with M = I.
  * Eq. (1) / Eq. (2) with M = I: log|M| = 0 and tr(M^-1 dM) = 0; the
    remainders are estimated by stochastic Lanczos quadrature (Ubaru et al.
    2017) and the Hutchinson estimator.
  * Eq. (1) / Eq. (2) with a Nystrom preconditioner M = s I + B W^-1 B^T on a
    fixed pivot set (``nystrom_precond``, ``est_nll_precond``): log|M| and
    tr(M^-1 dM/dtheta) exactly, the remainders by SLQ on M^-1/2 Kh M^-1/2 and
    by the Hutchinson estimator, with probes z ~ N(0, M).
  * §Statement of Need: the on-the-fly MatVec evaluates kernel blocks and
    uses them immediately; semantically it is the dense product Kh @ V.

Readings where the paper is silent (the kernel formulas and the form of the
regularised matrix are not printed in the paper):
  * Kh = f^2 K_l + s I  (s is the noise variance, added as is).
  * Gaussian (RBF) kernel  k(r) = exp(-r^2 / (2 l^2))      (Rasmussen &
    Williams, the textbook the paper cites for GPs).
  * Matern-3/2 kernel      k(r) = (1 + sqrt(3) r / l) exp(-sqrt(3) r / l).
  * l is one isotropic length-scale; gradients are w.r.t. raw (s, f, l).
  * Probes are Rademacher +-1, unnormalised (||z||^2 = n), drawn by the
    counter-based rule in ``rademacher_probes``; the preconditioned estimator
    takes standard normal e1, e2 (``gaussian_probes``: the same hash, then the
    Box-Muller transform) and forms z = L e1 + sqrt(s) e2 ~ N(0, M).
  * The preconditioner's derivatives are taken with its pivot set held fixed
    (the greedy pivot choice is piecewise constant in Theta).

Parity status per function (pins live in tests/test_oracle_pins.py):
  every public function below is pinned against a closed form, a brute-force
  computation, a library routine or a finite difference; none is "parity
  unpinned".
"""
from __future__ import annotations

import math

import numpy as np
import scipy.linalg as sla

GAUSSIAN = 0
MATERN32 = 1

_SQRT3 = math.sqrt(3.0)
_M64 = (1 << 64) - 1


# ---------------------------------------------------------------------------
# Counter-based Rademacher probes (SplitMix64, Steele, Lea & Flood 2014).
# ---------------------------------------------------------------------------

def splitmix64_next(state: int) -> tuple[int, int]:
    """One step of SplitMix64: returns (new_state, output).

    Written from the published definition: the state advances by the golden
    gamma 0x9e3779b97f4a7c15 and the output is the state passed through the
    variant-13 style xor-shift-multiply finaliser (shifts 30, 27, 31).
    """
    state = (state + 0x9E3779B97F4A7C15) & _M64
    z = state
    z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & _M64
    z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & _M64
    return state, z ^ (z >> 31)


def probe_hash(seed: int, col: int, row: int) -> int:
    """h = first SplitMix64 output from state key = seed xor (col << 40) xor row."""
    key = (seed ^ ((col << 40) & _M64) ^ row) & _M64
    return splitmix64_next(key)[1]


def rademacher_probes(n: int, p: int, seed: int) -> np.ndarray:
    """Z in {+-1}^{n x p}: z_ic = +1 if the top bit of probe_hash(seed, c, i) is 0.

    Pure-integer loops over the definition; vectorised with uint64 NumPy
    arithmetic (wrap-around multiplication is the definition's mod 2^64).
    """
    rows = np.arange(n, dtype=np.uint64)
    Z = np.empty((n, p), dtype=np.float64)
    with np.errstate(over="ignore"):
        for c in range(p):
            key = np.uint64(seed & _M64) ^ np.uint64((c << 40) & _M64) ^ rows
            z = key + np.uint64(0x9E3779B97F4A7C15)
            z = (z ^ (z >> np.uint64(30))) * np.uint64(0xBF58476D1CE4E5B9)
            z = (z ^ (z >> np.uint64(27))) * np.uint64(0x94D049BB133111EB)
            z = z ^ (z >> np.uint64(31))
            Z[:, c] = np.where((z >> np.uint64(63)) == 0, 1.0, -1.0)
    return Z


def gaussian_probes(rows: int, p: int, seed: int) -> np.ndarray:
    """Standard normal values G (rows x p) from the same counter-based hash:
    for row i and column c, h1 = probe_hash(seed ^ 2^39, c, 2i) and
    h2 = probe_hash(seed ^ 2^39, c, 2i + 1) (bit 39 of the key keeps these keys
    apart from the Rademacher ones); u1 = (h1 // 2^11 + 1) 2^-53 in (0, 1],
    u2 = (h2 // 2^11) 2^-53 in [0, 1); G_ic = sqrt(-2 ln u1) cos(2 pi u2)
    (the Box-Muller transform, Box & Muller 1958)."""
    G = np.empty((rows, p))
    tag = (seed ^ (1 << 39)) & _M64
    for c in range(p):
        for i in range(rows):
            h1 = probe_hash(tag, c, 2 * i)
            h2 = probe_hash(tag, c, 2 * i + 1)
            u1 = ((h1 >> 11) + 1) * 2.0 ** -53
            u2 = (h2 >> 11) * 2.0 ** -53
            G[i, c] = math.sqrt(-2.0 * math.log(u1)) * math.cos(2.0 * math.pi * u2)
    return G


# ---------------------------------------------------------------------------
# Kernel entries (§Gaussian Processes; formulas per the readings above).
# ---------------------------------------------------------------------------

def sqdist(A: np.ndarray, B: np.ndarray) -> np.ndarray:
    """R2_ij = sum_t (a_it - b_jt)^2, in difference form (no norm expansion)."""
    A = np.asarray(A, dtype=np.float64)
    B = np.asarray(B, dtype=np.float64)
    R2 = np.zeros((A.shape[0], B.shape[0]))
    for t in range(A.shape[1]):
        diff = A[:, t][:, None] - B[:, t][None, :]
        R2 += diff * diff
    return R2


def kernel_value(r2: np.ndarray, kind: int, l: float) -> np.ndarray:
    """k(r; l) from the squared distance."""
    if kind == GAUSSIAN:
        return np.exp(-r2 / (2.0 * l * l))
    if kind == MATERN32:
        a = _SQRT3 * np.sqrt(r2) / l
        return (1.0 + a) * np.exp(-a)
    raise ValueError(kind)


def kernel_dl(r2: np.ndarray, kind: int, l: float) -> np.ndarray:
    """dk/dl at fixed r (the entries of D_l = dK/dl)."""
    if kind == GAUSSIAN:
        return np.exp(-r2 / (2.0 * l * l)) * r2 / (l ** 3)
    if kind == MATERN32:
        a = _SQRT3 * np.sqrt(r2) / l
        return a * a * np.exp(-a) / l
    raise ValueError(kind)


def khat_dense(X, kind: int, theta) -> np.ndarray:
    """Kh = f^2 K + s I, formed densely (small n only)."""
    s, f, l = theta
    R2 = sqdist(X, X)
    K = kernel_value(R2, kind, l)
    return f * f * K + s * np.eye(K.shape[0])


def dkhat_dense(X, kind: int, theta):
    """(dKh/ds, dKh/df, dKh/dl) = (I, 2 f K, f^2 D_l), formed densely."""
    s, f, l = theta
    R2 = sqdist(X, X)
    K = kernel_value(R2, kind, l)
    D = kernel_dl(R2, kind, l)
    return np.eye(K.shape[0]), 2.0 * f * K, f * f * D


def kmv_rows(X, V, kind: int, theta, rows=None, block: int = 256):
    """Rows of (Kh V, dKh/df V, dKh/dl V) evaluated on the fly in FP64.

    Semantics of the on-the-fly MatVec (§Statement of Need): the product with
    the dense matrix, built block by block and discarded.  ``rows`` selects
    output rows (all by default); dKh/ds V is V itself and is not returned.
    """
    s, f, l = theta
    X = np.asarray(X, dtype=np.float64)
    V = np.asarray(V, dtype=np.float64)
    if V.ndim == 1:
        V = V[:, None]
    rows = np.arange(X.shape[0]) if rows is None else np.asarray(rows)
    Y = np.empty((rows.size, V.shape[1]))
    dYf = np.empty_like(Y)
    dYl = np.empty_like(Y)
    for b0 in range(0, rows.size, block):
        r = rows[b0:b0 + block]
        R2 = sqdist(X[r], X)
        KV = kernel_value(R2, kind, l) @ V
        DV = kernel_dl(R2, kind, l) @ V
        Y[b0:b0 + block] = f * f * KV + s * V[r]
        dYf[b0:b0 + block] = 2.0 * f * KV
        dYl[b0:b0 + block] = f * f * DV
    return Y, dYf, dYl


def cross_kmv(XA, XB, V, kind: int, theta, block: int = 256):
    """f^2 K(XA, XB) V: the noise-free cross-covariance product (prediction)."""
    s, f, l = theta
    XA = np.asarray(XA, dtype=np.float64)
    V = np.asarray(V, dtype=np.float64)
    if V.ndim == 1:
        V = V[:, None]
    out = np.empty((XA.shape[0], V.shape[1]))
    for b0 in range(0, XA.shape[0], block):
        R2 = sqdist(XA[b0:b0 + block], XB)
        out[b0:b0 + block] = f * f * (kernel_value(R2, kind, l) @ V)
    return out


def predict_mean(X, Xstar, alpha, kind: int, theta) -> np.ndarray:
    """Posterior mean mu* = f^2 K(X*, X) alpha (noise-free test outputs, §Gaussian Processes)."""
    return cross_kmv(Xstar, X, alpha, kind, theta)[:, 0]


def predict_var(X, Xstar, kind: int, theta) -> np.ndarray:
    """Posterior variance of the noise-free test outputs y* (§Gaussian Processes:
    y* and the noisy y are jointly Gaussian, Cov(y*) = f^2 K(X*, X*),
    Cov(y, y*) = f^2 K(X, X*), Cov(y) = Kh).  Conditioning on y gives, per test
    point c with k_c = f^2 K(X, x*_c):

        var_c = f^2 k(0) - k_c^T Kh^-1 k_c,   k(0) = 1 for both kernels,

    with Kh^-1 k_c by a Cholesky solve.
    """
    s, f, l = theta
    X = np.asarray(X, dtype=np.float64)
    Xs = np.asarray(Xstar, dtype=np.float64)
    Kc = f * f * kernel_value(sqdist(X, Xs), kind, l)          # n x m
    U = sla.cho_solve(sla.cho_factor(khat_dense(X, kind, theta)), Kc)
    return f * f - np.einsum("ij,ij->j", Kc, U)


# ---------------------------------------------------------------------------
# O-exact: the NLL and its gradient by Cholesky.
# ---------------------------------------------------------------------------

def exact_nll(X, y, kind: int, theta) -> dict:
    """L(Theta) and dL/d(s, f, l) by their definitions, through Cholesky.

    L = 1/2 (y^T alpha + log|Kh| + n log 2pi),  alpha = Kh^-1 y;
    g_theta = 1/2 (-alpha^T dKh alpha + sum_ij (Kh^-1)_ij (dKh)_ji).
    """
    y = np.asarray(y, dtype=np.float64)
    n = y.size
    Kh = khat_dense(X, kind, theta)
    C = sla.cho_factor(Kh, lower=True)
    alpha = sla.cho_solve(C, y)
    logdet = 2.0 * np.sum(np.log(np.diag(C[0])))
    loss = 0.5 * (y @ alpha + logdet + n * math.log(2.0 * math.pi))
    Kinv = sla.cho_solve(C, np.eye(n))
    grad = np.empty(3)
    quad = np.empty(3)
    trace = np.empty(3)
    for t, dK in enumerate(dkhat_dense(X, kind, theta)):
        quad[t] = alpha @ (dK @ alpha)
        trace[t] = np.sum(Kinv * dK.T)
        grad[t] = 0.5 * (-quad[t] + trace[t])
    return {"loss": loss, "grad": grad, "alpha": alpha, "logdet": logdet,
            "quad": quad, "trace": trace, "yalpha": float(y @ alpha)}


# ---------------------------------------------------------------------------
# Per-dimension length-scales (ARD): the "kernel parameters l" of §Gaussian
# Processes taken as one length-scale per coordinate, l = (l_1, ..., l_d).
# The kernel sees the scaled squared distance rho^2 = sum_t (x_t - y_t)^2 / l_t^2:
#   Gaussian    k = exp(-rho^2 / 2),
#   Matern-3/2  k = (1 + a) exp(-a),  a = sqrt(3) rho,
# and dk/dl_t = k (x_t - y_t)^2 / l_t^3 (Gaussian), 3 (x_t - y_t)^2 exp(-a) / l_t^3
# (Matern-3/2).  Theta = (s, f, l_1..l_d); gradients are w.r.t. those raw values.
# ---------------------------------------------------------------------------

def sqdist_ard(A, B, ls) -> np.ndarray:
    """rho2_ij = sum_t (a_it - b_jt)^2 / l_t^2, in difference form."""
    A = np.asarray(A, dtype=np.float64)
    B = np.asarray(B, dtype=np.float64)
    R2 = np.zeros((A.shape[0], B.shape[0]))
    for t in range(A.shape[1]):
        diff = A[:, t][:, None] - B[:, t][None, :]
        R2 += diff * diff / (ls[t] * ls[t])
    return R2


def kernel_ard(A, B, kind: int, ls) -> np.ndarray:
    """K_ij = k(rho_ij) with per-dimension length-scales."""
    rho2 = sqdist_ard(A, B, ls)
    if kind == GAUSSIAN:
        return np.exp(-rho2 / 2.0)
    if kind == MATERN32:
        a = _SQRT3 * np.sqrt(rho2)
        return (1.0 + a) * np.exp(-a)
    raise ValueError(kind)


def kernel_dls(A, B, kind: int, ls) -> list:
    """[dK/dl_1, ..., dK/dl_d] at fixed points."""
    A = np.asarray(A, dtype=np.float64)
    B = np.asarray(B, dtype=np.float64)
    rho2 = sqdist_ard(A, B, ls)
    if kind == GAUSSIAN:
        E = np.exp(-rho2 / 2.0)
    elif kind == MATERN32:
        E = 3.0 * np.exp(-_SQRT3 * np.sqrt(rho2))
    else:
        raise ValueError(kind)
    out = []
    for t in range(A.shape[1]):
        diff = A[:, t][:, None] - B[:, t][None, :]
        out.append(E * diff * diff / ls[t] ** 3)
    return out


def khat_dense_ard(X, kind: int, s: float, f: float, ls) -> np.ndarray:
    """Kh = f^2 K + s I with per-dimension length-scales."""
    K = kernel_ard(X, X, kind, ls)
    return f * f * K + s * np.eye(K.shape[0])


def dkhat_dense_ard(X, kind: int, s: float, f: float, ls) -> list:
    """[dKh/ds, dKh/df, dKh/dl_1, ..., dKh/dl_d] = [I, 2 f K, f^2 dK/dl_t ...]."""
    K = kernel_ard(X, X, kind, ls)
    return [np.eye(K.shape[0]), 2.0 * f * K] + [f * f * D for D in kernel_dls(X, X, kind, ls)]


def exact_nll_ard(X, y, kind: int, s: float, f: float, ls) -> dict:
    """L and dL/d(s, f, l_1, ..., l_d) by Cholesky (the NLL and gradient
    equations of §Gaussian Processes with Theta = (s, f, l_1..l_d))."""
    y = np.asarray(y, dtype=np.float64)
    n = y.size
    Kh = khat_dense_ard(X, kind, s, f, ls)
    C = sla.cho_factor(Kh, lower=True)
    alpha = sla.cho_solve(C, y)
    logdet = 2.0 * np.sum(np.log(np.diag(C[0])))
    loss = 0.5 * (y @ alpha + logdet + n * math.log(2.0 * math.pi))
    Kinv = sla.cho_solve(C, np.eye(n))
    dKs = dkhat_dense_ard(X, kind, s, f, ls)
    quad = np.array([alpha @ (dK @ alpha) for dK in dKs])
    trace = np.array([np.sum(Kinv * dK.T) for dK in dKs])
    return {"loss": loss, "grad": 0.5 * (-quad + trace), "alpha": alpha, "logdet": logdet,
            "quad": quad, "trace": trace, "yalpha": float(y @ alpha)}


def est_nll_ard(X, y, kind: int, s: float, f: float, ls, Z: np.ndarray, k: int) -> dict:
    """The same-probe estimator with per-dimension length-scales: SLQ for log|Kh|,
    Hutchinson with exact solves for the traces (Eq. 1, Eq. 2 with M = I)."""
    y = np.asarray(y, dtype=np.float64)
    n = y.size
    Kh = khat_dense_ard(X, kind, s, f, ls)
    dKs = dkhat_dense_ard(X, kind, s, f, ls)
    C = sla.cho_factor(Kh, lower=True)
    alpha = sla.cho_solve(C, y)
    logdet, _ = slq_logdet(Kh, Z, k)
    U = sla.cho_solve(C, Z)
    trace = np.array([np.mean(np.sum(U * (dK @ Z), axis=0)) for dK in dKs])
    quad = np.array([alpha @ (dK @ alpha) for dK in dKs])
    loss = 0.5 * (y @ alpha + logdet + n * math.log(2.0 * math.pi))
    return {"loss": loss, "grad": 0.5 * (-quad + trace), "alpha": alpha, "logdet": logdet,
            "quad": quad, "trace": trace, "yalpha": float(y @ alpha)}


# ---------------------------------------------------------------------------
# O-est: SLQ log-det and Hutchinson traces with given probes.
# ---------------------------------------------------------------------------

def lanczos(A: np.ndarray, z: np.ndarray, k: int, btol: float = 1e-14):
    """k Lanczos steps on symmetric A from q1 = z/||z||, full reorthogonalisation.

    Returns the diagonal a[0..m-1] and off-diagonal b[0..m-2] of T_m, m <= k;
    the run stops early when b_j < btol * ||T|| (an invariant subspace).
    """
    n = A.shape[0]
    Q = np.zeros((n, k))
    a = []
    b = []
    q = z / np.linalg.norm(z)
    q_prev = np.zeros(n)
    beta_prev = 0.0
    tnorm = 0.0
    for j in range(k):
        Q[:, j] = q
        w = A @ q
        aj = q @ w
        w = w - aj * q - beta_prev * q_prev
        for _ in range(2):  # full reorthogonalisation against q_1..q_j
            w = w - Q[:, :j + 1] @ (Q[:, :j + 1].T @ w)
        a.append(aj)
        bj = np.linalg.norm(w)
        tnorm = max(tnorm, abs(aj) + bj + beta_prev)
        if j == k - 1 or bj < btol * tnorm:
            break
        b.append(bj)
        q_prev, q, beta_prev = q, w / bj, bj
    return np.array(a), np.array(b)


def gauss_quadrature_log(a: np.ndarray, b: np.ndarray, znorm2: float) -> float:
    """||z||^2 * e1^T log(T) e1 = ||z||^2 sum_j U_1j^2 log(lambda_j) (Gauss rule from T)."""
    if a.size == 1:
        return znorm2 * math.log(a[0])
    lam, U = sla.eigh_tridiagonal(a, b)
    return znorm2 * float(np.sum(U[0, :] ** 2 * np.log(lam)))


def slq_logdet(A: np.ndarray, Z: np.ndarray, k: int):
    """Stochastic Lanczos quadrature: mean over probes of ||z||^2 e1^T log(T_k) e1.

    Returns (estimate, per-probe values).
    """
    vals = np.array([gauss_quadrature_log(*lanczos(A, Z[:, i], k), Z[:, i] @ Z[:, i])
                     for i in range(Z.shape[1])])
    return float(vals.mean()), vals


def hutchinson_traces(Kh: np.ndarray, dKs, Z: np.ndarray):
    """tr(Kh^-1 dK) ~ mean_i (Kh^-1 z_i)^T (dK z_i), exact solves (Eq. 2, M = I).

    Returns (estimates[3], per-probe values [3, p]).
    """
    C = sla.cho_factor(Kh, lower=True)
    U = sla.cho_solve(C, Z)
    vals = np.array([np.sum(U * (dK @ Z), axis=0) for dK in dKs])
    return vals.mean(axis=1), vals


def est_nll(X, y, kind: int, theta, Z: np.ndarray, k: int) -> dict:
    """The estimator the GPU computes, in FP64 with exact solves and the same probes.

    L~ = 1/2 (y^T alpha + logdet_SLQ + n log 2pi);
    g~_theta = 1/2 (-alpha^T dKh alpha + tr~_theta).
    """
    y = np.asarray(y, dtype=np.float64)
    n = y.size
    Kh = khat_dense(X, kind, theta)
    dKs = dkhat_dense(X, kind, theta)
    C = sla.cho_factor(Kh, lower=True)
    alpha = sla.cho_solve(C, y)
    logdet, ld_vals = slq_logdet(Kh, Z, k)
    tr, tr_vals = hutchinson_traces(Kh, dKs, Z)
    quad = np.array([alpha @ (dK @ alpha) for dK in dKs])
    grad = 0.5 * (-quad + tr)
    loss = 0.5 * (y @ alpha + logdet + n * math.log(2.0 * math.pi))
    return {"loss": loss, "grad": grad, "alpha": alpha, "logdet": logdet,
            "logdet_probes": ld_vals, "trace": tr, "trace_probes": tr_vals,
            "quad": quad, "yalpha": float(y @ alpha)}


# ---------------------------------------------------------------------------
# O-pcg: plain CG, M = I, x0 = 0 (§Gaussian Processes, PCG).
# ---------------------------------------------------------------------------

def cg(A: np.ndarray, B: np.ndarray, rtol: float, maxit: int):
    """Column-wise CG on A X = B from X = 0, stopping each column at
    ||r||_2 / ||b||_2 <= rtol (recurrence residual) or at maxit iterations.

    Returns (X, iterations per column, relres per column, alphas, betas) where
    alphas[c] / betas[c] list the CG step coefficients of column c.
    """
    B = np.asarray(B, dtype=np.float64)
    if B.ndim == 1:
        B = B[:, None]
    n, w = B.shape
    Xs = np.zeros((n, w))
    iters = np.zeros(w, dtype=int)
    relres = np.zeros(w)
    alphas, betas = [], []
    for c in range(w):
        b = B[:, c]
        bn = np.linalg.norm(b)
        x = np.zeros(n)
        r = b.copy()
        p = r.copy()
        rr = r @ r
        al, be = [], []
        it = 0
        while it < maxit and math.sqrt(rr) > rtol * bn:
            q = A @ p
            alpha = rr / (p @ q)
            x += alpha * p
            r -= alpha * q
            rr_new = r @ r
            beta = rr_new / rr
            al.append(alpha)
            be.append(beta)
            p = r + beta * p
            rr = rr_new
            it += 1
        Xs[:, c] = x
        iters[c] = it
        relres[c] = math.sqrt(rr) / bn if bn > 0 else 0.0
        alphas.append(np.array(al))
        betas.append(np.array(be))
    return Xs, iters, relres, alphas, betas


def lanczos_from_cg(alphas: np.ndarray, betas: np.ndarray, k: int):
    """T_k of the Lanczos process hidden in CG (the CG/Lanczos correspondence).

    diag_0 = 1/alpha_0; diag_j = 1/alpha_j + beta_{j-1}/alpha_{j-1};
    off_j = sqrt(beta_j)/alpha_j.  Uses the first min(k, len(alphas)) steps.
    """
    m = min(k, alphas.size)
    a = np.empty(m)
    b = np.empty(max(m - 1, 0))
    for j in range(m):
        a[j] = 1.0 / alphas[j] + (betas[j - 1] / alphas[j - 1] if j > 0 else 0.0)
        if j < m - 1:
            b[j] = math.sqrt(betas[j]) / alphas[j]
    return a, b


# ---------------------------------------------------------------------------
# Preconditioned CG (§Gaussian Processes: PCG with M ~ Kh).  M is the Nystrom
# approximation of f^2 K on landmark points chosen by greedy pivoting -- the
# rank-k partial pivoted Cholesky factor L of f^2 K (so f^2 K ~ L L^T, the
# Nystrom form K_{:,P} K_{P,P}^-1 K_{P,:} on the pivots P) -- plus the noise:
#     M = L L^T + s I,
# applied through the Woodbury identity
#     M^-1 v = (v - L (s I_k + L^T L)^-1 L^T v) / s.
# This is the low-rank (Nystrom) part of the AFN preconditioner the paper
# uses (Zhao et al. 2024), without AFN's sparse factor for the Schur
# complement and with the rank k given, not chosen adaptively.
# ---------------------------------------------------------------------------

def pivoted_cholesky(A: np.ndarray, k: int, tol: float = 0.0, pivot_dtype=np.float64,
                     pivots=None):
    """Rank-k partial Cholesky of the SPD matrix A with greedy diagonal pivoting.

    Step j takes the pivot p_j = argmax_i d_i of the residual diagonal
    d = diag(A - L L^T) (the smallest index among equal values; the argmax is
    taken over d rounded to pivot_dtype), stops early if d_{p_j} <= tol, and
    sets L[:, j] = (A[:, p_j] - L[:, :j] L[p_j, :j]^T) / sqrt(d_{p_j}).
    Returns (L (n x m), pivots (m,), residual diagonal d), m <= k.
    `pivots` (optional) replaces the greedy choice by a given sequence (the
    factor of another implementation is then checked on its own pivots).
    """
    A = np.asarray(A, dtype=np.float64)
    n = A.shape[0]
    L = np.zeros((n, k))
    d = np.diag(A).copy()
    piv = []
    for j in range(k):
        if pivots is not None:
            if j >= len(pivots):
                break
            p = int(pivots[j])
        else:
            p = int(np.argmax(d.astype(pivot_dtype)))
        if not d[p] > tol:
            break
        col = (A[:, p] - L[:, :j] @ L[p, :j]) / math.sqrt(d[p])
        L[:, j] = col
        d -= col * col
        d[p] = 0.0
        piv.append(p)
    m = len(piv)
    return L[:, :m], np.array(piv, dtype=np.int64), d


def nystrom_apply_inverse(L: np.ndarray, s: float, V: np.ndarray) -> np.ndarray:
    """(L L^T + s I)^-1 V by the Woodbury identity, with a Cholesky solve of the
    k x k matrix s I + L^T L."""
    V = np.asarray(V, dtype=np.float64)
    C = s * np.eye(L.shape[1]) + L.T @ L
    T = sla.cho_solve(sla.cho_factor(C), L.T @ V)
    return (V - L @ T) / s


def pcg(A: np.ndarray, B: np.ndarray, apply_minv, rtol: float, maxit: int):
    """Column-wise preconditioned CG on A X = B from X = 0 (Saad 2003, Alg. 9.1):
    z = M^-1 r, p = z; alpha = r^T z / p^T A p; x += alpha p; r -= alpha A p;
    z' = M^-1 r'; beta = r'^T z' / r^T z; p = z' + beta p.  Stops each column
    at ||r||_2 / ||b||_2 <= rtol (recurrence residual) or at maxit iterations.
    Returns (X, iterations per column, relres per column)."""
    B = np.asarray(B, dtype=np.float64)
    if B.ndim == 1:
        B = B[:, None]
    n, w = B.shape
    Xs = np.zeros((n, w))
    iters = np.zeros(w, dtype=int)
    relres = np.zeros(w)
    for c in range(w):
        b = B[:, c]
        bn = np.linalg.norm(b)
        x = np.zeros(n)
        r = b.copy()
        z = apply_minv(r[:, None])[:, 0]
        p = z.copy()
        rz = r @ z
        it = 0
        while it < maxit and np.linalg.norm(r) > rtol * bn:
            q = A @ p
            alpha = rz / (p @ q)
            x += alpha * p
            r -= alpha * q
            z = apply_minv(r[:, None])[:, 0]
            rz_new = r @ z
            p = z + (rz_new / rz) * p
            rz = rz_new
            it += 1
        Xs[:, c] = x
        iters[c] = it
        relres[c] = np.linalg.norm(r) / bn if bn > 0 else 0.0
    return Xs, iters, relres


# ---------------------------------------------------------------------------
# Eq. (1) / Eq. (2) with a Nystrom preconditioner on a fixed pivot set.
# ---------------------------------------------------------------------------

def nystrom_precond(X, kind: int, theta, piv):
    """M = s I + B W^-1 B^T, the Nystrom preconditioner on the pivot set P:
    A = f^2 K, B = A[:, P], W = A[P, P].  With P held fixed its derivatives are
      dM/ds = I,   dM/df = (2/f) B W^-1 B^T,
      dM/dl = B' W^-1 B^T + B W^-1 B'^T - B W^-1 W' W^-1 B^T,
    with B' = dB/dl and W' = dW/dl (f^2 times the dk/dl entries).
    Returns (M, [dM/ds, dM/df, dM/dl])."""
    s, f, l = theta
    X = np.asarray(X, dtype=np.float64)
    P = np.asarray(piv, dtype=int)
    n = X.shape[0]
    R2 = sqdist(X, X[P])
    B = f * f * kernel_value(R2, kind, l)
    Bd = f * f * kernel_dl(R2, kind, l)
    W = B[P, :]
    Wd = Bd[P, :]
    G = np.linalg.solve(W, B.T)          # W^-1 B^T
    N = B @ G
    N = 0.5 * (N + N.T)
    T = Bd @ G
    dl = T + T.T - G.T @ Wd @ G
    return s * np.eye(n) + N, [np.eye(n), (2.0 / f) * N, 0.5 * (dl + dl.T)]


def _inv_sqrt_spd(M: np.ndarray) -> np.ndarray:
    lam, U = np.linalg.eigh(M)
    return (U / np.sqrt(lam)) @ U.T


def est_nll_precond(X, y, kind: int, theta, piv, E1: np.ndarray, E2: np.ndarray, k: int) -> dict:
    """The preconditioned estimator: Eq. (1) and Eq. (2) with the Nystrom M on
    the pivots piv, exact solves, and probes z_i = L e1_i + sqrt(s) e2_i
    (L the partial Cholesky factor on piv, so L L^T = B W^-1 B^T and z_i ~ N(0, M)
    for standard normal e1 (r x p) and e2 (n x p)):
      log|Kh| ~ log|M| + mean_i ||zh_i||^2 e1^T log(T_i) e1,
        zh_i = M^-1/2 z_i, T_i from k Lanczos steps on M^-1/2 Kh M^-1/2 from zh_i;
      tr(Kh^-1 dKh) ~ tr(M^-1 dM) + mean_i [(Kh^-1 z_i)^T dKh (M^-1 z_i)
                                             - (M^-1 z_i)^T dM (M^-1 z_i)],
    the second an unbiased estimate of tr(Kh^-1 dKh - M^-1 dM) because
    E[z z^T] = M.  Loss and gradient then as in est_nll."""
    s, f, l = theta
    y = np.asarray(y, dtype=np.float64)
    n = y.size
    Kh = khat_dense(X, kind, theta)
    dKs = dkhat_dense(X, kind, theta)
    A = f * f * kernel_value(sqdist(X, X), kind, l)
    L, _, _ = pivoted_cholesky(A, len(piv), pivots=piv)
    Z = L @ np.asarray(E1, dtype=np.float64) + math.sqrt(s) * np.asarray(E2, dtype=np.float64)
    M, dMs = nystrom_precond(X, kind, theta, piv)
    logdet_M = float(np.linalg.slogdet(M)[1])
    trM = np.array([np.trace(np.linalg.solve(M, dM)) for dM in dMs])
    Mis = _inv_sqrt_spd(M)
    Ah = Mis @ Kh @ Mis
    Zh = Mis @ Z
    ld_vals = np.array([gauss_quadrature_log(*lanczos(Ah, Zh[:, i], k), Zh[:, i] @ Zh[:, i])
                        for i in range(Z.shape[1])])
    C = sla.cho_factor(Kh, lower=True)
    alpha = sla.cho_solve(C, y)
    U = sla.cho_solve(C, Z)
    V = np.linalg.solve(M, Z)
    corr = np.array([np.sum(U * (dK @ V), axis=0) - np.sum(V * (dM @ V), axis=0)
                     for dK, dM in zip(dKs, dMs)])
    tr = trM + corr.mean(axis=1)
    quad = np.array([alpha @ (dK @ alpha) for dK in dKs])
    logdet = logdet_M + float(ld_vals.mean())
    loss = 0.5 * (y @ alpha + logdet + n * math.log(2.0 * math.pi))
    return {"loss": loss, "grad": 0.5 * (-quad + tr), "logdet": logdet, "logdet_M": logdet_M,
            "logdet_probes": ld_vals, "trace": tr, "trace_M": trM, "trace_corr": corr,
            "quad": quad, "yalpha": float(y @ alpha), "Z": Z, "L": L}
