"""Seeded synthetic inputs shared by the tests, the bench and the oracle checks.

This module only builds input matrices; it holds none of the projection
method's arithmetic.  Every matrix is A = U diag(lam) U^T with U a product of
Householder reflectors H_t = I - 2 v_t v_t^T / (v_t^T v_t) built from Gaussian
vectors, formed in FP64 and rounded to FP32 once; that FP32 matrix is the
input both the CUDA path and the oracle see.  Because U is known, the exact
projection U diag(max(lam,0)) U^T (Thm 1) is known in closed form.

Recipes (seeds: U from seed_u, eigenvalues from seed_lam, both numpy PCG64):

* ``spectrum_small``   n=1000: 40 eigenvalues U[1,10], 960 N(0, 0.05^2).
* ``spectrum_decay``   n=20000 (any n >= 500): 200 positives decaying
  geometrically from 100 to 0.1, 300 negatives U[-5,-0.1], rest N(0, 0.01^2).
* ``spectrum_batch``   batched / served matrices: 10% U[0.5,5], rest
  N(0, 0.1^2) (10% rounded half-up).
* ``spectrum_cor3``    the block spectrum of Cor. 3 (quarters -b1, -b2, b3, b4).
* ``sdls_problem``     C, A_i, b of the semidefinite least-squares example
  (Sec. 6), the input of the dual gradient descent of Alg. 6.

Eigenvalues are placed on the diagonal in generation order before U is
applied (positives, negatives, noise).
"""
from __future__ import annotations

import math

import numpy as np


def round_half_up(x: float) -> int:
    """[a] of the notation section: round to nearest, halves upward."""
    return int(math.floor(x + 0.5))


def householder_vectors(n: int, r: int, seed: int) -> np.ndarray:
    """r Gaussian reflector vectors (rows), numpy PCG64 stream `seed`."""
    return np.random.default_rng(seed).standard_normal((r, n))


def spectrum_small(n: int = 1000, seed: int = 2) -> np.ndarray:
    rng = np.random.default_rng(seed)
    npos = min(40, n)
    return np.concatenate([rng.uniform(1.0, 10.0, npos),
                           rng.normal(0.0, 0.05, n - npos)])


def spectrum_decay(n: int = 20000, seed: int = 2) -> np.ndarray:
    rng = np.random.default_rng(seed)
    npos, nneg = 200, 300
    assert n >= npos + nneg
    i = np.arange(npos, dtype=np.float64)
    pos = 100.0 * (1e-3) ** (i / (npos - 1))
    neg = rng.uniform(-5.0, -0.1, nneg)
    noise = rng.normal(0.0, 0.01, n - npos - nneg)
    return np.concatenate([pos, neg, noise])


def spectrum_batch(n: int, seed: int) -> np.ndarray:
    rng = np.random.default_rng(seed)
    npos = round_half_up(0.1 * n)
    return np.concatenate([rng.uniform(0.5, 5.0, npos),
                           rng.normal(0.0, 0.1, n - npos)])


def spectrum_cor3(n: int, b1=3.0, b2=1.0, b3=6.0, b4=2.0) -> np.ndarray:
    assert n % 4 == 0
    q = n // 4
    return np.concatenate([np.full(q, -b1), np.full(q, -b2), np.full(q, b3),
                           np.full(q, b4)])


def form_A_numpy(Vr: np.ndarray, lam: np.ndarray) -> np.ndarray:
    """Dense FP64 U diag(lam) U^T, U = H_1 ... H_r (applied as H_t A H_t for
    t = r..1).  O(n^2 r)."""
    n = lam.shape[0]
    A = np.diag(np.asarray(lam, dtype=np.float64))
    for t in range(Vr.shape[0] - 1, -1, -1):
        v = Vr[t]
        beta = 2.0 / float(v @ v)
        w = A @ v
        u = w - 0.5 * beta * float(v @ w) * v
        A -= beta * (np.outer(v, u) + np.outer(u, v))
    return A


def form_A_torch(Vr: np.ndarray, lam: np.ndarray, device, out_dtype=None):
    """Same matrix formed with torch in FP64 on `device`, rounded to
    `out_dtype` (default float32) once."""
    import torch
    out_dtype = out_dtype or torch.float32
    lam_t = torch.as_tensor(np.asarray(lam, dtype=np.float64), device=device)
    A = torch.diag(lam_t)
    for t in range(Vr.shape[0] - 1, -1, -1):
        v = torch.as_tensor(np.asarray(Vr[t], dtype=np.float64), device=device)
        beta = 2.0 / float(v @ v)
        w = A @ v
        u = w - 0.5 * beta * float(v @ w) * v
        A.addr_(v, u, alpha=-beta)
        A.addr_(u, v, alpha=-beta)
    out = A.to(out_dtype)
    del A
    return out


def make_problem(kind: str, n: int, seed_u: int = 0, seed_lam: int = 2, r: int | None = None):
    """(Vr, lam) for one of the recipes above."""
    if kind == "small":
        lam = spectrum_small(n, seed_lam)
        r = 3 if r is None else r
    elif kind == "decay":
        lam = spectrum_decay(n, seed_lam)
        r = 4 if r is None else r
    elif kind == "batch":
        lam = spectrum_batch(n, seed_lam)
        r = 2 if r is None else r
    elif kind == "cor3":
        lam = spectrum_cor3(n)
        r = 3 if r is None else r
    else:
        raise ValueError(kind)
    return householder_vectors(n, r, seed_u), lam


def lowrank_problem(n: int, ranks, seed: int = 5, r: int = 2):
    """A with the given nonzero eigenvalues (list) and zeros elsewhere: the
    exact-recovery inputs (rank(A) <= sketch width)."""
    lam = np.zeros(n)
    vals = np.asarray(ranks, dtype=np.float64)
    lam[: vals.shape[0]] = vals
    return householder_vectors(n, r, seed), lam


def log_uniform_sizes(count: int, lo: int, hi: int, seed: int) -> np.ndarray:
    """Matrix sides log-uniform in [lo, hi] (batched and served recipes)."""
    rng = np.random.default_rng(seed)
    return np.floor(np.exp(rng.uniform(math.log(lo), math.log(hi), count))).astype(np.int64)


def sdls_problem(n: int, mc: int, seed: int = 0):
    """The semidefinite least-squares example of Sec. 6 (dual gradient
    descent, Alg. 6): A_i = (T_i + T_i^T) / (2 ||T_i||) with T_i Gaussian
    n x n and ||.|| the Frobenius norm (the paper writes ||.||_2 for the
    Frobenius norm of a matrix elsewhere, and only with it does its step
    size 0.5 lie below 2 / Lipschitz constant of the dual gradient);
    b_i = <A_i, X0> for a PSD X0 = G G^T / n (G Gaussian), so the problem is
    feasible; C = (H + H^T) / 2 with H Gaussian.  numpy PCG64 stream `seed`.
    Returns (C, [A_i], b) in FP64 (rounded to FP32 by the caller when it is
    the device input)."""
    rng = np.random.default_rng(seed)
    As = []
    for _ in range(mc):
        T = rng.standard_normal((n, n))
        As.append((T + T.T) / (2.0 * np.linalg.norm(T)))
    G = rng.standard_normal((n, n))
    X0 = G @ G.T / n
    b = np.array([float(np.sum(Ai * X0)) for Ai in As])
    H = rng.standard_normal((n, n))
    C = (H + H.T) / 2.0
    return C, As, b
