"""FP64 CPU oracle for the randomized PSD projections of arXiv 2410.19208.

TEST INFRASTRUCTURE ONLY.  This package is the plain, slow reference that the
CUDA library is checked against.  Only ``tests/``, ``__graft_entry__.smoke()``
and ``bench.py``'s cpu_baseline / reference arm may import it; the product
package ``paper_2410_19208_gb300`` never does.  The C source
``psdproj_oracle.c`` shares no code with the CUDA library.

Functions (each docstring cites the passage it follows):

* ``philox4x32_10``, ``gauss``, ``omega``  - the test-matrix generator (Alg. 1
  ``randn``; Philox4x32-10 of Salmon et al. SC'11 as our reading).
* ``omega_srht``                          - the structured test matrix of the
  footnote to Alg. 1 (subsampled randomized Hadamard transform reading).
* ``jacobi_eig``, ``exact_proj``          - Thm 1 (X+ = U D+ U^T).
* ``orth``, ``range_finder``              - Alg. 1 (QR 'econ').
* ``alg1``                                 - Alg. 2 (the C ABI's "Algorithm 1").
* ``power_iteration``, ``min_eig``         - Algs. 4 and 5.
* ``alg2``                                 - Alg. 3 (the C ABI's "Algorithm 2"),
  literal last step and the reduced form of Lemma 4.
* ``eps1``, ``eps2``                       - Eqs. (eps1), (eps2).
* ``sdls_dual_gd``                         - Alg. 6 (dual gradient descent for
  the semidefinite least-squares problem).
* ``factor_dist2``, ``exact_dist2``        - Frobenius errors in Gram form.

Parity status: every function above is pinned by a ``-m "not gpu"`` test in
``tests/test_oracle_*.py``; none is "parity unpinned".
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "psdproj_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_SO = os.path.join(_BUILD, "liboracle.so")
_lock = threading.Lock()
_lib = None

_D = ctypes.POINTER(ctypes.c_double)
_I = ctypes.POINTER(ctypes.c_int)
_U32 = ctypes.POINTER(ctypes.c_uint32)
_i64 = ctypes.c_int64
_u64 = ctypes.c_uint64


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (-O2, OpenMP) into oracle/_build/liboracle.so."""
    os.makedirs(_BUILD, exist_ok=True)
    if (not force and os.path.exists(_SO)
            and os.path.getmtime(_SO) >= os.path.getmtime(_SRC)):
        return _SO
    tmp = _SO + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-fopenmp", "-fPIC", "-shared", "-std=c11",
           "-D_GNU_SOURCE", "-o", tmp, _SRC, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _SO)
    return _SO


def _load():
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        lib = ctypes.CDLL(build())
        lib.orc_philox4x32_10.argtypes = [_U32, ctypes.c_uint32, ctypes.c_uint32, _U32]
        lib.orc_gauss.argtypes = [_u64, ctypes.c_uint32, ctypes.c_uint32, ctypes.c_uint32]
        lib.orc_gauss.restype = ctypes.c_double
        lib.orc_omega.argtypes = [_u64, _i64, ctypes.c_int, ctypes.c_uint32, _D]
        lib.orc_sym_mul.argtypes = [_D, _i64, _i64, _D, ctypes.c_int, ctypes.c_double, _D]
        lib.orc_jacobi_eig.argtypes = [ctypes.c_int, _D, _D, _D, ctypes.c_double,
                                       ctypes.c_int, _I]
        lib.orc_exact_proj.argtypes = [_D, _i64, _i64, _D]
        lib.orc_orth.argtypes = [_D, _i64, ctypes.c_int, ctypes.c_double]
        lib.orc_range_finder.argtypes = [_D, _i64, _i64, _D, ctypes.c_int, ctypes.c_int,
                                         ctypes.c_double, ctypes.c_double, ctypes.c_int,
                                         ctypes.c_double, _D]
        lib.orc_alg1.argtypes = [_D, _i64, _i64, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                 _u64, ctypes.c_int, _D, _D, _I, _I]
        lib.orc_power_iteration.argtypes = [_D, _i64, _i64, ctypes.c_double, ctypes.c_int,
                                            _u64, ctypes.c_uint32]
        lib.orc_power_iteration.restype = ctypes.c_double
        lib.orc_min_eig.argtypes = [_D, _i64, _i64, ctypes.c_int, _u64, _D, _D]
        lib.orc_min_eig.restype = ctypes.c_double
        lib.orc_alg2.argtypes = [_D, _i64, _i64, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                 _u64, ctypes.c_double, ctypes.c_int, ctypes.c_int,
                                 _D, _D, _D, _I, _I, _I]
        lib.orc_core_project.argtypes = [_D, _i64, _i64, _D, ctypes.c_int, _D]
        lib.orc_eps1.argtypes = [_D, _i64, ctypes.c_int, ctypes.c_int]
        lib.orc_eps1.restype = ctypes.c_double
        lib.orc_eps2.argtypes = [ctypes.c_double, _i64, ctypes.c_int, ctypes.c_int, ctypes.c_int]
        lib.orc_eps2.restype = ctypes.c_double
        lib.orc_factor_dist2.argtypes = [_D, ctypes.c_int, _D, ctypes.c_int, _i64]
        lib.orc_factor_dist2.restype = ctypes.c_double
        lib.orc_factor_norm2.argtypes = [_D, ctypes.c_int, _i64]
        lib.orc_factor_norm2.restype = ctypes.c_double
        lib.orc_apply_Ut.argtypes = [_D, ctypes.c_int, _i64, _D, ctypes.c_int]
        lib.orc_exact_dist2.argtypes = [_D, ctypes.c_int, _D, _i64, _D, ctypes.c_int]
        lib.orc_exact_dist2.restype = ctypes.c_double
        lib.orc_closed_form_proj.argtypes = [_D, ctypes.c_int, _D, _i64, _D]
        _lib = lib
        return lib


def _dp(a: np.ndarray):
    assert a.dtype == np.float64 and a.flags.c_contiguous
    return a.ctypes.data_as(_D)


def _mat(A) -> np.ndarray:
    A = np.ascontiguousarray(A, dtype=np.float64)
    assert A.ndim == 2 and A.shape[0] == A.shape[1]
    return A


class OracleError(RuntimeError):
    pass


def _check(st: int, what: str):
    if st != 0:
        raise OracleError(f"{what}: oracle status {st}")


# --------------------------------------------------------------------------
# Random test matrices (Alg. 1 line "Omega = randn"; Philox4x32-10 reading)
# --------------------------------------------------------------------------
def philox4x32_10(ctr, key):
    """Philox4x32-10 block function (Salmon et al., SC'11): 4 counter words,
    2 key words -> 4 output words."""
    lib = _load()
    c = (ctypes.c_uint32 * 4)(*[int(x) & 0xFFFFFFFF for x in ctr])
    o = (ctypes.c_uint32 * 4)()
    lib.orc_philox4x32_10(c, int(key[0]) & 0xFFFFFFFF, int(key[1]) & 0xFFFFFFFF, o)
    return [int(x) for x in o]


def gauss(seed: int, i: int, j: int, stream: int) -> float:
    """N(0,1) sample for element (i, j) of stream (Box-Muller, FP64)."""
    return float(_load().orc_gauss(seed, i, j, stream))


def omega(seed: int, n: int, m: int, stream: int = 0) -> np.ndarray:
    """n x m Gaussian test matrix, element (i,c) keyed by counter (i,c,stream,0)."""
    out = np.empty((n, m), dtype=np.float64)
    _load().orc_omega(seed, n, m, stream, _dp(out))
    return out


def omega_srht(seed: int, n: int, m: int) -> np.ndarray:
    """Structured test matrix for Alg. 1.  The footnote to Alg. 1 names the
    subsampled randomized Fourier transform; the reading taken is its real
    counterpart, the subsampled randomized Hadamard transform: with N the
    smallest power of two >= n, Omega = rows 0..n-1 of D H_N S, where
      D = diag(d), d_i = -1 when bit 0 of word 0 of Philox(counter (i, 0, 17, 0))
          is set, else +1;
      H_N = the Sylvester-Hadamard matrix, H_N[i, j] = (-1)^popcount(i & j);
      S = the columns s_0..s_{m-1}: s_c is the first word-0 value of
          Philox(counter (c, t, 16, 0)) mod N, t = 0, 1, ..., not already
          taken by an earlier column.
    Key = (seed low 32 bits, seed high 32 bits).  Entries are +-1."""
    N = 1
    while N < n:
        N *= 2
    key = (seed & 0xFFFFFFFF, (seed >> 32) & 0xFFFFFFFF)
    picks = []
    for c in range(m):
        t = 0
        while True:
            x = philox4x32_10((c, t, 16, 0), key)[0] % N
            if x not in picks:
                picks.append(x)
                break
            t += 1
    d = np.array([-1.0 if philox4x32_10((i, 0, 17, 0), key)[0] & 1 else 1.0 for i in range(n)])
    i = np.arange(n, dtype=np.uint64)[:, None]
    s = np.array(picks, dtype=np.uint64)[None, :]
    H = 1.0 - 2.0 * (np.bitwise_count(i & s) % 2)
    return d[:, None] * H


# --------------------------------------------------------------------------
# Dense symmetric helpers
# --------------------------------------------------------------------------
def sym_mul(A, X, shift: float = 0.0) -> np.ndarray:
    """Y = (A + shift I) X reading only the upper triangle of A."""
    A = _mat(A)
    X = np.ascontiguousarray(X, dtype=np.float64)
    if X.ndim == 1:
        X = X[:, None]
    Y = np.empty_like(X)
    _check(_load().orc_sym_mul(_dp(A), A.shape[0], A.shape[1], _dp(X), X.shape[1],
                               shift, _dp(Y)), "sym_mul")
    return Y


def jacobi_eig(C, rel_tol: float = 1e-15, max_sweeps: int = 100):
    """Cyclic Jacobi eigendecomposition (FP64).  Returns (d, V, sweeps)."""
    C = np.array(C, dtype=np.float64, order="C", copy=True)
    m = C.shape[0]
    V = np.empty((m, m))
    d = np.empty(m)
    sw = ctypes.c_int(0)
    _check(_load().orc_jacobi_eig(m, _dp(C), _dp(V), _dp(d), rel_tol, max_sweeps,
                                  ctypes.byref(sw)), "jacobi_eig")
    return d, V, sw.value


def exact_proj(A) -> np.ndarray:
    """Thm 1: X+ = U D+ U^T from the full Jacobi eigendecomposition."""
    A = _mat(A)
    n = A.shape[0]
    P = np.empty((n, n))
    _check(_load().orc_exact_proj(_dp(A), n, n, _dp(P)), "exact_proj")
    return P


def orth(Y, tau: float = 1e-10):
    """Economy orthonormal basis of range(Y) (MGS, two passes) with the
    dependent-column rule; returns (Q, rank)."""
    Q = np.array(Y, dtype=np.float64, order="C", copy=True)
    r = _load().orc_orth(_dp(Q), Q.shape[0], Q.shape[1], tau)
    return Q, r


def range_finder(A, Om, q: int, shift: float = 0.0, scale: float = 1.0,
                 reorth: bool = True, tau: float = 1e-10):
    """Alg. 1 on S = (A + shift I) * scale; returns (Q, rank)."""
    A = _mat(A)
    Om = np.ascontiguousarray(Om, dtype=np.float64)
    Q = np.empty_like(Om)
    r = _load().orc_range_finder(_dp(A), A.shape[0], A.shape[1], _dp(Om), Om.shape[1],
                                 q, shift, scale, int(reorth), tau, _dp(Q))
    if r < 0:
        raise OracleError(f"range_finder status {-r}")
    return Q, r


# --------------------------------------------------------------------------
# The two randomized projections
# --------------------------------------------------------------------------
def alg1(A, k: int, p: int, q: int, seed: int, reorth: bool = True):
    """Alg. 2 (ran_proj): returns dict(W, d, rank, rplus); P = W W^T."""
    A = _mat(A)
    n = A.shape[0]
    m = k + p
    W = np.empty((n, m))
    d = np.empty(m)
    rank = ctypes.c_int(0)
    rp = ctypes.c_int(0)
    _check(_load().orc_alg1(_dp(A), n, n, k, p, q, seed, int(reorth), _dp(W), _dp(d),
                            ctypes.byref(rank), ctypes.byref(rp)), "alg1")
    return dict(W=W, d=d, rank=rank.value, rplus=rp.value)


def power_iteration(A, N: int, seed: int, stream: int, shift: float = 0.0) -> float:
    """Alg. 4 on A + shift I with the start vector from `stream`."""
    A = _mat(A)
    return float(_load().orc_power_iteration(_dp(A), A.shape[0], A.shape[1], shift, N,
                                             seed, stream))


def min_eig(A, N: int, seed: int):
    """Alg. 5: returns (alpha, sigma1, sigma2)."""
    A = _mat(A)
    s1 = ctypes.c_double(0)
    s2 = ctypes.c_double(0)
    a = _load().orc_min_eig(_dp(A), A.shape[0], A.shape[1], N, seed, ctypes.byref(s1),
                            ctypes.byref(s2))
    return float(a), s1.value, s2.value


def alg2(A, k: int, p: int, q: int, seed: int, alpha: float = 0.0, N: int = 10,
         reorth: bool = True):
    """Alg. 3 (ran_proj_scal) with alpha from Alg. 5 when alpha <= 0.
    Returns dict(W_lit, W_red, alpha, degraded, rank, rplus)."""
    A = _mat(A)
    n = A.shape[0]
    m = k + p
    Wl = np.empty((n, m))
    Wr = np.empty((n, m))
    a = ctypes.c_double(0)
    deg = ctypes.c_int(0)
    rank = ctypes.c_int(0)
    rp = ctypes.c_int(0)
    _check(_load().orc_alg2(_dp(A), n, n, k, p, q, seed, alpha, N, int(reorth), _dp(Wl),
                            _dp(Wr), ctypes.byref(a), ctypes.byref(deg), ctypes.byref(rank),
                            ctypes.byref(rp)), "alg2")
    return dict(W_lit=Wl, W_red=Wr, alpha=a.value, degraded=deg.value, rank=rank.value,
                rplus=rp.value)


def sdls_dual_gd(C, As, b, rho: float, k: int, p: int, q: int, algorithm: int, beta: float,
                 eps: float, max_iter: int, seed: int, y0, N: int = 10, warm_start: bool = False,
                 exact: bool = False):
    """Alg. 6: dual gradient descent for min 1/2 ||X - C/rho||_F^2 over PSD X
    with <A_i, X> = b_i.  Each iteration forms X = C/rho + sum_i y_i A_i
    (Lemma: X*(y) = X_+), projects it (exact: Thm 1; else Alg. 2 or Alg. 3
    with alpha from Alg. 5, the sketch of iteration t drawn with seed + t,
    or with warm_start its Omega = the previous iteration's Q, columns that
    the orthonormalisation dropped taken from the fresh Gaussian draw), takes
    the gradient grad_i = <A_i, X_hat> - b_i and steps y <- y - beta grad;
    it stops after the iteration whose gradient norm is <= eps, or after
    max_iter iterations.  Returns dict(y, iters, gnorm, hist, W)."""
    C = _mat(C)
    n = C.shape[0]
    m = k + p
    As = [_mat(A) for A in As]
    b = np.asarray(b, dtype=np.float64)
    y = np.array(y0, dtype=np.float64)
    hist, Qprev, W, g = [], None, None, float("inf")
    t = -1
    for t in range(max_iter):
        X = C / rho
        for yi, Ai in zip(y, As):
            X = X + yi * Ai
        if exact:
            P = exact_proj(X)
            grad = np.array([float(np.sum(Ai * P)) for Ai in As]) - b
        else:
            s = seed + t
            Om = omega(s, n, m)
            if warm_start and Qprev is not None:
                alive = np.any(Qprev != 0.0, axis=0)
                Om[:, alive] = Qprev[:, alive]
            shift, scale = 0.0, 1.0
            if algorithm == 2:
                a = min_eig(X, N, s)[0]
                if np.isfinite(a) and a > 1e-300:
                    shift, scale = a, 1.0 / a
            Q, _ = range_finder(X, Om, q, shift=shift, scale=scale)
            W, _ = core_project(X, Q)
            Qprev = Q
            grad = np.array([float(np.sum(W * sym_mul(Ai, W))) for Ai in As]) - b
        g = float(np.linalg.norm(grad))
        hist.append(g)
        y = y - beta * grad
        if g <= eps:
            break
    return dict(y=y, iters=t + 1, gnorm=g, hist=hist, W=W)


def core_project(A, Q):
    """Alg. 2 lines 2-3 for a given orthonormal Q: returns (W, rplus)."""
    A = _mat(A)
    Q = np.ascontiguousarray(Q, dtype=np.float64)
    W = np.empty_like(Q)
    rp = _load().orc_core_project(_dp(A), A.shape[0], A.shape[1], _dp(Q), Q.shape[1],
                                  _dp(W))
    if rp < 0:
        raise OracleError(f"core_project status {-rp}")
    return W, rp


# --------------------------------------------------------------------------
# Bounds and error metrics
# --------------------------------------------------------------------------
def eps1(sigma, k: int, p: int) -> float:
    """Eq. (eps1); sigma sorted decreasingly; p is the paper's oversampling l."""
    s = np.ascontiguousarray(sigma, dtype=np.float64)
    return float(_load().orc_eps1(_dp(s), s.shape[0], k, p))


def eps2(sigma_k1: float, n: int, k: int, p: int, q: int) -> float:
    """Eq. (eps2) evaluated at sigma = sigma_{k+1}."""
    return float(_load().orc_eps2(sigma_k1, n, k, p, q))


def factor_dist2(W1, W2) -> float:
    """||W1 W1^T - W2 W2^T||_F^2 in Gram form."""
    W1 = np.ascontiguousarray(W1, dtype=np.float64)
    W2 = np.ascontiguousarray(W2, dtype=np.float64)
    assert W1.shape[0] == W2.shape[0]
    return float(_load().orc_factor_dist2(_dp(W1), W1.shape[1], _dp(W2), W2.shape[1],
                                          W1.shape[0]))


def factor_norm2(W) -> float:
    """||W W^T||_F^2 = ||W^T W||_F^2."""
    W = np.ascontiguousarray(W, dtype=np.float64)
    return float(_load().orc_factor_norm2(_dp(W), W.shape[1], W.shape[0]))


def exact_dist2(Vr, lam, W) -> float:
    """||X+ - W W^T||_F^2 for A = U diag(lam) U^T, U = H_1...H_r (rows of Vr)."""
    Vr = np.ascontiguousarray(Vr, dtype=np.float64)
    lam = np.ascontiguousarray(lam, dtype=np.float64)
    W = np.ascontiguousarray(W, dtype=np.float64)
    return float(_load().orc_exact_dist2(_dp(Vr), Vr.shape[0], _dp(lam), W.shape[0],
                                         _dp(W), W.shape[1]))


def apply_Ut(Vr, X) -> np.ndarray:
    """U^T X for U = H_1 ... H_r."""
    Vr = np.ascontiguousarray(Vr, dtype=np.float64)
    X = np.array(X, dtype=np.float64, order="C", copy=True)
    _load().orc_apply_Ut(_dp(Vr), Vr.shape[0], X.shape[0], _dp(X), X.shape[1])
    return X


def closed_form_proj(Vr, lam) -> np.ndarray:
    """X+ = U diag(max(lam,0)) U^T of a generated matrix (Thm 1 closed form)."""
    Vr = np.ascontiguousarray(Vr, dtype=np.float64)
    lam = np.ascontiguousarray(lam, dtype=np.float64)
    n = lam.shape[0]
    P = np.empty((n, n))
    _load().orc_closed_form_proj(_dp(Vr), Vr.shape[0], _dp(lam), n, _dp(P))
    return P
