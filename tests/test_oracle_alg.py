"""Pins of the oracle's range finder, both randomized projections, min_eig and
the error-bound terms.

* Range finder (Alg. 1): Q^T Q = I, Y = Q R, the one-shot and the
  re-orthonormalised forms span the same range, Halko's Frobenius bound in the
  mean (appendix theorem, q = 0).
* Alg. 2 (C ABI "Algorithm 1"): exact recovery when rank(A) <= k+p,
  Counterexample 1 with hand-picked Q, the invariants of Q (Q^T A Q)_+ Q^T,
  Cor. 1 bounds in the mean.
* Alg. 3 (C ABI "Algorithm 2"): the literal last step equals the reduced form
  (Lemma 4), zero error when the shifted tail vanishes (remark after Prop. 3),
  Prop. 3 bound in the mean.
* Algs. 4/5: the min-eigenvalue identity of the appendix lemma, convergence
  in N.
* Eqs. (eps1), (eps2): values evaluated by hand; Cor. 3's inequality.
"""
import json
import os

import numpy as np
import pytest

import synth_inputs as si

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def _P(W):
    return W @ W.T


def test_orth_properties(oracle_lib):
    rng = np.random.default_rng(0)
    Y = rng.standard_normal((80, 12)) @ np.diag(np.logspace(0, -4, 12))
    Q, r = oracle_lib.orth(Y)
    assert r == 12
    assert np.allclose(Q.T @ Q, np.eye(12), atol=1e-13)
    R = Q.T @ Y
    assert np.allclose(np.tril(R, -1), 0, atol=1e-12)
    assert np.allclose(Q @ R, Y, atol=1e-12)
    # dependent columns are zeroed and counted out of the rank
    Yd = np.concatenate([Y[:, :5], Y[:, :2] @ rng.standard_normal((2, 3))], axis=1)
    Qd, rd = oracle_lib.orth(Yd)
    assert rd == 5
    assert np.allclose(Qd[:, 5:], 0)
    assert np.allclose(Qd[:, :5].T @ Qd[:, :5], np.eye(5), atol=1e-13)


@pytest.mark.parametrize("q", [0, 1, 2])
def test_range_finder_oneshot_equals_reorth(oracle_lib, q):
    n, m = 200, 12
    Vr, lam = si.householder_vectors(n, 3, 1), np.concatenate(
        [np.linspace(10, 3, 8), np.linspace(-9, -4, 6), 0.2 * np.random.default_rng(2).standard_normal(n - 14)])
    A = si.form_A_numpy(Vr, lam)
    Om = oracle_lib.omega(1, n, m)
    Q1, _ = oracle_lib.range_finder(A, Om, q, reorth=True)
    Q0, _ = oracle_lib.range_finder(A, Om, q, reorth=False)
    # same subspace: singular values of Q1^T Q0 are all 1
    s = np.linalg.svd(Q1.T @ Q0, compute_uv=False)
    assert np.all(np.abs(s - 1) < 1e-8)


def test_halko_frobenius_bound_mean(oracle_lib):
    n, k, p = 150, 10, 5
    Vr, lam = si.householder_vectors(n, 3, 4), np.concatenate(
        [np.linspace(20, 5, 10), 0.5 * np.random.default_rng(5).standard_normal(n - 10)])
    A = si.form_A_numpy(Vr, lam)
    sig = np.sort(np.abs(lam))[::-1]
    bound = oracle_lib.eps1(sig, k, p)
    errs = []
    for seed in range(32):
        Q, _ = oracle_lib.range_finder(A, oracle_lib.omega(seed, n, k + p), 0)
        errs.append(np.linalg.norm(A - Q @ (Q.T @ A)))
    assert np.mean(errs) <= bound
    # and the optimum (Eckart-Young) is a lower bound
    assert min(errs) >= np.sqrt(np.sum(sig[k + p:] ** 2)) - 1e-9


def test_alg1_exact_recovery_mixed_sign(oracle_lib):
    n, k, p = 120, 8, 4
    Vr, lam = si.lowrank_problem(n, [7.0, 5.0, 3.0, 1.0, -2.0, -4.0, -6.0, 0.5, -0.3, 2.5], seed=3)
    A = si.form_A_numpy(Vr, lam)
    Xp = oracle_lib.closed_form_proj(Vr, lam)
    for q in [0, 1]:
        out = oracle_lib.alg1(A, k, p, q, seed=11)
        assert out["rank"] == 10
        assert out["rplus"] == 6
        assert np.abs(_P(out["W"]) - Xp).max() < 1e-11
        # Gram-form metric: resolution ~1e-13 in the squared distance
        assert oracle_lib.exact_dist2(Vr, lam, out["W"]) < 1e-12


def test_counterexample_1(oracle_lib):
    g = json.load(open(os.path.join(GOLD, "counterexample1.json")))
    X = np.array(g["X"], dtype=float)
    assert np.allclose(oracle_lib.exact_proj(X), g["X_plus"])
    e1 = np.array([[1.0], [0.0], [0.0]])
    e3 = np.array([[0.0], [0.0], [1.0]])
    W1, r1 = oracle_lib.core_project(X, e1)
    W3, r3 = oracle_lib.core_project(X, e3)
    assert r1 == 0 and np.allclose(_P(W1), g["Q_e1_projection"])
    assert r3 == 1 and np.allclose(_P(W3), g["Q_e3_projection"])


def _decay_problem(n=300, seed=0):
    rng = np.random.default_rng(seed + 100)
    lam = np.concatenate([10 * 0.8 ** np.arange(20), -rng.uniform(0.5, 6, 30),
                          rng.normal(0, 0.05, n - 50)])
    Vr = si.householder_vectors(n, 3, seed)
    return Vr, lam, si.form_A_numpy(Vr, lam)


def test_alg1_invariants(oracle_lib):
    Vr, lam, A = _decay_problem()
    k, p, q = 20, 6, 1
    out = oracle_lib.alg1(A, k, p, q, seed=3)
    P = _P(out["W"])
    assert np.linalg.matrix_rank(P, tol=1e-9 * np.abs(P).max()) <= k + p
    assert np.linalg.eigvalsh(P).min() > -1e-10
    # <P, A - P> = 0 follows from the interchange lemma with Q^T Q = I
    assert abs(np.sum(P * (A - P))) < 1e-9 * np.linalg.norm(A) ** 2
    # Q^T (A - P) Q <= 0 on the sketched subspace
    Q, _ = oracle_lib.range_finder(A, oracle_lib.omega(3, A.shape[0], k + p), q)
    assert np.linalg.eigvalsh(Q.T @ (A - P) @ Q).max() < 1e-9
    # factor-form distances agree with dense ones
    Xp = oracle_lib.closed_form_proj(Vr, lam)
    assert abs(oracle_lib.exact_dist2(Vr, lam, out["W"]) - np.sum((Xp - P) ** 2)) < 1e-8
    W2 = oracle_lib.alg1(A, k, p, q, seed=4)["W"]
    assert abs(oracle_lib.factor_dist2(out["W"], W2) - np.sum((P - _P(W2)) ** 2)) < 1e-8


def test_alg1_oneshot_vs_reorth(oracle_lib):
    Vr, lam, A = _decay_problem(200, 1)
    for q in [0, 1, 2]:
        a = oracle_lib.alg1(A, 15, 5, q, seed=2, reorth=True)["W"]
        b = oracle_lib.alg1(A, 15, 5, q, seed=2, reorth=False)["W"]
        # the Gram form cancels: its resolution is ~1e-8 ||P||_F
        d = max(oracle_lib.factor_dist2(a, b), 0.0)
        assert np.sqrt(d) < 1e-6 * np.sqrt(oracle_lib.factor_norm2(a))
        assert np.abs(a @ a.T - b @ b.T).max() < 1e-8 * np.abs(a @ a.T).max()


def test_alg2_literal_equals_reduced(oracle_lib):
    Vr, lam, A = _decay_problem(250, 2)
    for q in [0, 1, 2]:
        out = oracle_lib.alg2(A, 20, 6, q, seed=5, N=10)
        assert out["degraded"] == 0 and out["alpha"] > 0
        Pl, Pr = _P(out["W_lit"]), _P(out["W_red"])
        assert np.abs(Pl - Pr).max() < 1e-10 * np.abs(Pr).max()


def test_alg2_zero_error_when_shifted_tail_vanishes(oracle_lib):
    # lambda_i + alpha = 0 for every i beyond the sketch: exact output
    n, k, p = 100, 6, 4
    alpha = 2.5
    lam = np.full(n, -alpha)
    lam[:8] = [9.0, 6.0, 4.0, 3.0, 1.0, 0.5, -1.0, -2.0]
    Vr = si.householder_vectors(n, 3, 8)
    A = si.form_A_numpy(Vr, lam)
    out = oracle_lib.alg2(A, k, p, 0, seed=9, alpha=alpha)
    Xp = oracle_lib.closed_form_proj(Vr, lam)
    # dense check: the Gram-form metric cannot resolve below ~1e-13
    assert np.abs(_P(out["W_red"]) - Xp).max() < 1e-11
    assert np.abs(_P(out["W_lit"]) - Xp).max() < 1e-11
    # Alg. 2 (unscaled) cannot recover it: A is full rank
    w1 = oracle_lib.alg1(A, k, p, 0, seed=9)["W"]
    assert oracle_lib.exact_dist2(Vr, lam, w1) > 1e-2


def test_min_eig_identity_and_convergence(oracle_lib):
    n = 80
    lam = np.concatenate([[5.0, -8.0, 3.0], np.linspace(-2.0, 2.0, n - 3)])
    Vr = si.householder_vectors(n, 3, 6)
    A = si.form_A_numpy(Vr, lam)
    a, s1, s2 = oracle_lib.min_eig(A, 300, seed=1)
    assert abs(a - 8.0) < 1e-8
    assert abs(s1 - 8.0) < 1e-8 and abs(s2 - 16.0) < 1e-8
    # positive-dominant case: sigma1 = lambda_max
    lam2 = np.concatenate([[9.0, -4.0], np.linspace(-1.0, 1.0, n - 2)])
    A2 = si.form_A_numpy(si.householder_vectors(n, 3, 7), lam2)
    a2, s1b, s2b = oracle_lib.min_eig(A2, 400, seed=1)
    assert abs(a2 - 4.0) < 1e-7 and abs(s1b - 9.0) < 1e-8 and abs(s2b - 13.0) < 1e-7
    # the error shrinks with N
    errs = [abs(oracle_lib.min_eig(A, N, seed=2)[0] - 8.0) for N in [2, 10, 40]]
    assert errs[2] < errs[1] < errs[0]
    # power_iteration on a shifted matrix
    assert abs(oracle_lib.power_iteration(A, 300, 1, 3, shift=-8.0) - 16.0) < 1e-7


def test_eps_terms_by_hand(oracle_lib):
    sig = np.array([3.0, 2.0, 1.0, 1.0])
    # sqrt((1 + 2/(3-1)) * (1 + 1)) = 2
    assert abs(oracle_lib.eps1(sig, 2, 3) - 2.0) < 1e-15
    # n=4, k=2, p=3, q=0, sigma=1: 1 + sqrt(1) + e sqrt(5)/3 sqrt(2)
    ref = 2.0 + np.e * np.sqrt(5.0) / 3.0 * np.sqrt(2.0)
    assert abs(oracle_lib.eps2(1.0, 4, 2, 3, 0) - ref) < 1e-14
    assert abs(oracle_lib.eps2(2.0, 4, 2, 3, 1) - 2.0 * ref ** (1 / 3)) < 1e-14


def test_cor3_inequality(oracle_lib):
    g = json.load(open(os.path.join(GOLD, "cor3_class.json")))
    n = g["n"]
    b1, b2, b3, b4 = g["beta"]
    lam = si.spectrum_cor3(n, b1, b2, b3, b4)
    alpha = g["alpha"]
    assert alpha == -lam.min()
    sig = np.sort(np.abs(lam))[::-1]
    shifted = np.sort(lam + alpha)[::-1]
    l = g["oversampling"]
    assert oracle_lib.eps1(shifted, n // 2, l) < oracle_lib.eps1(sig, n // 2, l)


def test_cor3_class_crossover_of_the_two_algorithms(oracle_lib):
    # the first numerical example of Sec. 4 (Fig. 5): on the Cor. 3 class the
    # scaled projection (Alg. 3) is no better than Alg. 2 while k <= n/4 and
    # far better once k > n/4, where Alg. 2 spends its sketch on the beta_1
    # cluster of negative eigenvalues.  n = 400 instead of 1000 keeps k + p
    # inside the sketch widths the GPU path takes (<= 256) across the
    # crossover at n/4 = 100; beta, oversampling 5 and q = 2 as in the example.
    g = json.load(open(os.path.join(GOLD, "cor3_class.json")))
    n, (b1, b2, b3, b4), p, q = 400, g["beta"], g["oversampling"], g["q"]
    Vr = si.householder_vectors(n, 3, 0)
    lam = si.spectrum_cor3(n, b1, b2, b3, b4)
    A = si.form_A_numpy(Vr, lam).astype(np.float32).astype(np.float64)
    xp = np.sqrt(np.sum(np.maximum(lam, 0) ** 2))
    err = {}
    for k in (60, 100, 200, 250):
        w1 = oracle_lib.alg1(A, k, p, q, 1)["W"]
        w2 = oracle_lib.alg2(A, k, p, q, 1, N=10)["W_red"]
        err[k] = (np.sqrt(max(oracle_lib.exact_dist2(Vr, lam, w1), 0)) / xp,
                  np.sqrt(max(oracle_lib.exact_dist2(Vr, lam, w2), 0)) / xp)
    for k in (60, 100):
        assert err[k][1] >= 0.98 * err[k][0]
    for k in (200, 250):
        assert err[k][1] <= 0.5 * err[k][0]


def test_cor1_prop3_frobenius_bounds_mean(oracle_lib):
    Vr, lam, A = _decay_problem(200, 3)
    n, k, p = 200, 15, 5
    sig = np.sort(np.abs(lam))[::-1]
    alpha = -lam.min()
    shifted = np.sort(lam + alpha)[::-1]
    b1 = np.sqrt(2) * oracle_lib.eps1(sig, k, p)
    b2 = np.sqrt(2) * oracle_lib.eps1(shifted, k, p)
    e1, e2, s1 = [], [], []
    for seed in range(32):
        w1 = oracle_lib.alg1(A, k, p, 0, seed=seed)["W"]
        w2 = oracle_lib.alg2(A, k, p, 0, seed=seed, alpha=alpha)["W_red"]
        e1.append(np.sqrt(oracle_lib.exact_dist2(Vr, lam, w1)))
        e2.append(np.sqrt(oracle_lib.exact_dist2(Vr, lam, w2)))
        Xp = oracle_lib.closed_form_proj(Vr, lam)
        s1.append(np.linalg.norm(Xp - w1 @ w1.T, 2))
    assert np.mean(e1) <= b1
    assert np.mean(e2) <= b2
    # spectral bound of Cor. 1, first branch: (1 + sqrt(n)) eps2(sigma_{k+1})
    assert np.mean(s1) <= (1 + np.sqrt(n)) * oracle_lib.eps2(sig[k], n, k, p, 0)


def test_alg2_degrades_to_alg1_when_alpha_vanishes(oracle_lib):
    # A = 0: min_eig gives alpha = |0 - 0| = 0, so Alg. 3 is undefined and the
    # call falls back to Alg. 2 (degraded = 1) with output 0
    n = 40
    A = np.zeros((n, n))
    out = oracle_lib.alg2(A, 4, 2, 0, seed=3, N=10)
    assert out["degraded"] == 1 and out["alpha"] == 0.0
    assert np.all(out["W_red"] == 0)
    # a subnormal alpha also takes the fallback, and equals Alg. 2's output
    Vr, lam = si.lowrank_problem(n, [4.0, 2.0, -1.0], seed=2)
    A = si.form_A_numpy(Vr, lam)
    out = oracle_lib.alg2(A, 4, 2, 0, seed=3, alpha=1e-310)
    ref = oracle_lib.alg1(A, 4, 2, 0, seed=3)["W"]
    assert out["degraded"] == 1
    assert np.array_equal(out["W_red"], ref)


def test_ritz_alpha_is_a_lower_estimate_of_the_most_negative_eigenvalue(oracle_lib):
    # the variant's alpha = -(smallest Ritz value of Q0^T A Q0): by the
    # Poincare separation theorem every Ritz value of a symmetric A lies in
    # [lambda_min, lambda_max], so 0 <= alpha_ritz <= |lambda_min(A)|; with
    # the most negative eigenvector well inside the sketch it is close
    Vr, lam, A = _decay_problem(600, 4)
    for k in (20, 100):
        Om = oracle_lib.omega(3, 600, k + 10)
        Q0, _ = oracle_lib.range_finder(A, Om, 0)
        C = Q0.T @ oracle_lib.sym_mul(A, Q0)
        d, _, _ = oracle_lib.jacobi_eig(0.5 * (C + C.T))
        a = -min(d.min(), 0.0)
        assert 0.0 <= a <= -lam.min() + 1e-12
    assert a >= 0.5 * -lam.min()


# ----------------------------------------------------------------------------
# Alg. 6 (dual gradient descent for semidefinite least squares)
# ----------------------------------------------------------------------------
def _theta(oracle_lib, C, As, b, rho, y):
    # dual function theta(y) = L(X*(y), y), X*(y) = (C/rho + sum y_i A_i)_+
    X = C / rho + sum(yi * Ai for yi, Ai in zip(y, As))
    P = oracle_lib.exact_proj(X)
    return 0.5 * np.sum((P - C / rho) ** 2) - sum(yi * (np.sum(Ai * P) - bi) for yi, Ai, bi in zip(y, As, b))


def test_sdls_exact_gradient_descent_reaches_the_dual_optimum(oracle_lib):
    # with exact projections Alg. 6 is gradient ascent on the concave dual:
    # the gradient vanishes and theta is maximal there (checked by moving y)
    n, mc, rho = 100, 2, 1.0
    C, As, b = si.sdls_problem(n, mc, seed=3)
    r = oracle_lib.sdls_dual_gd(C, As, b, rho, 10, 5, 0, 2, 0.5, 1e-9, 400, 1, [1.2753, 0.2418], exact=True)
    assert r["gnorm"] <= 1e-9 and r["iters"] < 400
    assert all(h2 <= h1 * 1.0001 for h1, h2 in zip(r["hist"][5:], r["hist"][6:]))
    t0 = _theta(oracle_lib, C, As, b, rho, r["y"])
    for i in range(mc):
        for d in (-1e-3, 1e-3):
            yy = np.array(r["y"]); yy[i] += d
            assert _theta(oracle_lib, C, As, b, rho, yy) <= t0 + 1e-12


def test_sdls_full_width_sketch_follows_the_exact_iteration(oracle_lib):
    # a sketch as wide as the matrix spans everything: the randomized
    # projection is the exact one, so both iterations coincide
    n, mc = 60, 2
    C, As, b = si.sdls_problem(n, mc, seed=4)
    y0 = [0.3, -0.7]
    ex = oracle_lib.sdls_dual_gd(C, As, b, 1.0, 50, 10, 0, 1, 0.5, 0.0, 15, 1, y0, exact=True)
    for alg, warm in ((1, False), (2, False), (1, True)):
        rr = oracle_lib.sdls_dual_gd(C, As, b, 1.0, 50, 10, 0, alg, 0.5, 0.0, 15, 1, y0, warm_start=warm)
        assert np.allclose(rr["hist"], ex["hist"], rtol=1e-8, atol=1e-10)
        assert np.allclose(rr["y"], ex["y"], rtol=1e-8, atol=1e-10)
