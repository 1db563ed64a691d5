"""Pins of the oracle's eigensolver and exact projection (Thm 1).

* Jacobi against numpy.linalg.eigh (LAPACK) and against reconstruction.
* exact_proj against the Householder closed form U diag(lam+) U^T.
* The Fig. 3 pair (Prop. 1): Frobenius non-expansive, spectral not.
* The polar form X+ = (X + (X^T X)^(1/2)) / 2 (Prop. 1 proof).
* Moreau invariants P >= 0, A - P <= 0, <P, A - P> = 0, and Thm 1 optimality.
"""
import json
import os

import numpy as np
import pytest

import synth_inputs as si

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def _rand_sym(n, seed):
    rng = np.random.default_rng(seed)
    X = rng.standard_normal((n, n))
    return (X + X.T) / 2


@pytest.mark.parametrize("m,seed", [(1, 0), (2, 1), (7, 2), (40, 3), (113, 4)])
def test_jacobi_matches_eigh(oracle_lib, m, seed):
    C = _rand_sym(m, seed)
    d, V, sweeps = oracle_lib.jacobi_eig(C)
    ref = np.linalg.eigvalsh(C)
    assert np.allclose(np.sort(d), ref, atol=1e-12 * max(1, np.abs(ref).max()))
    assert np.allclose(V.T @ V, np.eye(m), atol=1e-13)
    assert np.allclose(V @ np.diag(d) @ V.T, C, atol=1e-12 * np.linalg.norm(C))
    assert sweeps <= 20


def test_jacobi_clustered_and_diagonal(oracle_lib):
    d0 = np.array([3.0, 3.0, 3.0, -1.0, -1.0, 0.0, 0.0, 5.0])
    Vr = si.householder_vectors(8, 3, 11)
    A = si.form_A_numpy(Vr, d0)
    d, V, _ = oracle_lib.jacobi_eig(A)
    assert np.allclose(np.sort(d), np.sort(d0), atol=1e-13)
    d2, V2, sw = oracle_lib.jacobi_eig(np.diag(d0))
    assert sw == 0 and np.array_equal(d2, d0)


def test_exact_proj_matches_closed_form(oracle_lib):
    n = 60
    Vr, lam = si.householder_vectors(n, 3, 0), np.random.default_rng(1).normal(0, 1, n)
    A = si.form_A_numpy(Vr, lam)
    P = oracle_lib.exact_proj(A)
    P_cf = oracle_lib.closed_form_proj(Vr, lam)
    assert np.abs(P - P_cf).max() < 1e-12 * np.abs(lam).max() * n
    # numpy reference of Thm 1
    w, U = np.linalg.eigh(A)
    P_np = (U * np.maximum(w, 0)) @ U.T
    assert np.abs(P - P_np).max() < 1e-12 * n


def test_exact_proj_reads_upper_triangle_only(oracle_lib):
    n = 30
    A = _rand_sym(n, 5)
    Apois = A.copy()
    Apois[np.tril_indices(n, -1)] = np.nan
    assert np.array_equal(oracle_lib.exact_proj(A), oracle_lib.exact_proj(Apois))


def test_fig3_pair(oracle_lib):
    g = json.load(open(os.path.join(GOLD, "fig3_pair.json")))
    A = np.array(g["A"], dtype=float)
    Ap = oracle_lib.exact_proj(A)
    assert np.allclose(Ap, A)
    spectral_violated = False
    for d in np.linspace(*g["d_range"], 41):
        B = np.array([[0.0, g["B_offdiag"]], [g["B_offdiag"], d]])
        Bp = oracle_lib.exact_proj(B)
        # closed form for the 2x2 B: eigenvalues (d +- sqrt(d^2 + 4 b^2)) / 2
        lam_max = (d + np.sqrt(d * d + 4 * g["B_offdiag"] ** 2)) / 2
        assert abs(np.trace(Bp) - lam_max) < 1e-9 * lam_max
        assert np.linalg.matrix_rank(Bp, tol=1e-9 * lam_max) == 1
        fro = np.linalg.norm(Ap - Bp)
        assert fro <= np.linalg.norm(A - B) + 1e-9
        if np.linalg.norm(Ap - Bp, 2) > np.linalg.norm(A - B, 2) + 1e-9:
            spectral_violated = True
        # Prop. 1 spectral bound with the sqrt(n) factor (n = 2)
        assert np.linalg.norm(Ap - Bp, 2) <= 0.5 * (np.sqrt(2) + 1) * np.linalg.norm(A - B, 2) + 1e-9
    assert spectral_violated


def test_polar_form(oracle_lib):
    from scipy.linalg import sqrtm
    X = _rand_sym(25, 9)
    polar = (X + np.real(sqrtm(X.T @ X))) / 2
    assert np.abs(oracle_lib.exact_proj(X) - polar).max() < 1e-9


def test_moreau_invariants_and_optimality(oracle_lib):
    X = _rand_sym(40, 13)
    P = oracle_lib.exact_proj(X)
    assert np.linalg.eigvalsh(P).min() > -1e-12
    assert np.linalg.eigvalsh(X - P).max() < 1e-12
    assert abs(np.sum(P * (X - P))) < 1e-10
    rng = np.random.default_rng(3)
    best = np.linalg.norm(X - P)
    for _ in range(20):
        G = rng.standard_normal((40, 40))
        Y = G @ G.T * rng.uniform(0.001, 0.1)
        assert np.linalg.norm(X - Y) >= best
        Y2 = P + 1e-3 * (G @ G.T) / 40
        assert np.linalg.norm(X - Y2) >= best
