"""Per-step parity of the CUDA path (through the C ABI) against the FP64 oracle.

Every input comes from synth_inputs / numpy generators; every expected value
from oracle/ (or, for library-pinned pieces, numpy / LAPACK).  Tolerances are
derived from FP32 arithmetic: an FP32 dot product of length n with FMA has
error <= gamma_n sum |a_i x_i|; the tests allow c * sqrt(n) * 2^-24 of that
bound (typical, not worst-case, rounding growth) with a margin.
"""
import numpy as np
import pytest

import synth_inputs as si

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import paper_2410_19208_gb300 as ps  # noqa: E402

EPS32 = 2.0 ** -24


@pytest.fixture(scope="module")
def ctx():
    c = ps.Context(0)
    yield c
    c.close()


def _tall_from_np(X, ld=None):
    n, m = X.shape
    T = ps.tall_empty(n, m, "cuda", ld=ld)
    T.copy_(torch.from_numpy(np.asarray(X, dtype=np.float32)))
    return T


def _np(T):
    return T.detach().cpu().numpy().astype(np.float64)


def _sym_A(n, seed, poison=False):
    rng = np.random.default_rng(seed)
    X = rng.standard_normal((n, n)).astype(np.float32)
    A = np.triu(X) + np.triu(X, 1).T
    if poison:
        A = A.copy()
        A[np.tril_indices(n, -1)] = np.nan
    return A


@pytest.mark.parametrize("n,m,stream", [(1000, 50, 0), (4099, 112, 0), (777, 1, 3), (5, 3, 4)])
def test_gaussian_matches_oracle(ctx, oracle_lib, n, m, stream):
    X = ps.tall_empty(n, m, "cuda", ld=n + 3)
    ctx.gaussian(7, stream, X)
    assert ctx.sync_status() == 0
    ref = oracle_lib.omega(7, n, m, stream)
    got = _np(X)
    assert np.all(np.abs(got - ref) <= 1e-6 * np.maximum(1.0, np.abs(ref)))


@pytest.mark.parametrize("n", [1, 2, 63, 64, 65, 127, 257, 1000, 4099])
@pytest.mark.parametrize("m", [1, 7, 50, 112])
def test_sym_pass_fp32(ctx, oracle_lib, n, m):
    if m > 50 and n in (1, 2):
        return
    A = _sym_A(n, seed=n * 7 + m)
    rng = np.random.default_rng(m)
    X = rng.standard_normal((n, m)).astype(np.float32)
    Xd = _tall_from_np(X, ld=n + 5)
    Y = ps.tall_empty(n, m, "cuda", ld=n + 1)
    Ad = torch.from_numpy(A).cuda()
    ctx.sym_pass(Ad, Xd, Y)
    assert ctx.sync_status() == 0
    A64 = A.astype(np.float64)
    ref = oracle_lib.sym_mul(A64, X.astype(np.float64))
    bound = np.abs(A64) @ np.abs(X.astype(np.float64))
    tol = 8.0 * np.sqrt(n) * EPS32 * bound + 1e-30
    assert np.all(np.abs(_np(Y) - ref) <= tol)


def test_sym_pass_reads_upper_only_and_shift(ctx, oracle_lib):
    n, m = 1000, 40
    A = _sym_A(n, seed=3)
    Ap = _sym_A(n, seed=3, poison=True)
    X = np.random.default_rng(4).standard_normal((n, m)).astype(np.float32)
    Xd = _tall_from_np(X)
    Y1 = ps.tall_empty(n, m)
    Y2 = ps.tall_empty(n, m)
    shift = torch.tensor([2.5], dtype=torch.float64, device="cuda")
    ctx.sym_pass(torch.from_numpy(A).cuda(), Xd, Y1, shift=shift)
    ctx.sym_pass(torch.from_numpy(Ap).cuda(), Xd, Y2, shift=shift)
    assert ctx.sync_status() == 0
    y1, y2 = _np(Y1), _np(Y2)
    assert np.all(np.isfinite(y2))
    ref = oracle_lib.sym_mul(A.astype(np.float64), X.astype(np.float64), shift=2.5)
    bound = np.abs(A.astype(np.float64)) @ np.abs(X.astype(np.float64)) + 2.5 * np.abs(X)
    assert np.all(np.abs(y1 - ref) <= 8 * np.sqrt(n) * EPS32 * bound)
    assert np.all(np.abs(y2 - ref) <= 8 * np.sqrt(n) * EPS32 * bound)


def _cond_tall(n, m, cond, seed):
    rng = np.random.default_rng(seed)
    U, _ = np.linalg.qr(rng.standard_normal((n, m)))
    Vt, _ = np.linalg.qr(rng.standard_normal((m, m)))
    s = np.logspace(0, -np.log10(cond), m)
    return ((U * s) @ Vt).astype(np.float32)


@pytest.mark.parametrize("n,m,cond", [(1000, 50, 10.0), (4099, 112, 100.0), (300, 7, 1e3),
                                      (129, 128, 10.0), (600, 200, 10.0),
                                      # 16-column block edges of the blocked factorization
                                      (500, 16, 10.0), (500, 17, 10.0), (700, 33, 100.0),
                                      (900, 127, 10.0),
                                      # Gram of condition 1e8: the double-float first pass
                                      (3000, 110, 1e4),
                                      # wider than 256 columns (global-memory factorization)
                                      (1000, 305, 10.0), (1200, 512, 10.0)])
def test_cholqr2_orthonormal_same_range(ctx, oracle_lib, n, m, cond):
    Y = _cond_tall(n, m, cond, seed=m)
    Yd = _tall_from_np(Y)
    Q = ps.tall_empty(n, m)
    qr = torch.zeros(1, dtype=torch.int32, device="cuda")
    ctx.cholqr2(Yd, Q, qrank=qr)
    assert ctx.sync_status() == 0
    q = _np(Q)
    assert int(qr.item()) == m
    assert np.abs(q.T @ q - np.eye(m)).max() < 2e-5
    Qo, r = oracle_lib.orth(Y.astype(np.float64))
    assert r == m
    # projector distance: same range (an FP32 Y of condition cond)
    d = np.linalg.norm(q @ (q.T @ Qo) - Qo) / np.sqrt(m)
    assert d < 50 * cond * EPS32 * np.sqrt(m)


def test_cholqr2_dependent_columns(ctx, oracle_lib):
    """Columns dependent exactly in FP32 (duplicates, a zero column, a power-
    of-two multiple) are detected on both sides and give zero Q columns.
    (The GPU Gram sums FP32 products in FP32 within 64-row chunks, so
    dependence is resolved to ~1e-6 relative, not to the oracle's 1e-10.)"""
    n, m = 500, 12
    rng = np.random.default_rng(1)
    B = rng.standard_normal((n, 8)).astype(np.float32)
    Y = np.concatenate([B, B[:, 2:3], np.zeros((n, 1), np.float32), 2.0 * B[:, 5:6],
                        B[:, 0:1]], axis=1)
    Yd = _tall_from_np(Y)
    Q = ps.tall_empty(n, m)
    qr = torch.zeros(1, dtype=torch.int32, device="cuda")
    ctx.cholqr2(Yd, Q, qrank=qr)
    assert ctx.sync_status() == 0
    q = _np(Q)
    Qo, r = oracle_lib.orth(Y.astype(np.float64))
    assert int(qr.item()) == r == 8
    assert np.all(q[:, 8:] == 0)
    live = q[:, :8]
    assert np.abs(live.T @ live - np.eye(8)).max() < 2e-5
    assert np.linalg.norm(live @ (live.T @ Qo[:, :8]) - Qo[:, :8]) < 1e-4


def test_cholqr2_dependent_columns_at_block_edges(ctx, oracle_lib):
    """Exactly dependent columns on both sides of the 16-column block edges
    (the last column of a block, the first of the next) and a zero column
    at the start of the last block: zero Q columns there, the rest
    orthonormal with the oracle's range."""
    n, m = 700, 50
    rng = np.random.default_rng(3)
    Y = rng.standard_normal((n, m)).astype(np.float32)
    Y[:, 15] = Y[:, 2]
    Y[:, 16] = 4.0 * Y[:, 9]
    Y[:, 32] = Y[:, 15] + 0.0
    Y[:, 48] = 0.0
    Yd = _tall_from_np(Y)
    Q = ps.tall_empty(n, m)
    qr = torch.zeros(1, dtype=torch.int32, device="cuda")
    ctx.cholqr2(Yd, Q, qrank=qr)
    assert ctx.sync_status() == 0
    q = _np(Q)
    Qo, r = oracle_lib.orth(Y.astype(np.float64))
    dead = [15, 16, 32, 48]
    assert int(qr.item()) == r == m - len(dead)
    assert np.all(q[:, dead] == 0)
    live_idx = [j for j in range(m) if j not in dead]
    live = q[:, live_idx]
    assert np.abs(live.T @ live - np.eye(len(live_idx))).max() < 2e-5
    Qr = Qo[:, np.abs(Qo).sum(axis=0) > 0]
    assert np.linalg.norm(live @ (live.T @ Qr) - Qr) < 1e-4 * np.sqrt(len(live_idx))


def test_cholqr2_nearly_dependent_columns_keep_range(ctx):
    """Columns dependent only up to FP32 rounding: whatever the rank decision,
    Q stays orthonormal on its live columns and spans range(Y)."""
    n, m = 500, 12
    rng = np.random.default_rng(2)
    B = rng.standard_normal((n, 8))
    Y = np.concatenate([B, B[:, :4] @ rng.standard_normal((4, 4))], axis=1).astype(np.float32)
    Q = ps.tall_empty(n, m)
    qr = torch.zeros(1, dtype=torch.int32, device="cuda")
    ctx.cholqr2(_tall_from_np(Y), Q, qrank=qr)
    assert ctx.sync_status() == 0
    q = _np(Q)
    r = int(qr.item())
    assert 8 <= r <= 12
    live = q[:, np.abs(q).sum(axis=0) > 0]
    assert live.shape[1] == r
    assert np.abs(live.T @ live - np.eye(r)).max() < 2e-4
    Y64 = Y.astype(np.float64)
    assert np.linalg.norm(Y64 - live @ (live.T @ Y64)) <= 1e-5 * np.linalg.norm(Y64)


def test_core_matches_oracle(ctx, oracle_lib):
    n, m = 2000, 60
    A = _sym_A(n, 5)
    Q, _ = np.linalg.qr(np.random.default_rng(2).standard_normal((n, m)))
    Q = Q.astype(np.float32)
    A64, Q64 = A.astype(np.float64), Q.astype(np.float64)
    Z = oracle_lib.sym_mul(A64, Q64).astype(np.float32)   # Z from the oracle
    C = torch.zeros(m, m, dtype=torch.float64, device="cuda")
    ctx.core(_tall_from_np(Q), _tall_from_np(Z), C)
    assert ctx.sync_status() == 0
    ref = Q64.T @ Z.astype(np.float64)
    ref = 0.5 * (ref + ref.T)
    got = C.cpu().numpy().T  # column-major
    bound = np.abs(Q64).T @ np.abs(Z.astype(np.float64))
    assert np.all(np.abs(got - ref) <= 8 * np.sqrt(n) * EPS32 * bound)
    assert np.array_equal(got, got.T)


@pytest.mark.parametrize("m", [1, 2, 3, 17, 60, 110, 112, 161, 210, 256, 305, 512])
@pytest.mark.parametrize("method", [ps.EIG_AUTO, ps.EIG_JACOBI, ps.EIG_TRIDIAG])
def test_eig_matches_lapack(ctx, m, method):
    rng = np.random.default_rng(m)
    X = rng.standard_normal((m, m))
    C = (X + X.T) / 2
    C[: m // 3, : m // 3] *= 10.0
    Cd = torch.from_numpy(np.ascontiguousarray(C.T)).cuda()  # column-major
    V = torch.zeros(m, m, dtype=torch.float32, device="cuda")
    d = torch.zeros(m, dtype=torch.float64, device="cuda")
    ctx.eig(Cd, V, d, method=method)
    assert ctx.sync_status() == 0
    dv = d.cpu().numpy()
    Vv = V.cpu().numpy().T.astype(np.float64)  # column-major -> (row, col)
    ref = np.linalg.eigvalsh(C)[::-1]
    nrm = np.linalg.norm(C)
    if method == ps.EIG_JACOBI:
        assert np.all(np.diff(dv) <= 0)
        assert np.abs(dv - ref).max() <= 2e-6 * nrm
    else:
        # the tridiagonal solver refines its eigenvalues in FP64 (Rayleigh
        # quotients of the FP32 vectors, error quadratic in theirs): within
        # 1e-9 ||C|| of LAPACK, against 2e-6 for FP32 eigenvalues; the
        # ordering is the FP32 one, so values closer than that may swap
        assert np.all(np.diff(dv) <= 1e-9 * nrm)
        assert np.abs(dv - ref).max() <= 1e-9 * nrm
    assert np.abs(Vv.T @ Vv - np.eye(m)).max() <= 2e-5
    assert np.linalg.norm(Vv @ np.diag(dv) @ Vv.T - C) <= 5e-6 * nrm * np.sqrt(m)


@pytest.mark.parametrize("method", [ps.EIG_AUTO, ps.EIG_JACOBI, ps.EIG_TRIDIAG])
def test_eig_degenerate_inputs(ctx, method):
    for C in [np.zeros((5, 5)), np.diag([3.0, 3.0, -1.0, 0.0]), np.eye(6) * 2.0,
              np.ones((1, 1)) * -2.0]:
        m = C.shape[0]
        V = torch.zeros(m, m, dtype=torch.float32, device="cuda")
        d = torch.zeros(m, dtype=torch.float64, device="cuda")
        ctx.eig(torch.from_numpy(np.ascontiguousarray(C.T)).cuda(), V, d, method=method)
        assert ctx.sync_status() == 0
        assert np.allclose(d.cpu().numpy(), np.sort(np.diag(C))[::-1])
        Vv = V.cpu().numpy().T
        assert np.allclose(Vv.T @ Vv, np.eye(m), atol=1e-6)


@pytest.mark.parametrize("method", [ps.EIG_AUTO, ps.EIG_TRIDIAG])
@pytest.mark.parametrize("m", [30, 110, 200])
def test_eig_clusters_in_random_basis(ctx, m, method):
    # exact multiplicities plus near-multiplicities (1e-7 apart) in a random
    # basis: the tridiagonal solver's cluster path; P = V max(D,0) V^T is
    # unique even where V is not
    rng = np.random.default_rng(100 + m)
    q = m // 3
    lam = np.concatenate([np.full(q, 3.0), np.full(q, -1.0), 1e-7 * np.arange(m - 2 * q)])
    U, _ = np.linalg.qr(rng.standard_normal((m, m)))
    C = (U * lam) @ U.T
    C = (C + C.T) / 2
    V = torch.zeros(m, m, dtype=torch.float32, device="cuda")
    d = torch.zeros(m, dtype=torch.float64, device="cuda")
    ctx.eig(torch.from_numpy(np.ascontiguousarray(C.T)).cuda(), V, d, method=method)
    assert ctx.sync_status() == 0
    dv = d.cpu().numpy()
    Vv = V.cpu().numpy().T.astype(np.float64)
    nrm = np.linalg.norm(C)
    assert np.abs(dv - np.sort(lam)[::-1]).max() <= 2e-6 * nrm
    assert np.abs(Vv.T @ Vv - np.eye(m)).max() <= 2e-5
    P = (Vv * np.maximum(dv, 0)) @ Vv.T
    Pe = (U * np.maximum(lam, 0)) @ U.T
    # FP32 Householder backward error grows like m * eps32 * ||C||
    assert np.linalg.norm(P - Pe) <= max(5e-6, 2 * m * EPS32) * nrm


@pytest.mark.parametrize("method", [ps.EIG_AUTO, ps.EIG_JACOBI, ps.EIG_TRIDIAG])
@pytest.mark.parametrize("m", [20, 110, 150])
def test_eig_zero_rows_give_exact_zero_eigenvalues(ctx, m, method):
    # zeroed rows / columns (the dependent columns of Q) must come back as
    # eigenvalue exactly 0 with a unit vector, never as a small positive
    rng = np.random.default_rng(300 + m)
    X = rng.standard_normal((m, m))
    C = (X + X.T) / 2
    dead = [1, 7, m // 2, m - 1]
    C[dead, :] = 0.0
    C[:, dead] = 0.0
    V = torch.zeros(m, m, dtype=torch.float32, device="cuda")
    d = torch.zeros(m, dtype=torch.float64, device="cuda")
    ctx.eig(torch.from_numpy(np.ascontiguousarray(C.T)).cuda(), V, d, method=method)
    assert ctx.sync_status() == 0
    dv = d.cpu().numpy()
    Vv = V.cpu().numpy().T.astype(np.float64)
    ref = np.linalg.eigvalsh(C)[::-1]
    assert np.all(np.diff(dv) <= 0)
    assert np.abs(dv - ref).max() <= 2e-6 * np.linalg.norm(C)
    assert int((dv == 0.0).sum()) >= len(dead)
    live = np.ones(m, bool); live[dead] = False
    assert int((dv > 0).sum()) == int((np.linalg.eigvalsh(C[np.ix_(live, live)]) > 0).sum())
    for i in dead:
        col = np.flatnonzero(np.abs(Vv[i, :]) == 1.0)
        assert col.size == 1 and dv[col[0]] == 0.0
    assert np.abs(Vv.T @ Vv - np.eye(m)).max() <= 2e-5


def test_eig_auto_skips_jacobi_when_tridiagonal_succeeds(ctx):
    # AUTO = the tridiagonal result bit for bit when no failure is flagged
    m = 110
    rng = np.random.default_rng(7)
    X = rng.standard_normal((m, m))
    Cd = torch.from_numpy(np.ascontiguousarray(((X + X.T) / 2).T)).cuda()
    out = []
    for method in (ps.EIG_AUTO, ps.EIG_TRIDIAG):
        V = torch.zeros(m, m, dtype=torch.float32, device="cuda")
        d = torch.zeros(m, dtype=torch.float64, device="cuda")
        ctx.eig(Cd, V, d, method=method)
        assert ctx.sync_status() == 0
        out.append((V.cpu(), d.cpu()))
    assert torch.equal(out[0][0], out[1][0]) and torch.equal(out[0][1], out[1][1])


def test_factor_and_syrk(ctx):
    n, m = 1500, 40
    rng = np.random.default_rng(9)
    Q, _ = np.linalg.qr(rng.standard_normal((n, m)))
    V, _ = np.linalg.qr(rng.standard_normal((m, m)))
    d = np.sort(rng.standard_normal(m))[::-1].copy()
    d[5] = 0.0
    Qd = _tall_from_np(Q)
    Vd = torch.from_numpy(np.ascontiguousarray(V.T).astype(np.float32)).cuda()
    dd = torch.from_numpy(d).cuda()
    W = ps.tall_empty(n, m)
    rank = torch.zeros(1, dtype=torch.int32, device="cuda")
    ctx.factor(Qd, Vd, dd, W, rank=rank)
    P = torch.full((n, n), float("nan"), device="cuda")
    ctx.syrk(W, P, rank=rank)
    Pu = torch.full((n, n), float("nan"), device="cuda")
    ctx.syrk(W, Pu, rank=rank, out_mode=ps.OUT_UPPER)
    assert ctx.sync_status() == 0
    rp = int((d > 0).sum())
    assert int(rank.item()) == rp
    Q32, V32 = Q.astype(np.float32).astype(np.float64), V.astype(np.float32).astype(np.float64)
    Wref = Q32 @ V32[:, :rp] * np.sqrt(d[:rp])
    w = _np(W)
    assert np.abs(w[:, :rp] - Wref).max() < 1e-5 * np.abs(Wref).max()
    assert np.all(w[:, rp:] == 0)
    Pref = w @ w.T
    p = _np(P)
    assert np.abs(p - Pref).max() <= 8 * np.sqrt(m) * EPS32 * (np.abs(w) @ np.abs(w).T).max()
    pu = _np(Pu)
    iu = np.triu_indices(n)
    assert np.array_equal(pu[iu], p[iu])
    assert np.all(np.isnan(pu[np.tril_indices(n, -1)]))


@pytest.mark.parametrize("n,N", [(500, 10), (2051, 10), (64, 0)])
def test_min_eig_matches_oracle(ctx, oracle_lib, n, N):
    Vr, lam = si.make_problem("small", n) if n >= 40 else (None, None)
    A = si.form_A_numpy(Vr, lam).astype(np.float32)
    alpha = torch.zeros(1, dtype=torch.float64, device="cuda")
    s1 = torch.zeros(1, dtype=torch.float64, device="cuda")
    s2 = torch.zeros(1, dtype=torch.float64, device="cuda")
    ctx.min_eig(torch.from_numpy(A).cuda(), N, 3, alpha, s1, s2)
    assert ctx.sync_status() == 0
    a_o, s1_o, s2_o = oracle_lib.min_eig(A.astype(np.float64), N, 3)
    assert abs(s1.item() - s1_o) <= 1e-5 * s1_o
    assert abs(s2.item() - s2_o) <= 1e-5 * s2_o
    assert abs(alpha.item() - a_o) <= 1e-5 * s2_o


# ----------------------------------------------------------------------------
# tensor-core (tcgen05) symmetric pass, BF16 products, FP32 accumulation
# ----------------------------------------------------------------------------
def _bf16(x):
    return torch.from_numpy(np.ascontiguousarray(x, dtype=np.float32)).to(torch.bfloat16).float().numpy()


def _padded_A(A, pad=4):
    """Row-major device copy with lda rounded up to a multiple of `pad`."""
    n = A.shape[0]
    lda = -(-n // pad) * pad
    buf = torch.full((n, lda), float("nan"), device="cuda")
    buf[:, :n] = torch.from_numpy(A).cuda()
    return buf[:, :n]


@pytest.mark.parametrize("n", [1, 63, 64, 65, 255, 256, 257, 1000, 4099])
@pytest.mark.parametrize("m", [1, 7, 50, 64, 65, 110, 112, 113, 128])
def test_sym_pass_bf16_tensor_cores(ctx, oracle_lib, n, m):
    A = _sym_A(n, seed=n + 13 * m)
    rng = np.random.default_rng(m + 1)
    X = rng.standard_normal((n, m)).astype(np.float32)
    Ad = _padded_A(A)
    Xd = _tall_from_np(X, ld=n + 4)
    Y = ps.tall_empty(n, m, "cuda", ld=-(-n // 4) * 4)
    shift = torch.tensor([0.75], dtype=torch.float64, device="cuda")
    ctx.sym_pass(Ad, Xd, Y, shift=shift, prec=ps.PREC_BF16)
    assert ctx.sync_status() == 0
    Ab, Xb = _bf16(A).astype(np.float64), _bf16(X).astype(np.float64)
    ref = oracle_lib.sym_mul(Ab, Xb) + 0.75 * X.astype(np.float64)
    bound = np.abs(Ab) @ np.abs(Xb) + 0.75 * np.abs(X)
    got = _np(Y)
    assert np.all(np.abs(got - ref) <= 8 * np.sqrt(n) * EPS32 * bound + 1e-30)


def test_sym_pass_bf16_lower_triangle_and_strides(ctx, oracle_lib):
    n, m = 777, 33
    A = _sym_A(n, seed=5)
    Ap = _sym_A(n, seed=5, poison=True)
    X = np.random.default_rng(6).standard_normal((n, m)).astype(np.float32)
    Y1 = ps.tall_empty(n, m, "cuda", ld=n + 3)   # ld not a multiple of 4: scalar atomics
    Y2 = ps.tall_empty(n, m, "cuda", ld=n + 1)
    ctx.sym_pass(_padded_A(A), _tall_from_np(X), Y1, prec=ps.PREC_BF16)
    ctx.sym_pass(_padded_A(Ap), _tall_from_np(X), Y2, prec=ps.PREC_BF16)
    assert ctx.sync_status() == 0
    y1, y2 = _np(Y1), _np(Y2)
    assert np.all(np.isfinite(y2))
    Ab, Xb = _bf16(A).astype(np.float64), _bf16(X).astype(np.float64)
    ref = oracle_lib.sym_mul(Ab, Xb)
    bound = np.abs(Ab) @ np.abs(Xb)
    for y in (y1, y2):
        assert np.all(np.abs(y - ref) <= 8 * np.sqrt(n) * EPS32 * bound)


def test_sym_pass_bf16_any_lda(ctx, oracle_lib):
    # lda = 10 (not a multiple of 4): the BF16 image is packed with scalar loads
    n, m = 10, 2
    A = _sym_A(n, seed=21)
    X = np.random.default_rng(22).standard_normal((n, m)).astype(np.float32)
    Y = ps.tall_empty(n, m)
    ctx.sym_pass(torch.from_numpy(A).cuda(), _tall_from_np(X), Y, prec=ps.PREC_BF16)
    assert ctx.sync_status() == 0
    Ab, Xb = _bf16(A).astype(np.float64), _bf16(X).astype(np.float64)
    ref = oracle_lib.sym_mul(Ab, Xb)
    bound = np.abs(Ab) @ np.abs(Xb)
    assert np.all(np.abs(_np(Y) - ref) <= 8 * np.sqrt(n) * EPS32 * bound + 1e-30)


@pytest.mark.parametrize("prec", [ps.PREC_BF16, ps.PREC_BF16X3, ps.PREC_TF32])
@pytest.mark.parametrize("m", [129, 256, 305])
def test_sym_pass_tensor_core_wide_sketch(ctx, oracle_lib, prec, m):
    # more than 128 columns: column slices of 128, one pass each
    n = 700
    A = _sym_A(n, seed=m + prec)
    X = np.random.default_rng(m).standard_normal((n, m)).astype(np.float32)
    Y = ps.tall_empty(n, m, "cuda", ld=704)
    shift = torch.tensor([-0.5], dtype=torch.float64, device="cuda")
    ctx.sym_pass(_padded_A(A), _tall_from_np(X), Y, shift=shift, prec=prec)
    assert ctx.sync_status() == 0
    if prec == ps.PREC_BF16:
        Ar, Xr, extra = _bf16(A), _bf16(X), 0.0
    elif prec == ps.PREC_TF32:
        Ar, Xr, extra = _tf32(A), _tf32(X), 0.0
    else:
        Ar, Xr, extra = A, X, 4 * 2.0 ** -16
    Ar, Xr = Ar.astype(np.float64), Xr.astype(np.float64)
    ref = oracle_lib.sym_mul(Ar, Xr) - 0.5 * X.astype(np.float64)
    bound = np.abs(Ar) @ np.abs(Xr) + 0.5 * np.abs(X)
    assert np.all(np.abs(_np(Y) - ref) <= (extra + 8 * np.sqrt(n) * EPS32) * bound + 1e-30)


def _tf32(x):
    # FP32 -> TF32 by rounding to nearest, ties away from zero: add half of the
    # last kept place to the magnitude bits, then clear the 13 dropped bits
    u = np.ascontiguousarray(x, dtype=np.float32).view(np.uint32)
    return ((u + np.uint32(0x1000)) & np.uint32(0xFFFFE000)).view(np.float32)


def test_tf32_rounding_helper():
    one_ulp = 2.0 ** -10                       # TF32 keeps 10 fraction bits
    x = np.array([1.0, 1.0 + one_ulp / 2, -(1.0 + one_ulp / 2), 1.0 + one_ulp / 4,
                  1.0 + 0.75 * one_ulp, 3.0 * 2.0 ** -130], dtype=np.float32)
    want = np.array([1.0, 1.0 + one_ulp, -(1.0 + one_ulp), 1.0, 1.0 + one_ulp, 3.0 * 2.0 ** -130])
    assert np.array_equal(_tf32(x).astype(np.float64), want)


@pytest.mark.parametrize("n", [1, 65, 257, 1000, 4099])
@pytest.mark.parametrize("m", [1, 50, 110, 128])
def test_sym_pass_tf32_tensor_cores(ctx, oracle_lib, n, m):
    # full TF32 image of A (mirrored from the upper triangle) and TF32 copy of
    # X, both rounded to nearest with ties away; products exact in FP32,
    # accumulation in FP32
    A = _sym_A(n, seed=n + 11 * m)
    rng = np.random.default_rng(m + 5)
    X = rng.standard_normal((n, m)).astype(np.float32)
    Y = ps.tall_empty(n, m, "cuda", ld=-(-n // 4) * 4)
    shift = torch.tensor([0.25], dtype=torch.float64, device="cuda")
    ctx.sym_pass(_padded_A(A), _tall_from_np(X, ld=n + 2), Y, shift=shift, prec=ps.PREC_TF32)
    assert ctx.sync_status() == 0
    At, Xt = _tf32(A).astype(np.float64), _tf32(X).astype(np.float64)
    ref = oracle_lib.sym_mul(At, Xt) + 0.25 * X.astype(np.float64)
    bound = np.abs(At) @ np.abs(Xt) + 0.25 * np.abs(X)
    assert np.all(np.abs(_np(Y) - ref) <= 8 * np.sqrt(n) * EPS32 * bound + 1e-30)


def test_sym_pass_tf32_lower_triangle_and_strides(ctx, oracle_lib):
    n, m = 777, 33
    A = _sym_A(n, seed=8)
    Ap = _sym_A(n, seed=8, poison=True)
    X = np.random.default_rng(9).standard_normal((n, m)).astype(np.float32)
    Y1 = ps.tall_empty(n, m, "cuda", ld=n + 3)   # ld not a multiple of 4: scalar atomics
    Y2 = ps.tall_empty(n, m, "cuda", ld=n + 1)
    ctx.sym_pass(torch.from_numpy(A).cuda(), _tall_from_np(X), Y1, prec=ps.PREC_TF32)   # lda = 777
    ctx.sym_pass(_padded_A(Ap), _tall_from_np(X), Y2, prec=ps.PREC_TF32)
    assert ctx.sync_status() == 0
    y1, y2 = _np(Y1), _np(Y2)
    assert np.all(np.isfinite(y2))
    At, Xt = _tf32(A).astype(np.float64), _tf32(X).astype(np.float64)
    ref = oracle_lib.sym_mul(At, Xt)
    bound = np.abs(At) @ np.abs(Xt)
    for y in (y1, y2):
        assert np.all(np.abs(y - ref) <= 8 * np.sqrt(n) * EPS32 * bound)


@pytest.mark.parametrize("n", [1, 65, 257, 1000, 4099])
@pytest.mark.parametrize("m", [1, 50, 112, 128])
def test_sym_pass_split_bf16(ctx, oracle_lib, n, m):
    # A X ~ A_hi X_hi + A_hi X_lo + A_lo X_hi with BF16 rounding (unit roundoff
    # 2^-8): |a - hi - lo| <= 2^-16 |a|, same for x, and the dropped lo lo term
    # is <= 2^-16 |a||x|, so each entry is within about 3 2^-16 |A||X| of the
    # exact product (4 2^-16 allowed), plus the FP32 accumulation
    A = _sym_A(n, seed=n + 7 * m)
    rng = np.random.default_rng(m + 3)
    X = rng.standard_normal((n, m)).astype(np.float32)
    Y = ps.tall_empty(n, m, "cuda", ld=-(-n // 4) * 4)
    shift = torch.tensor([0.5], dtype=torch.float64, device="cuda")
    ctx.sym_pass(_padded_A(A), _tall_from_np(X), Y, shift=shift, prec=ps.PREC_BF16X3)
    assert ctx.sync_status() == 0
    A64, X64 = A.astype(np.float64), X.astype(np.float64)
    ref = oracle_lib.sym_mul(A64, X64) + 0.5 * X64
    bound = np.abs(A64) @ np.abs(X64) + 0.5 * np.abs(X64)
    got = _np(Y)
    assert np.all(np.abs(got - ref) <= (4 * 2.0 ** -16 + 8 * np.sqrt(n) * EPS32) * bound + 1e-30)


# ----------------------------------------------------------------------------
# tensor-core SYRK P = W W^T (split BF16, FP32 accumulation)
# ----------------------------------------------------------------------------
@pytest.mark.parametrize("n,m,r", [(1, 1, 1), (100, 17, 17), (128, 128, 128), (129, 40, 33),
                                   (1000, 112, 87), (4099, 110, 110), (300, 50, 0)])
def test_syrk_split_bf16_tensor_cores(ctx, n, m, r):
    rng = np.random.default_rng(n + m)
    W = rng.standard_normal((n, m)).astype(np.float32)
    W[:, r:] = 0.0
    Wd = _tall_from_np(W, ld=n + 2)
    rank = torch.tensor([r], dtype=torch.int32, device="cuda")
    ldp = -(-n // 4) * 4
    Pbuf = torch.full((n, ldp), float("nan"), device="cuda")
    P = Pbuf[:, :n]
    ctx.syrk(Wd, P, rank=rank, prec=ps.PREC_BF16X3)
    Pub = torch.full((n, ldp), float("nan"), device="cuda")
    Pu = Pub[:, :n]
    ctx.syrk(Wd, Pu, rank=rank, out_mode=ps.OUT_UPPER, prec=ps.PREC_BF16X3)
    assert ctx.sync_status() == 0
    W64 = W.astype(np.float64)[:, :r]
    ref = W64 @ W64.T
    bound = np.abs(W64) @ np.abs(W64).T
    p = P.cpu().numpy().astype(np.float64)
    assert np.all(np.abs(p - ref) <= 3e-5 * bound + 1e-30)
    pu = Pu.cpu().numpy().astype(np.float64)
    iu = np.triu_indices(n)
    assert np.array_equal(pu[iu], p[iu])
    if n > 1:
        assert np.all(np.isnan(pu[np.tril_indices(n, -1)]))


# ----------------------------------------------------------------------------
# SRHT test matrix (footnote to Alg. 1): bit-exact against the oracle
# ----------------------------------------------------------------------------
@pytest.mark.parametrize("n,m,seed", [(64, 64, 5), (100, 40, 123456789012345), (1000, 110, 1),
                                      (777, 256, 2 ** 40 + 3), (20000, 112, 1)])
def test_srht_matches_oracle_bit_exactly(ctx, oracle_lib, n, m, seed):
    X = ps.tall_empty(n, m, "cuda", ld=n + 3)
    ctx.srht(seed, X)
    assert ctx.sync_status() == 0
    # integer work (Philox words, picks, popcounts) decides +-1: bit-exact
    assert np.array_equal(_np(X), oracle_lib.omega_srht(seed, n, m))
