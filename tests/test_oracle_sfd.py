"""Pins for the FP64 oracle of Sparse Frequent Directions.

Each check compares the oracle to something other than itself: a worked
example, brute-force eigendecompositions through a different library routine,
closed forms, or the inequalities the paper proves (Props. 1-3 of Sec. 4.3,
Lemma 4.1, Theorem 4.1, the FD bound of Sec. 2, mergeability of Sec. 3.1).
"""
import math
import os

import numpy as np
import pytest
import scipy.sparse as sp

from oracle import metrics, philox
from oracle import sfd as O
from paper_1602_00412_gb300 import synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def bbt(B):
    return B.T @ B


def brute_dense_shrink(M, ell):
    """DenseShrink through the eigendecomposition of M^T M (eigh), not an SVD."""
    w, V = np.linalg.eigh(M.T @ M)
    order = np.argsort(w)[::-1]
    w, V = np.maximum(w[order], 0.0), V[:, order]
    wl = w[ell - 1] if ell - 1 < len(w) else 0.0
    return (V[:, :ell] * np.maximum(w[:ell] - wl, 0.0)) @ V[:, :ell].T   # = B^T B


def random_sparse(rng, m, d, density, rank=None):
    if rank is None:
        A = sp.random(m, d, density=density, random_state=rng, data_rvs=rng.standard_normal)
        return A.tocsr()
    U = rng.standard_normal((m, rank))
    V = rng.standard_normal((rank, d))
    return sp.csr_matrix(U @ V)


# ----------------------------------------------------------------------------
# Alg. 5 DenseShrink
# ----------------------------------------------------------------------------
def test_dense_shrink_golden():
    with open(os.path.join(GOLDEN, "dense_shrink_diag.txt")) as f:
        cases = [ln for ln in f if ln.strip() and not ln.startswith("#")]
    assert len(cases) == 3
    for ln in cases:
        ell_s, m_s, want_s = ln.split("|")
        M = np.array([[float(x) for x in r.split()] for r in m_s.split(";")])
        B = O.dense_shrink(M, int(ell_s))
        assert B.shape == (int(ell_s), M.shape[1])
        np.testing.assert_allclose(np.diag(bbt(B)), [float(x) for x in want_s.split()], atol=1e-12)
        np.testing.assert_allclose(bbt(B) - np.diag(np.diag(bbt(B))), 0, atol=1e-12)


@pytest.mark.parametrize("rows,d,ell", [(8, 12, 4), (20, 15, 6), (10, 40, 10), (6, 6, 5)])
def test_dense_shrink_vs_eigh(rows, d, ell):
    rng = np.random.default_rng(rows * 100 + d)
    M = rng.standard_normal((rows, d)) * (0.7 ** np.arange(d))[None, :]
    B = O.dense_shrink(M, ell)
    np.testing.assert_allclose(bbt(B), brute_dense_shrink(M, ell), atol=1e-10)
    # last row is zero; Prop. 1: M^T M - B^T B is PSD
    assert np.allclose(B[-1], 0)
    assert np.linalg.eigvalsh(M.T @ M - bbt(B)).min() > -1e-9


def test_dense_shrink_of_zero_stack_is_identity():
    # first buffer: B = 0, DSh([0; B']) = B' up to rotation when B' has a zero last row
    rng = np.random.default_rng(1)
    Bp = O.dense_shrink(rng.standard_normal((9, 30)), 6)
    B = O.dense_shrink(np.vstack([np.zeros((6, 30)), Bp]), 6)
    np.testing.assert_allclose(bbt(B), bbt(Bp), atol=1e-10)


def test_dense_shrink_rank_deficient_exact():
    rng = np.random.default_rng(2)
    M = rng.standard_normal((3, 20))
    B = O.dense_shrink(M, 5)
    np.testing.assert_allclose(bbt(B), M.T @ M, atol=1e-10)


# ----------------------------------------------------------------------------
# schedules
# ----------------------------------------------------------------------------
def test_q_schedule_closed_form():
    # q = ceil(ln(4m)) at c_q = 1/4
    for m in [1, 2, 50, 2000, 50000, 200000, 10 ** 6]:
        assert O.q_fixed(m) == math.ceil(math.log(4 * m))
    assert [O.q_fixed(m) for m in (2000, 50000, 200000, 10 ** 6)] == [9, 13, 14, 16]
    assert O.q_fixed(2000, c_q=0.5) == math.ceil(2 * math.log(8000))


def test_delta_budget_sums_to_delta():
    tot = sum(O.delta_br(0.01, b, r) for b in range(20000) for r in range(40))
    # tail of sum 1/(b+1)^2 beyond 20000 is ~ 1/20000
    assert 0.01 * (1 - 1e-4) < tot <= 0.01
    assert O.delta_br(0.01, 0, 0) == pytest.approx(0.01 * 3 / math.pi ** 2)


def test_vs_steps_from_lemma_bound():
    # p is the least integer with 2^p * t >= 1 for t = delta_i / sqrt(2d/pi)
    for d in (10, 2000, 50000):
        for di in (1e-2, 1e-5):
            p = O.vs_steps(d, di)
            t = di / math.sqrt(2 * d / math.pi)
            assert 2 ** p * t >= 1 > 2 ** (p - 1) * t


def test_lemma41_anticoncentration():
    # Pr[|<v1, x>| <= t] <= t sqrt(2d/pi) for x uniform on the sphere (Lemma 4.1 proof)
    d = 200
    z = philox.normals(3, 0, 0, philox.TAG_VS, d * 20000).reshape(20000, d)
    x1 = z[:, 0] / np.linalg.norm(z, axis=1)
    for t in (0.01, 0.03, 0.05):
        assert (np.abs(x1) <= t).mean() <= t * math.sqrt(2 * d / math.pi) * 1.05 + 0.002


# ----------------------------------------------------------------------------
# Alg. 6 VerifySpectral
# ----------------------------------------------------------------------------
def _sym_with_spectrum(rng, d, eig):
    Q, _ = np.linalg.qr(rng.standard_normal((d, d)))
    return (Q * eig) @ Q.T


def test_vs_accepts_when_norm_at_most_one():
    rng = np.random.default_rng(4)
    d = 60
    for top in (1.0, 0.999, 0.5):
        eig = np.concatenate([[top], rng.uniform(0, top, d - 1)])
        C = _sym_with_spectrum(rng, d, eig)
        for s in range(30):
            x = philox.sphere_x(s, 0, 0, d)
            ok, _ = O.verify_spectral(lambda v: C @ v, x, O.vs_steps(d, 0.01))
            assert ok


@pytest.mark.parametrize("top", [2.0, 3.0])
def test_vs_rejects_norm_two_whp(top):
    rng = np.random.default_rng(5)
    d, di = 60, 0.05
    eig = np.concatenate([[top], rng.uniform(0, 0.9, d - 1)])
    C = _sym_with_spectrum(rng, d, eig)
    p = O.vs_steps(d, di)
    fails = 0
    trials = 2000
    for s in range(trials):
        ok, _ = O.verify_spectral(lambda v: C @ v, philox.sphere_x(s, 1, 0, d), p)
        fails += ok
    bound = 2.0 ** -p * math.sqrt(2 * d / math.pi)                 # <= delta_i by choice of p
    assert bound <= di
    assert fails / trials <= bound + 3 * math.sqrt(bound * (1 - bound) / trials)


def test_vs_logsum_matches_direct_power():
    rng = np.random.default_rng(6)
    d = 30
    C = _sym_with_spectrum(rng, d, rng.uniform(0, 1.5, d))
    x = philox.sphere_x(1, 0, 0, d)
    ok, L = O.verify_spectral(lambda v: C @ v, x, 7)
    direct = np.linalg.norm(np.linalg.matrix_power(C, 7) @ x)
    assert math.isclose(L, math.log(direct), rel_tol=1e-10)
    assert ok == (direct <= 1.0)


# ----------------------------------------------------------------------------
# Alg. 1 / Alg. 3 SimultaneousIteration + SparseShrink
# ----------------------------------------------------------------------------
def test_si_orthonormal_and_spectral_bound():
    # Musco-Musco spectral bound used in Sec. 4.3: ||(I - Z Z^T) A||_2 <= (1+eps) s_{l+1}
    rng = np.random.default_rng(7)
    for trial in range(5):
        m, d, ell = 80, 60, 8
        A = sp.csr_matrix(rng.standard_normal((m, d)) * (0.85 ** np.arange(d))[None, :])
        G = philox.gaussian_G(trial, 0, 0, d, ell)
        Z = O.simultaneous_iteration(A, ell, O.q_fixed(m), G)
        np.testing.assert_allclose(Z.T @ Z, np.eye(ell), atol=1e-12)
        s = np.linalg.svd(A.toarray(), compute_uv=False)
        R = A.toarray() - Z @ (Z.T @ A.toarray())
        assert np.linalg.norm(R, 2) <= 1.25 * s[ell]


@pytest.mark.parametrize("q", [0, 1, 2])
def test_si_span_equals_unnormalised_product(q):
    # R1: orthonormalising after every product leaves span(A (A^T A)^q G) unchanged
    rng = np.random.default_rng(30 + q)
    m, d, ell = 40, 30, 4
    A = sp.csr_matrix(rng.standard_normal((m, d)) * (0.9 ** np.arange(d))[None, :])
    G = philox.gaussian_G(q, 0, 0, d, ell)
    Ad = A.toarray()
    Y = Ad @ np.linalg.matrix_power(Ad.T @ Ad, q) @ G
    U, _, _ = np.linalg.svd(Y, full_matrices=False)
    Z = O.simultaneous_iteration(A, ell, q, G)
    np.testing.assert_allclose(Z @ Z.T, U @ U.T, atol=1e-9)


def test_si_finds_top_subspace_on_gap():
    rng = np.random.default_rng(8)
    m, d, ell = 50, 40, 5
    U, _ = np.linalg.qr(rng.standard_normal((m, m)))
    V, _ = np.linalg.qr(rng.standard_normal((d, d)))
    s = np.concatenate([np.linspace(10, 6, ell), np.linspace(1, 0.1, min(m, d) - ell)])
    A = sp.csr_matrix((U[:, :len(s)] * s) @ V[:, :len(s)].T)
    Z = O.simultaneous_iteration(A, ell, 12, philox.gaussian_G(0, 0, 0, d, ell))
    Pz = Z @ Z.T
    Pu = U[:, :ell] @ U[:, :ell].T
    assert np.linalg.norm(Pz - Pu) < 1e-9


def test_sparse_shrink_rank_deficient_equals_dense_shrink():
    rng = np.random.default_rng(9)
    m, d, ell = 30, 25, 6
    for rank in (3, 6):
        A = sp.csr_matrix(rng.standard_normal((m, rank)) @ rng.standard_normal((rank, d)))
        Bp, _ = O.sparse_shrink(A, ell, O.q_fixed(m), philox.gaussian_G(rank, 0, 0, d, ell))
        np.testing.assert_allclose(bbt(Bp), brute_dense_shrink(A.toarray(), ell), atol=1e-8)


def test_sparse_shrink_identities_and_props():
    """Sec. 4.3: ||P||_F^2 - ||B'||_F^2 = l lambda_l^2; Prop. 1 always; Props. 2
    (strengthened) and 3 with high probability, s_l from a brute-force SVD."""
    rng = np.random.default_rng(10)
    passes2 = passes3 = 0
    trials = 12
    for t in range(trials):
        m, d, ell = 120, 90, 10
        A = random_sparse(rng, m, d, 0.08)
        Bp, info = O.sparse_shrink(A, ell, O.q_fixed(m), philox.gaussian_G(t, 0, 0, d, ell))
        P, lam = info["P"], info["lam"]
        assert math.isclose((P ** 2).sum() - (Bp ** 2).sum(), ell * lam[ell - 1] ** 2,
                            rel_tol=1e-10)
        Ad = A.toarray()
        R = Ad.T @ Ad - bbt(Bp)
        w = np.linalg.eigvalsh(R)
        assert w[0] > -1e-9 * np.abs(w).max()                       # Prop. 1
        s = np.linalg.svd(Ad, compute_uv=False)
        passes2 += w[-1] <= 41 / 16 * s[ell - 1] ** 2              # Prop. 2 (strengthened)
        passes3 += (Ad ** 2).sum() - (Bp ** 2).sum() >= ell * 0.75 * s[ell - 1] ** 2   # Prop. 3
        assert np.allclose(Bp[-1], 0)
    assert passes2 >= trials - 1 and passes3 >= trials - 1


def test_sparse_shrink_converges_to_dense_shrink_on_gap():
    d = 2000
    X = synth.c1_gapped(seed=3, n=2000)
    A = X.to_scipy()
    Bp, _ = O.sparse_shrink(A, 50, 40, philox.gaussian_G(0, 0, 0, d, 50))
    ref = brute_dense_shrink(A.toarray(), 50)
    assert np.linalg.norm(bbt(Bp) - ref) / np.linalg.norm(ref) < 1e-8


# ----------------------------------------------------------------------------
# Alg. 4 BoostedSparseShrink
# ----------------------------------------------------------------------------
def test_boosted_sparse_shrink_retry_and_keys():
    rng = np.random.default_rng(11)
    A = random_sparse(rng, 60, 40, 0.1)
    Bp2, info = O.boosted_sparse_shrink(A, 6, 0.01, 17, 3, 5, inject_fail=2)
    assert info["attempts"] == 3 and info["verified"] and info["injected"] == 2
    # attempt r = 2 uses the draw keyed (b=3, r=2)
    direct, _ = O.sparse_shrink(A, 6, 5, philox.gaussian_G(17, 3, 2, 40, 6))
    np.testing.assert_allclose(Bp2, direct)
    _, info = O.boosted_sparse_shrink(A, 6, 0.01, 17, 3, 5, retry_cap=2, inject_fail=5)
    assert info["attempts"] == 2 and not info["verified"] and info["injected"] == 2


def _step_spectrum_matrix(m=250, d=300, seed=0):
    """l - 1 = 19 strong directions (sigma 10), one at sigma 4, 100 weak ones
    (sigma 0.3), random orthonormal singular vectors. With q = 0 the start
    block A'G often mixes the sigma-4 direction with the weak ones, so Z misses
    most of it; the shrink by lambda_l^2 is then small and the missed direction
    dominates the residual: ||A'^T A' - B'^T B'|| > Delta / 2."""
    rng = np.random.default_rng(seed)
    spec = np.concatenate([np.full(19, 10.0), [4.0], np.full(100, 0.3)])
    U, _ = np.linalg.qr(rng.standard_normal((m, spec.size)))
    V, _ = np.linalg.qr(rng.standard_normal((d, spec.size)))
    return sp.csr_matrix((U * spec) @ V.T)


def test_bssh_catches_a_failed_shrink():
    # q = 0 on a spectrum with a step at l: some runs miss the l-th direction.
    # Lemma 4.1: VS accepts every run whose residual norm is within Delta/2
    # (deterministically) and rejects those at or above Delta (w.h.p.)
    A = _step_spectrum_matrix()
    Ad = A.toarray()
    m, d = Ad.shape
    ell = 20
    seen = {"accept_small": 0, "reject_large": 0, "accept_large": 0}
    for s in range(24):
        Bp, _ = O.sparse_shrink(A, ell, 0, philox.gaussian_G(s, 0, 0, d, ell))
        Delta = ((Ad ** 2).sum() - (Bp ** 2).sum()) / (O.ALPHA * ell)
        nrm = np.linalg.eigvalsh(Ad.T @ Ad - bbt(Bp))[-1]
        ok, _ = O.verify_spectral(O.residual_operator(A, Bp, Delta), philox.sphere_x(s, 0, 0, d),
                                  O.vs_steps(d, 1e-3))
        if nrm <= Delta / 2:
            assert ok
            seen["accept_small"] += 1
        if nrm >= Delta:
            seen["reject_large" if not ok else "accept_large"] += 1
    assert seen["accept_small"] >= 3 and seen["reject_large"] >= 3, seen
    assert seen["accept_large"] <= 1, seen
    # and BoostedSparseShrink retries such a buffer until VS accepts
    _, info = O.boosted_sparse_shrink(A, ell, 0.01, 0, 0, 0)
    assert info["verified"] and info["attempts"] >= 2
    assert all(h["logsum"] > 0 for h in info["history"][:-1])


# ----------------------------------------------------------------------------
# Alg. 2 SFD end to end, FD, merge, flush
# ----------------------------------------------------------------------------
def _sfd_small(seed=0, n=1500, d=120, ell=12):
    X = synth.planted(n, d, 8, 1.1, 6, 10.0, 0.7, 0.1, seed)
    B, o = O.sfd_stream(X.indptr, X.indices, X.values, d, ell, seed)
    return X, B, o


def test_sfd_bounds_small():
    X, B, o = _sfd_small()
    A = X.to_scipy()
    lo, hi = metrics.residual_eigs(A, B)
    assert lo > -1e-8 * metrics.fro2(A)                            # Prop. 1 through the stream
    for k in (0, 1):                                               # Theorem 4.1, k < alpha l
        assert hi <= metrics.sfd_bound(A, 12, k)
    for k in (0, 2, 5, 8):                                         # FD bound (empirical target)
        assert hi <= metrics.fd_bound(A, 12, k)
    assert len(o.log) >= 10 and all(e["verified"] for e in o.log if e["q"] is not None)


def test_fd_classical_bound_deterministic():
    X = synth.planted(600, 80, 10, 1.1, 6, 10.0, 0.7, 0.1, 4)
    A = X.to_scipy()
    for ell in (8, 16):
        B = O.frequent_directions(A, ell)
        lo, hi = metrics.residual_eigs(A, B)
        assert lo > -1e-8 * metrics.fro2(A)
        for k in range(0, ell, 3):
            assert hi <= metrics.fd_bound(A, ell, k) * (1 + 1e-9)


def test_sfd_close_to_fd_error():
    X, B, _ = _sfd_small(seed=2)
    A = X.to_scipy()
    fd = metrics.cov_err(A, O.frequent_directions(A, 12))
    ours = metrics.cov_err(A, B)
    assert ours <= 2.0 * fd


def test_buffer_boundaries_chunking_invariant():
    X = synth.planted(900, 60, 10, 1.1, 4, 10.0, 0.7, 0.1, 5)
    ref, o1 = O.sfd_stream(X.indptr, X.indices, X.values, 60, 8, 9)
    o2 = O.SFDOracle(60, 8, 9)
    rng = np.random.default_rng(0)
    cuts = np.sort(rng.choice(np.arange(1, X.n), size=25, replace=False))
    prev = 0
    for c in list(cuts) + [X.n]:
        part = X.rows(prev, c)
        o2.append_rows(part.indptr, part.indices, part.values)
        prev = c
    np.testing.assert_array_equal(o2.sketch(), ref)
    assert [e["m"] for e in o1.log] == [e["m"] for e in o2.log]


def test_buffer_trigger_rules():
    # rows rule: m = d rows; nnz rule: first row where nnz >= l d
    ends, pr, pn = O.buffer_boundaries([1] * 25, 10, 3)
    assert ends == [10, 20] and (pr, pn) == (5, 5)
    ends, pr, pn = O.buffer_boundaries([4, 4, 4, 4, 4, 4], 5, 2)   # l d = 10
    assert ends == [3, 6] and (pr, pn) == (0, 0)
    ends, pr, pn = O.buffer_boundaries([5, 5, 2], 5, 2)            # nnz = l d exactly fires
    assert ends == [2] and (pr, pn) == (1, 2)
    # a pending buffer of 1 row / 5 nnz: 5+3 = 8 < l d = 10, then 11 >= 10
    ends, _, _ = O.buffer_boundaries([3, 3], 5, 2, start_rows=1, start_nnz=5)
    assert ends == [2]
    ends, _, _ = O.buffer_boundaries([3, 3], 5, 2, start_rows=4, start_nnz=1)
    assert ends == [1]                                             # rows rule: 4 + 1 = d


def test_short_stream_is_exact():
    # fewer than l rows in total: the flush takes DSh([0; A']) which keeps everything
    X = synth.planted(7, 40, 6, 1.1, 3, 10.0, 0.7, 0.1, 6)
    B, o = O.sfd_stream(X.indptr, X.indices, X.values, 40, 10, 0)
    A = X.to_scipy().toarray()
    np.testing.assert_allclose(bbt(B), A.T @ A, atol=1e-9)
    assert o.log[0]["q"] is None


def test_merge_identity_and_bounds():
    X = synth.planted(1200, 60, 8, 1.1, 5, 10.0, 0.7, 0.1, 7)
    a = O.SFDOracle(60, 10, 1)
    a.append_rows(X.rows(0, 600).indptr, X.rows(0, 600).indices, X.rows(0, 600).values)
    Ba = a.sketch()
    empty = O.SFDOracle(60, 10, 2)
    a.merge(empty)
    np.testing.assert_allclose(bbt(a.sketch()), bbt(Ba), atol=1e-9)
    b = O.SFDOracle(60, 10, 3)
    part = X.rows(600, 1200)
    b.append_rows(part.indptr, part.indices, part.values)
    a.merge(b)
    A = X.to_scipy()
    lo, hi = metrics.residual_eigs(A, a.sketch())
    assert lo > -1e-8 * metrics.fro2(A)
    assert hi <= metrics.fd_bound(A, 10, 0)


def test_shrink_outputs_have_orthogonal_rows():
    # The reading behind the GPU's cross-block Gram in DenseShrink: B' of
    # Alg. 3 and B of Alg. 5 have orthogonal rows, so the Gram of the stack
    # [B; B'] is [[diag, B B'^T], [B' B^T, diag]], and DenseShrink formed from
    # that block form equals Alg. 5 on the stack.
    d, ell = 300, 12
    A = synth.planted(900, d, 15, 1.1, 6, 10.0, 0.8, 0.1, 4).to_scipy().astype(np.float64)
    G = philox.gaussian_G(0, 0, 0, d, ell)
    Bp, _ = O.sparse_shrink(A, ell, 6, G)
    rng = np.random.default_rng(5)
    B = O.dense_shrink(rng.standard_normal((2 * ell, d)), ell)
    for R in (Bp, B):
        K = R @ R.T
        off = K - np.diag(np.diag(K))
        assert np.max(np.abs(off)) <= 1e-10 * np.max(np.diag(K))
    M = np.vstack([B, Bp])
    K = np.zeros((2 * ell, 2 * ell))
    K[:ell, :ell] = np.diag(np.sum(B * B, axis=1))
    K[ell:, ell:] = np.diag(np.sum(Bp * Bp, axis=1))
    K[:ell, ell:] = B @ Bp.T
    K[ell:, :ell] = K[:ell, ell:].T
    w, U = np.linalg.eigh(K)
    order = np.argsort(w)[::-1][:ell]
    w, U = np.maximum(w[order], 0.0), U[:, order]
    wt = np.sqrt(np.maximum(w - w[-1], 0.0)) / np.sqrt(np.where(w > 0, w, 1.0))
    Bnew = (wt[:, None] * U.T) @ M
    assert metrics.bbt_rel_diff(Bnew, O.dense_shrink(M, ell)) <= 1e-9


def test_bbt_rel_diff_matches_dense():
    rng = np.random.default_rng(3)
    B1, B2 = rng.standard_normal((5, 30)), rng.standard_normal((5, 30))
    want = np.linalg.norm(B1.T @ B1 - B2.T @ B2) / np.linalg.norm(B2.T @ B2)
    assert math.isclose(metrics.bbt_rel_diff(B1, B2), want, rel_tol=1e-9)


def test_cov_norm_operator_path_matches_dense():
    X = synth.planted(400, 3100, 30, 1.1, 4, 10.0, 0.7, 0.1, 8)
    A = X.to_scipy()
    B = np.random.default_rng(0).standard_normal((6, 3100)) * 0.1
    dense = metrics.cov_norm(A, B, dense_limit=4000)
    op = metrics.cov_norm(A, B, dense_limit=100)
    assert math.isclose(dense, op, rel_tol=1e-6)


def test_fd_stream_exact_below_l_and_bound():
    # fewer rows than l: the stack [0; A] has rank < l, its l-th singular value
    # is 0, nothing is shrunk and B^T B = A^T A exactly
    rng = np.random.default_rng(21)
    A = rng.standard_normal((7, 30))
    B = O.frequent_directions_stream(A, 10)
    assert np.allclose(B.T @ B, A.T @ A, atol=1e-10)
    # many rows: Prop. 1 and the FD bound for every k < l (Sec. 3.1)
    X = synth.headtail(400, 120, 12, 3)
    A = X.to_scipy()
    for ell in (5, 12):
        B = O.frequent_directions_stream(A, ell)
        lo, hi = metrics.residual_eigs(A, B)
        assert lo > -1e-9 * metrics.fro2(A)
        for k in range(ell):
            assert hi <= metrics.fd_bound(A, ell, k) * (1 + 1e-9)
    # the last shrink of a stream of exactly l rows is DenseShrink([0; A])
    A = rng.standard_normal((10, 40))
    assert np.allclose(O.frequent_directions_stream(A, 10),
                       O.dense_shrink(np.vstack([np.zeros((10, 40)), A]), 10))
