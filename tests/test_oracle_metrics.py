"""Pins of the oracle's error measures and bounds (Sec. 5 measurements,
the FD bound of Sec. 2 and the bound of Theorem 4.1) against closed forms.

Every test matrix here has singular values set by hand: A = H1 D H2 with D a
weighted permutation (one entry per row and column, so its singular values
are the absolute weights) and H1, H2 Householder reflections I - 2 v v^T /
v^T v (orthogonal), or D alone. So sigma_i, the right singular vectors and
every quantity below are known without calling an SVD routine, and a slip in
the oracle (sigma_i in place of sigma_i^2, k in place of k + 1, a wrong
denominator, a transposed operand) fails one of these checks.
"""
import math

import numpy as np
import pytest
import scipy.sparse as sp

from oracle import metrics
from oracle import sfd as O


def _householder(n, seed):
    v = np.random.default_rng(seed).standard_normal(n)
    return np.eye(n) - 2.0 * np.outer(v, v) / (v @ v)


def _known(m, d, sigma, seed, rotate=True):
    """(A, sigma sorted descending, V) with A = H1 D H2, D[p_i, c_i] = +-sigma_i,
    V[:, i] the right singular vector of sigma_i (sorted order)."""
    rng = np.random.default_rng(seed)
    r = len(sigma)
    rows = rng.permutation(m)[:r]
    cols = rng.permutation(d)[:r]
    signs = rng.choice([-1.0, 1.0], r)
    D = np.zeros((m, d))
    D[rows, cols] = signs * sigma
    E = np.zeros((d, r))                      # right singular vectors of D
    E[cols, np.arange(r)] = 1.0
    if rotate:
        H1, H2 = _householder(m, seed + 1), _householder(d, seed + 2)
        A = H1 @ D @ H2
        V = H2.T @ E                          # A^T A = H2^T D^T D H2
    else:
        A, V = D, E
    order = np.argsort(-np.asarray(sigma), kind="stable")
    return A, np.asarray(sigma, dtype=np.float64)[order], V[:, order]


SIGMA = [3.0, 7.0, 0.5, 5.0, 2.0, 1.0, 4.0, 0.25, 6.0, 1.5]   # unsorted on purpose


@pytest.mark.parametrize("rotate", [False, True])
def test_tail_mass_and_top_singular_values_closed_form(rotate):
    A, s, _ = _known(40, 60, SIGMA, 1, rotate)
    assert np.allclose(metrics.top_singular_values(A, 4), s[:4], rtol=1e-12, atol=1e-12)
    for k in range(len(s) + 1):
        want = float(np.sum(s[k:] ** 2))     # sum_{i > k} sigma_i^2
        assert math.isclose(metrics.tail_mass(A, k), want, rel_tol=1e-10, abs_tol=1e-10), k
    assert metrics.tail_mass(A, 0) == pytest.approx(metrics.fro2(A), rel=1e-12)


def test_tail_mass_sparse_iterative_path():
    # min(m, d) > 3000 takes the sparse partial SVD: D alone, kept sparse
    m, d = 3200, 3300
    rng = np.random.default_rng(5)
    sigma = np.concatenate([[9.0, 8.0, 6.5, 5.0, 4.0], rng.uniform(0.1, 1.0, 400)])
    rows, cols = rng.permutation(m)[:sigma.size], rng.permutation(d)[:sigma.size]
    A = sp.csr_matrix((sigma * rng.choice([-1.0, 1.0], sigma.size), (rows, cols)), shape=(m, d))
    top = metrics.top_singular_values(A, 5)
    assert np.allclose(top, [9.0, 8.0, 6.5, 5.0, 4.0], rtol=1e-8)
    assert metrics.tail_mass(A, 5) == pytest.approx(float(np.sum(sigma[5:] ** 2)), rel=1e-8)


@pytest.mark.parametrize("ell,k", [(8, 0), (8, 3), (12, 7), (41, 5)])
def test_fd_bound_closed_form(ell, k):
    A, s, _ = _known(30, 50, SIGMA, 2)
    tail = float(np.sum(s[k:] ** 2))
    assert metrics.fd_bound(A, ell, k) == pytest.approx(tail / (ell - k), rel=1e-10)


def test_sfd_bound_closed_form_and_domain():
    A, s, _ = _known(30, 50, SIGMA, 3)
    # Theorem 4.1: ||A - A_k||_F^2 / (alpha l - k), alpha = 6/41, needs k < alpha l
    for ell, k in [(41, 0), (41, 5), (100, 14), (7, 0)]:
        want = float(np.sum(s[k:] ** 2)) / (6.0 / 41.0 * ell - k)
        assert metrics.sfd_bound(A, ell, k) == pytest.approx(want, rel=1e-10)
    for ell, k in [(41, 6), (100, 15), (6, 1)]:
        with pytest.raises(ValueError):
            metrics.sfd_bound(A, ell, k)
    assert O.ALPHA == 6.0 / 41.0


@pytest.mark.parametrize("rotate", [False, True])
@pytest.mark.parametrize("k", [1, 3, 5])
def test_proj_err_closed_form(rotate, k):
    A, s, V = _known(40, 60, SIGMA, 4, rotate)
    tail = float(np.sum(s[k:] ** 2))
    # B = the top-k rows of A's SVD: the projection keeps sigma_1..sigma_k, ratio 1
    B = s[:k, None] * V[:, :k].T
    assert metrics.proj_err(A, B, k) == pytest.approx(1.0, rel=1e-10)
    # rows rescaled and in another order: B's top-k right subspace is still V_k
    B2 = np.arange(k, 0, -1.0)[:, None] * 0.3 * V[:, :k][:, ::-1].T
    B2 = np.vstack([B2, np.zeros((2, A.shape[1]))])
    assert metrics.proj_err(A, B2, k) == pytest.approx(1.0, rel=1e-10)
    # B spanning the next k directions keeps sigma_{k+1}..sigma_{2k} instead
    Bn = s[k:2 * k, None] * V[:, k:2 * k].T
    want = (float(np.sum(s ** 2)) - float(np.sum(s[k:2 * k] ** 2))) / tail
    assert metrics.proj_err(A, Bn, k) == pytest.approx(want, rel=1e-10)
    assert want > 1.0


@pytest.mark.parametrize("dense_limit", [4000, 10])
def test_cov_err_closed_form(dense_limit):
    A, s, V = _known(40, 60, SIGMA, 6)
    f = float(np.sum(s ** 2))
    assert metrics.fro2(A) == pytest.approx(f, rel=1e-12)
    # B = 0: ||A^T A||_2 = sigma_1^2
    assert metrics.cov_err(A, np.zeros((3, 60)), dense_limit) == pytest.approx(s[0] ** 2 / f, rel=1e-8)
    # B = A_k: the residual's top eigenvalue is sigma_{k+1}^2
    for k in (1, 4):
        B = s[:k, None] * V[:, :k].T
        assert metrics.cov_err(A, B, dense_limit) == pytest.approx(s[k] ** 2 / f, rel=1e-8)
    # the FD-style shrink of the exact SVD by sigma_l^2 leaves sigma_l^2 in every
    # kept direction and sigma_i^2 <= sigma_l^2 in the rest
    ell = 5
    B = np.sqrt(s[:ell] ** 2 - s[ell - 1] ** 2)[:, None] * V[:, :ell].T
    assert metrics.cov_norm(A, B, dense_limit) == pytest.approx(s[ell - 1] ** 2, rel=1e-8)


def test_residual_eigs_sign_and_extremes():
    A, s, V = _known(30, 45, SIGMA, 7, rotate=False)
    # B overshoots the top direction: A^T A - B^T B has eigenvalue s1^2 - 4 s1^2 there
    B = (2.0 * s[0]) * V[:, :1].T
    lo, hi = metrics.residual_eigs(A, B)
    assert lo == pytest.approx(-3.0 * s[0] ** 2, rel=1e-10)
    assert hi == pytest.approx(s[1] ** 2, rel=1e-10)
    assert metrics.cov_norm(A, B) == pytest.approx(3.0 * s[0] ** 2, rel=1e-10)


def test_cov_norm_psd_closed_form():
    A, s, V = _known(50, 3500, SIGMA, 8)
    As = sp.csr_matrix(A)
    for k in (0, 2, 6):
        B = s[:k, None] * V[:, :k].T if k else np.zeros((1, 3500))
        assert metrics.cov_norm_psd(As, B) == pytest.approx(s[k] ** 2, rel=1e-8)
    ell = 4
    B = np.sqrt(s[:ell] ** 2 - s[ell - 1] ** 2)[:, None] * V[:, :ell].T
    assert metrics.cov_norm_psd(As, B) == pytest.approx(s[ell - 1] ** 2, rel=1e-8)
