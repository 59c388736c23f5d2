"""Error measures and bounds used to assess sketches (oracle side).

Test infrastructure only (see the package docstring).

cov_err       ||A^T A - B^T B||_2 / ||A||_F^2            (Sec. 5, Measurements)
cov_norm_psd  ||A^T A - B^T B||_2 when that matrix is PSD (Prop. 1: every FD /
              SFD sketch), from its largest eigenvalue alone (large d)
proj_err      ||A - pi_{B_k}(A)||_F^2 / ||A - A_k||_F^2  (Sec. 5, Measurements)
tail_mass     ||A - A_k||_F^2                            (Sec. 1.1 notation)
fd_bound      ||A - A_k||_F^2 / (l - k)                  (FD bound, Sec. 2)
sfd_bound     ||A - A_k||_F^2 / (alpha l - k)            (Theorem 4.1)
bbt_rel_diff  ||B1^T B1 - B2^T B2||_F / ||B2^T B2||_F without forming d x d
"""
import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla

from .sfd import ALPHA


def _gram_apply(A, B):
    def mv(x):
        x = np.asarray(x).reshape(-1)
        return A.T @ (A @ x) - B.T @ (B @ x)
    return mv


def residual_eigs(A, B, dense_limit=3000):
    """(min, max) eigenvalue of A^T A - B^T B."""
    d = A.shape[1]
    if d <= dense_limit:
        Ad = A.toarray() if sp.issparse(A) else np.asarray(A)
        R = Ad.T @ Ad - B.T @ B
        w = np.linalg.eigvalsh(R)
        return float(w[0]), float(w[-1])
    op = spla.LinearOperator((d, d), matvec=_gram_apply(A, B), dtype=np.float64)
    hi = spla.eigsh(op, k=1, which="LA", tol=1e-10, maxiter=5000, return_eigenvectors=False)[0]
    lo = spla.eigsh(op, k=1, which="SA", tol=1e-10, maxiter=5000, return_eigenvectors=False)[0]
    return float(lo), float(hi)


def cov_norm(A, B, dense_limit=3000):
    """||A^T A - B^T B||_2."""
    lo, hi = residual_eigs(A, B, dense_limit)
    return max(abs(lo), abs(hi))


def cov_norm_psd(A, B, tol=1e-6, seed=0):
    """||A^T A - B^T B||_2 for a sketch B of A, whose residual A^T A - B^T B
    is positive semi-definite (Prop. 1), so its 2-norm is its largest
    eigenvalue: Lanczos on the operator from a seeded start vector."""
    d = A.shape[1]
    Bd = np.asarray(B, dtype=np.float64)
    op = spla.LinearOperator((d, d), matvec=_gram_apply(A, Bd), dtype=np.float64)
    v0 = np.random.default_rng(seed).standard_normal(d)
    return float(spla.eigsh(op, k=1, which="LA", tol=tol, ncv=40, v0=v0, maxiter=20000,
                            return_eigenvectors=False)[0])


def fro2(A):
    return float(A.multiply(A).sum()) if sp.issparse(A) else float((np.asarray(A) ** 2).sum())


def cov_err(A, B, dense_limit=3000):
    return cov_norm(A, B, dense_limit) / fro2(A)


def top_singular_values(A, k):
    if k <= 0:
        return np.zeros(0)
    m, d = A.shape
    if min(m, d) <= 3000 or k >= min(m, d) - 1:
        Ad = A.toarray() if sp.issparse(A) else np.asarray(A)
        return np.linalg.svd(Ad, compute_uv=False)[:k]
    s = spla.svds(A.astype(np.float64), k=k, return_singular_vectors=False, tol=1e-10)
    return np.sort(s)[::-1]


def tail_mass(A, k):
    """||A - A_k||_F^2 = ||A||_F^2 - sum_{i<=k} sigma_i^2."""
    s = top_singular_values(A, k)
    return fro2(A) - float((s ** 2).sum())


def fd_bound(A, ell, k):
    return tail_mass(A, k) / (ell - k)


def sfd_bound(A, ell, k):
    if not k < ALPHA * ell:
        raise ValueError("Theorem 4.1 needs k < alpha l")
    return tail_mass(A, k) / (ALPHA * ell - k)


def proj_err(A, B, k):
    """||A - A V_k V_k^T||_F^2 / ||A - A_k||_F^2 with V_k the top-k right
    singular vectors of B."""
    _, _, Vt = np.linalg.svd(B, full_matrices=False)
    Vk = Vt[:k].T
    AV = A @ Vk
    num = fro2(A) - float((np.asarray(AV) ** 2).sum())
    return num / tail_mass(A, k)


def bbt_rel_diff(B1, B2):
    """||B1^T B1 - B2^T B2||_F / ||B2^T B2||_F using l x l products only."""
    B1 = np.asarray(B1, dtype=np.float64)
    B2 = np.asarray(B2, dtype=np.float64)
    g11 = B1 @ B1.T
    g22 = B2 @ B2.T
    g12 = B1 @ B2.T
    num2 = (g11 ** 2).sum() + (g22 ** 2).sum() - 2.0 * (g12 ** 2).sum()
    return float(np.sqrt(max(num2, 0.0)) / np.sqrt((g22 ** 2).sum()))
