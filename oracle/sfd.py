"""Sparse Frequent Directions, step by step, in float64 on the CPU.

Test infrastructure only (see the package docstring). Each function follows
one algorithm of Ghashami, Liberty, Phillips, "Efficient Frequent Directions
Algorithm for Sparse Matrices", in the paper's order and notation:

  simultaneous_iteration  Alg. 1 (Sec. 3.2)
  sfd_stream / SFDOracle  Alg. 2 (Sec. 4)
  sparse_shrink           Alg. 3
  boosted_sparse_shrink   Alg. 4
  dense_shrink            Alg. 5
  verify_spectral         Alg. 6 (Sec. 4.1, Lemma 4.1)
  frequent_directions     the classical FD of Sec. 3.1 (baseline only)
  frequent_directions_stream
                          classical FD with a buffer of l rows, as the
                          comparison mode of the GPU library runs it (Sec. 5)

Readings of points the paper leaves open (the same on the CUDA side):

R1  Alg. 1 orthonormalises once, at the end. In floating point
    A (A^T A)^q G collapses onto the top direction, so every product is
    orthonormalised; the span after each step is unchanged in exact
    arithmetic. Householder QR, signs fixed so diag(R) >= 0.
R2  q = Theta(log(n/eps)/eps) with eps = 1/4 (Alg. 3 calls SI with 1/4); n is
    the buffer's row count m. q = ceil(c_q * ln(m/eps)/eps), c_q = 1/4 by
    default, i.e. ceil(ln(4m)).
R3  svd(P, l) of the l x d matrix P is complete; lambda_l is its l-th
    singular value and B' = diag(sqrt(max(0, lambda_i^2 - lambda_l^2))) V^T.
    Only B^T B is comparable between implementations (signs of singular
    vectors are arbitrary).
R4  VerifySpectral runs p = ceil(log2(sqrt(2d/pi)/delta_i)) power steps (the
    constant c from Lemma 4.1's proof: Pr[|<v1,x>| <= t] <= t sqrt(2d/pi)),
    with delta_i keyed on (buffer b, attempt r):
    delta_{b,r} = delta * (6/pi^2) / (b+1)^2 / 2^(r+1), whose double sum is
    delta, so the union bound of Sec. 4.1 still holds. ||C^p x|| is a running
    sum of log ||C x_t|| with x_t renormalised. When Delta/2 is at or below
    64 * 2^-24 * ||A'||_F^2 (the residual A'^T A' - B'^T B' is at the
    resolution of the fp32 arithmetic the GPU checks it in), VS accepts.
R5  BSSh retries at most `retry_cap` attempts; after that the last B' is
    used and the buffer is counted as unverified.
R6  End of stream (Alg. 2 drops the last partial buffer): `sketch()` flushes
    a pending buffer A' of m_p rows: BSSh + DSh if m_p >= l, else
    DSh([B; A']) with A' dense. Empty: nothing.
R7  A buffer that triggers with fewer than l rows (possible only through the
    nnz rule with rows holding many entries) takes the same m_p < l branch.
R8  nnz counts the entries the caller supplies for a row (duplicates summed
    in the arithmetic, counted as given).
"""
import math

import numpy as np
import scipy.sparse as sp

from . import philox

ALPHA = 6.0 / 41.0          # alpha of Alg. 4 / Theorem 4.1
EPS_SI = 0.25               # SimultaneousIteration is called with eps = 1/4 (Alg. 3)
VS_RESOLUTION = 64.0 * 2.0 ** -24   # R4: fp32 resolution guard


# ----------------------------------------------------------------------------
# schedules (R2, R4)
# ----------------------------------------------------------------------------
def q_fixed(m, c_q=0.25):
    """Power count of Alg. 1 for a buffer of m rows (R2)."""
    return max(0, int(math.ceil(c_q * math.log(m / EPS_SI) / EPS_SI)))


def delta_br(delta, b, r):
    """Failure budget of the VS call on buffer b, attempt r (R4)."""
    return delta * (6.0 / math.pi ** 2) / float(b + 1) ** 2 / 2.0 ** (r + 1)


def vs_steps(d, delta_i):
    """Power steps c * log(d / delta_i) of Alg. 6 with the constant of R4."""
    return max(1, int(math.ceil(math.log2(math.sqrt(2.0 * d / math.pi) / delta_i))))


# ----------------------------------------------------------------------------
# Alg. 1 SimultaneousIteration
# ----------------------------------------------------------------------------
def orthonormalize(X):
    """Orthonormal basis of the columns of X (Householder QR, diag(R) >= 0)."""
    Q, R = np.linalg.qr(X, mode="reduced")
    s = np.sign(np.diag(R))
    s[s == 0] = 1.0
    return Q * s


def simultaneous_iteration(A, k, q, G):
    """Alg. 1: Z = GramSchmidt(A (A^T A)^q G) with per-product
    orthonormalisation (R1). A is m x d (scipy sparse or dense), G is d x k."""
    Y = orthonormalize(A @ G)
    for _ in range(q):
        W = orthonormalize(A.T @ Y)
        Y = orthonormalize(A @ W)
    return Y


# ----------------------------------------------------------------------------
# Alg. 3 SparseShrink
# ----------------------------------------------------------------------------
def sparse_shrink(A, ell, q, G):
    """Alg. 3. Returns (B', info) with B' of shape l x d."""
    Z = simultaneous_iteration(A, ell, q, G)
    P = np.asarray((A.T @ Z).T)                    # P = Z^T A'  (l x d)
    H, lam, Vt = np.linalg.svd(P, full_matrices=False)
    lam_l = lam[ell - 1]
    lam_tilde = np.sqrt(np.maximum(lam ** 2 - lam_l ** 2, 0.0))
    Bp = lam_tilde[:, None] * Vt                   # B' = Lambda~ V^T
    return Bp, {"Z": Z, "P": P, "lam": lam}


# ----------------------------------------------------------------------------
# Alg. 6 VerifySpectral
# ----------------------------------------------------------------------------
def verify_spectral(apply_C, x0, p):
    """Alg. 6 on the operator apply_C, start vector x0 (unit), p steps.
    Returns (accepted, log ||C^p x0||)."""
    x = np.array(x0, dtype=np.float64)
    logsum = 0.0
    for _ in range(p):
        y = apply_C(x)
        nrm = float(np.linalg.norm(y))
        if nrm == 0.0:
            return True, -math.inf
        logsum += math.log(nrm)
        x = y / nrm
    return logsum <= 0.0, logsum


def residual_operator(A, Bp, Delta):
    """x -> (A'^T A' - B'^T B') x / (Delta / 2), the C of Alg. 4."""
    scale = 2.0 / Delta

    def apply_C(x):
        return (A.T @ (A @ x) - Bp.T @ (Bp @ x)) * scale
    return apply_C


# ----------------------------------------------------------------------------
# Alg. 4 BoostedSparseShrink
# ----------------------------------------------------------------------------
def boosted_sparse_shrink(A, ell, delta, seed, b, q, verify=True, retry_cap=8,
                          inject_fail=0):
    """Alg. 4 with the keyed delta_{b,r} of R4 and the retry cap of R5.

    inject_fail: this many VS verdicts, counted from this call on, are forced
    to False (host-side fault injection for the retry path).
    Returns (B', info); info["injected"] is how many were consumed."""
    m, d = A.shape
    fro2 = float(A.multiply(A).sum()) if sp.issparse(A) else float((A * A).sum())
    attempts = []
    Bp = None
    inject0 = inject_fail
    for r in range(retry_cap):
        G = philox.gaussian_G(seed, b, r, d, ell)
        Bp, inf = sparse_shrink(A, ell, q, G)
        fro2_b = float((Bp * Bp).sum())
        Delta = (fro2 - fro2_b) / (ALPHA * ell)
        if not verify:
            return Bp, {"attempts": 1, "Delta": Delta, "verified": True, "lam": inf["lam"],
                        "logsum": None, "p": 0}
        di = delta_br(delta, b, r)
        p = vs_steps(d, di)
        if Delta / 2.0 <= VS_RESOLUTION * fro2:
            ok, logsum = True, -math.inf
        else:
            x0 = philox.sphere_x(seed, b, r, d)
            ok, logsum = verify_spectral(residual_operator(A, Bp, Delta), x0, p)
        if inject_fail > 0:
            ok = False
            inject_fail -= 1
        attempts.append({"r": r, "Delta": Delta, "logsum": logsum, "ok": ok, "p": p})
        if ok:
            return Bp, {"attempts": r + 1, "Delta": Delta, "verified": True, "lam": inf["lam"],
                        "logsum": logsum, "p": p, "history": attempts,
                        "injected": inject0 - inject_fail}
    return Bp, {"attempts": retry_cap, "Delta": attempts[-1]["Delta"], "verified": False,
                "lam": None, "logsum": attempts[-1]["logsum"], "p": attempts[-1]["p"],
                "history": attempts, "injected": inject0 - inject_fail}


# ----------------------------------------------------------------------------
# Alg. 5 DenseShrink
# ----------------------------------------------------------------------------
def dense_shrink(M, ell):
    """Alg. 5: svd(M, l), shrink by lambda_l^2, return the l x d sketch."""
    M = np.asarray(M, dtype=np.float64)
    rows, d = M.shape
    _, lam, Vt = np.linalg.svd(M, full_matrices=False)
    lam_full = np.zeros(ell)
    k = min(ell, lam.size)
    lam_full[:k] = lam[:k]
    lam_l = lam_full[ell - 1]
    lam_tilde = np.sqrt(np.maximum(lam_full ** 2 - lam_l ** 2, 0.0))
    B = np.zeros((ell, d))
    B[:k] = lam_tilde[:k, None] * Vt[:k]
    return B


# ----------------------------------------------------------------------------
# Alg. 2 SparseFrequentDirections
# ----------------------------------------------------------------------------
def csr_from_arrays(indptr, indices, values, d):
    """scipy CSR (float64) of rows given as indptr / indices / values."""
    indptr = np.asarray(indptr, dtype=np.int64)
    base = indptr[0]
    ip = indptr - base
    nnz = int(ip[-1])
    idx = np.asarray(indices[base:base + nnz], dtype=np.int64)
    val = np.asarray(values[base:base + nnz], dtype=np.float64)
    return sp.csr_matrix((val, idx, ip), shape=(len(ip) - 1, d))


def buffer_boundaries(row_nnz, d, ell, start_rows=0, start_nnz=0):
    """Row positions after which Alg. 2's test nnz(A') >= l d or rows(A') = d
    fires, scanning one row at a time. start_rows / start_nnz describe a buffer
    already pending when the scan starts. Returns (ends, pending_rows,
    pending_nnz), ends being exclusive row indices into row_nnz."""
    ends = []
    rows, nnz = start_rows, start_nnz
    for i, c in enumerate(row_nnz):
        rows += 1
        nnz += int(c)
        if nnz >= ell * d or rows == d:
            ends.append(i + 1)
            rows, nnz = 0, 0
    return ends, rows, nnz


class SFDOracle:
    """Alg. 2 as a stream object: append rows, then read the sketch.

    State: B (l x d, float64), the pending buffer A' (rows kept as CSR
    pieces), the buffer counter b that keys the randomness."""

    def __init__(self, d, ell, seed, delta=0.01, verify=True, c_q=0.25, q_override=None,
                 retry_cap=8, inject_fail=0):
        if not (1 <= ell <= d):
            raise ValueError("need 1 <= l <= d")
        self.d, self.ell, self.seed = int(d), int(ell), int(seed)
        self.delta, self.verify, self.c_q = delta, verify, c_q
        self.q_override, self.retry_cap, self.inject_fail = q_override, retry_cap, inject_fail
        self.B = np.zeros((self.ell, self.d))
        self.b = 0
        self._pend = []          # list of CSR pieces of A'
        self._pend_rows = 0
        self._pend_nnz = 0
        self.log = []

    # -- Alg. 2 body ---------------------------------------------------------
    def append_rows(self, indptr, indices, values):
        indptr = np.asarray(indptr, dtype=np.int64)
        row_nnz = np.diff(indptr)
        ends, _, _ = buffer_boundaries(row_nnz, self.d, self.ell,
                                       self._pend_rows, self._pend_nnz)
        start = 0
        for e in ends:
            self._push(indptr[start:e + 1], indices, values)
            self._close_buffer()
            start = e
        if start < len(row_nnz):
            self._push(indptr[start:], indices, values)

    def _push(self, ip, indices, values):
        piece = csr_from_arrays(ip, indices, values, self.d)
        self._pend.append(piece)
        self._pend_rows += piece.shape[0]
        self._pend_nnz += int(ip[-1] - ip[0])

    def _take_buffer(self):
        A = sp.vstack(self._pend, format="csr") if self._pend else None
        self._pend, self._pend_rows, self._pend_nnz = [], 0, 0
        return A

    def _close_buffer(self):
        A = self._take_buffer()
        m = A.shape[0]
        if m >= self.ell:
            q = self.q_override if self.q_override is not None else q_fixed(m, self.c_q)
            Bp, info = boosted_sparse_shrink(A, self.ell, self.delta, self.seed, self.b, q,
                                             self.verify, self.retry_cap, self.inject_fail)
            self.inject_fail -= info.get("injected", 0)
            self.B = dense_shrink(np.vstack([self.B, Bp]), self.ell)
            self.log.append({"b": self.b, "m": m, "nnz": A.nnz, "q": q, **{
                k: v for k, v in info.items() if k in ("attempts", "Delta", "verified", "p", "lam")}})
        else:
            # R6 / R7: too few rows for SparseShrink; DenseShrink of [B; A']
            self.B = dense_shrink(np.vstack([self.B, A.toarray()]), self.ell)
            self.log.append({"b": self.b, "m": m, "nnz": A.nnz, "q": None, "attempts": 0})
        self.b += 1

    # -- R6 -------------------------------------------------------------------
    def flush(self):
        if self._pend_rows > 0:
            self._close_buffer()

    def sketch(self):
        self.flush()
        return self.B.copy()

    def merge(self, other):
        """Mergeability (Sec. 3.1): B <- DenseShrink([B; B_other])."""
        self.flush()
        other.flush()
        self.B = dense_shrink(np.vstack([self.B, other.B]), self.ell)


def sfd_stream(indptr, indices, values, d, ell, seed, **kw):
    """One-shot Alg. 2 over a whole CSR matrix, with the final flush (R6)."""
    o = SFDOracle(d, ell, seed, **kw)
    o.append_rows(indptr, indices, values)
    return o.sketch(), o


# ----------------------------------------------------------------------------
# Sec. 3.1 FrequentDirections (baseline for comparisons only)
# ----------------------------------------------------------------------------
def frequent_directions(A, ell):
    """Classical FD: grow the sketch to 2l rows, DenseShrink back to l."""
    A = A.toarray() if sp.issparse(A) else np.asarray(A, dtype=np.float64)
    n, d = A.shape
    B = np.zeros((0, d))
    for i in range(0, n, ell):
        B = np.vstack([B, A[i:i + ell]])
        if B.shape[0] >= 2 * ell:
            B = dense_shrink(B, ell)
    if B.shape[0] > ell:
        B = dense_shrink(B, ell)
    out = np.zeros((ell, d))
    out[:B.shape[0]] = B
    return out


def frequent_directions_stream(A, ell):
    """Classical FD (Sec. 3.1) driven like Alg. 2 with a buffer of l rows:
    B = 0 (l x d); after every l rows, and for the rows left at the end,
    B = DenseShrink([B; rows], l) (Alg. 5). Every shrink subtracts the l-th
    squared singular value of the stack in each kept direction, which is the
    FD step, so the FD guarantee of Sec. 3.1 holds for the result."""
    A = A.toarray() if sp.issparse(A) else np.asarray(A, dtype=np.float64)
    n, d = A.shape
    B = np.zeros((ell, d))
    for i in range(0, n, ell):
        B = dense_shrink(np.vstack([B, A[i:i + ell]]), ell)
    return B
