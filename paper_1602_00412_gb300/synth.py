"""Seeded synthetic sparse streams (CSR) for tests and the benchmark.

This module only makes input data: it holds none of the sketching method's
arithmetic, and both the CUDA path and the FP64 oracle consume the exact CSR
bytes it returns (indptr int64, indices int32, values float32).

Workloads (sizes from the method's evaluation and its scaled-up variants):

* ``planted``   nnz/row ~ Poisson(mu); columns Zipf(s) over d without repeats
  within a row (rank r -> column r-1, so hot columns come first, like the
  "head" of the paper's synthetic data in Sec. 5); value at (i, j) =
  x_i^T y_j + noise*N(0,1) with x_it = sigma_t g, sigma_t = scale*decay^t,
  y_jt ~ N(0,1).
* ``gapped``    rows are scaled copies of K = l + extra sparse prototypes
  (Zipf supports, unit-norm values): a_i = g_i c_{t_i} v_{t_i} + noise on the
  same support, with c_t = 10*0.95^t for t < l and 10x smaller for t >= l, so
  every buffer's spectrum has a planted gap at l.
* ``bow``       bag-of-words: nnz/row ~ round(LogNormal(mu, sigma)) capped,
  Zipf columns, value log(1+c) with c ~ zero-truncated Poisson(lam), rows
  L2-normalised.
* ``headtail``  the paper's own synthetic data (Sec. 5, Datasets): exactly z
  non-zeros of value +-1 per row; a non-zero lands in the first 1.5z columns
  ("head") w.p. 0.9, else in the tail, uniformly within each, no repeats.
"""
import numpy as np


class CSR:
    """A stream of sparse rows: indptr (n+1, int64), indices (int32), values (float32)."""

    __slots__ = ("indptr", "indices", "values", "n", "d", "name")

    def __init__(self, indptr, indices, values, d, name=""):
        self.indptr = np.ascontiguousarray(indptr, dtype=np.int64)
        self.indices = np.ascontiguousarray(indices, dtype=np.int32)
        self.values = np.ascontiguousarray(values, dtype=np.float32)
        self.n = len(self.indptr) - 1
        self.d = int(d)
        self.name = name

    @property
    def nnz(self):
        return int(self.indptr[-1])

    def rows(self, r0, r1):
        """Rows [r0, r1) as a new CSR with indptr starting at 0."""
        a, b = int(self.indptr[r0]), int(self.indptr[r1])
        return CSR(self.indptr[r0:r1 + 1] - a, self.indices[a:b], self.values[a:b], self.d,
                   self.name)

    def to_scipy(self):
        import scipy.sparse as sp
        return sp.csr_matrix((self.values.astype(np.float64), self.indices, self.indptr),
                             shape=(self.n, self.d))


def _zipf_cdf(d, s):
    w = np.arange(1, d + 1, dtype=np.float64) ** (-float(s))
    c = np.cumsum(w)
    return c / c[-1]


def _draw_cols(rng, cdf, k):
    u = rng.random(k)
    return np.minimum(np.searchsorted(cdf, u, side="right"), len(cdf) - 1)


def _unique_cols(rng, counts, cdf):
    """Column lists without repeats: slot j of row i drawn from cdf, repeats
    redrawn until none is left. Returns (indptr, cols) with sorted rows."""
    counts = np.asarray(counts, dtype=np.int64)
    n = len(counts)
    d = len(cdf)
    counts = np.minimum(counts, d)
    kmax = int(counts.max()) if n else 0
    indptr = np.zeros(n + 1, dtype=np.int64)
    np.cumsum(counts, out=indptr[1:])
    if kmax == 0:
        return indptr, np.zeros(0, dtype=np.int32)
    # padded [n, kmax] array; pad slots hold distinct values >= d
    pad = d + np.arange(kmax, dtype=np.int64)[None, :]
    valid = np.arange(kmax)[None, :] < counts[:, None]
    grid = np.where(valid, 0, pad)
    nv = int(valid.sum())
    grid[valid] = _draw_cols(rng, cdf, nv)
    active = np.arange(n)
    while active.size:
        sub = np.sort(grid[active], axis=1)
        dup = np.zeros_like(sub, dtype=bool)
        dup[:, 1:] = sub[:, 1:] == sub[:, :-1]
        has = dup.any(axis=1)
        sub_rows = active[has]
        sub = sub[has]
        dup = dup[has]
        if sub_rows.size == 0:
            grid[active] = np.sort(grid[active], axis=1)
            break
        nd = int(dup.sum())
        sub[dup] = _draw_cols(rng, cdf, nd)
        grid[sub_rows] = sub
        done = active[~has]
        grid[done] = np.sort(grid[done], axis=1)
        active = sub_rows
    cols = grid[np.arange(kmax)[None, :] < counts[:, None]]
    return indptr, cols.astype(np.int32)


def _chunks(n, size):
    for a in range(0, n, size):
        yield a, min(n, a + size)


def planted(n, d, mu, s, rank, scale, decay, noise, seed, cap=None, chunk=20000, name="planted",
            row_seed=None):
    """Poisson(mu) Zipf(s) rows with a planted rank-`rank` signal (see module doc).
    row_seed (optional): the column factors y_j come from `seed` and the rows
    from `row_seed`, so row blocks of one stream can be drawn independently."""
    rng = np.random.default_rng(seed)
    cdf = _zipf_cdf(d, s)
    sig = scale * decay ** np.arange(rank, dtype=np.float64)
    Y = rng.standard_normal((d, rank))
    if row_seed is not None:
        rng = np.random.default_rng(row_seed)
    counts = rng.poisson(mu, size=n)
    if cap is not None:
        counts = np.minimum(counts, cap)
    ip_all = np.zeros(n + 1, dtype=np.int64)
    idx_parts, val_parts = [], []
    for a, b in _chunks(n, chunk):
        ip, cols = _unique_cols(rng, counts[a:b], cdf)
        X = rng.standard_normal((b - a, rank)) * sig[None, :]
        rows = np.repeat(np.arange(b - a), np.diff(ip))
        vals = np.einsum("ij,ij->i", X[rows], Y[cols]) + noise * rng.standard_normal(len(cols))
        ip_all[a + 1:b + 1] = ip[1:] + ip_all[a]
        idx_parts.append(cols)
        val_parts.append(vals.astype(np.float32))
    return CSR(ip_all, np.concatenate(idx_parts), np.concatenate(val_parts), d, name)


def gapped(n, d, ell, mu, s, seed, extra=10, gap=0.1, noise=1e-3, name="gapped"):
    """Prototype rows with a planted spectral gap at l (see module doc)."""
    rng = np.random.default_rng(seed)
    cdf = _zipf_cdf(d, s)
    K = ell + extra
    pcounts = np.maximum(rng.poisson(mu, size=K), 1)
    pip, pcols = _unique_cols(rng, pcounts, cdf)
    pvals = rng.standard_normal(len(pcols))
    for t in range(K):
        seg = slice(pip[t], pip[t + 1])
        pvals[seg] /= np.linalg.norm(pvals[seg])
    c = 10.0 * 0.95 ** np.arange(K, dtype=np.float64)
    c[ell:] *= gap
    t_i = rng.integers(0, K, size=n)
    g_i = rng.standard_normal(n)
    counts = pcounts[t_i]
    indptr = np.zeros(n + 1, dtype=np.int64)
    np.cumsum(counts, out=indptr[1:])
    starts = pip[t_i]
    offs = np.arange(indptr[-1]) - np.repeat(indptr[:-1], counts)
    src = np.repeat(starts, counts) + offs
    cols = pcols[src]
    vals = np.repeat(g_i * c[t_i], counts) * pvals[src] + noise * rng.standard_normal(len(src))
    return CSR(indptr, cols, vals.astype(np.float32), d, name)


def bow(n, d, mu, sigma, s, lam, seed, cap=2000, chunk=20000, name="bow"):
    """Bag-of-words counts with row L2 normalisation (see module doc)."""
    rng = np.random.default_rng(seed)
    cdf = _zipf_cdf(d, s)
    counts = np.minimum(np.rint(rng.lognormal(mu, sigma, size=n)).astype(np.int64), cap)
    ip_all = np.zeros(n + 1, dtype=np.int64)
    idx_parts, val_parts = [], []
    for a, b in _chunks(n, chunk):
        ip, cols = _unique_cols(rng, counts[a:b], cdf)
        k = len(cols)
        c = rng.poisson(lam, size=k)
        while (c == 0).any():
            z = c == 0
            c[z] = rng.poisson(lam, size=int(z.sum()))
        v = np.log1p(c.astype(np.float64))
        rows = np.repeat(np.arange(b - a), np.diff(ip))
        nrm = np.sqrt(np.bincount(rows, weights=v * v, minlength=b - a))
        nrm[nrm == 0] = 1.0
        v = v / nrm[rows]
        ip_all[a + 1:b + 1] = ip[1:] + ip_all[a]
        idx_parts.append(cols)
        val_parts.append(v.astype(np.float32))
    return CSR(ip_all, np.concatenate(idx_parts), np.concatenate(val_parts), d, name)


def headtail(n, d, z, seed, name="headtail"):
    """The paper's synthetic data (Sec. 5): z non-zeros of +-1 per row."""
    rng = np.random.default_rng(seed)
    head = int(1.5 * z)
    cols = np.empty((n, z), dtype=np.int64)
    for i in range(n):
        chosen = set()
        row = []
        while len(row) < z:
            if rng.random() < 0.9:
                c = int(rng.integers(0, head))
            else:
                c = int(rng.integers(head, d))
            if c not in chosen:
                chosen.add(c)
                row.append(c)
        cols[i] = np.sort(row)
    vals = rng.choice(np.array([-1.0, 1.0]), size=(n, z))
    indptr = np.arange(0, n * z + 1, z, dtype=np.int64)
    return CSR(indptr, cols.reshape(-1), vals.reshape(-1), d, name)


# ----------------------------------------------------------------------------
# named workloads
# ----------------------------------------------------------------------------
def c1(seed=0, n=10000):
    """n=10,000, d=2,000, l=50: Poisson(20), Zipf(1.1), rank-10 planted 10*0.7^t, noise 0.1."""
    return planted(n, 2000, 20, 1.1, 10, 10.0, 0.7, 0.1, seed, name="c1")


def c1_gapped(seed=0, n=10000):
    """d=2,000 rows of the c1 shape with a planted gap at l=50 (prototype rows)."""
    return gapped(n, 2000, 50, 20, 1.1, seed, name="c1_gapped")


def c2(seed=0, n=1_000_000):
    """n=1,000,000, d=50,000, l=100: Poisson(50), Zipf(1.1), rank-20 planted 10*0.8^t, noise 0.1."""
    return planted(n, 50000, 50, 1.1, 20, 10.0, 0.8, 0.1, seed, name="c2")


def c3(seed=0, n=5_000_000):
    """n=5,000,000, d=200,000, l=200: round(LogNormal(4.2,0.8)) capped at 2000, Zipf(1.05), log(1+Poisson(2))."""
    return bow(n, 200000, 4.2, 0.8, 1.05, 2.0, seed, name="c3")


def c5(seed=0, n=2_000_000):
    """n=2,000,000, d=1,000,000, l=256: Poisson(80), Zipf(1.1), rank-64 planted 10*0.9^t, noise 0.05."""
    return planted(n, 1000000, 80, 1.1, 64, 10.0, 0.9, 0.05, seed, name="c5")


def c3_chunk(seed, i, n=625_000):
    """Chunk i of the chunk-parallel bag-of-words stream of c3 (d=200,000; 8
    chunks of 625,000 rows make its 5,000,000 rows): c3's row distribution
    drawn from seed (seed, 3, i)."""
    return bow(n, 200000, 4.2, 0.8, 1.05, 2.0, [seed, 3, i], name="c3")


def c5_chunk(seed, i, n=500_000):
    """Chunk i of the c5 stream (d=1,000,000; 4 chunks of 500,000 rows make its
    2,000,000 rows): planted column factors from `seed`, rows from (seed, 5, i)."""
    return planted(n, 1000000, 80, 1.1, 64, 10.0, 0.9, 0.05, seed, name="c5",
                   row_seed=[seed, 5, i])


def _call(args):
    fn, a = args
    return fn(*a)


def parallel(fn, arg_list, processes=None):
    """[fn(*a) for a in arg_list] in spawned worker processes (generation only)."""
    import multiprocessing as mp
    import os
    procs = processes or min(len(arg_list), os.cpu_count() or 1)
    if procs <= 1:
        return [fn(*a) for a in arg_list]
    with mp.get_context("spawn").Pool(procs) as pool:
        return pool.map(_call, [(fn, a) for a in arg_list])


def concat(parts, name=None):
    """Rows of several CSR blocks (same d) one after another."""
    ip = [np.asarray(parts[0].indptr, dtype=np.int64)]
    off = ip[0][-1]
    for p in parts[1:]:
        q = np.asarray(p.indptr, dtype=np.int64)
        ip.append(q[1:] - q[0] + off)
        off = ip[-1][-1]
    return CSR(np.concatenate(ip), np.concatenate([p.indices for p in parts]),
               np.concatenate([p.values for p in parts]), parts[0].d, name or parts[0].name)


WORKLOADS = {
    "c1": (c1, 2000, 50, 10),
    "c1_gapped": (c1_gapped, 2000, 50, 10),
    "c2": (c2, 50000, 100, 20),
    "c3": (c3, 200000, 200, 20),
    "c5": (c5, 1000000, 256, 64),
}
