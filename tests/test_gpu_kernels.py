"""GPU parity of the individual stages through the C ABI: the sparse products
of Alg. 1, CholeskyQR orthonormalisation, the symmetric eigensolver behind
svd(P, l) / svd([B; B'], l), and DenseShrink (Alg. 5) against the FP64 oracle
or float64 library routines on the same inputs."""
import numpy as np
import pytest
import scipy.sparse as sp

from oracle import sfd as O
from paper_1602_00412_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__ as g
    g.build()
    from paper_1602_00412_gb300 import sfd
    return sfd


def dev(a, dtype=None):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda() if dtype is None else \
        torch.from_numpy(np.ascontiguousarray(a, dtype=dtype)).cuda()


def csr_case(kind, seed=0):
    rng = np.random.default_rng(seed)
    if kind == "zipf":
        X = synth.planted(3000, 700, 20, 1.1, 5, 10.0, 0.7, 0.1, seed)
        return X.to_scipy().astype(np.float32), 700
    if kind == "edges":
        # empty rows, one dense column longer than the 2048-entry split, a full row
        m, d = 5000, 300
        A = sp.random(m, d, density=0.01, random_state=rng, format="lil", dtype=np.float32)
        A[::3, :] = 0
        A[:, 7] = rng.standard_normal((m, 1)).astype(np.float32)
        A[11, :] = 1.5
        return sp.csr_matrix(A), d
    if kind == "tiny":
        A = sp.csr_matrix(np.array([[0, 2, 0], [0, 0, 0], [1, 0, -3]], dtype=np.float32))
        return A, 3
    raise KeyError(kind)


@pytest.mark.parametrize("kind", ["zipf", "edges", "tiny"])
@pytest.mark.parametrize("k", [1, 4, 20, 50, 104, 200, 256])
@pytest.mark.parametrize("transpose", [0, 1])
def test_spmm_matches_fp64(lib, kind, k, transpose):
    A, d = csr_case(kind)
    m = A.shape[0]
    rng = np.random.default_rng(k)
    ld = (k + 7) // 8 * 8
    rows_in = m if transpose else d
    Xh = np.zeros((rows_in, ld), np.float32)
    Xh[:, :k] = rng.standard_normal((rows_in, k))
    want = (A.T if transpose else A).astype(np.float64) @ Xh[:, :k].astype(np.float64)
    Y = torch.full((want.shape[0], ld), 7.0, device="cuda")
    lib.sfd_csr_spmm(m, d, dev(A.indptr, np.int32), dev(A.indices, np.int32),
                     dev(A.data, np.float32), k, dev(Xh), ld, Y, ld, transpose)
    got = Y.cpu().numpy()[:, :k].astype(np.float64)
    # fp32 accumulation: error <= ~n u sum |a||x|
    scale = (abs(A.T if transpose else A).astype(np.float64) @ np.abs(Xh[:, :k].astype(np.float64)))
    err = np.abs(got - want)
    assert np.all(err <= 1e-5 * scale + 1e-30), err.max()


@pytest.mark.parametrize("kind", ["zipf", "edges", "tiny", "wide"])
@pytest.mark.parametrize("k", [1, 8, 20, 50, 100, 128])
@pytest.mark.parametrize("transpose", [0, 1])
def test_spmm_forms_are_bit_identical(lib, kind, k, transpose):
    # every kernel form the autotuner may pick (gathers with different
    # unrolling) gives the same bits, and the fp16 forms match FP64 on the
    # fp16 inputs
    if kind == "wide":   # C2's row shape: Poisson(50) entries per row, Zipf(1.1) columns
        X = synth.planted(20000, 5000, 50, 1.1, 5, 10.0, 0.8, 0.1, 3)
        A, d = X.to_scipy().astype(np.float32), 5000
    else:
        A, d = csr_case(kind)
    m = A.shape[0]
    ld = (k + 7) // 8 * 8
    rows_in = m if transpose else d
    rng = np.random.default_rng(k + transpose)
    X32 = np.zeros((rows_in, ld), np.float32)
    X32[:, :k] = rng.uniform(-1, 1, (rows_in, k))
    X16 = X32.astype(np.float16)
    args = (m, d, dev(A.indptr, np.int32), dev(A.indices, np.int32), dev(A.data, np.float32), k)
    n_out = d if transpose else m
    for Xin, half in ((dev(X32), False), (dev(X16), True)):
        outs = []
        for v in range(lib.sfd_spmm_variant_count(half)):
            Y = torch.full((n_out, ld), 7.0, device="cuda")
            lib.sfd_csr_spmm_ex(*args, Xin, ld, Y, ld, transpose, v)
            outs.append(Y.cpu().numpy())
        for v, o in enumerate(outs[1:], 1):
            assert np.array_equal(o[:, :k], outs[0][:, :k]), (half, v)
        if half:
            Af = (A.T if transpose else A).astype(np.float64)
            want = Af @ X16[:, :k].astype(np.float64)
            scale = abs(Af) @ np.abs(X16[:, :k].astype(np.float64))
            assert np.all(np.abs(outs[0][:, :k] - want) <= 1e-5 * scale + 1e-30)


def test_spmm_is_deterministic(lib):
    A, d = csr_case("edges")
    m = A.shape[0]
    X = dev(np.random.default_rng(0).standard_normal((m, 104)).astype(np.float32))
    outs = []
    for _ in range(3):
        Y = torch.zeros((d, 104), device="cuda")
        lib.sfd_csr_spmm(m, d, dev(A.indptr, np.int32), dev(A.indices, np.int32),
                         dev(A.data, np.float32), 104, X, 104, Y, 104, 1)
        outs.append(Y.cpu().numpy())
    assert np.array_equal(outs[0], outs[1]) and np.array_equal(outs[1], outs[2])


@pytest.mark.parametrize("rows,k,cond", [(5000, 50, 10.0), (50000, 100, 1e3), (3000, 200, 1e2),
                                         (700, 256, 10.0), (64, 8, 1.0), (1000, 1, 1.0),
                                         (999, 17, 10.0), (2000, 127, 1e2), (4000, 128, 1e3),
                                         (500, 16, 1e3), (800, 33, 1e2), (20000, 64, 1e4),
                                         (20000, 100, 1e5), (10000, 50, 1e6)])
def test_orthonormalize(lib, rows, k, cond):
    rng = np.random.default_rng(rows + k)
    U, _ = np.linalg.qr(rng.standard_normal((rows, k)))
    V, _ = np.linalg.qr(rng.standard_normal((k, k)))
    s = np.logspace(0, -np.log10(cond), k)
    X = ((U * s) @ V.T * 3.0).astype(np.float32)
    ld = (k + 7) // 8 * 8
    Xp = np.zeros((rows, ld), np.float32)
    Xp[:, :k] = X
    T = dev(Xp)
    lib.sfd_orthonormalize(rows, k, T, ld)
    Q = T.cpu().numpy()[:, :k].astype(np.float64)
    assert np.linalg.norm(Q.T @ Q - np.eye(k)) < 5e-5 * k
    # same column span as X (projectors agree)
    Qr, _ = np.linalg.qr(X.astype(np.float64))
    assert np.linalg.norm(Q @ (Q.T @ Qr) - Qr) < 1e-4 * cond * np.sqrt(k)


def _sym(rng, n, kind):
    if kind == "random":
        A = rng.standard_normal((n, n))
        return (A + A.T) / 2
    if kind == "gram":      # PSD, decaying, rank-deficient (like [B; B'][B; B']^T)
        r = max(1, n // 2 - 1)
        M = rng.standard_normal((n, 4 * n)) * np.concatenate([0.9 ** np.arange(r), np.zeros(n - r)])[:, None]
        return M @ M.T
    if kind == "cluster":   # repeated eigenvalues
        Q, _ = np.linalg.qr(rng.standard_normal((n, n)))
        ev = np.repeat(np.linspace(10, 1, (n + 3) // 4), 4)[:n]
        return (Q * ev) @ Q.T
    raise KeyError(kind)


@pytest.mark.parametrize("n", [1, 2, 3, 17, 50, 100, 200, 224, 256, 400, 512])
@pytest.mark.parametrize("kind", ["random", "gram", "cluster"])
def test_symeig(lib, n, kind):
    rng = np.random.default_rng(n)
    S = _sym(rng, n, kind)
    nwant = max(1, n // 2) if n > 2 else n
    ev = torch.zeros(nwant, device="cuda")
    V = torch.zeros((n, nwant), device="cuda")
    Sf = S.astype(np.float32)
    lib.sfd_symeig(n, dev(Sf), nwant, ev, V)
    w_ref = np.linalg.eigvalsh(Sf.astype(np.float64))[::-1][:nwant]
    w = ev.cpu().numpy().astype(np.float64)
    nrm = np.abs(w_ref).max() + 1e-30
    assert np.all(np.abs(w - w_ref) <= 2e-5 * nrm * max(1, np.sqrt(n) / 4)), np.abs(w - w_ref).max() / nrm
    Vh = V.cpu().numpy().astype(np.float64)
    R = Sf.astype(np.float64) @ Vh - Vh * w
    assert np.linalg.norm(R, axis=0).max() <= 1e-4 * nrm * max(1, np.sqrt(n) / 4)
    assert np.linalg.norm(Vh.T @ Vh - np.eye(nwant)) <= 1e-3 * max(1, nwant / 16)


@pytest.mark.parametrize("rows,d,ell", [(100, 500, 50), (200, 2000, 100), (60, 300, 50),
                                        (7, 40, 10), (512, 3000, 256)])
def test_dense_shrink_matches_oracle(lib, rows, d, ell):
    rng = np.random.default_rng(rows)
    M = (rng.standard_normal((rows, d)) * (0.97 ** np.arange(d))[None, :]).astype(np.float32)
    B = torch.zeros((ell, d), device="cuda")
    lib.sfd_dense_shrink(rows, d, ell, dev(M), B)
    got = B.cpu().numpy().astype(np.float64)
    ref = O.dense_shrink(M.astype(np.float64), ell)
    from oracle.metrics import bbt_rel_diff
    # fp32 Gram + eigensolve of an n x n problem (n = rows): relative error ~ n u
    tol = max(1e-5, 2 * rows * 2.0 ** -24)
    assert bbt_rel_diff(got, ref) < tol
