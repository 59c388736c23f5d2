"""The two dense products of CholeskyQR (the GramSchmidt step of Alg. 1),
G = X^T X and Y = X T, on the CUDA cores (precision 0) and on the tcgen05
tensor cores (precision 1, TF32 inputs, FP32 accumulation), against FP64 on
the same inputs; and the whole stream with precision 1 against the oracle.

Error bounds. An input rounded to TF32 (10 stored mantissa bits) has relative
error at most 2^-10 (also when the conversion truncates), so a product of two
has at most 2 * 2^-10 + 2^-20; FP32 accumulation of r terms adds at most
r * 2^-24 of the sum of magnitudes. Elementwise:
  |G_tc - G| <= (3 * 2^-10 + r * 2^-23) * (|X|^T |X|),
  |G_fp32 - G| <= r * 2^-23 * (|X|^T |X|).
The split form (precision 2) writes x = x_hi + x_lo with x_hi exactly TF32 and
|x_lo| <= 2^-10 |x|, and forms x_hi y_hi + x_hi y_lo + x_lo y_hi with x_lo, y_lo
rounded to TF32 by the MMA: the dropped x_lo y_lo and the two roundings of the
lo parts leave at most 3 * 2^-20 |x y| per product, and each product adds
three terms to the FP32 accumulator:
  |G_split - G| <= (3 * 2^-20 + 3 r * 2^-23) * (|X|^T |X|).
On random inputs its error is also far below the TF32 form's (the per-product
term is 2^-10 times smaller): the tests check a factor 16."""
import numpy as np
import pytest

from oracle import metrics
from oracle import sfd as O
from paper_1602_00412_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

U_TF32 = 2.0 ** -10
U_F32 = 2.0 ** -24


@pytest.fixture(scope="module")
def lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__ as g
    g.build()
    from paper_1602_00412_gb300 import sfd
    return sfd


def _x(rows, k, ld, seed, scale_cols=False):
    rng = np.random.default_rng(seed)
    X = np.zeros((rows, ld), np.float32)
    X[:, :k] = rng.standard_normal((rows, k)).astype(np.float32)
    if scale_cols:  # columns of very different norms, as before an orthonormalisation
        X[:, :k] *= np.logspace(0, 4, k).astype(np.float32)
    return X


def _gram(lib, X, rows, k, ld, precision):
    G = torch.full((k, k), np.nan, device="cuda")
    lib.sfd_gram(rows, k, torch.from_numpy(X).cuda(), ld, G, precision)
    return G.cpu().numpy().astype(np.float64)


def _bound(precision, r):
    if precision == 2:
        return 3 * 2.0 ** -20 + 6 * r * U_F32
    return (3 * U_TF32 if precision else 0.0) + 2 * r * U_F32


@pytest.mark.parametrize("precision", [0, 1, 2])
@pytest.mark.parametrize("rows,k,ld", [(0, 8, 8), (1, 1, 4), (31, 50, 56), (33, 100, 104),
                                       (1000, 128, 128), (4097, 64, 64), (50000, 100, 104),
                                       (777, 17, 20)])
def test_gram(lib, precision, rows, k, ld):
    X = _x(rows, k, ld, rows + k, scale_cols=(rows % 2 == 1))
    got = _gram(lib, X, rows, k, ld, precision)
    X64 = X[:, :k].astype(np.float64)
    ref = X64.T @ X64
    mag = np.abs(X64).T @ np.abs(X64)
    u = _bound(precision, rows)
    assert np.all(np.abs(got - ref) <= u * mag + 1e-30), np.max(np.abs(got - ref) / (mag + 1e-30))
    if precision == 2 and rows > 0:
        e1 = np.max(np.abs(_gram(lib, X, rows, k, ld, 1) - ref) / (mag + 1e-30))
        e2 = np.max(np.abs(got - ref) / (mag + 1e-30))
        print("gram rows %d k %d: max rel err tf32 %.2e split %.2e" % (rows, k, e1, e2))
        assert e2 <= e1 / 16


@pytest.mark.parametrize("precision", [0, 1, 2])
@pytest.mark.parametrize("rows,n,kout,ldx,ldy", [(0, 8, 8, 8, 8), (1, 1, 1, 4, 4),
                                                  (127, 50, 50, 56, 56), (129, 100, 100, 104, 104),
                                                  (1000, 128, 128, 128, 128),
                                                  (50000, 100, 100, 104, 104),
                                                  (333, 17, 33, 20, 36), (300, 64, 7, 64, 8),
                                                  (500, 112, 112, 112, 112)])
def test_gemm_ts(lib, precision, rows, n, kout, ldx, ldy):
    X = _x(rows, n, ldx, 7 * rows + n)
    rng = np.random.default_rng(n * kout)
    T = np.triu(rng.standard_normal((n, kout))).astype(np.float32)
    Y = torch.full((max(rows, 1), ldy), 12345.0, device="cuda")
    args = (rows, n, torch.from_numpy(X).cuda(), ldx, torch.from_numpy(T).cuda(), kout, Y, ldy)
    if precision == 2 and max(n, kout) > 112:   # hi and lo of both operands exceed shared memory
        with pytest.raises(lib.SfdError) as ei:
            lib.sfd_gemm_ts(*args, precision)
        assert ei.value.code == lib.SFD_EINVAL
        return
    lib.sfd_gemm_ts(*args, precision)
    got = Y.cpu().numpy().astype(np.float64)
    if rows == 0:
        assert np.all(got == 12345.0)
        return
    X64, T64 = X[:, :n].astype(np.float64), T.astype(np.float64)
    ref = X64 @ T64
    mag = np.abs(X64) @ np.abs(T64)
    u = _bound(precision, n)
    assert np.all(np.abs(got[:rows, :kout] - ref) <= u * mag + 1e-30)
    assert np.all(got[:rows, kout:] == 12345.0)   # columns beyond kout untouched
    if precision == 2:
        Y1 = torch.full((max(rows, 1), ldy), 12345.0, device="cuda")
        lib.sfd_gemm_ts(*args[:6], Y1, ldy, 1)
        rel = lambda a: np.max(np.abs(a[:rows, :kout] - ref) / (mag + 1e-30))
        e1, e2 = rel(Y1.cpu().numpy().astype(np.float64)), rel(got)
        print("gemm rows %d n %d: max rel err tf32 %.2e split %.2e" % (rows, n, e1, e2))
        assert e2 <= e1 / 16


def test_tc_rejects_wide_blocks(lib):
    X = torch.zeros((10, 136), device="cuda")
    G = torch.zeros((136, 136), device="cuda")
    with pytest.raises(lib.SfdError) as ei:
        lib.sfd_gram(10, 136, X, 136, G, 1)
    assert ei.value.code == lib.SFD_EINVAL
    lib.sfd_gram(10, 136, X, 136, G, 0)   # the CUDA-core path takes it


def _stream(lib, X, d, ell, seed, **opts):
    s = lib.SFD(d, ell, seed, **opts)
    s.append(X.indptr, X.indices, X.values)
    B = s.sketch().astype(np.float64)
    st = s.stats()
    s.close()
    return B, st


@pytest.mark.parametrize("kind", ["gapped", "c1"])
def test_mixed_precision_stream(lib, kind):
    d, ell, k, seed = 2000, 50, 10, 0
    X = (synth.c1_gapped if kind == "gapped" else synth.c1)(seed=seed)
    B, st = _stream(lib, X, d, ell, seed, precision=1)
    ref, o = O.sfd_stream(X.indptr, X.indices, X.values, d, ell, seed)
    A = X.to_scipy()
    ce_gpu, ce_ref = metrics.cov_err(A, B), metrics.cov_err(A, ref)
    rel = metrics.bbt_rel_diff(B, ref)
    print("%s mixed: bbt rel %.2e  cov-err gpu %.4e oracle %.4e" % (kind, rel, ce_gpu, ce_ref))
    assert st["buffers"] == len(o.log)
    assert st["vs_rejects"] == 0
    assert abs(ce_gpu - ce_ref) <= 0.02 * ce_ref
    assert metrics.cov_norm(A, B) <= metrics.fd_bound(A, ell, k)
    if kind == "gapped":
        assert rel <= 1e-3, rel


def test_mixed_precision_is_deterministic(lib):
    d, ell, seed = 2000, 100, 3
    X = synth.c1_gapped(seed=seed, n=6000)
    B1, _ = _stream(lib, X, d, ell, seed, precision=1)
    B2, _ = _stream(lib, X, d, ell, seed, precision=1, slots=1)
    assert np.array_equal(B1, B2)


def test_invalid_precision_rejected(lib):
    with pytest.raises(lib.SfdError) as ei:
        lib.SFD(100, 10, 0, precision=2)
    assert ei.value.code == lib.SFD_EINVAL
