"""Many streams on one GPU (sfd_batch_*): every stream of a batch gives the
sketch its own context gives (same seed), streams of different shapes run side
by side, errors of queued work surface at the next wait, and the chunk-parallel
merge tree matches the FP64 oracle running the same tree of DenseShrinks."""
import numpy as np
import pytest

from oracle import metrics
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


def _single(lib, X, d, ell, seed):
    s = lib.SFD(d, ell, seed, slots=1)
    s.append(X.indptr, X.indices, X.values)
    B = s.sketch()
    s.close()
    return B


def test_streams_of_mixed_shapes_match_single_contexts(lib):
    rng = np.random.default_rng(0)
    shapes = [(int(rng.integers(300, 2000)), int(rng.choice([20, 50]))) for _ in range(12)]
    data = [synth.planted(int(rng.integers(800, 4000)), d, 15, 1.1, max(2, ell // 4), 10.0, 0.9,
                          0.1, 100 + i) for i, (d, ell) in enumerate(shapes)]
    bt = lib.Batch([d for d, _ in shapes], [ell for _, ell in shapes], seed=40, workers=4)
    # rows arrive interleaved across streams, in uneven pieces
    cuts = [sorted(set(rng.integers(1, X.n, 5).tolist())) for X in data]
    pieces = [list(zip([0] + c, c + [X.n])) for c, X in zip(cuts, data)]
    for k in range(max(len(p) for p in pieces)):
        for i, X in enumerate(data):
            if k < len(pieces[i]):
                a, b = pieces[i][k]
                part = X.rows(a, b)
                bt.append(i, part.indptr, part.indices, part.values)
    for i, (X, (d, ell)) in enumerate(zip(data, shapes)):
        B = bt.sketch(i)
        assert np.array_equal(B, _single(lib, X, d, ell, 40 + i))
        A = X.to_scipy()
        k = max(1, ell // 4)
        assert metrics.cov_norm(A, B.astype(np.float64)) <= metrics.fd_bound(A, ell, k)
        assert bt.stats(i)["rows_seen"] == X.n
    bt.close()


def test_device_input_and_error_reporting(lib):
    d, ell = 500, 20
    X = synth.planted(1200, d, 10, 1.1, 3, 10.0, 0.7, 0.1, 9)
    bt = lib.Batch([d, d], [ell, ell], seed=3, workers=2)
    dev = lambda a, t: torch.from_numpy(np.ascontiguousarray(a, dtype=t)).cuda()
    bt.append(0, dev(X.indptr, np.int64), dev(X.indices, np.int32), dev(X.values, np.float32))
    bad = X.indices.copy()
    bad[7] = d   # out of range: the worker's append fails
    bt.append(1, X.indptr, bad, X.values)
    with pytest.raises(lib.SfdError) as ei:
        bt.wait()
    assert ei.value.code == lib.SFD_EINVAL
    assert np.array_equal(bt.sketch(0), _single(lib, X, d, ell, 3))
    bt.append(1, X.indptr, X.indices, X.values)   # the stream is still usable
    assert np.array_equal(bt.sketch(1), _single(lib, X, d, ell, 4))
    bt.close()


@pytest.mark.parametrize("nchunks", [8, 5])
def test_merge_tree_matches_oracle(lib, nchunks):
    d, ell, seed = 2000, 50, 7
    X = synth.c1_gapped(seed=1, n=12000)
    bounds = np.linspace(0, X.n, nchunks + 1).astype(int)
    bt = lib.Batch([d] * nchunks, [ell] * nchunks, seed=seed, workers=4)
    orc = [O.SFDOracle(d, ell, seed + c) for c in range(nchunks)]
    for c in range(nchunks):
        part = X.rows(bounds[c], bounds[c + 1])
        bt.append(c, part.indptr, part.indices, part.values)
        orc[c].append_rows(part.indptr, part.indices, part.values)
    B = bt.merge_tree().astype(np.float64)
    step = 1
    while step < nchunks:
        for i in range(0, nchunks - step, 2 * step):
            orc[i].merge(orc[i + step])
        step *= 2
    ref = orc[0].sketch()
    assert metrics.bbt_rel_diff(B, ref) <= 1e-4
    A = X.to_scipy()
    # the tree keeps the guarantee of the sequential stream
    assert metrics.cov_norm(A, B) <= metrics.fd_bound(A, ell, 10)
    seq = _single(lib, X, d, ell, seed).astype(np.float64)
    print("cov-err tree %.4e sequential %.4e" % (metrics.cov_err(A, B), metrics.cov_err(A, seq)))
    bt.close()
