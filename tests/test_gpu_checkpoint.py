"""Checkpoint / resume (sfd_save, sfd_load) and the sharded merge through the
C ABI on the GPU.

  - a stream checkpointed at any row and resumed in a new context gives the
    same sketch, bit for bit, as the uninterrupted stream (plain and mixed
    precision, another slot count for the resumed context);
  - the library's checkpoint bytes follow the layout sharded.py reads and
    writes (pack(parse(blob)) == blob; B in the blob equals B before flush);
  - damaged blobs are rejected with SFD_EINVAL;
  - the sharded path (per-rank streams with seed + rank, flushed, saved,
    resumed and folded by the merge tree) equals sfd_batch_merge_tree on the
    same chunks bit for bit, and its sketch stays within 2% of the FP64
    oracle's fold of the same chunks in cov-err.
"""
import numpy as np
import pytest

from oracle import metrics
from oracle import sfd as O
from paper_1602_00412_gb300 import sharded as S
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


def _feed(s, X, a, b):
    part = X.rows(a, b)
    s.append(part.indptr, part.indices, part.values)


@pytest.mark.parametrize("precision", [0, 1])
@pytest.mark.parametrize("cut", [1, 2000, 3517, 6999])
def test_resume_is_bit_identical(lib, precision, cut):
    d, ell, seed = 2000, 50, 9
    X = synth.c1_gapped(seed=seed, n=7000)
    ref = lib.SFD(d, ell, seed, precision=precision)
    _feed(ref, X, 0, X.n)
    B_ref = ref.sketch()
    st_ref = ref.stats()
    ref.close()
    s = lib.SFD(d, ell, seed, precision=precision)
    _feed(s, X, 0, cut)
    blob = s.save()
    s.close()
    r = lib.SFD.load(blob, slots=2)
    _feed(r, X, cut, X.n)
    assert np.array_equal(r.sketch(), B_ref)
    st = r.stats()
    assert (st["buffers"], st["attempts"], st["rows_seen"]) == \
        (st_ref["buffers"], st_ref["attempts"], st_ref["rows_seen"])
    r.close()


def test_checkpoint_bytes_follow_the_layout(lib):
    d, ell, seed = 2000, 50, 4
    X = synth.c1(seed=seed, n=5100)             # two buffers closed, 1,100 rows open
    s = lib.SFD(d, ell, seed, precision=1, q_override=5)
    _feed(s, X, 0, X.n)
    blob = s.save()
    f = S.parse_checkpoint(blob)
    assert (f["d"], f["ell"], f["seed"], f["b"]) == (d, ell, seed, 2)
    assert f["options"]["precision"] == 1 and f["options"]["q_override"] == 5
    part = X.rows(4000, X.n)
    assert np.array_equal(f["ptr"], part.indptr - part.indptr[0])
    assert np.array_equal(f["idx"], part.indices) and np.array_equal(f["val"], part.values)
    assert S.pack_checkpoint(f) == blob
    # B before the flush: the same bits the first 4,000 rows give as a stream
    s2 = lib.SFD(d, ell, seed, precision=1, q_override=5)
    _feed(s2, X, 0, 4000)
    assert np.array_equal(f["B"], s2.sketch())
    s.close()
    s2.close()


def test_damaged_checkpoints_are_rejected(lib):
    d, ell = 500, 20
    X = synth.planted(900, d, 10, 1.1, 3, 10.0, 0.7, 0.1, 2)
    s = lib.SFD(d, ell, 1)
    _feed(s, X, 0, X.n)
    blob = s.save()
    s.close()
    for bad in (blob[:-1], blob[:100], b"x" * len(blob),
                blob[:S.HEADER_BYTES + 3] + bytes([blob[S.HEADER_BYTES + 3] ^ 4]) +
                blob[S.HEADER_BYTES + 4:]):
        with pytest.raises(lib.SfdError) as ei:
            lib.SFD.load(bad)
        assert ei.value.code == lib.SFD_EINVAL
    r = lib.SFD.load(blob)        # the intact blob still loads
    r.close()


@pytest.mark.parametrize("world", [2, 5])
def test_sharded_fold_equals_batch_merge_tree(lib, world):
    d, ell, seed = 2000, 50, 21
    X = synth.c1(seed=seed, n=9000)
    ranges = S.row_ranges(X.n, world)
    # the per-rank half of sketch_sharded, ranks run one after another here
    blobs = []
    for r, (a, b) in enumerate(ranges):
        s = lib.SFD(d, ell, seed + r, precision=1)
        _feed(s, X, a, b)
        s.sketch()
        blobs.append(s.save())
        s.close()
    ctxs = [lib.SFD.load(b) for b in blobs]

    def merge(x, y):
        x.merge(y)
        return x
    B = S.fold(ctxs, merge).sketch()
    for c in ctxs:
        c.close()
    bt = lib.Batch([d] * world, [ell] * world, seed, precision=1)
    for r, (a, b) in enumerate(ranges):
        part = X.rows(a, b)
        bt.append(r, part.indptr, part.indices, part.values)
    Bt = bt.merge_tree()
    bt.close()
    assert np.array_equal(B, Bt)
    # the oracle: each chunk sketched in FP64 with its seed, folded in the same order
    refs = []
    for r, (a, b) in enumerate(ranges):
        part = X.rows(a, b)
        refs.append(O.sfd_stream(part.indptr, part.indices, part.values, d, ell, seed + r)[0])
    ref = S.fold(refs, lambda x, y: O.dense_shrink(np.vstack([x, y]), ell))
    A = X.to_scipy()
    ce, ce_ref = metrics.cov_err(A, B.astype(np.float64)), metrics.cov_err(A, ref)
    assert abs(ce - ce_ref) <= 0.02 * ce_ref, (ce, ce_ref)
    assert metrics.cov_norm(A, B.astype(np.float64)) <= metrics.fd_bound(A, ell, 10)
