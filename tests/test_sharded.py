"""The multi-process path (paper_1602_00412_gb300/sharded.py) on CPU: gloo
ranks exchange real serialized sketches and fold them by the merge tree.

Each rank sketches its contiguous range of one stream (Sec. 3.1
mergeability); here the per-rank sketch comes from the FP64 oracle (the GPU
does that step in the -m gpu tests), is serialized in the checkpoint layout
of sfd_save, gathered over gloo, parsed on rank 0 and folded with the
oracle's DenseShrink in the order of merge_schedule. The result must equal
the same fold done in one process, and satisfy the FD bound of the whole
stream. No GPU and no kernel runs here; the checkpoint layout itself is
checked against the library's own bytes in tests/test_gpu_checkpoint.py.
"""
import json
import os
import socket

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

from oracle import metrics  # noqa: E402
from oracle import sfd as O  # noqa: E402
from paper_1602_00412_gb300 import sharded as S  # noqa: E402
from paper_1602_00412_gb300 import synth  # noqa: E402

D, ELL, SEED, N = 300, 12, 7, 2400
OPTS = {"delta": 0.01, "verify": 1, "c_q": 0.25, "q_override": -1, "retry_cap": 8,
        "precision": 0, "q_mode": 0, "strict": 0, "q_margin": 1.0, "q_tau": 0.01, "mode": 0}


def _stream():
    return synth.planted(N, D, 10, 1.1, 6, 10.0, 0.7, 0.1, 3)


def _rank_blob(X, rank, world):
    a, b = S.row_ranges(X.n, world)[rank]
    part = X.rows(a, b)
    B, o = O.sfd_stream(part.indptr, part.indices, part.values, D, ELL, SEED + rank)
    return S.pack_checkpoint({"d": D, "ell": ELL, "seed": SEED + rank, "b": o.b, "B": B,
                              "options": OPTS, "stats": {"rows_seen": part.n}})


def _merge(Ba, Bb):
    return O.dense_shrink(np.vstack([Ba, Bb]), ELL).astype(np.float32).astype(np.float64)


def _fold_blobs(blobs):
    states = [S.parse_checkpoint(b)["B"].astype(np.float64) for b in blobs]
    return S.fold(states, _merge)


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out_dir):
    dist.init_process_group("gloo", init_method="tcp://127.0.0.1:%d" % port, rank=rank,
                            world_size=world)
    try:
        X = _stream()
        blob = _rank_blob(X, rank, world)
        blobs = S.gather_bytes(blob)
        assert blobs[rank] == blob
        out = {"sizes": [len(b) for b in blobs],
               "seeds": [S.parse_checkpoint(b)["seed"] for b in blobs]}
        if rank == 0:
            np.save(os.path.join(out_dir, "merged.npy"), _fold_blobs(blobs))
        with open(os.path.join(out_dir, "rank%d.json" % rank), "w") as f:
            json.dump(out, f)
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("world", [2, 3])
def test_gloo_ranks_gather_and_fold_real_sketches(tmp_path, world):
    mp.spawn(_rank_main, args=(world, _free_port(), str(tmp_path)), nprocs=world, join=True)
    res = [json.load(open(tmp_path / ("rank%d.json" % r))) for r in range(world)]
    for r in res:  # every rank saw every rank's bytes, in rank order
        assert r == res[0]
        assert r["seeds"] == [SEED + i for i in range(world)]
    merged = np.load(tmp_path / "merged.npy")
    X = _stream()
    ref = _fold_blobs([_rank_blob(X, r, world) for r in range(world)])
    assert np.array_equal(merged, ref)
    A = X.to_scipy()
    lo, hi = metrics.residual_eigs(A, merged)
    assert lo >= -1e-5 * metrics.fro2(A)          # Prop. 1 through the merges
    assert hi <= metrics.fd_bound(A, ELL, 4)      # the FD bound of the union


def test_merge_schedule_is_the_batch_tree():
    # level s merges i + s into i for i a multiple of 2 s; every state but 0 is
    # merged exactly once, after everything merged into it
    for n in range(1, 12):
        lv = S.merge_schedule(n)
        assert len(lv) == (n - 1).bit_length()
        seen_src, done = [], set()
        for s, level in enumerate(lv):
            step = 1 << s
            assert level == [(i, i + step) for i in range(0, n, 2 * step) if i + step < n]
            for dst, src in level:
                assert dst not in done and src not in done
                done.add(src)
                seen_src.append(src)
        assert sorted(seen_src) == list(range(1, n))
    # fold with string concatenation shows the order of the merges
    assert S.fold(list("abcde"), lambda x, y: "(%s%s)" % (x, y)) == "(((ab)(cd))e)"


def test_row_ranges_cover_the_stream():
    for n, w in [(10, 3), (7, 7), (5, 8), (1000001, 4)]:
        r = S.row_ranges(n, w)
        assert r[0][0] == 0 and r[-1][1] == n and len(r) == w
        assert all(a1 == b0 for (_, b0), (a1, _) in zip(r, r[1:]))
        sizes = [b - a for a, b in r]
        assert max(sizes) - min(sizes) <= 1


def test_checkpoint_layout_round_trip_and_hash():
    rng = np.random.default_rng(0)
    f = {"d": 9, "ell": 3, "seed": 123, "b": 17, "B": rng.standard_normal((3, 9)),
         "ptr": np.array([0, 2, 5]), "idx": np.array([1, 4, 0, 2, 8]),
         "val": rng.standard_normal(5), "options": OPTS, "inject_left": 2,
         "stats": {"rows_seen": 40, "buffers": 4, "last_delta": 0.5}}
    blob = S.pack_checkpoint(f)
    assert len(blob) == S.HEADER_BYTES + 4 * (27 + 3 + 5 + 5) + 8
    g = S.parse_checkpoint(blob)
    assert (g["d"], g["ell"], g["seed"], g["b"], g["inject_left"]) == (9, 3, 123, 17, 2)
    assert np.array_equal(g["B"], f["B"].astype(np.float32))
    assert np.array_equal(g["ptr"], f["ptr"]) and np.array_equal(g["idx"], f["idx"])
    assert g["stats"]["rows_seen"] == 40 and g["stats"]["last_delta"] == 0.5
    assert g["options"] == pytest.approx(OPTS)
    assert S.pack_checkpoint(g) == blob
    bad = bytearray(blob)
    bad[S.HEADER_BYTES + 5] ^= 1
    with pytest.raises(ValueError):
        S.parse_checkpoint(bytes(bad))
    with pytest.raises(ValueError):
        S.parse_checkpoint(blob[:-9] + blob[-8:])
