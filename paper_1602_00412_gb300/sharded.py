"""One stream sketched by several processes (one GPU each) through
mergeability (Sec. 3.1: merge(B1, B2) = DenseShrink([B1; B2]) keeps the FD
guarantee of the union).

  row_ranges       contiguous row ranges, one per rank (any cut is allowed:
                   a rank's first buffer simply starts at its first row)
  merge_schedule   the binary tree of merges, level by level: level s merges
                   rank i + s into rank i for i a multiple of 2 s (the order
                   of sfd_batch_merge_tree, so the same chunks give the same
                   bits either way)
  fold             apply the schedule to a list of states with a merge function
  gather_bytes     the one exchange step: every rank's checkpoint bytes to every
                   rank (torch.distributed all-gather of a length, then of the
                   padded bytes)
  sketch_sharded   each rank sketches its rows (seed + rank, like stream i of a
                   batch), checkpoints the flushed stream (sfd_save), the blobs
                   are gathered and rank 0 resumes each (sfd_load) and folds
                   them with sfd_merge
  pack_checkpoint / parse_checkpoint
                   the checkpoint layout of sfd_save, field by field (host code;
                   the tests check it against the library's own bytes)

Host code only: the sketching and every merge run in the library's kernels.
"""
import struct

import numpy as np

MAGIC = b"SFDCKPT1"
ABI_VERSION = 4
_HEAD = "<8sIIqiiQqqqii"          # magic .. inject_left, mode
_OPTS = "<didiiiiiff"             # delta verify c_q q_override retry_cap precision q_mode strict q_margin q_tau
_STATS_I = ("rows_seen", "nnz_seen", "buffers", "attempts", "vs_rejects", "unverified",
            "q_total", "pending_rows", "pending_nnz")
_STATS_F = ("last_delta", "last_logsum", "last_fro2")
_STATS = "<9q3dqqdd"
HEADER_BYTES = struct.calcsize(_HEAD) + struct.calcsize(_OPTS) + struct.calcsize(_STATS)
QPARAMS = 5313


def _fnv1a(data):
    h = 0xcbf29ce484222325
    for c in data:
        h ^= c
        h = (h * 0x100000001b3) & 0xFFFFFFFFFFFFFFFF
    return h


def parse_checkpoint(blob, check_hash=True):
    """The fields of a checkpoint blob (dict); raises ValueError on a bad blob.
    check_hash=False skips the hash (a byte-serial loop, slow for large d)."""
    blob = bytes(blob)
    if len(blob) < HEADER_BYTES + 8:
        raise ValueError("checkpoint too short")
    (stored,) = struct.unpack_from("<Q", blob, len(blob) - 8)
    if check_hash and _fnv1a(blob[:-8]) != stored:
        raise ValueError("checkpoint hash mismatch")
    f = {}
    (magic, abi, hb, f["d"], f["ell"], has_q, f["seed"], f["b"], prow, pnnz, f["inject_left"],
     mode) = struct.unpack_from(_HEAD, blob, 0)
    if magic != MAGIC or abi != ABI_VERSION or hb != HEADER_BYTES:
        raise ValueError("not a checkpoint of this library version")
    at = struct.calcsize(_HEAD)
    o = struct.unpack_from(_OPTS, blob, at)
    f["options"] = dict(zip(("delta", "verify", "c_q", "q_override", "retry_cap", "precision",
                             "q_mode", "strict", "q_margin", "q_tau"), o))
    f["options"]["mode"] = mode
    at += struct.calcsize(_OPTS)
    st = struct.unpack_from(_STATS, blob, at)
    f["stats"] = dict(zip(_STATS_I + _STATS_F + ("kernel_launches", "spmm_launches", "spmm_ms",
                                                   "spmm_bytes"), st))
    at += struct.calcsize(_STATS)
    d, ell = f["d"], f["ell"]
    f["B"] = np.frombuffer(blob, dtype="<f4", count=ell * d, offset=at).reshape(ell, d).copy()
    at += 4 * ell * d
    f["ptr"] = np.frombuffer(blob, dtype="<i4", count=prow + 1, offset=at).copy()
    at += 4 * (prow + 1)
    f["idx"] = np.frombuffer(blob, dtype="<i4", count=pnnz, offset=at).copy()
    at += 4 * pnnz
    f["val"] = np.frombuffer(blob, dtype="<f4", count=pnnz, offset=at).copy()
    at += 4 * pnnz
    f["qparams"] = None
    if has_q:
        f["qparams"] = np.frombuffer(blob, dtype="<f4", count=QPARAMS, offset=at).copy()
        at += 4 * QPARAMS
    if at != len(blob) - 8:
        raise ValueError("checkpoint size does not match its header")
    return f


def pack_checkpoint(f):
    """The bytes of a checkpoint with the fields of parse_checkpoint (same
    layout as the library's sfd_save)."""
    d, ell = int(f["d"]), int(f["ell"])
    B = np.ascontiguousarray(f["B"], dtype="<f4").reshape(ell, d)
    ptr = np.ascontiguousarray(f.get("ptr", np.zeros(1)), dtype="<i4")
    idx = np.ascontiguousarray(f.get("idx", np.zeros(0)), dtype="<i4")
    val = np.ascontiguousarray(f.get("val", np.zeros(0)), dtype="<f4")
    qp = f.get("qparams")
    o = f["options"]
    st = f.get("stats") or {}
    parts = [
        struct.pack(_HEAD, MAGIC, ABI_VERSION, HEADER_BYTES, d, ell, int(qp is not None),
                    int(f["seed"]), int(f["b"]), len(ptr) - 1, len(idx),
                    int(f.get("inject_left", 0)), int(o.get("mode", 0))),
        struct.pack(_OPTS, o["delta"], o["verify"], o["c_q"], o["q_override"], o["retry_cap"],
                    o["precision"], o["q_mode"], o["strict"], o["q_margin"], o["q_tau"]),
        struct.pack(_STATS, *[int(st.get(k, 0)) for k in _STATS_I],
                    *[float(st.get(k, 0.0)) for k in _STATS_F],
                    int(st.get("kernel_launches", 0)), int(st.get("spmm_launches", 0)),
                    float(st.get("spmm_ms", 0.0)), float(st.get("spmm_bytes", 0.0))),
        B.tobytes(), ptr.tobytes(), idx.tobytes(), val.tobytes(),
    ]
    if qp is not None:
        parts.append(np.ascontiguousarray(qp, dtype="<f4").tobytes())
    body = b"".join(parts)
    return body + struct.pack("<Q", _fnv1a(body))


# ------------------------------------------------------------------ the tree
def row_ranges(n, world):
    """[(a_r, b_r)] for r < world: contiguous, sizes differing by at most 1."""
    if world < 1:
        raise ValueError("world >= 1")
    q, r = divmod(int(n), world)
    out, a = [], 0
    for i in range(world):
        b = a + q + (1 if i < r else 0)
        out.append((a, b))
        a = b
    return out


def merge_schedule(n):
    """Levels of (dst, src) merges folding n states into state 0: at level s
    (s = 1, 2, 4, ...) state i + s is merged into state i for i a multiple of 2s."""
    levels, step = [], 1
    while step < n:
        levels.append([(i, i + step) for i in range(0, n - step, 2 * step)])
        step *= 2
    return levels


def fold(states, merge):
    """Apply merge_schedule(len(states)): states[dst] = merge(states[dst],
    states[src]) level by level; returns states[0]."""
    states = list(states)
    for level in merge_schedule(len(states)):
        for dst, src in level:
            states[dst] = merge(states[dst], states[src])
    return states[0]


def gather_bytes(blob, group=None):
    """Every rank's `blob` (bytes) on every rank, in rank order: the one
    collective of the sharded path. CPU tensors for gloo, CUDA tensors for
    NCCL."""
    import torch
    import torch.distributed as dist
    world = dist.get_world_size(group)
    device = torch.device("cuda", torch.cuda.current_device()) \
        if dist.get_backend(group) == "nccl" else torch.device("cpu")
    n = torch.tensor([len(blob)], dtype=torch.int64, device=device)
    sizes = [torch.zeros_like(n) for _ in range(world)]
    dist.all_gather(sizes, n, group=group)
    sizes = [int(x.item()) for x in sizes]
    cap = max(sizes)
    mine = torch.zeros(cap, dtype=torch.uint8, device=device)
    if len(blob):
        mine[:len(blob)] = torch.frombuffer(bytearray(blob), dtype=torch.uint8).to(device)
    bufs = [torch.zeros(cap, dtype=torch.uint8, device=device) for _ in range(world)]
    dist.all_gather(bufs, mine, group=group)
    return [bytes(b[:k].cpu().numpy().tobytes()) for b, k in zip(bufs, sizes)]


def sketch_sharded(indptr, indices, values, d, ell, seed, group=None, **opts):
    """This rank's rows (its range of the stream) through SFD on the current
    GPU with seed + rank; the flushed sketches are gathered and folded on
    rank 0 by the merge tree. Returns the l x d sketch on rank 0, None elsewhere."""
    import torch.distributed as dist
    from . import sfd
    rank = dist.get_rank(group)
    s = sfd.SFD(d, ell, seed + rank, **opts)
    try:
        s.append(indptr, indices, values)
        s.sketch()                       # flush the open buffer (R6)
        blob = s.save()
    finally:
        s.close()
    blobs = gather_bytes(blob, group)
    if rank != 0:
        return None
    ctxs = [sfd.SFD.load(b) for b in blobs]
    try:
        def merge(a, b):
            a.merge(b)
            return a
        return fold(ctxs, merge).sketch()
    finally:
        for c in ctxs:
            c.close()
