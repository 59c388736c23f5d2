"""ctypes binding of libsfd.so (include/sfd.h): the same entry points, with
argument marshalling only. Host arrays are numpy arrays; device arrays are
torch CUDA tensors (PyTorch supplies device memory and streams). Every
computation runs in the library's CUDA kernels; if the library is missing,
loading fails loudly.
"""
import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "lib", "libsfd.so")

SFD_ABI_VERSION = 4
SFD_OK, SFD_EINVAL, SFD_ENOMEM, SFD_ECUDA, SFD_EVERIFY, SFD_ETIMEOUT = 0, 1, 2, 3, 4, 5
SFD_HOST, SFD_DEVICE = 0, 1


class SfdError(RuntimeError):
    def __init__(self, code, msg=""):
        self.code = code
        super().__init__("sfd error %d (%s)%s" % (code, _strerror(code), (": " + msg) if msg else ""))


class sfd_options(ctypes.Structure):
    _fields_ = [("abi_version", ctypes.c_uint32), ("delta", ctypes.c_double),
                ("verify", ctypes.c_int32), ("c_q", ctypes.c_double),
                ("q_override", ctypes.c_int32), ("retry_cap", ctypes.c_int32),
                ("precision", ctypes.c_int32), ("q_mode", ctypes.c_int32),
                ("strict", ctypes.c_int32), ("inject_vs_fail", ctypes.c_int32),
                ("cuda_stream", ctypes.c_void_p), ("profile", ctypes.c_int32),
                ("slots", ctypes.c_int32), ("q_margin", ctypes.c_float), ("q_tau", ctypes.c_float),
                ("autotune", ctypes.c_int32), ("mode", ctypes.c_int32)]


class sfd_stats(ctypes.Structure):
    _fields_ = [(n, ctypes.c_int64) for n in ("rows_seen", "nnz_seen", "buffers", "attempts",
                                               "vs_rejects", "unverified", "q_total",
                                               "pending_rows", "pending_nnz")] + \
               [(n, ctypes.c_double) for n in ("last_delta", "last_logsum", "last_fro2")] + \
               [("kernel_launches", ctypes.c_int64), ("spmm_launches", ctypes.c_int64),
                ("spmm_ms", ctypes.c_double), ("spmm_bytes", ctypes.c_double)]


class sfd_shrink_info(ctypes.Structure):
    _fields_ = [("q", ctypes.c_int32), ("attempts", ctypes.c_int32), ("verified", ctypes.c_int32),
                ("vs_steps", ctypes.c_int32), ("delta_shrink", ctypes.c_double),
                ("logsum", ctypes.c_double), ("fro2_a", ctypes.c_double),
                ("fro2_b", ctypes.c_double), ("captured", ctypes.c_double)]


EXPORTS = ["sfd_options_init", "sfd_create", "sfd_append_rows", "sfd_sketch", "sfd_merge",
           "sfd_get_stats", "sfd_reset", "sfd_destroy", "sfd_strerror", "sfd_last_error", "sfd_bssh_buffer",
           "sfd_dense_shrink", "sfd_csr_spmm", "sfd_spmm_variant_count", "sfd_csr_spmm_ex",
           "sfd_orthonormalize", "sfd_symeig",
           "sfd_symeig_noalloc", "sfd_gram", "sfd_gemm_ts", "sfd_set_wait_limit", "sfd_wait_selftest",
           "sfd_set_q_model", "sfd_q_log",
           "sfd_q_features", "sfd_q_predict", "sfd_q_grad", "sfd_q_train", "sfd_batch_create",
           "sfd_batch_append", "sfd_batch_wait", "sfd_batch_sketch", "sfd_batch_merge_tree",
           "sfd_batch_stats", "sfd_batch_destroy", "sfd_save", "sfd_load"]
QF, QPARAMS = 16, 5313

_lib = None


def load(path=None):
    """Load libsfd.so (raises if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    p = path or LIB_PATH
    if not os.path.exists(p):
        raise RuntimeError("libsfd.so not found at %s: build it with "
                           "paper_1602_00412_gb300.build.build()" % p)
    L = ctypes.CDLL(p)
    vp, i32, i64, u64 = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_uint64
    L.sfd_options_init.argtypes = [ctypes.POINTER(sfd_options)]
    L.sfd_options_init.restype = None
    L.sfd_create.argtypes = [i64, i32, u64, ctypes.POINTER(sfd_options), ctypes.POINTER(vp)]
    L.sfd_append_rows.argtypes = [vp, i64, vp, vp, vp, ctypes.c_int]
    L.sfd_sketch.argtypes = [vp, vp, ctypes.c_int]
    L.sfd_merge.argtypes = [vp, vp]
    L.sfd_get_stats.argtypes = [vp, ctypes.POINTER(sfd_stats)]
    L.sfd_reset.argtypes = [vp]
    L.sfd_destroy.argtypes = [vp]
    L.sfd_destroy.restype = None
    L.sfd_strerror.argtypes = [ctypes.c_int]
    L.sfd_strerror.restype = ctypes.c_char_p
    L.sfd_last_error.argtypes = [vp]
    L.sfd_last_error.restype = ctypes.c_char_p
    L.sfd_bssh_buffer.argtypes = [i64, i64, i32, vp, vp, vp, u64, i64, ctypes.POINTER(sfd_options),
                                  vp, ctypes.POINTER(sfd_shrink_info)]
    L.sfd_dense_shrink.argtypes = [i64, i64, i32, vp, vp]
    L.sfd_csr_spmm.argtypes = [i64, i64, vp, vp, vp, i32, vp, i32, vp, i32, i32]
    L.sfd_spmm_variant_count.argtypes = [i32]
    L.sfd_csr_spmm_ex.argtypes = [i64, i64, vp, vp, vp, i32, vp, i32, i32, vp, i32, i32, i32]
    L.sfd_orthonormalize.argtypes = [i64, i32, vp, i32]
    L.sfd_symeig.argtypes = [i32, vp, i32, vp, vp]
    L.sfd_symeig_noalloc.argtypes = [i32, vp, i32, vp, vp]
    L.sfd_gram.argtypes = [i64, i32, vp, i32, vp, i32]
    L.sfd_gemm_ts.argtypes = [i64, i32, vp, i32, vp, i32, vp, i32, i32]
    L.sfd_set_wait_limit.argtypes = [i64]
    L.sfd_wait_selftest.argtypes = [i64, ctypes.POINTER(ctypes.c_float)]
    L.sfd_set_q_model.argtypes = [vp, vp]
    L.sfd_q_log.argtypes = [vp, i64, vp, vp, vp, ctypes.POINTER(i64)]
    L.sfd_q_features.argtypes = [i64, i64, i32, vp, vp, vp, u64, i64, i32, vp]
    L.sfd_q_predict.argtypes = [i64, vp, vp, vp]
    L.sfd_q_grad.argtypes = [i64, vp, vp, vp, vp, vp]
    L.sfd_q_train.argtypes = [i64, vp, vp, i32, i32, ctypes.c_float, u64, vp, vp]
    L.sfd_batch_create.argtypes = [i32, vp, vp, u64, ctypes.POINTER(sfd_options), i32,
                                   ctypes.POINTER(vp)]
    L.sfd_batch_append.argtypes = [vp, i32, i64, vp, vp, vp, ctypes.c_int]
    L.sfd_batch_wait.argtypes = [vp]
    L.sfd_batch_sketch.argtypes = [vp, i32, vp, ctypes.c_int]
    L.sfd_batch_merge_tree.argtypes = [vp, vp, ctypes.c_int]
    L.sfd_batch_stats.argtypes = [vp, i32, ctypes.POINTER(sfd_stats)]
    L.sfd_batch_destroy.argtypes = [vp]
    L.sfd_save.argtypes = [vp, vp, i64, ctypes.POINTER(i64)]
    L.sfd_load.argtypes = [vp, i64, ctypes.POINTER(sfd_options), ctypes.POINTER(vp)]
    for name in EXPORTS:
        fn = getattr(L, name)
        if name not in ("sfd_options_init", "sfd_destroy", "sfd_strerror", "sfd_last_error",
                        "sfd_batch_destroy"):
            fn.restype = ctypes.c_int
    _lib = L
    return L


def _strerror(code):
    try:
        return load().sfd_strerror(code).decode()
    except Exception:
        return "?"


def _check(rc, ctx=None):
    if rc != SFD_OK:
        msg = ""
        if ctx is not None:
            msg = (load().sfd_last_error(ctx) or b"").decode()
        raise SfdError(rc, msg)


def _is_torch_cuda(x):
    return hasattr(x, "is_cuda") and x.is_cuda


def _ptr(x, dtype):
    """(pointer, where) for a numpy array or a torch CUDA tensor of `dtype`."""
    if x is None:
        return None, SFD_HOST
    if _is_torch_cuda(x):
        import torch
        tdt = {np.int64: torch.int64, np.int32: torch.int32, np.float32: torch.float32}[dtype]
        if x.dtype != tdt or not x.is_contiguous():
            raise TypeError("device array must be a contiguous %s tensor" % tdt)
        return ctypes.c_void_p(x.data_ptr()), SFD_DEVICE
    a = np.asarray(x)
    if a.dtype != dtype or not a.flags["C_CONTIGUOUS"]:
        raise TypeError("host array must be a C-contiguous %s array" % np.dtype(dtype))
    return ctypes.c_void_p(a.ctypes.data), SFD_HOST


def options(**kw):
    o = sfd_options()
    load().sfd_options_init(ctypes.byref(o))
    for k, v in kw.items():
        if not hasattr(o, k):
            raise KeyError(k)
        setattr(o, k, v)
    return o


# --------------------------------------------------------------- entry points
def sfd_create(d, ell, seed, opts=None):
    h = ctypes.c_void_p()
    _check(load().sfd_create(d, ell, seed, ctypes.byref(opts) if opts is not None else None,
                             ctypes.byref(h)))
    return h


def sfd_append_rows(ctx, indptr, indices, values):
    """indptr (n+1 int64), indices (int32), values (float32): all numpy, or all
    torch CUDA tensors."""
    n = len(indptr) - 1
    pi, w1 = _ptr(indptr, np.int64)
    px, w2 = _ptr(indices, np.int32)
    pv, w3 = _ptr(values, np.float32)
    if not (w1 == w2 == w3):
        raise TypeError("indptr, indices and values must all be host or all device arrays")
    _check(load().sfd_append_rows(ctx, n, pi, px, pv, w1), ctx)


def sfd_sketch(ctx, out):
    """Write B (l x d float32) into `out` (numpy array or torch CUDA tensor)."""
    p, w = _ptr(out, np.float32)
    _check(load().sfd_sketch(ctx, p, w), ctx)
    return out


def sfd_merge(dst, src):
    _check(load().sfd_merge(dst, src), dst)


def sfd_get_stats(ctx):
    s = sfd_stats()
    _check(load().sfd_get_stats(ctx, ctypes.byref(s)))
    return {f: getattr(s, f) for f, _ in sfd_stats._fields_}


def sfd_reset(ctx):
    _check(load().sfd_reset(ctx), ctx)


def sfd_destroy(ctx):
    load().sfd_destroy(ctx)


def sfd_save(ctx):
    """The context's state as bytes (sfd_save): sketch, open buffer, counters."""
    n = ctypes.c_int64()
    _check(load().sfd_save(ctx, None, 0, ctypes.byref(n)), ctx)
    buf = ctypes.create_string_buffer(n.value)
    _check(load().sfd_save(ctx, buf, n.value, ctypes.byref(n)), ctx)
    return buf.raw[:n.value]


def sfd_load(blob, runtime=None):
    """A context resumed from sfd_save bytes; `runtime` options supply only
    cuda_stream, slots, profile and autotune."""
    h = ctypes.c_void_p()
    b = bytes(blob)
    _check(load().sfd_load(b, len(b), ctypes.byref(runtime) if runtime is not None else None,
                           ctypes.byref(h)))
    return h


def sfd_bssh_buffer(m, d, ell, rowptr, colidx, vals, seed, b, Bp_out, opts=None):
    info = sfd_shrink_info()
    _check(load().sfd_bssh_buffer(m, d, ell, ctypes.c_void_p(rowptr.data_ptr()),
                                  ctypes.c_void_p(colidx.data_ptr()),
                                  ctypes.c_void_p(vals.data_ptr()), seed, b,
                                  ctypes.byref(opts) if opts is not None else None,
                                  ctypes.c_void_p(Bp_out.data_ptr()), ctypes.byref(info)))
    return {f: getattr(info, f) for f, _ in sfd_shrink_info._fields_}


def sfd_dense_shrink(rows, d, ell, M, B_out):
    _check(load().sfd_dense_shrink(rows, d, ell, ctypes.c_void_p(M.data_ptr()),
                                   ctypes.c_void_p(B_out.data_ptr())))


def sfd_csr_spmm(m, d, rowptr, colidx, vals, k, X, ldx, Y, ldy, transpose):
    _check(load().sfd_csr_spmm(m, d, ctypes.c_void_p(rowptr.data_ptr()),
                               ctypes.c_void_p(colidx.data_ptr()), ctypes.c_void_p(vals.data_ptr()),
                               k, ctypes.c_void_p(X.data_ptr()), ldx, ctypes.c_void_p(Y.data_ptr()),
                               ldy, int(transpose)))


def sfd_spmm_variant_count(x_fp16):
    return int(load().sfd_spmm_variant_count(int(bool(x_fp16))))


def sfd_csr_spmm_ex(m, d, rowptr, colidx, vals, k, X, ldx, Y, ldy, transpose, variant):
    """sfd_csr_spmm with the kernel form chosen; X fp16 (torch.float16) or fp32."""
    import torch
    half = X.dtype == torch.float16
    _check(load().sfd_csr_spmm_ex(m, d, ctypes.c_void_p(rowptr.data_ptr()),
                                  ctypes.c_void_p(colidx.data_ptr()),
                                  ctypes.c_void_p(vals.data_ptr()), k,
                                  ctypes.c_void_p(X.data_ptr()), int(half), ldx,
                                  ctypes.c_void_p(Y.data_ptr()), ldy, int(transpose), int(variant)))


def sfd_orthonormalize(rows, k, X, ld):
    _check(load().sfd_orthonormalize(rows, k, ctypes.c_void_p(X.data_ptr()), ld))


def sfd_gram(rows, k, X, ldx, G, precision=0):
    _check(load().sfd_gram(rows, k, ctypes.c_void_p(X.data_ptr()), ldx,
                           ctypes.c_void_p(G.data_ptr()), int(precision)))


def sfd_set_wait_limit(spins):
    """Iteration limit of the tensor-core stages' first waits (< 0: the default;
    0: they give up at once and the stage reports SFD_ETIMEOUT)."""
    _check(load().sfd_set_wait_limit(int(spins)))


def sfd_wait_selftest(spins):
    """Run one bounded wait that nothing ends; returns (status, milliseconds)."""
    ms = ctypes.c_float(0.0)
    rc = load().sfd_wait_selftest(int(spins), ctypes.byref(ms))
    if rc not in (SFD_OK, SFD_ETIMEOUT):
        _check(rc)
    return rc, ms.value


def sfd_gemm_ts(rows, n, X, ldx, T, kout, Y, ldy, precision=0):
    _check(load().sfd_gemm_ts(rows, n, ctypes.c_void_p(X.data_ptr()), ldx,
                              ctypes.c_void_p(T.data_ptr()), kout, ctypes.c_void_p(Y.data_ptr()),
                              ldy, int(precision)))


def sfd_symeig(n, S, nwant, evals, evecs):
    _check(load().sfd_symeig(n, ctypes.c_void_p(S.data_ptr()), nwant,
                             ctypes.c_void_p(evals.data_ptr()), ctypes.c_void_p(evecs.data_ptr())))


def sfd_symeig_noalloc(n, S, nwant, evals, evecs):
    """Same eigensolver, scratch in the library's fixed array (no allocation)."""
    _check(load().sfd_symeig_noalloc(n, ctypes.c_void_p(S.data_ptr()), nwant,
                                     ctypes.c_void_p(evals.data_ptr()),
                                     ctypes.c_void_p(evecs.data_ptr())))


def _f32(a, n=None):
    a = np.ascontiguousarray(a, dtype=np.float32)
    if n is not None and a.size != n:
        raise ValueError("expected %d values, got %d" % (n, a.size))
    return a


def _hptr(a):
    return ctypes.c_void_p(a.ctypes.data) if a.size else None


def q_init_params(seed=0):
    """Initial network parameters: He-scaled normal weights from a seeded
    generator, zero biases, output bias 4 (a middle power count)."""
    rng = np.random.default_rng(seed)
    W1 = rng.standard_normal((QF, 64)) * np.sqrt(2.0 / QF)
    W2 = rng.standard_normal((64, 64)) * np.sqrt(2.0 / 64)
    w3 = rng.standard_normal(64) * np.sqrt(1.0 / 64)
    P = np.concatenate([W1.ravel(), np.zeros(64), W2.ravel(), np.zeros(64), w3, [4.0]])
    return P.astype(np.float32)


def sfd_q_features(m, d, ell, rowptr, colidx, vals, seed, b, q_fixed):
    out = np.empty(QF, dtype=np.float32)
    _check(load().sfd_q_features(m, d, ell, ctypes.c_void_p(rowptr.data_ptr()),
                                 ctypes.c_void_p(colidx.data_ptr()), ctypes.c_void_p(vals.data_ptr()),
                                 seed, b, q_fixed, _hptr(out)))
    return out


def sfd_q_predict(features, params):
    X = _f32(features).reshape(-1, QF)
    P = _f32(params, QPARAMS)
    y = np.empty(len(X), dtype=np.float32)
    _check(load().sfd_q_predict(len(X), _hptr(X), _hptr(P), _hptr(y)))
    return y


def sfd_q_grad(features, targets, params):
    X = _f32(features).reshape(-1, QF)
    T = _f32(targets, len(X))
    P = _f32(params, QPARAMS)
    g = np.empty(QPARAMS, dtype=np.float32)
    loss = ctypes.c_float()
    _check(load().sfd_q_grad(len(X), _hptr(X), _hptr(T), _hptr(P), _hptr(g), ctypes.byref(loss)))
    return float(loss.value), g


def sfd_q_train(features, targets, params, epochs, batch, lr, seed=0):
    """Adam on the squared error; returns (trained parameters, final loss)."""
    X = _f32(features).reshape(-1, QF)
    T = _f32(targets, len(X))
    P = _f32(params, QPARAMS).copy()
    loss = ctypes.c_float()
    _check(load().sfd_q_train(len(X), _hptr(X), _hptr(T), int(epochs), int(batch), float(lr), seed,
                              _hptr(P), ctypes.byref(loss)))
    return P, float(loss.value)


class SFD:
    """Stream object over one context: append rows, read the sketch, merge."""

    def __init__(self, d, ell, seed=0, **opts):
        self.d, self.ell = int(d), int(ell)
        self._opts = options(**opts) if opts else None
        self.ctx = sfd_create(self.d, self.ell, seed, self._opts)

    def append(self, indptr, indices, values):
        sfd_append_rows(self.ctx, indptr, indices, values)

    def sketch(self, out=None):
        if out is None:
            out = np.empty((self.ell, self.d), dtype=np.float32)
        return sfd_sketch(self.ctx, out)

    def merge(self, other):
        sfd_merge(self.ctx, other.ctx)

    def stats(self):
        return sfd_get_stats(self.ctx)

    def save(self):
        """Checkpoint: bytes that sfd_load / SFD.load turn back into this stream."""
        return sfd_save(self.ctx)

    @classmethod
    def load(cls, blob, **runtime):
        """Resume a stream from SFD.save bytes (same d, l, seed, options)."""
        import struct
        d, ell = struct.unpack_from("<qi", blob, 16)
        self = cls.__new__(cls)
        self.d, self.ell = int(d), int(ell)
        self._opts = options(**runtime) if runtime else None
        self.ctx = sfd_load(blob, self._opts)
        return self

    def set_q_model(self, params):
        P = None if params is None else _f32(params, QPARAMS)
        _check(load().sfd_set_q_model(self.ctx, None if P is None else _hptr(P)), self.ctx)

    def q_log(self):
        """(features n x 16, labels n, q_fixed n) logged in q_mode 2."""
        n = ctypes.c_int64()
        _check(load().sfd_q_log(self.ctx, 0, None, None, None, ctypes.byref(n)))
        F = np.empty((n.value, QF), dtype=np.float32)
        lab = np.empty(n.value, dtype=np.float32)
        qf = np.empty(n.value, dtype=np.int32)
        if n.value:
            _check(load().sfd_q_log(self.ctx, n.value, _hptr(F), _hptr(lab), _hptr(qf), ctypes.byref(n)))
        return F, lab, qf

    def reset(self):
        sfd_reset(self.ctx)

    def close(self):
        if self.ctx is not None:
            sfd_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Batch:
    """Independent SFD streams driven concurrently (sfd_batch_*): stream i has
    d[i] columns, l = ell[i] and seed `seed + i`."""

    def __init__(self, d, ell, seed=0, workers=0, **opts):
        self.d = [int(x) for x in d]
        self.ell = [int(x) for x in ell]
        da = np.asarray(self.d, dtype=np.int64)
        ea = np.asarray(self.ell, dtype=np.int32)
        o = options(**opts) if opts else None
        h = ctypes.c_void_p()
        _check(load().sfd_batch_create(len(da), _hptr(da), _hptr(ea), seed,
                                       ctypes.byref(o) if o is not None else None, int(workers),
                                       ctypes.byref(h)))
        self.h = h
        self._keep = []  # device arrays the workers have not read yet

    def append(self, stream, indptr, indices, values):
        pi, w1 = _ptr(indptr, np.int64)
        px, w2 = _ptr(indices, np.int32)
        pv, w3 = _ptr(values, np.float32)
        if not (w1 == w2 == w3):
            raise TypeError("indptr, indices and values must all be host or all device arrays")
        if w1 == SFD_DEVICE:
            self._keep.append((indptr, indices, values))
        _check(load().sfd_batch_append(self.h, int(stream), len(indptr) - 1, pi, px, pv, w1))

    def wait(self):
        try:
            _check(load().sfd_batch_wait(self.h))
        finally:
            self._keep.clear()

    def sketch(self, stream, out=None):
        if out is None:
            out = np.empty((self.ell[stream], self.d[stream]), dtype=np.float32)
        p, w = _ptr(out, np.float32)
        try:
            _check(load().sfd_batch_sketch(self.h, int(stream), p, w))
        finally:
            self._keep.clear()
        return out

    def merge_tree(self, out=None):
        if out is None:
            out = np.empty((self.ell[0], self.d[0]), dtype=np.float32)
        p, w = _ptr(out, np.float32)
        try:
            _check(load().sfd_batch_merge_tree(self.h, p, w))
        finally:
            self._keep.clear()
        return out

    def stats(self, stream):
        s = sfd_stats()
        _check(load().sfd_batch_stats(self.h, int(stream), ctypes.byref(s)))
        return {f: getattr(s, f) for f, _ in sfd_stats._fields_}

    def close(self):
        if self.h is not None:
            load().sfd_batch_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
