"""The C-ABI library builds, loads and exports every function include/sfd.h
declares; argument checks that need no GPU reject bad input."""
import os
import re

import pytest

from paper_1602_00412_gb300 import build as B
from paper_1602_00412_gb300 import sfd

HEADER = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "include", "sfd.h")


@pytest.fixture(scope="module")
def lib():
    B.build()
    return sfd.load()


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(sfd_[a-z_]+)\s*\(", text)))


def test_every_declared_symbol_is_exported(lib):
    names = declared_functions()
    assert len(names) >= 10
    for n in names:
        assert hasattr(lib, n), n
    assert sorted(sfd.EXPORTS) == names


def test_status_strings(lib):
    assert sfd._strerror(0) == "ok"
    assert "invalid" in sfd._strerror(1)
    assert sfd._strerror(99) == "unknown status"


def test_options_defaults(lib):
    o = sfd.options()
    assert o.abi_version == sfd.SFD_ABI_VERSION
    assert (o.delta, o.verify, o.c_q, o.q_override, o.retry_cap) == (0.01, 1, 0.25, -1, 8)
    assert o.cuda_stream is None
    assert (o.precision, o.q_mode, o.slots) == (0, 0, 0)
    assert o.q_margin == 1.0 and abs(o.q_tau - 1e-2) < 1e-9 and o.autotune == 1


def test_create_rejects_bad_shapes_without_gpu(lib):
    import ctypes
    h = ctypes.c_void_p()
    for d, ell in [(0, 1), (10, 0), (10, 11), (1000, 257)]:
        assert lib.sfd_create(d, ell, 0, None, ctypes.byref(h)) == sfd.SFD_EINVAL
    bad = sfd.options()
    bad.abi_version = 99
    assert lib.sfd_create(100, 10, 0, ctypes.byref(bad), ctypes.byref(h)) == sfd.SFD_EINVAL


def test_null_context_is_rejected(lib):
    assert lib.sfd_append_rows(None, 1, None, None, None, 0) == sfd.SFD_EINVAL
    assert lib.sfd_sketch(None, None, 0) == sfd.SFD_EINVAL
    assert lib.sfd_merge(None, None) == sfd.SFD_EINVAL
    lib.sfd_destroy(None)


def test_dense_product_forms_rejected_without_gpu(lib):
    # argument checks that return before any CUDA call
    assert lib.sfd_gram(10, 8, None, 8, None, 0) == sfd.SFD_EINVAL          # G null
    p = 1  # a non-null dummy address: the checks below reject before using it
    assert lib.sfd_gram(10, 8, p, 8, p, 3) == sfd.SFD_EINVAL               # no form 3
    assert lib.sfd_gram(10, 136, p, 136, p, 2) == sfd.SFD_EINVAL           # tensor cores: k <= 128
    assert lib.sfd_gemm_ts(10, 120, p, 120, p, 120, p, 120, 2) == sfd.SFD_EINVAL  # split: <= 112
    assert lib.sfd_gemm_ts(10, 8, p, 4, p, 8, p, 8, 0) == sfd.SFD_EINVAL   # ldx < n


def test_spmm_forms_without_gpu(lib):
    assert lib.sfd_spmm_variant_count(0) == 2
    assert lib.sfd_spmm_variant_count(1) == 3
    p = 1
    # variant out of range, fp16 needs k <= 128 and ld % 8 == 0
    assert lib.sfd_csr_spmm_ex(4, 4, p, p, p, 4, p, 0, 4, p, 4, 0, 2) == sfd.SFD_EINVAL
    assert lib.sfd_csr_spmm_ex(4, 4, p, p, p, 4, p, 1, 4, p, 4, 0, 0) == sfd.SFD_EINVAL
    assert lib.sfd_csr_spmm_ex(4, 4, p, p, p, 136, p, 1, 136, p, 136, 0, 0) == sfd.SFD_EINVAL
    assert lib.sfd_csr_spmm_ex(4, 4, p, p, p, 4, p, 0, 4, p, 4, 0, -1) == sfd.SFD_EINVAL
