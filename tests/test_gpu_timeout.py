"""Failure detection of the bounded device waits, without a GPU fault.

Every tensor-core stage (the Gram, X T and cross-Gram products of Alg. 1,
Alg. 3 and Alg. 5) waits on mbarriers for its copies and its MMAs, and each
wait gives up after an iteration limit. Here the limit is made to run out on
purpose, with nothing broken:

  - a wait that nothing ends (an mbarrier no thread or copy arrives at) gives
    up after its limit, in bounded time, and reports SFD_ETIMEOUT;
  - with the first-wait limit at 0, the real stages give up at their first
    wait, drain the copies and MMAs they started, and report SFD_ETIMEOUT:
    through sfd_gram and sfd_gemm_ts (both tensor-core forms, both staging
    paths of the Gram) and through a stream (sfd_append_rows / sfd_sketch);
  - once the limit is restored, the same calls and a new stream give the
    correct results, bit for bit where the path is deterministic: the stage
    that gave up left nothing running.
"""
import numpy as np
import pytest

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


@pytest.fixture(autouse=True)
def default_limit(lib):
    yield
    torch.cuda.synchronize()
    lib.sfd_set_wait_limit(-1)


def test_a_wait_that_nothing_ends_gives_up(lib):
    times = {}
    for spins in (0, 1, 1000, 100000):
        rc, ms = lib.sfd_wait_selftest(spins)
        assert rc == lib.SFD_ETIMEOUT, spins
        assert ms < 5000.0, (spins, ms)
        times[spins] = ms
    # the default limit (2^18 tries) bounds a wait at about (2^18 / 1e5) times
    # the last figure; run it too when that stays within a few seconds
    est = times[100000] * (2 ** 18) / 1e5
    print("wait self-test: %s ms; default limit about %.0f ms" % (times, est))
    if est < 5000.0:
        rc, ms = lib.sfd_wait_selftest(-1)
        assert rc == lib.SFD_ETIMEOUT and ms < 10000.0
    # the context is still usable
    x = torch.arange(1000, device="cuda", dtype=torch.float32)
    assert float(x.sum()) == 499500.0


def _gram_ref(X, k):
    Xd = X.double().cpu().numpy()[:, :k]
    return Xd.T @ Xd


@pytest.mark.parametrize("precision", [1, 2])
@pytest.mark.parametrize("ldx", [104, 101])   # bulk-copy staging / per-element staging
def test_gram_gives_up_then_recovers(lib, precision, ldx):
    rows, k = 50000, 100
    g = torch.Generator(device="cpu").manual_seed(precision * 1000 + ldx)
    X = torch.zeros((rows, ldx), dtype=torch.float32)
    X[:, :k] = torch.randn((rows, k), generator=g)
    X = X.cuda()
    G = torch.full((k, k), 7.0, device="cuda")
    lib.sfd_set_wait_limit(0)
    with pytest.raises(lib.SfdError) as ei:
        lib.sfd_gram(rows, k, X, ldx, G, precision)
    assert ei.value.code == lib.SFD_ETIMEOUT
    lib.sfd_set_wait_limit(-1)
    lib.sfd_gram(rows, k, X, ldx, G, precision)
    ref = _gram_ref(X, k)
    err = np.linalg.norm(G.double().cpu().numpy() - ref) / np.linalg.norm(ref)
    assert err < (2e-3 if precision == 1 else 1e-5), err


@pytest.mark.parametrize("precision", [1, 2])
def test_gemm_gives_up_then_recovers(lib, precision):
    rows, n, kout, ld = 50000, 100, 100, 104
    g = torch.Generator(device="cpu").manual_seed(7 + precision)
    X = torch.zeros((rows, ld), dtype=torch.float32)
    X[:, :n] = torch.randn((rows, n), generator=g)
    T = torch.randn((n, kout), generator=g)
    X, T = X.cuda(), T.cuda()
    Y = torch.zeros((rows, ld), device="cuda")
    lib.sfd_set_wait_limit(0)
    with pytest.raises(lib.SfdError) as ei:
        lib.sfd_gemm_ts(rows, n, X, ld, T, kout, Y, ld, precision)
    assert ei.value.code == lib.SFD_ETIMEOUT
    lib.sfd_set_wait_limit(-1)
    lib.sfd_gemm_ts(rows, n, X, ld, T, kout, Y, ld, precision)
    ref = X.double().cpu().numpy()[:, :n] @ T.double().cpu().numpy()
    got = Y.double().cpu().numpy()[:, :kout]
    err = np.linalg.norm(got - ref) / np.linalg.norm(ref)
    assert err < (2e-3 if precision == 1 else 1e-5), err


def _stream_sketch(lib, X, d, ell, seed):
    s = lib.SFD(d, ell, seed, precision=1)
    try:
        s.append(X.indptr, X.indices, X.values)
        return s.sketch()
    finally:
        s.close()


def test_stream_gives_up_then_a_new_stream_is_exact(lib):
    d, ell, seed = 2000, 50, 3
    X = synth.c1(seed=seed, n=6000)    # three buffers close, the last one is flushed
    ref = _stream_sketch(lib, X, d, ell, seed)
    lib.sfd_set_wait_limit(0)
    s = lib.SFD(d, ell, seed, precision=1)
    codes = []
    try:
        try:
            s.append(X.indptr, X.indices, X.values)
            s.sketch()
        except lib.SfdError as e:
            codes.append(e.code)
    finally:
        torch.cuda.synchronize()
        s.close()
    assert codes == [lib.SFD_ETIMEOUT]
    lib.sfd_set_wait_limit(-1)
    again = _stream_sketch(lib, X, d, ell, seed)
    assert np.array_equal(again, ref)
