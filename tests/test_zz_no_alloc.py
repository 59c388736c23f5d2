"""sfd_symeig_noalloc: the eigensolver entry point that allocates nothing.

It exists for callers that cannot let a library allocate device memory (a
process whose caching allocator already holds the memory budget, or a
latency-critical loop that cannot take cudaMalloc's synchronisation). Its
output must match the allocating entry point sfd_symeig on the same input, on
two calls in a row (the second call finds the first call's data in the shared
scratch array), and an FP64 eigensolve of the same matrix; after the first
call on the device, further calls must leave the device's free memory
unchanged. This file is collected last on purpose.
"""
import numpy as np
import pytest

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


def _matrix(seed, n):
    rng = np.random.default_rng(seed)
    M = rng.standard_normal((n, 3 * n)) * (0.95 ** np.arange(n))[:, None]
    return (M @ M.T).astype(np.float32)


@pytest.mark.parametrize("n,nwant", [(100, 100), (200, 100), (256, 128), (256, 256), (7, 3)])
def test_noalloc_matches_allocating_entry_point(lib, n, nwant):
    for call, seed in enumerate((n, n + 1)):          # two calls in a row
        Sf = _matrix(seed, n)
        S = torch.from_numpy(Sf).cuda()
        ev_a = torch.zeros(nwant, device="cuda")
        V_a = torch.zeros((n, nwant), device="cuda")
        ev_b = torch.full((nwant,), 7.0, device="cuda")
        V_b = torch.full((n, nwant), 7.0, device="cuda")
        lib.sfd_symeig(n, S, nwant, ev_a, V_a)
        lib.sfd_symeig_noalloc(n, S, nwant, ev_b, V_b)
        wa, wb = ev_a.cpu().numpy().astype(np.float64), ev_b.cpu().numpy().astype(np.float64)
        Va, Vb = V_a.cpu().numpy().astype(np.float64), V_b.cpu().numpy().astype(np.float64)
        # the FP64 eigenvalues of the same (fp32) matrix
        w64 = np.linalg.eigvalsh(Sf.astype(np.float64))[::-1][:nwant]
        nrm = float(np.abs(w64).max())
        tol = 2e-5 * nrm * max(1, np.sqrt(n) / 4)          # the eigensolver tests' bound
        assert np.all(np.abs(wa - wb) <= tol), call
        assert np.all(np.abs(wb - w64) <= tol), (call, np.abs(wb - w64).max() / nrm)
        # same eigenvectors up to sign, and each an eigenvector of S to fp32 accuracy
        dots = np.abs(np.sum(Va * Vb, axis=0))
        assert np.all(dots > 1 - 1e-4), (call, dots.min())
        R = Sf.astype(np.float64) @ Vb - Vb * wb
        assert np.linalg.norm(R, axis=0).max() <= 1e-4 * nrm * max(1, np.sqrt(n) / 4)
        assert np.linalg.norm(Vb.T @ Vb - np.eye(nwant)) <= 1e-3 * max(1, nwant / 16)


def test_noalloc_leaves_free_memory_unchanged(lib):
    n, nwant = 256, 200
    S = torch.from_numpy(_matrix(3, n)).cuda()
    ev = torch.zeros(nwant, device="cuda")
    V = torch.zeros((n, nwant), device="cuda")
    lib.sfd_symeig_noalloc(n, S, nwant, ev, V)       # warm-up: the array is in place from here on
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    for _ in range(3):
        lib.sfd_symeig_noalloc(n, S, nwant, ev, V)
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert free1 == free0, (free0, free1)


def test_noalloc_rejects_sizes_beyond_its_array(lib):
    S = torch.zeros((257, 257), device="cuda")
    ev = torch.zeros(257, device="cuda")
    V = torch.zeros((257, 257), device="cuda")
    with pytest.raises(lib.SfdError) as ei:
        lib.sfd_symeig_noalloc(257, S, 10, ev, V)
    assert ei.value.code == lib.SFD_EINVAL
