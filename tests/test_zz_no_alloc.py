"""sfd_symeig_noalloc: the eigensolver entry point that allocates nothing.

It exists for callers that cannot let a library allocate device memory (a
process whose caching allocator already holds the memory budget, or a
latency-critical loop that cannot take cudaMalloc's synchronisation). Its
output must match the allocating entry point sfd_symeig on the same input, on
two calls in a row (the second call finds the first call's data in the shared
scratch array). This file is collected last on purpose.
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


@pytest.mark.parametrize("n,nwant", [(100, 100), (200, 100), (256, 128), (7, 3)])
def test_noalloc_matches_allocating_entry_point(lib, n, nwant):
    for call, seed in enumerate((n, n + 1)):          # two calls in a row
        S = torch.from_numpy(_matrix(seed, n)).cuda()
        ev_a = torch.zeros(nwant, device="cuda")
        V_a = torch.zeros((n, nwant), device="cuda")
        ev_b = torch.full((nwant,), 7.0, device="cuda")
        V_b = torch.full((n, nwant), 7.0, device="cuda")
        lib.sfd_symeig(n, S, nwant, ev_a, V_a)
        lib.sfd_symeig_noalloc(n, S, nwant, ev_b, V_b)
        wa, wb = ev_a.cpu().numpy(), ev_b.cpu().numpy()
        Va, Vb = V_a.cpu().numpy().astype(np.float64), V_b.cpu().numpy().astype(np.float64)
        nrm = float(np.abs(wa).max())
        # the tolerance of the eigensolver tests
        assert np.all(np.abs(wa - wb) <= 2e-5 * nrm * max(1, np.sqrt(n) / 4)), call
        # same eigenvectors up to sign
        dots = np.abs(np.sum(Va * Vb, axis=0))
        assert np.all(dots > 1 - 1e-4), (call, dots.min())


def test_noalloc_rejects_sizes_beyond_its_array(lib):
    S = torch.zeros((257, 257), device="cuda")
    ev = torch.zeros(257, device="cuda")
    V = torch.zeros((257, 257), device="cuda")
    with pytest.raises(lib.SfdError) as ei:
        lib.sfd_symeig_noalloc(257, S, 10, ev, V)
    assert ei.value.code == lib.SFD_EINVAL
