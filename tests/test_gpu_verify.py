"""GPU VerifySpectral (Alg. 6) and BoostedSparseShrink (Alg. 4) against the
FP64 oracle, through the C ABI:

  - the power-step count p of every (buffer b, attempt r) key equals the
    oracle's schedule (Lemma 4.1's constant, keyed delta_{b,r});
  - the log-sum log ||C^p x|| of the GPU equals the oracle's VerifySpectral run
    on the GPU's own B' (the same C, the same Philox x) to the FP32 resolution
    of the residual;
  - natural rejections (no injection): with q = 0 on a spectrum with a step at
    l, SimultaneousIteration misses the l-th direction in some runs; the GPU
    makes the same accept / reject decisions and the same number of attempts
    as the oracle under the same Philox keys;
  - SparseShrink without VerifySpectral (verify = 0, the mode of the paper's
    experiments in Sec. 5) matches the oracle's verify=False stream at the
    1e-4 parity bar, and equals the verified sketch bit for bit when
    VerifySpectral rejects nothing.
"""
import numpy as np
import pytest
import scipy.sparse as sp

from oracle import metrics, philox
from oracle import sfd as O
from paper_1602_00412_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

U32 = 2.0 ** -24


@pytest.fixture(scope="module")
def lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__ as g
    g.build()
    from paper_1602_00412_gb300 import sfd
    return sfd


def dev(a, dtype):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=dtype)).cuda()


def _bssh(lib, A, ell, seed, b, **opts):
    A = sp.csr_matrix(A)
    m, d = A.shape
    Bp = torch.zeros((ell, d), device="cuda")
    info = lib.sfd_bssh_buffer(m, d, ell, dev(A.indptr, np.int32), dev(A.indices, np.int32),
                               dev(A.data, np.float32), seed, b, Bp, lib.options(**opts))
    return Bp.cpu().numpy().astype(np.float64), info


def _step_spectrum_matrix(m=250, d=300, seed=0):
    """19 directions at sigma 10, one at 4, 100 at 0.3 (l = 20): with q = 0,
    Z often misses the sigma-4 direction and VerifySpectral rejects."""
    rng = np.random.default_rng(seed)
    spec = np.concatenate([np.full(19, 10.0), [4.0], np.full(100, 0.3)])
    U, _ = np.linalg.qr(rng.standard_normal((m, spec.size)))
    V, _ = np.linalg.qr(rng.standard_normal((d, spec.size)))
    return sp.csr_matrix(((U * spec) @ V.T).astype(np.float32).astype(np.float64))


def _logsum_tol(info, p):
    # one power step forms C x = (A'^T A' x - B'^T B' x) / (Delta / 2): a
    # difference of terms up to ||A'||_F^2 scaled by 2 / Delta, so its fp32
    # relative error is a few units of 2^-24 ||A'||_F^2 / (Delta / 2); the
    # log-sum adds p such steps (64 units per step, the constant of the
    # resolution guard of VerifySpectral)
    kappa = info["fro2_a"] / (info["delta_shrink"] / 2.0)
    return p * 64.0 * U32 * kappa


@pytest.mark.parametrize("kind", ["gapped", "c1", "step"])
@pytest.mark.parametrize("b,r", [(0, 0), (3, 0), (17, 2)])
def test_vs_steps_and_logsum_match_oracle(lib, kind, b, r):
    seed = 5
    if kind == "step":
        A, ell, q = _step_spectrum_matrix(seed=b), 20, 0
    else:
        X = (synth.c1_gapped if kind == "gapped" else synth.c1)(seed=seed, n=2000)
        A, ell, q = X.to_scipy(), 50, None
    m, d = A.shape
    opts = {"inject_vs_fail": r, "retry_cap": r + 1}
    if q is not None:
        opts["q_override"] = q
    Bp, info = _bssh(lib, A, ell, seed, b, **opts)
    p = O.vs_steps(d, O.delta_br(0.01, b, r))
    assert info["vs_steps"] == p                 # keyed schedule of Lemma 4.1
    assert info["attempts"] == r + 1
    # the oracle's VerifySpectral on the GPU's B' with the GPU's Delta
    Delta = info["delta_shrink"]
    assert Delta / 2.0 > O.VS_RESOLUTION * info["fro2_a"]
    ok, ls = O.verify_spectral(O.residual_operator(A, Bp, Delta), philox.sphere_x(seed, b, r, d), p)
    tol = _logsum_tol(info, p)
    assert tol < 0.05 * abs(ls) + 0.05          # the bound is not vacuous
    assert abs(info["logsum"] - ls) <= tol, (info["logsum"], ls, tol)
    if abs(ls) > tol:
        # the first r attempts were forced False on the host; the last is VS's own
        assert bool(info["verified"]) == ok


def test_natural_rejections_match_oracle(lib):
    # no injection: q = 0 makes SimultaneousIteration miss the l-th direction in
    # some runs; per seed, the GPU's attempts and final verdict equal the
    # oracle's (same Philox keys), skipping seeds with a log-sum near 0
    A = _step_spectrum_matrix()
    d, ell = A.shape[1], 20
    compared = rejected = 0
    for seed in range(12):
        _, rinfo = O.boosted_sparse_shrink(A, ell, 0.01, seed, 0, 0)
        if any(abs(h["logsum"]) < 1.0 for h in rinfo["history"]):
            continue
        _, info = _bssh(lib, A, ell, seed, 0, q_override=0)
        assert info["attempts"] == rinfo["attempts"], seed
        assert bool(info["verified"]) == rinfo["verified"], seed
        compared += 1
        rejected += rinfo["attempts"] - 1
    assert compared >= 6 and rejected >= 3, (compared, rejected)


def _step_stream(nbuf, seed, d=2400, r=120, ell=20):
    """A stream of nbuf buffers (d rows each, 20 entries per row) whose every
    buffer has singular values exactly 19 x 10, one 6 and 100 x 0.3: row i of a
    buffer is a multiple of prototype t = i mod r (unit rows V_t on disjoint
    column sets, so orthonormal), the multiples of each prototype normalised
    within the buffer."""
    rng = np.random.default_rng(seed)
    spec = np.concatenate([np.full(ell - 1, 10.0), [6.0], np.full(r - ell, 0.3)])
    supp = d // r
    perm = rng.permutation(d)
    V = np.zeros((r, d))
    for t in range(r):
        v = rng.standard_normal(supp)
        V[t, perm[t * supp:(t + 1) * supp]] = v / np.linalg.norm(v)
    t_i = np.tile(np.arange(r), d // r)
    blocks = []
    for _ in range(nbuf):
        g = rng.standard_normal(d)
        for t in range(r):
            g[t_i == t] /= np.linalg.norm(g[t_i == t])
        blocks.append((g * spec[t_i])[:, None] * V[t_i])
    A = sp.csr_matrix(np.vstack(blocks).astype(np.float32))
    A.sort_indices()
    return A


def test_stream_rejections_without_injection(lib):
    # SimultaneousIteration with q = 0 misses the l-th direction of these
    # buffers in most attempts; BoostedSparseShrink retries each buffer with
    # the next Philox key until VerifySpectral accepts. The GPU stream's
    # attempts and rejections equal the oracle's on the same keys (compared
    # when no oracle log-sum lies within 0.5 of the decision threshold 0)
    d, ell, seed, nbuf = 2400, 20, 3, 4
    A = _step_stream(nbuf, 0)
    hist = []
    for b in range(nbuf):
        _, info = O.boosted_sparse_shrink(A[b * d:(b + 1) * d], ell, 0.01, seed, b, 0)
        hist.append(info)
    margin = min(abs(h["logsum"]) for info in hist for h in info["history"])
    want_attempts = sum(info["attempts"] for info in hist)
    s = lib.SFD(d, ell, seed, q_override=0)
    s.append(A.indptr.astype(np.int64), A.indices.astype(np.int32), A.data.astype(np.float32))
    B = s.sketch().astype(np.float64)
    st = s.stats()
    s.close()
    assert st["buffers"] == nbuf
    assert st["vs_rejects"] == st["attempts"] - (nbuf - st["unverified"])
    assert st["vs_rejects"] > 0                      # no injection anywhere
    if margin > 0.5:
        assert st["attempts"] == want_attempts, (st["attempts"], want_attempts)
        assert st["unverified"] == sum(not info["verified"] for info in hist)
    ref, o = O.sfd_stream(A.indptr, A.indices, A.data, d, ell, seed, q_override=0)
    assert [e["attempts"] for e in o.log] == [info["attempts"] for info in hist]
    Ad = A.astype(np.float64)
    assert metrics.cov_norm(Ad, B) <= metrics.fd_bound(Ad, ell, 10)


@pytest.mark.parametrize("precision", [0, 1])
def test_verify_off_matches_oracle(lib, precision):
    d, ell, k, seed = 2000, 50, 10, 0
    X = synth.c1_gapped(seed=seed, n=8000)
    s = lib.SFD(d, ell, seed, verify=0, precision=precision)
    s.append(X.indptr, X.indices, X.values)
    B = s.sketch().astype(np.float64)
    st = s.stats()
    s.close()
    ref, o = O.sfd_stream(X.indptr, X.indices, X.values, d, ell, seed, verify=False)
    assert st["buffers"] == len(o.log) and st["attempts"] == st["buffers"]
    assert st["vs_rejects"] == 0
    rel = metrics.bbt_rel_diff(B, ref)
    assert rel <= (1e-4 if precision == 0 else 1e-3), rel
    A = X.to_scipy()
    assert metrics.cov_norm(A, B) <= metrics.fd_bound(A, ell, k)
    # VerifySpectral only judges B'; when it accepts every buffer, the verified
    # stream's sketch is the same bits
    s2 = lib.SFD(d, ell, seed, verify=1, precision=precision)
    s2.append(X.indptr, X.indices, X.values)
    B2 = s2.sketch().astype(np.float64)
    st2 = s2.stats()
    s2.close()
    if st2["vs_rejects"] == 0:
        assert np.array_equal(B, B2)
