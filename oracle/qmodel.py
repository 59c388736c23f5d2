"""Learned power count q of SimultaneousIteration, in float64 on the CPU.

Test infrastructure only: imported by tests/, by the smoke check and by the
baseline leg of bench.py, never by the CUDA path.

Sec. 3.2 fixes q only up to a constant, q = Theta(log(n/eps)/eps) (Alg. 1,
called with eps = 1/4 by Alg. 3), and BoostedSparseShrink (Alg. 4) checks each
result with VerifySpectral (Alg. 6), so a buffer run with a smaller q that
still passes the check keeps the guarantee of Theorem 4.1. The learned form
predicts q per buffer from 16 numbers that are known before the power loop
starts, with a 16 -> 64 -> 64 -> 1 ReLU network. This module defines, for the
CUDA path to be checked against:

  buffer_features     the 16 inputs (statistics of A' and of S0 = (A'G)^T A'G)
  ladder, label       the training label of a buffer
  mlp_forward / mlp_backward / mse_loss / adam_step
                      the network, its gradient (hand-derived backpropagation)
                      and Adam (Kingma & Ba 2015, Algorithm 1)
"""
import math

import numpy as np

from . import philox

NF = 16          # features (feature 0 is the constant 1)
NH = 64          # hidden width of both hidden layers
# parameter vector layout (float32 on the device, float64 here)
SIZES = (("W1", (NF, NH)), ("b1", (NH,)), ("W2", (NH, NH)), ("b2", (NH,)), ("w3", (NH,)),
         ("b3", (1,)))
NPARAM = sum(int(np.prod(s)) for _, s in SIZES)   # 5313
LADDER = (1, 2, 3, 4, 6, 8, 11, 16, 23, 32, 45, 64)
ADAM_B1, ADAM_B2, ADAM_EPS = 0.9, 0.999, 1e-8


def unpack(theta):
    """Views W1 (16 x 64, input-major), b1, W2 (64 x 64), b2, w3 (64), b3 (1)."""
    theta = np.asarray(theta)
    out, o = {}, 0
    for name, shape in SIZES:
        k = int(np.prod(shape))
        out[name] = theta[o:o + k].reshape(shape)
        o += k
    return out


def init_params(seed):
    """He-style initial weights from a seeded generator (biases 0, b3 = 4)."""
    rng = np.random.default_rng(seed)
    theta = np.zeros(NPARAM)
    p = unpack(theta)
    p["W1"][...] = rng.standard_normal((NF, NH)) * math.sqrt(2.0 / NF)
    p["W2"][...] = rng.standard_normal((NH, NH)) * math.sqrt(2.0 / NH)
    p["w3"][...] = rng.standard_normal(NH) * math.sqrt(1.0 / NH)
    p["b3"][...] = 4.0
    return theta


# ---------------------------------------------------------------- features
def buffer_features(indptr, indices, values, d, ell, S0, q_fixed):
    """The 16 inputs for a buffer A' (CSR, m x d) whose first product
    Y0 = A' G has Gram S0 = Y0^T Y0 (l x l):

      0  1
      1  ln m / 10                 2  ln N / 20 (N = nnz)
      3  ln d / 15                 4  l / 256
      5  ln(N / m) / 5             6  ln(||A'||_F^2 / N) / 10
      7  max_i ||a_i||^2 / ||A'||_F^2            (row energy concentration)
      8  max_j c_j / N             9  sum_j c_j^2 / N^2   (c_j: column counts)
     10  m sum_i r_i^2 / N^2 - 1                  (r_i: row counts)
     11  ln q_fixed / 3
     12  ||S0||_F^2 / tr(S0)^2     13  max_j S0_jj / tr(S0)
     14  ln(1 + N / (m l))        15  1 - (nonempty columns) / d
    Empty or all-zero quantities give 0 for the terms they would divide by."""
    indptr = np.asarray(indptr, dtype=np.int64)
    indices = np.asarray(indices, dtype=np.int64)
    v = np.asarray(values, dtype=np.float64)
    base = int(indptr[0])
    m = len(indptr) - 1
    N = int(indptr[-1] - base)
    rows = np.diff(indptr)
    f = np.zeros(NF)
    f[0] = 1.0
    f[1] = math.log(m) / 10.0 if m > 0 else 0.0
    f[2] = math.log(N) / 20.0 if N > 0 else 0.0
    f[3] = math.log(d) / 15.0
    f[4] = ell / 256.0
    if N > 0:
        seg = v[base:base + N]
        idx = indices[base:base + N]
        fro2 = float(np.dot(seg, seg))
        rowsq = np.bincount(np.repeat(np.arange(m), rows), weights=seg * seg, minlength=m)
        c = np.bincount(idx, minlength=d).astype(np.float64)
        f[5] = math.log(N / m) / 5.0
        f[6] = math.log(fro2 / N) / 10.0 if fro2 > 0 else 0.0
        f[7] = float(rowsq.max()) / fro2 if fro2 > 0 else 0.0
        f[8] = float(c.max()) / N
        f[9] = float(np.dot(c, c)) / (float(N) * N)
        f[10] = m * float(np.dot(rows.astype(np.float64), rows)) / (float(N) * N) - 1.0
        f[14] = math.log(1.0 + N / (m * ell))
        f[15] = 1.0 - float(np.count_nonzero(c)) / d
    else:
        f[15] = 1.0
    f[11] = math.log(q_fixed) / 3.0
    S0 = np.asarray(S0, dtype=np.float64)
    tr = float(np.trace(S0))
    if tr > 0:
        f[12] = float((S0 * S0).sum()) / (tr * tr)
        f[13] = float(np.diag(S0).max()) / tr
    return f


def first_gram(A, seed, b, ell):
    """S0 = (A' G)^T (A' G) for the G of attempt 0 of buffer b (Alg. 1's start
    block, drawn as in Alg. 4)."""
    d = A.shape[1]
    Y = A @ philox.gaussian_G(seed, b, 0, d, ell)
    return np.asarray(Y.T @ Y)


# ------------------------------------------------------------------ labels
def ladder(q_fixed):
    """The q values tried for a label: LADDER entries below q_fixed, then q_fixed."""
    return [q for q in LADDER if q < q_fixed] + [q_fixed]


def label(qs, energies, oks, tau):
    """Smallest q of the ladder whose run passed VerifySpectral and kept the
    captured energy ||P||_F^2 = ||Z^T A'||_F^2 within a fraction tau of the
    run at the largest q (the last entry); that q if none does."""
    e_ref = energies[-1]
    for q, e, ok in zip(qs, energies, oks):
        if ok and e >= (1.0 - tau) * e_ref:
            return q
    return qs[-1]


# ---------------------------------------------------------------- network
def mlp_forward(theta, X):
    """X: B x 16 -> (y (B), cache). h1 = relu(X W1 + b1), h2 = relu(h1 W2 + b2),
    y = h2 w3 + b3."""
    p = unpack(theta)
    X = np.asarray(X, dtype=np.float64)
    z1 = X @ p["W1"] + p["b1"]
    h1 = np.maximum(z1, 0.0)
    z2 = h1 @ p["W2"] + p["b2"]
    h2 = np.maximum(z2, 0.0)
    y = h2 @ p["w3"] + p["b3"][0]
    return y, (X, z1, h1, z2, h2)


def mse_loss(y, t):
    """L = (1 / 2B) sum (y - t)^2."""
    r = np.asarray(y, dtype=np.float64) - np.asarray(t, dtype=np.float64)
    return 0.5 * float(np.dot(r, r)) / len(r)


def mlp_backward(theta, X, t):
    """Gradient of mse_loss(mlp_forward(theta, X), t) with respect to theta,
    by the chain rule layer by layer. Returns (loss, grad)."""
    p = unpack(theta)
    y, (X, z1, h1, z2, h2) = mlp_forward(theta, X)
    B = len(y)
    dy = (y - np.asarray(t, dtype=np.float64)) / B
    g = np.zeros(NPARAM)
    gp = unpack(g)
    gp["w3"][...] = h2.T @ dy
    gp["b3"][...] = dy.sum()
    dz2 = np.outer(dy, p["w3"]) * (z2 > 0)
    gp["W2"][...] = h1.T @ dz2
    gp["b2"][...] = dz2.sum(axis=0)
    dz1 = (dz2 @ p["W2"].T) * (z1 > 0)
    gp["W1"][...] = X.T @ dz1
    gp["b1"][...] = dz1.sum(axis=0)
    return mse_loss(y, t), g


def adam_step(theta, grad, m, v, step, lr):
    """One Adam update (step counts from 1). Returns (theta, m, v)."""
    m = ADAM_B1 * m + (1.0 - ADAM_B1) * grad
    v = ADAM_B2 * v + (1.0 - ADAM_B2) * grad * grad
    mhat = m / (1.0 - ADAM_B1 ** step)
    vhat = v / (1.0 - ADAM_B2 ** step)
    return theta - lr * mhat / (np.sqrt(vhat) + ADAM_EPS), m, v


def predict_q(theta, f, q_fixed, margin=1.0):
    """q = ceil(prediction + margin), clamped to [1, q_fixed]."""
    y, _ = mlp_forward(theta, np.asarray(f)[None, :])
    return int(min(q_fixed, max(1, math.ceil(float(y[0]) + margin))))
