"""CPU oracle of the learned first-pass bound -- TEST INFRASTRUCTURE ONLY.

Only ``tests/``, ``__graft_entry__.smoke()`` and bench.py's CPU legs may use this
module; the CUDA library never does, and the two share no code.

The paper has no learned part: FastSearch (Sec. 2.2) grows a release horizon
until every register is filled.  The library replaces the horizon of the first
pass by a per-row prediction of ln y* (y* = the largest register) from a small
network; any horizon gives the same registers, so the network only decides the
work.  This module states, plainly and in FP64, what the library's model
kernels compute:

* ``features``   -- the 8 row features;
* ``forward``    -- the 8 -> 64 -> 64 -> 1 GELU network and its ln y* output;
* ``loss_and_grad`` -- mean pinball loss and its exact gradient (backprop);
* ``adam_step``  -- one Adam update (Kingma & Ba, 2015, Algorithm 1).

Parameters are one flat vector: W1[64][8], b1[64], W2[64][64], b2[64], w3[64], b3.
"""
import math

import numpy as np

F, H = 8, 64
P = H * F + H + H * H + H + H + 1
PCT = (10, 50, 90, 99)
BIN_MIN, BIN_MAX = -512, 511


def unpack(theta):
    """Split the flat parameter vector into (W1, b1, W2, b2, w3, b3)."""
    theta = np.asarray(theta, dtype=np.float64)
    assert theta.shape == (P,)
    o = 0
    W1 = theta[o:o + H * F].reshape(H, F); o += H * F
    b1 = theta[o:o + H]; o += H
    W2 = theta[o:o + H * H].reshape(H, H); o += H * H
    b2 = theta[o:o + H]; o += H
    w3 = theta[o:o + H]; o += H
    b3 = theta[o]
    return W1, b1, W2, b2, w3, b3


def pack(W1, b1, W2, b2, w3, b3):
    return np.concatenate([np.ravel(W1), b1, np.ravel(W2), b2, w3, [b3]]).astype(np.float64)


# --- features -----------------------------------------------------------------

def weight_bin(v):
    """floor(4 log2 v) for a positive finite double, the quarter-octave points
    2^(j/4) (j = 1, 2, 3) taken as the doubles nearest to them; clamped to
    [-512, 511].  Subnormal weights fall in the lowest bin."""
    v = float(v)
    if v < 2.0 ** -1022:
        return BIN_MIN
    m, e = math.frexp(v)          # v = m 2^e, m in [1/2, 1)
    sig, e = 2.0 * m, e - 1       # v = sig 2^e, sig in [1, 2), exact
    b = 4 * e + sum(1 for j in (1, 2, 3) if sig >= 2.0 ** (j / 4.0))
    return min(max(b, BIN_MIN), BIN_MAX)


def features(w, k):
    """The 8 features of one row's weights (non-positive / non-finite skipped):
    ln n+, ln sum v, ln max v, the 10/50/90/99 % quantile bins of the weights as
    (b + 1/2) ln2 / 4 (the bin of the ceil(p n+)-th smallest weight), ln k.
    A row without positive weights gives zeros there (ln k still set)."""
    w = np.asarray(w, dtype=np.float64)
    pos = w[(w > 0) & np.isfinite(w)]
    f = np.zeros(F, dtype=np.float64)
    f[7] = math.log(k)
    n = pos.size
    if n == 0:
        return f
    f[0] = math.log(n)
    f[1] = math.log(math.fsum(pos))
    f[2] = math.log(pos.max())
    bins = sorted(weight_bin(x) for x in pos)
    for i, pct in enumerate(PCT):
        r = max(1, -(-n * pct // 100))  # ceil(n pct / 100), integer
        f[3 + i] = (bins[r - 1] + 0.5) * math.log(2.0) / 4.0
    return f


def features_rows(row_ptr, w, k):
    return np.stack([features(w[row_ptr[r]:row_ptr[r + 1]], k) for r in range(len(row_ptr) - 1)])


# --- network --------------------------------------------------------------------

def gelu(x):
    """x Phi(x), Phi the standard normal CDF."""
    return 0.5 * x * (1.0 + np.vectorize(math.erf)(x / math.sqrt(2.0)))


def gelu_grad(x):
    """d/dx [x Phi(x)] = Phi(x) + x phi(x)."""
    cdf = 0.5 * (1.0 + np.vectorize(math.erf)(x / math.sqrt(2.0)))
    return cdf + x * np.exp(-0.5 * x * x) / math.sqrt(2.0 * math.pi)


def forward(theta, X):
    """Predicted ln y* per sample: net(x) - x[1] (the skip subtracts ln sum v).
    Returns (pred, cache) with the activations backprop needs."""
    W1, b1, W2, b2, w3, b3 = unpack(theta)
    X = np.asarray(X, dtype=np.float64)
    a1 = X @ W1.T + b1
    h1 = gelu(a1)
    a2 = h1 @ W2.T + b2
    h2 = gelu(a2)
    out = h2 @ w3 + b3
    pred = out - X[:, 1]
    return pred, (X, a1, h1, a2, h2)


def pinball(r, tau):
    """rho_tau(r) = tau r for r > 0, (tau - 1) r otherwise."""
    return np.where(r > 0, tau * r, (tau - 1.0) * r)


def loss_and_grad(theta, X, t, tau):
    """Mean pinball loss of (t - pred) and its gradient in theta, by the chain
    rule layer by layer (the subgradient of the r <= 0 branch at r = 0)."""
    W1, b1, W2, b2, w3, b3 = unpack(theta)
    pred, (X, a1, h1, a2, h2) = forward(theta, X)
    t = np.asarray(t, dtype=np.float64)
    n = t.size
    r = t - pred
    loss = float(np.mean(pinball(r, tau)))
    g = np.where(r > 0, -tau, 1.0 - tau) / n     # dL/dpred = dL/dout, per sample
    dw3 = h2.T @ g
    db3 = g.sum()
    da2 = np.outer(g, w3) * gelu_grad(a2)        # [n, H]
    dW2 = da2.T @ h1
    db2 = da2.sum(axis=0)
    da1 = (da2 @ W2) * gelu_grad(a1)
    dW1 = da1.T @ X
    db1 = da1.sum(axis=0)
    return loss, pack(dW1, db1, dW2, db2, dw3, db3)


def adam_step(theta, m, v, g, lr, step, beta1=0.9, beta2=0.999, eps=1e-8):
    """One Adam update; returns (theta, m, v)."""
    m = beta1 * m + (1.0 - beta1) * g
    v = beta2 * v + (1.0 - beta2) * g * g
    mhat = m / (1.0 - beta1 ** step)
    vhat = v / (1.0 - beta2 ** step)
    return theta - lr * mhat / (np.sqrt(vhat) + eps), m, v


def ystar_quantile(p, k):
    """The p-quantile of ln(y* sum v) = ln max of k iid Exp(1): (1 - e^-x)^k = p."""
    return math.log(-math.log1p(-p ** (1.0 / k)))
