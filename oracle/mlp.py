"""FP64 numpy oracle of the learned Newton initial guess (test infrastructure).

Only tests/, __graft_entry__.smoke() and the benchmark's CPU-baseline leg may
use it; the CUDA path shares none of this code.

The guess (not a part of the paper; it replaces the plain start X^n of
Algorithm 2 by a predicted one, and the JFNK still converges every solve):

  features of cell i: for each stencil offset o = -2..2 (index mirrored at the
  column ends, j < 0 -> -j-1, j >= N -> 2N-1-j) the five values
      n_e^n / s_n, phi^n / s_phi, f_phi / s_n, T / 2000 K, E h / s_phi,
  with E h = -(phi_{k+1} - phi_{k-1}) / 2 (mirrored neighbours) and the
  per-column scales s_n, s_phi of Eq. newton_sc taken at X^n; 25 values in
  stencil-major order, zero-padded to 32.

  network: y = W3 silu(W2 silu(W1 x + b1) + b2) + b3, 32 -> 128 -> 128 -> 2,
  silu(z) = z / (1 + e^{-z}).

  guess: n_e = n_e^n + s_n y_0, phi = phi^n + s_phi y_1.

  training target: y* = ((n_e* - n_e^n) / s_n, (phi* - phi^n) / s_phi) from
  converged solves, loss = mean over samples and both outputs of (y - y*)^2,
  optimiser Adam (Kingma & Ba 2015) with bias correction.
"""
from __future__ import annotations

import numpy as np

NF = 25
NF_PAD = 32
HIDDEN = 128
NOUT = 2
T_SCALE = 2000.0


def column_scales(batch):
    """(s_n, s_phi) per column, from the plain start X^n (Eq. newton_sc)."""
    sn = np.empty(batch.ncol)
    sp = np.empty(batch.ncol)
    fphi = (batch.valence[:, None] * np.atleast_2d(batch.n_ion)).sum(axis=0)
    for c in range(batch.ncol):
        s = slice(batch.col_off[c], batch.col_off[c + 1])
        sn[c] = max(np.abs(batch.ne_old[s]).max(), np.abs(fphi[s]).max(), 1.0)
        sp[c] = max(np.abs(batch.phi_old[s]).max(), abs(batch.v_left[c]), abs(batch.v_right[c]), 1.0)
    return sn, sp


def features(batch):
    """[cells, 32] float64 feature matrix of every cell of the batch."""
    fphi = (batch.valence[:, None] * np.atleast_2d(batch.n_ion)).sum(axis=0)
    sn, sp = column_scales(batch)
    X = np.zeros((batch.ncells, NF_PAD))
    for c in range(batch.ncol):
        a, b = int(batch.col_off[c]), int(batch.col_off[c + 1])
        N = b - a
        ne, phi, q, T = batch.ne_old[a:b], batch.phi_old[a:b], fphi[a:b], batch.T[a:b]

        def mirror(j):
            j = np.where(j < 0, -j - 1, j)
            return np.where(j >= N, 2 * N - 1 - j, j)
        i = np.arange(N)
        for o in range(-2, 3):
            k = mirror(i + o)
            kp, km = mirror(k + 1), mirror(k - 1)
            base = 5 * (o + 2)
            X[a:b, base + 0] = ne[k] / sn[c]
            X[a:b, base + 1] = phi[k] / sp[c]
            X[a:b, base + 2] = q[k] / sn[c]
            X[a:b, base + 3] = T[k] / T_SCALE
            X[a:b, base + 4] = -(phi[kp] - phi[km]) / 2.0 / sp[c]
    return X


def targets(batch, ne_star, phi_star):
    sn, sp = column_scales(batch)
    Y = np.zeros((batch.ncells, NOUT))
    for c in range(batch.ncol):
        s = slice(batch.col_off[c], batch.col_off[c + 1])
        Y[s, 0] = (ne_star[s] - batch.ne_old[s]) / sn[c]
        Y[s, 1] = (phi_star[s] - batch.phi_old[s]) / sp[c]
    return Y


def guess(batch, Y):
    sn, sp = column_scales(batch)
    ne = batch.ne_old.copy()
    phi = batch.phi_old.copy()
    for c in range(batch.ncol):
        s = slice(batch.col_off[c], batch.col_off[c + 1])
        ne[s] += sn[c] * Y[s, 0]
        phi[s] += sp[c] * Y[s, 1]
    return ne, phi


def init_params(seed=0):
    """He-style initialisation, FP64: dict W1 [128,32], b1, W2 [128,128], b2, W3 [2,128], b3."""
    rng = np.random.default_rng(seed)
    return dict(W1=rng.standard_normal((HIDDEN, NF_PAD)) * np.sqrt(2.0 / NF),
                b1=np.zeros(HIDDEN),
                W2=rng.standard_normal((HIDDEN, HIDDEN)) * np.sqrt(2.0 / HIDDEN),
                b2=np.zeros(HIDDEN),
                W3=rng.standard_normal((NOUT, HIDDEN)) * np.sqrt(1.0 / HIDDEN) * 0.1,
                b3=np.zeros(NOUT))


def silu(z):
    return z / (1.0 + np.exp(-z))


def silu_grad(z):
    s = 1.0 / (1.0 + np.exp(-z))
    return s * (1.0 + z * (1.0 - s))


def forward(p, X):
    Z1 = X @ p["W1"].T + p["b1"]
    H1 = silu(Z1)
    Z2 = H1 @ p["W2"].T + p["b2"]
    H2 = silu(Z2)
    Y = H2 @ p["W3"].T + p["b3"]
    return Y, dict(X=X, Z1=Z1, H1=H1, Z2=Z2, H2=H2)


def mse(Y, T):
    """loss = mean((Y - T)^2) over samples and outputs, and dL/dY."""
    d = Y - T
    return float(np.mean(d * d)), 2.0 * d / d.size


def backward(p, cache, dY):
    """Gradients of a scalar loss with dL/dY = dY (chain rule through the layers)."""
    g = {}
    g["W3"] = dY.T @ cache["H2"]
    g["b3"] = dY.sum(axis=0)
    dH2 = dY @ p["W3"]
    dZ2 = dH2 * silu_grad(cache["Z2"])
    g["W2"] = dZ2.T @ cache["H1"]
    g["b2"] = dZ2.sum(axis=0)
    dH1 = dZ2 @ p["W2"]
    dZ1 = dH1 * silu_grad(cache["Z1"])
    g["W1"] = dZ1.T @ cache["X"]
    g["b1"] = dZ1.sum(axis=0)
    return g


def adam_step(p, g, m, v, t, lr=1e-3, beta1=0.9, beta2=0.999, eps=1e-8):
    """One Adam update (in place) of every parameter; t is the 1-based step."""
    for k in p:
        m[k] = beta1 * m[k] + (1 - beta1) * g[k]
        v[k] = beta2 * v[k] + (1 - beta2) * g[k] * g[k]
        mh = m[k] / (1 - beta1 ** t)
        vh = v[k] / (1 - beta2 ** t)
        p[k] = p[k] - lr * mh / (np.sqrt(vh) + eps)


def bf16_round(a):
    """Round float64 values to the nearest bfloat16 (ties to even), as float64."""
    f = np.asarray(a, dtype=np.float32)
    u = f.view(np.uint32).astype(np.uint64)
    r = ((u + 0x7FFF + ((u >> 16) & 1)) >> 16) << 16
    return r.astype(np.uint32).view(np.float32).astype(np.float64)
