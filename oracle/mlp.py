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
  stencil-major order, followed by seven values of the column context:
      25: x_i / L = (i + 1/2) / N               (cell position)
      26: log10(s_n / 1 m^-3) - 16               (density level)
      27: (V_R - V_L) / 1000 V                   (applied voltage)
      28: (log2 N - 10) / 2                      (resolution)
      29: log10(dt / 1 s) + 5                    (time step)
      30: asinh(phi_ion,i / s_phi)
      31: asinh(E_ion,i L / s_phi)
  where phi_ion is the potential of the ion charge alone: the root of the
  Poisson residual F_phi (Sec. 2, Eq. nls) with n_e = 0 and both electrodes
  at 0 V (eps_r = 1), and E_ion,i = -(G_{i-1/2} + G_{i+1/2}) / 2 the mean of
  its two face gradients (electrode faces by the residual's one-sided
  formulas). A column of one cell has no Poisson system: 30, 31 are 0.

  network: y = W3 silu(W2 silu(W1 x + b1) + b2) + b3, 32 -> 128 -> 128 -> 2,
  silu(z) = z / (1 + e^{-z}).

  guess (components, a bit set): bit 0 adds the n_e increment s_n y_0; bit 1
  adds the potential increment s_phi y_1; bit 2 instead takes as potential the
  root of F_phi at the guessed n_e (the potential consistent with the guessed
  charge, eps_r = 1; columns of one cell keep phi^n).

  training target: y* = ((n_e* - n_e^n) / s_n, (phi* - phi^n) / s_phi) from
  converged solves, loss = mean over samples and both outputs of (y - y*)^2,
  optimiser Adam (Kingma & Ba 2015) with bias correction.
"""
from __future__ import annotations

import numpy as np

NF = 25          # stencil features
NF_CTX = 7       # column-context features (slots 25..31)
NF_PAD = 32
HIDDEN = 128
NOUT = 2
T_SCALE = 2000.0
E_CHARGE = 1.602176634e-19      # C (CODATA 2018)
EPS0 = 8.8541878128e-12         # F/m
KAPPA = EPS0 / E_CHARGE         # eps_0 eps_r / e with eps_r = 1


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


def poisson_potential(n_minus_f, h, v_left, v_right):
    """Cell potentials phi [N] (N >= 2) with F_phi = -n + f + kappa (G_{i+1/2} -
    G_{i-1/2}) / h = 0 for every cell, given n - f [N] (m^-3): interior face
    gradients (phi_{i+1} - phi_i) / h, electrode faces (9 phi_0 - phi_1 - 8 V_L)
    / (3h) and (8 V_R - 9 phi_{N-1} + phi_{N-2}) / (3h). A banded solve of the
    N tridiagonal rows written out from those faces."""
    from scipy.linalg import solve_banded
    N = n_minus_f.shape[0]
    k = KAPPA / (h * h)
    ab = np.zeros((3, N))            # ab[0, j+1] = A[j, j+1], ab[1, j] = A[j, j], ab[2, j] = A[j+1, j]
    rhs = np.asarray(n_minus_f, dtype=np.float64).copy()
    ab[1, :] = -2.0 * k
    ab[0, 1:] = k
    ab[2, :-1] = k
    # row 0: kappa/h [(phi_1 - phi_0)/h - (9 phi_0 - phi_1 - 8 V_L)/(3h)]
    ab[1, 0] = -4.0 * k
    ab[0, 1] = 4.0 / 3.0 * k
    rhs[0] -= 8.0 / 3.0 * k * v_left
    # row N-1: kappa/h [(8 V_R - 9 phi_{N-1} + phi_{N-2})/(3h) - (phi_{N-1} - phi_{N-2})/h]
    ab[1, N - 1] = -4.0 * k
    ab[2, N - 2] = 4.0 / 3.0 * k
    rhs[N - 1] -= 8.0 / 3.0 * k * v_right
    return solve_banded((1, 1), ab, rhs)


def face_gradients(phi, h, v_left, v_right):
    """G_{-1/2}, G_{1/2}, ..., G_{N-1/2} of the Poisson residual (N + 1 faces)."""
    G = np.empty(phi.shape[0] + 1)
    G[1:-1] = np.diff(phi) / h
    G[0] = (9.0 * phi[0] - phi[1] - 8.0 * v_left) / (3.0 * h)
    G[-1] = (8.0 * v_right - 9.0 * phi[-1] + phi[-2]) / (3.0 * h)
    return G


def ion_field(q, h):
    """(phi_ion, E_ion) of a column: the potential of the ion charge f (n_e = 0,
    electrodes at 0 V) and the mean of each cell's two face gradients, negated."""
    phi = poisson_potential(-np.asarray(q, dtype=np.float64), h, 0.0, 0.0)
    G = face_gradients(phi, h, 0.0, 0.0)
    return phi, -0.5 * (G[:-1] + G[1:])


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
        L = batch.length[c]
        X[a:b, 25] = (i + 0.5) / N
        X[a:b, 26] = np.log10(sn[c]) - 16.0
        X[a:b, 27] = (batch.v_right[c] - batch.v_left[c]) / 1000.0
        X[a:b, 28] = (np.log2(N) - 10.0) / 2.0
        X[a:b, 29] = np.log10(batch.dt[c]) + 5.0
        if N >= 2:
            pi, ei = ion_field(q, L / N)
            X[a:b, 30] = np.arcsinh(pi / sp[c])
            X[a:b, 31] = np.arcsinh(ei * L / sp[c])
    return X


def targets(batch, ne_star, phi_star):
    sn, sp = column_scales(batch)
    Y = np.zeros((batch.ncells, NOUT))
    for c in range(batch.ncol):
        s = slice(batch.col_off[c], batch.col_off[c + 1])
        Y[s, 0] = (ne_star[s] - batch.ne_old[s]) / sn[c]
        Y[s, 1] = (phi_star[s] - batch.phi_old[s]) / sp[c]
    return Y


def guess(batch, Y, components=3):
    sn, sp = column_scales(batch)
    ne = batch.ne_old.copy()
    phi = batch.phi_old.copy()
    fphi = (batch.valence[:, None] * np.atleast_2d(batch.n_ion)).sum(axis=0)
    for c in range(batch.ncol):
        s = slice(batch.col_off[c], batch.col_off[c + 1])
        N = s.stop - s.start
        if components & 1:
            ne[s] += sn[c] * Y[s, 0]
        if components & 4:
            if N >= 2:
                phi[s] = poisson_potential(ne[s] - fphi[s], batch.length[c] / N,
                                           batch.v_left[c], batch.v_right[c])
        elif components & 2:
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
