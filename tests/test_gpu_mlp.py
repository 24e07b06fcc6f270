"""GPU kernels of the learned initial guess against the FP64 numpy oracle.

BF16 bar: features match the oracle rounded to bfloat16 to one BF16 ulp; the
network output and every parameter gradient match the oracle evaluated on the
same BF16-rounded weights and inputs element by element: |gpu - oracle| <=
2e-2 x the max-norm of the oracle's output column or parameter tensor (BF16
activations and operands carry 8 significant bits; accumulation is FP32). A
numpy emulation of the kernels' rounding points stays below 7e-3 on these
cases. The rows of the last, ragged 128-row tile are scaled up (inputs x3 for
the forward pass, targets x300 for the gradients), so that a wrong or dropped
last tile moves the compared values by far more than the bar.
"""
import numpy as np
import pytest

from oracle import mlp as M
from paper_1904_08510_gb300.workload import make_batch

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_1904_08510_gb300 import sdcef as S  # noqa: E402
from paper_1904_08510_gb300 import learned as Lrn  # noqa: E402


def dev():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return "cuda:0"


def rounded_params(seed=3):
    p = M.init_params(seed)
    rng = np.random.default_rng(seed)
    for k in ("b1", "b2", "b3"):
        p[k] = 0.1 * rng.standard_normal(p[k].shape)
    flat = S.pack_params(p).astype(np.float32)
    q = S.unpack_params(flat.astype(np.float64))
    for k in ("W1", "W2", "W3"):
        q[k] = M.bf16_round(q[k])
    return flat, q


def tail_rows(n):
    """Rows of the last, ragged 128-row tile."""
    return n - 128 * ((n - 1) // 128)


def assert_elementwise(a, r, rel, what):
    """|a - r| <= rel * max|r| for every element of each column (axis 0 scale)."""
    a = np.atleast_2d(np.asarray(a, dtype=np.float64).T).T
    r = np.atleast_2d(np.asarray(r, dtype=np.float64).T).T
    scale = np.abs(r).max(axis=0)
    err = np.abs(a - r) / np.maximum(scale, 1e-30)
    assert err.max() <= rel, (what, float(err.max()), np.unravel_index(err.argmax(), err.shape))


@pytest.mark.parametrize("n_range", [(3, 300), (1, 4)])
def test_features_match_oracle(n_range):
    """One BF16 ulp. The ion potential and field (features 30, 31) come from
    FP32 prefix sums on the GPU and an FP64 banded solve in the oracle: near the
    electrodes, where the potential tends to 0, and where the field changes
    sign they differ by the FP32 rounding of the sums (relative 1e-6 of the
    column's largest terms), hence an absolute floor of 1e-4 on those two (a
    BF16 ulp of a feature of order 1 is 4e-3); log10(dt) + 5 is 0 up to
    rounding at dt = 1e-5 s: an absolute floor of 1e-6 on the context features."""
    d = dev()
    b = make_batch("ragged", 5, 31, n_range=n_range)
    db = S.DeviceBatch.from_host(b, d)
    mlp = S.MLP(16)
    X = mlp.features(db).float().cpu().numpy()
    ref = M.bf16_round(M.features(b))
    tol = 2.0 ** -7 * np.abs(ref) + 1e-30
    tol[:, 25:] += 1e-6   # context features that are 0 up to rounding (log10(dt) + 5)
    tol[:, 30:] += 1e-4   # the ion field from FP32 prefix sums
    assert np.all(np.abs(X - ref) <= tol), np.argwhere(np.abs(X - ref) > tol)[:5]
    mlp.close()


def test_features_and_poisson_start_with_two_species_and_varied_steps():
    """The general charge f_phi = sum nu_s n_s (a cation and a 5 % anion) and
    per-column time steps and electrode potentials: features against the
    oracle (one BF16 ulp), and the Poisson start against the oracle's banded
    solve of F_phi = 0 with the kernel's own n_e (1e-9)."""
    d = dev()
    b = make_batch("ragged", 7, 57, n_range=(2, 400))
    rng = np.random.default_rng(4)
    b.n_ion = np.vstack([b.n_ion, 0.05 * b.n_ion * np.abs(rng.standard_normal(b.ncells))])
    b.valence = np.array([1, -1], dtype=np.int32)
    b.dt = 10.0 ** rng.uniform(-7, -4, b.ncol)
    b.v_left = rng.uniform(-50, 50, b.ncol)
    db = S.DeviceBatch.from_host(b, d)
    mlp = S.MLP(b.ncells)
    X = mlp.features(db).float().cpu().numpy()
    ref = M.bf16_round(M.features(b))
    tol = 2.0 ** -7 * np.abs(ref) + 1e-30
    tol[:, 25:] += 1e-6
    tol[:, 30:] += 1e-4
    assert np.all(np.abs(X - ref) <= tol), np.argwhere(np.abs(X - ref) > tol)[:5]
    flat, _ = rounded_params(17)
    mlp.set_params(flat)
    ne, phi = mlp.guess(db, components=S.GUESS_NE | S.GUESS_PHI_POISSON)
    mlp.check()
    ne, phi = ne.cpu().numpy(), phi.cpu().numpy()
    f = (b.valence[:, None] * b.n_ion).sum(axis=0)
    for c in range(b.ncol):
        sl = slice(b.col_off[c], b.col_off[c + 1])
        N = sl.stop - sl.start
        pr = M.poisson_potential(ne[sl] - f[sl], b.length[c] / N, b.v_left[c], b.v_right[c])
        assert np.abs(phi[sl] - pr).max() <= 1e-9 * np.abs(pr).max(), c
    mlp.close()


def test_targets_and_guess_round_trip():
    d = dev()
    b = make_batch("ragged", 4, 8, n_range=(20, 200))
    db = S.DeviceBatch.from_host(b, d)
    rng = np.random.default_rng(0)
    ne = b.ne_old * (1 + 0.2 * rng.standard_normal(b.ncells))
    phi = b.phi_old + 3 * rng.standard_normal(b.ncells)
    mlp = S.MLP(16)
    T = mlp.targets(db, torch.as_tensor(ne, device=d), torch.as_tensor(phi, device=d))
    ref = M.targets(b, ne, phi)
    np.testing.assert_allclose(T.cpu().numpy(), ref, rtol=1e-6, atol=1e-7)


# 1000 rows: 8 tiles with a ragged last one; 40001: 313 tiles, more than the
# 2 x 152 co-resident CTAs of the fused forward
@pytest.mark.parametrize("n", [1000, 40001])
def test_forward_matches_oracle_on_bf16_weights(n):
    d = dev()
    flat, q = rounded_params()
    rng = np.random.default_rng(1)
    Xh = M.bf16_round(rng.standard_normal((n, 32)))
    Xh[:, 25:] = 0.0
    Xh[-tail_rows(n):] *= 3.0          # the ragged last tile carries the largest outputs
    mlp = S.MLP(n)
    mlp.set_params(flat)
    X = torch.as_tensor(Xh, dtype=torch.float32, device=d).to(torch.bfloat16)
    Y = mlp.forward(X).cpu().numpy()
    Yr, _ = M.forward(q, Xh)
    assert_elementwise(Y, Yr, 2e-2, "Y")


# 37 and 700 rows: one ragged 128-row tile and several; 20011 rows: 157 tiles,
# two per CTA of the persistent training kernel, the last one ragged; 40001
# rows: three tiles per CTA, so that each CTA accumulates its weight and bias
# gradients in TMEM across tiles and reuses both of its X buffers
@pytest.mark.parametrize("n", [37, 700, 20011, 40001])
def test_gradients_match_fp64_backprop(n):
    d = dev()
    flat, q = rounded_params(5)
    rng = np.random.default_rng(n)
    Xh = M.bf16_round(rng.standard_normal((n, 32)))
    Xh[:, 25:] = 0.0
    Th = rng.standard_normal((n, 2))
    # the samples of the ragged last tile dominate every weight gradient:
    # dropping them changes each by > 80 %
    Th[-tail_rows(n):] *= 300.0
    mlp = S.MLP(n)
    mlp.set_params(flat)
    X = torch.as_tensor(Xh, dtype=torch.float32, device=d).to(torch.bfloat16)
    T = torch.as_tensor(Th, dtype=torch.float32, device=d)
    g, loss = mlp.grad(X, T)
    g = S.unpack_params(g.cpu().numpy())
    Y, cache = M.forward(q, Xh)
    lr, dY = M.mse(Y, Th)
    gr = M.backward(q, cache, dY)
    assert float(loss.item()) == pytest.approx(lr, rel=2e-2)
    for k in ("W1", "b1", "W2", "b2", "W3", "b3"):
        a, r = g[k], gr[k]
        if k == "W1":
            a, r = a[:, :25], r[:, :25]
        # one scale per tensor: the max-norm of the oracle's gradient
        assert_elementwise(np.ravel(a), np.ravel(r), 2e-2, k)


def test_gradients_from_unaligned_features_match_aligned():
    """Features 8 bytes off a 16-byte boundary cannot be described by a tensor
    map: the training kernel then stages them by element-wise copies into the
    same layout. The gradients must be bit-identical to those of the same
    features at an aligned address (read by TMA)."""
    d = dev()
    flat, _ = rounded_params(6)
    n = 700
    rng = np.random.default_rng(8)
    Xh = M.bf16_round(rng.standard_normal((n, 32)))
    Xh[:, 25:] = 0.0
    Th = rng.standard_normal((n, 2))
    T = torch.as_tensor(Th, dtype=torch.float32, device=d)
    mlp = S.MLP(n)
    mlp.set_params(flat)
    Xa = torch.as_tensor(Xh, dtype=torch.float32, device=d).to(torch.bfloat16)
    buf = torch.zeros(n * 32 + 8, dtype=torch.bfloat16, device=d)
    Xu = buf[4:4 + n * 32].view(n, 32)
    Xu.copy_(Xa)
    assert Xu.data_ptr() % 16 == 8
    ga, la = mlp.grad(Xa, T)
    gu, lu = mlp.grad(Xu, T)
    mlp.check()
    assert np.array_equal(gu.cpu().numpy(), ga.cpu().numpy())
    assert float(lu.item()) == float(la.item())
    mlp.close()


def test_adam_step_matches_oracle():
    d = dev()
    flat, q = rounded_params(7)
    rng = np.random.default_rng(2)
    n = 256
    Xh = M.bf16_round(rng.standard_normal((n, 32)))
    Xh[:, 25:] = 0.0
    Th = rng.standard_normal((n, 2))
    mlp = S.MLP(n)
    mlp.set_params(flat)
    X = torch.as_tensor(Xh, dtype=torch.float32, device=d).to(torch.bfloat16)
    T = torch.as_tensor(Th, dtype=torch.float32, device=d)
    mlp.train_step(X, T, 1e-3)
    mlp.check()                       # no tensor-core wait ran out
    got = S.unpack_params(mlp.get_params())
    p0 = S.unpack_params(flat.astype(np.float64))
    # first Adam step moves every parameter with a non-negligible gradient by ~lr
    Y, cache = M.forward(q, Xh)
    _, dY = M.mse(Y, Th)
    gr = M.backward(q, cache, dY)
    for k in ("W2", "b2", "W3"):
        big = np.abs(gr[k]) > 1e-3 * np.abs(gr[k]).max()
        step = (p0[k] - got[k])[big]
        np.testing.assert_allclose(np.abs(step), 1e-3, rtol=2e-2)
        assert np.mean(np.sign(step) == np.sign(gr[k][big])) > 0.97


def test_training_reduces_loss_and_newton_iterations():
    """A short training run on converged solves lowers the loss and the Newton
    iterations of held-out columns of the same cell-count range (what the
    learned guess is for). The predicted n_e increment is applied and phi is
    the potential of the guessed charge (the predicted phi increment is too
    coarse for the exponential Scharfetter-Gummel fluxes)."""
    dev()
    X, T, nok = Lrn.generate(2048, 3_000_000, n_range=(256, 1024))
    mlp, hist = Lrn.train(X, T, steps=1500, batch=16384, lr=2e-3, log_every=100)
    assert hist[-1][1] < 0.5 * hist[0][1], hist
    params = mlp.get_params()
    b, res = Lrn.evaluate(params, 128, 4_000_000, n_range=(256, 1024), reps=1,
                          variants=(("learned", S.GUESS_NE | S.GUESS_PHI_POISSON),))
    assert res["plain"]["status_ok"] == b.ncol and res["learned"]["status_ok"] == b.ncol
    assert res["learned"]["newton_mean"] < res["plain"]["newton_mean"], res
    # the guess changes the start, not the root
    for c in range(b.ncol):
        s = slice(b.col_off[c], b.col_off[c + 1])
        e = np.abs(res["learned"]["ne"][s] - res["plain"]["ne"][s]).max() / np.abs(res["plain"]["ne"][s]).max()
        assert e < 1e-8


@pytest.mark.parametrize("components", [S.GUESS_NE, S.GUESS_NE | S.GUESS_PHI,
                                        S.GUESS_NE | S.GUESS_PHI_POISSON, S.GUESS_PHI_POISSON])
def test_fused_guess_matches_oracle_network(components):
    d = dev()
    flat, q = rounded_params(11)
    b = make_batch("ragged", 9, 55, n_range=(2, 700))
    db = S.DeviceBatch.from_host(b, d)
    mlp = S.MLP(b.ncells)
    mlp.set_params(flat)
    ne, phi = mlp.guess(db, components=components)
    ne, phi = ne.cpu().numpy(), phi.cpu().numpy()
    Y, _ = M.forward(q, M.bf16_round(M.features(b)))
    sn, sp = M.column_scales(b)
    yn = np.empty(b.ncells)
    yp = np.empty(b.ncells)
    for c in range(b.ncol):
        s = slice(b.col_off[c], b.col_off[c + 1])
        yn[s] = (ne[s] - b.ne_old[s]) / sn[c]
        yp[s] = (phi[s] - b.phi_old[s]) / sp[c]
        if components & S.GUESS_PHI_POISSON:
            # the root of the Poisson residual at the kernel's own n_e: prefix
            # sums on the GPU against the oracle's banded solve
            N = s.stop - s.start
            ref = M.poisson_potential(ne[s] - b.n_ion[0, s], b.length[c] / N, b.v_left[c],
                                      b.v_right[c])
            assert np.abs(phi[s] - ref).max() <= 1e-9 * np.abs(ref).max(), c
        elif not components & S.GUESS_PHI:
            assert np.array_equal(phi[s], b.phi_old[s])
        if not components & S.GUESS_NE:
            assert np.array_equal(ne[s], b.ne_old[s])
    # every cell of every column against the network's output scale
    if components & S.GUESS_NE:
        assert_elementwise(yn, Y[:, 0], 2e-2, "dn")
    if (components & 6) == S.GUESS_PHI:
        assert_elementwise(yp, Y[:, 1], 2e-2, "dphi")
    mlp.close()


def test_poisson_start_keeps_one_cell_columns_and_zeroes_f_phi():
    """Columns of one cell keep phi^n; elsewhere the oracle's Poisson residual
    at the start vanishes to rounding of its largest terms."""
    import oracle as O
    d = dev()
    flat, _ = rounded_params(13)
    b = make_batch("ragged", 12, 90, n_range=(1, 8))
    assert (b.lengths() == 1).any()
    db = S.DeviceBatch.from_host(b, d)
    mlp = S.MLP(b.ncells)
    mlp.set_params(flat)
    ne, phi = mlp.guess(db, components=S.GUESS_NE | S.GUESS_PHI_POISSON)
    torch.cuda.synchronize()
    ne, phi = ne.cpu().numpy(), phi.cpu().numpy()
    _, Fp = O.residual(b, ne, phi, O.default_params())
    for c in range(b.ncol):
        s = slice(b.col_off[c], b.col_off[c + 1])
        if s.stop - s.start == 1:
            assert phi[s][0] == b.phi_old[s][0]
        else:
            # the terms of F_phi: the densities and kappa/h^2 times the potential
            h = b.length[c] / (s.stop - s.start)
            scale = max(np.abs(ne[s]).max(), np.abs(b.n_ion[0, s]).max(),
                        M.KAPPA / h ** 2 * np.abs(phi[s]).max())
            assert np.abs(Fp[s]).max() <= 1e-12 * scale, c
    mlp.close()
