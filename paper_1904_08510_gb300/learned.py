"""Training and evaluation of the learned Newton initial guess.

Data: converged solves of seeded columns of one profile family (--family):
the single-flame family of workload.make_batch(kind="single") with a fixed cell
count or cell counts drawn uniformly from a range (--train-cells), or the ragged
family of the benchmark workload (kind="ragged", training seeds disjoint from
the benchmark's), solved by the batched FP64 JFNK on the GPU; features and targets are produced by the library's own kernels
(sdcef_mlp_features / sdcef_mlp_targets). Training runs the library's BF16
forward/backward kernels and its Adam step. Evaluation solves held-out columns
with and without the guess and compares Newton and GMRES iteration counts.
"""
from __future__ import annotations

import os
import time

import numpy as np

from . import sdcef as S
from .workload import make_batch, sdc_batch

HERE = os.path.dirname(os.path.abspath(__file__))
WEIGHTS = os.path.join(HERE, "data", "mlp_weights.npz")                 # single-flame family
WEIGHTS_RAGGED = os.path.join(HERE, "data", "mlp_weights_ragged.npz")   # ragged (bench) family
WEIGHTS_SWEEP = os.path.join(HERE, "data", "mlp_weights_sweep.npz")     # first SDC iteration


def init_params(seed=0):
    """He-style initial parameters, flat FP32 in the order of the C ABI; the
    weights of the 7 column-context inputs start at 0 (training brings them in)."""
    rng = np.random.default_rng(seed)
    p = dict(W1=rng.standard_normal((128, 32)) * np.sqrt(2.0 / 25),
             b1=np.zeros(128),
             W2=rng.standard_normal((128, 128)) * np.sqrt(2.0 / 128),
             b2=np.zeros(128),
             W3=rng.standard_normal((2, 128)) * np.sqrt(1.0 / 128) * 0.1,
             b3=np.zeros(2))
    p["W1"][:, 25:] = 0.0
    return S.pack_params(p).astype(np.float32)


def generate(ncol: int, seed: int, *, kind="single", n_cells=256, n_range=None, chunk=8192,
             device="cuda:0", eps_F=1e-10):
    """Solve ncol seeded columns of profile family `kind` on the GPU; return
    (features bf16 [cells,32], targets f32 [cells,2]) device tensors and the
    number of converged solves. For kind="ragged" the cell counts follow the
    family's own draw unless n_range is given. kind="sweep": the first SDC
    iteration of the MISDC electric sweep (Algorithm 1) on workload.sdc_batch
    columns of n_cells cells at the ion-CFL step: the features are those of X^n
    with the ion densities n^n (what the guess sees before the sweep), the
    target is the root of the implicit solve with the provisional ions of the
    first iteration."""
    import torch
    Xs, Ts, stats = [], [], []
    mlp = S.MLP(1, )
    for c0 in range(0, ncol, chunk):
        n = min(chunk, ncol - c0)
        if kind == "ragged":
            b = make_batch("ragged", n, seed + c0, n_range=n_range)
        elif kind == "sweep":
            b = sdc_batch(n, seed + c0, n_cells=n_cells)
        else:
            b = make_batch("single", n, seed + c0, n_cells=None if n_range else n_cells,
                           n_range=n_range)
        db = S.DeviceBatch.from_host(b, device)
        solver = S.Solver(S.default_params(eps_F=eps_F), max_cols=n, max_cells=b.ncells,
                          max_col_cells=int(b.lengths().max()))
        if kind == "sweep":
            ions = solver.ion_provisional(db, db.tensors["phi_old"])
            out = solver.solve(S.DeviceBatch(db.ncol, db.ncells, dict(db.tensors, n_ion=ions),
                                             db.valence))
        else:
            out = solver.solve(db)
        X = mlp.features(db)
        T = mlp.targets(db, out["ne"], out["phi"])
        ok = out["status"] == S.STATUS_OK
        torch.cuda.synchronize()
        Xs.append(X)
        Ts.append(T)
        stats.append(int(ok.sum().item()))
        solver.close()
    mlp.close()
    return torch.cat(Xs), torch.cat(Ts), sum(stats)


def save_checkpoint(path, mlp, it, rng):
    """Training checkpoint: parameters, Adam moments and step, the iteration
    and the window generator's state."""
    st = mlp.get_state()
    np.savez(path, params=st["params"], adam_m=st["adam_m"], adam_v=st["adam_v"],
             step=np.int64(st["step"]), it=np.int64(it),
             rng=np.array(repr(rng.bit_generator.state)))


def load_checkpoint(path):
    import ast
    with np.load(path) as z:
        return ({"params": z["params"], "adam_m": z["adam_m"], "adam_v": z["adam_v"],
                 "step": int(z["step"])}, int(z["it"]), ast.literal_eval(str(z["rng"])))


def train(X, T, *, steps: int, batch: int = 32768, lr: float = 2e-3, lr_end: float = 1e-4,
          seed: int = 0, params=None, log_every: int = 0, checkpoint=None, checkpoint_every=0,
          resume=None):
    """Adam on contiguous random windows of (X, T); cosine learning-rate decay.
    checkpoint / checkpoint_every: save a checkpoint every so many iterations;
    resume: continue from a checkpoint (parameters, Adam state, iteration and
    window sequence), reproducing the uninterrupted run's updates.
    Returns (mlp handle with the trained parameters, loss history)."""
    import torch
    rows = X.shape[0]
    batch = min(batch, rows)
    mlp = S.MLP(batch)
    rng = np.random.default_rng(seed)
    start = 0
    if resume is not None:
        state, start, rng_state = load_checkpoint(resume)
        mlp.set_state(state)
        rng.bit_generator.state = rng_state
    else:
        mlp.set_params(init_params(seed) if params is None else params)
    loss = torch.zeros(1, dtype=torch.float32, device=X.device)
    hist = []
    for it in range(start, steps):
        if checkpoint and checkpoint_every and it > start and it % checkpoint_every == 0:
            torch.cuda.synchronize()
            save_checkpoint(checkpoint, mlp, it, rng)
        o = int(rng.integers(0, rows - batch + 1))
        a = lr_end + 0.5 * (lr - lr_end) * (1 + np.cos(np.pi * it / max(steps - 1, 1)))
        mlp.train_step(X[o:o + batch], T[o:o + batch], a, loss)
        if log_every and (it % log_every == 0 or it == steps - 1):
            torch.cuda.synchronize()
            hist.append((it, float(loss.item())))
    torch.cuda.synchronize()
    return mlp, hist


def evaluate(params, ncol: int, seed: int, *, kind="single", n_range=(512, 2048), device="cuda:0",
             reps=3, variants=(("learned", 5),)):
    """Held-out solves with and without the learned guess (FP64 batched JFNK).
    variants: (name, components) pairs; components = 1 applies the predicted
    n_e increment only, 3 applies n_e and phi, 5 the n_e increment with the
    potential of the guessed charge (root of the Poisson residual)."""
    import torch
    b = make_batch(kind, ncol, seed, n_range=n_range)
    db = S.DeviceBatch.from_host(b, device)
    solver = S.Solver(S.default_params(), max_cols=b.ncol, max_cells=b.ncells,
                      max_col_cells=int(b.lengths().max()))
    mlp = S.MLP(b.ncells)
    mlp.set_params(params)
    res = {}
    comps = dict(variants)
    for name in ("plain",) + tuple(comps):
        times = []
        for _ in range(reps):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            if name != "plain":
                ne, phi = mlp.guess(db, components=comps[name])
                out = solver.solve(db.with_guess(ne, phi))
            else:
                out = solver.solve(db)
            e1.record()
            torch.cuda.synchronize()
            times.append(e0.elapsed_time(e1))
        st = out["status"].cpu().numpy()
        nw = out["newton_it"].cpu().numpy()
        kr = out["krylov_it"].cpu().numpy()
        res[name] = dict(ms=float(np.median(times)), status_ok=int((st == 0).sum()),
                         newton_mean=float(nw.mean()), newton_p50=float(np.median(nw)),
                         newton_p99=float(np.percentile(nw, 99)), krylov_mean=float(kr.mean()),
                         solves_per_s=b.ncol / (np.median(times) / 1e3),
                         ne=out["ne"].cpu().numpy(), phi=out["phi"].cpu().numpy())
    solver.close()
    mlp.close()
    return b, res


def evaluate_sweep(params, ncol: int, seed: int, *, n_cells=1024, device="cuda:0", reps=3,
                   components=5):
    """The MISDC electric sweep's first SDC iteration (workload.sdc_batch columns)
    with and without the learned start: Newton and GMRES iterations and time of
    that iteration (guess kernel included)."""
    import torch
    b = sdc_batch(ncol, seed, n_cells=n_cells)
    db = S.DeviceBatch.from_host(b, device)
    solver = S.Solver(S.default_params(), max_cols=b.ncol, max_cells=b.ncells,
                      max_col_cells=n_cells)
    work = solver.sweep_work(db)
    out = solver.alloc_result(db)
    mlp = S.MLP(b.ncells)
    mlp.set_params(params)
    ne_g = torch.empty(b.ncells, dtype=torch.float64, device=device)
    ph_g = torch.empty_like(ne_g)
    gdb = db.with_guess(ne_g, ph_g)
    res = {}
    for name in ("plain", "learned"):
        def one():
            if name == "learned":
                mlp.guess(db, ne_g, ph_g, components=components)
                return solver.sdc_sweep(gdb, 1, work=work, out=out)
            return solver.sdc_sweep(db, 1, work=work, out=out)
        one()
        times = []
        for _ in range(reps):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            o = one()
            e1.record()
            torch.cuda.synchronize()
            times.append(e0.elapsed_time(e1))
        res[name] = dict(ms=float(np.median(times)), status_ok=int((o["status"] == 0).sum().item()),
                         newton_mean=float(o["newton_it"].float().mean().item()),
                         krylov_mean=float(o["krylov_it"].float().mean().item()))
    solver.close()
    mlp.close()
    return res


def save(params, path=WEIGHTS, meta=None):
    os.makedirs(os.path.dirname(path), exist_ok=True)
    np.savez(path, params=np.asarray(params, dtype=np.float32), meta=np.array(repr(meta or {})))


def load(path=WEIGHTS):
    with np.load(path) as z:
        return z["params"].astype(np.float32)


def main():
    """Train on converged single-flame solves and report held-out gains."""
    import argparse
    import json
    ap = argparse.ArgumentParser()
    ap.add_argument("--ncol", type=int, default=None,
                    help="training columns (default: 400k single, 600k ragged, 262144 sweep, "
                         "the sets of the shipped networks)")
    ap.add_argument("--steps", type=int, default=480_000)
    ap.add_argument("--batch", type=int, default=32768)
    ap.add_argument("--lr", type=float, default=2e-3)
    ap.add_argument("--eval-ncol", type=int, default=None,
                    help="held-out columns (default: 4096; 16384 for the sweep family)")
    ap.add_argument("--out", default=None,
                    help="weights file (default: the family's file under data/)")
    ap.add_argument("--train-cells", default="512:2048",
                    help="cells per training column: an integer, or lo:hi for U{lo..hi}")
    ap.add_argument("--family", default="single", choices=["single", "ragged", "sweep"],
                    help="profile family of the training and evaluation columns (sweep: the "
                         "first SDC iteration of the electric sweep, 1024-cell columns)")
    args = ap.parse_args()
    if args.ncol is None:
        args.ncol = {"single": 400_000, "ragged": 600_000, "sweep": 262_144}[args.family]
    if args.eval_ncol is None:
        args.eval_ncol = 16384 if args.family == "sweep" else 4096
    if args.out is None:
        args.out = {"single": WEIGHTS, "ragged": WEIGHTS_RAGGED, "sweep": WEIGHTS_SWEEP}[args.family]
    t0 = time.perf_counter()
    if args.family == "ragged":
        # training seeds 3e6 + i, disjoint from the evaluation / benchmark seeds 2e6 + i
        X, T, nok = generate(args.ncol, 3_000_000, kind="ragged")
    elif args.family == "sweep":
        # training seeds 6e6 + i, disjoint from the sweep benchmark's 5e6 + i
        X, T, nok = generate(args.ncol, 6_000_000, kind="sweep", n_cells=1024)
    elif ":" in args.train_cells:
        lo, hi = (int(v) for v in args.train_cells.split(":"))
        X, T, nok = generate(args.ncol, 1_000_000, n_range=(lo, hi))
    else:
        X, T, nok = generate(args.ncol, 1_000_000, n_cells=int(args.train_cells))
    t1 = time.perf_counter()
    mlp, hist = train(X, T, steps=args.steps, batch=args.batch, lr=args.lr, log_every=500)
    t2 = time.perf_counter()
    params = mlp.get_params()
    save(params, args.out, dict(ncol=args.ncol, steps=args.steps, batch=args.batch, lr=args.lr,
                                train_cells=args.train_cells, family=args.family))
    if args.family == "sweep":
        ev = {f"components_{c}": evaluate_sweep(params, args.eval_ncol, 5_000_000, components=c)
              for c in (1, 5)}
    else:
        b, res = evaluate(params, args.eval_ncol, 2_000_000, kind=args.family,
                          n_range=None if args.family == "ragged" else (512, 2048),
                          variants=(("learned_ne", 1), ("learned_ne_poisson_phi", 5)))
        ev = {k: {kk: vv for kk, vv in v.items() if kk not in ("ne", "phi")} for k, v in res.items()}
    summary = dict(family=args.family, train_columns=args.ncol, train_cells=args.train_cells,
                   train_samples=int(X.shape[0]), converged=nok,
                   data_s=t1 - t0, train_s=t2 - t1, loss=hist, eval=ev)
    print(json.dumps(summary))


if __name__ == "__main__":
    main()
