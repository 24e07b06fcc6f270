"""Cases run against the bounds-checking build of libsdcef.so (SDCEF_LIB points
at it); used by tests/test_gpu_checks.py in a child process. Prints one JSON
object: per case the check word read after the calls (0 = no failed bounds
test) and the largest relative error against the CPU oracle or the expected
values."""
import json
import sys

import numpy as np
import torch

import oracle as O
from oracle import mlp as M
from paper_1904_08510_gb300 import sdcef as S
from paper_1904_08510_gb300.workload import make_batch, sdc_batch, transport_table

D = "cuda:0"


def colerr(b, a, ref):
    return max(float(np.abs(a[s] - ref[s]).max() / max(np.abs(ref[s]).max(), 1e-300))
               for s in (slice(b.col_off[c], b.col_off[c + 1]) for c in range(b.ncol)))


def solve_case(b, gkw, okw, guess=None, table=None, oracle_guess=True):
    p = S.default_params(**gkw)
    s = S.Solver(p, max_cols=b.ncol, max_cells=b.ncells, max_col_cells=int(b.lengths().max()))
    if table is not None:
        s.set_transport_table(table)
    g = None if guess is None else (torch.as_tensor(guess[0], device=D),
                                    torch.as_tensor(guess[1], device=D))
    db = S.DeviceBatch.from_host(b, D)
    if g is not None:
        db = db.with_guess(*g)
    out = s.solve(db)
    torch.cuda.synchronize()
    out = {k: v.cpu().numpy() for k, v in out.items()}
    word = s.check_word()
    s.close()
    op = O.default_params(**okw)
    if table is not None:
        op = O.default_params(table=table, **okw)
    ref = O.solve(b, op, guess=guess if oracle_guess else None)
    ok = (ref["status"] == 0) & (out["status"] == 0)
    cols = [slice(b.col_off[c], b.col_off[c + 1]) for c in np.where(ok)[0]]
    err = max([float(np.abs(out[k][s] - ref[k][s]).max() / max(np.abs(ref[k][s]).max(), 1e-300))
               for k in ("ne", "phi") for s in cols] or [0.0])
    return {"word": word, "err": err, "ok": int(ok.sum()), "ncol": b.ncol}


def main():
    assert S.lib().sdcef_checks_compiled() == 1, "not the bounds-checking build"
    res = {}
    b = make_batch("ragged", 24, 1000, n_range=(2, 900))
    for tpc in (0, 32, 64, 256):
        res[f"fp64_exact_tpc{tpc}"] = solve_case(b, dict(eps_F=1e-12, threads_per_column=tpc),
                                                 dict(precond=2, eps_F=1e-12))
    br = make_batch("ragged", 8, 500, n_range=(100, 700), dt=1e-7)
    res["fp64_recast"] = solve_case(br, dict(eps_F=1e-12, precond=S.PREC_RECAST, restart_m=30),
                                    dict(precond=1, eps_F=1e-12, restart_m=30))
    res["mg"] = solve_case(br, dict(eps_F=1e-12, precond=S.PREC_MG, restart_m=30),
                           dict(precond=3, eps_F=1e-12, restart_m=30))
    bs = make_batch("single", 8, 1)
    res["mixed_fp32"] = solve_case(bs, dict(eps_F=1e-12, precision=S.MIXED, restart_m=16),
                                   dict(precond=2, eps_F=1e-12))
    res["mixed_df"] = solve_case(b, dict(eps_F=1e-12, precision=S.MIXED_DF),
                                 dict(precond=2, eps_F=1e-12))
    bt = make_batch("ragged", 10, 12, n_range=(2, 900), dt=1e-7)
    tab = transport_table()
    res["transport_table"] = solve_case(bt, dict(eps_F=1e-12, transport=S.TRANSPORT_TABLE),
                                        dict(precond=2, eps_F=1e-12, transport=1), table=tab)
    # the error test at the bench tolerance, and a rejected guess (restart path)
    bb = make_batch("ragged", 48, 4242)
    res["bench_tolerance_error_test"] = solve_case(bb, dict(), dict(precond=2))
    bg = make_batch("single", 6, 77, n_cells=300)
    rng = np.random.default_rng(9)
    guess = (bg.ne_old * (1 + 0.2 * rng.standard_normal(bg.ncells)),
             bg.phi_old + 5.0 * rng.standard_normal(bg.ncells))
    # the judged start is replaced by X^n: the root is the plain one
    res["rejected_guess"] = solve_case(bg, dict(eps_F=1e-12), dict(precond=2, eps_F=1e-12),
                                       guess=guess, oracle_guess=False)
    # provisional ions, current and the SDC sweep
    sb = sdc_batch(16, 5_000_000, n_cells=256)
    s = S.Solver(S.default_params(), max_cols=sb.ncol, max_cells=sb.ncells, max_col_cells=256)
    db = S.DeviceBatch.from_host(sb, D)
    phi = torch.as_tensor(sb.phi_old, device=D)
    ions = s.ion_provisional(db, phi).cpu().numpy()
    ref_ions = O.ion_provisional(sb, sb.phi_old)
    jp, jn = s.current(db, torch.as_tensor(sb.ne_old, device=D), phi)
    rjp, rjn = O.current(sb, sb.ne_old, sb.phi_old)
    out = s.sdc_sweep(db, 2)
    torch.cuda.synchronize()
    ne_s, phi_s, _ = O.sdc_sweep(sb, 2)
    res["fields_and_sweep"] = {
        "word": s.check_word(),
        "err": max(float(np.abs(ions - ref_ions).max() / np.abs(ref_ions).max()),
                   float(np.abs(jp.cpu().numpy() - rjp).max() / max(np.abs(rjp).max(), 1e-300)),
                   float(np.abs(jn.cpu().numpy() - rjn).max() / max(np.abs(rjn).max(), 1e-300)),
                   colerr(sb, out["ne"].cpu().numpy(), ne_s), colerr(sb, out["phi"].cpu().numpy(), phi_s)),
        "ok": int((out["status"] == 0).sum().item()), "ncol": sb.ncol}
    s.close()
    # the learned-guess kernels: features, fused guess, forward and gradients
    bm = make_batch("ragged", 9, 55, n_range=(2, 700))
    p = M.init_params(11)
    p["W1"][:, 25:] = 0.0
    flat = S.pack_params(p).astype(np.float32)
    q = S.unpack_params(flat.astype(np.float64))
    for k in ("W1", "W2", "W3"):
        q[k] = M.bf16_round(q[k])
    n = 700
    mlp = S.MLP(max(bm.ncells, n))
    mlp.set_params(flat)
    dbm = S.DeviceBatch.from_host(bm, D)
    X = mlp.features(dbm).float().cpu().numpy()
    ne_g, _ = mlp.guess(dbm, components=S.GUESS_NE)
    rng = np.random.default_rng(1)
    Xh = M.bf16_round(rng.standard_normal((n, 32)))
    Xh[:, 25:] = 0.0
    Xt = torch.as_tensor(Xh, dtype=torch.float32, device=D).to(torch.bfloat16)
    Th = rng.standard_normal((n, 2))
    g, _ = mlp.grad(Xt, torch.as_tensor(Th, dtype=torch.float32, device=D))
    Y = mlp.forward(Xt).cpu().numpy()
    mlp.check()
    Yr, cache = M.forward(q, Xh)
    _, dY = M.mse(Yr, Th)
    gr = M.backward(q, cache, dY)
    gg = S.unpack_params(g.cpu().numpy())
    Yg, _ = M.forward(q, M.bf16_round(M.features(bm)))
    sn, _ = M.column_scales(bm)
    yn = np.concatenate([(ne_g.cpu().numpy()[s] - bm.ne_old[s]) / sn[c]
                         for c, s in enumerate(slice(bm.col_off[c], bm.col_off[c + 1])
                                               for c in range(bm.ncol))])
    ref_feat = M.bf16_round(M.features(bm))
    errs = [float(np.abs(X - ref_feat).max() / np.abs(ref_feat).max()),
            float(np.abs(Y - Yr).max() / np.abs(Yr).max()),
            float(np.abs(yn - Yg[:, 0]).max() / np.abs(Yg[:, 0]).max())]
    for k in ("W2", "W3", "b2"):
        errs.append(float(np.abs(gg[k] - gr[k]).max() / np.abs(gr[k]).max()))
    res["mlp"] = {"word": mlp.check_word(), "err": max(errs), "ok": 1, "ncol": 1}
    mlp.close()
    print(json.dumps(res))
    return 0


if __name__ == "__main__":
    sys.exit(main())
