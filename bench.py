#!/usr/bin/env python
"""Benchmark: batched JFNK column-solves/s on one GB300 (per rank).

Workload (default): 4096 independent columns, cells per column uniform in
128..2048 on L = 1 cm, dt = 1e-5 s, flame position U(3, 7) mm, ion peak
log-uniform in [1e15, 1e17] m^-3, V_R ~ U(-500, 500) V (seeded synthetic
profiles standing in for the paper's flame data). One step = one
sdcef_solve_batch over the whole batch to ||S_F^-1 F||_inf < 1e-10.

Prints ONE JSON line (rank 0). Keys follow the benchmark contract: metric,
value (device-timed, inputs resident in HBM), e2e (host buffers through
sdcef_solve_batch_host, copies inside the timed region), roofline of the
solver kernel, cpu_baseline (the CPU oracle on a bounded sample), clocks.

--impl reference times the CPU oracle itself (the reference arm).
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "column-solves/s at rel. residual 1e-10 (batched/learned vs plain JFNK); HBM %"
# the learned Newton start: the predicted n_e increment and the potential of
# the guessed charge (root of the Poisson residual at that n_e)
LEARNED_START = 5
UNIT = "column-solves/s"
WORKLOAD = "4096 ragged columns, 128-2048 cells, L=1cm, dt=1e-5s, V_R~U(-500,500)V"
PEAKS_FILE = os.path.join(ROOT, "MEASURED_PEAKS.json")
# FP64 FMA pipe: 2 DFMA/clk/SM (the recipe's 1.25 TFLOP/s / (152 SM x 2.07 GHz x 2))
FP64_DFMA_PER_CLK_SM = 2.0


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=30)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="native", choices=["native", "reference"])
    ap.add_argument("--ncol", type=int, default=4096)
    ap.add_argument("--precision", default="fp64", choices=["fp64", "mixed", "mixed_df"])
    ap.add_argument("--precond", default="exact", choices=["exact", "recast"])
    ap.add_argument("--seed", type=int, default=2_000_000)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--cpu-seconds", type=float, default=15.0)
    ap.add_argument("--tpc", type=int, default=0, help="threads per column (0 = library default)")
    ap.add_argument("--krylov-on-chip", type=int, default=-1, choices=[-1, 0, 1],
                    help="Krylov vectors in the solver kernel's spare shared memory (1), all in "
                         "the workspace slot (0), or picked by the autotuner (-1)")
    ap.add_argument("--no-extras", action="store_true",
                    help="skip the unbatched / learned / SDC-sweep comparison legs")
    ap.add_argument("--sdc-ncol", type=int, default=16384)
    return ap.parse_args()


from paper_1904_08510_gb300.replicas import dist_info, job_throughput, max_over_ranks, shard_seed  # noqa: E402


def load_peaks():
    try:
        with open(PEAKS_FILE) as f:
            return json.load(f), "measured"
    except Exception:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "sm_max_mhz": 2070.0}, "fallback"


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.path = None

    def __enter__(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.Q}", "--format=csv,noheader,nounits",
                 "-lms", "100", "-f", self.path], stdout=subprocess.DEVNULL, stderr=subprocess.DEVNULL)
            # the timed region starts only once the sampler is producing samples
            t0 = time.time()
            while time.time() - t0 < 5.0 and os.path.getsize(self.path) == 0:
                time.sleep(0.02)
        except Exception:
            self.proc = None
        return self

    def __exit__(self, *exc):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        if not self.path or not os.path.exists(self.path):
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unavailable"]}
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx.append(float(f[2]))
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        os.unlink(self.path)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(mx) if mx else None, "samples": len(sm),
                "reasons": sorted(reasons)}


def kernel_digest():
    """Digest of the solver kernel sources (ties an ncu capture to the code it measured)."""
    import hashlib
    h = hashlib.sha256()
    for f in ("solver.cuh", "blockalg.cuh", "checks.cuh", "dfloat.cuh", "mg.cuh", "expm1_table.cuh",
              "kern_inst.cu"):
        with open(os.path.join(ROOT, "paper_1904_08510_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def ncu_traffic(ncells, tpc, on_chip):
    """DRAM bytes per launch of the solver kernel from the committed ncu summary, if it
    was taken on the current kernel sources and launch shape (else None), scaled to
    this batch's cells."""
    path = os.path.join(ROOT, "profiles", "jfnk_kernel_counters.json")
    try:
        with open(path) as f:
            c = json.load(f)
    except Exception:
        return None
    if c.get("kernel_digest") != kernel_digest() or int(c.get("threads_per_column", -1)) != tpc:
        return None
    cap = c.get("captures", {}).get(str(int(on_chip)))
    if not cap:
        return None
    return float(cap["dram_bytes_per_launch"]) * ncells / float(c["cells"])


def algorithmic_model(lengths, newton, krylov, res_evals, precond, kr_bytes):
    """Algorithmic FP64 flops and streaming-model bytes of the solve (per batch).

    Per cell: a residual evaluation ~ 40 FP64 flops + one e^x - 1 and one
    reciprocal per face (counted as 26 + 9 flop-equivalents: 13 and ~4.5
    FMA-class operations), 75 in all, inside the 60-80 per cell per residual
    of the path's scope analysis; a block
    factorisation ~ 120 flops per Newton step; a preconditioner application
    ~ 40 flops (exact form) or 30 (recast); Arnoldi CGS2 with a basis of p
    vectors ~ 8 (p+1) flops per iteration. Streaming-model bytes per cell
    follow the same count with 8-byte state and `kr_bytes` Krylov data:
    residual 56 B, factorisation 40 + 18 s, iteration 40 + 19 s + 4 s (p+1).
    """
    N = lengths.astype(np.float64)
    res = res_evals.astype(np.float64)
    nw = newton.astype(np.float64)
    kr = krylov.astype(np.float64)
    it_per = np.where(nw > 0, kr / np.maximum(nw, 1), 0.0)
    p_mean = 0.5 * it_per + 1.0
    pa = 40.0 if precond == "exact" else 30.0
    flop_cell = res * 75.0 + nw * 120.0 + (kr + nw) * 2 * pa + kr * 8.0 * (p_mean + 1) * 2
    s = float(kr_bytes)
    byte_cell = 56.0 + res * 56.0 + nw * (40 + 18 * s) + kr * (40 + 19 * s + 4 * s * (p_mean + 1)) + 48 * nw
    return float(np.sum(flop_cell * N)), float(np.sum(byte_cell * N))


def parity_sample(b, n_rand=54, seed=0):
    """Columns compared with the oracle: the shortest, the longest, the eight
    with the smallest |V_R| (the worst-conditioned scaled Jacobians) and a
    seeded draw."""
    lens = b.lengths()
    cols = {int(np.argmin(lens)), int(np.argmax(lens))}
    cols |= set(int(c) for c in np.argsort(np.abs(b.v_right))[:8])
    rng = np.random.default_rng(seed)
    cols |= set(int(c) for c in rng.choice(b.ncol, min(n_rand, b.ncol), replace=False))
    return sorted(cols)


def err_vs_oracle(parity):
    """Max-norm relative error per column and field of each GPU leg against the
    oracle's root converged to its rounding floor (eps_F = 1e-13, error test at
    1e-14), on a sample of each batch's columns."""
    import oracle as O
    out = {}
    for family, (b, legs) in parity.items():
        cols = parity_sample(b)
        sub = b.subset(cols)
        ref = O.solve(sub, O.default_params(precond=2, eps_F=1e-13, max_linesearch=6, eps_E=1e-14))
        ok = np.isin(ref["status"], [0, 3]) & (ref["final_res"] < 1e-10)
        fam = {"columns": len(cols), "reference_ok": int(ok.sum())}
        for leg, (ne, phi) in legs.items():
            en, ep = [], []
            for k, c in enumerate(cols):
                if not ok[k]:
                    continue
                s = slice(int(b.col_off[c]), int(b.col_off[c + 1]))
                r = slice(int(sub.col_off[k]), int(sub.col_off[k + 1]))
                en.append(np.abs(ne[s] - ref["ne"][r]).max() / np.abs(ref["ne"][r]).max())
                ep.append(np.abs(phi[s] - ref["phi"][r]).max() / np.abs(ref["phi"][r]).max())
            fam[leg] = {"ne_max": float(np.max(en)), "phi_max": float(np.max(ep)),
                        "ne_median": float(np.median(en)), "phi_median": float(np.median(ep))}
        out[family] = fam
    return out


def cpu_baseline(batch, seconds, precond, parity=None):
    """The CPU oracle on a bounded prefix sample of the same workload; with
    parity, also the GPU legs' errors against the oracle's converged root."""
    import oracle as O
    P = O.default_params(precond=2 if precond == "exact" else 1,
                         restart_m=30 if precond == "recast" else 30)
    threads = O.max_threads()
    # calibrate on a few columns, then size the sample to ~`seconds`
    k = min(batch.ncol, 2 * threads)
    t0 = time.perf_counter()
    O.solve(batch.subset(range(k)), P, threads=threads)
    dt = max(time.perf_counter() - t0, 1e-3)
    m = int(min(batch.ncol, max(k, k * seconds / dt)))
    sub = batch.subset(range(m))
    t0 = time.perf_counter()
    r = O.solve(sub, P, threads=threads)
    el = time.perf_counter() - t0
    # one core: a prefix sized to about 2 s from the all-core rate
    m1 = int(min(m, max(min(m, 8), 2.0 * m / (el * threads))))
    t0 = time.perf_counter()
    O.solve(batch.subset(range(m1)), P, threads=1)
    el1 = time.perf_counter() - t0
    errs = err_vs_oracle(parity) if parity else None
    return {"value": m / el, "unit": UNIT, "cores": threads, "kind": "oracle",
            "value_1core": m1 / el1, "err_vs_oracle": errs,
            "sample": f"first {m} of {batch.ncol} columns ({int(sub.ncells)} cells), "
                      f"{el:.1f} s on {threads} threads, status OK {int((r['status'] == 0).sum())}/{m}; "
                      f"1 core: first {m1} columns, {el1:.2f} s"}


def run_reference(args):
    ws, rank, _ = dist_info()
    if rank != 0:
        return 0
    from paper_1904_08510_gb300.workload import make_batch
    b = make_batch("ragged", args.ncol, args.seed)
    import oracle as O
    P = O.default_params(precond=2 if args.precond == "exact" else 1)
    threads = O.max_threads()
    # bounded sample per step: columns costing ~ (budget / (steps+warmup)) seconds
    budget = 150.0
    k = min(b.ncol, 2 * threads)
    t0 = time.perf_counter()
    O.solve(b.subset(range(k)), P, threads=threads)
    per_col = max(time.perf_counter() - t0, 1e-3) / k
    m = int(max(k, min(b.ncol, budget / (args.steps + args.warmup) / per_col)))
    sub = b.subset(range(m))
    for _ in range(args.warmup):
        O.solve(sub, P, threads=threads)
    times = []
    for _ in range(args.steps):
        t0 = time.perf_counter()
        O.solve(sub, P, threads=threads)
        times.append(time.perf_counter() - t0)
    tot = sum(times)
    val = m * args.steps / tot
    line = {"impl": "reference", "metric": METRIC, "value": val, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * tot / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic (seeded profiles; the paper's flame data is not available)",
            "config": {"workload": WORKLOAD, "ncol": args.ncol, "sample_columns": m,
                       "precond": args.precond, "eps_F": 1e-10},
            "cpu_baseline": {"value": val, "unit": UNIT, "cores": threads, "kind": "oracle",
                             "sample": f"first {m} of {b.ncol} columns per step"},
            "e2e": {"value": val, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))
    return 0


def main():
    args = parse()
    if args.impl == "reference":
        return run_reference(args)
    import torch
    ws, rank, local = dist_info()
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    torch.cuda.set_device(local)
    dev = f"cuda:{local}"
    from paper_1904_08510_gb300 import sdcef as S
    from paper_1904_08510_gb300.workload import make_batch
    # weak scaling: each rank solves its own batch (independent columns, no exchange)
    b = make_batch("ragged", args.ncol, shard_seed(args.seed, rank, args.ncol))
    lengths = b.lengths()
    prec = {"fp64": S.FP64, "mixed": S.MIXED, "mixed_df": S.MIXED_DF}[args.precision]
    pc = S.PREC_EXACT if args.precond == "exact" else S.PREC_RECAST
    params = S.default_params(precision=prec, precond=pc, threads_per_column=args.tpc,
                              restart_m=30 if pc == S.PREC_RECAST else (16 if prec == S.MIXED else 8),
                              krylov_on_chip=max(args.krylov_on_chip, 0))
    solver = S.Solver(params, max_cols=b.ncol, max_cells=b.ncells,
                      max_col_cells=int(lengths.max()))
    db = S.DeviceBatch.from_host(b, dev)
    tuned = None
    if args.tpc == 0:
        tuned = solver.autotune(db, reps=1)   # before warm-up and timing
    tuned_oc = None
    if args.krylov_on_chip < 0:
        tuned_oc = solver.autotune_on_chip(db, reps=2)
    on_chip = int(solver.params.krylov_on_chip)
    out = solver.alloc_result(db)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    stream = torch.cuda.current_stream()
    for _ in range(max(args.warmup, 3)):
        solver.solve(db, out)
    torch.cuda.synchronize()
    launches_per_step = solver.launches()

    def barrier():
        if ws > 1:
            import torch.distributed as dist
            dist.barrier()
        torch.cuda.synchronize()

    # device-timed steps: inputs resident in HBM; L2 flushed between steps
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for _ in range(args.steps)]
    with ClockSampler(local) as clk:
        barrier()
        for i in range(args.steps):
            flush.zero_()
            ev[i][0].record(stream)
            solver.solve(db, out)
            ev[i][1].record(stream)
        barrier()
    ms = [a.elapsed_time(bb) for a, bb in ev]
    tot_ms = max_over_ranks(float(sum(ms)), device=dev)
    # denominators of the ALU roofline, measured on this GPU after the timed region
    fp64_peak = S.fma_peak_probe(S.FP64, 100)
    fp32_peak = S.fma_peak_probe(S.MIXED, 4000)
    value = job_throughput(b.ncol, ws, args.steps, tot_ms / 1e3)
    st = out["status"].cpu().numpy()
    nw = out["newton_it"].cpu().numpy()
    kr = out["krylov_it"].cpu().numpy()
    re = out["res_evals"].cpu().numpy()
    fr = out["final_res"].cpu().numpy()

    # end to end: host buffers through sdcef_solve_batch_host (copies timed)
    e2e = None
    if not args.no_e2e:
        pin = lambda a: torch.as_tensor(np.ascontiguousarray(a)).pin_memory()
        hb = type(b)(col_off=pin(b.col_off), length=pin(b.length), dt=pin(b.dt),
                     v_left=pin(b.v_left), v_right=pin(b.v_right), ne_old=pin(b.ne_old),
                     phi_old=pin(b.phi_old), n_ion=pin(np.atleast_2d(b.n_ion)),
                     valence=b.valence, T=pin(b.T), rho=pin(b.rho))
        hb.col_off_np = b.col_off
        hout = {k: torch.empty(v.shape, dtype=v.dtype).pin_memory() for k, v in out.items()}
        solver.solve_host(_HostView(hb, b), hout)
        e2e_t = []
        for _ in range(args.steps):
            flush.zero_()
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            solver.solve_host(_HostView(hb, b), hout)
            e2e_t.append(time.perf_counter() - t0)
        serial = b.ncol * ws * args.steps / sum(e2e_t)
        # the same K steps through one sdcef_solve_batches_host call: step k+1's
        # inputs and step k-1's results cross PCIe/C2C while step k is solved
        # (inputs larger than L2, so no flush between the steps of the call)
        hout2 = [hout, {k: torch.empty_like(v).pin_memory() for k, v in hout.items()}]
        solver.solve_host_many([_HostView(hb, b)] * 2, hout2)
        flush.zero_()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        solver.solve_host_many([_HostView(hb, b)] * args.steps,
                               [hout2[k & 1] for k in range(args.steps)])
        piped_s = time.perf_counter() - t0
        h2d = int(8 * (b.ncol + 1) + 4 * 8 * b.ncol + 8 * b.ncells * (3 + b.n_ion.shape[0]))
        d2h = int(16 * b.ncells + b.ncol * (4 * 4 + 8))
        e2e = {"value": b.ncol * ws * args.steps / piped_s, "unit": UNIT,
               "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h,
               "api": "sdcef_solve_batches_host (copies of the neighbouring steps overlap each solve)",
               "serial_value": serial,
               "serial_api": "sdcef_solve_batch_host per step (copy in, solve, copy out; L2 flushed between steps)"}

    extra = None
    parity = {"headline": (b, {f"plain_{args.precision}": (out["ne"].cpu().numpy(),
                                                         out["phi"].cpu().numpy())})}
    if not args.no_extras and ws == 1:
        extra = extras(args, S, b, db, solver, params, dev, parity)
    if rank != 0:
        return 0
    peaks, peak_kind = load_peaks()
    flops, sbytes = algorithmic_model(lengths, nw, kr, re, args.precond, 4 if prec == S.MIXED else 8)
    t_launch = tot_ms / args.steps / 1e3
    clocks = clk.summary()
    sm_clk = clocks.get("sm_mhz") or peaks.get("sm_max_mhz", 2070.0)
    fp64_nominal = 152 * FP64_DFMA_PER_CLK_SM * 2 * float(peaks.get("sm_max_mhz", 2070.0)) * 1e6 / 1e12
    achieved_tf = flops / t_launch / 1e12
    hbm_gbs = sbytes / t_launch / 1e9
    roofline = {"bound": "alu", "achieved": achieved_tf, "peak": fp64_peak, "unit": "TFLOP/s",
                "frac": achieved_tf / fp64_peak, "traffic": ncu_traffic(b.ncells, tuned[0] if tuned else args.tpc,
                                                       on_chip),
                "kernel": "jfnk_kernel (persistent solver)",
                "peak_source": "measured in this run: sdcef_fma_peak_probe, FP64 FMA chains on every SM, "
                               "best of 5 CUDA-event timings",
                "peak_nominal": {"value": fp64_nominal, "unit": "TFLOP/s",
                                 "how": "2 DFMA/clk/SM x 152 SM x max SM clock"},
                "fp32_fma_measured_tflops": fp32_peak,
                "streaming_model": {"achieved": hbm_gbs, "peak": peaks["hbm_gbs"], "unit": "GB/s",
                                    "frac": hbm_gbs / peaks["hbm_gbs"], "peak_kind": peak_kind}}
    if roofline["traffic"] is not None:
        # measured DRAM bytes (ncu) over the live launch time: the third figure
        dram = roofline["traffic"] / t_launch / 1e9
        roofline["ncu_dram"] = {"achieved": dram, "peak": peaks["hbm_gbs"], "unit": "GB/s",
                                "frac": dram / peaks["hbm_gbs"], "peak_kind": peak_kind}
    cpu = None
    if not args.no_cpu_baseline and ws == 1:
        cpu = cpu_baseline(b, args.cpu_seconds, args.precond, parity)
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
            "warmup": max(args.warmup, 3), "ms_per_step": tot_ms / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": {S.FP64: "f64", S.MIXED: "f64+f32", S.MIXED_DF: "f64+f32x2"}[prec],
            "data": "synthetic (seeded profiles; the paper's flame data is not available)",
            "config": {"workload": WORKLOAD, "ncol": b.ncol, "cells": int(b.ncells),
                       "precision": args.precision, "precond": args.precond, "eps_F": 1e-10,
                       "threads_per_column": (tuned[0] if tuned else args.tpc),
                       "krylov_on_chip": on_chip,
                       "krylov_on_chip_ms": (tuned_oc[1] if tuned_oc else None),
                       "autotune_ms": (tuned[1] if tuned else None),
                       "l2": "flushed between steps (256 MB write); inputs 5 x 8 B x cells > L2",
                       "parallelism": f"replicas x{ws}"},
            "e2e": e2e, "gpu_launches": launches_per_step * args.steps,
            "err_vs_oracle": cpu["err_vs_oracle"] if cpu else None,
            "roofline": roofline, "cpu_baseline": cpu, "clocks": clocks, "comparisons": extra,
            "solve_stats": {"status_ok": int((st == 0).sum()), "ncol": int(b.ncol),
                            "status_hist": np.bincount(st, minlength=6).tolist(),
                            "newton_mean": float(nw.mean()), "krylov_mean": float(kr.mean()),
                            "res_evals_mean": float(re.mean()), "final_res_max": float(fr.max()),
                            "step_ms": ms}}
    if extra and "headline_workload_learned" in extra:
        # the learned start on this batch, beside the plain batched solve above
        # (the network, the guess kernel and the solve; details in comparisons)
        lw, ld = extra["headline_workload_learned"], extra.get("headline_workload_mixed_df_learned", {})
        line["learned_start"] = {
            "value": lw["value"], "unit": UNIT, "vs_plain_batched": lw["value"] / value,
            "mixed_df_value": ld.get("value"),
            "newton_per_column": [float(nw.mean()), lw.get("newton_mean")],
            "gmres_per_column": [float(kr.mean()), lw.get("krylov_mean")],
            "status_ok": lw.get("status_ok"),
            "note": "FP64 solve from the learned start (n_e from the network, phi the root of the "
                    "Poisson residual at that n_e), timed including the guess kernel; "
                    "iterations as [plain, learned]"}
    print(json.dumps(line))
    return 0


def _timed(fn, reps=3):
    """Best-of-reps CUDA-event time (s) of fn() on the current stream, after one warm-up."""
    import torch
    fn()
    torch.cuda.synchronize()
    best = None
    for _ in range(reps):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        out = fn()
        e1.record()
        torch.cuda.synchronize()
        t = e0.elapsed_time(e1) / 1e3
        best = t if best is None or t < best else best
    return best, out


def _colerr(b, a, ref):
    return np.array([np.abs(a[s] - ref[s]).max() / max(np.abs(ref[s]).max(), 1e-300)
                     for s in (slice(b.col_off[c], b.col_off[c + 1]) for c in range(b.ncol))])


def extras(args, S, b, db, solver, params, dev, parity):
    """The other configurations of the benchmark, reported beside the headline
    (not part of `value`): single column, unbatched comparator, mixed precision,
    learned guess, SDC electric sweep. The learned legs' roots are added to
    `parity` (family -> (batch, {leg: (ne, phi)})) for the comparison with the
    oracle in the CPU-baseline leg."""
    import torch
    from paper_1904_08510_gb300 import learned as Lrn
    from paper_1904_08510_gb300.workload import make_batch, sdc_batch
    res = {}
    # config 1: one 256-cell column, one launch
    b1 = make_batch("single", 1, 1)
    db1 = S.DeviceBatch.from_host(b1, dev)
    s1 = S.Solver(params, max_cols=1, max_cells=256, max_col_cells=256)
    o1 = s1.alloc_result(db1)
    t1, _ = _timed(lambda: s1.solve(db1, o1), reps=5)
    res["config1_single_column_fp64"] = {"ms_per_solve": 1e3 * t1, "cells": 256,
                                         "newton": int(o1["newton_it"].item()),
                                         "status": int(o1["status"].item())}
    s1.close()
    # plain unbatched FP64 JFNK on the headline workload: one column per launch, looped
    m = min(64, b.ncol)
    cols = [S.DeviceBatch.from_host(b.column(c), dev) for c in range(m)]
    one = S.Solver(params, max_cols=1, max_cells=int(b.lengths()[:m].max()),
                   max_col_cells=int(b.lengths()[:m].max()))
    outs = [one.alloc_result(c) for c in cols]

    def loop():
        for c, o in zip(cols, outs):
            one.solve(c, o)
    t, _ = _timed(loop, reps=2)
    res["plain_unbatched_fp64"] = {"value": m / t, "unit": "column-solves/s", "columns": m,
                                   "launches_per_column": 2}
    one.close()
    # config 3: the 256-cell batch in the mixed modes (FP32 and double-float
    # preconditioner), error against the FP64 GPU path; then the double-float
    # mode on the headline workload
    b3 = make_batch("single", 4096, 1)
    db3 = S.DeviceBatch.from_host(b3, dev)
    s64 = S.Solver(params, max_cols=b3.ncol, max_cells=b3.ncells, max_col_cells=256)
    t64, o64 = _timed(lambda: s64.solve(db3))
    res["config3_mixed_vs_fp64"] = {"columns": b3.ncol, "cells": 256, "unit": "column-solves/s",
                                    "fp64_value": b3.ncol / t64,
                                    "fp64_status_ok": int((o64["status"] == 0).sum().item())}
    for name, prec, m in (("mixed", S.MIXED, 16), ("mixed_df", S.MIXED_DF, 8)):
        sm = S.Solver(S.default_params(precision=prec, restart_m=m), max_cols=b3.ncol,
                      max_cells=b3.ncells, max_col_cells=256)
        tm, om = _timed(lambda: sm.solve(db3))
        okc = ((o64["status"] == 0) & (om["status"] == 0)).cpu().numpy()
        en = _colerr(b3, om["ne"].cpu().numpy(), o64["ne"].cpu().numpy())[okc]
        ep = _colerr(b3, om["phi"].cpu().numpy(), o64["phi"].cpu().numpy())[okc]
        res["config3_mixed_vs_fp64"].update({
            f"{name}_value": b3.ncol / tm, f"{name}_status_ok": int((om["status"] == 0).sum().item()),
            f"{name}_krylov_mean": float(om["krylov_it"].float().mean().item()),
            f"{name}_err_vs_fp64_ne": {"max": float(en.max()), "median": float(np.median(en))},
            f"{name}_err_vs_fp64_phi": {"max": float(ep.max()), "median": float(np.median(ep))}})
        sm.close()
    res["config3_mixed_vs_fp64"]["note"] = ("the FP64 GPU path itself matches the CPU oracle to 1e-9 "
                                            "(tests/test_gpu_parity.py)")
    s64.close()
    if args.precision == "fp64":
        pdf = S.default_params(precision=S.MIXED_DF, precond=params.precond, restart_m=8,
                               threads_per_column=params.threads_per_column)
        sdf = S.Solver(pdf, max_cols=b.ncol, max_cells=b.ncells, max_col_cells=int(b.lengths().max()))
        if not pdf.threads_per_column:
            sdf.autotune(db, reps=1)
        o_ref = solver.solve(db)
        tdf, odf = _timed(lambda: sdf.solve(db))
        okc = ((o_ref["status"] == 0) & (odf["status"] == 0)).cpu().numpy()
        en = _colerr(b, odf["ne"].cpu().numpy(), o_ref["ne"].cpu().numpy())[okc]
        ep = _colerr(b, odf["phi"].cpu().numpy(), o_ref["phi"].cpu().numpy())[okc]
        res["headline_workload_mixed_df"] = {
            "value": b.ncol / tdf, "unit": "column-solves/s",
            "status_ok": int((odf["status"] == 0).sum().item()),
            "newton_mean": float(odf["newton_it"].float().mean().item()),
            "krylov_mean": float(odf["krylov_it"].float().mean().item()),
            "err_vs_fp64_ne": {"max": float(en.max()), "median": float(np.median(en))},
            "err_vs_fp64_phi": {"max": float(ep.max()), "median": float(np.median(ep))}}
        sdf.close()
    # learned Newton start on the headline workload, with the network trained on
    # the same (ragged) profile family from disjoint seeds; timed including the
    # guess kernel, plain FP64 and with the double-float preconditioner
    if args.precision == "fp64" and os.path.exists(Lrn.WEIGHTS_RAGGED):
        mlp = S.MLP(b.ncells)
        mlp.set_params(Lrn.load(Lrn.WEIGHTS_RAGGED))
        ne_g = torch.empty(b.ncells, dtype=torch.float64, device=dev)
        ph_g = torch.empty_like(ne_g)
        gdb = db.with_guess(ne_g, ph_g)
        o_ref = solver.solve(db)
        legs = {}
        for name, prec, rm in (("headline_workload_learned", S.FP64, 8),
                               ("headline_workload_mixed_df_learned", S.MIXED_DF, 8),
                               ("headline_workload_mixed_learned", S.MIXED, 16)):
            sl = S.Solver(S.default_params(precision=prec, precond=params.precond, restart_m=rm,
                                           threads_per_column=params.threads_per_column),
                          max_cols=b.ncol, max_cells=b.ncells, max_col_cells=int(b.lengths().max()))
            ol_ = sl.alloc_result(db)

            def learned(sl=sl, ol_=ol_):
                mlp.guess(db, ne_g, ph_g, components=LEARNED_START)
                return sl.solve(gdb, ol_)
            tl, ol = _timed(learned)
            okc = ((o_ref["status"] == 0) & (ol["status"] == 0)).cpu().numpy()
            en = _colerr(b, ol["ne"].cpu().numpy(), o_ref["ne"].cpu().numpy())[okc]
            ep = _colerr(b, ol["phi"].cpu().numpy(), o_ref["phi"].cpu().numpy())[okc]
            res[name] = {"value": b.ncol / tl, "unit": "column-solves/s",
                         "status_ok": int((ol["status"] == 0).sum().item()), **_iterations(ol),
                         "err_vs_plain_fp64_ne": {"max": float(en.max()), "median": float(np.median(en))},
                         "err_vs_plain_fp64_phi": {"max": float(ep.max()), "median": float(np.median(ep))},
                         "err_vs_oracle": "see err_vs_oracle.headline." + name}
            parity["headline"][1][name] = (ol["ne"].cpu().numpy(), ol["phi"].cpu().numpy())
            sl.close()
        res["headline_workload_plain_iterations"] = _iterations(o_ref)
        mlp.close()
    # config 4: learned initial guess on held-out columns (512-2048 cells)
    if os.path.exists(Lrn.WEIGHTS):
        b4 = make_batch("single", 4096, 2_000_000, n_range=(512, 2048))
        db4 = S.DeviceBatch.from_host(b4, dev)
        s4 = S.Solver(params, max_cols=b4.ncol, max_cells=b4.ncells,
                      max_col_cells=int(b4.lengths().max()))
        mlp = S.MLP(b4.ncells)
        mlp.set_params(Lrn.load())
        ne_g = torch.empty(b4.ncells, dtype=torch.float64, device=dev)
        ph_g = torch.empty_like(ne_g)
        out4 = s4.alloc_result(db4)
        tp, op = _timed(lambda: s4.solve(db4))

        def learned():
            mlp.guess(db4, ne_g, ph_g, components=LEARNED_START)
            return s4.solve(db4.with_guess(ne_g, ph_g), out4)
        tl, ol = _timed(learned)
        parity["holdout"] = (b4, {"plain_fp64": (op["ne"].cpu().numpy(), op["phi"].cpu().numpy()),
                                  "learned_fp64": (ol["ne"].cpu().numpy(), ol["phi"].cpu().numpy())})
        tg, _ = _timed(lambda: mlp.guess(db4, ne_g, ph_g, components=LEARNED_START))
        res["config4_learned_guess"] = {
            "columns": b4.ncol, "cells": "512-2048",
            "plain": {"value": b4.ncol / tp, **_iterations(op),
                      "status_ok": int((op["status"] == 0).sum().item())},
            "learned": {"value": b4.ncol / tl, **_iterations(ol),
                        "status_ok": int((ol["status"] == 0).sum().item()),
                        "guess_kernel_ms": 1e3 * tg},
            "unit": "column-solves/s",
            "components": "n_e increment; potential of the guessed charge (root of F_phi)"}
        mlp.close()
        s4.close()
    # config 5: SDC electric sweep, k_max = 4 solves per MISDC step, ion-CFL step, CUDA graph
    sb = sdc_batch(args.sdc_ncol, 5_000_000, n_cells=1024)
    sdb = S.DeviceBatch.from_host(sb, dev)
    st_ = torch.cuda.Stream()
    ssolver = S.Solver(params, max_cols=sb.ncol, max_cells=sb.ncells, max_col_cells=1024, stream=st_)
    sout = ssolver.alloc_result(sdb)
    work = ssolver.sweep_work(sdb)
    with torch.cuda.stream(st_):
        te, _ = _timed(lambda: ssolver.sdc_sweep(sdb, 4, work=work, out=sout), reps=2)
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g, stream=st_):
            ssolver.sdc_sweep(sdb, 4, work=work, out=sout)
        tg, _ = _timed(lambda: g.replay(), reps=2)
    sst = sout["status"].cpu().numpy()
    res["config5_sdc_sweep_fp64"] = {
        "columns": sb.ncol, "cells_per_column": 1024, "k_max": 4,
        "ms_per_sweep_eager": 1e3 * te, "ms_per_sweep_graph": 1e3 * tg,
        "column_solves_per_s_graph": 4 * sb.ncol / tg,
        "status_ok_last_iteration": int((sst == 0).sum()),
        "newton_mean_last_iteration": float(sout["newton_it"].float().mean().item())}
    # the same sweep with the double-float preconditioner, without and with the
    # learned Newton start of the first SDC iteration (the network trained on
    # that iteration's solves, learned.py --family sweep): guess kernel + 4
    # solves in one CUDA graph
    wpath = Lrn.WEIGHTS_SWEEP if os.path.exists(Lrn.WEIGHTS_SWEEP) else Lrn.WEIGHTS
    if os.path.exists(wpath):
        pdf = S.default_params(precision=S.MIXED_DF, restart_m=8,
                               threads_per_column=params.threads_per_column)
        dsolver = S.Solver(pdf, max_cols=sb.ncol, max_cells=sb.ncells, max_col_cells=1024, stream=st_)
        dout0 = dsolver.alloc_result(sdb)
        with torch.cuda.stream(st_):
            g1 = torch.cuda.CUDAGraph()
            with torch.cuda.graph(g1, stream=st_):
                dsolver.sdc_sweep(sdb, 4, work=work, out=dout0)
            tdg, _ = _timed(lambda: g1.replay(), reps=2)
        res["config5_sdc_sweep_mixed_df"] = {
            "ms_per_sweep_graph": 1e3 * tdg, "column_solves_per_s_graph": 4 * sb.ncol / tdg,
            "speedup_vs_fp64_graph": tg / tdg,
            "status_ok_last_iteration": int((dout0["status"] == 0).sum().item())}
        mlp5 = S.MLP(sb.ncells, stream=st_)
        mlp5.set_params(Lrn.load(wpath))
        g_ne = torch.empty(sb.ncells, dtype=torch.float64, device=dev)
        g_ph = torch.empty_like(g_ne)
        gdb = sdb.with_guess(g_ne, g_ph)
        dout = dsolver.alloc_result(sdb)

        def mixed_learned():
            mlp5.guess(sdb, g_ne, g_ph, components=LEARNED_START)
            return dsolver.sdc_sweep(gdb, 4, work=work, out=dout)
        with torch.cuda.stream(st_):
            tme, _ = _timed(mixed_learned, reps=2)
            g2 = torch.cuda.CUDAGraph()
            with torch.cuda.graph(g2, stream=st_):
                mixed_learned()
            tmg, _ = _timed(lambda: g2.replay(), reps=2)
        okc = ((sout["status"] == 0) & (dout["status"] == 0)).cpu().numpy()
        en = _colerr(sb, dout["ne"].cpu().numpy(), sout["ne"].cpu().numpy())[okc]
        ep = _colerr(sb, dout["phi"].cpu().numpy(), sout["phi"].cpu().numpy())[okc]
        res["config5_sdc_sweep_mixed_df_learned"] = {
            "weights": os.path.basename(wpath),
            "ms_per_sweep_eager": 1e3 * tme, "ms_per_sweep_graph": 1e3 * tmg,
            "column_solves_per_s_graph": 4 * sb.ncol / tmg, "speedup_vs_fp64_graph": tg / tmg,
            "status_ok_last_iteration": int((dout["status"] == 0).sum().item()),
            "newton_mean_last_iteration": float(dout["newton_it"].float().mean().item()),
            "err_vs_fp64_sweep_ne": {"max": float(en.max()), "median": float(np.median(en))},
            "err_vs_fp64_sweep_phi": {"max": float(ep.max()), "median": float(np.median(ep))}}
        mlp5.close()
        dsolver.close()
        # the first SDC iteration alone (the one the learned start applies to):
        # Newton / GMRES iterations and time with and without it, FP64
        res["config5_first_iteration_learned"] = {
            "weights": os.path.basename(wpath), "columns": sb.ncol, "cells_per_column": 1024,
            **Lrn.evaluate_sweep(Lrn.load(wpath), sb.ncol, 5_000_000, n_cells=1024, device=dev)}
    ssolver.close()
    res["multigrid_block_solver"] = mg_study(S, dev)
    res["current_iv_sweep"] = iv_sweep(S, dev)
    res["field_dependent_transport"] = transport_leg(S, b, db, dev)
    res["mlp_training"] = mlp_training_leg(S, dev)
    return res


# One training step is one fused kernel (forward, loss, backward; activations
# never leave the chip) and the Adam / partial-sum kernel. Algorithmic work per
# sample: the BF16 products forward 2 (32 128 + 128 128 + 128 2) and backward
# dH1 2 128 128, gW2 2 128 128, gW1 2 128 32, gW3 2 2 128 flops; compulsory
# bytes X 64 + T 8. Per step: the weights (44 KB per CTA, from L2) and the
# per-CTA partial gradients (84 KB each, written and summed).
MLP_STEP_FLOPS_PER_SAMPLE = (2 * (32 * 128 + 128 * 128 + 128 * 2) + 2 * 128 * 128 * 2
                             + 2 * 128 * 32 + 2 * 2 * 128)
MLP_STEP_BYTES_PER_SAMPLE = 64 + 8
# the earlier unfused step (forward kernel, four split-K backward GEMMs, Adam)
# moved each operand once through HBM: 2960 bytes per sample
MLP_UNFUSED_BYTES_PER_SAMPLE = 1100 + 260 + 512 + 768 + 320


def mlp_training_leg(S, dev):
    """One Adam step of the learned-guess network (forward, MSE loss and the
    whole backward pass in one persistent tcgen05 kernel, then Adam over its
    per-CTA partial gradients) on synthetic features, at the training batch and
    at a streaming size; the epoch estimate is for the 51.2 M samples of 200k
    solves x 256 cells."""
    import torch
    peaks, peak_kind = load_peaks()
    out = {}
    rng = np.random.default_rng(12)
    for n in (32768, 262144):
        X = torch.as_tensor(rng.standard_normal((n, 32)), dtype=torch.float32)
        X[:, 25:] = 0.0
        X = X.to(torch.bfloat16).to(dev)
        T = torch.as_tensor(rng.standard_normal((n, 2)), dtype=torch.float32, device=dev)
        mlp = S.MLP(n)
        mlp.set_params((0.05 * rng.standard_normal(S.MLP_NPARAM)).astype(np.float32))
        reps = 10

        def steps():
            for _ in range(reps):
                mlp.train_step(X, T, 1e-4)
        t, _ = _timed(steps, reps=3)
        t /= reps
        tf = MLP_STEP_FLOPS_PER_SAMPLE * n / t / 1e12
        out[f"batch_{n}"] = {
            "us_per_step": 1e6 * t, "samples_per_s": n / t, "epoch_s_51_2M": 51.2e6 * t / n,
            "launches_per_step": mlp.launches(),
            "algorithmic": {"flops_per_sample": MLP_STEP_FLOPS_PER_SAMPLE, "achieved": tf,
                            "peak": peaks["bf16_tflops"], "unit": "TFLOP/s",
                            "frac": tf / peaks["bf16_tflops"], "peak_kind": peak_kind,
                            "bound": "latency: the per-tile chain of MMA waits and epilogues"},
            "bytes": {"per_sample": MLP_STEP_BYTES_PER_SAMPLE,
                      "achieved": MLP_STEP_BYTES_PER_SAMPLE * n / t / 1e9, "unit": "GB/s",
                      "frac": MLP_STEP_BYTES_PER_SAMPLE * n / t / 1e9 / peaks["hbm_gbs"]},
            "unfused_equivalent": {
                "bytes_per_sample": MLP_UNFUSED_BYTES_PER_SAMPLE,
                "frac": MLP_UNFUSED_BYTES_PER_SAMPLE * n / t / 1e9 / peaks["hbm_gbs"],
                "note": "the HBM traffic of the earlier unfused step per unit time at this "
                        "step's rate, against the measured HBM copy rate (a throughput "
                        "figure: the fused kernel does not move these bytes)"}}
        mlp.close()
    return out


def transport_leg(S, b, db, dev):
    """The headline workload with field-dependent electron transport (Sec. 2.2:
    mobility and diffusivity from tables over the progress variable and E/N;
    synthetic tables stand in for BOLSIG+) against constant transport."""
    from paper_1904_08510_gb300.workload import transport_table
    out = {"table": "workload.transport_table(): 21 x 161 nodes, E/N 0..400 Td"}
    ref = None
    for name, kw in (("constant", {}), ("table", dict(transport=S.TRANSPORT_TABLE))):
        for m in (8, 30):
            p = S.default_params(threads_per_column=128, restart_m=m, **kw)
            sv = S.Solver(p, max_cols=b.ncol, max_cells=b.ncells, max_col_cells=int(b.lengths().max()))
            if kw:
                sv.set_transport_table(transport_table())
            t, o = _timed(lambda: sv.solve(db), reps=2)
            r = {"ms": 1e3 * t, "column_solves_per_s": b.ncol / t,
                 "status_ok": int((o["status"] == 0).sum().item())}
            r.update(_iterations(o))
            if ref is None:
                ref = o
            elif kw:
                ok = ((o["status"] == 0) & (ref["status"] == 0)).cpu().numpy()
                e = _colerr(b, o["ne"].cpu().numpy(), ref["ne"].cpu().numpy())[ok]
                r["root_change_vs_constant_ne"] = {"max": float(e.max()), "median": float(np.median(e))}
            out[f"{name}_restart{m}"] = r
            sv.close()
    return out


def iv_sweep(S, dev):
    """Charge flux (Sec. 4.4) after one implicit electric step over a sweep of
    the applied voltage: J = J+ + J- at both electrodes and its mean over the
    interior faces, i = J S with the burner cross-section S = 7.04 cm^2 of the
    paper's i-V comparison (synthetic columns: no chemistry, no steady state,
    no experimental comparison)."""
    import torch
    from paper_1904_08510_gb300.workload import make_batch
    s_expe = 7.04e-4                      # m^2
    rows = []
    kt = []
    for dv in (-1000.0, -500.0, -250.0, -100.0, -50.0, 0.0, 50.0, 100.0, 250.0, 500.0, 1000.0):
        b, dt = _dv_batch(make_batch, 256, 7_200_000, dv)
        db = S.DeviceBatch.from_host(b, dev)
        sv = S.Solver(S.default_params(), max_cols=b.ncol, max_cells=b.ncells, max_col_cells=512)
        o = sv.solve(db)
        t, (jp, jn) = _timed(lambda: sv.current(db, o["ne"], o["phi"]), reps=3)
        kt.append(t)
        J = (jp + jn).cpu().numpy().reshape(b.ncol, 513)
        ok = (o["status"] == 0).cpu().numpy()
        rows.append({"dv_V": dv, "dt_s": dt, "status_ok": int(ok.sum()),
                     "i_left_uA": float(J[ok, 0].mean() * s_expe * 1e6),
                     "i_right_uA": float(J[ok, -1].mean() * s_expe * 1e6),
                     "i_interior_mean_uA": float(J[ok, 1:-1].mean() * s_expe * 1e6)})
        sv.close()
    return {"workload": "256 columns x 512 cells per voltage (single-flame family), dt from an "
                        "ion-drift CFL of 0.5, one implicit step from X^n",
            "cross_section_m2": s_expe, "rows": rows,
            "current_kernel_us": 1e6 * float(np.median(kt)),
            "current_kernel_faces": 256 * 513}


def _dv_batch(make_batch, ncol, seed, dv, n_cells=512):
    """The paper's n_x = 512 flame columns with the electrode potential
    difference fixed at dv and the time step of a constant ion-drift CFL of 0.5
    (gas velocity 0.4 m/s plus the ion drift kappa_ion |dv| / L), so that dt
    shrinks as |dv| grows."""
    from paper_1904_08510_gb300.workload import KAPPA_ION, L_DOMAIN
    h = L_DOMAIN / n_cells
    dt = 0.5 * h / (0.4 + KAPPA_ION * abs(dv) / L_DOMAIN)
    b = make_batch("single", ncol, seed, n_cells=n_cells, dt=dt)
    b.v_right[:] = dv
    x = (np.arange(n_cells) + 0.5) * h
    b.phi_old = np.tile(dv * x / L_DOMAIN, ncol)
    return b, dt


def mg_study(S, dev):
    """The multigrid block solver (SDCEF_PREC_MG) and the preconditioner studies
    of Sec. 4.2: GMRES iterations and V-cycles against the V-cycle tolerance
    gamma_MG, one block inexact while the other is solved exactly; and the
    recast preconditioner against none over dv = 0..1000 V."""
    import torch
    from paper_1904_08510_gb300.workload import make_batch
    out = {"workload": "1024 columns x 512 cells (single-flame family), V_R = dv, "
                       "dt from an ion-drift CFL of 0.5"}

    def run(b, db, **kw):
        p = S.default_params(**kw)
        sv = S.Solver(p, max_cols=b.ncol, max_cells=b.ncells, max_col_cells=int(b.lengths().max()))
        t, o = _timed(lambda: sv.solve(db), reps=2)
        nw = o["newton_it"].float()
        kr = o["krylov_it"].float()
        r = {"status_ok": int((o["status"] == 0).sum().item()),
             "newton_mean": float(nw.mean().item()),
             "krylov_per_newton": float((kr.sum() / nw.sum().clamp(min=1)).item()),
             "ms": 1e3 * t, "column_solves_per_s": b.ncol / t}
        if p.precond == S.PREC_MG:
            r["vcycles_per_column"] = float(o["mg_cycles"].float().mean().item())
        sv.close()
        return r, o

    # gamma_MG study at dv = 100 V
    b, dt = _dv_batch(make_batch, 1024, 7_000_000, 100.0)
    db = S.DeviceBatch.from_host(b, dev)
    exact, oref = run(b, db, precond=S.PREC_RECAST)
    study = {"dv_V": 100.0, "dt_s": dt, "recast_exact_blocks": exact}
    rows = []
    for g in (1e-1, 1e-2, 1e-3, 1e-4, 1e-6, 1e-8):
        row = {"gamma_MG": g}
        row["S_linear_A_exact"], _ = run(b, db, precond=S.PREC_MG, mg_transfer=S.MG_LINEAR,
                                         mg_gamma_A=0.0, mg_gamma_S=g)
        row["A_operator_S_exact"], _ = run(b, db, precond=S.PREC_MG, mg_transfer=S.MG_OPERATOR,
                                           mg_gamma_A=g, mg_gamma_S=0.0)
        row["both_operator"], o = run(b, db, precond=S.PREC_MG, mg_transfer=S.MG_OPERATOR,
                                      mg_gamma_A=g, mg_gamma_S=g)
        ok = ((o["status"] == 0) & (oref["status"] == 0)).cpu().numpy()
        row["both_operator"]["max_root_diff_vs_exact_ne"] = float(
            _colerr(b, o["ne"].cpu().numpy(), oref["ne"].cpu().numpy())[ok].max()) if ok.any() else None
        rows.append(row)
    study["rows"] = rows
    lin_a, _ = run(b, db, precond=S.PREC_MG, mg_transfer=S.MG_LINEAR, mg_gamma_A=1e-4,
                   mg_gamma_S=1e-4)
    study["A_linear_transfers_gamma_1e-4"] = lin_a
    out["gamma_MG_study"] = study
    # recast preconditioner against none, dv = 0 .. 1000 V (128 columns each):
    # GMRES(32) iterations to gamma = 1e-4 on the first Newton system (one
    # Newton step, at most 5000 iterations)
    pre = []
    cap = 5000
    for dv in (0.0, 10.0, 50.0, 100.0, 500.0, 1000.0):
        bq, dtq = _dv_batch(make_batch, 128, 7_100_000, dv)
        dbq = S.DeviceBatch.from_host(bq, dev)
        row = {"dv_V": dv, "dt_s": dtq}
        for name, pc in (("recast", S.PREC_RECAST), ("none", S.PREC_NONE)):
            p = S.default_params(precond=pc, restart_m=32, max_newton=1, max_krylov=cap,
                                 stall_ratio=0.0)
            sv = S.Solver(p, max_cols=bq.ncol, max_cells=bq.ncells, max_col_cells=512)
            o = sv.solve(dbq)
            torch.cuda.synchronize()
            k = o["krylov_it"].cpu().numpy()
            row[name] = {"krylov_mean": float(k.mean()), "krylov_max": int(k.max()),
                         "converged_columns": int((k < cap).sum())}
            sv.close()
        row["ratio_none_over_recast"] = row["none"]["krylov_mean"] / max(row["recast"]["krylov_mean"], 1e-30)
        pre.append(row)
    out["with_without_preconditioner_first_newton_system"] = {"gmres": "GMRES(32), gamma 1e-4",
                                                               "cap": cap, "rows": pre}
    return out


def _iterations(o):
    """Mean, median and 99th percentile of the Newton and GMRES iteration counts."""
    out = {}
    for k, name in (("newton_it", "newton"), ("krylov_it", "krylov")):
        v = o[k].float().cpu().numpy()
        out.update({f"{name}_mean": float(v.mean()), f"{name}_p50": float(np.median(v)),
                    f"{name}_p99": float(np.percentile(v, 99))})
    return out


class _HostView:
    """Adapter giving Solver.solve_host the attributes of a workload.Batch with
    pinned tensors as the array storage."""

    def __init__(self, hb, b):
        self._hb = hb
        self.ncol = b.ncol
        self.ncells = b.ncells

    def __getattr__(self, k):
        return getattr(self._hb, k)


if __name__ == "__main__":
    sys.exit(main())
