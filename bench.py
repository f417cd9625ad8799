"""Benchmark: ADMM iterations/s of the HSDE ADMM for SOS programs on GB300.

Default workload: the constrained quartic POP on the unit ball with n = 20
(Gram blocks 231x231 and a weighted 21x21, m = 10626 monomial rows), plain
FP64 form.  One "step" is one full ADMM iteration (eq. (20): affine step,
PSD projection of every Gram block, dual/embedding update) of that instance.

JSON line (rank 0): value = ADMM iterations/s (device-timed with CUDA events
on the solver's stream, L2 flushed between steps), e2e = the same metric
through the C-ABI with host buffers (iterate copied in and out every step),
roofline of the dominant kernel, the CPU oracle as a bounded baseline,
time to a 1e-4 residual for the plain FP64 form and the FP32 form, and SM
clocks sampled during the timed region.

``--impl reference`` times the CPU oracle (the reference arm)
on the same workload and metric.
"""

from __future__ import annotations

import argparse
import json
import math
import os
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

WORKLOADS = {
    "ball_pop_n20": dict(desc="constrained quartic POP on the unit ball, n=20, 2d=4: Gram 231x231 + weighted "
                              "21x21, m=10626 (Lasserre order 2)", make=("ball_pop", 20, 0)),
    "quartic_pop_n6": dict(desc="unconstrained quartic POP, n=6, 2d=4: Gram 28x28, m=210",
                           make=("quartic_pop", 6, 0)),
    "quartic_pop_n30": dict(desc="unconstrained quartic POP, n=30, 2d=4: Gram 496x496, m=46376",
                            make=("quartic_pop", 30, 0)),
}


METRIC = "ADMM iterations/s (one iteration = affine step + PSD projections + update)"


def alu_peaks(sm_mhz: float):
    """ALU peaks from unit counts and the SM clock (GFLOP/s): 152 SMs, each
    with 2 FP64 and 128 FP32 fused multiply-adds per cycle (a multiply-add
    counts as two flops).  An FMA-loop probe on GB300 measured 2.00 FP64 and
    123.6 FP32 multiply-adds per cycle per SM at 2070 MHz."""
    ghz = sm_mhz / 1e3
    return {"fp64": 152 * 2 * 2 * ghz, "fp32": 152 * 128 * 2 * ghz}


def source_hash(*paths) -> str:
    import hashlib

    h = hashlib.sha256()
    for q in paths:
        with open(os.path.join(ROOT, q), "rb") as f:
            h.update(f.read())
    return h.hexdigest()


def recorded_traffic(kernel: str, workload: str):
    """DRAM bytes per launch of a kernel from the ncu capture recorded in
    profiles/traffic.json, if the kernel's source is unchanged since."""
    path = os.path.join(ROOT, "profiles", "traffic.json")
    if not os.path.exists(path):
        return None
    with open(path) as f:
        rec = json.load(f)
    e = rec.get(kernel, {}).get(workload)
    if not e or e.get("source_sha256") != source_hash(*e.get("sources", [])):
        return None
    return e.get("dram_bytes_per_launch")


def make_program(name):
    from instances import workloads as W

    fn, n, seed = WORKLOADS[name]["make"]
    return getattr(W, fn)(n, seed)


def clock_dir() -> str:
    """Where the nvidia-smi clock samples of the timed region are written
    (SOS_CLOCKS_DIR, else the system's temporary directory)."""
    import tempfile

    d = os.environ.get("SOS_CLOCKS_DIR") or tempfile.gettempdir()
    os.makedirs(d, exist_ok=True)
    return d


class L2Flush:
    """Evicts L2 between timed steps: writes a 256 MB buffer (> 129 MB of L2)
    and then reads a second one, so L2 holds clean unrelated lines and the
    write-back of the flush itself is not charged to the next timed step."""

    def __init__(self, torch):
        n = 256 * 1024 * 1024 // 4
        self.w = torch.empty(n, dtype=torch.float32, device="cuda")
        self.r = torch.zeros(n, dtype=torch.float32, device="cuda")
        self.out = torch.zeros((), dtype=torch.float32, device="cuda")
        self.torch = torch

    def __call__(self):
        self.w.zero_()
        self.torch.sum(self.r, dim=0, out=self.out)


def peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as f:
            return json.load(f), "measured"
    return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0}, "fallback"


class ClockSampler:
    def __init__(self, out_path):
        self.proc = None
        self.path = out_path

    def __enter__(self):
        try:
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(
                ["nvidia-smi", "--query-gpu=index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
                 "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
                 "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap",
                 "--format=csv,noheader,nounits", "-lms", "200"], stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None
        return self

    def __exit__(self, *a):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()
            self.f.close()

    def summary(self, dev_index=0):
        if self.proc is None or not os.path.exists(self.path):
            return None
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                if int(parts[0]) != dev_index:
                    continue
                sm.append(float(parts[1]))
                mx = float(parts[2])
            except ValueError:
                continue
            for nm, val in zip(names, parts[5:9]):
                if val.lower() == "active":
                    reasons.add(nm)
        if not sm:
            return None
        return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": mx, "reasons": sorted(reasons), "samples": len(sm)}


def reduce_max(x: float, dist, device: str) -> float:
    """Maximum of x over the ranks of the default process group."""
    import torch

    t = torch.tensor([x], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def aggregate_rate(units_per_rank: float, world: int, max_seconds: float) -> float:
    """Whole-job throughput of independent replicas: all units over the
    slowest rank's time."""
    return world * units_per_rank / max_seconds


def run_oracle_iters(prog, seconds: float, max_iters: int):
    """Times the CPU oracle's ADMM iterations (bounded sample)."""
    from oracle import admm, conic

    cd = conic.build(prog)
    hs = admm.HSDE(cd)
    u, v = hs.start()
    u, v = hs.step(u, v)  # warm-up
    t0 = time.perf_counter()
    k = 0
    while k < max_iters and (time.perf_counter() - t0) < seconds:
        u, v = hs.step(u, v)
        k += 1
    dt = time.perf_counter() - t0
    return k, dt


def cpu_cores():
    try:
        return len(os.sched_getaffinity(0))
    except Exception:
        return os.cpu_count()


def reference_arm(args, rank):
    if rank != 0:
        return
    prog = make_program(args.workload)
    k, dt = run_oracle_iters(prog, seconds=max(2.0, 8.0 * (args.steps + args.warmup) / 20), max_iters=10**9)
    ips = k / dt
    line = {"impl": "reference", "metric": METRIC, "value": ips, "unit": "iter/s",
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 / ips,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": args.workload, "desc": WORKLOADS[args.workload]["desc"]},
            "cpu_baseline": {"value": ips, "unit": "iter/s", "cores": cpu_cores(), "kind": "oracle",
                             "sample": f"{k} ADMM iterations of the FP64 NumPy/SciPy oracle from a cold start"},
            "e2e": {"value": ips, "unit": "iter/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def measure_warmstart(args, n_train: int, n_test: int, epochs: int, full: bool):
    """Learned warm start (parametric quartic POP, n = 10, Gram 66, m = 1001):
    time to a 1e-4 residual for unseen members, batched, in three forms on
    the SAME members: plain FP64 batched from the cold start, FP32
    projections batched from the cold start, and FP32 projections batched
    from the network's prediction.  The network is trained on n_train
    members solved to args.train_tol by the batched solver.  ``full`` adds
    the starts at the exact and at a noisy solution (what a better predictor
    could gain) and the plain FP64 form one instance at a time (sample)."""
    import torch

    from instances import workloads as W
    from paper_1708_04174_gb300 import capi, warmstart

    fam = W.ParametricPOP(n=10, K=16, seed=0)
    th_train = W.ParametricPOP.thetas(n_train, 100)
    th_test = W.ParametricPOP.thetas(n_test, 200)
    ws = warmstart.WarmStart(fam, hidden=512, seed=0)
    t0 = time.perf_counter()
    mi = args.max_iter
    res, dims, t_solve_train, tune = ws.solve(th_train, args.train_tol, mi)
    ok = np.array([r["status"] == capi.SOLVED for r in res])
    if not ok.any():
        raise RuntimeError(f"no training member reached {args.train_tol} within {mi} iterations")
    targets = warmstart.solution_vectors([r for r, k in zip(res, ok) if k], [d for d, k in zip(dims, ok) if k])
    t_data = time.perf_counter() - t0
    losses = ws.train(th_train[ok], targets, epochs=epochs, batch=256, lr=1e-3)
    pred = ws.predict(th_test)
    torch.cuda.synchronize()
    warm, _, t_warm, _ = ws.solve(th_test, 1e-4, mi, start=pred)
    cold, _, t_cold, _ = ws.solve(th_test, 1e-4, mi)
    sol_c = warmstart.solution_vectors(cold, ws.last_dims)
    fp64, _, t_fp64, _ = ws.solve(th_test, 1e-4, mi, precision=capi.PREC_FP64)

    def summary(rs, secs):
        it = np.array([r["iters"] for r in rs])
        return {"seconds": secs, "per_instance_s": secs / n_test, "iters_mean": float(it.mean()),
                "iters_median": float(np.median(it)), "iters_max": int(it.max()),
                "solved": int(sum(r["status"] == capi.SOLVED for r in rs))}

    def obj_diff(xs, ys):
        d = np.array([abs(a["obj_primal"] - b["obj_primal"]) / max(1.0, abs(b["obj_primal"]))
                      for a, b in zip(xs, ys) if a["status"] == capi.SOLVED and b["status"] == capi.SOLVED])
        return {"max": float(d.max()) if d.size else None, "median": float(np.median(d)) if d.size else None,
                "members": int(d.size)}

    pred_err = np.linalg.norm(pred - sol_c, axis=1) / np.maximum(np.linalg.norm(sol_c, axis=1), 1e-30)
    out = {"config": {"family": "p0 + sum_k theta_k q_k, n=10, K=16, Gram 66, m=1001", "train": int(n_train),
                      "test": int(n_test), "mlp": "16-512-512-5425", "epochs": int(epochs),
                      "train_tol": args.train_tol, "max_iter": mi},
           "plain_fp64_batched": summary(fp64, t_fp64),
           "mixed_batched_cold": summary(cold, t_cold),
           "mixed_batched_warm": summary(warm, t_warm),
           "speedup_warm_mixed_vs_plain_fp64_batched": t_fp64 / t_warm,
           "speedup_cold_mixed_vs_plain_fp64_batched": t_fp64 / t_cold,
           "speedup_warm_vs_cold_mixed": t_cold / t_warm,
           "objective_rel_diff": {"warm_vs_fp64": obj_diff(warm, fp64), "cold_vs_fp64": obj_diff(cold, fp64)},
           "prediction_rel_err": {"median": float(np.median(pred_err)), "p90": float(np.percentile(pred_err, 90))},
           "training": {"data_seconds": t_data, "solve_seconds": t_solve_train, "solved": int(ok.sum()),
                        "iters_mean": float(np.mean([r["iters"] for r in res])),
                        "train_seconds": ws.log["train_seconds"], "loss_first": losses[0], "loss_last": losses[-1]},
           "tuning": tune}
    if full:
        # what a better predictor could gain: starts at the cold-start solution
        # itself and at that solution with 5% relative Gaussian noise
        rng = np.random.default_rng(0)
        noisy = sol_c + 0.05 * np.linalg.norm(sol_c, axis=1, keepdims=True) / np.sqrt(sol_c.shape[1]) * \
            rng.standard_normal(sol_c.shape)
        bounds = {}
        for name, start in (("exact_solution", sol_c), ("solution_5pct_noise", noisy)):
            rb, _, tb, _ = ws.solve(th_test, 1e-4, mi, start=start.astype(np.float32))
            bounds[name] = summary(rb, tb)
        out["start_bounds"] = bounds
        # plain FP64 form, one instance at a time, on a sample of the same members
        sample = list(range(0, n_test, max(1, n_test // 4)))
        t_plain = 0.0
        it_plain = []
        for i in sample:
            s = capi.Solver(fam.program(th_test[i]), precision=capi.PREC_FP64, k_check=10)
            t1 = time.perf_counter()
            r = s.solve(1e-4, mi, want_solution=False)[0]
            t_plain += time.perf_counter() - t1
            it_plain.append(r["iters"])
            s.close()
        out["plain_fp64_single"] = {"seconds_per_instance": t_plain / len(sample),
                                    "iters_mean": float(np.mean(it_plain)), "sample": len(sample)}
    return out


def warmstart_arm(args):
    r = measure_warmstart(args, args.train, 1024, args.epochs, full=True)
    warm = r["mixed_batched_warm"]
    line = {"metric": "time to a 1e-4 residual per instance (learned warm start + FP32 projections + batched)",
            "value": warm["per_instance_s"], "unit": "s/instance", "n_gpus": 1, "steps": 1, "warmup": 0,
            "higher_is_better": False, "scaling": "weak", "vs_baseline": None, "dtype": "f64 iterates, f32 proj",
            "data": "synthetic", "config": dict(workload="parametric_warmstart", **r.pop("config"))}
    line.update(r)
    print(json.dumps(line), flush=True)


def measure_batch(args, steps: int, with_tt: bool, with_cpu: bool):
    """Batched form: 4096 cubic Lyapunov searches (n uniform in 2..6, Gram
    blocks 3x3 .. 84x84) advanced together.  One step = one ADMM iteration of
    every instance.  Mixed form (FP64 iterates, Woodbury and residuals; FP32
    Jacobi projections with the compensated refinement).  Also reported: time
    to a 1e-4 residual for the whole batch, the plain FP64 form's rate on the
    same batch, and the HBM roofline fraction of each memory-bound kernel of
    the FP64 affine step (timed alone, L2 flushed before each launch)."""
    import torch

    from instances import workloads as W
    from paper_1708_04174_gb300 import capi

    count = 4096
    t0 = time.perf_counter()
    progs = W.lyapunov_batch(count, 0, 2, 6)
    t_gen = time.perf_counter() - t0
    pk, pk_kind = peaks()
    hbm = float(pk["hbm_gbs"])
    flush = L2Flush(torch)

    def timed(solver, fn, reps, flush_each=True):
        st = torch.cuda.ExternalStream(solver.stream)
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(reps)]
        for a, b in ev:
            with torch.cuda.stream(st):
                if flush_each:
                    flush()
                a.record(st)
            fn()
            with torch.cuda.stream(st):
                b.record(st)
        solver.sync()
        return [a.elapsed_time(b) for a, b in ev]

    t0 = time.perf_counter()
    s = capi.Solver(progs, precision=capi.PREC_MIXED, k_check=10)
    t_setup = time.perf_counter() - t0
    s.iterate(args.warmup)
    s.sync()
    clk = ClockSampler(os.path.join(clock_dir(), "clocks_rank0.csv"))
    torch.cuda.synchronize()
    with clk:
        step_ms = timed(s, lambda: s.iterate(1), steps)
    total_ms = float(np.sum(step_ms))
    ips = steps / (total_ms / 1e3)
    stage_ms = {name: float(np.mean(timed(s, lambda st=st: s.run_stage(st), 5)))
                for st, name in ((0, "affine"), (1, "psd_small"))}
    dims = s.dims
    Ns = []
    for prog in progs:
        for con in prog.constraints:
            for blk in con.blocks:
                from math import comb

                Ns.append(blk.size(prog.n))
    flops = sum(9.0 * N ** 3 for N in Ns)
    fp32_peak = alu_peaks(2070.0)["fp32"]
    roof = {"kernel": "k_psd_small<double,float> (FP32 Jacobi + compensated refinement, one CTA per block)",
            "bound": "alu", "achieved": flops / (stage_ms["psd_small"] / 1e3) / 1e9, "peak": fp32_peak,
            "unit": "GFLOP/s", "frac": flops / (stage_ms["psd_small"] / 1e3) / 1e9 / fp32_peak,
            "traffic": recorded_traffic("k_psd_small", "lyapunov_batch4096"),
            "note": "algorithmic flops 9 N^3 per block over all 8192 blocks; peak = FP32 multiply-add rate from "
                    "unit counts at 2070 MHz", "stage_ms": stage_ms,
            "stage_bytes": {"affine": s.stage_bytes(0), "psd_small": s.stage_bytes(1)}}
    tuning = s.tuning()
    launches = s.launches_per_iteration()
    # end-to-end through the C-ABI with host buffers
    u0, v0 = s.get_iterate()
    e2e_steps = 10
    s.sync()
    t0 = time.perf_counter()
    for _ in range(e2e_steps):
        s.set_iterate(u0, v0)
        s.iterate(1)
        u0, v0 = s.get_iterate()
    e2e_dt = time.perf_counter() - t0
    nbytes = int(u0.nbytes + v0.nbytes)
    e2e = {"value": e2e_steps / e2e_dt, "unit": "iter/s", "h2d_bytes_per_step": nbytes, "d2h_bytes_per_step": nbytes}
    s.close()

    # time to a 1e-4 residual for the whole batch, from the cold start
    tt = None
    if with_tt:
        sm = capi.Solver(progs, precision=capi.PREC_MIXED, k_check=10)
        t0 = time.perf_counter()
        res = sm.solve(1e-4, args.max_iter, want_solution=False)
        t_solve = time.perf_counter() - t0
        sm.close()
        st = np.array([r["status"] for r in res])
        it = np.array([r["iters"] for r in res])
        tt = {"seconds": t_solve, "per_instance_s": t_solve / count,
              "status_counts": {str(k): int(v) for k, v in zip(*np.unique(st, return_counts=True))},
              "iters": {"median": float(np.median(it)), "p90": float(np.percentile(it, 90)), "max": int(it.max())}}

    # plain FP64 form on the same batch: rate, and the HBM roofline of the
    # memory-bound kernels of its affine step
    s64 = capi.Solver(progs, precision=capi.PREC_FP64, k_check=10, solve_mode=1)
    s64.iterate(3)
    s64.sync()
    fp64_ms = float(np.mean(timed(s64, lambda: s64.iterate(1), 10)))
    names = {4: "k_rows_r", 5: "k_lr_y", 6: "k_woodbury", 7: "k_rows_sigma2", 8: "k_inst_scalar", 9: "k_rows_y"}
    hbm_kernels = {}
    for stg, name in names.items():
        ms = float(np.mean(timed(s64, lambda stg=stg: s64.run_stage(stg), 10)))
        nb = s64.stage_bytes(stg)
        gbs = nb / (ms / 1e3) / 1e9
        hbm_kernels[name] = {"ms": ms, "algorithmic_bytes": nb, "achieved_gbs": gbs, "frac": gbs / hbm}
    s64.close()

    cpu = None
    if with_cpu:
        # the oracle, as it stands, on a sample of the batch (one instance at a time)
        tot_k, tot_t, used = 0, 0.0, 0
        for prog in progs[::256]:
            k, dt = run_oracle_iters(prog, seconds=1.0, max_iters=10 ** 9)
            tot_k += k
            tot_t += dt
            used += 1
        inst_rate = tot_k / tot_t
        cpu = {"value": inst_rate / count, "unit": "iter/s", "cores": cpu_cores(), "kind": "oracle",
               "sample": f"{used} of the {count} instances (every 256th), about 1 s of oracle iterations each; "
                         f"batch iterations/s = instance-iterations/s / {count}"}

    line = {"metric": "ADMM iterations/s of the whole batch (one iteration of all 4096 instances)",
            "value": ips, "unit": "iter/s", "n_gpus": 1, "steps": steps, "warmup": args.warmup,
            "ms_per_step": total_ms / steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64 iterates, f32 proj", "data": "synthetic",
            "config": {"workload": "lyapunov_batch4096",
                       "desc": "4096 cubic Lyapunov searches, n uniform in 2..6, V degree 2..4, eps 1e-3; "
                               "Gram blocks 3x3 .. 84x84",
                       "form": "FP64 iterates/Woodbury/residuals, FP32 Jacobi projections + compensated refinement",
                       "l2": "flushed between steps (256 MB write, then 256 MB read); working set > L2",
                       "n_x_total": int(sum(d[0] for d in dims)), "m_total": int(sum(d[1] for d in dims)),
                       "setup_s": t_setup, "generate_s": t_gen},
            "instance_iters_per_s": ips * count, "e2e": e2e, "roofline": roof,
            "hbm_kernels_fp64": {"peak_gbs": hbm, "peak_source": pk_kind, "kernels": hbm_kernels},
            "fp64_form": {"ms_per_step": fp64_ms, "value": 1e3 / fp64_ms, "unit": "iter/s"},
            "time_to_1e-4": tt, "tuning": tuning,
            "gpu_launches": int(launches * steps), "clocks": clk.summary(0)}
    if cpu is not None:
        line["cpu_baseline"] = cpu
    return line


def batched_arm(args):
    print(json.dumps(measure_batch(args, args.steps, not args.no_tt, not args.no_cpu_baseline)), flush=True)


# Published numbers for the constrained POP of eq. (46) (context only: a
# MATLAB solver on a 2.8 GHz Intel Core i7, tolerance 1e-3, at most 2000
# iterations).  Table I: CDCS-sos total solve time in seconds; Table II:
# terminal objective of the interior-point solvers and of CDCS-sos.
PAPER_TABLE1_CDCS_S = {10: 0.4, 12: 0.7, 14: 1.4, 17: 3.5, 20: 8.5, 24: 22.8, 29: 67.1, 35: 216.9, 42: 686.6}
PAPER_TABLE2_IPM = {10: -9.11, 12: -11.12, 14: -13.12, 17: -16.12, 20: -19.12, 24: -23.12}
PAPER_TABLE2_CDCS = {10: -9.10, 12: -11.11, 14: -13.12, 17: -16.06, 20: -19.08, 24: -23.15, 29: -28.17, 35: -34.08,
                     42: -41.05}


# Table III: CDCS-sos total solve time (s) of the local Lyapunov search with a
# quadratic V in the ball |x|^2 <= 0.1 (same hardware and stopping rule as
# Table I; context only).
PAPER_TABLE3_CDCS_S = {10: 0.3, 12: 0.4, 14: 0.6, 17: 1.1, 20: 2.4, 24: 5.1, 29: 14.3, 35: 37.4, 42: 92.8}


def local_lyapunov_arm(args):
    """Local stability of a random cubic system with a linearly stable origin
    in the ball |x|^2 <= 0.1, quadratic V, Positivstellensatz multiplier
    (instances.workloads.lyapunov_local, seed = n), for the n of the paper's
    Table III, at tolerance 1e-3 and at most 2000 iterations, plain FP64 and
    mixed; wall time of sos_solve next to the paper's CDCS-sos times (other
    hardware: context)."""
    from instances import workloads as W
    from paper_1708_04174_gb300 import capi

    ns = [10, 12, 14, 17, 20, 24, 29, 35, 42] if not args.paper_n else [int(x) for x in args.paper_n.split(",")]
    rows = []
    for n in ns:
        prog = W.lyapunov_local(n, n)
        entry = {"n": n, "N": max(b.size(n) for c in prog.constraints for b in c.blocks),
                 "paper_cdcs_s": PAPER_TABLE3_CDCS_S.get(n)}
        for name, prec in (("fp64", capi.PREC_FP64), ("mixed", capi.PREC_MIXED)):
            t0 = time.perf_counter()
            s = capi.Solver(prog, precision=prec, k_check=10)
            t_setup = time.perf_counter() - t0
            t0 = time.perf_counter()
            r = s.solve(1e-3, 2000, want_solution=False)[0]
            dt = time.perf_counter() - t0
            d = s.dims[0]
            s.close()
            entry["m"], entry["t_eff"] = d[1], d[3]
            entry[name] = {"solve_s": dt, "setup_s": t_setup, "iters": r["iters"], "status": r["status"],
                           "trace_P": r["obj_primal"], "res": max(r["res_primal"], r["res_dual"], r["gap"])}
        if entry["paper_cdcs_s"]:
            entry["speedup_fp64_vs_paper_cdcs"] = entry["paper_cdcs_s"] / entry["fp64"]["solve_s"]
        rows.append(entry)
        print(json.dumps({"n": n, "fp64_s": entry["fp64"]["solve_s"], "mixed_s": entry["mixed"]["solve_s"],
                          "status": [entry["fp64"]["status"], entry["mixed"]["status"]]}), file=sys.stderr, flush=True)
    line = {"metric": "time to solve the local Lyapunov search at tolerance 1e-3 (paper's Table III workload shape, "
                      "plain FP64)", "value": None, "unit": "s", "n_gpus": 1, "higher_is_better": False,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": "lyapunov_local_table3", "tol": 1e-3, "max_iter": 2000, "r2": 0.1,
                       "note": "paper times: MATLAB CDCS-sos on a 2.8 GHz Intel Core i7 on its own random systems "
                               "(context)"},
            "rows": rows}
    print(json.dumps(line), flush=True)


def paper_pop_arm(args):
    """The constrained POP of eq. (46) on the unit ball (Lasserre order 2,
    Gram N = C(n+2, 2) plus the weighted multiplier block) for the n of the
    paper's Table I, solved at the paper's stopping rule (tolerance 1e-3, at
    most 2000 iterations) in the plain FP64 form and the mixed form.  Wall
    time of sos_solve (setup excluded) next to the paper's CDCS-sos times
    (other hardware: context), terminal objective next to Table II."""
    from instances import workloads as W
    from paper_1708_04174_gb300 import capi

    ns = [10, 12, 14, 17, 20, 24, 29, 35, 42] if not args.paper_n else [int(x) for x in args.paper_n.split(",")]
    rows = []
    for n in ns:
        prog = W.paper_pop(n)
        entry = {"n": n, "paper_cdcs_s": PAPER_TABLE1_CDCS_S.get(n), "paper_ipm_obj": PAPER_TABLE2_IPM.get(n),
                 "paper_cdcs_obj": PAPER_TABLE2_CDCS.get(n)}
        for name, prec in (("fp64", capi.PREC_FP64), ("mixed", capi.PREC_MIXED)):
            t0 = time.perf_counter()
            s = capi.Solver(prog, precision=prec, k_check=10)
            t_setup = time.perf_counter() - t0
            t0 = time.perf_counter()
            r = s.solve(1e-3, 2000, want_solution=False)[0]
            dt = time.perf_counter() - t0
            d = s.dims[0]
            s.close()
            entry[name] = {"solve_s": dt, "setup_s": t_setup, "iters": r["iters"], "status": r["status"],
                           "objective": -r["obj_primal"], "res": max(r["res_primal"], r["res_dual"], r["gap"])}
            entry["m"] = d[1]
        entry["N"] = math.comb(n + 2, 2)
        if entry["paper_cdcs_s"]:
            entry["speedup_fp64_vs_paper_cdcs"] = entry["paper_cdcs_s"] / entry["fp64"]["solve_s"]
        rows.append(entry)
        print(json.dumps({"n": n, "fp64_s": entry["fp64"]["solve_s"], "mixed_s": entry["mixed"]["solve_s"],
                          "obj": entry["fp64"]["objective"]}), file=sys.stderr, flush=True)
    line = {"metric": "time to solve eq. (46) at tolerance 1e-3 (paper's Table I workload, plain FP64)",
            "value": rows[0]["fp64"]["solve_s"] if len(rows) == 1 else None, "unit": "s", "n_gpus": 1,
            "higher_is_better": False, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": "paper_pop_table1", "tol": 1e-3, "max_iter": 2000,
                       "note": "paper times: MATLAB CDCS-sos on a 2.8 GHz Intel Core i7 (context, other hardware)"},
            "rows": rows}
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=20)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--workload", default="ball_pop_n20",
                    choices=sorted(WORKLOADS) + ["parametric_warmstart", "lyapunov_batch4096", "paper_pop_table1",
                                                 "lyapunov_local_table3"])
    ap.add_argument("--paper-n", default="",
                    help="comma-separated n for paper_pop_table1 / lyapunov_local_table3 (default: the tables' n)")
    ap.add_argument("--train", type=int, default=20000, help="training members (parametric_warmstart)")
    ap.add_argument("--epochs", type=int, default=200, help="training epochs (parametric_warmstart)")
    ap.add_argument("--max-iter", type=int, default=20000, help="iteration cap of every solve (parametric_warmstart)")
    ap.add_argument("--train-tol", type=float, default=1e-3, help="tolerance of the training solves (parametric_warmstart)")
    ap.add_argument("--precision", default="fp64", choices=["fp64", "mixed", "fp32"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-tt", action="store_true", help="skip the time-to-1e-4 solves")
    ap.add_argument("--no-extras", action="store_true",
                    help="skip the batch and warm-start keys of the default line")
    ap.add_argument("--extras-train", type=int, default=4096, help="training members of the warm-start key")
    ap.add_argument("--extras-test", type=int, default=256, help="unseen members of the warm-start key")
    ap.add_argument("--extras-epochs", type=int, default=100, help="epochs of the warm-start key")
    args = ap.parse_args()
    args.warmup = max(args.warmup, 3)

    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    if args.impl == "reference":
        return reference_arm(args, rank)
    if args.workload == "parametric_warmstart":
        return warmstart_arm(args)
    if args.workload == "lyapunov_batch4096":
        return batched_arm(args)
    if args.workload == "paper_pop_table1":
        return paper_pop_arm(args)
    if args.workload == "lyapunov_local_table3":
        return local_lyapunov_arm(args)

    import torch

    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist

        dist.init_process_group("nccl")

    from paper_1708_04174_gb300 import capi

    prog = make_program(args.workload)
    prec = {"fp64": capi.PREC_FP64, "mixed": capi.PREC_MIXED, "fp32": capi.PREC_FP32}[args.precision]
    solver = capi.Solver(prog, precision=prec, k_check=10)
    stream = torch.cuda.ExternalStream(solver.stream)
    flush = L2Flush(torch)

    # warm-up
    solver.iterate(args.warmup)
    solver.sync()

    def barrier():
        if dist is not None:
            dist.barrier()
        torch.cuda.synchronize()

    starts = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    ends = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    clk = ClockSampler(os.path.join(clock_dir(), f"clocks_rank{rank}.csv"))
    barrier()
    with clk:
        t_wall0 = time.perf_counter()
        for k in range(args.steps):
            with torch.cuda.stream(stream):
                flush()  # L2 flush between steps, outside the step's events
                starts[k].record(stream)
            solver.iterate(1)
            with torch.cuda.stream(stream):
                ends[k].record(stream)
        solver.sync()
        barrier()
        t_wall = time.perf_counter() - t_wall0
    step_ms = [s.elapsed_time(e) for s, e in zip(starts, ends)]
    total_ms = float(np.sum(step_ms))
    if dist is not None:
        total_ms = reduce_max(total_ms, dist, "cuda")
    ips = aggregate_rate(args.steps, world, total_ms / 1e3)

    # dominant kernel: a fresh handle replays the timed iteration range
    # (warm-up, then the steps) kernel group by kernel group (stages 0, 1 and
    # 10..14 in order make one iteration), each bracketed by events on that
    # handle's stream and L2 flushed before each iteration as in the timed
    # region.  In the timed steps the small-block projections run on a side
    # stream beside the large-block ones, so a step is affine + max(small,
    # large); the replay is trusted only if that sum is within 10% of it.
    blocks = [blk.size(prog.n) for con in prog.constraints for blk in con.blocks]
    # Gram blocks above 112 go to the tensor-core Newton-Schulz kernel in the
    # FP32-projection forms; stage 2 (every large-block projection) times it
    ns_blocks = [N for N in blocks if N > 112] if prec != capi.PREC_FP64 else []
    if ns_blocks:
        stage_names = ((0, "affine"), (1, "psd_small"), (2, "psd_large_ns"))
    else:
        stage_names = ((0, "affine"), (1, "psd_small"), (15, "tri_warm"), (10, "tri_gather"), (11, "tri_reduce"),
                       (12, "tri_vectors"), (13, "tri_recon"), (14, "psd_large_jacobi"))
    sk = capi.Solver(prog, precision=prec, k_check=10)
    sk.iterate(args.warmup)
    sk.sync()
    stk = torch.cuda.ExternalStream(sk.stream)
    evs = {name: [] for _, name in stage_names}
    ns_steps = []  # Newton-Schulz steps of each replayed iteration (largest over the blocks)
    for _ in range(args.steps):
        with torch.cuda.stream(stk):
            flush()
        for stage, name in stage_names:
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            with torch.cuda.stream(stk):
                a.record(stk)
            sk.run_stage(stage)
            with torch.cuda.stream(stk):
                b.record(stk)
            evs[name].append((a, b))
        if ns_blocks:
            ns_steps.append(sk.stats()["max_sweeps"])
    sk.sync()
    sk.close()
    stage_all = {name: [a.elapsed_time(b) for a, b in evs[name]] for _, name in stage_names}
    stage_ms = {name: float(np.mean(v)) for name, v in stage_all.items()}
    # launches that did the work: once a warm attempt projects the block, the
    # cold kernels after it return at once (a few microseconds)
    worked = {name: [x for x in v if x > 0.02] for name, v in stage_all.items()}
    large_ms = sum(stage_ms[k] for k in ("tri_warm", "tri_gather", "tri_reduce", "tri_vectors", "tri_recon",
                                         "psd_large_jacobi", "psd_large_ns") if k in stage_ms)
    replay_ms = stage_ms["affine"] + max(stage_ms["psd_small"], large_ms)
    step_ms = total_ms / args.steps
    consistent = abs(replay_ms - step_ms) <= 0.1 * step_ms

    d = solver.dims[0]
    clk_sum = clk.summary(local)
    sm_mhz = (clk_sum or {}).get("sm_max_mhz") or 2070.0
    alu = alu_peaks(sm_mhz)
    big = [N for N in blocks if 33 <= N <= 232] if prec == capi.PREC_FP64 else []
    note_tail = (f"; kernel times from a replay of the timed iterations; replay affine + max(small, large) = "
                 f"{replay_ms:.3f} ms against {step_ms:.3f} ms per step"
                 + ("" if consistent else " (more than 10% apart: achieved and frac withheld)"))
    if big:
        # The dominant unit is the large-block projection: kernels in a row
        # on one stream (the warm attempt, which returns at once early in a
        # solve, then gather, FP32 tridiagonal reduction, FP32 eigenvectors,
        # FP64 refinement and reconstruction), ~90% of a step.
        # Algorithmic work: 9 N^3 flops, the count of a dense symmetric
        # eigendecomposition plus the reconstruction V max(L, 0) V^T (the
        # figure the grid Jacobi kernel was measured against before), bound
        # by the GPU's FP64 multiply-add rate.
        proj_ms = sum(stage_ms[k] for k in ("tri_warm", "tri_gather", "tri_reduce", "tri_vectors", "tri_recon"))
        flops = sum(9.0 * N ** 3 for N in big)
        achieved = flops / (proj_ms / 1e3) / 1e9
        # per kernel: the reduction is one CTA, so its own ceiling is one SM's
        # FP32 rate (4/3 N^3 flops); the refinement and reconstruction run on
        # every SM (at least 7 N^3 FP64 flops: V^T V, W V, V^T W V lower half,
        # V M, V M V^T lower half, plus 2 N^3 per Newton-Schulz or Newton pass)
        per = {"k_tri_reduce": {"ms": stage_ms["tri_reduce"], "flops": sum(4.0 / 3.0 * N ** 3 for N in big),
                                "peak": alu["fp32"] / 152, "peak_scope": "one SM, FP32 (the kernel is one CTA)"},
               "k_tri_recon": {"ms": stage_ms["tri_recon"], "flops": sum(7.0 * N ** 3 for N in big),
                               "peak": alu["fp64"], "peak_scope": "all SMs, FP64"},
               "k_tri_vectors": {"ms": stage_ms["tri_vectors"], "flops": None, "peak": None,
                                 "peak_scope": "latency bound: bisection and inverse iteration, O(N^2) per eigenvalue"},
               "k_tri_gather": {"ms": stage_ms["tri_gather"], "flops": None, "peak": None, "peak_scope": "copy"},
               "k_tri_recon (warm attempt)": {"ms": stage_ms["tri_warm"], "flops": None, "peak": None,
                                              "peak_scope": "returns at once unless it starts from the last eigenvectors"}}
        stage_of = {"k_tri_reduce": "tri_reduce", "k_tri_recon": "tri_recon", "k_tri_vectors": "tri_vectors",
                    "k_tri_gather": "tri_gather", "k_tri_recon (warm attempt)": "tri_warm"}
        for kname, v in per.items():
            # per kernel: mean over the launches that did the work (the mean
            # over all launches, early returns included, is "ms")
            w = worked[stage_of[kname]]
            v["launches"] = len(stage_all[stage_of[kname]])
            v["launches_worked"] = len(w)
            v["ms_worked"] = float(np.mean(w)) if w else None
            ok = bool(v["flops"]) and bool(w)
            v["achieved_gflops"] = v["flops"] / (v["ms_worked"] / 1e3) / 1e9 if ok else None
            v["frac"] = v["achieved_gflops"] / v["peak"] if ok else None
        roof = {"kernel": "large-block FP64 projection (warm attempt, k_tri_gather, k_tri_reduce, k_tri_vectors, "
                          "k_tri_recon)",
                "bound": "alu", "achieved": achieved if consistent else None, "peak": alu["fp64"],
                "unit": "GFLOP/s", "frac": achieved / alu["fp64"] if consistent else None,
                "traffic": recorded_traffic("large_projection_fp64", args.workload),
                "work_flops": flops, "ms_per_launch": proj_ms, "kernels": per,
                "note": f"peak = FP64 multiply-add rate from unit counts and the SM clock ({sm_mhz:.0f} MHz)"
                        + note_tail
                        + (f"; in {len(stage_all['tri_reduce']) - len(worked['tri_reduce'])} of "
                           f"{len(stage_all['tri_reduce'])} iterations the warm attempt projected the block "
                           "(refinement from the last eigenvectors) and the cold kernels returned at once; the "
                           "work is counted as 9 N^3 in every iteration"
                           if len(worked['tri_reduce']) < len(stage_all['tri_reduce']) else ""),
                "stage_ms": stage_ms}
    elif ns_blocks:
        # The dominant unit is the tensor-core Newton-Schulz projection of the
        # large blocks: per step two products of the padded Np x Np iterate
        # (Np = N rounded up to 128), each as six BF16 products of the
        # three-part split (2 Np^3 flops each), plus the final product W S;
        # bound by the BF16 tensor rate (the sustained measured peak: the
        # kernel runs inside a long step).
        pk, pk_kind = peaks()
        peak_tf = pk.get("bf16_tflops_sustained") or pk.get("bf16_tflops")
        steps_mean = float(np.mean(ns_steps)) if ns_steps else 0.0
        tflop = sum(6 * 2.0 * (-(-N // 128) * 128) ** 3 * (2 * steps_mean + 1) for N in ns_blocks) / 1e12
        fp32_equiv = sum(2.0 * N ** 3 * (2 * steps_mean + 1) for N in ns_blocks) / 1e12
        ns_ms = stage_ms["psd_large_ns"]
        achieved = tflop / (ns_ms / 1e3)
        roof = {"kernel": "k_psd_ns (tensor-core Newton-Schulz projection)", "bound": "tensor",
                "achieved": achieved if consistent else None, "peak": peak_tf, "unit": "TFLOP/s",
                "frac": achieved / peak_tf if consistent else None, "traffic": None,
                "ns_steps_mean": steps_mean, "ms_per_launch": ns_ms,
                "note": f"BF16 tensor flops of the three-part split products ({tflop * 1e3:.2f} GFLOP per launch; "
                        f"{fp32_equiv * 1e3:.2f} GFLOP as FP32-equivalent products of the N x N iterate) over "
                        f"the sustained BF16 peak ({pk_kind})" + note_tail,
                "stage_ms": stage_ms}
    else:
        flops = sum(9.0 * N ** 3 for N in blocks)
        dom_ms = stage_ms["psd_small"] if stage_ms["psd_small"] >= large_ms else large_ms
        peak = alu["fp64"] if prec == capi.PREC_FP64 else alu["fp32"]
        prec_name = "FP64" if prec == capi.PREC_FP64 else "FP32"
        achieved = flops / (dom_ms / 1e3) / 1e9
        roof = {"kernel": "PSD projection (Jacobi kernels)", "bound": "alu",
                "achieved": achieved if consistent else None, "peak": peak, "unit": "GFLOP/s",
                "frac": achieved / peak if consistent else None, "traffic": None,
                "note": f"peak = {prec_name} multiply-add rate from unit counts and the SM clock ({sm_mhz:.0f} MHz)"
                        + note_tail,
                "stage_ms": stage_ms}

    # end-to-end through the C-ABI with host buffers, on a fresh handle over
    # the same iteration range as the timed steps (warm-up, then the steps)
    se = capi.Solver(prog, precision=prec, k_check=10)
    se.iterate(args.warmup)
    se.sync()
    # the step's input and result live in pinned host memory
    pin = [torch.empty(se.total, dtype=torch.float64).pin_memory() for _ in range(2)]
    u0, v0 = se.get_iterate(out=(pin[0].numpy(), pin[1].numpy()))
    e2e_steps = args.steps
    t0 = time.perf_counter()
    for _ in range(e2e_steps):
        se.set_iterate(u0, v0)
        se.iterate(1)
        se.get_iterate(out=(u0, v0))
    e2e_dt = time.perf_counter() - t0
    se.close()
    esz = 8 if prec == capi.PREC_FP64 else 4
    nbytes = 2 * ((d[0] + d[1]) * esz + 8)
    e2e = {"value": world * e2e_steps / e2e_dt, "unit": "iter/s", "h2d_bytes_per_step": nbytes,
           "d2h_bytes_per_step": nbytes}

    out = {"metric": METRIC,
           "value": ips, "unit": "iter/s", "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
           "ms_per_step": total_ms / args.steps, "higher_is_better": True, "scaling": "weak",
           "vs_baseline": None, "dtype": "f64" if prec == capi.PREC_FP64 else "f32", "data": "synthetic",
           "config": {"workload": args.workload, "desc": WORKLOADS[args.workload]["desc"],
                      "form": "plain FP64" if prec == capi.PREC_FP64 else "FP32 projections, FP64 Woodbury",
                      "l2": "flushed between steps (256 MB write, then 256 MB read)", "parallelism": "replicas" if world > 1 else "1 GPU",
                      "n_x": d[0], "m": d[1], "t_eff": d[3]},
           "wall_s": t_wall, "e2e": e2e, "roofline": roof,
           "gpu_launches": None}
    out["gpu_launches"] = int(solver.launches_per_iteration() * args.steps)
    out["roofline"]["peak_source"] = ("MEASURED_PEAKS.json bf16_tflops_sustained" if ns_blocks else
                                      "unit counts x SM clock (derivation in the design notes)")
    out["clocks"] = clk_sum

    # the FP32-projection form (tensor-core Newton-Schulz for the large block)
    # on the same instance and the same step definition, for comparison
    if prec == capi.PREC_FP64 and not args.no_tt:
        sm = capi.Solver(prog, precision=capi.PREC_MIXED, k_check=10)
        sm.iterate(args.warmup)
        sm.sync()
        stm = torch.cuda.ExternalStream(sm.stream)
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
        for a0, a1 in ev:
            with torch.cuda.stream(stm):
                flush()
                a0.record(stm)
            sm.iterate(1)
            with torch.cuda.stream(stm):
                a1.record(stm)
        sm.sync()
        mixed_ms = float(np.sum([a0.elapsed_time(a1) for a0, a1 in ev]))
        out_mixed = {"value": args.steps / (mixed_ms / 1e3), "unit": "iter/s", "ms_per_step": mixed_ms / args.steps,
                     "form": "FP64 iterates, FP32 projections (tensor-core Newton-Schulz for N=231)",
                     "stats": sm.stats()}
        sm.close()
    else:
        out_mixed = None

    if not args.no_tt:
        tt = {}
        for nm, pr in (("fp64", capi.PREC_FP64), ("mixed_fp32_projections", capi.PREC_MIXED)):
            s2 = capi.Solver(prog, precision=pr, k_check=10)
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            r = s2.solve(1e-4, 3000, want_solution=False)[0]
            dt = time.perf_counter() - t0
            tt[nm] = {"seconds": dt, "iters": r["iters"], "status": r["status"], "obj": r["obj_primal"]}
            s2.close()
        out["time_to_1e-4"] = tt
    if out_mixed is not None:
        out["mixed_form"] = out_mixed

    if rank == 0 and not args.no_cpu_baseline:
        k, dt = run_oracle_iters(prog, seconds=15.0, max_iters=10**9)
        out["cpu_baseline"] = {"value": k / dt, "unit": "iter/s", "cores": cpu_cores(), "kind": "oracle",
                               "sample": f"{k} ADMM iterations of the FP64 NumPy/SciPy oracle on the same "
                                         f"instance (about 15 s), BLAS threads at their default"}
    if world == 1 and not args.no_extras and args.workload == "ball_pop_n20":
        # The targets of the other forms as extra keys of the headline line
        # (one GPU only): the 4096-search batch (rate of the mixed and plain
        # FP64 forms, HBM fraction of each FP64 affine kernel, short runs),
        # and time to 1e-4 on the same unseen parametric members for plain
        # FP64 batched, mixed batched cold and mixed batched warm (training
        # set, test set and epochs scaled down from the full arm to keep the
        # default run within minutes; stated in its config).
        solver.close()
        solver = None
        b = measure_batch(args, 10, with_tt=False, with_cpu=False)
        out["batch_lyapunov4096"] = {
            "value": b["value"], "unit": "batch iter/s", "steps": 10,
            "instance_iters_per_s": b["instance_iters_per_s"], "form": b["config"]["form"],
            "ms_per_step": b["ms_per_step"], "fp64_form": b["fp64_form"],
            "hbm_kernels_fp64": b["hbm_kernels_fp64"], "setup_s": b["config"]["setup_s"],
            "roofline_psd_small": {k: b["roofline"][k] for k in ("kernel", "achieved", "peak", "unit", "frac")}}
        out["warmstart_parametric"] = measure_warmstart(args, args.extras_train, args.extras_test,
                                                        args.extras_epochs, full=False)
    if rank == 0:
        print(json.dumps(out), flush=True)
    if solver is not None:
        solver.close()
    if dist is not None:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
