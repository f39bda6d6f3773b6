#!/usr/bin/env python
"""Benchmark of the self-learning DQMC hot path on GB300.

Workload (the configuration the headline metric is quoted on): SLDQMC on a
16x16 lattice, t=1, mu=-0.5, xi=1, beta=8, dtau=0.05 (M=160), n_wrap from the
autotuner (paper_1612_03804_gb300/tune.py),
bare Ising weight J=1, h=2.774; effective action with J1/J2/J3 (space) and
J_tau couplings, fitted (Eq. 3) on local-DQMC configurations of an 8x8
lattice at the same couplings and transferred to 16x16, as the paper does
with its L=8 fit.

Training (untimed): 8x8 chains are pre-thermalised by effective sweeps of
the bare Ising action, run 20 local-DQMC sweeps, then contribute one
configuration per sweep until 2000 are collected.  The 16x16 chains start in
equilibrium of the fitted H_eff (300 effective sweeps) before the warm-up.

One step = one cumulative update (steps iii+iv) of B independent chains:
one sweep of N*M effective-model flips per chain, the exact log weight of
every proposal (two flavours -> 2B fermion-weight evaluations through the
stabilised B-chain) and the Eq. 4 acceptance.  The metric is fermion-weight
evaluations per second (single-flavour det(1+B) evaluations) with the
slice products in split-TF32 (mixed) precision; the FP64-product path and
decorrelated samples/s are reported beside it.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]

Under torchrun each rank runs its own chains (weak scaling, no data-path
collective); the timed region is bracketed by a barrier and a device
synchronisation and the time is the maximum over ranks.
"""
import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

WL = dict(L=16, t=1.0, mu=-0.5, xi=1.0, beta=8.0, dtau=0.05, n_wrap=10, J=1.0, h=2.774)
CLASSES = [[(1, 0, 0), (0, 1, 0)], [(1, 1, 0), (1, -1, 0)], [(2, 0, 0), (0, 2, 0)], [(0, 0, 1)]]
METRIC = "fermion-weight evals/s and decorrelated samples/s, mixed vs FP64, 1 GB300"
UNIT = "weight evals/s"
NOMINAL = {"bf16": 2250.0, "tf32": 1100.0, "fp64": 1.25}  # TFLOP/s, dense, per GPU
FALLBACK = {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0}


def workload_name():
    return ("SLDQMC cumulative update, 16x16 lattice, beta=8, dtau=0.05 (M=160), mu=-0.5, xi=1, "
            "J1/J2/J3/Jtau effective action")


def env_rank():
    return (int(os.environ.get("RANK", 0)), int(os.environ.get("WORLD_SIZE", 1)),
            int(os.environ.get("LOCAL_RANK", 0)))


def peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    src = "fallback"
    vals = dict(FALLBACK)
    if os.path.exists(path):
        try:
            d = json.load(open(path))
            flat = {}

            def walk(o):
                for k, v in o.items():
                    if isinstance(v, dict):
                        walk(v)
                    else:
                        flat[k] = v
            walk(d)
            if "hbm_gbs" in flat:
                vals["hbm_gbs"] = float(flat["hbm_gbs"])
            if "bf16_tflops" in flat:
                vals["bf16_tflops"] = float(flat["bf16_tflops"])
            src = "measured (burst)"
            # the roofline kernels are timed inside a step of seconds-long runs:
            # the sustained (power-capped) figure applies where it was measured
            if "bf16_tflops_sustained" in flat:
                vals["bf16_tflops"] = float(flat["bf16_tflops_sustained"])
                src = "measured (sustained)"
        except Exception:
            pass
    vals["fp64_tflops"] = vals["bf16_tflops"] * NOMINAL["fp64"] / NOMINAL["bf16"]
    vals["tf32_tflops"] = vals["bf16_tflops"] * NOMINAL["tf32"] / NOMINAL["bf16"]
    vals["source"] = src
    return vals


class ClockSampler:
    """nvidia-smi clock and throttle-reason samples during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu):
        self.gpu = gpu
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits", "-lms", "200",
                 "-i", str(self.gpu)], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            threading.Thread(target=self._read, daemon=True).start()
        except OSError:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for l in self.lines:
            p = [x.strip() for x in l.split(",")]
            if len(p) < 9:
                continue
            try:
                sm.append(float(p[1]))
                mx = float(p[2])
            except ValueError:
                continue
            for n, v in zip(names, p[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(n)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": mx,
                "reasons": sorted(reasons), "samples": len(sm)}


def traffic_record(kernel_class):
    """Per-launch DRAM traffic of a kernel class from a committed ncu summary,
    valid only while the sources it depends on (the kernel, and the code that
    decides which launches it gets) are unchanged."""
    path = os.path.join(ROOT, "profiles", "traffic.json")
    if not os.path.exists(path):
        return None
    try:
        d = json.load(open(path)).get(kernel_class)
        if not d:
            return None
        h = hashlib.sha256()
        for f in d["sources"]:
            h.update(open(os.path.join(ROOT, "paper_1612_03804_gb300", "csrc", f), "rb").read())
        if h.hexdigest()[:16] != d["sha"]:
            return None
        return d
    except Exception:
        return None


def max_over_ranks(x, dist=None, device="cpu"):
    """Max of a per-rank scalar over all ranks (timing: the slowest rank sets the time)."""
    import torch
    if dist is None or not dist.is_initialized():
        return x
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def weak_scaling_value(units_per_rank, world, t_max):
    """Whole-job throughput: every rank processed units_per_rank in at most t_max."""
    return units_per_rank * world / t_max


def oracle_weight_sample(seed=1):
    """One single-flavour weight evaluation of the workload by the FP64 CPU
    oracle (as it stands, with the workload's n_wrap)."""
    from oracle import oracle as O
    from paper_1612_03804_gb300.inputs import uniform_field
    m = O.Model(WL["L"], WL["L"], t=WL["t"], mu=WL["mu"], xi=WL["xi"], beta=WL["beta"], dtau=WL["dtau"],
                n_wrap=WL["n_wrap"], J=WL["J"], h=WL["h"])
    s = uniform_field(seed, m.M, m.N)
    t0 = time.perf_counter()
    O.weight(m, s, -1)
    return time.perf_counter() - t0


def run_reference(args):
    rank, world, _ = env_rank()
    if rank != 0:
        return
    from oracle import oracle as O
    O.build()
    for w in range(args.warmup):
        oracle_weight_sample(100 + w)
    t0 = time.perf_counter()
    for k in range(args.steps):
        oracle_weight_sample(200 + k)
    T = time.perf_counter() - t0
    value = args.steps / T
    sample = "one single-flavour weight evaluation (16x16, M=160, n_wrap=10) per step, FP64 CPU oracle"
    out = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
           "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * T / args.steps,
           "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
           "data": "synthetic", "config": {"workload": workload_name(), "global_batch": 1, "seq_len": 160,
                                           "parallelism": "cpu-1-thread"},
           "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle", "sample": sample},
           "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out), flush=True)


def bare_couplings():
    """The bare Ising action log phi as an effective model over the same classes:
    -beta H = dtau J f_1 + K_tau f_tau, K_tau = -ln tanh(dtau h) / 2."""
    import math
    kt = -0.5 * math.log(math.tanh(WL["dtau"] * WL["h"]))
    return [-WL["dtau"] * WL["J"] / WL["beta"], 0.0, 0.0, -kt / WL["beta"]]


def train_effective_model(torch, sldqmc, args, dev_seed):
    """Steps i-ii: local DQMC on 8x8 at the workload couplings (started from
    configurations pre-thermalised under the bare Ising action), then the Eq. 3 fit."""
    import numpy as np
    from paper_1612_03804_gb300.inputs import batch_uniform
    Bt = args.train_chains
    ctx8 = sldqmc.Context(8, 8, t=WL["t"], mu=WL["mu"], xi=WL["xi"], beta=WL["beta"], dtau=WL["dtau"],
                          n_wrap=WL["n_wrap"], J=WL["J"], h=WL["h"], prec="fp64", max_batch=Bt)
    s = torch.from_numpy(batch_uniform(dev_seed, Bt, ctx8.M, ctx8.N)).cuda()
    ctx8.set_effective_model(CLASSES, np.array(bare_couplings()))
    for k in range(args.bare_sweeps):
        ctx8.eff_sweeps_batch_dev(s, 1, dev_seed, k, -1)
    ctx8.local_sweep_batch_dev(s, dev_seed, 0, args.thermalize, want_stats=False)
    cfgs = []
    sweep = args.thermalize
    while len(cfgs) * Bt < args.train_configs:
        ctx8.local_sweep_batch_dev(s, dev_seed, sweep, 1, want_stats=False)
        sweep += 1
        cfgs.append(s.cpu().numpy().copy())
    import numpy as np
    cfgs = np.concatenate(cfgs)[: args.train_configs]
    J, E0, r2 = ctx8.fit_effective_action(cfgs)
    ctx8.close()
    return J, E0, r2, len(cfgs)


def critical_point_context(torch, sldqmc, args, rank):
    """Decorrelation at the paper's finite-temperature critical point (beta=1,
    dtau=0.05, M=20, h=2.774, 16x16; fit on 8x8 as in the paper): acceptance and
    tau_int of |sum s| for 16 chains over args.tau_steps cumulative updates, with
    1, 10 and 100 effective-model sweeps per update (the paper moves the
    proposal through many effective sweeps so that one exact accept step
    decorrelates the chain)."""
    import math
    import numpy as np
    from paper_1612_03804_gb300.analysis import tau_int
    from paper_1612_03804_gb300.inputs import batch_uniform
    wl = dict(WL, beta=1.0)
    kt = -0.5 * math.log(math.tanh(wl["dtau"] * wl["h"]))
    bare = np.array([-wl["dtau"] * wl["J"] / wl["beta"], 0.0, 0.0, -kt / wl["beta"]])
    Bt = args.train_chains
    c8 = sldqmc.Context(8, 8, t=wl["t"], mu=wl["mu"], xi=wl["xi"], beta=wl["beta"], dtau=wl["dtau"], n_wrap=20,
                        J=wl["J"], h=wl["h"], prec="fp64", max_batch=Bt)
    s = torch.from_numpy(batch_uniform(8100 + rank, Bt, c8.M, c8.N)).cuda()
    c8.set_effective_model(CLASSES, bare)
    for k in range(args.bare_sweeps):
        c8.eff_sweeps_batch_dev(s, 1, 81, k, -1)
    c8.local_sweep_batch_dev(s, 81, 0, args.thermalize, want_stats=False)
    cfgs, sw = [], args.thermalize
    while len(cfgs) * Bt < args.train_configs:
        c8.local_sweep_batch_dev(s, 81, sw, 1, want_stats=False)
        sw += 1
        cfgs.append(s.cpu().numpy().copy())
    J, E0, r2 = c8.fit_effective_action(np.concatenate(cfgs)[: args.train_configs])
    c8.close()
    B = min(args.tau_chains, args.batch)
    ctx = sldqmc.Context(wl["L"], wl["L"], t=wl["t"], mu=wl["mu"], xi=wl["xi"], beta=wl["beta"], dtau=wl["dtau"],
                         n_wrap=20, J=wl["J"], h=wl["h"], prec=args.prec, max_batch=B)
    ctx.set_effective_model(CLASSES, J, E0)
    d_s = torch.from_numpy(batch_uniform(8200 + rank, B, ctx.M, ctx.N)).cuda()
    for k in range(args.eff_thermalize):
        ctx.eff_sweeps_batch_dev(d_s, 1, 82, k, -1)
    d_lw = torch.zeros(B, dtype=torch.float64, device="cuda")
    ctx.log_weight_batch_dev(d_s, d_lw)
    d_acc = torch.zeros(B, dtype=torch.int32, device="cuda")
    for w in range(args.warmup):
        ctx.cumulative_batch_dev(d_s, d_lw, 1, 83, w, 1, d_acc)
    # the same equilibrated start for every number of effective sweeps per update
    s0, lw0 = d_s.clone(), d_lw.clone()
    scan = []
    for n_eff in (1, 10, 100):
        d_s.copy_(s0)
        d_lw.copy_(lw0)
        d_acc.zero_()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        series = magnetisation_series(torch, ctx, d_s, d_lw, d_acc, 83 + n_eff, 100, args.tau_steps,
                                      n_eff).astype(np.float64)
        dt = time.perf_counter() - t0
        tau, window = tau_int(series)
        scan.append({"n_eff": n_eff, "accept_rate": float(d_acc.sum().item()) / (B * args.tau_steps),
                     "tau_int": tau, "tau_window": window, "steps_per_s": args.tau_steps / dt,
                     "decorrelated_samples_per_s": B * args.tau_steps / dt / tau,
                     "note": ("window reached" if window < args.tau_steps - 1 else
                              "window not reached: tau_int is a lower bound")})
    ctx.close()
    first = scan[0]
    return {"point": "16x16, beta=1, dtau=0.05 (M=20), h=2.774, mu=-0.5 (the paper's critical point), "
                     f"{B} chains, effective model fitted on 8x8 (R^2={r2:.6f})",
            "accept_rate": first["accept_rate"], "tau_int": first["tau_int"],
            "tau_window": first["tau_window"], "tau_steps": args.tau_steps,
            "steps_per_s": first["steps_per_s"],
            "n_eff_scan": scan}


def steps_timed(torch, ctx, d_s, d_lw, d_acc, seed, step0, K):
    st = torch.cuda.current_stream()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(st)
    for k in range(K):
        ctx.cumulative_batch_dev(d_s, d_lw, 1, seed, step0 + k, 1, d_acc)
    e1.record(st)
    e1.synchronize()
    return e0.elapsed_time(e1) / 1e3


def magnetisation_series(torch, ctx, d_s, d_lw, d_acc, seed, step0, K, n_eff=1):
    """|total magnetisation| of every chain after each of K further (untimed)
    cumulative updates of n_eff effective sweeps each."""
    out = torch.zeros((K, d_s.shape[0]), dtype=torch.float32, device="cuda")
    for k in range(K):
        ctx.cumulative_batch_dev(d_s, d_lw, n_eff, seed, step0 + k, 1, d_acc)
        out[k] = d_s.float().sum(dim=(1, 2)).abs()
    return out.cpu().numpy()


def run_ours(args):
    import numpy as np
    import torch
    rank, world, local = env_rank()
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    if rank == 0:
        import __graft_entry__
        __graft_entry__.build()
    if dist:
        dist.barrier()
    from paper_1612_03804_gb300 import sldqmc
    from paper_1612_03804_gb300.analysis import tau_int
    from paper_1612_03804_gb300.inputs import batch_uniform
    sldqmc.load()

    def barrier_sync():
        torch.cuda.synchronize()
        if dist:
            dist.barrier()
        torch.cuda.synchronize()

    def rank_max(x):
        return max_over_ranks(x, dist, "cuda")

    t_setup = time.perf_counter()
    if args.no_train:
        J, E0, r2, ncfg = bare_couplings(), 0.0, None, 0
    else:
        J, E0, r2, ncfg = train_effective_model(torch, sldqmc, args, 7000 + rank)
    t_setup = time.perf_counter() - t_setup
    B = args.batch
    seed = 123456789 + (rank << 20)
    nwrap = {}
    tune_log = {}
    for prec in {args.prec, "fp64"}:
        if args.n_wrap == "auto":
            from paper_1612_03804_gb300.tune import autotune_nwrap
            nwrap[prec], res = autotune_nwrap(WL["L"], WL["beta"], WL["dtau"], WL["mu"], prec, t=WL["t"], xi=WL["xi"])
            tune_log[prec] = [[r[0], round(r[1], 2), r[2]] for r in res]
        else:
            nwrap[prec] = int(args.n_wrap)

    def make_ctx(prec):
        c = sldqmc.Context(WL["L"], WL["L"], t=WL["t"], mu=WL["mu"], xi=WL["xi"], beta=WL["beta"],
                           dtau=WL["dtau"], n_wrap=nwrap[prec], J=WL["J"], h=WL["h"], prec=prec, max_batch=B)
        c.set_effective_model(CLASSES, J, E0)
        return c

    ctx = make_ctx(args.prec)
    V = ctx.V
    d_s = torch.from_numpy(batch_uniform(5000 + rank, B, ctx.M, ctx.N)).cuda()
    d_lw = torch.zeros(B, dtype=torch.float64, device="cuda")
    d_acc = torch.zeros(B, dtype=torch.int32, device="cuda")
    # start the chains in equilibrium of H_eff (cheap effective sweeps), where
    # the fitted model is accurate, then compute their exact log weights
    for k in range(args.eff_thermalize):
        ctx.eff_sweeps_batch_dev(d_s, 1, seed ^ 0x5A5A, k, -1)
    ctx.log_weight_batch_dev(d_s, d_lw)
    ctx.sync()
    # warm-up cumulative updates
    for w in range(args.warmup):
        ctx.cumulative_batch_dev(d_s, d_lw, 1, seed, w, 1, d_acc)
    ctx.sync()
    d_acc.zero_()
    sampler = ClockSampler(local)
    sampler.start()
    n0 = ctx.kernel_launches()
    barrier_sync()
    T = steps_timed(torch, ctx, d_s, d_lw, d_acc, seed, args.warmup, args.steps)
    barrier_sync()
    launches = ctx.kernel_launches() - n0
    clocks = sampler.stop()
    ctx.sync()
    Tmax = rank_max(T)
    value = weak_scaling_value(2 * B * args.steps, world, Tmax)
    accept_rate = float(d_acc.sum().item()) / (B * args.steps)
    # decorrelation: |magnetisation| series of a separate set of chains (fewer
    # chains, more steps; the per-chain dynamics does not depend on the batch)
    tau, window, tau_note = None, None, None
    samples_per_s = None
    if args.tau_steps > 0:
        Bt = min(args.tau_chains, B)
        t_s = d_s[:Bt].clone()
        t_lw = d_lw[:Bt].clone()
        t_acc = torch.zeros(Bt, dtype=torch.int32, device="cuda")
        series = magnetisation_series(torch, ctx, t_s, t_lw, t_acc, seed ^ 0x77, 10 ** 5,
                                      args.tau_steps).astype(np.float64)
        tau, window = tau_int(series)
        tau_note = ("window reached" if window < args.tau_steps - 1 else
                    "window not reached: tau_int is a lower bound, samples/s an upper bound")
        samples_per_s = (B * world * args.steps / Tmax) / tau

    # roofline: a profiled pass (CUDA events around every launch)
    ctx.profile(True)
    ctx.cumulative_batch_dev(d_s, d_lw, 1, seed, 10 ** 6, args.profile_steps, d_acc)
    prof = ctx.profile_read()
    ctx.profile(False)
    pk = peaks()
    dom = max(prof, key=lambda k: prof[k]["ms"])
    rec = prof[dom]
    achieved = rec["flops"] / (rec["ms"] * 1e-3) / 1e12 if rec["ms"] > 0 and rec["flops"] > 0 else None
    unit, note = "TFLOP/s", None
    if dom == "gemm_tc":
        # algorithmic flops (2 N^3 per slice product) against the ceiling of the
        # split mode: the tensor peak of its operand type / MMAs issued per product
        mmas = {"3xtf32": 5, "bf16x3": 6, "bf16": 1}[args.prec]
        base = pk["tf32_tflops"] if args.prec == "3xtf32" else pk["bf16_tflops"]
        bound, peak = "tensor", base / mmas
        note = f"{args.prec} ceiling = {'TF32' if args.prec == '3xtf32' else 'BF16'} peak / {mmas} MMAs per product"
    elif dom == "gemm_oz":
        # FP64-accurate products by digit splitting: 36 BF16 MMAs per product
        bound, peak = "tensor", pk["bf16_tflops"] / 36.0
        note = "FP64-equivalent flops; ceiling = BF16 peak / 36 digit products"
    else:
        bound, peak = "alu", pk["fp64_tflops"]
        note = "FP64 pipe"
    tr = traffic_record(dom)
    roofline = {"kernel": dom, "bound": bound, "achieved": achieved, "peak": peak, "unit": unit,
                "frac": (achieved / peak) if achieved else None,
                "traffic": tr["bytes_per_launch"] if tr else None,
                "peak_source": f"{pk['source']} (fp64 = bf16 x 1.25/2250, tf32 = bf16 x 1100/2250 nominal ratios)",
                "peak_note": note,
                "launches": rec["launches"], "ms_per_launch": rec["ms"] / max(rec["launches"], 1),
                "share": rec["ms"] / sum(v["ms"] for v in prof.values()),
                "breakdown_ms": {k: round(v["ms"], 3) for k, v in prof.items()}}

    # FP64-product path on the same workload
    fp64 = None
    if not args.skip_fp64:
        c64 = make_ctx("fp64")
        d_s64 = d_s.clone()
        d_lw64 = torch.zeros(B, dtype=torch.float64, device="cuda")
        c64.log_weight_batch_dev(d_s64, d_lw64)
        c64.cumulative_batch_dev(d_s64, d_lw64, 1, seed, 0, 1, d_acc)
        c64.sync()
        K64 = max(2, args.steps // 3)
        barrier_sync()
        T64 = steps_timed(torch, c64, d_s64, d_lw64, d_acc, seed, 1, K64)
        barrier_sync()
        T64 = rank_max(T64)
        fp64 = {"value": 2 * B * K64 * world / T64, "unit": UNIT, "steps": K64, "ms_per_step": 1e3 * T64 / K64}
        c64.close()

    # end to end through the host-buffer C ABI call (copies inside the timed region)
    h_s = torch.empty((B, ctx.M, ctx.N), dtype=torch.int8).pin_memory()
    h_s.copy_(d_s.cpu())
    h_lw = torch.empty(B, dtype=torch.float64).pin_memory()
    h_lw.copy_(d_lw.cpu())
    h_acc = np.zeros(B, dtype=np.int32)
    hs, hl = h_s.numpy(), h_lw.numpy()
    Ke = max(2, args.steps // 2)
    barrier_sync()
    t0 = time.perf_counter()
    for k in range(Ke):
        ctx.cumulative_batch(hs, hl, 1, seed, 2 * 10 ** 6 + k, 1, h_acc)
    torch.cuda.synchronize()
    Te = rank_max(time.perf_counter() - t0)
    e2e = {"value": 2 * B * Ke * world / Te, "unit": UNIT, "h2d_bytes_per_step": B * V + 8 * B,
           "d2h_bytes_per_step": B * V + 8 * B + 4 * B}

    crit = None
    if args.tau_steps > 0 and not args.no_train and not args.skip_critical:
        crit = critical_point_context(torch, sldqmc, args, rank)

    cpu = None
    if rank == 0 and not args.skip_cpu:
        from oracle import oracle as O
        O.build()
        t1 = oracle_weight_sample(1)
        cpu = {"value": 1.0 / t1, "unit": UNIT, "cores": 1, "kind": "oracle",
               "sample": "one single-flavour weight evaluation (16x16, M=160, n_wrap=10, uniform random field) "
                         "by the FP64 CPU oracle, one host thread"}
    if rank == 0:
        out = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
               "warmup": args.warmup, "ms_per_step": 1e3 * Tmax / args.steps, "higher_is_better": True,
               "scaling": "weak", "vs_baseline": None,
               "dtype": "tf32x2/fp32-acc products, f64 stabilisation" if args.prec == "3xtf32" else args.prec,
               "data": "synthetic (seeded random fields; effective model fitted on seeded local-DQMC runs)",
               "config": {"workload": workload_name(), "global_batch": B * world, "seq_len": ctx.M,
                          "lattice": f"{WL['L']}x{WL['L']}", "chains_per_gpu": B, "precision": args.prec,
                          "n_wrap": nwrap, "n_wrap_tuning": tune_log or None,
                          "parallelism": f"replicas x{world}", "l2": "working set > L2 (no flush)",
                          "fit": {"lattice": "8x8", "configs": ncfg, "J": [float(x) for x in J],
                                  "E0": E0, "r2": r2}, "setup_s": round(t_setup, 2)},
               "fp64": fp64, "decorrelated_samples_per_s": samples_per_s, "tau_int": tau,
               "tau_window": window, "tau_observable": "|sum s| per chain",
               "tau_series": {"chains": min(args.tau_chains, B), "steps": args.tau_steps, "note": tau_note}, "accept_rate": accept_rate,
               "critical_point": crit,
               "roofline": roofline, "cpu_baseline": cpu, "e2e": e2e, "clocks": clocks,
               "gpu_launches": launches}
        print(json.dumps(out), flush=True)
    ctx.close()
    if dist:
        dist.barrier()
        dist.destroy_process_group()


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--batch", type=int, default=128)
    ap.add_argument("--prec", default="3xtf32", choices=["3xtf32", "bf16x3", "bf16", "fp64"])
    ap.add_argument("--train-configs", type=int, default=2000)
    ap.add_argument("--train-chains", type=int, default=64)
    ap.add_argument("--thermalize", type=int, default=20)
    ap.add_argument("--bare-sweeps", type=int, default=200)
    ap.add_argument("--eff-thermalize", type=int, default=300)
    ap.add_argument("--tau-steps", type=int, default=300)
    ap.add_argument("--tau-chains", type=int, default=16)
    ap.add_argument("--n-wrap", default="auto", help="stabilisation interval, or 'auto' for the autotuner")
    ap.add_argument("--profile-steps", type=int, default=1)
    ap.add_argument("--skip-fp64", action="store_true")
    ap.add_argument("--no-train", action="store_true",
                    help="use the bare Ising couplings as H_eff (no local-DQMC training; for profiling runs)")
    ap.add_argument("--skip-cpu", action="store_true")
    ap.add_argument("--skip-critical", action="store_true")
    args = ap.parse_args()
    if args.warmup < 3:
        ap.error("--warmup must be >= 3")
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
