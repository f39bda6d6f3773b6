#!/usr/bin/env python
"""Benchmark of the self-learning DQMC hot path on one GB300.

Headline workload (the largest single-GPU configuration): one SLDQMC chain on
a 100x100 periodic lattice (N = 10^4 sites), t=1, mu=-0.5, xi=1, beta=10,
dtau=0.1 (M = 100 slices), n_wrap=10, dense exp(-dtau K) slice products in
split-TF32 on the tensor cores with FP64-accurate stabilisation, bare Ising
weight J=1, h=2.774; effective action with J1/J2/J3 (space) and J_tau
couplings fitted (Eq. 3) on local-DQMC configurations of an 8x8 lattice at
the same couplings and transferred to 100x100, as the paper transfers its
L=8 fit.  Only the running U, D, V factors, the chain buffers and E stay in
HBM (about 13 GB per flavour).

One step = one cumulative update (steps iii+iv): one sweep of N*M = 10^6
effective-model flips, the exact log weight of the proposal (both flavours,
i.e. two single-flavour fermion-weight evaluations through the stabilised
B-chain) and the Eq. 4 acceptance.  value = fermion-weight evaluations/s.
Beside it, in the same JSON line:
  fp64           -- the FP64-product path on the same lattice, extrapolated
                    from one timed block of n_wrap slices (labelled so);
  precision      -- log|det| relative/absolute error and max|dG| of the
                    benched mode against the uniform-field closed form;
  roofline       -- the dominant kernel class of a profiled step against
                    the peak of its own operand type (of measured);
  e2e            -- the same metric through the host-buffer C call, with the
                    copies inside the timed region;
  cpu_baseline   -- the FP64 CPU oracle on all host cores, extrapolated from
                    a timed sample of smaller weights by the N^3 M cost law;
  workloads      -- the other configurations:
     chains16  : 128 chains at 16x16, beta=8, dtau=0.05 (M=160), n_wrap by
                 the autotuner, with its own FP64 arm, e2e, decorrelation
                 and errors against the oracle on sampled configurations;
     uneven    : 64 chains, L in {12,16,20,24,32}, beta in {4,8}, split-TF32,
                 n_wrap per bucket by the autotuner, one CUDA graph per step,
                 with its fill fraction;
     precision : 32x32, beta=10, dtau=0.05 (M=200), n_wrap in {5,10,20},
                 FP64 / split-TF32 / split-BF16 / BF16 products;
     local4    : plain FP64 DQMC on 4x4 (weight, then local sweeps);
     critical  : decorrelation at the paper's critical point (beta=1);
     effmodel16: the paper's 16-coupling effective model, its 1 - R^2 range
                 scans and tau_int of local against cumulative updates for
                 L = 8, 12, 16, 24;
     local_delayed: local sweeps with immediate rank-1 against delayed
                 rank-32 Green's-function updates.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]
                  [--workloads large,chains16,uneven,precision,local4,critical]

Under torchrun each rank runs its own chains (weak scaling, no data-path
collective); every timed region is bracketed by a barrier and a device
synchronisation and its time is the maximum over ranks.
"""
import argparse
import hashlib
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

LARGE = dict(L=100, t=1.0, mu=-0.5, xi=1.0, beta=10.0, dtau=0.1, n_wrap=10, J=1.0, h=2.774)
CH16 = dict(L=16, t=1.0, mu=-0.5, xi=1.0, beta=8.0, dtau=0.05, n_wrap=10, J=1.0, h=2.774)
CLASSES = [[(1, 0, 0), (0, 1, 0)], [(1, 1, 0), (1, -1, 0)], [(2, 0, 0), (0, 2, 0)], [(0, 0, 1)]]
METRIC = "fermion-weight evals/s and decorrelated samples/s, mixed vs FP64, 1 GB300"
UNIT = "weight evals/s"
NOMINAL = {"bf16": 2250.0, "tf32": 1100.0, "fp64": 1.25}  # TFLOP/s, dense, per GPU
FALLBACK = {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0}
MMAS = {"3xtf32": 5, "bf16x3": 6, "bf16": 1}
SMS, SM_MAX_MHZ = 152, 2070.0
ALL_WORKLOADS = ("large", "chains16", "uneven", "precision", "local4", "critical", "effmodel16", "local_delayed")
# oracle sample for the CPU baseline and the reference arm: single-flavour
# weights at 16x16 with the headline's beta, dtau and n_wrap
CPU_SAMPLE = dict(L=16, beta=10.0, dtau=0.1, n_wrap=10)


def workload_name(wl=LARGE):
    M = int(round(wl["beta"] / wl["dtau"]))
    return (f"SLDQMC cumulative update, {wl['L']}x{wl['L']} lattice (N={wl['L'] ** 2}), beta={wl['beta']:g}, "
            f"dtau={wl['dtau']:g} (M={M}), n_wrap={wl['n_wrap']}, mu={wl['mu']:g}, xi={wl['xi']:g}, "
            "dense exp(-dtau K), J1/J2/J3/Jtau effective action")


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
    # FP32 CUDA-core peak from the unit counts and the maximum SM clock:
    # 152 SMs x 128 FP32 lanes x 2 flops per FMA x 2070 MHz
    vals["fp32_tflops"] = SMS * 128 * 2 * SM_MAX_MHZ * 1e6 / 1e12
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


def traffic_record(kernel_class, workload="chains16"):
    """Per-launch DRAM traffic of a kernel class on a workload from a committed
    ncu summary, valid only while the sources it depends on (the kernel, and
    the code that decides which launches it gets) are unchanged."""
    path = os.path.join(ROOT, "profiles", "traffic.json")
    if not os.path.exists(path):
        return None
    try:
        d = json.load(open(path)).get(workload, {}).get(kernel_class)
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


def dominant_site(sites):
    """The launch site (one kernel instantiation) with the most event time."""
    return max(sites, key=lambda k: sites[k]["ms"]) if sites else None


def roofline_entry(prof, prec, pk, workload, sites=None):
    """Roofline of the dominant kernel class of a profiled step.

    achieved = algorithmic flops of the class (2 N^3 per slice product; the
    FP64-equivalent flops of the digit-split products) / summed CUDA-event
    time of its launches.  peak = the measured peak of the operand type the
    class computes in: TF32 (measured BF16 x 1100/2250) for split-TF32 slice
    products, BF16 for split-BF16 / BF16 products and for the digit-split
    products (BF16 integer digits), FP64 (x 1.25/2250) for the FP64 pipe.
    issue_efficiency divides instead by that peak over the MMAs one
    algorithmic product issues (5 split-TF32, 6 split-BF16, 36 digit
    products)."""
    site = dominant_site(sites) if sites else None
    if site:
        # the dominant kernel: one launch site, classed for its peak
        rec = sites[site]
        dom = rec["cls"]
    else:
        dom = max(prof, key=lambda k: prof[k]["ms"])
        rec = prof[dom]
    achieved = rec["flops"] / (rec["ms"] * 1e-3) / 1e12 if rec["ms"] > 0 and rec["flops"] > 0 else None
    issue = None
    if dom == "gemm_tc":
        base = pk["tf32_tflops"] if prec == "3xtf32" else pk["bf16_tflops"]
        dtype = "tf32" if prec == "3xtf32" else "bf16"
        bound, peak, per = "tensor", base, MMAS.get(prec, 1)
        note = (f"{prec} slice products: algorithmic 2N^3 per product against the {dtype.upper()} peak; "
                f"issue_efficiency against {dtype.upper()} peak / {per} MMAs per product")
    elif dom == "sep":
        if prec == "fp64":
            bound, peak, per, dtype = "alu", pk["fp64_tflops"], 1, "fp64"
            note = "separable exp(-dtau K) convolutions in FP64 against the FP64 pipe"
        else:
            bound, peak, per, dtype = "alu", pk["fp32_tflops"], 3, "fp32"
            note = ("separable exp(-dtau K) convolutions in split FP32: algorithmic flops (2 N^2 (Lx+Ly) per slice) "
                    "against the FP32 CUDA-core peak (152 SMs x 128 lanes x 2 x 2070 MHz); issue_efficiency "
                    "against that peak / 3 FMAs per multiply-add")
    elif dom == "gemm_oz":
        bound, peak, per, dtype = "tensor", pk["bf16_tflops"], 36, "bf16"
        note = ("FP64-accurate digit-split products (Gram, Cholesky-QR updates and panels, R2R1, V update, "
                "LU updates): FP64-equivalent flops against the BF16 peak; issue_efficiency against "
                "BF16 peak / 36 digit products")
    else:
        bound, peak, per, dtype = "alu", pk["fp64_tflops"], 1, "fp64"
        note = "FP64 pipe (nominal FP64 rate scaled from the measured BF16 peak)"
    if achieved and per > 1:
        issue = achieved / (peak / per)
    tr = traffic_record(dom, workload)
    return {"kernel": site or dom, "class": dom, "bound": bound, "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
            "frac": (achieved / peak) if achieved else None, "dtype": dtype,
            "issue_efficiency": issue, "mmas_per_product": per,
            "traffic": tr["bytes_per_launch"] if tr else None,
            "peak_source": f"{pk['source']} (fp64 = bf16 x 1.25/2250, tf32 = bf16 x 1100/2250 nominal ratios), of measured",
            "peak_note": note,
            "launches": rec["launches"], "ms_per_launch": rec["ms"] / max(rec["launches"], 1),
            "share": rec["ms"] / max(sum(v["ms"] for v in prof.values()), 1e-30),
            "class_share": prof[dom]["ms"] / max(sum(v["ms"] for v in prof.values()), 1e-30),
            "breakdown_ms": {k: round(v["ms"], 3) for k, v in prof.items()},
            "breakdown_tflops": {k: (v["flops"] / (v["ms"] * 1e-3) / 1e12 if v["ms"] > 0 and v["flops"] > 0
                                     else None) for k, v in prof.items()}}


def profile_step(ctx, run):
    """One profiled pass (CUDA events around every launch, flavours
    serialised): returns (per-class record, per-site record)."""
    ctx.profile(True)
    run()
    sites = ctx.profile_read_sites()
    ctx.profile(False)
    prof = {k: {"launches": 0, "ms": 0.0, "flops": 0.0} for k in ctx.KERNEL_CLASSES}
    for v in sites.values():
        p = prof[v["cls"]]
        p["launches"] += v["launches"]
        p["ms"] += v["ms"]
        p["flops"] += v["flops"]
    return prof, sites


def site_table(sites, top=16):
    rows = sorted(sites.items(), key=lambda kv: -kv[1]["ms"])[:top]
    return {k: {"launches": v["launches"], "ms": round(v["ms"], 3),
                "tflops": (v["flops"] / (v["ms"] * 1e-3) / 1e12 if v["ms"] > 0 and v["flops"] > 0 else None)}
            for k, v in rows}


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


def weight_work(N, M, n_wrap):
    """Algorithmic flops of one single-flavour weight: dense slice products
    2 M N^3, one stabilisation of about 3.67 N^3 per block, the LU (2/3) N^3."""
    return 2.0 * M * N ** 3 + math.ceil(M / n_wrap) * 3.67 * N ** 3 + (2.0 / 3.0) * N ** 3


def closed_form_logdet(L, beta, t, mu_eff):
    """log det(1 + e^{-beta (K - shift)}) of the uniform field: sum_k log(1 + e^{-beta (eps_k - mu_eff)})."""
    import numpy as np
    k = 2 * np.pi * np.arange(L) / L
    eps = (-2 * t * (np.cos(k)[None, :] + np.cos(k)[:, None])).ravel() - mu_eff
    return float(np.sum(np.logaddexp(0.0, -beta * eps)))


def closed_form_green_row(L, beta, t, mu_eff):
    """g[dy, dx] with G_ij = g(r_i - r_j) for the uniform field: the inverse
    Fourier transform of 1 / (1 + e^{-beta (eps_k - mu_eff)}) on the L x L torus."""
    import numpy as np
    k = 2 * np.pi * np.arange(L) / L
    eps = -2 * t * (np.cos(k)[None, :] + np.cos(k)[:, None]) - mu_eff
    occ = 1.0 / (1.0 + np.exp(np.clip(-beta * eps, -700, 700)))
    return np.real(np.fft.ifft2(occ))


# ------------------------------------------------------------------ oracle
def oracle_sample_rate(n_weights, seed=1):
    """The FP64 CPU oracle as it stands, timed on every host core: n_weights
    independent single-flavour weight evaluations of the CPU_SAMPLE lattice,
    one per process.  Returns (weights/s at the sample size, cores, seconds)."""
    from oracle import oracle as O
    from paper_1612_03804_gb300.inputs import batch_uniform
    O.build()
    c = CPU_SAMPLE
    m = O.Model(c["L"], c["L"], t=1.0, mu=-0.5, xi=1.0, beta=c["beta"], dtau=c["dtau"], n_wrap=c["n_wrap"])
    fields = batch_uniform(seed, n_weights, m.M, m.N)
    cores = len(os.sched_getaffinity(0))
    t0 = time.perf_counter()
    O.weight_many(m, fields, -1, workers=cores)
    dt = time.perf_counter() - t0
    return n_weights / dt, min(cores, n_weights), dt


def extrapolate_oracle(rate, wl):
    """Scale an oracle rate at CPU_SAMPLE to the workload by the cost law
    M N^3 of its dense products and per-slice Householder QR."""
    c = CPU_SAMPLE
    Ns, Ms = c["L"] ** 2, int(round(c["beta"] / c["dtau"]))
    N, M = wl["L"] ** 2, int(round(wl["beta"] / wl["dtau"]))
    return rate * (Ns / N) ** 3 * (Ms / M)


def run_reference(args):
    rank, world, _ = env_rank()
    if rank != 0:
        return
    cores = len(os.sched_getaffinity(0))
    for w in range(args.warmup):
        oracle_sample_rate(cores, seed=100 + w)
    t_tot = 0.0
    for k in range(args.steps):
        _, _, dt = oracle_sample_rate(cores, seed=200 + k)
        t_tot += dt
    rate = args.steps * cores / t_tot
    value = extrapolate_oracle(rate, LARGE)
    c = CPU_SAMPLE
    sample = (f"each step: {cores} independent single-flavour weight evaluations ({c['L']}x{c['L']}, "
              f"beta={c['beta']:g}, dtau={c['dtau']:g}, n_wrap={c['n_wrap']}) by the FP64 CPU oracle, one per "
              f"host core; {rate:.4g} weights/s there, extrapolated to 100x100, M=100 by the M N^3 cost law "
              "(labelled extrapolated)")
    out = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
           "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * t_tot / args.steps,
           "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
           "data": "synthetic", "extrapolated": True,
           "config": {"workload": workload_name(LARGE), "global_batch": 1, "seq_len": 100,
                      "parallelism": f"cpu-{cores}-processes"},
           "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": sample},
           "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out), flush=True)


# ---------------------------------------------------------------- helpers
def bare_couplings(wl):
    """The bare Ising action log phi as an effective model over the same classes:
    -beta H = dtau J f_1 + K_tau f_tau, K_tau = -ln tanh(dtau h) / 2."""
    kt = -0.5 * math.log(math.tanh(wl["dtau"] * wl["h"]))
    return [-wl["dtau"] * wl["J"] / wl["beta"], 0.0, 0.0, -kt / wl["beta"]]


def train_effective_model(torch, sldqmc, wl, args, dev_seed, n_wrap=None):
    """Steps i-ii: local DQMC on 8x8 at the workload couplings (started from
    configurations pre-thermalised under the bare Ising action), then the Eq. 3 fit."""
    import numpy as np
    from paper_1612_03804_gb300.inputs import batch_uniform
    Bt = args.train_chains
    ctx8 = sldqmc.Context(8, 8, t=wl["t"], mu=wl["mu"], xi=wl["xi"], beta=wl["beta"], dtau=wl["dtau"],
                          n_wrap=n_wrap or wl["n_wrap"], J=wl["J"], h=wl["h"], prec="fp64", max_batch=Bt)
    s = torch.from_numpy(batch_uniform(dev_seed, Bt, ctx8.M, ctx8.N)).cuda()
    ctx8.set_effective_model(CLASSES, np.array(bare_couplings(wl)))
    for k in range(args.bare_sweeps):
        ctx8.eff_sweeps_batch_dev(s, 1, dev_seed, k, -1)
    ctx8.local_sweep_batch_dev(s, dev_seed, 0, args.thermalize, want_stats=False)
    cfgs = []
    sweep = args.thermalize
    while len(cfgs) * Bt < args.train_configs:
        ctx8.local_sweep_batch_dev(s, dev_seed, sweep, 1, want_stats=False)
        sweep += 1
        cfgs.append(s.cpu().numpy().copy())
    cfgs = np.concatenate(cfgs)[: args.train_configs]
    J, E0, r2 = ctx8.fit_effective_action(cfgs)
    ctx8.close()
    return J, E0, r2, len(cfgs)


def steps_timed(torch, ctx, d_s, d_lw, d_acc, seed, step0, K, n_eff=1):
    st = torch.cuda.current_stream()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(st)
    for k in range(K):
        ctx.cumulative_batch_dev(d_s, d_lw, n_eff, seed, step0 + k, 1, d_acc)
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


def make_ctx(sldqmc, wl, prec, B, n_wrap, J=None, E0=0.0, beta=None):
    c = sldqmc.Context(wl["L"], wl["L"], t=wl["t"], mu=wl["mu"], xi=wl["xi"], beta=beta or wl["beta"],
                       dtau=wl["dtau"], n_wrap=n_wrap, J=wl["J"], h=wl["h"], prec=prec, max_batch=B)
    if J is not None:
        c.set_effective_model(CLASSES, J, E0)
    return c


class Env:
    """Per-process state shared by the workloads: torch, the binding, the
    process group and the timing helpers."""

    def __init__(self, args):
        import torch
        self.args = args
        self.torch = torch
        self.rank, self.world, self.local = env_rank()
        torch.cuda.set_device(self.local)
        self.dist = None
        if self.world > 1:
            import torch.distributed as dist
            dist.init_process_group("nccl")
            self.dist = dist
        if self.rank == 0:
            import __graft_entry__
            __graft_entry__.build()
        if self.dist:
            self.dist.barrier()
        from paper_1612_03804_gb300 import sldqmc
        self.sldqmc = sldqmc
        sldqmc.load()

    def barrier_sync(self):
        self.torch.cuda.synchronize()
        if self.dist:
            self.dist.barrier()
        self.torch.cuda.synchronize()

    def rank_max(self, x):
        return max_over_ranks(x, self.dist, "cuda")


# --------------------------------------------------------- headline: 100x100
def run_large(env):
    """Config 5: one chain on 100x100, the headline line."""
    import numpy as np
    from paper_1612_03804_gb300.inputs import uniform_field
    torch, sldqmc, args = env.torch, env.sldqmc, env.args
    wl = dict(LARGE, L=args.large_L)
    N, M, nw = wl["L"] ** 2, int(round(wl["beta"] / wl["dtau"])), wl["n_wrap"]
    B = 1
    t_setup = time.perf_counter()
    if args.no_train:
        J, E0, r2, ncfg = bare_couplings(wl), 0.0, None, 0
    else:
        J, E0, r2, ncfg = train_effective_model(torch, sldqmc, wl, args, 9000 + env.rank)
    ctx = make_ctx(sldqmc, wl, args.prec, B, nw, J, E0)
    if args.prec != "fp64":
        ctx.set_tile_n(args.large_tile)
    seed = 987654321 + (env.rank << 20)
    d_s = torch.from_numpy(uniform_field(5100 + env.rank, M, N)[None]).cuda()
    d_lw = torch.zeros(B, dtype=torch.float64, device="cuda")
    d_acc = torch.zeros(B, dtype=torch.int32, device="cuda")
    for k in range(args.large_eff_thermalize):
        ctx.eff_sweeps_batch_dev(d_s, 1, seed ^ 0x5A5A, k, -1)
    ctx.log_weight_batch_dev(d_s, d_lw)
    ctx.sync()
    t_setup = time.perf_counter() - t_setup
    for w in range(args.warmup):
        ctx.cumulative_batch_dev(d_s, d_lw, 1, seed, w, 1, d_acc)
    ctx.sync()
    d_acc.zero_()
    sampler = ClockSampler(env.local)
    sampler.start()
    n0 = ctx.kernel_launches()
    env.barrier_sync()
    T = steps_timed(torch, ctx, d_s, d_lw, d_acc, seed, args.warmup, args.steps)
    env.barrier_sync()
    launches = ctx.kernel_launches() - n0
    clocks = sampler.stop()
    ctx.sync()
    Tmax = env.rank_max(T)
    value = weak_scaling_value(2 * B * args.steps, env.world, Tmax)
    accept_rate = float(d_acc.sum().item()) / (B * args.steps)

    # roofline: one profiled step (CUDA events around every launch; flavours serialised)
    prof, sites = profile_step(ctx, lambda: ctx.cumulative_batch_dev(d_s, d_lw, 1, seed, 10 ** 6, 1, d_acc))
    pk = peaks()
    roof = roofline_entry(prof, args.prec, pk, "large", sites)
    roof["serialised_step_ms"] = sum(v["ms"] for v in prof.values())
    roof["sites"] = site_table(sites)

    # error of the benched mode: the uniform field has a closed form (the
    # oracle's dense FP64 at N = 10^4, ~10^14 flops per weight, is beyond the
    # host cores); eta = -1, s = +1 shifts mu by -xi
    u = torch.ones((1, M, N), dtype=torch.int8, device="cuda")
    ld = torch.zeros(1, dtype=torch.float64, device="cuda")
    ctx.weight_batch_dev(u, -1, ld)
    G = torch.zeros((1, N, N), dtype=torch.float64, device="cuda")
    ctx.green_batch_dev(u, -1, 0, G)
    ctx.sync()
    mu_eff = wl["mu"] - wl["xi"]
    cf = closed_form_logdet(wl["L"], wl["beta"], wl["t"], mu_eff)
    g = torch.from_numpy(closed_form_green_row(wl["L"], wl["beta"], wl["t"], mu_eff)).cuda()
    L = wl["L"]
    idx = torch.arange(N, device="cuda")
    x, y = idx % L, idx // L
    dG = 0.0
    for r0 in range(0, N, 1000):
        rows = idx[r0:r0 + 1000]
        ref = g[(y[rows, None] - y[None, :]) % L, (x[rows, None] - x[None, :]) % L]
        dG = max(dG, float((G[0, r0:r0 + 1000] - ref).abs().max()))
    precision = {"reference": "uniform-field closed form sum_k log(1+e^{-beta(eps_k-mu+xi)}) and its "
                              "translation-invariant G (eta=-1, s=+1)",
                 "logdet": float(ld.item()), "closed_form": cf,
                 "logdet_rel_err": abs(float(ld.item()) - cf) / abs(cf),
                 "logdet_abs_err": abs(float(ld.item()) - cf), "max_abs_dG": dG,
                 "bound": "1e-6 relative (log det), stated per result"}
    del G

    # end to end through the host-buffer C call (copies inside the timed region)
    h_s = torch.empty((B, M, N), dtype=torch.int8).pin_memory()
    h_s.copy_(d_s.cpu())
    h_lw = torch.empty(B, dtype=torch.float64).pin_memory()
    h_lw.copy_(d_lw.cpu())
    h_acc = np.zeros(B, dtype=np.int32)
    hs, hl = h_s.numpy(), h_lw.numpy()
    Ke = max(2, args.steps // 5)
    env.barrier_sync()
    t0 = time.perf_counter()
    for k in range(Ke):
        ctx.cumulative_batch(hs, hl, 1, seed, 2 * 10 ** 6 + k, 1, h_acc)
    torch.cuda.synchronize()
    Te = env.rank_max(time.perf_counter() - t0)
    e2e = {"value": 2 * B * Ke * env.world / Te, "unit": UNIT, "steps": Ke,
           "h2d_bytes_per_step": B * M * N + 8 * B, "d2h_bytes_per_step": B * M * N + 8 * B + 4 * B}
    sep = separable_arm(env, ctx, d_s, d_lw, d_acc, seed, u, mu_eff, cf) if not args.skip_separable else None
    if sep:
        sep["dense_slice_products_ms_per_step"] = prof["gemm_tc"]["ms"] + prof["gemm_f64"]["ms"]
    ctx.close()
    del d_s, u

    # FP64-product path: one block of n_wrap slices (a beta = n_wrap dtau chain:
    # products, one stabilisation, the LU) timed, times the M / n_wrap blocks
    fp64 = None
    if not args.skip_fp64:
        c64 = make_ctx(sldqmc, wl, "fp64", 1, nw, beta=nw * wl["dtau"])
        s1 = torch.from_numpy(uniform_field(5200, nw, N)[None]).cuda()
        l1 = torch.zeros(1, dtype=torch.float64, device="cuda")
        env.barrier_sync()
        st = torch.cuda.current_stream()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(st)
        c64.weight_batch_dev(s1, -1, l1)
        e1.record(st)
        c64.sync()
        t_block = env.rank_max(e0.elapsed_time(e1) / 1e3)
        c64.close()
        t_w = t_block * (M // nw)
        fp64 = {"value": env.world / t_w, "unit": UNIT, "extrapolated": True,
                "s_per_block": t_block, "s_per_weight": t_w,
                "note": f"one block of {nw} FP64 slice products + stabilisation + LU timed, x {M // nw} blocks"}

    cpu = None
    if env.rank == 0 and not args.skip_cpu:
        cores = len(os.sched_getaffinity(0))
        rate, used, dt = oracle_sample_rate(cores, seed=1)
        c = CPU_SAMPLE
        cpu = {"value": extrapolate_oracle(rate, wl), "unit": UNIT, "cores": used, "kind": "oracle",
               "extrapolated": True,
               "sample": (f"{cores} independent single-flavour weights ({c['L']}x{c['L']}, beta={c['beta']:g}, "
                          f"dtau={c['dtau']:g}, n_wrap={c['n_wrap']}) by the FP64 CPU oracle, one per host core, "
                          f"{dt:.1f} s: {rate:.4g} weights/s, scaled to 100x100, M=100 by the M N^3 cost law")}
    out = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": env.world, "steps": args.steps,
           "warmup": args.warmup, "ms_per_step": 1e3 * Tmax / args.steps, "higher_is_better": True,
           "scaling": "weak", "vs_baseline": None,
           "dtype": "tf32x2/fp32-acc products, f64 stabilisation" if args.prec == "3xtf32" else args.prec,
           "data": "synthetic (seeded random fields; effective model fitted on seeded local-DQMC runs)",
           "config": {"workload": workload_name(wl), "global_batch": B * env.world, "seq_len": M,
                      "lattice": f"{wl['L']}x{wl['L']}", "chains_per_gpu": B, "precision": args.prec,
                      "n_wrap": nw, "tile_n": args.large_tile if args.prec != "fp64" else None,
                      "parallelism": f"replicas x{env.world}",
                      "l2": "working set > L2 (each N x N FP64 matrix is 800 MB; no flush)",
                      "fit": {"lattice": "8x8", "configs": ncfg, "J": [float(x) for x in J], "E0": E0, "r2": r2},
                      "setup_s": round(t_setup, 2)},
           "ms_per_weight": 1e3 * Tmax / (2 * B * args.steps),
           "ms_per_accept_step": 1e3 * Tmax / args.steps,
           "accept_rate": accept_rate, "fp64": fp64, "precision": precision, "separable": sep,
           "decorrelated_samples_per_s": None,
           "decorrelation_note": ("tau_int needs a series of many cumulative steps (seconds each at 100x100); "
                                  "it is measured on the chains16 workload (workloads.chains16)"),
           "roofline": roof, "cpu_baseline": cpu, "e2e": e2e, "clocks": clocks, "gpu_launches": launches}
    return out


def separable_arm(env, ctx, d_s, d_lw, d_acc, seed, u=None, mu_eff=None, cf=None, prec=None):
    """The same chains with exp(-dtau K) in its exact separable form (two
    circular convolutions per slice instead of a dense product): weight
    evaluations/s, the closed-form error and the slice-product time of a
    profiled step against the dense one."""
    torch, args = env.torch, env.args
    B = d_s.shape[0]
    ctx.set_kinetic_form("separable")
    ctx.cumulative_batch_dev(d_s, d_lw, 1, seed, 3 * 10 ** 6, 1, d_acc)
    ctx.sync()
    K = 2
    env.barrier_sync()
    T = env.rank_max(steps_timed(torch, ctx, d_s, d_lw, d_acc, seed, 3 * 10 ** 6 + 1, K))
    prof, sites = profile_step(ctx, lambda: ctx.cumulative_batch_dev(d_s, d_lw, 1, seed, 4 * 10 ** 6, 1, d_acc))
    out = {"value": 2 * B * K * env.world / T, "unit": UNIT, "steps": K, "ms_per_step": 1e3 * T / K,
           "slice_products_ms_per_step": prof["sep"]["ms"],
           "roofline": roofline_entry(prof, prec or args.prec, peaks(), "none", sites),
           "note": "exp(-dtau K) = e^{dtau mu} E1x (x) E1y applied as two circular convolutions per row of the "
                   "running product, rows resident in shared memory for a whole block"}
    if u is not None:
        ld = torch.zeros(1, dtype=torch.float64, device="cuda")
        ctx.weight_batch_dev(u, -1, ld)
        ctx.sync()
        out["closed_form_rel_err"] = abs(float(ld.item()) - cf) / abs(cf)
    ctx.set_kinetic_form("dense")
    return out


# ------------------------------------------------ 16x16 x 128 chains (config 2)
def oracle_errors(torch, ctx, d_s, m_kw, n_sample):
    """Errors of the context's mode against the FP64 CPU oracle on the first
    n_sample configurations of d_s (both flavours), and max|dG| on the first."""
    import numpy as np
    from oracle import oracle as O
    fields = d_s[:n_sample].cpu().numpy()
    m = O.Model(**m_kw)
    rel, ab = [], []
    for eta in (1, -1):
        ref = O.weight_many(m, fields, eta)
        ld = torch.zeros(n_sample, dtype=torch.float64, device="cuda")
        ctx.weight_batch_dev(d_s[:n_sample], eta, ld)
        ctx.sync()
        ld = ld.cpu().numpy()
        r = np.array([x[0] for x in ref])
        rel.append(np.abs(ld - r) / np.abs(r))
        ab.append(np.abs(ld - r))
    _, _, Gref = O.weight(m, fields[0], -1, want_G=True)
    G = torch.zeros((1, m.N, m.N), dtype=torch.float64, device="cuda")
    ctx.green_batch_dev(d_s[:1], -1, 0, G)
    ctx.sync()
    return {"reference": f"FP64 CPU oracle (n_wrap={m.n_wrap}), {n_sample} sampled chain configurations, both flavours",
            "logdet_rel_err": float(np.max(rel)), "logdet_abs_err": float(np.max(ab)),
            "max_abs_dG": float(np.abs(G[0].cpu().numpy() - Gref).max())}


def run_chains16(env):
    import numpy as np
    from paper_1612_03804_gb300.analysis import tau_int
    from paper_1612_03804_gb300.inputs import batch_uniform
    torch, sldqmc, args = env.torch, env.sldqmc, env.args
    wl = CH16
    t_setup = time.perf_counter()
    if args.no_train:
        J, E0, r2, ncfg = bare_couplings(wl), 0.0, None, 0
    else:
        J, E0, r2, ncfg = train_effective_model(torch, sldqmc, wl, args, 7000 + env.rank)
    t_setup = time.perf_counter() - t_setup
    B = args.batch
    seed = 123456789 + (env.rank << 20)
    nwrap, tiles, tune_log = {}, {}, {}
    for prec in {args.prec, "fp64"}:
        if args.n_wrap == "auto":
            from paper_1612_03804_gb300.tune import autotune_schedule
            nwrap[prec], tiles[prec], res = autotune_schedule(wl["L"], wl["beta"], wl["dtau"], wl["mu"], prec,
                                                              t=wl["t"], xi=wl["xi"])
            tune_log[prec] = [[r[0], r[1], round(r[2], 2), r[3]] for r in res]
        else:
            nwrap[prec], tiles[prec] = int(args.n_wrap), 64
    ctx = make_ctx(sldqmc, wl, args.prec, B, nwrap[args.prec], J, E0)
    ctx.set_tile_n(tiles[args.prec])
    d_s = torch.from_numpy(batch_uniform(5000 + env.rank, B, ctx.M, ctx.N)).cuda()
    d_lw = torch.zeros(B, dtype=torch.float64, device="cuda")
    d_acc = torch.zeros(B, dtype=torch.int32, device="cuda")
    for k in range(args.eff_thermalize):
        ctx.eff_sweeps_batch_dev(d_s, 1, seed ^ 0x5A5A, k, -1)
    ctx.log_weight_batch_dev(d_s, d_lw)
    ctx.sync()
    for w in range(args.warmup):
        ctx.cumulative_batch_dev(d_s, d_lw, 1, seed, w, 1, d_acc)
    ctx.sync()
    d_acc.zero_()
    K = args.steps
    n0 = ctx.kernel_launches()
    env.barrier_sync()
    T = steps_timed(torch, ctx, d_s, d_lw, d_acc, seed, args.warmup, K)
    env.barrier_sync()
    launches = ctx.kernel_launches() - n0
    Tmax = env.rank_max(T)
    value = weak_scaling_value(2 * B * K, env.world, Tmax)
    accept_rate = float(d_acc.sum().item()) / (B * K)

    # decorrelation: |magnetisation| series of 16 of the chains, long enough
    # for the Madras-Sokal window
    tau = window = tau_note = samples_per_s = None
    if args.tau_steps > 0:
        Bt = min(args.tau_chains, B)
        t_s, t_lw = d_s[:Bt].clone(), d_lw[:Bt].clone()
        t_acc = torch.zeros(Bt, dtype=torch.int32, device="cuda")
        series = magnetisation_series(torch, ctx, t_s, t_lw, t_acc, seed ^ 0x77, 10 ** 5,
                                      args.tau_steps).astype(np.float64)
        tau, window = tau_int(series)
        tau_note = ("window reached" if window < args.tau_steps - 1 else
                    "window not reached: tau_int is a lower bound, samples/s an upper bound")
        samples_per_s = (B * env.world * K / Tmax) / tau

    prof, sites = profile_step(ctx, lambda: ctx.cumulative_batch_dev(d_s, d_lw, 1, seed, 10 ** 6, 1, d_acc))
    roof = roofline_entry(prof, args.prec, peaks(), "chains16", sites)
    roof["sites"] = site_table(sites)

    errors = None
    if env.rank == 0 and args.oracle_sample > 0:
        errors = oracle_errors(torch, ctx, d_s, dict(Lx=wl["L"], Ly=wl["L"], t=wl["t"], mu=wl["mu"], xi=wl["xi"],
                                                     beta=wl["beta"], dtau=wl["dtau"], n_wrap=10, J=wl["J"],
                                                     h=wl["h"]), args.oracle_sample)

    fp64 = None
    if not args.skip_fp64:
        c64 = make_ctx(sldqmc, wl, "fp64", B, nwrap["fp64"], J, E0)
        d_s64 = d_s.clone()
        d_lw64 = torch.zeros(B, dtype=torch.float64, device="cuda")
        c64.log_weight_batch_dev(d_s64, d_lw64)
        c64.cumulative_batch_dev(d_s64, d_lw64, 1, seed, 0, 1, d_acc)
        c64.sync()
        K64 = max(2, K // 3)
        env.barrier_sync()
        T64 = env.rank_max(steps_timed(torch, c64, d_s64, d_lw64, d_acc, seed, 1, K64))
        fp64 = {"value": 2 * B * K64 * env.world / T64, "unit": UNIT, "steps": K64, "ms_per_step": 1e3 * T64 / K64}
        if not args.skip_separable:
            p_dense, _ = profile_step(c64, lambda: c64.cumulative_batch_dev(d_s64, d_lw64, 1, seed, 5 * 10 ** 6, 1,
                                                                            d_acc))
            sp = separable_arm(env, c64, d_s64, d_lw64, d_acc, seed, prec="fp64")
            # in the FP64 mode the stabilisation also runs on the FP64 GEMM: the dense
            # slice products are what the separable step no longer spends there
            sp["dense_slice_products_ms_per_step"] = p_dense["gemm_f64"]["ms"] - sp["roofline"]["breakdown_ms"]["gemm_f64"]
            fp64["separable"] = sp
        c64.close()

    sep = separable_arm(env, ctx, d_s, d_lw, d_acc, seed) if not args.skip_separable else None
    if sep:
        sep["dense_slice_products_ms_per_step"] = prof["gemm_tc"]["ms"] + prof["gemm_f64"]["ms"]
    V = ctx.V
    h_s = torch.empty((B, ctx.M, ctx.N), dtype=torch.int8).pin_memory()
    h_s.copy_(d_s.cpu())
    h_lw = torch.empty(B, dtype=torch.float64).pin_memory()
    h_lw.copy_(d_lw.cpu())
    h_acc = np.zeros(B, dtype=np.int32)
    hs, hl = h_s.numpy(), h_lw.numpy()
    Ke = max(2, K // 2)
    env.barrier_sync()
    t0 = time.perf_counter()
    for k in range(Ke):
        ctx.cumulative_batch(hs, hl, 1, seed, 2 * 10 ** 6 + k, 1, h_acc)
    torch.cuda.synchronize()
    Te = env.rank_max(time.perf_counter() - t0)
    e2e = {"value": 2 * B * Ke * env.world / Te, "unit": UNIT, "h2d_bytes_per_step": B * V + 8 * B,
           "d2h_bytes_per_step": B * V + 8 * B + 4 * B}
    ctx.close()

    cpu = None
    if env.rank == 0 and not args.skip_cpu:
        from oracle import oracle as O
        from paper_1612_03804_gb300.inputs import batch_uniform as bu
        cores = len(os.sched_getaffinity(0))
        m = O.Model(wl["L"], wl["L"], t=wl["t"], mu=wl["mu"], xi=wl["xi"], beta=wl["beta"], dtau=wl["dtau"],
                    n_wrap=10)
        t0 = time.perf_counter()
        O.weight_many(m, bu(1, cores, m.M, m.N), -1, workers=cores)
        dt = time.perf_counter() - t0
        cpu = {"value": cores / dt, "unit": UNIT, "cores": cores, "kind": "oracle",
               "sample": f"{cores} single-flavour weights of this workload (n_wrap=10), one per host core, {dt:.1f} s"}
    return {"workload": workload_name(dict(wl, n_wrap=nwrap[args.prec])), "value": value, "unit": UNIT,
            "chains": B * env.world, "steps": K, "ms_per_step": 1e3 * Tmax / K, "precision": args.prec,
            "n_wrap": nwrap, "tile_n": tiles, "tuning": tune_log or None,
            "tuning_columns": ["n_wrap", "tile_n", "ms per batch of 16", "max rel log-det deviation"],
            "accept_rate": accept_rate,
            "fit": {"lattice": "8x8", "configs": ncfg, "J": [float(x) for x in J], "E0": E0, "r2": r2},
            "setup_s": round(t_setup, 2), "fp64": fp64, "separable": sep, "errors_vs_oracle": errors,
            "decorrelated_samples_per_s": samples_per_s, "tau_int": tau, "tau_window": window,
            "tau_observable": "|sum s| per chain",
            "tau_series": {"chains": min(args.tau_chains, B), "steps": args.tau_steps, "note": tau_note},
            "roofline": roof, "cpu_baseline": cpu, "e2e": e2e, "gpu_launches": launches}


# ------------------------------------------------- 64 uneven chains (config 4)
UNEVEN_L = (12, 16, 20, 24, 32)
UNEVEN_BETA = (4.0, 8.0)


def uneven_buckets(n_chains=64):
    """Chain c: L = UNEVEN_L[c mod 5], beta = UNEVEN_BETA[(c div 5) mod 2]."""
    counts = {}
    for c in range(n_chains):
        key = (UNEVEN_L[c % 5], UNEVEN_BETA[(c // 5) % 2])
        counts[key] = counts.get(key, 0) + 1
    return counts


def fill_fraction(work_uneven, t_uneven, work_full, t_full):
    """Algorithmic flop rate of the uneven batch relative to that of a full
    uniform batch measured in the same run (1.0: the uneven chains keep the
    GPU as busy as the best-filled workload)."""
    return (work_uneven / t_uneven) / (work_full / t_full)


def run_uneven(env, full_rate=None):
    import numpy as np
    from paper_1612_03804_gb300.inputs import batch_uniform
    from paper_1612_03804_gb300.tune import autotune_schedule
    torch, sldqmc, args = env.torch, env.sldqmc, env.args
    dtau, mu = 0.05, -0.5
    members, tuned, work = [], {}, 0.0
    t_setup = time.perf_counter()
    for k, ((L, beta), B) in enumerate(sorted(uneven_buckets().items())):
        nw, tile, _ = autotune_schedule(L, beta, dtau, mu, args.prec, batch=2, reps=1)
        tuned[f"{L}x{L} beta={beta:g}"] = {"chains": B, "n_wrap": nw, "tile_n": tile}
        wl = dict(CH16, L=L, beta=beta)
        ctx = make_ctx(sldqmc, wl, args.prec, B, nw, bare_couplings(wl))
        ctx.set_tile_n(tile)
        s = torch.from_numpy(batch_uniform(900 + k + 100 * env.rank, B, ctx.M, ctx.N)).cuda()
        ctx.eff_sweeps_batch_dev(s, 20, 5, 0, -1)
        lw = torch.zeros(B, dtype=torch.float64, device="cuda")
        ctx.log_weight_batch_dev(s, lw)
        acc = torch.zeros(B, dtype=torch.int32, device="cuda")
        ctx.sync()
        members.append((ctx, s, lw, acc, 7000 + k + (env.rank << 20)))
        work += B * 2 * weight_work(L * L, ctx.M, nw)
    g = sldqmc.Graph(members, n_eff=1, step0=0)
    for _ in range(args.warmup):
        g.launch(1)
    g.sync()
    t_setup = time.perf_counter() - t_setup
    K = max(2, min(args.steps, 10))
    env.barrier_sync()
    t0 = time.perf_counter()
    g.launch(K)
    g.sync()
    T = env.rank_max(time.perf_counter() - t0)
    launches = sum(m[0].kernel_launches() for m in members)
    accepted = sum(int(m[3].sum().item()) for m in members)
    g.close()
    for m in members:
        m[0].close()
    out = {"workload": "64 SLDQMC chains, L in {12,16,20,24,32} x beta in {4,8}, dtau=0.05, mu=-0.5, xi=1, "
                       f"{args.prec} products, FP64 stabilisation, one CUDA graph per step (replay)",
           "value": 2 * 64 * K * env.world / T, "unit": UNIT, "steps": K, "ms_per_step": 1e3 * T / K,
           "buckets": tuned, "accept_rate": accepted / (64.0 * (K + args.warmup)),
           "algorithmic_tflops": work * K / T / 1e12, "setup_s": round(t_setup, 2),
           "kernel_launches_total": launches}
    if full_rate:
        out["fill_fraction"] = (work * K / T) / full_rate
        out["fill_note"] = ("algorithmic flop rate (2 M N^3 products + 3.67 N^3 per block + 2/3 N^3 LU per weight) "
                            "relative to the 128-chain 16x16 workload of the same run")
    return out


# ------------------------------------------------ precision sweep (config 3)
def run_precision(env):
    import numpy as np
    from paper_1612_03804_gb300.inputs import batch_uniform
    torch, sldqmc, args = env.torch, env.sldqmc, env.args
    L, beta, dtau, mu = 32, 10.0, 0.05, -0.5
    M = int(round(beta / dtau))
    nf = args.precision_fields
    fields = torch.from_numpy(batch_uniform(1003, nf, M, L * L)).cuda()
    uniform = torch.ones((1, M, L * L), dtype=torch.int8, device="cuda")
    cf = closed_form_logdet(L, beta, 1.0, mu - 1.0)
    out = []
    for nw in (5, 10, 20):
        res = {}
        for prec in ("fp64", "3xtf32", "bf16x3", "bf16"):
            wl = dict(CH16, L=L, beta=beta, dtau=dtau, mu=mu)
            with make_ctx(sldqmc, wl, prec, nf, nw) as ctx:
                ld = torch.zeros(nf, dtype=torch.float64, device="cuda")
                ctx.weight_batch_dev(fields, -1, ld)
                ctx.sync()
                st = torch.cuda.current_stream()
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record(st)
                ctx.weight_batch_dev(fields, -1, ld)
                e1.record(st)
                ctx.sync()
                dt = e0.elapsed_time(e1) / 1e3
                G = torch.zeros((1, L * L, L * L), dtype=torch.float64, device="cuda")
                ctx.green_batch_dev(fields[:1], -1, 0, G)
                lu = torch.zeros(1, dtype=torch.float64, device="cuda")
                ctx.weight_batch_dev(uniform, -1, lu)
                ctx.sync()
                res[prec] = (ld.cpu().numpy(), G.cpu().numpy()[0], float(lu.item()), dt)
        ref_ld, ref_G = res["fp64"][0], res["fp64"][1]
        for prec in ("fp64", "3xtf32", "bf16x3", "bf16"):
            ld, G, lu, dt = res[prec]
            out.append({"n_wrap": nw, "prec": prec,
                        "logdet_rel_err_max": float(np.max(np.abs(ld - ref_ld) / np.abs(ref_ld))),
                        "logdet_abs_err_max": float(np.max(np.abs(ld - ref_ld))),
                        "max_abs_dG": float(np.max(np.abs(G - ref_G))),
                        "closed_form_rel_err": abs(lu - cf) / abs(cf),
                        "weights_per_s": nf / dt})
    return {"workload": f"32x32, beta=10, dtau=0.05 (M=200), mu=-0.5, {nf} seeded random fields; errors against "
                        "the FP64-product GPU path at the same n_wrap (parity-checked against the oracle at "
                        "smaller sizes) and the uniform-field closed form", "rows": out}


# ------------------------------------------------------- 4x4 DQMC (config 1)
def run_local4(env):
    from paper_1612_03804_gb300.inputs import uniform_field
    torch, sldqmc = env.torch, env.sldqmc
    wl = dict(CH16, L=4, mu=0.0, beta=2.0, dtau=0.1)
    n_sw = 1000
    with make_ctx(sldqmc, wl, "fp64", 1, 10) as ctx:
        s = torch.from_numpy(uniform_field(1001, ctx.M, ctx.N)[None]).cuda()
        ld = torch.zeros(1, dtype=torch.float64, device="cuda")
        ctx.weight_batch_dev(s, -1, ld)
        ctx.sync()
        st = torch.cuda.current_stream()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(st)
        for _ in range(100):
            ctx.weight_batch_dev(s, -1, ld)
        e1.record(st)
        ctx.sync()
        us_w = e0.elapsed_time(e1) * 10.0
        ctx.local_sweep_batch_dev(s, 17, 0, 5, want_stats=False)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        stats = ctx.local_sweep_batch_dev(s, 17, 5, n_sw)
        torch.cuda.synchronize()
        dt = time.perf_counter() - t0
    # the same configuration for 1024 independent chains (one launch serves them all)
    from paper_1612_03804_gb300.inputs import batch_uniform
    Bb = 1024
    with make_ctx(sldqmc, wl, "fp64", Bb, 10) as ctx:
        sb = torch.from_numpy(batch_uniform(1002, Bb, ctx.M, ctx.N)).cuda()
        ctx.local_sweep_batch_dev(sb, 18, 0, 2, want_stats=False)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        ctx.local_sweep_batch_dev(sb, 18, 2, 50, want_stats=False)
        torch.cuda.synchronize()
        batched = Bb * 50 / (time.perf_counter() - t0)
    cpu = None
    if env.rank == 0 and not env.args.skip_cpu:
        # the FP64 CPU oracle on one host core: one weight and a few local sweeps
        from oracle import oracle as O
        m = O.Model(4, 4, t=1.0, mu=0.0, xi=1.0, beta=2.0, dtau=0.1, n_wrap=10)
        s0 = uniform_field(1001, m.M, m.N)
        t0 = time.perf_counter()
        for _ in range(20):
            O.weight(m, s0, -1)
        tw = (time.perf_counter() - t0) / 20
        t0 = time.perf_counter()
        O.local_sweep(m, s0, 17, 0, 20)
        ts = (time.perf_counter() - t0) / 20
        cpu = {"us_per_weight": 1e6 * tw, "us_per_sweep": 1e6 * ts, "cores": 1, "kind": "oracle",
               "sample": "20 weights and 20 local sweeps of this configuration, one host core"}
    return {"workload": "plain FP64 DQMC, 4x4, mu=0, beta=2, dtau=0.1 (M=20), n_wrap=10, one chain",
            "us_per_weight": us_w, "us_per_sweep": 1e6 * dt / n_sw, "sweeps": n_sw,
            "accept_rate": stats[0]["accepted"] / max(stats[0]["proposed"], 1),
            "max_drift": stats[0]["max_drift"], "batched_chains": Bb, "batched_sweeps_per_s": batched,
            "note": "one chain is launch-latency bound (about ten launches per slice and a stabilised "
                    "recomputation of G every n_wrap slices); chains batch into the same launches",
            "cpu_baseline": cpu}


# ----------------------------------------- decorrelation at the critical point
def run_critical(env):
    """Decorrelation at the paper's finite-temperature critical point (beta=1,
    dtau=0.05, M=20, h=2.774, 16x16; fit on 8x8 as in the paper): acceptance and
    tau_int of |sum s| for 16 chains with 1, 10 and 100 effective-model sweeps
    per cumulative update."""
    import numpy as np
    from paper_1612_03804_gb300.analysis import tau_int
    from paper_1612_03804_gb300.inputs import batch_uniform
    torch, sldqmc, args = env.torch, env.sldqmc, env.args
    wl = dict(CH16, beta=1.0)
    J, E0, r2, _ = train_effective_model(torch, sldqmc, wl, args, 8100 + env.rank, n_wrap=20)
    B = min(args.tau_chains, args.batch)
    ctx = make_ctx(sldqmc, wl, args.prec, B, 20, J, E0)
    d_s = torch.from_numpy(batch_uniform(8200 + env.rank, B, ctx.M, ctx.N)).cuda()
    for k in range(args.eff_thermalize):
        ctx.eff_sweeps_batch_dev(d_s, 1, 82, k, -1)
    d_lw = torch.zeros(B, dtype=torch.float64, device="cuda")
    ctx.log_weight_batch_dev(d_s, d_lw)
    d_acc = torch.zeros(B, dtype=torch.int32, device="cuda")
    for w in range(args.warmup):
        ctx.cumulative_batch_dev(d_s, d_lw, 1, 83, w, 1, d_acc)
    s0, lw0 = d_s.clone(), d_lw.clone()
    scan = []
    steps = args.critical_steps
    for n_eff in (1, 10, 100):
        d_s.copy_(s0)
        d_lw.copy_(lw0)
        d_acc.zero_()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        series = magnetisation_series(torch, ctx, d_s, d_lw, d_acc, 83 + n_eff, 100, steps, n_eff).astype(np.float64)
        dt = time.perf_counter() - t0
        tau, window = tau_int(series)
        scan.append({"n_eff": n_eff, "accept_rate": float(d_acc.sum().item()) / (B * steps),
                     "tau_int": tau, "tau_window": window, "steps_per_s": steps / dt,
                     "decorrelated_samples_per_s": B * steps / dt / tau,
                     "note": ("window reached" if window < steps - 1 else
                              "window not reached: tau_int is a lower bound")})
    ctx.close()
    return {"point": "16x16, beta=1, dtau=0.05 (M=20), h=2.774, mu=-0.5 (the paper's critical point), "
                     f"{B} chains, effective model fitted on 8x8 (R^2={r2:.6f})", "steps": steps, "n_eff_scan": scan}


# ------------------------- the paper's 16-coupling model and its range scans
def run_effmodel16(env):
    """"Results" of the paper at its critical point (beta=1, dtau=0.05, M=20,
    h=2.774): the 1 - R^2 curves of the temporal range (space fixed at
    nearest neighbours) and of the spatial range (time fixed at 10), the fit
    of the 16-coupling model on 8x8 local-DQMC configurations, and tau_int of
    |sum s| for local DQMC sweeps against cumulative updates with that model
    transferred to L = 8, 12, 16, 24."""
    import numpy as np
    from paper_1612_03804_gb300 import effmodel as EM
    from paper_1612_03804_gb300.analysis import tau_int
    from paper_1612_03804_gb300.inputs import batch_uniform
    torch, sldqmc, args = env.torch, env.sldqmc, env.args
    wl = dict(CH16, beta=1.0)
    Bt = args.train_chains
    t0 = time.perf_counter()
    c8 = make_ctx(sldqmc, wl, "fp64", Bt, 20, bare_couplings(wl))
    s = torch.from_numpy(batch_uniform(8300 + env.rank, Bt, c8.M, c8.N)).cuda()
    for k in range(args.bare_sweeps):
        c8.eff_sweeps_batch_dev(s, 1, 84, k, -1)
    c8.local_sweep_batch_dev(s, 84, 0, args.thermalize, want_stats=False)
    cfgs, sw = [], args.thermalize
    while len(cfgs) * Bt < args.train_configs:
        c8.local_sweep_batch_dev(s, 84, sw, 1, want_stats=False)
        sw += 1
        cfgs.append(s.cpu().numpy().copy())
    cfgs = np.concatenate(cfgs)[: args.train_configs]
    d_c = torch.from_numpy(cfgs).cuda()
    lw = torch.zeros(len(cfgs), dtype=torch.float64, device="cuda")
    for k in range(0, len(cfgs), Bt):
        c8.log_weight_batch_dev(d_c[k:k + Bt], lw[k:k + Bt])
    c8.sync()
    logw = lw.cpu().numpy()

    def fit(classes):
        c8.set_effective_model(classes, np.zeros(len(classes)))
        return c8.fit_effective_action(cfgs, logw)

    temporal = [{"range": k, "one_minus_r2": 1.0 - fit(cls)[2]} for k, cls in EM.temporal_range_scan(10)]
    spatial = [{"shells": sh, "one_minus_r2": 1.0 - fit(cls)[2]} for sh, cls in EM.spatial_range_scan(5)]
    cls16 = EM.paper_classes()
    J16, E016, r2_16 = fit(cls16)
    c8.close()
    t_fit = time.perf_counter() - t0

    taus = []
    B = args.tau_chains
    for L in args.effmodel_sizes:
        wlL = dict(wl, L=L)
        row = {"L": L}
        # local DQMC sweeps
        cl = make_ctx(sldqmc, wlL, "fp64", B, 20)
        if L >= 16:
            cl.set_local_update_rank(32)
        sl = torch.from_numpy(batch_uniform(8400 + L, B, cl.M, cl.N)).cuda()
        cl.set_effective_model(cls16, J16, E016)
        for k in range(100):
            cl.eff_sweeps_batch_dev(sl, 1, 85, k, -1)
        cl.local_sweep_batch_dev(sl, 85, 0, 5, want_stats=False)
        # local sweeps cost O(N^2) per accepted flip: the largest lattice gets a shorter series
        S = args.effmodel_steps if L <= 16 else max(50, args.effmodel_steps // 3)
        out = torch.zeros((S, B), dtype=torch.float32, device="cuda")
        torch.cuda.synchronize()
        ta = time.perf_counter()
        for k in range(S):
            cl.local_sweep_batch_dev(sl, 85, 5 + k, 1, want_stats=False)
            out[k] = sl.float().sum(dim=(1, 2)).abs()
        torch.cuda.synchronize()
        dt = time.perf_counter() - ta
        tau, win = tau_int(out.cpu().numpy().astype(np.float64))
        row["local"] = {"tau_int_sweeps": tau, "window": win, "sweeps_per_s": S / dt,
                        "note": "window reached" if win < S - 1 else "window not reached: lower bound"}
        # cumulative updates with the 16-coupling model fitted on 8x8
        d_lw = torch.zeros(B, dtype=torch.float64, device="cuda")
        cl.log_weight_batch_dev(sl, d_lw)
        d_acc = torch.zeros(B, dtype=torch.int32, device="cuda")
        torch.cuda.synchronize()
        ta = time.perf_counter()
        S = args.effmodel_steps
        ser = magnetisation_series(torch, cl, sl, d_lw, d_acc, 86, 0, S, args.effmodel_neff).astype(np.float64)
        dt = time.perf_counter() - ta
        tau, win = tau_int(ser)
        row["cumulative"] = {"n_eff": args.effmodel_neff, "tau_int_steps": tau, "window": win,
                             "steps_per_s": S / dt, "accept_rate": float(d_acc.sum().item()) / (B * S),
                             "note": "window reached" if win < S - 1 else "window not reached: lower bound"}
        cl.close()
        taus.append(row)
    return {"point": "beta=1, dtau=0.05 (M=20), h=2.774, mu=-0.5, xi=1 (the paper's critical point); fits on "
                     f"{len(cfgs)} local-DQMC configurations of 8x8",
            "temporal_range_scan": temporal, "spatial_range_scan": spatial,
            "model16": {"classes": EM.class_names(), "J": [float(x) for x in J16], "E0": E016, "r2": r2_16,
                        "one_minus_r2": 1.0 - r2_16},
            "fit_s": round(t_fit, 2), "tau_vs_L": taus, "chains": B, "series": args.effmodel_steps}


# ------------------------------------------- delayed (rank-k) local updates
def run_local_delayed(env):
    """Local DQMC sweeps (the step-i training path) with immediate rank-1
    Sherman-Morrison updates against delayed rank-32 updates, 16 chains at the
    paper's critical point (beta=1, dtau=0.05, M=20) on 16x16 and 24x24."""
    from paper_1612_03804_gb300.inputs import batch_uniform
    torch, sldqmc, args = env.torch, env.sldqmc, env.args
    rows = []
    B = args.tau_chains
    for L in (16, 24):
        wl = dict(CH16, L=L, beta=1.0)
        row = {"L": L, "chains": B}
        for k in (1, 32):
            ctx = make_ctx(sldqmc, wl, "fp64", B, 20)
            ctx.set_local_update_rank(k)
            d_s = torch.from_numpy(batch_uniform(8500 + L, B, ctx.M, ctx.N)).cuda()
            ctx.local_sweep_batch_dev(d_s, 87, 0, 1, want_stats=False)
            torch.cuda.synchronize()
            n_sw = 3
            st = torch.cuda.current_stream()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(st)
            ctx.local_sweep_batch_dev(d_s, 87, 1, n_sw, want_stats=False)
            e1.record(st)
            e1.synchronize()
            dt = e0.elapsed_time(e1) / 1e3
            row[f"rank{k}_sweeps_per_s"] = n_sw / dt
            ctx.close()
        row["speedup"] = row["rank32_sweeps_per_s"] / row["rank1_sweeps_per_s"]
        rows.append(row)
    return {"workload": "local DQMC sweeps, beta=1, dtau=0.05 (M=20), n_wrap=20, mu=-0.5, xi=1, FP64",
            "rows": rows}


def run_ours(args):
    env = Env(args)
    chosen = ALL_WORKLOADS if args.workloads == "all" else tuple(w for w in args.workloads.split(",") if w)
    head = run_large(env) if "large" in chosen else None
    wls = {}
    if "chains16" in chosen:
        wls["chains16"] = run_chains16(env)
    if "uneven" in chosen:
        full = None
        if "chains16" in wls:
            c = wls["chains16"]
            nw = c["n_wrap"][args.prec]
            full = c["chains"] / env.world * 2 * weight_work(256, 160, nw) / (c["ms_per_step"] * 1e-3)
        wls["uneven"] = run_uneven(env, full)
    if "precision" in chosen:
        wls["precision"] = run_precision(env)
    if "local4" in chosen:
        wls["local4"] = run_local4(env)
    if "critical" in chosen and not args.no_train:
        wls["critical"] = run_critical(env)
    if "effmodel16" in chosen:
        wls["effmodel16"] = run_effmodel16(env)
    if "local_delayed" in chosen:
        wls["local_delayed"] = run_local_delayed(env)
    if env.rank == 0:
        if head is None:
            # a partial run (no headline workload): the first workload's numbers head the line
            first = next(iter(wls.values()))
            head = {"metric": METRIC, "value": first.get("value"), "unit": UNIT, "n_gpus": env.world,
                    "steps": args.steps, "warmup": args.warmup, "ms_per_step": first.get("ms_per_step"),
                    "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": args.prec,
                    "data": "synthetic", "config": {"workload": first.get("workload")},
                    "partial": "headline workload not run"}
        head["workloads"] = wls
        print(json.dumps(head), flush=True)
    if env.dist:
        env.dist.barrier()
        env.dist.destroy_process_group()


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workloads", default="all", help="comma-separated subset of " + ",".join(ALL_WORKLOADS))
    ap.add_argument("--batch", type=int, default=128)
    ap.add_argument("--prec", default="3xtf32", choices=["3xtf32", "bf16x3", "bf16", "fp64"])
    ap.add_argument("--train-configs", type=int, default=2000)
    ap.add_argument("--train-chains", type=int, default=64)
    ap.add_argument("--thermalize", type=int, default=20)
    ap.add_argument("--bare-sweeps", type=int, default=200)
    ap.add_argument("--eff-thermalize", type=int, default=300)
    ap.add_argument("--large-eff-thermalize", type=int, default=100)
    ap.add_argument("--large-tile", type=int, default=64, choices=[64, 128],
                    help="tensor-core tile width of the headline workload's slice products")
    ap.add_argument("--large-L", type=int, default=LARGE["L"],
                    help="lattice of the headline workload (profiling captures use a smaller one)")
    ap.add_argument("--tau-steps", type=int, default=1000)
    ap.add_argument("--tau-chains", type=int, default=16)
    ap.add_argument("--critical-steps", type=int, default=300)
    ap.add_argument("--precision-fields", type=int, default=4)
    ap.add_argument("--oracle-sample", type=int, default=2)
    ap.add_argument("--effmodel-sizes", type=lambda v: [int(x) for x in v.split(",")], default=[8, 12, 16, 24])
    ap.add_argument("--effmodel-steps", type=int, default=300)
    ap.add_argument("--effmodel-neff", type=int, default=10)
    ap.add_argument("--n-wrap", default="auto", help="stabilisation interval of chains16, or 'auto' for the autotuner")
    ap.add_argument("--skip-fp64", action="store_true")
    ap.add_argument("--skip-separable", action="store_true")
    ap.add_argument("--no-train", action="store_true",
                    help="use the bare Ising couplings as H_eff (no local-DQMC training; for profiling runs)")
    ap.add_argument("--skip-cpu", action="store_true")
    args = ap.parse_args()
    if args.warmup < 3:
        ap.error("--warmup must be >= 3")
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
