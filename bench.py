#!/usr/bin/env python
"""Benchmark of the cognitive-model hot path on GB300.

One step = one pass of the whole hot path over one batch of synthetic input:
  Stroop (4 x 1,000 trials), DDM (2^20 trials), LCA (262,144 trials at
  N = 4, 8, 16), predator-prey grid search (27,000 candidates x 64 trials)
  and the wide multitask network, launched together as one CUDA-graph batch
  (each job on its own branch, so their tails overlap).
value = trial-steps per second of that pass (a grid evaluation counts as one
trial-step). Also reported: the plain one-launch-per-job form on the same
GPU, the dominant kernel's roofline, an end-to-end number through the serving
API with host buffers, served-mix p50/p99 latency, and the CPU oracle.

python bench.py [--gpus N --steps K --warmup W] [--impl reference]
Multi-GPU: launched by torchrun, one process per GPU, weak scaling: rank r
runs the same pass on its own trials (global ids r*n .. r*n + n - 1, so its
noise differs) and its own predator-prey positions; no data-path collective.
"""
from __future__ import annotations

import argparse
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

import numpy as np  # noqa: E402

METRIC = "trial-steps/sec (hot-path pass: DDM, LCA, Stroop, wide Stroop, grid search)"
UNIT = "trial-steps/s"
WORKLOAD = ("hot-path pass: Stroop 4x1000 (weights seed 0) + DDM 2^20 + LCA 262144 x N{4,8,16} "
            "+ predator-prey grid 27000 cand x 64 trials + wide Stroop 16384 (16+16 -> 256 -> 16)")
# Algorithmic FP32/INT32 lane-operations per unit of each kernel (the count a
# minimal implementation of the same arithmetic needs; the kernels' own
# instruction counts are higher):
#   normal (a quarter Philox4x32-10 block: 10 rounds x 4 ops / 4 = 10; one
#   uniform and half a Box-Muller pair: 9)                          19
#   DDM trial-step: normal + fixed-point update, bound test         32
#   LCA unit-step: normal + drive, update, rectify, sum and max     31
#   logistic unit-step: normal + integrate (3) + logistic (4)       26
#   Stroop trial-step: 6 logistic units, 24 edges, stop test        200
#   wide trial-step: 272 logistic units (26 each) + the 16-way stop
#     test (60); the 256 x 16 response GEMM runs on tensor cores and
#     the kernel's own precision device (bf16 hi/lo activations) is not
#     counted                                                      7,132
#   grid evaluation: 6 normals, 3 normalisations, distance, FP64 add   120
DDM_OPS_PER_TRIAL_STEP = 32
OPS_PER_UNIT = {"ddm": 32, "lca4": 4 * 31, "lca8": 8 * 31, "lca16": 16 * 31, "stroop": 200,
                "wide": 7132, "grid": 120}
# DRAM bytes (read + write) of one ddm_batched launch over the 2^20-trial job,
# from `ncu --set full --clock-control none -k regex:ddm_batched -s 1 -c 1
# python bench.py --only ddm` on the current kernel: 12,602,624 read + 512 written
# (the 5 MB of outputs stay in L2 within the launch). Algorithmic: 8 B of
# parameters in and 5 B out per trial = 13.6 MB.
DDM_TRAFFIC_BYTES = 12_603_136
# DRAM bytes of one wide_block_kernel launch over the 16,384-trial job, from
# `ncu --set full --clock-control none -k regex:wide_block -s 1 -c 1 python bench.py --only wide`
# on the current kernel: 314,112 read (9,816 sectors) + 0 written (the outputs stay in
# L2 within the launch). Algorithmic: the weights (16 KB BF16 operand image, 32 KB hidden
# weights), the 256 condition rows and 5 B of outputs per trial: 0.16 MB; the reads are
# about twice that, a few hundred KB against a 3 ms ALU-bound launch.
WIDE_TRAFFIC_BYTES = 314_112
TRAFFIC_BYTES = {"ddm": DDM_TRAFFIC_BYTES, "wide": WIDE_TRAFFIC_BYTES}
LANES_PER_SM = 128
PEAK_OPS = [40.27e12]   # SMs x lanes x max SM clock, set from the device in main()
# Order in which the pass's graph branches are created (and served jobs
# submitted). The LCA jobs go first: their longest trials end in a
# latency-bound tail on a few SMs, which then runs beside the later jobs
# instead of after them (8.21-8.23 ms per pass against 8.34-8.37 ms with the
# wide network first, two runs each; job order was 2-4 % slower still).
JOB_ORDER = ("lca4", "lca8", "lca16", "ddm", "wide", "grid", "stroop")


def in_job_order(jobs):
    rank = {n: i for i, n in enumerate(JOB_ORDER)}
    return sorted(jobs, key=lambda j: rank.get(j["name"], len(rank)))
WIDE_TRIALS = 16384


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-serving", action="store_true")
    ap.add_argument("--no-extensions", action="store_true",
                    help="skip the episode / coarse-to-fine / tie-break measurements")
    ap.add_argument("--profile-once", action="store_true",
                    help="run warmup + 1 step only (for ncu launch lists)")
    ap.add_argument("--only", default=None,
                    choices=["ddm", "lca4", "lca8", "lca16", "grid", "stroop", "wide", "refine",
                             "episodes", "grid_batch", "small_jobs", "extended"],
                    help="one job of this kind, default launch shape, 1 warm + 1 timed launch "
                         "(the small case for per-kernel ncu captures)")
    ap.add_argument("--n", type=int, default=0, help="trials (or candidates) for --only")
    ap.add_argument("--hidden", type=int, default=256,
                    help="hidden units of the wide network for --only wide (64, 128, 192, 256)")
    return ap.parse_args()


def dist_env():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, local, world


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f), "measured"
    except OSError:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "sm_max_mhz": 2070.0}, "fallback"


# ------------------------------------------------------------------ step ---

class Step:
    """Device inputs/outputs and models of one hot-path pass (this rank's shard)."""

    def __init__(self, B, W, torch, ctx, rank, world):
        def shard_range(n, rank, world):
            # weak scaling: every rank takes a full job of its own trials
            return rank * n, rank * n + n
        self.B, self.torch = B, torch
        cuda = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()  # noqa: E731
        self.jobs = []      # (name, kind, model, desc, outputs)
        self.inputs_bytes = 0

        def out_run(n, state=0):
            return dict(choice=torch.zeros(max(n, 1), dtype=torch.int8, device="cuda"),
                        step=torch.zeros(max(n, 1), dtype=torch.int32, device="cuda"))

        # Stroop small
        s = W.stroop_small()
        lo, hi = shard_range(s["n_trials"], rank, world)
        m = B.compose_network(ctx, s["layers"], s["projections"], rate=s["rate"],
                              noise_sd=s["noise_sd"], stop_layer=s["stop_layer"],
                              stop_threshold=s["stop_threshold"], max_steps=s["max_steps"])
        cond = cuda(s["cond_inputs"])
        d = B.run_desc(hi - lo, s["seed"], cond_inputs=cond, n_cond=4, cond_block=s["cond_block"],
                       trial_offset=lo)
        self.jobs.append(dict(name="stroop", model=m, desc=d, out=out_run(hi - lo), keep=[cond],
                              host_in=[s["cond_inputs"]], n=hi - lo))
        # DDM
        w = W.ddm()
        n = w["A"].shape[0]
        lo, hi = shard_range(n, rank, world)
        m = B.compose_ddm(ctx, dt=w["dt"], sigma=w["sigma"], max_steps=w["max_steps"])
        hp = np.concatenate([w["A"], w["z"]])
        p = cuda(hp)
        d = B.run_desc(hi - lo, w["seed"], trial_params=p, trial_offset=lo)
        self.jobs.append(dict(name="ddm", model=m, desc=d, out=out_run(hi - lo), keep=[p],
                              host_in=[hp], n=hi - lo))
        # LCA
        for N in (4, 8, 16):
            l = W.lca(N=N)
            n = l["I"].shape[0]
            lo, hi = shard_range(n, rank, world)
            m = B.compose_lca(ctx, N, leak=l["leak"], inhibition=l["inhibition"], sigma=l["sigma"],
                              dt=l["dt"], threshold=l["threshold"], max_steps=l["max_steps"])
            hp = l["I"]
            p = cuda(hp)
            d = B.run_desc(hi - lo, l["seed"], trial_params=p, trial_offset=lo)
            self.jobs.append(dict(name=f"lca{N}", model=m, desc=d, out=out_run(hi - lo), keep=[p],
                                  host_in=[hp], n=hi - lo))
        # wide Stroop (tensor cores); skipped when this build has no wide kernel
        wd = W.stroop_wide(n_trials=WIDE_TRIALS)
        try:
            m = B.compose_network(ctx, wd["layers"], wd["projections"], rate=wd["rate"],
                                  noise_sd=wd["noise_sd"], stop_layer=wd["stop_layer"],
                                  stop_threshold=wd["stop_threshold"], max_steps=wd["max_steps"],
                                  bf16_edges=(2,))
            lo, hi = shard_range(WIDE_TRIALS, rank, world)
            cond = cuda(wd["cond_inputs"])
            d = B.run_desc(hi - lo, wd["seed"], cond_inputs=cond, n_cond=cond.shape[0],
                           cond_block=1, trial_offset=lo)
            probe = out_run(1)
            B.dg_run(m, B.run_desc(1, wd["seed"], cond_inputs=cond, n_cond=cond.shape[0],
                                   cond_block=1), probe["choice"], probe["step"])
            self.jobs.append(dict(name="wide", model=m, desc=d, out=out_run(hi - lo), keep=[cond],
                                  host_in=[wd["cond_inputs"]], n=hi - lo))
        except B.DGError:
            self.wide_missing = True
        # predator-prey grid
        g = W.predator_prey(pos_seed=3 + rank)
        lo, hi = 0, 30 * 30 * 30
        m = B.compose_predator_prey(ctx, obs_offset=g["obs_offset"], pred_weight=g["pred_weight"])
        lv = [cuda(x) for x in g["levels"]]
        pos = cuda(g["pos"])
        d = B.grid_desc(lv, pos, g["seed"])
        res = torch.zeros(3, dtype=torch.float64, device="cuda")
        self.jobs.append(dict(name="grid", model=m, desc=d, grid=True,
                              out=dict(result=res), keep=lv + [pos],
                              host_in=[g["pos"]] + g["levels"], n=hi - lo,
                              evals=(hi - lo) * g["pos"].shape[0]))
        self.batch = None

    def run_plain(self):
        B = self.B
        for j in self.jobs:
            if j.get("grid"):
                d = j["desc"]
                d.mode = B.DG_MODE_PLAIN
                B.dg_grid_search(j["model"], d, j["out"]["result"])
                d.mode = B.DG_MODE_BATCHED
            else:
                d = j["desc"]
                d.mode = B.DG_MODE_PLAIN
                B.dg_run(j["model"], d, j["out"]["choice"], j["out"]["step"])
                d.mode = B.DG_MODE_BATCHED

    def launch(self, ctx):
        B = self.B
        if self.batch is None:
            self.batch = B.dg_batch_create(ctx)
            for j in in_job_order(self.jobs):
                if j.get("grid"):
                    B.dg_batch_add_grid(self.batch, j["model"], j["desc"], j["out"]["result"])
                else:
                    B.dg_batch_add_run(self.batch, j["model"], j["desc"], j["out"]["choice"],
                                       j["out"]["step"])
        B.dg_batch_launch(self.batch)

    def trial_steps(self):
        """Per-job trial-steps of the pass (from the step outputs)."""
        self.torch.cuda.synchronize()
        ts = {}
        for j in self.jobs:
            if j.get("grid"):
                ts[j["name"]] = j["evals"]
            else:
                ts[j["name"]] = int(j["out"]["step"][:j["n"]].to(self.torch.int64).sum().item())
        return ts

    def kernels_per_step(self):
        """Kernels of one pass: the kernel nodes of the batch's CUDA graph, as
        the library counts them (one per job, plus the three-kernel trial-order
        sort wherever the launch-shape tuner chose the sorted hand-out)."""
        return self.B.dg_batch_kernels(self.batch)


# ---------------------------------------------------------------- clocks ---

class ClockSampler:
    def __init__(self, device):
        self.device = device
        self.proc = None
        self.out = None

    def __enter__(self):
        q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--query-gpu={q}", "--format=csv,noheader,nounits", "-lms", "100",
                 "-i", str(self.device)], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL,
                text=True)
        except OSError:
            self.proc = None
        return self

    def __exit__(self, *a):
        if self.proc is None:
            return
        time.sleep(0.25)
        self.proc.terminate()
        try:
            self.out, _ = self.proc.communicate(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
            self.out, _ = self.proc.communicate()

    def summary(self):
        if not self.out:
            return None
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in self.out.strip().splitlines():
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx.append(float(f[2]))
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "samples": len(sm),
                "reasons": sorted(reasons)}


class NvmlClockSampler:
    """SM clock and clock-event reasons read through NVML every 5 ms, strictly
    inside the timed region (a thread polls between __enter__ and __exit__).
    Falls back to the nvidia-smi sampler when NVML cannot be loaded."""

    REASONS = {0x4: "sw_power_cap", 0x8: "hw_slowdown", 0x20: "sw_thermal_slowdown",
               0x40: "hw_thermal_slowdown", 0x80: "hw_power_brake_slowdown"}

    def __init__(self, device, period_s=0.005):
        self.device, self.period = device, period_s
        self.samples, self.max_mhz = [], None
        self.fallback = None
        self._stop = threading.Event()
        self._thread = None
        self._nvml = None
        self._handle = None

    def _open(self):
        import ctypes as C
        lib = C.CDLL("libnvidia-ml.so.1")
        if lib.nvmlInit_v2() != 0:
            raise OSError("nvmlInit failed")
        h = C.c_void_p()
        bus = self._pci_bus_id()
        # NVML numbers all GPUs of the machine; the CUDA device is found by its PCI address
        if bus is None or lib.nvmlDeviceGetHandleByPciBusId_v2(bus, C.byref(h)) != 0:
            if lib.nvmlDeviceGetHandleByIndex_v2(C.c_uint(self.device), C.byref(h)) != 0:
                raise OSError("no NVML handle")
        self._nvml, self._handle = lib, h
        mx = C.c_uint()
        if lib.nvmlDeviceGetMaxClockInfo(h, C.c_int(1), C.byref(mx)) == 0:   # NVML_CLOCK_SM
            self.max_mhz = float(mx.value)
        fn = getattr(lib, "nvmlDeviceGetCurrentClocksEventReasons", None)
        self._reasons_fn = fn or lib.nvmlDeviceGetCurrentClocksThrottleReasons

    def _pci_bus_id(self):
        try:
            import torch
            p = torch.cuda.get_device_properties(self.device)
            return b"%08x:%02x:%02x.0" % (p.pci_domain_id, p.pci_bus_id, p.pci_device_id)
        except (AttributeError, RuntimeError, ImportError):
            return None

    def _poll(self):
        import ctypes as C
        clk, rs = C.c_uint(), C.c_ulonglong()
        while not self._stop.is_set():
            if self._nvml.nvmlDeviceGetClockInfo(self._handle, C.c_int(1), C.byref(clk)) == 0:
                r = rs.value if self._reasons_fn(self._handle, C.byref(rs)) == 0 else 0
                self.samples.append((float(clk.value), int(r)))
            time.sleep(self.period)

    def __enter__(self):
        try:
            self._open()
        except (OSError, AttributeError):
            self.fallback = ClockSampler(self.device).__enter__()
            return self
        self._thread = threading.Thread(target=self._poll, daemon=True)
        self._thread.start()
        return self

    def __exit__(self, *a):
        if self.fallback is not None:
            self.fallback.__exit__(*a)
            return
        self._stop.set()
        self._thread.join(timeout=1.0)

    def summary(self):
        if self.fallback is not None:
            return self.fallback.summary()
        if not self.samples:
            return None
        reasons = set()
        for _, r in self.samples:
            for bit, name in self.REASONS.items():
                if r & bit:
                    reasons.add(name)
        return {"sm_mhz": statistics.median(c for c, _ in self.samples),
                "sm_max_mhz": self.max_mhz, "samples": len(self.samples),
                "reasons": sorted(reasons), "source": "NVML every 5 ms inside the timed region"}


# ----------------------------------------------------------- CPU oracle ---

def cpu_baseline(threads=None, every=1):
    """The oracle as it stands, on this host's cores, over a bounded sample of
    the same pass: every `every`-th trial (or candidate) of each job, and every
    2*`every`-th trial of the wide job. Returns (value, threads, sample)."""
    import oracle
    from paper_2110_15425_gb300 import workloads as W
    threads = threads or (os.cpu_count() or 1)
    wide_every = 2 * every
    t0 = time.perf_counter()
    steps = 0
    s = W.stroop_small()
    ids = np.arange(0, s["n_trials"], every, dtype=np.uint32)
    o = oracle.transfer_run(s["layers"], s["projections"], s["cond_inputs"], s["cond_block"],
                            s["seed"], trial_ids=ids, threads=threads)
    steps += int(o["step"].sum())
    w = W.ddm()
    ids = np.arange(0, w["A"].shape[0], every, dtype=np.uint32)
    o = oracle.ddm_run(w["A"], w["z"], w["seed"], trial_ids=ids, threads=threads)
    steps += int(o["step"].sum())
    for N in (4, 8, 16):
        l = W.lca(N=N)
        ids = np.arange(0, l["I"].shape[0], every, dtype=np.uint32)
        o = oracle.lca_run(l["I"], l["seed"], trial_ids=ids, threads=threads)
        steps += int(o["step"].sum())
    wd = W.stroop_wide(n_trials=WIDE_TRIALS)
    ids = np.arange(0, WIDE_TRIALS, wide_every, dtype=np.uint32)
    o = oracle.transfer_run(wd["layers"], wd["projections"], wd["cond_inputs"], 1, wd["seed"],
                            trial_ids=ids, threads=threads)
    steps += int(o["step"].sum())
    g = W.predator_prey()
    ids = np.arange(0, 27000, every, dtype=np.uint32)
    oracle.pp_means(g["pos"], g["levels"], g["seed"], cand_ids=ids, threads=threads)
    steps += ids.shape[0] * g["pos"].shape[0]
    dt = time.perf_counter() - t0
    sample = (f"every {every} trial(s) or candidate(s) of the Stroop, DDM, LCA and grid jobs and "
              f"every {wide_every} trials of the wide job on {threads} thread(s): {steps} "
              f"trial-steps in {dt:.1f} s")
    return steps / dt, threads, sample


def cpu_baselines():
    """All-core and single-thread rates of the oracle (the single-thread one
    over a 16 times sparser sample, so that both take seconds)."""
    v, cores, sample = cpu_baseline()
    v1, _, sample1 = cpu_baseline(threads=1, every=16)
    return {"value": v, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": sample,
            "single_thread": {"value": v1, "unit": UNIT, "cores": 1, "sample": sample1}}


# ------------------------------------------------------------- reference ---

# Each reference step runs the oracle on every REF_EVERY-th trial of every job,
# so that the default --steps/--warmup run ends within a few minutes.
REF_EVERY = 4


def run_reference(args):
    rank, local, world = dist_env()
    if rank != 0:
        return
    for _ in range(args.warmup):
        cpu_baseline(every=REF_EVERY)
    vals = []
    sample = cores = None
    t0 = time.perf_counter()
    for _ in range(max(1, args.steps)):
        v, cores, sample = cpu_baseline(every=REF_EVERY)
        vals.append(v)
    wall = time.perf_counter() - t0
    value = statistics.mean(vals)
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT,
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1000.0 * wall / max(1, args.steps), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": WORKLOAD, "sample": sample},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ------------------------------------------------------------------ main ---

def run_only(args):
    """One job of one kind: the small case for single-kernel profiles."""
    os.environ["DG_AUTOTUNE"] = "0"
    import torch
    from paper_2110_15425_gb300 import binding as B
    from paper_2110_15425_gb300 import workloads as W
    ctx = B.dg_create(0)
    cuda = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()  # noqa: E731
    k = args.only
    if k == "small_jobs":   # the many-small-jobs serving measurement alone
        w, l8 = W.ddm(n_trials=1), W.lca(n_trials=1, N=8)
        st = W.stroop_small()
        models = [dict(name="stroop", model=B.compose_network(
                      ctx, st["layers"], st["projections"], rate=st["rate"],
                      noise_sd=st["noise_sd"], stop_layer=st["stop_layer"],
                      stop_threshold=st["stop_threshold"], max_steps=st["max_steps"])),
                  dict(name="ddm", model=B.compose_ddm(ctx, dt=w["dt"], sigma=w["sigma"],
                                                       max_steps=w["max_steps"])),
                  dict(name="lca8", model=B.compose_lca(
                      ctx, 8, leak=l8["leak"], inhibition=l8["inhibition"], sigma=l8["sigma"],
                      dt=l8["dt"], threshold=l8["threshold"], max_steps=l8["max_steps"]))]

        class _Models:
            jobs = models
        print(json.dumps(served_small_jobs(B, W, torch, ctx, _Models, n_jobs=args.n or SERVE_JOBS)))
        for j in models:
            B.dg_model_free(j["model"])
        B.dg_destroy(ctx)
        return
    if k == "grid":
        L = max(2, round(args.n ** (1 / 3))) if args.n else 30
        g = W.predator_prey(levels=L)
        m = B.compose_predator_prey(ctx)
        lv = [cuda(x) for x in g["levels"]]
        pos = cuda(g["pos"])
        res = torch.zeros(3, dtype=torch.float64, device="cuda")
        go = lambda: B.dg_grid_search(m, B.grid_desc(lv, pos, g["seed"]), res)  # noqa: E731
    elif k == "grid_batch":
        nb = args.n or 16   # searches of the 30^3 x 64 grid, each its own positions and seed
        bw = [W.predator_prey(pos_seed=3 + i, noise_seed=13 + i) for i in range(nb)]
        m = B.compose_predator_prey(ctx)
        bkeep = [([cuda(l) for l in w_["levels"]], cuda(w_["pos"])) for w_ in bw]
        bdesc = [B.grid_desc(lv_, pos_, w_["seed"]) for (lv_, pos_), w_ in zip(bkeep, bw)]
        res = torch.zeros(nb * 3, dtype=torch.float64, device="cuda")
        go = lambda: B.dg_grid_search_batch(m, bdesc, res)  # noqa: E731
    elif k == "episodes":
        w = W.predator_prey_episodes(n_episodes=args.n or 64)
        m = B.compose_predator_prey(ctx)
        E, T = w["start"].shape[0], w["max_steps"]
        d = B.episode_desc([cuda(x) for x in w["levels"]], cuda(w["start"]), w["n_trials"], T,
                           w["seed"], speed=w["speed"], radius=w["radius"])
        oc = torch.zeros(E, dtype=torch.int8, device="cuda")
        st = torch.zeros(E, dtype=torch.int32, device="cuda")
        o = B.episode_out(oc, st)
        go = lambda: B.dg_run_episodes(m, d, o)  # noqa: E731
    elif k == "refine":
        G, R = (args.n or 5), 7
        g = W.predator_prey()
        m = B.compose_predator_prey(ctx)
        pos = cuda(g["pos"])
        out = torch.zeros(64 * R, dtype=torch.uint8, device="cuda")
        d = B.refine_desc(pos, [0, 0, 0], [1, 1, 1], G, R, g["seed"])
        go = lambda: B.dg_grid_refine(m, d, out)  # noqa: E731
    else:
        if k == "ddm":
            w = W.ddm(n_trials=args.n or (1 << 20))
            m = B.compose_ddm(ctx)
            p = cuda(np.concatenate([w["A"], w["z"]]))
            d = B.run_desc(w["A"].shape[0], w["seed"], trial_params=p)
        elif k.startswith("lca"):
            w = W.lca(n_trials=args.n or 262144, N=int(k[3:]))
            m = B.compose_lca(ctx, w["N"])
            p = cuda(w["I"])
            d = B.run_desc(w["I"].shape[0], w["seed"], trial_params=p)
        elif k == "extended":
            w = W.extended_stroop()
            m = B.compose_extended_stroop(
                ctx, w["layers"], w["projections"],
                [dict(W=w["ddm_W"][q:q + 1], bias=w["ddm_bias"], dt=w["ddm_dt"],
                      sigma=w["ddm_sigma"], bound=w["ddm_bound"], max_steps=w["ddm_max"])
                 for q in range(2)],
                rate=w["rate"], noise_sd=w["noise_sd"], stop_layer=w["stop_layer"],
                stop_threshold=w["stop_threshold"], max_steps=w["max_steps"])
            p = cuda(w["cond_inputs"])
            d = B.run_desc(w["n_trials"], w["seed"], cond_inputs=p, n_cond=p.shape[0],
                           cond_block=w["cond_block"])
        else:
            w = (W.stroop_small() if k == "stroop" else
                 W.stroop_wide(n_trials=args.n or WIDE_TRIALS, hidden=args.hidden))
            m = B.compose_network(ctx, w["layers"], w["projections"], rate=w["rate"],
                                  noise_sd=w["noise_sd"], stop_layer=w["stop_layer"],
                                  stop_threshold=w["stop_threshold"], max_steps=w["max_steps"],
                                  bf16_edges=(2,) if k == "wide" else ())
            p = cuda(w["cond_inputs"])
            d = B.run_desc(w["n_trials"], w["seed"], cond_inputs=p, n_cond=p.shape[0],
                           cond_block=w["cond_block"])
        n = d.n_trials
        ch = torch.zeros(n, dtype=torch.int8, device="cuda")
        st = torch.zeros(n, dtype=torch.int32, device="cuda")
        go = lambda: B.dg_run(m, d, ch, st)  # noqa: E731
    go()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    go()
    e1.record()
    torch.cuda.synchronize()
    out = {"only": k, "n": args.n, "ms": e0.elapsed_time(e1)}
    if k not in ("grid", "refine", "episodes", "grid_batch"):
        out["trial_steps"] = int(st.to(torch.int64).sum().item())
    print(json.dumps(out))
    B.dg_model_free(m)
    B.dg_destroy(ctx)


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
        return
    if args.only:
        run_only(args)
        return
    rank, local, world = dist_env()
    import torch
    torch.cuda.set_device(local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    from paper_2110_15425_gb300 import binding as B
    from paper_2110_15425_gb300 import workloads as W
    try:
        B.lib()
    except RuntimeError:
        from paper_2110_15425_gb300 import build as BB
        BB.build()
    ctx = B.dg_create(local)
    step = Step(B, W, torch, ctx, rank, world)
    pk, pk_kind = peaks()
    sms = torch.cuda.get_device_properties(local).multi_processor_count

    def barrier():
        torch.cuda.synchronize()
        if world > 1:
            torch.distributed.barrier()

    # warm-up: the first launch tunes shapes and captures the graph
    for _ in range(max(3, args.warmup)):
        step.launch(ctx)
    ts = step.trial_steps()
    total_ts = sum(ts.values())
    l2_flush = torch.empty(512 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")

    K = 1 if args.profile_once else args.steps
    starts = [torch.cuda.Event(enable_timing=True) for _ in range(K)]
    ends = [torch.cuda.Event(enable_timing=True) for _ in range(K)]
    barrier()
    with NvmlClockSampler(local) as clk:
        for i in range(K):
            l2_flush.zero_()
            starts[i].record()
            step.launch(ctx)
            ends[i].record()
        barrier()
    step_ms = [s.elapsed_time(e) for s, e in zip(starts, ends)]
    ms = sum(step_ms) / K
    if world > 1:
        t = torch.tensor([ms, float(total_ts)], dtype=torch.float64, device="cuda")
        mx = t.clone()
        torch.distributed.all_reduce(mx[:1], op=torch.distributed.ReduceOp.MAX)
        torch.distributed.all_reduce(t[1:], op=torch.distributed.ReduceOp.SUM)
        ms, all_ts = float(mx[0]), float(t[1])
    else:
        all_ts = float(total_ts)
    if args.profile_once:
        if rank == 0:
            print(json.dumps({"profile_once": True, "ms": ms}))
        return
    value = all_ts / (ms / 1000.0)

    # plain form: one launch per job, no refill, no graph, one stream
    barrier()
    pe0, pe1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    step.run_plain()
    barrier()
    plain_ms = []
    for _ in range(3):
        l2_flush.zero_()
        pe0.record()
        step.run_plain()
        pe1.record()
        torch.cuda.synchronize()
        plain_ms.append(pe0.elapsed_time(pe1))
    plain_ms = statistics.mean(plain_ms)
    ts_plain = step.trial_steps()
    plain_same = ts_plain == ts
    # restore batched outputs for later checks
    step.launch(ctx)

    # per-job kernel times (each alone, batched form) and the dominant kernel
    per_job = {}
    ddm_ms = None
    for j in step.jobs:
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        times = []
        for _ in range(3):
            l2_flush.zero_()
            e0.record()
            if j.get("grid"):
                B.dg_grid_search(j["model"], j["desc"], j["out"]["result"])
            else:
                B.dg_run(j["model"], j["desc"], j["out"]["choice"], j["out"]["step"])
            e1.record()
            torch.cuda.synchronize()
            times.append(e0.elapsed_time(e1))
        t_ms = statistics.mean(times)
        per_job[j["name"]] = {"ms": round(t_ms, 4), "trial_steps": ts[j["name"]],
                              "trial_steps_per_s": ts[j["name"]] / (t_ms / 1000.0)}
        if j["name"] == "grid":
            per_job["grid"]["candidates_per_s"] = j["n"] / (t_ms / 1000.0)
        if j["name"] == "ddm":
            ddm_ms = t_ms
    dominant = max(per_job, key=lambda k: per_job[k]["ms"])
    sm_max = pk.get("sm_max_mhz", 2070.0)
    peak_ops = sms * LANES_PER_SM * sm_max * 1e6
    PEAK_OPS[0] = peak_ops
    peak_src = (f"{sms} SMs x {LANES_PER_SM} FP32/INT32 lanes x {sm_max:.0f} MHz "
                f"({pk_kind} max SM clock)")
    by_kernel = {}
    for name, job in per_job.items():
        ach = ts[name] * OPS_PER_UNIT[name] / (job["ms"] / 1000.0)
        by_kernel[name] = {"achieved": ach / 1e12, "frac": ach / peak_ops,
                           "ops_per_unit": OPS_PER_UNIT[name]}
    kernel_names = {"ddm": "ddm_batched", "wide": "wide_block_kernel<256> (tensor cores)",
                    "lca4": "lca_batched<4,*>", "lca8": "lca_batched<8,*>",
                    "lca16": "lca_batched<16,*>", "stroop": "net_group<8>",
                    "grid": "grid_batched"}
    # the dominant kernel of the pass (the longest job); DRAM traffic is known
    # for the DDM kernel from the ncu capture named above
    roofline = {"bound": "alu", "kernel": kernel_names[dominant],
                "achieved": by_kernel[dominant]["achieved"], "peak": peak_ops / 1e12,
                "unit": "Tlane-op/s", "frac": by_kernel[dominant]["frac"],
                "traffic": TRAFFIC_BYTES.get(dominant),
                "peak_source": peak_src, "ops_per_unit": OPS_PER_UNIT[dominant],
                "by_kernel": by_kernel,
                "ddm": {"kernel": "ddm_batched", "frac": by_kernel["ddm"]["frac"],
                        "traffic": DDM_TRAFFIC_BYTES, "traffic_unit": "bytes per launch"}}

    # end to end through the serving API with pinned host buffers
    e2e = None
    serving = None
    if not args.no_serving:
        e2e = e2e_serving(B, torch, ctx, step, all_ts, world, rank)
        if world == 1:
            serving = served_mix(B, W, torch, ctx, step)
            serving["small_jobs"] = served_small_jobs(B, W, torch, ctx, step)

    gpu_launches = step.kernels_per_step() * K
    clocks = clk.summary()
    ext = None
    if rank == 0 and world == 1 and not args.no_extensions:
        ext = extensions(B, W, torch, ctx, per_job["grid"]["ms"])
    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cpu = cpu_baselines()
    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": K,
            "warmup": max(3, args.warmup), "ms_per_step": ms, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": WORKLOAD, "l2": "flushed between timed steps (512 MB write)",
                       "parallelism": f"dp{world} (independent passes)" if world > 1 else "1 GPU",
                       "wide_member": "missing" if getattr(step, "wide_missing", False) else "on"},
            "plain_form": {"ms_per_step": plain_ms, "value": all_ts / (plain_ms / 1000.0),
                           "speedup_batched_vs_plain": plain_ms / ms,
                           "same_trial_steps_as_batched": plain_same},
            "per_job": per_job,
            "grid_candidates_per_s": per_job["grid"]["candidates_per_s"],
            "roofline": roofline, "e2e": e2e, "serving": serving, "gpu_launches": gpu_launches,
            "clocks": clocks, "cpu_baseline": cpu, "extensions": ext,
        }
        print(json.dumps(line), flush=True)
    for j in step.jobs:
        B.dg_model_free(j["model"])
    B.dg_destroy(ctx)
    if world > 1:
        torch.distributed.destroy_process_group()


def _time_ms(torch, fn, reps=3, stream=None):
    """Mean CUDA-event time of fn() on `stream` (torch's current stream if None)."""
    s = stream or torch.cuda.current_stream()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    out = []
    for _ in range(reps):
        torch.cuda.synchronize()
        e0.record(s)
        fn()
        e1.record(s)
        torch.cuda.synchronize()
        out.append(e0.elapsed_time(e1))
    return statistics.mean(out)


def extensions(B, W, torch, ctx, grid_ms):
    """Measurements of the paths beyond the hot-path pass: time-stepped
    predator-prey episodes, the coarse-to-fine grid search, and the reservoir
    tie-break. Each is timed alone with CUDA events after a warm-up call."""
    cuda = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()  # noqa: E731
    out = {}
    pp = B.compose_predator_prey(ctx)
    try:
        # episodes: 64 x up to 100 steps, each step a 27,000 x 64 search per episode
        w = W.predator_prey_episodes()
        E, T = w["start"].shape[0], w["max_steps"]
        d = B.episode_desc([cuda(x) for x in w["levels"]], cuda(w["start"]), w["n_trials"], T,
                           w["seed"], speed=w["speed"], radius=w["radius"])
        oc = torch.zeros(E, dtype=torch.int8, device="cuda")
        st = torch.zeros(E, dtype=torch.int32, device="cuda")
        o = B.episode_out(oc, st)
        B.dg_run_episodes(pp, d, o)
        ms = _time_ms(torch, lambda: B.dg_run_episodes(pp, d, o))
        steps = int(st.sum().item())
        nc = 30 ** 3
        res = oc.cpu().numpy()
        out["episodes"] = {
            "episodes": E, "max_steps": T, "candidates": nc, "trials": w["n_trials"],
            "episode_steps": steps, "ms": ms, "episode_steps_per_s": steps / (ms / 1e3),
            "evaluations_per_s": steps * nc * w["n_trials"] / (ms / 1e3),
            "outcomes": {"prey_caught": int((res == 1).sum()),
                         "player_caught": int((res == -1).sum()), "none": int((res == 0).sum())},
            "kernel_launches": 1 + T}
        # coarse-to-fine: 5 points x 7 rounds against the 30^3 grid, same positions
        g = W.predator_prey()
        pos = cuda(g["pos"])
        G, R = 5, 7
        rounds = torch.zeros(64 * R, dtype=torch.uint8, device="cuda")
        rd = B.refine_desc(pos, [0, 0, 0], [1, 1, 1], G, R, g["seed"])
        side = torch.cuda.Stream()
        with torch.cuda.stream(side):
            B.dg_grid_refine(pp, rd, rounds, stream=side)
        side.synchronize()
        ms_eager = _time_ms(torch, lambda: B.dg_grid_refine(pp, rd, rounds, stream=side),
                            stream=side)
        try:
            graph = torch.cuda.CUDAGraph()
            with torch.cuda.graph(graph, stream=side):
                B.dg_grid_refine(pp, rd, rounds, stream=side)
            graph.replay()  # replays on torch's current stream
            ms_graph = _time_ms(torch, graph.replay)
        except Exception as exc:  # capture refused: report it, keep the eager number
            ms_graph = f"capture failed: {exc}"
        # the launch-per-round form of the same search, for comparison
        os.environ["DG_REFINE_FUSED"] = "0"
        try:
            B.dg_grid_refine(pp, rd, rounds, stream=side)
            side.synchronize()
            graph2 = torch.cuda.CUDAGraph()
            with torch.cuda.graph(graph2, stream=side):
                B.dg_grid_refine(pp, rd, rounds, stream=side)
            graph2.replay()
            ms_graph_rounds = _time_ms(torch, graph2.replay)
        except Exception as exc:
            ms_graph_rounds = f"capture failed: {exc}"
        finally:
            del os.environ["DG_REFINE_FUSED"]
        B.dg_grid_refine(pp, rd, rounds, stream=side)
        side.synchronize()
        rr = B.refine_rounds(rounds.cpu().numpy())
        full = torch.zeros(3, dtype=torch.float64, device="cuda")
        lv = [cuda(x) for x in g["levels"]]
        B.dg_grid_search(pp, B.grid_desc(lv, pos, g["seed"]), full)
        fb = int(full.cpu().numpy()[:1].view(np.int64)[0])
        L = g["levels"][0].shape[0]
        full_alloc = [g["levels"][0][fb // (L * L)], g["levels"][1][(fb // L) % L],
                      g["levels"][2][fb % L]]
        # both answers re-evaluated on 1,024 fresh perceptions per position set
        ev = W.predator_prey(n_trials=1024, pos_seed=31)
        evpos = cuda(ev["pos"])

        def value_of(alloc):
            r = torch.zeros(3, dtype=torch.float64, device="cuda")
            B.dg_grid_search(pp, B.grid_desc([cuda(np.array([a], np.float32)) for a in alloc],
                                             evpos, 4242), r)
            return float(r.cpu().numpy()[1])
        out["coarse_to_fine"] = {
            "points": G, "rounds": R, "trials": 64, "candidates": R * G ** 3,
            "ms_eager": ms_eager, "ms_graph": ms_graph, "kernel_launches": 1,
            "form": "one 8-CTA cluster launch", "ms_graph_launch_per_round": ms_graph_rounds,
            "full_grid_candidates": nc, "full_grid_ms": grid_ms,
            "alloc": [float(a) for a in rr["alloc"][-1]], "full_grid_alloc": [float(a) for a in full_alloc],
            "value_fresh_1024": value_of(rr["alloc"][-1]),
            "full_grid_value_fresh_1024": value_of(full_alloc)}
        # Extended Stroop: the 4 x 1,000 Stroop trials, then two DDM nodes each
        ex = W.extended_stroop()
        xm = B.compose_extended_stroop(
            ctx, ex["layers"], ex["projections"],
            [dict(W=ex["ddm_W"][q:q + 1], bias=ex["ddm_bias"], dt=ex["ddm_dt"],
                  sigma=ex["ddm_sigma"], bound=ex["ddm_bound"], max_steps=ex["ddm_max"])
             for q in range(2)],
            rate=ex["rate"], noise_sd=ex["noise_sd"], stop_layer=ex["stop_layer"],
            stop_threshold=ex["stop_threshold"], max_steps=ex["max_steps"])
        try:
            n = ex["n_trials"]
            cond = cuda(ex["cond_inputs"])
            xc = torch.zeros(n, dtype=torch.int8, device="cuda")
            xs = torch.zeros(n, dtype=torch.int32, device="cuda")
            xf = torch.zeros(n * 8, dtype=torch.float32, device="cuda")
            xd = B.run_desc(n, ex["seed"], cond_inputs=cond, n_cond=cond.shape[0],
                            cond_block=ex["cond_block"])
            B.dg_run(xm, xd, xc, xs, xf)
            xms = _time_ms(torch, lambda: B.dg_run(xm, xd, xc, xs, xf))
            # final state per trial: y_0, y_1, then (x, choice, steps) per node
            f = xf.cpu().numpy().reshape(n, 8).astype(np.int64)
            ch, st = xc.cpu().numpy(), xs.cpu().numpy().astype(np.int64)
            winner = np.maximum(ch, 0) // 2
            winner_steps = np.where(ch >= 0, f[np.arange(n), 4 + 3 * winner], ex["ddm_max"])
            net_steps = int((st - winner_steps).sum())
            node_steps = int(f[:, 4].sum() + f[:, 7].sum())
            out["extended_stroop"] = {
                "trials": n, "ddm_nodes": 2, "ms": xms, "network_trial_steps": net_steps,
                "ddm_node_steps": node_steps,
                "trial_steps_per_s": (net_steps + node_steps) / (xms / 1e3)}
        finally:
            B.dg_model_free(xm)
        # a batch of 16 searches (the 30^3 x 64 grid, each its own positions and
        # seed) in one launch, against the same searches one call each
        nb = 16
        bw = [W.predator_prey(pos_seed=3 + i, noise_seed=13 + i) for i in range(nb)]
        bkeep = [([cuda(l) for l in w_["levels"]], cuda(w_["pos"])) for w_ in bw]
        bdesc = [B.grid_desc(lv_, pos_, w_["seed"]) for (lv_, pos_), w_ in zip(bkeep, bw)]
        bres = torch.zeros(nb * 3, dtype=torch.float64, device="cuda")
        B.dg_grid_search_batch(pp, bdesc, bres)
        ms_batch = _time_ms(torch, lambda: B.dg_grid_search_batch(pp, bdesc, bres))
        ms_single = _time_ms(torch, lambda: [B.dg_grid_search(pp, d_, bres[3 * i:3 * i + 3])
                                             for i, d_ in enumerate(bdesc)])
        evals = nb * nc * 64
        out["grid_search_batch"] = {
            "searches": nb, "candidates_per_search": nc, "trials": 64, "ms": ms_batch,
            "candidates_per_s": nb * nc / (ms_batch / 1e3),
            "frac_alu": evals * OPS_PER_UNIT["grid"] / (ms_batch / 1e3) / PEAK_OPS[0],
            "ms_one_call_each": ms_single,
            "candidates_per_s_one_call_each": nb * nc / (ms_single / 1e3)}
        # a larger batch: 64 searches (the ramp and drain of one launch spread wider)
        nb4 = 64
        bw4 = [W.predator_prey(pos_seed=3 + i, noise_seed=13 + i) for i in range(nb4)]
        bkeep4 = [([cuda(l) for l in w_["levels"]], cuda(w_["pos"])) for w_ in bw4]
        bdesc4 = [B.grid_desc(lv_, pos_, w_["seed"]) for (lv_, pos_), w_ in zip(bkeep4, bw4)]
        bres4 = torch.zeros(nb4 * 3, dtype=torch.float64, device="cuda")
        B.dg_grid_search_batch(pp, bdesc4, bres4)
        ms4 = _time_ms(torch, lambda: B.dg_grid_search_batch(pp, bdesc4, bres4))
        out["grid_search_batch"]["searches_64"] = {
            "ms": ms4, "candidates_per_s": nb4 * nc / (ms4 / 1e3),
            "frac_alu": nb4 * nc * 64 * OPS_PER_UNIT["grid"] / (ms4 / 1e3) / PEAK_OPS[0]}
        # reservoir tie-break: the 30^3 search with either rule
        res0 = torch.zeros(3, dtype=torch.float64, device="cuda")
        d0 = B.grid_desc(lv, pos, g["seed"])
        d1 = B.grid_desc(lv, pos, g["seed"], tie_break=B.DG_TIE_RESERVOIR)
        B.dg_grid_search(pp, d1, res0)
        out["tie_break"] = {
            "ms_lowest_index": _time_ms(torch, lambda: B.dg_grid_search(pp, d0, res0)),
            "ms_reservoir": _time_ms(torch, lambda: B.dg_grid_search(pp, d1, res0))}
    finally:
        B.dg_model_free(pp)
    return out


def _pinned(torch, a):
    t = torch.from_numpy(np.ascontiguousarray(a)).pin_memory()
    return t, t.numpy()


def e2e_serving(B, torch, ctx, step, all_ts, world, rank):
    """The pass through dg_submit/dg_wait: host inputs copied in, outputs
    copied back, every step."""
    host_jobs = []
    h2d = d2h = 0
    for j in in_job_order(step.jobs):
        job = B.dg_job()
        job.model = j["model"].value
        keep = []
        if j.get("grid"):
            d = j["desc"]
            job.is_grid = 1
            job.grid = B.dg_grid_desc.from_buffer_copy(d)
            pos_t, pos = _pinned(torch, j["host_in"][0])
            keep.append(pos_t)
            job.grid.positions = pos.ctypes.data
            for i in range(3):
                lt, lv = _pinned(torch, j["host_in"][1 + i])
                keep.append(lt)
                job.grid.levels[i] = lv.ctypes.data
                h2d += lv.nbytes
            h2d += pos.nbytes
            rt, res = _pinned(torch, np.zeros(3, np.float64))
            keep.append(rt)
            job.grid_result = res.ctypes.data
            d2h += 24
        else:
            d = j["desc"]
            job.run = B.dg_run_desc.from_buffer_copy(d)
            pt, hp = _pinned(torch, j["host_in"][0])
            keep.append(pt)
            if d.trial_params:
                job.run.trial_params = hp.ctypes.data
            else:
                job.run.cond_inputs = hp.ctypes.data
            h2d += hp.nbytes
            ct, ch = _pinned(torch, np.zeros(max(1, j["n"]), np.int8))
            st, sp = _pinned(torch, np.zeros(max(1, j["n"]), np.int32))
            keep += [ct, st]
            job.choice = ch.ctypes.data
            job.step = sp.ctypes.data
            d2h += j["n"] * 5
        host_jobs.append((job, keep))

    def one():
        tickets = [B.dg_submit(ctx, jb) for jb, _ in host_jobs]
        for t in tickets:
            B.dg_wait(ctx, t, 600000)

    one()
    one()
    times = []
    for _ in range(3):
        if world > 1:
            torch.distributed.barrier()
        t0 = time.perf_counter()
        one()
        times.append(time.perf_counter() - t0)
    sec = statistics.mean(times)
    if world > 1:
        t = torch.tensor([sec], dtype=torch.float64, device="cuda")
        torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
        sec = float(t[0])
    return {"value": all_ts / sec, "unit": UNIT, "h2d_bytes_per_step": h2d,
            "d2h_bytes_per_step": d2h, "ms_per_step": 1000 * sec,
            "api": "dg_submit/dg_wait (serving loop, pinned host buffers)"}


SERVE_JOBS = 256


def _mix(B, W, torch, step, n_jobs, seed, kinds=("stroop", "ddm", "lca", "grid", "wide"),
         log_trials=(3, 6)):
    """The served mix: jobs drawn uniformly from the five workloads, trial
    counts log-uniform in [1e3, 1e6] (grid jobs: levels per signal
    clamp(round((n / 64)^(1/3)), 2, 30) at 64 trials per candidate). Each job
    carries its pinned host buffers, a dg_job for the serving API and the device
    buffers of the plain form."""
    rng = np.random.default_rng(seed)
    models = {j["name"]: j["model"] for j in step.jobs}
    kinds = [k for k in kinds if k != "wide" or "wide" in models]
    jobs = []
    for _ in range(n_jobs):
        k = kinds[rng.integers(0, len(kinds))]
        n = int(round(10 ** rng.uniform(*log_trials)))
        jobs.append((k, n, int(rng.integers(0, 1 << 31))))
    cuda = lambda t: torch.empty_like(t, device="cuda")  # noqa: E731
    prepared = []
    for k, n, sd in jobs:
        job = B.dg_job()
        rec = {"kind": k, "n": n, "seed": sd, "job": job}
        if k == "grid":
            L = int(min(30, max(2, round((n / 64) ** (1 / 3)))))
            g = W.predator_prey(levels=L, noise_seed=sd)
            rec["model"] = models["grid"]
            job.model = models["grid"].value
            job.is_grid = 1
            pt, pos = _pinned(torch, g["pos"])
            job.grid.positions = pos.ctypes.data
            job.grid.n_trials = 64
            job.grid.seed = sd
            lts = []
            for i in range(3):
                lt, lv = _pinned(torch, g["levels"][i])
                lts.append(lt)
                job.grid.levels[i] = lv.ctypes.data
                job.grid.n_levels[i] = L
            rt, res = _pinned(torch, np.zeros(3, np.float64))
            job.grid_result = res.ctypes.data
            rec.update(host_in=[pt] + lts, host_out=[rt], dev_in=[cuda(pt)] + [cuda(t) for t in lts],
                       dev_out=[cuda(rt)], steps=L ** 3 * 64)
        else:
            if k == "stroop":
                s_ = W.stroop_small()
                rec["model"] = models["stroop"]
                ht, h = _pinned(torch, s_["cond_inputs"])
                job.run.cond_inputs = h.ctypes.data
                job.run.n_cond, job.run.cond_block = 4, max(1, n // 4)
            elif k == "wide":
                wd = W.stroop_wide(n_trials=n)
                rec["model"] = models["wide"]
                ht, h = _pinned(torch, wd["cond_inputs"])
                job.run.cond_inputs = h.ctypes.data
                job.run.n_cond, job.run.cond_block = 256, 1
            elif k == "ddm":
                w = W.ddm(n_trials=n, param_seed=sd)
                rec["model"] = models["ddm"]
                ht, h = _pinned(torch, np.concatenate([w["A"], w["z"]]))
                job.run.trial_params = h.ctypes.data
            else:
                l_ = W.lca(n_trials=n, N=8, input_seed=sd)
                rec["model"] = models["lca8"]
                ht, h = _pinned(torch, l_["I"])
                job.run.trial_params = h.ctypes.data
            job.model = rec["model"].value
            job.run.n_trials = n
            job.run.seed = sd
            ct, ch = _pinned(torch, np.zeros(n, np.int8))
            st, sp = _pinned(torch, np.zeros(n, np.int32))
            job.choice = ch.ctypes.data
            job.step = sp.ctypes.data
            rec.update(host_in=[ht], host_out=[ct, st], dev_in=[cuda(ht)],
                       dev_out=[cuda(ct), cuda(st)], cond=bool(job.run.cond_inputs),
                       n_cond=job.run.n_cond, cond_block=job.run.cond_block)
        prepared.append(rec)
    return prepared


def _plain_job(B, rec, stream):
    """One job in the plain form: inputs copied in, one plain launch, outputs
    copied back, on one stream; returns when the outputs are on the host."""
    for d, h in zip(rec["dev_in"], rec["host_in"]):
        d.copy_(h, non_blocking=True)
    if rec["kind"] == "grid":
        pos, l0, l1, l2 = rec["dev_in"]
        d = B.grid_desc([l0, l1, l2], pos, rec["seed"], mode=B.DG_MODE_PLAIN)
        B.dg_grid_search(rec["model"], d, rec["dev_out"][0], stream=stream)
    else:
        x = rec["dev_in"][0]
        d = (B.run_desc(rec["n"], rec["seed"], cond_inputs=x, n_cond=rec["n_cond"],
                        cond_block=rec["cond_block"], mode=B.DG_MODE_PLAIN) if rec["cond"] else
             B.run_desc(rec["n"], rec["seed"], trial_params=x, mode=B.DG_MODE_PLAIN))
        B.dg_run(rec["model"], d, rec["dev_out"][0], rec["dev_out"][1], stream=stream)
    for h, d in zip(rec["host_out"], rec["dev_out"]):
        h.copy_(d, non_blocking=True)
    stream.synchronize()


def _tune_mix(B, prepared, stream):
    """Tune the launch shapes of the mix's size buckets before serving it, as a
    deployment would from its tuning cache: one batched run per (kind, trial
    count bucket) on this thread (the serving thread never times shapes)."""
    seen = set()
    for rec in prepared:
        key = (rec["kind"], int(math.ceil(math.log2(max(rec["n"], 1)))))
        if key in seen:
            continue
        seen.add(key)
        for d, h in zip(rec["dev_in"], rec["host_in"]):
            d.copy_(h, non_blocking=True)
        if rec["kind"] == "grid":
            pos, l0, l1, l2 = rec["dev_in"]
            B.dg_grid_search(rec["model"], B.grid_desc([l0, l1, l2], pos, rec["seed"]),
                             rec["dev_out"][0], stream=stream)
        else:
            x = rec["dev_in"][0]
            d = (B.run_desc(rec["n"], rec["seed"], cond_inputs=x, n_cond=rec["n_cond"],
                            cond_block=rec["cond_block"]) if rec["cond"] else
                 B.run_desc(rec["n"], rec["seed"], trial_params=x))
            B.dg_run(rec["model"], d, rec["dev_out"][0], rec["dev_out"][1], stream=stream)
    stream.synchronize()


def _trial_steps(prepared):
    return sum(r["steps"] if r["kind"] == "grid" else int(r["host_out"][1].numpy().sum())
               for r in prepared)


def _lat_stats(lat, wall, n_jobs, steps):
    lat = sorted(lat)
    p99 = lat[min(len(lat) - 1, int(math.ceil(0.99 * len(lat))) - 1)]
    return {"p50_ms": 1000 * lat[len(lat) // 2], "p99_ms": 1000 * p99,
            "max_ms": 1000 * lat[-1], "wall_s": wall, "jobs_per_s": n_jobs / wall,
            "trial_steps_per_s": steps / wall}


def _serve(B, ctx, prepared, arrivals):
    """Submit each job at its arrival time (seconds from the start) through
    dg_submit; latency = completion - submission (the library's clock)."""
    t0 = time.perf_counter()
    tickets = []
    for rec, a in zip(prepared, arrivals):
        while time.perf_counter() - t0 < a:
            time.sleep(min(0.0005, max(0.0, a - (time.perf_counter() - t0))))
        tickets.append(B.dg_submit(ctx, rec["job"]))
    lat = []
    for t in tickets:
        r = B.dg_wait(ctx, t, 600000)
        lat.append(r.t_done - r.t_submit)
    return lat, time.perf_counter() - t0


def _plain(B, prepared, arrivals, stream):
    """The same jobs one after another on one stream in arrival order, each
    started at its arrival time or when the previous one ends, whichever is
    later; latency = completion - arrival."""
    t0 = time.perf_counter()
    lat = []
    for rec, a in zip(prepared, arrivals):
        while time.perf_counter() - t0 < a:
            time.sleep(min(0.0005, max(0.0, a - (time.perf_counter() - t0))))
        _plain_job(B, rec, stream)
        lat.append(time.perf_counter() - t0 - a)
    return lat, time.perf_counter() - t0


def served_small_jobs(B, W, torch, ctx, step, n_jobs=SERVE_JOBS, seed=17):
    """Many small jobs: DDM, LCA (N = 8) and Stroop jobs of 1e3-1e4 trials, all
    arriving at once, through the serving API and through the plain form:
    jobs/s, trial-steps/s and latency."""
    prepared = _mix(B, W, torch, step, n_jobs, seed, kinds=("ddm", "lca", "stroop"),
                    log_trials=(3, 4))
    stream = torch.cuda.Stream()
    zero = [0.0] * n_jobs
    # a second context whose serving loop gives every job its own launch
    os.environ["DG_SERVE_GROUP_TRIALS"] = "0"
    try:
        ctx_each = B.dg_create(0)
        _serve(B, ctx_each, prepared, zero)
    finally:
        del os.environ["DG_SERVE_GROUP_TRIALS"]
    _serve(B, ctx, prepared, zero)
    with torch.cuda.stream(stream):
        _plain(B, prepared, zero, stream)
    steps = _trial_steps(prepared)
    res = {}
    for r in range(3):   # best of three per form, the forms interleaved
        for name, fn in (("served", lambda: _serve(B, ctx, prepared, zero)),
                         ("served_per_job", lambda: _serve(B, ctx_each, prepared, zero))):
            lat, wall = fn()
            if name not in res or wall < res[name][1]:
                res[name] = (lat, wall)
    with torch.cuda.stream(stream):
        lat_p, wall_p = _plain(B, prepared, zero, stream)
    B.dg_destroy(ctx_each)
    return {"jobs": n_jobs, "mix": "ddm/lca8/stroop, trials log-uniform 1e3-1e4, all at once",
            "trial_steps": steps,
            "served": dict(_lat_stats(*res["served"], n_jobs, steps),
                           form="serving loop, small jobs of one model share a launch"),
            "served_per_job": dict(_lat_stats(*res["served_per_job"], n_jobs, steps),
                                   form="serving loop, a launch and a stream per job"),
            "plain": _lat_stats(lat_p, wall_p, n_jobs, steps)}


def served_mix(B, W, torch, ctx, step, n_jobs=SERVE_JOBS, seed=7):
    """The served mix against the plain one-launch-per-job form on the same
    jobs. Capacity: all jobs arriving at once (jobs/s until the last result is
    on the host). Then Poisson arrivals at 0.7x each form's capacity, the same
    arrival sequence (scaled) replayed through both forms: p50/p99 latency
    (arrival to results on the host), jobs/s and trial-steps/s."""
    prepared = _mix(B, W, torch, step, n_jobs, seed)
    stream = torch.cuda.Stream()
    zero = [0.0] * n_jobs
    with torch.cuda.stream(stream):
        _tune_mix(B, prepared, stream)
    # warm-up: the serving pool and the plain form's per-stream scratch
    _serve(B, ctx, prepared, zero)
    with torch.cuda.stream(stream):
        _plain(B, prepared, zero, stream)
    steps = _trial_steps(prepared)
    untuned0 = B.dg_tune_stats(ctx)[1]
    lat_s, wall_s = _serve(B, ctx, prepared, zero)
    with torch.cuda.stream(stream):
        lat_p, wall_p = _plain(B, prepared, zero, stream)
    cap_s, cap_p = n_jobs / wall_s, n_jobs / wall_p
    gaps = np.random.default_rng(seed + 1).exponential(1.0, n_jobs)
    unit = np.cumsum(gaps) - gaps[0]          # unit-rate Poisson arrival times

    def at(rate):
        arr = list(unit / rate)
        ls, ws = _serve(B, ctx, prepared, arr)
        with torch.cuda.stream(stream):
            lp, wp = _plain(B, prepared, arr, stream)
        return {"arrival_rate_per_s": rate, "served": _lat_stats(ls, ws, n_jobs, steps),
                "plain": _lat_stats(lp, wp, n_jobs, steps)}
    at_served = at(0.7 * cap_s)
    at_plain = at(0.7 * cap_p)
    tuned_keys, untuned1 = B.dg_tune_stats(ctx)
    out = dict(at_served["served"])
    # the serving thread never times launch shapes: served launches whose size
    # bucket had no tuned shape ran the default one
    out["tuner"] = {"tuned_keys": tuned_keys,
                    "untuned_launches_in_served_runs": untuned1 - untuned0}
    out.update({
        "jobs": n_jobs, "mix": "stroop/ddm/lca8/grid/wide, trials log-uniform 1e3-1e6",
        "arrival_rate_per_s": at_served["arrival_rate_per_s"],
        "capacity_jobs_per_s": cap_s, "capacity_trial_steps_per_s": steps / wall_s,
        "saturated": _lat_stats(lat_s, wall_s, n_jobs, steps),
        "plain": dict(at_served["plain"], capacity_jobs_per_s=cap_p,
                      capacity_trial_steps_per_s=steps / wall_p,
                      saturated=_lat_stats(lat_p, wall_p, n_jobs, steps),
                      form="dg_run / dg_grid_search DG_MODE_PLAIN, one job after another on "
                           "one stream, host copies included"),
        "at_plain_capacity_rate": at_plain,
        "trial_steps": steps})
    return out


if __name__ == "__main__":
    main()
