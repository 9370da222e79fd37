"""Parity of the configuration the benchmark times: the whole hot-path pass at
full size (Stroop 4 x 1,000, DDM 2^20, LCA 262,144 x N in {4, 8, 16}, wide
network 16,384, predator-prey 27,000 x 64), built by bench.py as one CUDA-graph
batch with tuned launch shapes, launched twice (capture, then a replay).
Sampled trials of every job, the whole Stroop job and the grid search's
choice are compared with the oracle."""
import numpy as np
import pytest

from gpu_util import compare_decisions, host

pytestmark = pytest.mark.gpu


def _bf16(a):
    """round-to-nearest-even bfloat16, returned as float32"""
    u = np.ascontiguousarray(a, np.float32).view(np.uint32).astype(np.uint64)
    u = (u + 0x7FFF + ((u >> 16) & 1)) & 0xFFFF0000
    return u.astype(np.uint32).view(np.float32)


def test_bench_pass_matches_oracle(orc, threads):
    import torch

    import bench
    from paper_2110_15425_gb300 import binding as B
    from paper_2110_15425_gb300 import workloads as W
    torch.cuda.init()
    ctx = B.dg_create(0)
    step = None
    try:
        step = bench.Step(B, W, torch, ctx, 0, 1)
        step.launch(ctx)   # tunes shapes, captures the batch graph, runs it
        for j in step.jobs:
            for t in j["out"].values():
                t.zero_()
        step.launch(ctx)   # replay of the graph
        torch.cuda.synchronize()
        jobs = {j["name"]: j for j in step.jobs}
        assert set(jobs) == {"stroop", "ddm", "lca4", "lca8", "lca16", "wide", "grid"}
        assert B.dg_batch_kernels(step.batch) >= len(jobs)

        def out(name):
            o = jobs[name]["out"]
            return host(o["choice"])[:jobs[name]["n"]], host(o["step"])[:jobs[name]["n"]]

        rng = np.random.default_rng(2024)
        # DDM: 2,048 sampled trials of 2^20
        w = W.ddm()
        c, s = out("ddm")
        ids = np.sort(rng.choice(w["A"].shape[0], 2048, replace=False)).astype(np.uint32)
        ref = orc.ddm_run(w["A"], w["z"], w["seed"], dt=w["dt"], sigma=w["sigma"],
                          max_steps=w["max_steps"], trial_ids=ids, threads=threads)
        compare_decisions(c[ids], s[ids], ref, "pass ddm")
        # LCA: 1,024 sampled trials of each job
        for N in (4, 8, 16):
            w = W.lca(N=N)
            c, s = out(f"lca{N}")
            ids = np.sort(rng.choice(w["I"].shape[0], 1024, replace=False)).astype(np.uint32)
            ref = orc.lca_run(w["I"], w["seed"], leak=w["leak"], inhibition=w["inhibition"],
                              sigma=w["sigma"], dt=w["dt"], threshold=w["threshold"],
                              max_steps=w["max_steps"], trial_ids=ids, threads=threads)
            compare_decisions(c[ids], s[ids], ref, f"pass lca{N}")
        # Stroop: every trial
        w = W.stroop_small()
        c, s = out("stroop")
        ref = orc.transfer_run(w["layers"], w["projections"], w["cond_inputs"], w["cond_block"],
                               w["seed"], rate=w["rate"], noise_sd=w["noise_sd"],
                               stop_layer=w["stop_layer"], stop_threshold=w["stop_threshold"],
                               max_steps=w["max_steps"], n_trials=w["n_trials"], threads=threads)
        compare_decisions(c, s, ref, "pass stroop")
        # wide network: 256 sampled trials, oracle fed the device's bf16 response weights
        w = W.stroop_wide(n_trials=bench.WIDE_TRIALS)
        c, s = out("wide")
        ids = np.sort(rng.choice(bench.WIDE_TRIALS, 256, replace=False)).astype(np.uint32)
        proj = list(w["projections"])
        snd, rcv, Wr = proj[2]
        proj[2] = (snd, rcv, _bf16(Wr))
        ref = orc.transfer_run(w["layers"], proj, w["cond_inputs"], w["cond_block"], w["seed"],
                               rate=w["rate"], noise_sd=w["noise_sd"], stop_layer=w["stop_layer"],
                               stop_threshold=w["stop_threshold"], max_steps=w["max_steps"],
                               trial_ids=ids, threads=threads)
        compare_decisions(c[ids], s[ids], ref, "pass wide")
        # predator-prey grid: the choice and its mean against the oracle's means
        g = W.predator_prey(pos_seed=3)
        r = host(jobs["grid"]["out"]["result"])
        best, val, gap = int(r[:1].view(np.int64)[0]), float(r[1]), float(r[2])
        means = orc.pp_means(g["pos"], g["levels"], g["seed"], obs_offset=g["obs_offset"],
                             pred_weight=g["pred_weight"], threads=threads)
        srt = np.sort(means)
        if srt[-1] - srt[-2] >= 1e-5:
            assert best == int(np.argmax(means))
        assert abs(val - means.max()) <= 1e-5 * max(1.0, abs(means.max()))
        assert abs(gap - (srt[-1] - srt[-2])) <= 1e-5 * max(1.0, abs(means.max()))
    finally:
        if step is not None:
            torch.cuda.synchronize()
            if step.batch is not None:
                B.dg_batch_free(step.batch)
            for j in step.jobs:
                B.dg_model_free(j["model"])
        B.dg_destroy(ctx)
