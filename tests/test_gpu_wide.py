"""GPU parity: the wide multitask network (tensor-core batched form and
CUDA-core comparison form) against the oracle.

The response weights are bfloat16 on the device, so the oracle is fed the
same bf16-rounded values (as FP32): the remaining difference is FP32 state
and the hi+lo bf16 split of the hidden outputs (~2^-17 relative), well inside
the FP32-state tolerance. The error of the bf16 weights themselves, against
an oracle with the original FP32 weights, is measured and reported.
"""
import numpy as np
import pytest

from gpu_util import FLOAT_RTOL, compare_decisions, dev, host, rel_err

pytestmark = pytest.mark.gpu


def _bf16(a):
    """round-to-nearest-even bfloat16, returned as float32"""
    u = np.ascontiguousarray(a, np.float32).view(np.uint32).astype(np.uint64)
    u = (u + 0x7FFF + ((u >> 16) & 1)) & 0xFFFF0000
    return u.astype(np.uint32).view(np.float32)


@pytest.fixture(scope="module")
def ctx():
    import torch
    from paper_2110_15425_gb300 import binding as B
    torch.cuda.init()
    c = B.dg_create(0)
    yield c
    B.dg_destroy(c)


def _wide(ctx, w, mode, n, trial_offset=0):
    import torch
    from paper_2110_15425_gb300 import binding as B
    model = B.compose_network(ctx, w["layers"], w["projections"], rate=w["rate"],
                              noise_sd=w["noise_sd"], stop_layer=w["stop_layer"],
                              stop_threshold=w["stop_threshold"], max_steps=w["max_steps"],
                              bf16_edges=(2,))
    try:
        kind, ss = B.dg_model_info(model)
        assert B.MODEL_KINDS[kind] == "transfer_wide" and ss == 16
        cond = dev(w["cond_inputs"])
        choice = torch.zeros(max(n, 1), dtype=torch.int8, device="cuda")
        step = torch.zeros(max(n, 1), dtype=torch.int32, device="cuda")
        ys = torch.zeros(max(n, 1) * 16, dtype=torch.float32, device="cuda")
        B.dg_run(model, B.run_desc(n, w["seed"], cond_inputs=cond, n_cond=cond.shape[0],
                                   cond_block=w["cond_block"], mode=mode,
                                   trial_offset=trial_offset), choice, step, ys)
        B.dg_stream_status(ctx)
        return host(choice)[:n], host(step)[:n], host(ys)[:n * 16].reshape(n, 16)
    finally:
        B.dg_model_free(model)


def _ref(orc, w, threads, n=None, trial_ids=None, exact_weights=False):
    proj = list(w["projections"])
    if not exact_weights:
        s, r, W = proj[2]
        proj[2] = (s, r, _bf16(W))
    return orc.transfer_run(w["layers"], proj, w["cond_inputs"], w["cond_block"], w["seed"],
                            rate=w["rate"], noise_sd=w["noise_sd"], stop_layer=w["stop_layer"],
                            stop_threshold=w["stop_threshold"], max_steps=w["max_steps"],
                            n_trials=n, trial_ids=trial_ids, threads=threads)


@pytest.mark.parametrize("mode", [0, 1])
def test_wide_parity(ctx, orc, threads, mode):
    from paper_2110_15425_gb300 import workloads as W
    w = W.stroop_wide(n_trials=389, max_steps=120)
    c, s, y = _wide(ctx, w, mode, 389)
    ref = _ref(orc, w, threads, n=389)
    compare_decisions(c, s, ref, f"wide mode={mode}")
    assert rel_err(y, ref["y"], 1e-2) < FLOAT_RTOL
    assert (ref["choice"] >= 0).any() and (ref["choice"] < 0).any()


@pytest.mark.parametrize("H", [64, 128, 192])
def test_wide_sizes_noise_free(ctx, orc, threads, H):
    from paper_2110_15425_gb300 import workloads as W
    w = W.stroop_wide(n_trials=300, max_steps=60)
    rng = np.random.default_rng(H)
    w["layers"][2]["size"] = H
    w["projections"] = [(0, 2, rng.uniform(-6, 6, (H, 16)).astype(np.float32)),
                        (1, 2, rng.uniform(-6, 6, (H, 16)).astype(np.float32)),
                        (2, 3, rng.uniform(-2, 2, (16, H)).astype(np.float32) * 2)]
    w["noise_sd"] = 0.0
    for mode in (0, 1):
        c, s, y = _wide(ctx, w, mode, 300)
        ref = _ref(orc, w, threads, n=300)
        compare_decisions(c, s, ref, f"wide H={H} mode={mode}")
        assert rel_err(y, ref["y"], 1e-2) < FLOAT_RTOL


def test_wide_bench_size_sampled(ctx, orc, threads):
    """16,384 trials (the benchmark's wide member), 512 sampled trials
    replayed by the oracle; the error of bf16 weights against the FP32-weight
    oracle is reported."""
    from paper_2110_15425_gb300 import workloads as W
    w = W.stroop_wide(n_trials=16384)
    c, s, y = _wide(ctx, w, 0, 16384)
    ids = np.sort(np.random.default_rng(1).choice(16384, 512, replace=False)).astype(np.uint32)
    ref = _ref(orc, w, threads, trial_ids=ids)
    compare_decisions(c[ids], s[ids], ref, "wide full")
    assert rel_err(y[ids], ref["y"], 1e-2) < FLOAT_RTOL
    exact = _ref(orc, w, threads, trial_ids=ids, exact_weights=True)
    same = (exact["choice"] == c[ids]).mean()
    print(f"wide: bf16 response weights vs FP32-weight oracle: choice agreement {same:.4f}, "
          f"max rel err of outputs {rel_err(y[ids], exact['y'], 1e-2):.2e}")


def test_wide_tc_equals_cuda_core_decisions(ctx):
    from paper_2110_15425_gb300 import workloads as W
    w = W.stroop_wide(n_trials=5000, max_steps=200)
    a = _wide(ctx, w, 0, 5000)
    b = _wide(ctx, w, 1, 5000)
    assert (a[0] == b[0]).mean() > 0.999 and (a[1] == b[1]).mean() > 0.999
    assert rel_err(a[2], b[2], 1e-2) < FLOAT_RTOL
