"""GPU parity: Philox words, normals and the DDM kernels against the oracle."""
import numpy as np
import pytest

from gpu_util import FLOAT_RTOL, compare_decisions, dev, host, rel_err

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    import torch
    from paper_2110_15425_gb300 import binding as B
    torch.cuda.init()
    c = B.dg_create(0)
    yield c
    B.dg_destroy(c)


@pytest.mark.parametrize("seed,trial,cand,purpose,block0,n", [
    (0, 0, 0, 0, 0, 1000), (11, 5, 0, 0, 2000, 333), ((7 << 32) | 99, 123456, 26999, 0, 0, 64),
    (0xFFFFFFFFFFFFFFFF, 0xFFFFFFFF, 0xFFFFFFFF, 3, 0xFFFFFFF0, 16)])
def test_philox_words_bitwise(orc, seed, trial, cand, purpose, block0, n):
    import torch
    from paper_2110_15425_gb300 import binding as B
    out = torch.zeros(4 * n, dtype=torch.int32, device="cuda")
    B.dg_philox_words(seed, trial, cand, purpose, block0, n, out)
    got = host(out).view(np.uint32)
    ref = orc.philox_words(seed, trial, cand, purpose, block0, n)
    assert np.array_equal(got, ref)


def test_normals_match_oracle(orc):
    """FP32 Box-Muller with the hardware log2 / sine / cosine approximations
    (and a series for ln u near u = 1) against the FP64 oracle: error below
    2e-6 x max(1, |z|) on 4 million draws, including the draws nearest u = 1."""
    import torch
    from paper_2110_15425_gb300 import binding as B
    n = 1 << 22
    out = torch.zeros(n, dtype=torch.float32, device="cuda")
    B.dg_normals(42, 7, 3, 5, n, out)
    got = host(out).astype(np.float64)
    ref = orc.normals(42, 7, 3, 5, n)
    rel = np.abs(got - ref) / np.maximum(np.abs(ref), 1.0)
    print("normals: max err / max(1,|z|) =", rel.max(), " mean =", rel.mean())
    assert rel.max() < 2e-6


def _ddm_run(ctx, A, z, seed, mode, max_steps=10000, dt=1e-3, sigma=1.0):
    import torch
    from paper_2110_15425_gb300 import binding as B
    n = A.shape[0]
    model = B.compose_ddm(ctx, dt=dt, sigma=sigma, max_steps=max_steps)
    try:
        params = dev(np.concatenate([A, z]).astype(np.float32))
        choice = torch.zeros(max(n, 1), dtype=torch.int8, device="cuda")
        step = torch.zeros(max(n, 1), dtype=torch.int32, device="cuda")
        xs = torch.zeros(max(n, 1), dtype=torch.float32, device="cuda")
        B.dg_run(model, B.run_desc(n, seed, trial_params=params, mode=mode), choice, step, xs)
        return host(choice)[:n], host(step)[:n], host(xs)[:n]
    finally:
        B.dg_model_free(model)


@pytest.mark.parametrize("mode", [0, 1])
@pytest.mark.parametrize("n", [1, 37, 5000])
def test_ddm_parity_small(ctx, orc, threads, mode, n):
    from paper_2110_15425_gb300 import workloads as W
    w = W.ddm(n_trials=n, param_seed=5)
    c, s, x = _ddm_run(ctx, w["A"], w["z"], w["seed"], mode)
    ref = orc.ddm_run(w["A"], w["z"], w["seed"], threads=threads)
    excl = compare_decisions(c, s, ref, f"ddm mode={mode}")
    assert excl <= max(2, n // 200)
    keep = ref["margin"] >= 1e-5
    assert rel_err(x[keep], ref["x"][keep], w["z"][keep]) < FLOAT_RTOL


@pytest.mark.parametrize("max_steps", [1, 2, 7, 13])
def test_ddm_short_caps(ctx, orc, max_steps):
    from paper_2110_15425_gb300 import workloads as W
    w = W.ddm(n_trials=300, param_seed=6)
    w["A"][:10] = 50.0  # crosses within the first steps
    for mode in (0, 1):
        c, s, x = _ddm_run(ctx, w["A"], w["z"], 3, mode, max_steps=max_steps)
        ref = orc.ddm_run(w["A"], w["z"], 3, max_steps=max_steps)
        compare_decisions(c, s, ref, f"cap {max_steps}")
        assert np.all(s <= max_steps)


def test_ddm_bounds_on_both_state_formats(ctx, orc, threads):
    """Bounds up to 6 keep the state in 32-bit fixed point, larger ones in 64
    bits: a mix of both (and bounds right at the switch) against the oracle,
    and the two forms bit for bit."""
    rng = np.random.default_rng(11)
    n = 3000
    A = rng.uniform(2.0, 5.0, n).astype(np.float32)
    z = rng.uniform(4.0, 9.0, n).astype(np.float32)
    z[:50] = 6.0
    z[50:100] = np.nextafter(np.float32(6.0), np.float32(7.0))
    out = []
    for mode in (0, 1):
        c, s, x = _ddm_run(ctx, A, z, 21, mode)
        ref = orc.ddm_run(A, z, 21, threads=threads)
        assert compare_decisions(c, s, ref, f"wide bounds mode={mode}") <= n // 200
        keep = ref["margin"] >= 1e-5
        assert rel_err(x[keep], ref["x"][keep], z[keep]) < FLOAT_RTOL
        out.append((c, s, x))
    for u, v in zip(*out):
        assert np.array_equal(u, v)


def test_ddm_empty(ctx):
    c, s, x = _ddm_run(ctx, np.zeros(0, np.float32), np.zeros(0, np.float32), 1, 0)
    assert c.size == 0


def test_ddm_plain_equals_batched(ctx):
    from paper_2110_15425_gb300 import workloads as W
    w = W.ddm(n_trials=20000, param_seed=7)
    a = _ddm_run(ctx, w["A"], w["z"], 9, 0)
    b = _ddm_run(ctx, w["A"], w["z"], 9, 1)
    for u, v in zip(a, b):
        assert np.array_equal(u, v)


def test_ddm_full_size_sampled(ctx, orc, threads):
    """2^20 trials in the benchmark's launch configuration; 4096 sampled
    trials replayed by the oracle."""
    from paper_2110_15425_gb300 import workloads as W
    w = W.ddm()
    c, s, x = _ddm_run(ctx, w["A"], w["z"], w["seed"], 0)
    rng = np.random.default_rng(0)
    ids = np.sort(rng.choice(w["A"].shape[0], 4096, replace=False)).astype(np.uint32)
    ref = orc.ddm_run(w["A"], w["z"], w["seed"], trial_ids=ids, threads=threads)
    compare_decisions(c[ids], s[ids], ref, "ddm full")
    keep = ref["margin"] >= 1e-5
    assert rel_err(x[ids][keep], ref["x"][keep], w["z"][ids][keep]) < FLOAT_RTOL
    # properties at any size: decisions are +-1 or timeouts; steps in range
    assert set(np.unique(c)).issubset({-1, 0, 1})
    assert s.min() >= 1 and s.max() <= 10000
    assert np.all(s[c == -1] == 10000)
