"""GPU parity: LCA (every threads-per-trial layout) and the small logistic
network (Botvinick Stroop) against the oracle."""
import os

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


def _lca(ctx, I, seed, mode, **kw):
    import torch
    from paper_2110_15425_gb300 import binding as B
    n, N = I.shape
    model = B.compose_lca(ctx, N, **kw)
    try:
        choice = torch.zeros(max(n, 1), dtype=torch.int8, device="cuda")
        step = torch.zeros(max(n, 1), dtype=torch.int32, device="cuda")
        xs = torch.zeros(max(n, 1) * N, dtype=torch.float32, device="cuda")
        B.dg_run(model, B.run_desc(n, seed, trial_params=dev(I), mode=mode), choice, step, xs)
        return host(choice)[:n], host(step)[:n], host(xs)[:n * N].reshape(n, N)
    finally:
        B.dg_model_free(model)


@pytest.mark.parametrize("N,tpt", [(4, 1), (8, 1), (8, 2), (16, 1), (16, 2), (16, 4), (5, 1),
                                   (3, 1), (1, 1), (4, -1), (8, -1), (16, -1), (5, -1), (1, -1)])
def test_lca_parity(ctx, orc, threads, monkeypatch, N, tpt):
    from paper_2110_15425_gb300 import workloads as W
    monkeypatch.setenv("DG_LCA_TPT", str(tpt))
    w = W.lca(n_trials=3000 + 7, N=N)
    kw = dict(leak=w["leak"], inhibition=w["inhibition"], sigma=w["sigma"], dt=w["dt"],
              threshold=w["threshold"], max_steps=w["max_steps"])
    # tpt -1: one lane per trial with block-level compaction of the running trials
    for mode in ((0, 1) if tpt == 1 else (0,)):
        c, s, x = _lca(ctx, w["I"], w["seed"], mode, **kw)
        ref = orc.lca_run(w["I"], w["seed"], threads=threads, **kw)
        compare_decisions(c, s, ref, f"lca N={N} tpt={tpt} mode={mode}")
        keep = ref["margin"] >= 1e-5
        assert rel_err(x[keep], ref["x"][keep], w["threshold"]) < FLOAT_RTOL
        assert np.all(x >= 0)


@pytest.mark.parametrize("tpt", ["1", "-1"])
def test_lca_batched_equals_plain_bitwise(ctx, monkeypatch, tpt):
    """The batched form hands trials out longest-expected-first, splits a
    trial over several lanes or moves it between lanes when it compacts the
    running trials; none of this changes any result bit."""
    from paper_2110_15425_gb300 import workloads as W
    monkeypatch.setenv("DG_LCA_TPT", tpt)
    for N in (4, 8, 16):
        w = W.lca(n_trials=30000, N=N)
        a = _lca(ctx, w["I"], w["seed"], 0)
        b = _lca(ctx, w["I"], w["seed"], 1)
        for u, v in zip(a, b):
            assert np.array_equal(u, v), N


@pytest.mark.parametrize("order", ["0", "1"])
def test_lca_hand_out_orders(ctx, orc, threads, monkeypatch, order):
    """Both hand-out orders (as given; longest expected first) at a size that
    is sorted (>= 4,096 trials) give the plain form's results bit for bit, and
    the oracle's on a sample of trials."""
    from paper_2110_15425_gb300 import workloads as W
    monkeypatch.setenv("DG_LCA_ORDER", order)
    for N in (4, 16):
        w = W.lca(n_trials=20000, N=N)
        a = _lca(ctx, w["I"], w["seed"], 0)
        b = _lca(ctx, w["I"], w["seed"], 1)
        for u, v in zip(a, b):
            assert np.array_equal(u, v), (N, order)
        ids = np.arange(0, 20000, 37, dtype=np.uint32)
        ref = orc.lca_run(w["I"], w["seed"], trial_ids=ids, threads=threads)
        compare_decisions(a[0][ids], a[1][ids], ref, f"lca N={N} order={order}")


def test_lca_ddm_mapping(ctx, orc, threads):
    """Sec. 4.4: LCA(N=1, leak 0, no competition, unit noise, two-sided, no
    rectification) decides like the DDM on the same draws."""
    n = 4000
    rng = np.random.default_rng(3)
    A = rng.uniform(0.1, 1.0, n).astype(np.float32)
    z = np.full(n, 1.25, np.float32)
    c, s, x = _lca(ctx, A.reshape(n, 1), 77, 0, leak=0.0, inhibition=0.0, sigma=1.0, dt=1e-3,
                   threshold=1.25, max_steps=10000, rectify=False, two_sided=True)
    ref = orc.ddm_run(A, z, 77, threads=threads)
    compare_decisions(c, s, ref, "lca as ddm")


def test_lca_full_size_sampled(ctx, orc, threads):
    from paper_2110_15425_gb300 import workloads as W
    for N in (4, 8, 16):
        w = W.lca(N=N)
        kw = dict(leak=w["leak"], inhibition=w["inhibition"], sigma=w["sigma"], dt=w["dt"],
                  threshold=w["threshold"], max_steps=w["max_steps"])
        c, s, x = _lca(ctx, w["I"], w["seed"], 0, **kw)
        ids = np.sort(np.random.default_rng(N).choice(w["I"].shape[0], 2048, replace=False))
        ref = orc.lca_run(w["I"], w["seed"], trial_ids=ids.astype(np.uint32), threads=threads, **kw)
        compare_decisions(c[ids], s[ids], ref, f"lca full N={N}")
        assert c.min() >= -1 and c.max() < N and s.min() >= 1 and s.max() <= w["max_steps"]


# ------------------------------------------------------------ small network ---

def _net(ctx, w, mode, n=None, trial_ids=None):
    import torch
    from paper_2110_15425_gb300 import binding as B
    n = w["n_trials"] if n is None else n
    model = B.compose_network(ctx, w["layers"], w["projections"], rate=w["rate"],
                              noise_sd=w["noise_sd"], stop_layer=w["stop_layer"],
                              stop_threshold=w["stop_threshold"], max_steps=w["max_steps"])
    try:
        kind, ss = B.dg_model_info(model)
        assert B.MODEL_KINDS[kind] == "transfer"
        cond = dev(w["cond_inputs"])
        choice = torch.zeros(max(n, 1), dtype=torch.int8, device="cuda")
        step = torch.zeros(max(n, 1), dtype=torch.int32, device="cuda")
        ys = torch.zeros(max(n, 1) * ss, dtype=torch.float32, device="cuda")
        B.dg_run(model, B.run_desc(n, w["seed"], cond_inputs=cond, n_cond=cond.shape[0],
                                   cond_block=w["cond_block"], mode=mode), choice, step, ys)
        return host(choice)[:n], host(step)[:n], host(ys)[:n * ss].reshape(n, ss)
    finally:
        B.dg_model_free(model)


def _net_ref(orc, w, n, threads):
    return orc.transfer_run(w["layers"], w["projections"], w["cond_inputs"], w["cond_block"],
                            w["seed"], rate=w["rate"], noise_sd=w["noise_sd"],
                            stop_layer=w["stop_layer"], stop_threshold=w["stop_threshold"],
                            max_steps=w["max_steps"], n_trials=n, threads=threads)


@pytest.mark.parametrize("weight_seed", [0, 4])
@pytest.mark.parametrize("mode", [0, 1])
def test_stroop_parity(ctx, orc, threads, weight_seed, mode):
    from paper_2110_15425_gb300 import workloads as W
    w = W.stroop_small(weight_seed=weight_seed)
    c, s, y = _net(ctx, w, mode)
    ref = _net_ref(orc, w, w["n_trials"], threads)
    compare_decisions(c, s, ref, f"stroop seed={weight_seed}")
    assert rel_err(y, ref["y"], 1e-2) < FLOAT_RTOL
    assert np.all((y > 0) & (y < 1))


def test_stroop_ragged_and_strong_weights(ctx, orc, threads):
    """A test-only network with strong weights so most trials stop, at a
    ragged trial count."""
    from paper_2110_15425_gb300 import workloads as W
    w = W.stroop_small(weight_seed=4, trials_per_condition=250, weight_range=6.0)
    n = 999
    for mode in (0, 1):
        c, s, y = _net(ctx, w, mode, n=n)
        ref = _net_ref(orc, w, n, threads)
        compare_decisions(c, s, ref, "strong")
        assert rel_err(y, ref["y"], 1e-2) < FLOAT_RTOL
    assert (ref["choice"] >= 0).mean() > 0.2


def test_network_with_feedback(ctx, orc, threads):
    """Recurrent edges (response -> hidden) are read from the previous step."""
    rng = np.random.default_rng(9)
    layers = [dict(size=3, input=True), dict(size=4, bias=-1.0), dict(size=3, bias=0.0)]
    projections = [(0, 1, rng.uniform(-3, 3, (4, 3)).astype(np.float32)),
                   (1, 2, rng.uniform(-3, 3, (3, 4)).astype(np.float32)),
                   (2, 1, rng.uniform(-2, 2, (4, 3)).astype(np.float32)),
                   (2, 2, rng.uniform(-1, 1, (3, 3)).astype(np.float32))]
    cond = rng.uniform(0, 1, (5, 3)).astype(np.float32)
    w = dict(layers=layers, projections=projections, cond_inputs=cond, cond_block=7,
             n_trials=700, rate=0.2, noise_sd=0.05, stop_layer=2, stop_threshold=0.3,
             max_steps=300, seed=31)
    c, s, y = _net(ctx, w, 0)
    ref = _net_ref(orc, w, 700, threads)
    compare_decisions(c, s, ref, "feedback")
    assert rel_err(y, ref["y"], 1e-2) < FLOAT_RTOL


def _random_net(seed, sizes, n_in=3, dup=False):
    """A layered network with an input layer, logistic layers of the given
    sizes, feed-forward and recurrent edges (and, with dup, a second
    projection between the same layers, whose weights the library adds)."""
    rng = np.random.default_rng(seed)
    layers = [dict(size=n_in, input=True)] + [
        dict(size=s, bias=float(rng.uniform(-1, 1)), gain=float(rng.uniform(0.5, 2)))
        for s in sizes]
    projections = [(0, 1, rng.uniform(-2, 2, (sizes[0], n_in)).astype(np.float32))]
    for i in range(1, len(sizes)):
        projections.append((i, i + 1, rng.uniform(-3, 3, (sizes[i], sizes[i - 1])).astype(np.float32)))
    last = len(sizes)
    projections.append((last, 1, rng.uniform(-1, 1, (sizes[0], sizes[-1])).astype(np.float32)))
    projections.append((last, last, rng.uniform(-1, 1, (sizes[-1], sizes[-1])).astype(np.float32)))
    if dup:
        projections.append((1, last if last > 1 else 1,
                            rng.uniform(-1, 1, (sizes[-1], sizes[0])).astype(np.float32)))
    cond = rng.uniform(0, 1, (5, n_in)).astype(np.float32)
    return dict(layers=layers, projections=projections, cond_inputs=cond, cond_block=3,
                n_trials=1500, rate=0.2, noise_sd=0.05, stop_layer=last, stop_threshold=0.25,
                max_steps=400, seed=seed + 1)


NETS = [(11, [2], False), (12, [1, 2], True), (13, [3], False), (14, [3, 2], False),
        (15, [4, 3], True), (16, [2, 2, 4], False), (17, [4, 4], True), (18, [1, 3], False)]


@pytest.mark.parametrize("seed,sizes,dup", NETS)
def test_net_lane_form_equals_group_form_and_oracle(ctx, orc, threads, monkeypatch, seed, sizes,
                                                    dup):
    """Networks of 2 to 8 logistic units: the one-lane-per-trial form gives the
    lane-group form's results bit for bit (outputs included) and the oracle's
    decisions."""
    w = _random_net(seed, sizes, dup=dup)
    a = _net(ctx, w, 0)
    monkeypatch.setenv("DG_NET_LANE", "0")
    b = _net(ctx, w, 0)
    for u, v in zip(a, b):
        assert np.array_equal(u.view(np.uint8), v.view(np.uint8)), (seed, sizes)
    ref = _net_ref(orc, w, w["n_trials"], threads)
    compare_decisions(a[0], a[1], ref, f"lane form {sizes}")
    assert rel_err(a[2], ref["y"], 1e-2) < FLOAT_RTOL


def test_stroop_lane_form_equals_group_form(ctx, monkeypatch):
    from paper_2110_15425_gb300 import workloads as W
    for ws in (0, 4):
        w = W.stroop_small(weight_seed=ws)
        a = _net(ctx, w, 0)
        monkeypatch.setenv("DG_NET_LANE", "0")
        b = _net(ctx, w, 0)
        monkeypatch.delenv("DG_NET_LANE")
        c = _net(ctx, w, 1)
        for u, v, x in zip(a, b, c):
            assert np.array_equal(u.view(np.uint8), v.view(np.uint8))
            assert np.array_equal(u.view(np.uint8), x.view(np.uint8))
