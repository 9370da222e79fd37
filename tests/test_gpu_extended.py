"""GPU parity of the Extended Stroop model (Sec. 5: DDM nodes for colour
naming and finger pointing on the Stroop network's response layer) against
the oracle, and the A/B equivalence of two graphs of the same model."""
import numpy as np
import pytest

from gpu_util import FLOAT_RTOL, MARGIN, dev, host, rel_err

# A node's drift comes from the network's FP32 outputs (about 1e-6 off the
# FP64 oracle's), and over up to 10,000 steps of dt = 1e-3 that moves its
# path by up to ~4e-5: node decisions are compared bit for bit where the
# oracle's path stays at least this far from the bound.
NODE_MARGIN = 1e-4

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    import torch
    from paper_2110_15425_gb300 import binding as B
    torch.cuda.init()
    c = B.dg_create(0)
    yield c
    B.dg_destroy(c)


def _nodes(w, W_=None, bias=None, bound=None):
    Wd = w["ddm_W"] if W_ is None else W_
    return [dict(W=Wd[q:q + 1], bias=w["ddm_bias"] if bias is None else bias, dt=w["ddm_dt"],
                 sigma=w["ddm_sigma"], bound=w["ddm_bound"] if bound is None else bound,
                 max_steps=w["ddm_max"]) for q in range(Wd.shape[0])]


def _run_model(ctx, model, w, n, mode):
    import torch
    from paper_2110_15425_gb300 import binding as B
    kind, ss = B.dg_model_info(model)
    cond = dev(w["cond_inputs"])
    choice = torch.zeros(n, dtype=torch.int8, device="cuda")
    step = torch.zeros(n, dtype=torch.int32, device="cuda")
    fs = torch.zeros(n * ss, dtype=torch.float32, device="cuda")
    B.dg_run(model, B.run_desc(n, w["seed"], cond_inputs=cond, n_cond=cond.shape[0],
                               cond_block=w["cond_block"], mode=mode), choice, step, fs)
    return host(choice), host(step), host(fs).reshape(n, ss)


def _gpu(ctx, w, n, mode, **kw):
    from paper_2110_15425_gb300 import binding as B
    model = B.compose_extended_stroop(ctx, w["layers"], w["projections"], _nodes(w, **kw),
                                      rate=w["rate"], noise_sd=w["noise_sd"],
                                      stop_layer=w["stop_layer"],
                                      stop_threshold=w["stop_threshold"], max_steps=w["max_steps"])
    try:
        return _run_model(ctx, model, w, n, mode)
    finally:
        B.dg_model_free(model)


def _ref(orc, w, n, threads, W_=None, bias=None, bound=None):
    Wd = w["ddm_W"] if W_ is None else W_
    q = Wd.shape[0]
    return orc.extended_run(
        w["layers"], w["projections"], w["cond_inputs"], w["cond_block"], w["seed"], Wd,
        [w["ddm_bias"] if bias is None else bias] * q, [w["ddm_dt"]] * q, [w["ddm_sigma"]] * q,
        [w["ddm_bound"] if bound is None else bound] * q, [w["ddm_max"]] * q, rate=w["rate"],
        noise_sd=w["noise_sd"], stop_layer=w["stop_layer"], stop_threshold=w["stop_threshold"],
        max_steps=w["max_steps"], n_trials=n, threads=threads)


def _compare(c, s, fs, ref, ss=2):
    q = ref["d_choice"].shape[1]
    clear = ref["s_margin"] >= MARGIN
    for k in range(q):
        clear &= ref["d_margin"][:, k] >= NODE_MARGIN
    assert clear.mean() > 0.95
    y = fs[:, :ss]
    assert rel_err(y[clear], ref["y"][clear], 1e-2) < FLOAT_RTOL
    for k in range(q):
        x, dc, dst = fs[:, ss + 3 * k], fs[:, ss + 3 * k + 1], fs[:, ss + 3 * k + 2]
        assert np.array_equal(dc[clear].astype(np.int8), ref["d_choice"][clear, k]), k
        assert np.array_equal(dst[clear].astype(np.int32), ref["d_step"][clear, k]), k
        assert rel_err(x[clear], ref["d_x"][clear, k], 1.0) < FLOAT_RTOL
    assert np.array_equal(c[clear], ref["choice"][clear])
    assert np.array_equal(s[clear], ref["step"][clear])


@pytest.mark.parametrize("weight_seed", [0, 4])
@pytest.mark.parametrize("mode", [0, 1])
def test_extended_parity(ctx, orc, threads, weight_seed, mode):
    from paper_2110_15425_gb300 import workloads as W
    w = W.extended_stroop(weight_seed=weight_seed)
    n = w["n_trials"]
    c, s, fs = _gpu(ctx, w, n, mode)
    _compare(c, s, fs, _ref(orc, w, n, threads))
    assert set(np.unique(c)) <= {-1, 0, 1, 2, 3}


def test_extended_ragged_and_strong(ctx, orc, threads):
    """Strong test-only network weights (most trials stop early), a ragged
    trial count, and bounds some nodes do not reach within 10,000 steps."""
    from paper_2110_15425_gb300 import workloads as W
    w = W.extended_stroop(weight_seed=4)
    w2 = W.stroop_small(weight_seed=4, trials_per_condition=250, weight_range=6.0)
    for k in ("layers", "projections", "cond_inputs", "cond_block"):
        w[k] = w2[k]
    for bound in (1.0, 3.0):
        for mode in (0, 1):
            c, s, fs = _gpu(ctx, w, 999, mode, bound=bound)
            _compare(c, s, fs, _ref(orc, w, 999, threads, bound=bound))


@pytest.mark.parametrize("lane", ["1", "0"])
def test_extended_batched_equals_plain_bitwise(ctx, monkeypatch, lane):
    """The batched form (one lane per trial, or a lane group per trial with
    DG_NET_LANE=0) gives the plain form's results bit for bit."""
    from paper_2110_15425_gb300 import workloads as W
    monkeypatch.setenv("DG_NET_LANE", lane)
    w = W.extended_stroop(weight_seed=4)
    a = _gpu(ctx, w, w["n_trials"], 0)
    b = _gpu(ctx, w, w["n_trials"], 1)
    for u, v in zip(a, b):
        assert np.array_equal(u.view(np.uint8), v.view(np.uint8))


def test_extended_a_equals_b(ctx):
    """Version A: two one-unit DDM mechanisms, one projection each. Version B:
    one two-unit DDM mechanism fed by two projections listed in reverse order
    whose weights add up to the same matrix. Both compose to the same layout
    and give identical bits."""
    from paper_2110_15425_gb300 import binding as B
    from paper_2110_15425_gb300 import workloads as W
    w = W.extended_stroop(weight_seed=4)
    n = w["n_trials"]
    a = _gpu(ctx, w, n, 0)
    ms, ps, keep = [], [], []
    for l in w["layers"]:
        if l.get("input", False):
            ms.append(B.mech(B.DG_INPUT, int(l["size"])))
        else:
            ms.append(B.mech(B.DG_TRANSFER_LOGISTIC, int(l["size"]), gain=float(l.get("gain", 1.0)),
                             bias=float(l.get("bias", 0.0)), rate=w["rate"], noise=w["noise_sd"]))
    for (s_, r_, Wp) in w["projections"]:
        keep.append(np.ascontiguousarray(Wp, np.float32))
        ps.append(B.proj(s_, r_, keep[-1]))
    ms.append(B.mech(B.DG_DDM, 2, bias=w["ddm_bias"], dt=w["ddm_dt"], noise=w["ddm_sigma"],
                     threshold=w["ddm_bound"], max_steps=w["ddm_max"]))
    half = np.ascontiguousarray(w["ddm_W"] * 0.5, np.float32)    # exact halves
    keep += [half, half.copy()]
    ps.insert(0, B.proj(w["stop_layer"], len(ms) - 1, keep[-1]))
    ps.append(B.proj(w["stop_layer"], len(ms) - 1, keep[-2]))
    model = B.dg_compose(ctx, ms, ps, B.stop(w["stop_layer"], w["max_steps"], w["stop_threshold"]))
    try:
        b = _run_model(ctx, model, w, n, 0)
    finally:
        B.dg_model_free(model)
    for u, v in zip(a, b):
        assert np.array_equal(u, v)


def test_extended_compose_errors(ctx):
    from paper_2110_15425_gb300 import binding as B
    from paper_2110_15425_gb300 import workloads as W
    w = W.extended_stroop(weight_seed=4)
    bad = [dict(n) for n in _nodes(w)]
    bad[0]["bound"] = 0.0
    with pytest.raises(B.DGError):
        B.compose_extended_stroop(ctx, w["layers"], w["projections"], bad)
    many = _nodes(w) * 5   # 10 DDM units
    with pytest.raises(B.DGError):
        B.compose_extended_stroop(ctx, w["layers"], w["projections"], many)
