"""A model composed from a weight seed alone (projections with NULL weights
and a range, Sec. 3.3 static parameters): the library's weights equal the
oracle's bit for bit, and the Stroop workload composed that way matches the
oracle fed the oracle's weights."""
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


@pytest.mark.parametrize("weight_seed,lo,hi", [(0, -2.5, 2.5), (123456789012, -6.0, 6.0)])
def test_seeded_stroop(ctx, orc, threads, weight_seed, lo, hi):
    import torch
    from paper_2110_15425_gb300 import binding as B
    from paper_2110_15425_gb300 import workloads as W
    w = W.stroop_small()
    sizes = [l["size"] for l in w["layers"]]
    seeded = [(s, r, (lo, hi)) for (s, r, _) in w["projections"]]
    m = B.compose_network(ctx, w["layers"], seeded, rate=w["rate"], noise_sd=w["noise_sd"],
                          stop_layer=w["stop_layer"], stop_threshold=w["stop_threshold"],
                          max_steps=w["max_steps"], weight_seed=weight_seed)
    try:
        proj = []
        for i, (s, r, _) in enumerate(w["projections"]):
            n = sizes[r] * sizes[s]
            got = B.dg_model_weights(m, i, n)
            ref = orc.weights(weight_seed, i, n, lo, hi)
            assert np.array_equal(got.view(np.uint32), ref.view(np.uint32)), i
            proj.append((s, r, ref.reshape(sizes[r], sizes[s])))
        n = w["n_trials"]
        c = torch.zeros(n, dtype=torch.int8, device="cuda")
        st = torch.zeros(n, dtype=torch.int32, device="cuda")
        y = torch.zeros(n * 2, dtype=torch.float32, device="cuda")
        B.dg_run(m, B.run_desc(n, w["seed"], cond_inputs=dev(w["cond_inputs"]), n_cond=4,
                               cond_block=w["cond_block"]), c, st, y)
        refr = orc.transfer_run(w["layers"], proj, w["cond_inputs"], w["cond_block"], w["seed"],
                                rate=w["rate"], noise_sd=w["noise_sd"],
                                stop_layer=w["stop_layer"], stop_threshold=w["stop_threshold"],
                                max_steps=w["max_steps"], n_trials=n, threads=threads)
        compare_decisions(host(c), host(st), refr, "seeded stroop")
        keep = refr["margin"] >= 1e-5
        assert rel_err(host(y).reshape(n, 2)[keep], refr["y"][keep], 1e-2) < FLOAT_RTOL
    finally:
        B.dg_model_free(m)


def test_seeded_weight_errors(ctx):
    from paper_2110_15425_gb300 import binding as B
    from paper_2110_15425_gb300 import workloads as W
    w = W.stroop_small()
    bad = [(s, r, (1.0, -1.0)) for (s, r, _) in w["projections"]]
    with pytest.raises(B.DGError) as e:
        B.compose_network(ctx, w["layers"], bad, weight_seed=1)
    assert e.value.status == B.DG_E_ARG
    m = B.compose_network(ctx, w["layers"], w["projections"])
    try:
        got = B.dg_model_weights(m, 0, 4)   # given weights are read back as given
        assert np.array_equal(got, np.asarray(w["projections"][0][2], np.float32).ravel())
        with pytest.raises(B.DGError):
            B.dg_model_weights(m, 0, 5)
        with pytest.raises(B.DGError):
            B.dg_model_weights(m, 99, 0)
    finally:
        B.dg_model_free(m)
