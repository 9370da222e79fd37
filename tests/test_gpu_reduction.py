"""The per-candidate reduction of the grid search and the episodes, pinned on
its own: given FP32 values go through the kernels' lane-group layout,
compensated (TwoSum) FP32 pair sums and FP64 mean (dg_selftest_pair_sum), and
are compared with the exact mean of the same values (math.fsum is exact before
its one final rounding). The FP64 means feed the argmax (Sec. 3.6); a mistake
in the compensation would hide under the 1e-5 tolerance of the grid parity
tests, not here."""
import math

import numpy as np
import pytest

from gpu_util import dev, host

pytestmark = pytest.mark.gpu


def _exact_means(x, per):
    return np.array([math.fsum(float(v) for v in row) / per for row in x.reshape(-1, per)])


def _gpu_means(B, x, per, lanes):
    import torch
    n = x.size // per
    out = torch.zeros(n, dtype=torch.float64, device="cuda")
    B.dg_selftest_pair_sum(dev(x), n, per, lanes, out)
    return host(out)


def _plain_f32_means(x, per, lanes):
    """The same lane layout with plain FP32 additions (what the compensation
    protects against), for the discrimination check."""
    out = []
    for row in x.reshape(-1, per):
        parts = []
        for l in range(lanes):
            acc = np.float32(0)
            for v in row[l::lanes]:
                acc = np.float32(acc + v)
            parts.append(acc)
        tot = np.float32(0)
        for p in parts:
            tot = np.float32(tot + p)
        out.append(float(tot) / per)
    return np.array(out)


@pytest.mark.parametrize("lanes", [8, 32])
@pytest.mark.parametrize("per", [64, 37, 1024])
def test_pair_sum_matches_exact_mean(lanes, per):
    """Outcomes of the grid's range (-|P + act - Y| - cost, in [-30, 0]).
    Bound: each lane's pair keeps every rounding error of its additions, and
    only the sum of the errors is rounded again, so the mean is off by at most
    per^2 2^-48 of the mean magnitude."""
    from paper_2110_15425_gb300 import binding as B
    rng = np.random.default_rng(per * 100 + lanes)
    n = 4096 if per <= 64 else 256
    x = (-rng.uniform(0.0, 30.0, n * per)).astype(np.float32)
    got = _gpu_means(B, x, per, lanes)
    ref = _exact_means(x, per)
    mag = np.abs(x.astype(np.float64)).reshape(-1, per).mean(axis=1)
    err = np.abs(got - ref) / mag
    assert err.max() <= per * per * 2.0**-48, err.max()
    # the plain FP32 sum of the same values misses by far more
    plain = _plain_f32_means(x[:64 * per], per, lanes)
    assert (np.abs(plain - ref[:64]) / mag[:64]).max() > 1e3 * max(err.max(), 2.0**-60)


@pytest.mark.parametrize("lanes", [8, 32])
def test_pair_sum_recovers_cancelled_terms(lanes):
    """Large terms that cancel exactly, +-3e7 (FP32 spacing 2 there), around
    small ones: a plain FP32 sum drops the small terms, the compensated pair
    keeps them."""
    from paper_2110_15425_gb300 import binding as B
    rng = np.random.default_rng(lanes)
    per, n = 64, 512
    x = np.empty((n, per), np.float32)
    big = np.float32(3.0e7)
    for g in range(n):
        small = rng.uniform(0.0, 1.0, per // 2).astype(np.float32)
        signs = np.where(np.arange(per // 2) % 2 == 0, big, -big).astype(np.float32)
        x[g, 0::2] = signs
        x[g, 1::2] = small
    x = x.reshape(-1)
    got = _gpu_means(B, x, per, lanes)
    ref = _exact_means(x, per)
    assert np.abs(got - ref).max() <= 2.0**-20, np.abs(got - ref).max()
    plain = _plain_f32_means(x[:8 * per], per, lanes)
    assert np.abs(plain - ref[:8]).max() > 1e-3


def test_pair_sum_argument_errors():
    from paper_2110_15425_gb300 import binding as B
    import torch
    x = torch.zeros(64, dtype=torch.float32, device="cuda")
    out = torch.zeros(1, dtype=torch.float64, device="cuda")
    with pytest.raises(B.DGError) as e:
        B.dg_selftest_pair_sum(x, 1, 64, 16, out)
    assert e.value.status == B.DG_E_ARG
