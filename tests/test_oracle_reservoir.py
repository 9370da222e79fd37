"""Pins of the oracle's reservoir tie-break (Sec. 3.3: when several parameter
choices reach the best value, one of them is picked at random with reservoir
sampling, Vitter's Algorithm R with a reservoir of one)."""
import numpy as np
import pytest
from scipy import stats


def _rank_form(orc, v, seed):
    """Restatement over the final tie set: ties t_1 < ... < t_m; t_k (k >= 2)
    is accepted when its Philox word w satisfies w k < 2^32; the choice is the
    last accepted tie (t_1 always accepts)."""
    v = np.asarray(v, np.float64)
    ties = np.flatnonzero(v == v.max())
    key = [seed & 0xFFFFFFFF, seed >> 32]
    choice = int(ties[0])
    for k, t in enumerate(ties, start=1):
        if k == 1:
            continue
        w = int(orc.philox([t & 0xFFFFFFFF, t >> 32, 0, 4], key)[0])
        if w * k < (1 << 32):
            choice = int(t)
    return choice, len(ties)


def test_no_ties_is_plain_argmax(orc):
    rng = np.random.default_rng(0)
    for n in (1, 2, 7, 1000):
        for s in range(5):
            v = rng.standard_normal(n)
            b, bv, g, k = orc.argmax_reservoir(v, 1234 + s)
            assert (b, bv, g) == orc.argmax(v)
            assert k == 1


def test_single_value_and_all_equal(orc):
    assert orc.argmax_reservoir(np.array([3.5]), 9) == (0, 3.5, 0.0, 1)
    v = np.full(50, -2.0)
    b, bv, g, k = orc.argmax_reservoir(v, 9)
    assert 0 <= b < 50 and bv == -2.0 and g == 0.0 and k == 50


@pytest.mark.parametrize("seed", [0, 1, 77, 2**40 + 3])
def test_matches_rank_restatement(orc, seed):
    """Planted ties, with earlier groups of equal values that a larger value
    later supersedes (the streaming pass must restart its count there)."""
    rng = np.random.default_rng(seed & 0xFFFF)
    for trial in range(40):
        n = int(rng.integers(2, 400))
        v = rng.integers(-3, 3, n).astype(np.float64)   # many equal values
        if trial % 3 == 0:
            v[rng.integers(0, n)] = 10.0                   # a unique maximum
        b, bv, g, k = orc.argmax_reservoir(v, seed)
        rb, m = _rank_form(orc, v, seed)
        assert (b, k) == (rb, m)
        assert v[b] == v.max() == bv
        assert (g == 0.0) == (m > 1)


@pytest.mark.parametrize("m", [2, 3, 7])
def test_uniform_over_ties(orc, m):
    """Each of m tied positions is chosen with probability 1/m over seeds."""
    n = 40
    pos = np.sort(np.random.default_rng(m).choice(n, m, replace=False))
    v = np.zeros(n)
    v[pos] = 1.0
    runs = 6000
    counts = np.zeros(m, np.int64)
    for s in range(runs):
        b = orc.argmax_reservoir(v, 1000 + s)[0]
        counts[np.searchsorted(pos, b)] += 1
        assert b in pos
    p = stats.chisquare(counts).pvalue
    assert p > 1e-4, (counts, p)
