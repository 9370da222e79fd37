"""Pins for the oracle's drift-diffusion and leaky-competing-accumulator models.

DDM: Euler-Maruyama with discrete monitoring of the +-z barriers. For x0 = 0
the continuous process has P(upper) = 1 / (1 + exp(-2 A z / s^2)) and mean
decision time (z / A) tanh(A z / s^2). Checking the barrier only every dt
shifts it outward by beta s sqrt(dt), beta = -zeta(1/2)/sqrt(2 pi) ~ 0.5826
(Broadie, Glasserman & Kou 1997); the closed forms are evaluated at the
shifted barrier, and at dt = 1e-4 and 1e-5 on nine fixed points too, where
the shift is small.

LCA: the equivalence mapping of Sec. 4.4 (Fig. clones: LCA with zero rate and
offset, unit-normal noise is the DDM integrator), the noise-free fixed point,
the closed-form leak-only crossing step, rectification and exchangeability.
"""
import math

import numpy as np
import pytest

BETA = 0.5825971579390106  # -zeta(1/2) / sqrt(2 pi)


def _p_upper(A, z, s=1.0):
    return 1.0 / (1.0 + math.exp(-2.0 * A * z / s**2))


def _mean_dt(A, z, s=1.0):
    return (z / A) * math.tanh(A * z / s**2)


@pytest.mark.parametrize("dt,points,n", [
    (1e-3, [(0.2, 1.0), (0.5, 1.0), (1.0, 0.5), (0.5, 2.0), (1.0, 1.5)], 20000),
    (1e-4, [(0.5, 1.0), (1.0, 0.5), (0.3, 1.5)], 4000),
])
def test_ddm_closed_forms(orc, threads, dt, points, n):
    zscores = []
    for pi, (A, z) in enumerate(points):
        Aa = np.full(n, A, np.float32)
        zz = np.full(n, z, np.float32)
        # slowest decay rate of the survival probability; 25/lambda1 leaves
        # mass ~exp(-25) undecided
        lam1 = A * A / 2 + math.pi**2 / (8 * z * z)
        o = orc.ddm_run(Aa, zz, seed=1000 + pi, dt=dt, max_steps=int(25.0 / lam1 / dt),
                        threads=threads)
        assert np.all(o["choice"] >= 0), "survival mass must be negligible"
        Af, zf = float(np.float32(A)), float(np.float32(z))
        zeff = zf + BETA * math.sqrt(dt)
        p = _p_upper(Af, zeff)
        phat = (o["choice"] == 1).mean()
        zp = (phat - p) / math.sqrt(p * (1 - p) / n)
        t = o["step"] * dt
        zt = (t.mean() - _mean_dt(Af, zeff)) / (t.std() / math.sqrt(n))
        zscores.append((A, z, zp, zt))
        assert abs(zp) < 4.0, (A, z, phat, p)
        assert abs(zt) < 4.0, (A, z, t.mean(), _mean_dt(Af, zeff))
    # the unshifted barrier must be rejected at dt = 1e-3 for the mean DT: the
    # correction is visible, so the test can tell the barrier convention apart
    if dt == 1e-3:
        A, z = points[1]
        o = orc.ddm_run(np.full(n, A, np.float32), np.full(n, z, np.float32), seed=1001, dt=dt,
                        max_steps=25000, threads=threads)
        t = o["step"] * dt
        zt_raw = (t.mean() - _mean_dt(A, z)) / (t.std() / math.sqrt(n))
        assert zt_raw > 4.0


# Nine fixed (A, z) points spanning the workload's drift and bound ranges.
SMALL_DT_POINTS = [(A, z) for A in (0.4, 0.7, 1.0) for z in (0.5, 1.0, 1.5)]


@pytest.mark.parametrize("dt,n", [(1e-4, 2000), (1e-5, 1000)])
def test_ddm_closed_forms_small_dt(orc, threads, dt, n):
    """At small dt the barrier shift beta s sqrt(dt) shrinks (0.0058 at 1e-4,
    0.0018 at 1e-5) and the discrete walk approaches the continuous closed
    forms: P(upper) and mean DT on nine fixed points, each |z-score| < 4, and
    the pooled z-scores over the nine points < 4 as well."""
    sum_dev_p = sum_var_p = 0.0
    zts = []
    for pi, (A, z) in enumerate(SMALL_DT_POINTS):
        lam1 = A * A / 2 + math.pi**2 / (8 * z * z)
        o = orc.ddm_run(np.full(n, A, np.float32), np.full(n, z, np.float32), seed=5000 + pi,
                        dt=dt, max_steps=int(25.0 / lam1 / dt), threads=threads)
        assert np.all(o["choice"] >= 0), "survival mass must be negligible"
        Af, zf = float(np.float32(A)), float(np.float32(z))
        zeff = zf + BETA * math.sqrt(dt)
        p = _p_upper(Af, zeff)
        k = int((o["choice"] == 1).sum())
        zp = (k - n * p) / math.sqrt(n * p * (1 - p))
        assert abs(zp) < 4.0, (A, z, k / n, p)
        sum_dev_p += k - n * p
        sum_var_p += n * p * (1 - p)
        t = o["step"] * dt
        zt = (t.mean() - _mean_dt(Af, zeff)) / (t.std() / math.sqrt(n))
        assert abs(zt) < 4.0, (A, z, t.mean(), _mean_dt(Af, zeff))
        zts.append(zt)
    assert abs(sum_dev_p / math.sqrt(sum_var_p)) < 4.0
    assert abs(sum(zts) / math.sqrt(len(zts))) < 4.0


def test_ddm_noise_free_crossing(orc):
    """sigma = 0: x_k = k A dt, first k with x_k >= z."""
    A = np.array([0.3, 0.7, 0.45], np.float32)
    z = np.array([0.77, 1.33, 1.91], np.float32)
    o = orc.ddm_run(A, z, seed=0, dt=1e-3, sigma=0.0)
    for i in range(3):
        k = math.ceil(float(z[i]) / (float(A[i]) * 1e-3))
        assert o["step"][i] == k and o["choice"][i] == 1


def test_ddm_timeout_and_margin(orc):
    A = np.array([0.1], np.float32)
    z = np.array([2.0], np.float32)
    o = orc.ddm_run(A, z, seed=3, max_steps=5)
    assert o["choice"][0] == -1 and o["step"][0] == 5
    # margin: distance of |x| to z, minimised over the 5 steps
    x = 0.0
    eps = orc.normals(3, 0, 0, 0, 5)
    m = math.inf
    for j in range(5):
        x = x + (float(A[0]) * 1e-3 + math.sqrt(1e-3) * eps[j])
        m = min(m, abs(abs(x) - 2.0))
    assert math.isclose(o["margin"][0], m, rel_tol=1e-12)


def test_lca_ddm_equivalence(orc):
    """Sec. 4.4: LCA with leak 0, no competition, N(0,1) noise, no
    rectification and a two-sided bound is the DDM: identical steps, choices
    and states for the same draws."""
    n = 2000
    rng = np.random.default_rng(0)
    A = rng.uniform(0.1, 1.0, n).astype(np.float32)
    z = np.full(n, 1.25, np.float32)
    d = orc.ddm_run(A, z, seed=42, dt=1e-3, sigma=1.0, max_steps=10000)
    l = orc.lca_run(A.reshape(n, 1), seed=42, leak=0.0, inhibition=0.0, sigma=1.0, dt=1e-3,
                    threshold=1.25, max_steps=10000, rectify=False, two_sided=True)
    assert np.array_equal(d["choice"], l["choice"])
    assert np.array_equal(d["step"], l["step"])
    assert np.array_equal(d["x"], l["x"][:, 0])


def test_lca_fixed_point(orc):
    """Noise-free, leak > inhibition: x*_i = (I_i - beta S)/(k - beta) with
    S = sum I / (k - beta + N beta)."""
    I = np.array([[0.6, 0.7, 0.5, 0.65]], np.float32)
    k, b = 0.5, 0.1
    o = orc.lca_run(I, seed=0, leak=k, inhibition=b, sigma=0.0, dt=0.01, threshold=10.0,
                    max_steps=6000)
    Id = I[0].astype(np.float64)
    S = Id.sum() / (k - b + 4 * b)
    xs = (Id - b * S) / (k - b)
    assert np.all(xs > 0)
    assert o["choice"][0] == -1
    np.testing.assert_allclose(o["x"][0], xs, rtol=1e-9, atol=1e-12)


def test_lca_leak_only_crossing_step(orc):
    """N = 1, sigma = 0: x_n = (I/k)(1 - (1 - k dt)^n); first n with x_n >= 1 is
    ceil(ln(1 - k/I) / ln(1 - k dt))."""
    for I0, k in [(0.5, 0.2), (0.9, 0.5), (0.35, 0.1)]:
        o = orc.lca_run(np.array([[I0]], np.float32), seed=0, leak=k, inhibition=0.3, sigma=0.0,
                        dt=0.01, threshold=1.0, max_steps=3000)
        Id = float(np.float32(I0))
        nstar = math.log(1 - k / Id) / math.log(1 - k * 0.01)
        assert abs(nstar - round(nstar)) > 1e-3
        assert o["step"][0] == math.ceil(nstar) and o["choice"][0] == 0


def test_lca_rectification(orc):
    rng = np.random.default_rng(1)
    I = rng.uniform(0, 1, (200, 8)).astype(np.float32)
    r = orc.lca_run(I, seed=5, inhibition=2.0, max_steps=400)
    assert np.all(r["x"] >= 0.0)
    u = orc.lca_run(I, seed=5, inhibition=2.0, max_steps=400, rectify=False)
    assert np.any(u["x"] < 0.0)


def test_lca_exchangeability(orc):
    """Noise-free dynamics commute with a permutation of the inputs."""
    rng = np.random.default_rng(2)
    I = rng.uniform(0, 1, (50, 6)).astype(np.float32)
    perm = rng.permutation(6)
    a = orc.lca_run(I, seed=0, sigma=0.0)
    b = orc.lca_run(I[:, perm], seed=0, sigma=0.0)
    assert np.array_equal(a["step"], b["step"])
    # unit i of the permuted run is unit perm[i] of the original one
    assert np.array_equal(perm[b["choice"]], a["choice"])
    assert np.all(a["choice"] == np.argmax(I, axis=1))


def test_lca_noise_index(orc):
    """Unit i at step j (1-based) takes normal (j-1)*N + i: with zero inputs,
    no leak or competition, the first step is sigma sqrt(dt) eps, rectified."""
    N = 5
    o = orc.lca_run(np.zeros((1, N), np.float32), seed=8, leak=0.0, inhibition=0.0, sigma=1.0,
                    dt=0.01, threshold=100.0, max_steps=1, rectify=False)
    eps = orc.normals(8, 0, 0, 0, N)
    np.testing.assert_allclose(o["x"][0], 0.1 * eps, rtol=1e-15)


def test_ddm_run_offset_matches_trial_ids(orc):
    """A run starting at global id trial0 is the same computation as the
    id-indexed run over ids trial0 .. trial0 + n - 1."""
    import numpy as np
    rng = np.random.default_rng(3)
    A = rng.uniform(0.1, 1.0, 50).astype(np.float32)
    z = rng.uniform(0.5, 2.0, 50).astype(np.float32)
    a = orc.ddm_run_offset(A, z, 7, 20)
    Apad = np.concatenate([np.zeros(20, np.float32), A])
    zpad = np.concatenate([np.ones(20, np.float32), z])
    b = orc.ddm_run(Apad, zpad, 7, trial_ids=np.arange(20, 70, dtype=np.uint32))
    for k in ("choice", "step", "x"):
        assert np.array_equal(a[k], b[k])
