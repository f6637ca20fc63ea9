"""Pins of the oracle's model arithmetic against things other than itself.

* Philox4x64-10 against numpy's independent implementation.
* Arrival times against the paper's worked two-event example (golden file).
* The log-likelihood against a hand-derived closed form evaluated with
  scipy's Gaussian log-density.
* The variance formula against Monte-Carlo draws of the generative story
  (worldgen), so a dropped square or a wrong envelope rate fails.
* The windowed log-likelihood change of a proposal against the brute-force
  difference of two full log-likelihoods.
* The prior against the Poisson / uniform / exponential densities.
* The same three likelihood pins for the additive-mean reading (arrivals add
  to the mean, the variance is the noise's).
"""
import math
import os

import numpy as np
import pytest
from scipy import stats

import worldgen

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _world(stations, signals, **kw):
    p = worldgen.ModelParams(**kw)
    st = np.asarray(stations, dtype=np.float64).reshape(-1, 2)
    sig = np.asarray(signals, dtype=np.float64)
    sig = sig.reshape(st.shape[0], sig.shape[-1] if sig.ndim else 0)
    return worldgen.World(params=p, stations=st, signals=sig, events=np.zeros((0, 4)))


def test_philox_matches_numpy(orc):
    rng = np.random.default_rng(5)
    for _ in range(50):
        key = rng.integers(0, 2**63, size=2, dtype=np.uint64)
        ctr = rng.integers(0, 2**63, size=4, dtype=np.uint64)
        ctr[0] = max(int(ctr[0]), 1)
        c0 = ctr.copy()
        c0[0] -= np.uint64(1)
        bg = np.random.Philox(key=key, counter=c0)
        ref = bg.random_raw(4)  # numpy increments the counter before each block
        assert np.array_equal(orc.philox4x64(ctr, key), ref)


def test_philox_counter_edge(orc):
    # all-ones counter wraps in numpy's increment: compare at counter (2^64-1, 0, 0, 0)
    bg = np.random.Philox(key=np.array([3, 9], dtype=np.uint64),
                          counter=np.array([2**64 - 2, 0, 0, 0], dtype=np.uint64))
    ref = bg.random_raw(4)
    assert np.array_equal(orc.philox4x64([2**64 - 1, 0, 0, 0], [3, 9]), ref)


def test_arrivals_match_paper_example(orc):
    rows = np.loadtxt(os.path.join(GOLDEN, "paper_fig1_arrivals.txt"))
    f = 2.0  # half-second samples: every arrival of the example falls on a sample
    stations = [(xs, 0.0) for xs in (0.0, 33.0, 66.0, 100.0)]
    ns = 1200
    w = _world(stations, np.zeros((4, ns)), W=200.0, T=ns / f, Lambda=1.0, v=2.0, alpha=0.0,
               beta_att=0.0, tau=5.0, t_s=10.0, f_hz=f, R_max=1000.0)
    o = orc.World(w)
    for t, x, xs, arrival in rows:
        j = [s[0] for s in stations].index(xs)
        V = o.variance(np.array([[x, 0.0, t, 2.0]]), j, 0, ns)
        k_first = int(np.nonzero(V > 1.0)[0][0])
        assert k_first == int(round(arrival * f))
        # amplitude 1 (alpha = beta_att = 0): the arrival sample adds exactly 1
        assert V[k_first] == pytest.approx(2.0, rel=1e-15)
        assert V[k_first + 1] == pytest.approx(1.0 + math.exp(-2.0 * (1.0 / f) / 5.0), rel=1e-14)
        # the window holds t_s * f samples
        assert np.count_nonzero(V > 1.0) == 20


def test_loglik_closed_form(orc):
    # one station at the origin, f = 1 Hz, three samples; one event at the
    # station at t = 0 with alpha*m = 1 and no attenuation: amplitude e, envelope
    # exp(-u) for u in {0, 1} (t_s = 2 s): variances 1 + e^2, 1 + 1, 1.
    s = np.array([0.0, 1.0, -2.0])
    w = _world([(0.0, 0.0)], s[None, :], W=10.0, T=3.0, Lambda=1.0, v=6.0, alpha=0.5,
               beta_att=0.0, tau=1.0, t_s=2.0, f_hz=1.0, R_max=5.0)
    o = orc.World(w)
    ev = np.array([[0.0, 0.0, 0.0, 2.0]])
    V = np.array([1.0 + math.e**2, 2.0, 1.0])
    assert np.allclose(o.variance(ev, 0, 0, 3), V, rtol=1e-15, atol=0)
    want = stats.norm.logpdf(s, 0.0, np.sqrt(V)).sum()
    assert o.log_likelihood(ev) == pytest.approx(want, rel=1e-14)
    # empty world: noise only
    assert o.log_likelihood(np.zeros((0, 4))) == pytest.approx(stats.norm.logpdf(s).sum(), rel=1e-14)
    # an event just beyond R_max adds nothing (footprint test d < R_max)
    far = np.array([[5.0, 0.0, 0.0, 2.0]])
    assert o.log_likelihood(far) == o.log_likelihood(np.zeros((0, 4)))


def test_log_prior_closed_form(orc):
    W, T, lam = 300.0, 500.0, 7.5
    w = _world(np.zeros((0, 2)), np.zeros((0, 10)), W=W, T=T, Lambda=lam)
    o = orc.World(w)
    ev = np.array([[10.0, 20.0, 30.0, 2.0], [299.0, 1.0, 499.0, 4.5], [150.0, 150.0, 0.0, 3.25]])
    n = len(ev)
    # Poisson count x n! orderings x uniform(x) uniform(y) uniform(t) x Exp(1) magnitudes
    want = (stats.poisson.logpmf(n, lam) + math.lgamma(n + 1) - n * math.log(W * W * T)
            + stats.expon.logpdf(ev[:, 3] - 2.0).sum())
    assert o.log_prior(ev) == pytest.approx(want, rel=1e-14)
    assert o.log_prior(np.zeros((0, 4))) == pytest.approx(stats.poisson.logpmf(0, lam), rel=1e-14)
    assert o.log_prior(np.array([[10.0, 20.0, 30.0, 1.999]])) == -math.inf
    assert o.log_prior(np.array([[300.0, 20.0, 30.0, 3.0]])) == -math.inf


def test_variance_matches_generative_draws(orc):
    # Monte-Carlo of the generative story: E[s^2] = V at every sample.
    p = worldgen.ModelParams(W=100.0, T=40.0, Lambda=1.0, tau=4.0, t_s=20.0, f_hz=5.0, R_max=50.0,
                             alpha=1.0, beta_att=0.02)
    st = np.array([[40.0, 50.0]])
    ev = np.array([[55.0, 45.0, 3.3, 2.7]])
    n_rep = 4000
    sq = np.zeros(p.n_samples)
    for r in range(n_rep):
        wr = worldgen.make_world(p, st, seed=10_000 + r, events=ev)
        sq += wr.signals[0] ** 2
    sq /= n_rep
    o = orc.World(worldgen.World(params=p, stations=st, signals=np.zeros((1, p.n_samples)),
                                 events=ev))
    V = o.variance(ev, 0, 0, p.n_samples)
    # s^2 / V has mean 1 and variance 2 per draw: 5 sigma per sample
    z = (sq / V - 1.0) / math.sqrt(2.0 / n_rep)
    assert np.max(np.abs(z)) < 5.5
    # and the window-averaged ratio is tight (catches a wrong decay rate)
    blocks = (sq / V).reshape(-1, 20).mean(axis=1)
    assert np.max(np.abs(blocks - 1.0)) < 6 * math.sqrt(2.0 / (n_rep * 20))


@pytest.mark.parametrize("seed", [1, 2, 3])
def test_delta_matches_full_difference(orc, seed):
    rng = np.random.default_rng(seed)
    p = worldgen.ModelParams(W=300.0, T=300.0, Lambda=8.0, f_hz=2.0, t_s=60.0, tau=10.0)
    st = worldgen.jittered_grid_stations(3, p.W, seed)
    w = worldgen.make_world(p, st, seed)
    o = orc.World(w)
    ev = w.events.copy()
    base = o.log_likelihood(ev)
    for trial in range(12):
        kind = trial % 3
        if kind == 0 or len(ev) == 0:   # birth
            cand = np.array([rng.uniform(0, p.W), rng.uniform(0, p.W), rng.uniform(0, p.T),
                             2 + rng.exponential()])
            new = np.vstack([ev, cand])
            d = o.delta_loglik(ev, -1, cand)
        elif kind == 1:                 # death
            i = int(rng.integers(len(ev)))
            new = np.delete(ev, i, axis=0)
            d = o.delta_loglik(ev, i, None)
        else:                           # move
            i = int(rng.integers(len(ev)))
            cand = ev[i] + rng.normal(0, [5.0, 5.0, 2.0, 0.1])
            new = ev.copy()
            new[i] = cand
            d = o.delta_loglik(ev, i, cand)
        full = o.log_likelihood(new) - base
        assert d == pytest.approx(full, rel=1e-9, abs=1e-7)
        ev, base = new, o.log_likelihood(new)


# ---- the additive-mean reading: arrivals add A g(u) to the mean of a sample
# whose variance is the noise's --------------------------------------------
def test_mean_reading_loglik_closed_form(orc):
    # the world of test_loglik_closed_form with noise variance 2: amplitude e
    # (alpha m = 1), envelope exp(-u) for u in {0, 1}: means e, 1, 0
    s = np.array([0.0, 1.0, -2.0])
    w = _world([(0.0, 0.0)], s[None, :], W=10.0, T=3.0, Lambda=1.0, v=6.0, alpha=0.5,
               beta_att=0.0, tau=1.0, t_s=2.0, f_hz=1.0, R_max=5.0, noise_var=2.0, likelihood="mean")
    o = orc.World(w)
    ev = np.array([[0.0, 0.0, 0.0, 2.0]])
    mu = np.array([math.e, 1.0, 0.0])
    assert np.allclose(o.variance(ev, 0, 0, 3), mu, rtol=1e-15, atol=0)
    want = stats.norm.logpdf(s, mu, math.sqrt(2.0)).sum()
    assert o.log_likelihood(ev) == pytest.approx(want, rel=1e-14)
    assert o.log_likelihood(np.zeros((0, 4))) == pytest.approx(
        stats.norm.logpdf(s, 0.0, math.sqrt(2.0)).sum(), rel=1e-14)


def test_mean_reading_matches_generative_draws(orc):
    # E[s] = mu and Var[s] = noise at every sample of the generative story
    p = worldgen.ModelParams(W=100.0, T=40.0, Lambda=1.0, tau=4.0, t_s=20.0, f_hz=5.0, R_max=50.0,
                             alpha=1.0, beta_att=0.02, noise_var=1.5, likelihood="mean")
    st = np.array([[40.0, 50.0]])
    ev = np.array([[55.0, 45.0, 3.3, 2.7]])
    n_rep = 3000
    s1 = np.zeros(p.n_samples)
    s2 = np.zeros(p.n_samples)
    for r in range(n_rep):
        x = worldgen.make_world(p, st, seed=20_000 + r, events=ev).signals[0]
        s1 += x
        s2 += x * x
    mean = s1 / n_rep
    var = s2 / n_rep - mean ** 2
    o = orc.World(worldgen.World(params=p, stations=st, signals=np.zeros((1, p.n_samples)), events=ev))
    mu = o.variance(ev, 0, 0, p.n_samples)
    assert mu.max() > 5.0   # the event is visible
    z = (mean - mu) / math.sqrt(p.noise_var / n_rep)
    assert np.max(np.abs(z)) < 5.5
    assert np.max(np.abs(var / p.noise_var - 1.0)) < 6 * math.sqrt(2.0 / n_rep)


@pytest.mark.parametrize("seed", [4, 5])
def test_mean_reading_delta_matches_full_difference(orc, seed):
    rng = np.random.default_rng(seed)
    p = worldgen.ModelParams(W=300.0, T=300.0, Lambda=8.0, f_hz=2.0, t_s=60.0, tau=10.0, likelihood="mean")
    w = worldgen.make_world(p, worldgen.jittered_grid_stations(3, p.W, seed), seed)
    o = orc.World(w)
    ev = w.events.copy()
    base = o.log_likelihood(ev)
    for trial in range(9):
        kind = trial % 3
        if kind == 0 or len(ev) == 0:
            cand = np.array([rng.uniform(0, p.W), rng.uniform(0, p.W), rng.uniform(0, p.T), 2 + rng.exponential()])
            new, d = np.vstack([ev, cand]), o.delta_loglik(ev, -1, cand)
        elif kind == 1:
            i = int(rng.integers(len(ev)))
            new, d = np.delete(ev, i, axis=0), o.delta_loglik(ev, i, None)
        else:
            i = int(rng.integers(len(ev)))
            cand = ev[i] + rng.normal(0, [5.0, 5.0, 2.0, 0.1])
            new = ev.copy()
            new[i] = cand
            d = o.delta_loglik(ev, i, cand)
        assert d == pytest.approx(o.log_likelihood(new) - base, rel=1e-9, abs=1e-7)
        ev, base = new, o.log_likelihood(new)
