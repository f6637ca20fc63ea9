"""Pins of the oracle's latent arrival times and arrival-time move.

The paper's arrival of event i at station j is Gaussian around
t_i + d_ij / v (§Generative Model, Event Detections), and the sampler changes
one arrival by a Gaussian offset (§MH moves, "Arrival Time Move").  The
oracle keeps one latent offset delta_ij = a_ij - (t_i + d_ij / v) per
(event, reached station), with prior N(0, sig_a^2).

* The prior with offsets against scipy's Poisson / exponential / normal
  densities; the likelihood of an arrival shifted by delta against a
  hand-derived closed form (both readings).
* The arrival-time move's ratio equals the brute-force change of the full
  log-density (prior + likelihood summed from scratch): it is symmetric.
* A birth's ratio equals the full change less the offsets' prior density,
  which its proposal draws them from, and less its uniform proposal terms:
  the cancellation the sampler relies on.
* With signals that carry no information (amplitudes ~e^-10), chains with
  births, deaths, location, pair and arrival moves keep every offset
  N(0, sig_a^2); planted mistakes fail this: mutant 8 (the arrival move
  without its prior ratio) widens the offsets, mutant 9 (newly reached
  stations given offset 0 instead of a prior draw) piles them at 0.
* With informative signals, arrival moves started from zero offsets move
  toward the offsets the world was generated with.
"""
import math

import numpy as np
import pytest
from scipy import stats

import worldgen

SIG_A = 2.5


def _reach(p, ev, st):
    return np.hypot(ev[:, None, 0] - st[None, :, 0], ev[:, None, 1] - st[None, :, 1]) < p.R_max


def test_latent_prior_closed_form(orc):
    p = worldgen.ModelParams(W=300.0, T=400.0, Lambda=6.0, R_max=120.0, f_hz=1.0, t_s=20.0)
    st = worldgen.jittered_grid_stations(3, p.W, 4)
    w = worldgen.World(params=p, stations=st, signals=np.zeros((len(st), p.n_samples)),
                       events=np.zeros((0, 4)))
    o = orc.World(w, sig_a=SIG_A)
    rng = np.random.default_rng(3)
    ev = np.column_stack([rng.uniform(0, p.W, 5), rng.uniform(0, p.W, 5), rng.uniform(0, p.T, 5),
                          2.0 + rng.exponential(size=5)])
    off = rng.normal(0, 3.0, size=(5, len(st)))
    r = _reach(p, ev, st)
    assert 0 < r.sum() < r.size
    want = (stats.poisson.logpmf(5, p.Lambda) + math.lgamma(6) - 5 * math.log(p.W * p.W * p.T)
            + stats.expon.logpdf(ev[:, 3] - 2.0).sum() + stats.norm.logpdf(off[r], 0.0, SIG_A).sum())
    assert o.log_prior(ev, off) == pytest.approx(want, rel=1e-13)
    # entries of stations an event does not reach carry nothing
    off2 = off.copy()
    off2[~r] = 17.0
    assert o.log_prior(ev, off2) == o.log_prior(ev, off)
    # without latent arrivals the offsets are not part of the model
    o0 = orc.World(w)
    assert o0.log_prior(ev, off) == o0.log_prior(ev)


@pytest.mark.parametrize("likelihood", ["variance", "mean"])
def test_shifted_arrival_closed_form(orc, likelihood):
    # one station at the origin, f = 1 Hz; an event at the station at t = 0
    # with offset delta = 1.5: arrival 1.5, window from sample 2 for t_s = 2 s,
    # envelope e^{-u} at u = 0.5, 1.5 with amplitude e (alpha m = 1)
    s = np.array([0.3, 1.0, -2.0, 0.7, 0.1])
    p = worldgen.ModelParams(W=10.0, T=5.0, Lambda=1.0, v=6.0, alpha=0.5, beta_att=0.0, tau=1.0, t_s=2.0,
                             f_hz=1.0, R_max=5.0, likelihood=likelihood)
    w = worldgen.World(params=p, stations=np.zeros((1, 2)), signals=s[None, :], events=np.zeros((0, 4)))
    o = orc.World(w, sig_a=SIG_A)
    ev = np.array([[0.0, 0.0, 0.0, 2.0]])
    g = np.array([0.0, 0.0, math.e * math.exp(-0.5), math.e * math.exp(-1.5), 0.0])
    if likelihood == "variance":
        want = stats.norm.logpdf(s, 0.0, np.sqrt(1.0 + g ** 2)).sum()
    else:
        want = stats.norm.logpdf(s, g, 1.0).sum()
    assert o.log_likelihood(ev, np.array([[1.5]])) == pytest.approx(want, rel=1e-13)
    # offset 0 is the deterministic arrival
    assert o.log_likelihood(ev, np.array([[0.0]])) == orc.World(w).log_likelihood(ev)


def _informative_world(seed, likelihood="variance", sig_a=SIG_A):
    p = worldgen.ModelParams(W=300.0, T=300.0, Lambda=8.0, f_hz=2.0, t_s=60.0, tau=10.0, R_max=120.0,
                             likelihood=likelihood)
    st = worldgen.jittered_grid_stations(3, p.W, seed)
    return worldgen.make_world(p, st, seed, sig_a=sig_a)


@pytest.mark.parametrize("likelihood", ["variance", "mean"])
def test_arrival_move_ratio_matches_full_difference(orc, likelihood):
    w = _informative_world(2, likelihood)
    p = w.params
    o = orc.World(w, sig_a=SIG_A)
    ev, off = w.events.copy(), w.offsets.copy()
    r = _reach(p, ev, w.stations)
    rng = np.random.default_rng(5)
    pairs = np.argwhere(r)
    assert len(pairs) >= 8
    for i, j in pairs[rng.choice(len(pairs), size=8, replace=False)]:
        new = off[i, j] + rng.normal(0, 2.0)
        la, ok = o.log_alpha_off(0.0, 0.0, -1, ev, off, 4, i, j, cand_off=new)
        assert ok
        off2 = off.copy()
        off2[i, j] = new
        full = o.log_density(ev, off2) - o.log_density(ev, off)
        assert la == pytest.approx(full, rel=1e-9, abs=1e-8)
        off = off2
    # a station the event does not reach has no offset to move
    i, j = np.argwhere(~r)[0]
    assert not o.log_alpha_off(0.0, 0.0, -1, ev, off, 4, i, j, cand_off=1.0)[1]


def test_birth_and_move_ratios_cancel_the_offset_prior(orc):
    w = _informative_world(3)
    p = w.params
    o = orc.World(w, sig_a=SIG_A, p_birth=0.25, p_death=0.25)
    ev, off = w.events.copy(), w.offsets.copy()
    n = len(ev)
    rng = np.random.default_rng(8)
    c = np.array([140.0, 150.0, 120.0, 3.1])
    rc = _reach(p, c[None, :], w.stations)[0]
    c_off = np.where(rc, rng.normal(0, SIG_A, len(w.stations)), 0.0)
    la, ok = o.log_alpha_off(0.0, 0.0, -1, ev, off, 0, cand=c, cand_off=c_off)
    assert ok and rc.sum() >= 2
    full = o.log_density(np.vstack([ev, c]), np.vstack([off, c_off])) - o.log_density(ev, off)
    # births draw the offsets from their prior: their density leaves the ratio
    # with the uniform proposal of (x, y, t) and the Exp(1) magnitude
    want = (full - stats.norm.logpdf(c_off[rc], 0.0, SIG_A).sum() + math.log(p.W * p.W * p.T) + (c[3] - 2.0)
            + math.log(0.25 / 0.25) - math.log(n + 1))
    assert la == pytest.approx(want, rel=1e-9, abs=1e-8)
    # a location move that keeps the reached set carries the offsets along:
    # symmetric, the ratio is the full change
    i = int(np.argmax(_reach(p, ev, w.stations).sum(axis=1)))
    mv = ev[i] + np.array([0.5, -0.5, 0.3, 0.01])
    assert np.array_equal(_reach(p, mv[None, :], w.stations)[0], _reach(p, ev[i:i + 1], w.stations)[0])
    la, ok = o.log_alpha_off(0.0, 0.0, -1, ev, off, 2, i, cand=mv, cand_off=off[i])
    new = ev.copy()
    new[i] = mv
    assert ok and la == pytest.approx(o.log_density(new, off) - o.log_density(ev, off), rel=1e-9, abs=1e-8)


def _silent_chain(orc, mutant=0, n_iter=900):
    """Stations whose signals carry nothing (amplitude e^{-5 m} <= e^{-10}):
    the posterior of every offset is its prior."""
    p = worldgen.ModelParams(W=200.0, T=100.0, Lambda=12.0, R_max=50.0, L=100.0, alpha=-5.0, beta_att=0.0,
                             f_hz=1.0, t_s=20.0, tau=5.0)
    st = worldgen.jittered_grid_stations(4, p.W, 6)
    w = worldgen.make_world(p, st, 6, events=np.zeros((0, 4)))
    o = orc.World(w, p_birth=0.2, p_death=0.2, p_pair=0.1, p_arr=0.3, sig_a=SIG_A, sig_da=SIG_A,
                  sig_xy=20.0, sig_t=5.0, sig_m=0.3, k_per_phase=8, seed=13, mutant=mutant)
    ev, ids, off = np.zeros((0, 4)), None, None
    samples, counts = [], []
    for it in range(n_iter):
        ev, ids, _, _ = o.run_chromatic(ev, 1, ids=ids, sweep0=it, off=off)
        off = o.last_offsets
        counts.append(len(ev))
        if it >= 100 and it % 4 == 0 and len(ev):
            r = _reach(p, ev, st)
            samples.extend(off[r])
            assert np.all(off[~r] == 0.0)
    return np.array(samples), np.array(counts), p


def test_offsets_keep_their_prior_without_information(orc):
    d, counts, p = _silent_chain(orc)
    assert len(d) > 3000
    assert abs(d.mean()) < 0.15 * SIG_A, d.mean()
    assert abs(d.var() / SIG_A ** 2 - 1.0) < 0.12, d.var() / SIG_A ** 2
    assert abs(np.mean(np.abs(d) < SIG_A) - 0.6827) < 0.04
    assert abs(counts[100:].mean() - p.Lambda) < 1.5


def test_offset_mutants_leave_the_prior(orc):
    d, _, _ = _silent_chain(orc, mutant=8, n_iter=500)
    assert d.var() / SIG_A ** 2 > 1.5, d.var()
    d, _, _ = _silent_chain(orc, mutant=9, n_iter=500)
    assert np.mean(np.abs(d) < 0.05 * SIG_A) > 0.2


def test_arrival_moves_recover_generated_offsets(orc):
    """Arrival moves only (sig_a = 4 s, 0.5 s samples), from the true events
    with every offset at 0: the chain's offsets end near the ones the signals
    were generated with, the strong arrivals within a second (one of them
    14 s away from the start)."""
    w = _informative_world(7, sig_a=4.0)
    p = w.params
    r = _reach(p, w.events, w.stations)
    d = np.hypot(w.events[:, None, 0] - w.stations[None, :, 0], w.events[:, None, 1] - w.stations[None, :, 1])
    strong = r & (np.exp(2.0 * (p.alpha * w.events[:, 3][:, None] - p.beta_att * d)) > 300.0)
    o = orc.World(w, p_birth=0.0, p_death=0.0, p_arr=1.0, sig_a=4.0, sig_da=1.0, k_per_phase=32, seed=3)
    ev, ids = w.events.copy(), None
    off = np.zeros_like(w.offsets)
    for it in range(60):
        ev, ids, _, _ = o.run_serial(ev, 200, ids=ids, step0=it * 200, off=off)
        off = o.last_offsets
    assert np.array_equal(ev, w.events)
    err = np.abs(off - w.offsets)
    # measured: median error 0.3 s against a median |offset| of 1.0 s
    assert np.median(err[r]) < 0.5 * np.median(np.abs(w.offsets[r]))
    assert strong.sum() >= 4 and err[strong].max() < 1.0, err[strong]
    assert np.abs(w.offsets[strong]).max() > 10.0


def test_world_rejects_reach_sets_beyond_the_oracle_bound(orc):
    p = worldgen.ModelParams(W=100.0, T=10.0, Lambda=1.0, R_max=50.0, f_hz=1.0, t_s=2.0)
    st = worldgen.jittered_grid_stations(12, p.W, 1)   # 144 stations within 2 R_max of each other
    w = worldgen.World(params=p, stations=st, signals=np.zeros((len(st), p.n_samples)), events=np.zeros((0, 4)))
    orc.World(w)   # fine without latent arrivals
    with pytest.raises(ValueError):
        orc.World(w, sig_a=1.0)


def test_scale_world_with_latent_offsets():
    """The bench's scale world at a small size with latent offsets: one
    offset per (event, station it reaches), zero elsewhere, of the stated
    scale, and the signals they shift differ from the deterministic ones."""
    w = worldgen.config_scale(seed=11, side_regions=6, T=36000.0, sig_a=2.0)
    w0 = worldgen.config_scale(seed=11, side_regions=6, T=36000.0)
    off = w.offsets
    assert off.shape == (len(w.events), len(w.stations))
    reach = _reach(w.params, w.events, w.stations)
    assert np.all(off[~reach] == 0.0) and np.count_nonzero(off[reach]) == reach.sum()
    assert reach.sum() > 50
    assert 1.5 < np.std(off[reach]) < 2.5   # +-25%: over 3 sd of the estimate at these counts
    assert np.array_equal(w.events, w0.events) and not np.array_equal(w.signals, w0.signals)
