"""Pins of the oracle's joint move of a pair of events (§MH moves, "Joint
Events Move"; §Chromatic MH with Dynamic Coloring on why pairs cut by a fixed
boundary need the shifting partition).

* Its acceptance ratio equals the brute-force change of the full log-density
  (prior + likelihood summed from scratch over every station and sample): the
  proposal is symmetric, so nothing else may enter it.  Both readings.
* Geometry: stations on the perpendicular bisector of two events cannot tell
  the exchange of their locations apart, so the exchange is priced exactly
  0; a station off the bisector sees it.
* The sampler's exchange keeps each event's time and magnitude: on a world
  whose stations all lie on the bisector, every exchange the chain proposes
  is priced exactly 0 and the two locations are only ever permuted.
* A planted mistake (mutant 7: the joint move drops the prior ratio) shows
  in a prior-only chain as magnitudes drifting off the Exp(1) law.
* The pair the paper draws: two events whose assignment of origin times to
  locations is wrong.  Starting from it, dynamic colouring with joint moves
  reaches the true assignment; a fixed boundary between the two locations
  keeps the joint move from firing.
"""
import math

import numpy as np
import pytest

import worldgen
from test_oracle_sampler import _prior_only_chain


@pytest.mark.parametrize("likelihood", ["variance", "mean"])
@pytest.mark.parametrize("seed", [1, 2])
def test_pair_ratio_matches_full_difference(orc, seed, likelihood):
    rng = np.random.default_rng(seed)
    p = worldgen.ModelParams(W=300.0, T=300.0, Lambda=8.0, f_hz=2.0, t_s=60.0, tau=10.0,
                             likelihood=likelihood)
    st = worldgen.jittered_grid_stations(3, p.W, seed)
    w = worldgen.make_world(p, st, seed)
    o = orc.World(w)
    ev = w.events.copy()
    assert len(ev) >= 3
    n_tried = 0
    for trial in range(16):
        i, j = rng.choice(len(ev), size=2, replace=False)
        c1, c2 = ev[i].copy(), ev[j].copy()
        if trial % 2 == 0:                      # exchange of locations
            c1[:2], c2[:2] = ev[j][:2], ev[i][:2]
        else:                                   # one common offset
            off = rng.normal(0, [5.0, 5.0, 2.0, 0.1])
            c1, c2 = c1 + off, c2 + off
        la, ok = o.log_alpha_pair(0.0, 0.0, -1, ev, i, j, c1, c2)
        new = ev.copy()
        new[i], new[j] = c1, c2
        inside = all(0 <= c[0] < p.W and 0 <= c[1] < p.W and 0 <= c[2] < p.T and c[3] >= 2 for c in (c1, c2))
        assert ok == inside
        if not ok:
            continue
        full = o.log_density(new) - o.log_density(ev)
        assert la == pytest.approx(full, rel=1e-9, abs=1e-7)
        n_tried += 1
        ev = new
    assert n_tried >= 10


def _bisector_world(likelihood, off_axis=False):
    p = worldgen.ModelParams(W=300.0, T=200.0, Lambda=2.0, f_hz=2.0, t_s=40.0, tau=8.0, R_max=200.0,
                             L=150.0, likelihood=likelihood)
    st = [[150.0, 60.0], [150.0, 150.0], [150.0, 260.0]]
    if off_axis:
        st.append([40.0, 120.0])
    truth = np.array([[100.0, 120.0, 30.0, 3.4], [200.0, 120.0, 50.0, 2.8]])
    return p, worldgen.make_world(p, np.array(st), seed=5, events=truth), truth


@pytest.mark.parametrize("likelihood", ["variance", "mean"])
def test_exchange_is_invisible_on_the_bisector(orc, likelihood):
    p, w, ev = _bisector_world(likelihood)
    o = orc.World(w)
    c1, c2 = ev[0].copy(), ev[1].copy()
    c1[:2], c2[:2] = ev[1][:2], ev[0][:2]
    la, ok = o.log_alpha_pair(0.0, 0.0, -1, ev, 0, 1, c1, c2)
    assert ok and la == 0.0
    # a station off the bisector tells the two assignments apart
    p, w, ev = _bisector_world(likelihood, off_axis=True)
    o = orc.World(w)
    la, ok = o.log_alpha_pair(0.0, 0.0, -1, ev, 0, 1, c1, c2)
    assert ok and abs(la) > 1.0
    assert la == pytest.approx(o.log_density(np.array([c1, c2])) - o.log_density(ev), rel=1e-9)


def test_sampler_exchange_permutes_locations_only(orc):
    """Joint moves only, no location steps (sig_xy = 0): exchanges must be
    priced exactly 0 on the bisector world and leave the two locations in
    place as a set; the common offsets move times and magnitudes."""
    p, w, ev = _bisector_world("variance")
    o = orc.World(w, p_birth=0.0, p_death=0.0, p_pair=1.0, sig_xy=0.0, sig_t=2.0, sig_m=0.05)
    out, ids, tr, _ = o.run_serial(ev, 400, trace_cap=400)
    assert np.all(tr["type"] == 3)
    zero = np.sum(tr["evaluated"].astype(bool) & (tr["dll"] == 0.0))
    # half the joint moves are exchanges (bit 36 of the pick word)
    assert 150 < zero < 250, zero
    locs = sorted(map(tuple, out[:, :2]))
    assert locs == [(100.0, 120.0), (200.0, 120.0)]
    # the accepted exchanges did permute them
    assert np.sum(tr["accepted"]) > zero // 2


def test_pair_prior_mutant_drifts_magnitudes(orc):
    """Mostly joint moves with wide magnitude steps: the oracle keeps the
    Exp(1) law, the mutant's unweighted steps push magnitudes up."""
    kw = dict(n_iter=1200, p_bd=0.1, sig_m=2.0)
    _, _, _, ms = _prior_only_chain(orc, "dynamic", 0.8, **kw)
    assert abs(ms.mean() - 1.0) < 0.12, ms.mean()
    _, _, _, ms = _prior_only_chain(orc, "dynamic", 0.8, mutant=7, **kw)
    assert ms.mean() > 1.8, ms.mean()   # measured 2.44


def _swapped_pair_world():
    """Two events 20 s and ~54 km apart across x = 150, eight stations on a
    ring around them: the true assignment of times and magnitudes to the two
    locations, and its exchange as the starting hypothesis."""
    p = worldgen.ModelParams(W=300.0, T=200.0, Lambda=2.0, f_hz=2.0, t_s=40.0, tau=8.0, R_max=200.0,
                             L=150.0, noise_var=1.0)
    ang = np.linspace(0.0, 2 * np.pi, 8, endpoint=False)
    st = np.stack([150.0 + 90.0 * np.cos(ang), 150.0 + 90.0 * np.sin(ang)], axis=1)
    truth = np.array([[125.0, 140.0, 40.0, 3.2], [175.0, 160.0, 60.0, 3.0]])
    w = worldgen.make_world(p, st, seed=9, events=truth)
    start = truth.copy()
    start[0, :2], start[1, :2] = truth[1, :2], truth[0, :2]
    return p, w, truth, start


def _reached(ev, truth, tol=8.0):
    if len(ev) < 2:
        return False
    for t in truth:
        d = np.hypot(ev[:, 0] - t[0], ev[:, 1] - t[1])
        k = int(np.argmin(d))
        if d[k] > tol or abs(ev[k, 2] - t[2]) > 2.0:
            return False
    return True


def test_dynamic_colouring_lets_the_pair_reach_its_true_mode(orc):
    p, w, truth, start = _swapped_pair_world()
    o0 = orc.World(w)
    assert o0.log_density(truth) > o0.log_density(start) + 1000.0   # measured 2141
    res = {}
    for name, p_pair, shift_mode in (("pairs, dynamic", 0.2, 1), ("pairs, static", 0.2, 0),
                                     ("no pairs, dynamic", 0.0, 1)):
        hits = 0
        for seed in range(8):
            o = orc.World(w, k_per_phase=16, seed=100 + seed, p_pair=p_pair, sig_xy=3.0, sig_t=1.0,
                          sig_m=0.05)
            # static boundary at x = 150 separates the two locations
            ev, ids, _, _ = o.run_chromatic(start, 40, shift_mode=shift_mode, sx=0.0, sy=0.0)
            hits += _reached(ev, truth)
        res[name] = hits
    assert res["pairs, dynamic"] >= 6, res   # measured 7 of 8, the others 0
    assert res["pairs, static"] <= 1, res
    assert res["no pairs, dynamic"] <= 1, res
