"""Latent arrival times and the arrival-time move (§Generative Model, Event
Detections; §MH moves) in the float64 replay form and the float32 form
against the CPU oracle, through the C ABI.

Worlds are generated with Gaussian arrival offsets; both sides start from the
same events and offsets (or the empty set) and run the same chain: every
step's type (4: the arrival-time move), validity, picks and accept decision
equal the oracle's, Δℓ and log α agree to 1e-9 relative, and the final
events and their offsets are the oracle's.  The running log-density (which
counts the offsets' prior) tracks the oracle's and a recomputation, and a
checkpoint carries the offsets.
"""
import numpy as np
import pytest

import worldgen
from gpu_helpers import TRACE_KEYS, assert_traces_match, lib

pytestmark = pytest.mark.gpu

SIG_A = 2.5
MIX = dict(p_pair=0.1, sig_a=SIG_A, p_arr=0.2, sig_da=1.0)


@pytest.fixture(scope="module")
def cm():
    return lib()


def _world(seed=5):
    p = worldgen.ModelParams(W=500.0, T=1200.0, Lambda=60.0)
    return worldgen.make_world(p, worldgen.jittered_grid_stations(5, p.W, seed), seed, sig_a=SIG_A)


def _gpu(cm, w, ev0, off0, sweeps, k=16, seed=11, shift_mode=1):
    params = cm.make_params(w.params, k_per_phase=k, seed=seed, dtype=cm.F64, **MIX)
    m = cm.create_model(ev0, w.stations, w.signals, params)
    if ev0 is not None and len(ev0):
        m.set_arrival_offsets(off0)
    m.partition_and_color(w.params.L, shift_mode=shift_mode, sx=37.0, sy=81.5)
    ncx = int(np.floor(w.params.W / w.params.L)) + 2
    m.set_trace(sweeps * ncx * ncx * k)
    m.run_sweeps(sweeps)
    ev, ids, logp, stats = m.read_state()
    off = m.read_arrival_offsets(len(w.stations))
    tr = np.sort(m.read_trace(), order=TRACE_KEYS)
    return m, ev, ids, off, logp, stats, tr


def _oracle(orc, w, ev0, off0, sweeps, k=16, seed=11, shift_mode=1):
    o = orc.World(w, k_per_phase=k, seed=seed, **MIX)
    ncx = int(np.floor(w.params.W / w.params.L)) + 2
    start = np.zeros((0, 4)) if ev0 is None else ev0
    ev, ids, tr, dlp = o.run_chromatic(start, sweeps, shift_mode=shift_mode, sx=37.0, sy=81.5,
                                       trace_cap=sweeps * ncx * ncx * k + 16, off=off0)
    return o, ev, ids, o.last_offsets, np.sort(tr, order=TRACE_KEYS), dlp


@pytest.mark.parametrize("init", ["empty", "truth"])
@pytest.mark.parametrize("shift_mode", [1, 0])
def test_replay_latent_arrivals_bit_exact(cm, orc, init, shift_mode):
    w = _world()
    ev0 = w.events if init == "truth" else None
    off0 = w.offsets if init == "truth" else None
    m, ev, ids, off, logp, stats, tr = _gpu(cm, w, ev0, off0, 6, shift_mode=shift_mode)
    o, oev, oids, ooff, otr, odlp = _oracle(orc, w, ev0, off0, 6, shift_mode=shift_mode)
    assert_traces_match(tr, otr)
    assert np.array_equal(ids, oids)
    assert np.array_equal(ev[:, :3], oev[:, :3])
    assert np.allclose(ev[:, 3], oev[:, 3], rtol=1e-14, atol=0)
    # offsets: drawn with the same rounding on both sides, stepped exactly
    assert off.shape == ooff.shape
    assert np.allclose(off, ooff, rtol=0, atol=1e-12)
    arr = tr["type"] == 4
    assert stats["arrival"] == [int(arr.sum()), int(tr["evaluated"][arr].sum()), int(tr["accepted"][arr].sum())]
    assert tr["accepted"][arr].sum() > 10
    lp0 = o.log_density(np.zeros((0, 4)) if ev0 is None else ev0, off0)
    assert logp == pytest.approx(lp0 + odlp, rel=1e-11)
    assert m.log_density() == pytest.approx(logp, rel=1e-10)
    m.destroy()


def test_set_offsets_gives_the_oracles_log_density(cm, orc):
    w = _world(seed=7)
    params = cm.make_params(w.params, k_per_phase=8, seed=3, dtype=cm.F64, **MIX)
    m = cm.create_model(w.events, w.stations, w.signals, params)
    o = orc.World(w, **MIX)
    lp_zero = m.log_density()
    assert lp_zero == pytest.approx(o.log_density(w.events, None), rel=1e-12)
    m.set_arrival_offsets(w.offsets)
    assert m.log_density() == pytest.approx(o.log_density(w.events, w.offsets), rel=1e-12)
    # the generated offsets explain the signals better than zeros
    assert o.log_likelihood(w.events, w.offsets) > o.log_likelihood(w.events, None)
    # read back unchanged before any sweep
    assert np.array_equal(m.read_arrival_offsets(len(w.stations)), w.offsets)
    m.destroy()


def test_checkpoint_carries_the_offsets(cm):
    w = _world(seed=9)
    params = cm.make_params(w.params, k_per_phase=8, seed=5, dtype=cm.F64, **MIX)
    m = cm.create_model(w.events, w.stations, w.signals, params)
    m.set_arrival_offsets(w.offsets)
    m.partition_and_color(w.params.L, shift_mode=1)
    m.run_sweeps(3)
    ck = m.checkpoint()
    m.run_sweeps(4)
    ev_a, ids_a, lp_a, _ = m.read_state()
    off_a = m.read_arrival_offsets(len(w.stations))
    m.restore(ck)
    m.run_sweeps(4)
    ev_b, ids_b, lp_b, _ = m.read_state()
    off_b = m.read_arrival_offsets(len(w.stations))
    assert np.array_equal(ids_a, ids_b) and np.array_equal(ev_a, ev_b) and np.array_equal(off_a, off_b)
    assert lp_a == lp_b
    m.destroy()


# ---- the float32 form -------------------------------------------------------
# Latent offsets are float64 in both forms; the float32 kernel prices with
# float32 terms (windows start at the float64 definition's sample, see the
# float32 parity tests), so its changes of the log-likelihood agree with the
# oracle's to the float32 tolerance and its chains track the oracle's
# log-density of the events and offsets they reach.

def _f32_world(seed):
    p = worldgen.ModelParams(W=1000.0, T=3600.0, Lambda=500.0)
    return worldgen.make_world(p, worldgen.jittered_grid_stations(10, p.W, seed), seed, np.float32, sig_a=SIG_A)


def _reach(w, ev):
    dx = ev[:, None, 0] - w.stations[None, :, 0]
    dy = ev[:, None, 1] - w.stations[None, :, 1]
    return np.sqrt(dx * dx + dy * dy) < w.params.R_max


def test_fp32_latent_arrivals_dry_run_match_oracle(cm, orc):
    """Commit off, from the ground truth and its offsets, every move type in
    the mix (births draw offsets, moves keep or draw them, the arrival-time
    move steps one): every step's type, validity and event count equal the
    oracle's, each float32 change of the log-likelihood is within 1e-4 (to
    max(|x|, 1)) of the oracle's, and the arrival-move counters equal the
    trace's."""
    import os
    w = _f32_world(71)
    k, sweeps = 32, 4
    params = cm.make_params(w.params, k_per_phase=k, seed=13, dtype=cm.F32, commit=False, **MIX)
    m = cm.create_model(w.events, w.stations, w.signals, params)
    m.set_arrival_offsets(w.offsets)
    m.partition_and_color(w.params.L, shift_mode=1)
    ncx = int(np.floor(w.params.W / w.params.L)) + 2
    m.set_trace(sweeps * ncx * ncx * k)
    m.run_sweeps(sweeps)
    ev, _, _, stats = m.read_state()
    tr = np.sort(m.read_trace(), order=TRACE_KEYS)
    o = orc.World(w, k_per_phase=k, seed=13, commit=False, **MIX)
    _, _, otr, _ = o.run_chromatic(w.events, sweeps, shift_mode=1, trace_cap=sweeps * ncx * ncx * k + 16,
                                   threads=min(16, os.cpu_count() or 1), off=w.offsets)
    otr = np.sort(otr, order=TRACE_KEYS)
    assert len(tr) == len(otr) > 0
    for key in ("sweep", "cell", "step", "type", "n_before", "evaluated"):
        assert np.array_equal(tr[key], otr[key]), key
    ev_ = otr["evaluated"] == 1
    err = np.abs(tr["dll"][ev_] - otr["dll"][ev_]) / np.maximum(np.abs(otr["dll"][ev_]), 1.0)
    arr = (otr["type"] == 4) & ev_
    print("dll: %d evaluated (%d arrival-time moves), max err %.3g" % (ev_.sum(), arr.sum(), err.max()))
    assert arr.sum() > 300 and ((otr["type"] == 3) & ev_).sum() > 100
    assert err.max() <= 1e-4, err.max()
    assert np.count_nonzero(tr["accepted"][ev_] != otr["accepted"][ev_]) <= max(2, err.size // 10000)
    t4 = tr["type"] == 4
    assert stats["arrival"] == [int(t4.sum()), int(tr["evaluated"][t4].sum()), int(tr["accepted"][t4].sum())]
    # nothing committed: the offsets read back (in the store's event order)
    # are the ones set
    off = m.read_arrival_offsets(len(w.stations))
    mine, theirs = np.lexsort((ev[:, 1], ev[:, 0])), np.lexsort((w.events[:, 1], w.events[:, 0]))
    assert np.array_equal(ev[mine], w.events[theirs])
    assert np.array_equal(off[mine], w.offsets[theirs])
    m.destroy()


@pytest.mark.parametrize("init", ["empty", "truth"])
def test_fp32_latent_arrivals_chain_tracks_oracle_log_density(cm, orc, init):
    """With commits: the running log-density (likelihood, event prior and the
    offsets' prior) equals the oracle's log-density of the final events and
    offsets, summed from scratch in float64, within 1e-7 of the magnitudes it
    summed (the start's log-density and the accepted changes: each change is
    priced from float32 terms, rounded at 2^-24 and evaluated by the SFU at
    2^-22, so its error is a few 1e-8 of the terms' sizes; from the empty set
    the first births change the log-density by up to ~1e9); the GPU's
    recomputation agrees with the oracle's to float32 rounding of the
    synthesis.  Every offset sits at a station its event reaches, and
    arrival-time moves were accepted."""
    w = _f32_world(72)
    ev0 = w.events if init == "truth" else None
    k, sweeps = 32, 20
    params = cm.make_params(w.params, k_per_phase=k, seed=15, dtype=cm.F32, **MIX)
    m = cm.create_model(ev0, w.stations, w.signals, params)
    if ev0 is not None:
        m.set_arrival_offsets(w.offsets)
    m.partition_and_color(w.params.L, shift_mode=1)
    ncx = int(np.floor(w.params.W / w.params.L)) + 2
    m.set_trace(sweeps * ncx * ncx * k)
    m.run_sweeps(sweeps)
    ev, ids, logp, stats = m.read_state()
    tr = m.read_trace()
    off = m.read_arrival_offsets(len(w.stations))
    assert stats["arrival"][2] > 20 and len(ev) > 10
    assert off.shape == (len(ev), len(w.stations))
    assert np.all(off[~_reach(w, ev)] == 0.0)
    assert np.count_nonzero(off) > 0.9 * _reach(w, ev).sum()
    o = orc.World(w, **MIX)
    lp0 = o.log_density(w.events, w.offsets) if ev0 is not None else o.log_density(np.zeros((0, 4)), None)
    acc = tr["accepted"] == 1
    scale = abs(lp0) + float(np.abs(tr["dll"][acc]).sum())
    want = o.log_density(ev, off)
    rec = m.log_density()
    print("running - oracle %.4f (%.3g of %.3e summed); recomputed - oracle %.4f"
          % (logp - want, abs(logp - want) / scale, scale, rec - want))
    assert abs(logp - want) <= 1e-7 * scale
    assert rec == pytest.approx(want, rel=1e-6)
    assert len(np.unique(ids)) == len(ids)
    m.destroy()


def test_fp32_offsets_give_the_oracles_log_density(cm, orc):
    """The float32 synthesis of V with offsets: the model's log-density of the
    ground truth with its offsets equals the oracle's to float32 rounding, and
    the offsets explain the signals better than zeros."""
    w = _f32_world(73)
    params = cm.make_params(w.params, k_per_phase=8, seed=3, dtype=cm.F32, **MIX)
    m = cm.create_model(w.events, w.stations, w.signals, params)
    o = orc.World(w, **MIX)
    lp_zero = m.log_density()
    m.set_arrival_offsets(w.offsets)
    lp = m.log_density()
    assert lp == pytest.approx(o.log_density(w.events, w.offsets), rel=1e-6)
    assert lp_zero == pytest.approx(o.log_density(w.events, None), rel=1e-6)
    assert lp > lp_zero
    m.destroy()


def test_fp32_latent_persistent_sweep_matches_colour_by_colour(cm):
    """The instantiation with latent offsets: one persistent launch per sweep
    gives the chain (events, offsets, trace, log-density) of the
    colour-by-colour schedule bit for bit."""
    w = _f32_world(74)
    runs = []
    for schedule in (0, 1):
        params = cm.make_params(w.params, k_per_phase=32, seed=17, dtype=cm.F32, schedule=schedule, **MIX)
        m = cm.create_model(w.events, w.stations, w.signals, params)
        m.set_arrival_offsets(w.offsets)
        m.partition_and_color(w.params.L, shift_mode=1)
        ncx = int(np.floor(w.params.W / w.params.L)) + 2
        m.set_trace(8 * ncx * ncx * 32)
        m.run_sweeps(8)
        ev, ids, logp, stats = m.read_state()
        runs.append((ev, ids, logp, np.sort(m.read_trace(), order=TRACE_KEYS), stats,
                     m.read_arrival_offsets(len(w.stations))))
        m.destroy()
    assert runs[0][4]["arrival"][2] > 10
    assert runs[0][4]["kernel_launches"] < runs[1][4]["kernel_launches"]
    assert np.array_equal(runs[0][0], runs[1][0]) and np.array_equal(runs[0][1], runs[1][1])
    assert runs[0][2] == runs[1][2]
    assert np.array_equal(runs[0][3], runs[1][3])
    assert np.array_equal(runs[0][5], runs[1][5])


def test_batch_refuses_latent_offsets(cm):
    """A batch runs the kernel without latent offsets: a model with them is
    refused."""
    w = _f32_world(75)
    m = cm.create_model(w.events, w.stations, w.signals,
                        cm.make_params(w.params, k_per_phase=16, seed=3, dtype=cm.F32, **MIX))
    m.partition_and_color(w.params.L, 1)
    with pytest.raises(cm.ChromhError):
        cm.create_batch([m])
    m.destroy()
