"""Latent arrival times and the arrival-time move (§Generative Model, Event
Detections; §MH moves) in the float64 replay form against the CPU oracle,
through the C ABI.

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
