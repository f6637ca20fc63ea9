"""The joint move of a pair of events (§MH moves, "Joint Events Move") in the
float64 replay form and in the float32 form against the CPU oracle, through
the C ABI.

With p_pair > 0 every step's type (3 for the joint move), validity, picks and
accept decision equal the oracle's, the log-likelihood changes and ratios
agree to 1e-9 relative, and the final event sets are identical.  The
swapped-pair world (two events with their locations exchanged, across the
boundary a static partition would keep) reaches its true mode on the GPU
under dynamic colouring, as the oracle's chains do.
"""
import os

import numpy as np
import pytest

import worldgen
from gpu_helpers import assert_traces_match, lib, run_gpu, run_oracle, small_world

pytestmark = pytest.mark.gpu

PAIR = 0.2


@pytest.fixture(scope="module")
def cm():
    return lib()


def _pair_counts(tr):
    p = tr["type"] == 3
    return [int(p.sum()), int(tr["evaluated"][p].sum()), int(tr["accepted"][p].sum())]


@pytest.mark.parametrize("init", ["empty", "truth"])
@pytest.mark.parametrize("shift_mode", [1, 0])
def test_replay_pairs_bit_exact(cm, orc, init, shift_mode):
    w = small_world()
    ev0 = w.events if init == "truth" else None
    sweeps = 6
    m, ev, ids, logp, stats, tr = run_gpu(cm, w, sweeps=sweeps, events=ev0, shift_mode=shift_mode,
                                          sx=37.0, sy=81.5, p_pair=PAIR)
    o, oev, oids, otr, odlp = run_oracle(orc, w, sweeps=sweeps, events=ev0, shift_mode=shift_mode,
                                         sx=37.0, sy=81.5, p_pair=PAIR)
    assert_traces_match(tr, otr)
    assert np.array_equal(ids, oids)
    assert np.array_equal(ev[:, :3], oev[:, :3])
    assert np.allclose(ev[:, 3], oev[:, 3], rtol=1e-14, atol=0)
    counts = _pair_counts(tr)
    assert stats["pair"] == counts
    assert counts[0] > 0.1 * len(tr)
    if init == "truth":
        assert counts[1] > 50
    lp0 = o.log_density(w.events if init == "truth" else np.zeros((0, 4)))
    assert logp == pytest.approx(lp0 + odlp, rel=1e-11)
    assert m.log_density() == pytest.approx(logp, rel=1e-10)
    m.destroy()


def test_replay_pairs_config_world(cm, orc):
    """The 1000 x 1000 km, 100-station, 36000-sample world of the replay
    workload, from the ground truth, with joint moves on."""
    w = worldgen.config_replay(seed=1000)
    threads = min(16, os.cpu_count() or 1)
    m, ev, ids, logp, stats, tr = run_gpu(cm, w, sweeps=3, k=32, seed=7, events=w.events, p_pair=PAIR)
    o, oev, oids, otr, odlp = run_oracle(orc, w, sweeps=3, k=32, seed=7, events=w.events, threads=threads,
                                         p_pair=PAIR)
    assert_traces_match(tr, otr)
    assert np.array_equal(ids, oids)
    assert np.array_equal(ev[:, :3], oev[:, :3])
    assert _pair_counts(tr)[1] > 100
    m.destroy()


def _swapped_pair_world():
    p = worldgen.ModelParams(W=300.0, T=200.0, Lambda=2.0, f_hz=2.0, t_s=40.0, tau=8.0, R_max=200.0,
                             L=150.0, noise_var=1.0)
    ang = np.linspace(0.0, 2 * np.pi, 8, endpoint=False)
    st = np.stack([150.0 + 90.0 * np.cos(ang), 150.0 + 90.0 * np.sin(ang)], axis=1)
    truth = np.array([[125.0, 140.0, 40.0, 3.2], [175.0, 160.0, 60.0, 3.0]])
    w = worldgen.make_world(p, st, seed=9, events=truth)
    start = truth.copy()
    start[0, :2], start[1, :2] = truth[1, :2], truth[0, :2]
    return w, truth, start


def _reached(ev, truth, tol=8.0):
    if len(ev) < 2:
        return False
    for t in truth:
        d = np.hypot(ev[:, 0] - t[0], ev[:, 1] - t[1])
        k = int(np.argmin(d))
        if d[k] > tol or abs(ev[k, 2] - t[2]) > 2.0:
            return False
    return True


def test_swapped_pair_reaches_its_true_mode(cm, orc):
    w, truth, start = _swapped_pair_world()
    steps = dict(sig_xy=3.0, sig_t=1.0, sig_m=0.05)
    # one chain step for step against the oracle
    m, ev, ids, logp, stats, tr = run_gpu(cm, w, sweeps=40, k=16, seed=100, events=start, p_pair=PAIR, **steps)
    o, oev, oids, otr, odlp = run_oracle(orc, w, sweeps=40, k=16, seed=100, events=start, p_pair=PAIR, **steps)
    assert_traces_match(tr, otr)
    assert np.array_equal(ev[:, :3], oev[:, :3])
    m.destroy()
    hits = {}
    for shift_mode in (1, 0):
        n = 0
        for seed in range(100, 108):
            m, ev, _, _, _, _ = run_gpu(cm, w, sweeps=40, k=16, seed=seed, events=start, shift_mode=shift_mode,
                                        trace=False, p_pair=PAIR, **steps)
            n += _reached(ev, truth)
            m.destroy()
        hits[shift_mode] = n
    # the oracle's chains of the same seeds: 7 of 8 dynamic, 0 of 8 static
    assert hits[1] >= 6 and hits[0] <= 1, hits


# ---- the float32 form -------------------------------------------------------

def _f32_world(seed):
    return small_world(seed=seed, W=1000.0, T=3600.0, Lambda=500.0, n_side=10, dtype=np.float32)


def test_fp32_pairs_dry_run_match_oracle(cm, orc):
    """Commit off, from the ground truth, joint moves at 0.2: every step's
    type, validity and event count equal the oracle's, and every float32
    change of the log-likelihood is within 1e-4 (to max(|x|, 1)) of the
    oracle's for the same pair of candidates; the pair counters of the
    statistics equal the trace's."""
    w = _f32_world(61)
    m, ev, ids, logp, stats, tr = run_gpu(cm, w, sweeps=4, k=32, seed=13, events=w.events, commit=False,
                                          p_pair=PAIR)
    o, oev, oids, otr, odlp = run_oracle(orc, w, sweeps=4, k=32, seed=13, events=w.events, commit=False,
                                         p_pair=PAIR, threads=min(16, os.cpu_count() or 1))
    assert len(tr) == len(otr)
    for key in ("sweep", "cell", "step", "type", "n_before", "evaluated"):
        assert np.array_equal(tr[key], otr[key]), key
    ev_ = otr["evaluated"] == 1
    err = np.abs(tr["dll"][ev_] - otr["dll"][ev_]) / np.maximum(np.abs(otr["dll"][ev_]), 1.0)
    pairs = (otr["type"] == 3) & ev_
    assert pairs.sum() > 300
    assert err.max() <= 1e-4, err.max()
    assert np.count_nonzero(tr["accepted"][ev_] != otr["accepted"][ev_]) <= max(2, err.size // 10000)
    assert stats["pair"] == _pair_counts(tr)
    m.destroy()


@pytest.mark.parametrize("init", ["empty", "truth"])
def test_fp32_pairs_chain_tracks_oracle_log_density(cm, orc, init):
    """With commits and joint moves: the running log-density equals the
    oracle's log-density of the final events and the GPU's recomputation, so
    the variance re-synthesised after a pair's commit matches its events."""
    w = _f32_world(62)
    ev0 = w.events if init == "truth" else None
    m, ev, ids, logp, stats, tr = run_gpu(cm, w, sweeps=20, k=32, seed=14, events=ev0, p_pair=PAIR)
    assert stats["pair"][2] > 20
    want = orc.World(w).log_density(ev)
    print("running %.4f oracle %.4f gpu recomputed %.4f" % (logp, want, m.log_density()))
    assert logp == pytest.approx(want, rel=1e-6)
    assert logp == pytest.approx(m.log_density(), rel=1e-6)
    assert len(np.unique(ids)) == len(ids)
    m.destroy()


def test_fp32_swapped_pair_reaches_its_true_mode(cm):
    """The swapped-pair world with float32 signals: joint moves under dynamic
    colouring reach the true mode in most chains, across a fixed boundary in
    (almost) none, as in the float64 form and the oracle."""
    w64, truth, start = _swapped_pair_world()
    w = worldgen.make_world(w64.params, w64.stations, seed=9, events=truth, dtype=np.float32)
    steps = dict(sig_xy=3.0, sig_t=1.0, sig_m=0.05)
    hits = {}
    for shift_mode in (1, 0):
        n = 0
        for seed in range(100, 108):
            m, ev, _, _, _, _ = run_gpu(cm, w, sweeps=40, k=16, seed=seed, events=start, shift_mode=shift_mode,
                                        trace=False, p_pair=PAIR, **steps)
            n += _reached(ev, truth)
            m.destroy()
        hits[shift_mode] = n
    assert hits[1] >= 5 and hits[0] <= 1, hits


def test_fp32_pairs_persistent_sweep_matches_colour_by_colour(cm):
    """The instantiation with joint moves: one persistent launch per sweep
    (regions waiting only for their lower-colour neighbours) gives the chain
    of the colour-by-colour schedule bit for bit."""
    w = _f32_world(63)
    runs = []
    for schedule in (0, 1):
        m, ev, ids, logp, stats, tr = run_gpu(cm, w, sweeps=8, k=32, events=w.events, seed=15, schedule=schedule,
                                              p_pair=PAIR)
        runs.append((ev, ids, logp, tr, stats))
        m.destroy()
    assert runs[0][4]["pair"][2] > 10
    assert runs[0][4]["kernel_launches"] < runs[1][4]["kernel_launches"]
    assert np.array_equal(runs[0][0], runs[1][0]) and np.array_equal(runs[0][1], runs[1][1])
    assert runs[0][2] == runs[1][2]
    assert np.array_equal(runs[0][3], runs[1][3])


def test_batch_refuses_joint_moves(cm):
    """A batch runs the kernel without joint moves: a model with them is
    refused."""
    w = _f32_world(64)
    m = cm.create_model(w.events, w.stations, w.signals,
                        cm.make_params(w.params, k_per_phase=16, seed=3, dtype=cm.F32, p_pair=PAIR))
    m.partition_and_color(w.params.L, 1)
    with pytest.raises(cm.ChromhError):
        cm.create_batch([m])
    m.destroy()
