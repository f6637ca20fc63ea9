"""CUDA path vs the CPU oracle, through the C ABI.

float64 replay: every MH step's move type, validity, event pick and accept
decision are bit-identical to the oracle's; log-likelihood changes and log
acceptance ratios agree to 1e-9 relative (to max(|x|, 1)); the final event
sets are identical (ids and coordinates).  The oracle never sees anything
the GPU produced: both start from the same seeded world and seed.
"""
import math
import os

import numpy as np
import pytest

import worldgen
from gpu_helpers import assert_traces_match, lib, run_gpu, run_oracle, small_world

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def cm():
    return lib()


def assert_running_log_density(o, w, init, logp, oev, otr):
    """The GPU's running log-density (its start plus every accepted step's
    change) equals the oracle's log-density of the final state, summed from
    scratch.  The running value is a sum of terms as large as the start's
    log-density and the accepted changes (up to ~1e9 when the chain starts
    empty under a large event), so it is held to 1e-12 of that magnitude,
    a few float64 roundings of the largest term."""
    lp0 = o.log_density(w.events if init == "truth" else np.zeros((0, 4)))
    acc = otr["accepted"] == 1
    scale = abs(lp0) + float(np.abs(otr["dll"][acc]).sum())
    want = o.log_density(oev)
    assert abs(logp - want) <= 1e-12 * scale, (logp, want, scale)


def test_philox_device_matches_oracle(cm, orc):
    rng = np.random.default_rng(3)
    ctr = rng.integers(0, 2**63, size=(2048, 4), dtype=np.uint64)
    ctr[:4] = [[0, 0, 0, 0], [2**64 - 1, 2**64 - 1, 2**64 - 1, 2**64 - 1], [1, 2, 3, 4], [7, 0, 0, 1]]
    for key in ([0, 0], [11, 0], [2**64 - 1, 1], [12345, 2]):
        dev = cm.philox4x64(ctr, key)
        ref = np.array([orc.philox4x64(c, key) for c in ctr])
        assert np.array_equal(dev, ref)


@pytest.mark.parametrize("init", ["empty", "truth"])
@pytest.mark.parametrize("shift_mode", [1, 0])
def test_replay_small_bit_exact(cm, orc, init, shift_mode):
    w = small_world()
    ev0 = w.events if init == "truth" else None
    sweeps = 6
    m, ev, ids, logp, stats, tr = run_gpu(cm, w, sweeps=sweeps, events=ev0, shift_mode=shift_mode,
                                          sx=37.0, sy=81.5)
    o, oev, oids, otr, odlp = run_oracle(orc, w, sweeps=sweeps, events=ev0, shift_mode=shift_mode,
                                         sx=37.0, sy=81.5)
    assert_traces_match(tr, otr)
    assert np.array_equal(ids, oids)
    # x, y, t are sums of exactly rounded operations on both sides; m goes
    # through log() at birth, which may differ by an ulp between libraries
    assert np.array_equal(ev[:, :3], oev[:, :3])
    assert np.allclose(ev[:, 3], oev[:, 3], rtol=1e-14, atol=0)
    assert stats["accepted"][0] + stats["accepted"][1] + stats["accepted"][2] == int(tr["accepted"].sum())
    assert sum(stats["proposed"]) == len(tr)
    assert_running_log_density(o, w, init, logp, oev, otr)
    m.destroy()


@pytest.mark.parametrize("seed,init", [(1000, "empty"), (1001, "empty"), (1002, "empty"), (1000, "truth")])
def test_tiny_config_bit_exact(cm, orc, seed, init):
    """The small configuration (200 x 200 km, 600 s, Lambda 10, 4 stations on a
    2 x 2 grid, 6000 float64 samples, regions of side 100 km, 4 colours) at
    k = 500 steps per region and phase: 18,000 MH steps over 4 sweeps, step
    for step against the oracle.  A region may hold its events plus k births,
    hence the event capacity of 640."""
    w = worldgen.config_tiny(seed=seed)
    ev0 = w.events if init == "truth" else None
    m, ev, ids, logp, stats, tr = run_gpu(cm, w, sweeps=4, k=500, seed=seed, events=ev0, ev_capacity=640)
    o, oev, oids, otr, odlp = run_oracle(orc, w, sweeps=4, k=500, seed=seed, events=ev0)
    assert len(tr) >= 10000
    assert_traces_match(tr, otr)
    assert np.array_equal(ids, oids)
    assert np.array_equal(ev[:, :3], oev[:, :3])
    assert_running_log_density(o, w, init, logp, oev, otr)
    m.destroy()


def test_replay_shift_matches_oracle(cm, orc):
    w = small_world(seed=8)
    params = cm.make_params(w.params, k_per_phase=4, seed=99, dtype=cm.F64)
    m = cm.create_model(None, w.stations, w.signals, params)
    m.partition_and_color(w.params.L, shift_mode=1)
    o = orc.World(w, seed=99)
    for s in range(5):
        m.run_sweeps(1)
        assert m.read_shift() == o.shift(s)
    m.destroy()


def test_replay_config2_world(cm, orc):
    """The 1000 x 1000 km, 100-station, 36000-sample world of the replay
    workload: a few sweeps from the ground truth and from the empty set."""
    w = worldgen.config_replay(seed=1000)
    threads = min(16, os.cpu_count() or 1)
    for init in (w.events, None):
        m, ev, ids, logp, stats, tr = run_gpu(cm, w, sweeps=3, k=32, seed=7, events=init)
        o, oev, oids, otr, odlp = run_oracle(orc, w, sweeps=3, k=32, seed=7, events=init, threads=threads)
        assert_traces_match(tr, otr)
        assert np.array_equal(ids, oids)
        assert np.array_equal(ev[:, :3], oev[:, :3])
        m.destroy()


def test_log_density_recompute_matches_oracle(cm, orc):
    w = small_world(seed=9)
    params = cm.make_params(w.params, k_per_phase=8, seed=5, dtype=cm.F64)
    m = cm.create_model(w.events, w.stations, w.signals, params)
    o = orc.World(w)
    want = o.log_density(w.events)
    assert m.log_density() == pytest.approx(want, rel=1e-12)
    _, _, lp_run, _ = m.read_state()
    assert lp_run == pytest.approx(want, rel=1e-12)
    # after sweeps, the running value tracks a from-scratch recomputation
    m.partition_and_color(w.params.L, 1)
    m.run_sweeps(10)
    _, _, lp_run, _ = m.read_state()
    assert m.log_density() == pytest.approx(lp_run, rel=1e-10)
    m.destroy()


def test_device_signals_and_empty_start(cm, orc):
    w = small_world(seed=12)
    a = run_gpu(cm, w, sweeps=3, on_device=True)
    b = run_gpu(cm, w, sweeps=3, on_device=False)
    assert np.array_equal(a[1], b[1]) and np.array_equal(a[5], b[5])
    a[0].destroy()
    b[0].destroy()


def test_ragged_samples_and_single_step(cm, orc):
    # n_samples not a multiple of 4 or 64; windows cut by the record's end
    w = small_world(seed=13, T=1234.5, Lambda=40.0)
    assert w.signals.shape[1] % 4 != 0
    m, ev, ids, logp, stats, tr = run_gpu(cm, w, sweeps=4, k=1, events=w.events)
    o, oev, oids, otr, odlp = run_oracle(orc, w, sweeps=4, k=1, events=w.events)
    assert_traces_match(tr, otr)
    assert np.array_equal(ids, oids)
    m.destroy()


def test_prior_only_world(cm, orc):
    """No stations: the chain samples the prior; still bit-identical."""
    p = worldgen.ModelParams(W=300.0, T=100.0, Lambda=15.0)
    w = worldgen.World(params=p, stations=np.zeros((0, 2)), signals=np.zeros((0, p.n_samples)),
                       events=np.zeros((0, 4)))
    m, ev, ids, logp, stats, tr = run_gpu(cm, w, sweeps=20, k=8)
    o, oev, oids, otr, odlp = run_oracle(orc, w, sweeps=20, k=8)
    assert_traces_match(tr, otr)
    assert np.array_equal(ids, oids) and 0 < len(ev) < 60
    m.destroy()


def test_capacity_overflow_is_reported_not_faulted(cm):
    w = small_world(seed=14, Lambda=400.0)
    params = cm.make_params(w.params, k_per_phase=16, seed=1, dtype=cm.F64, ev_capacity=17)
    m = cm.create_model(w.events, w.stations, w.signals, params)
    with pytest.raises(cm.ChromhError) as ei:
        m.partition_and_color(w.params.L, 1)
        m.run_sweeps(1)
        m.read_state()
    assert ei.value.code == -5
    with pytest.raises(cm.ChromhError) as ei:
        m.run_sweeps(1)
    assert ei.value.code == -8
    m.destroy()


def test_checkpoint_restore_continues_the_chain(cm):
    w = small_world(seed=15)
    params = cm.make_params(w.params, k_per_phase=8, seed=4, dtype=cm.F64)
    a = cm.create_model(None, w.stations, w.signals, params)
    a.partition_and_color(w.params.L, 1)
    a.run_sweeps(10)
    ev_a, ids_a, lp_a, _ = a.read_state()
    b = cm.create_model(None, w.stations, w.signals, params)
    b.partition_and_color(w.params.L, 1)
    b.run_sweeps(5)
    blob = b.checkpoint()
    c = cm.create_model(None, w.stations, w.signals, params)
    c.restore(blob)
    c.run_sweeps(5)
    ev_c, ids_c, lp_c, _ = c.read_state()
    assert np.array_equal(ids_a, ids_c)
    assert np.array_equal(ev_a[:, :3], ev_c[:, :3])
    assert lp_c == pytest.approx(lp_a, rel=1e-11)
    with pytest.raises(cm.ChromhError):
        c.restore(blob[:40])
    for x in (a, b, c):
        x.destroy()


def test_fp32_dry_run_deltas(cm, orc):
    """float32 per-sample terms vs the float64 oracle on the same proposals:
    with commit off, every proposal is priced against the ground-truth state,
    so the two sides price identical (state, candidate) pairs."""
    w = small_world(seed=16, W=1000.0, T=3600.0, Lambda=500.0, n_side=10, dtype=np.float32)
    m, ev, ids, logp, stats, tr = run_gpu(cm, w, sweeps=4, k=32, events=w.events, commit=False, seed=21)
    o, oev, oids, otr, odlp = run_oracle(orc, w, sweeps=4, k=32, events=w.events, commit=False, seed=21,
                                         threads=min(16, os.cpu_count() or 1))
    missing = sorted(set(zip(otr["sweep"], otr["cell"])) - set(zip(tr["sweep"], tr["cell"])))
    assert len(tr) == len(otr), ("region phases without records (sweep, cell)", missing[:8], stats)
    for key in ("sweep", "cell", "step", "type", "n_before"):
        assert np.array_equal(tr[key], otr[key]), key
    # the float32 Box-Muller may round a Gaussian offset to the neighbouring
    # 2^-20 quantum (a few micrometres), which can flip validity only for a
    # candidate that close to a region boundary
    assert np.count_nonzero(tr["evaluated"] != otr["evaluated"]) <= max(2, len(tr) // 10000)
    ev_ = (otr["evaluated"] == 1) & (tr["evaluated"] == 1)
    err = np.abs(tr["dll"][ev_] - otr["dll"][ev_]) / np.maximum(np.abs(otr["dll"][ev_]), 1.0)
    print("fp32 dll rel err: n=%d median %.2e p99 %.2e p99.9 %.2e max %.2e" % (
        err.size, np.median(err), np.quantile(err, 0.99), np.quantile(err, 0.999), err.max()))
    assert err.max() <= 1e-4
    mism = np.count_nonzero(tr["accepted"][ev_] != otr["accepted"][ev_])
    assert mism <= max(2, err.size // 10000)
    m.destroy()


def test_fp32_precision_at_scale_density(cm, orc):
    """The float32 sweep kernel at the density and record length of the
    4000 x 4000 km, 24 h workload: a 1000 x 1000 km world of that density
    (100 jittered stations x 864,000 float32 samples, ~625 events, regions
    of 100 km), dry run (commit off) from the ground truth, 40 sweeps of
    k = 32.  Every evaluated proposal's float32 change of the log-likelihood
    is compared with the float64 oracle's for the same (state, candidate):
    at least 1e5 of them, each within 1e-4 relative (to max(|x|, 1)).  The
    error distribution is printed as one JSON line (FP32_ERROR)."""
    import json
    w = worldgen.config_scale(seed=1000, side_regions=10)
    sweeps = 40
    m, ev, ids, logp, stats, tr = run_gpu(cm, w, sweeps=sweeps, k=32, events=w.events, commit=False, seed=23)
    o, oev, oids, otr, odlp = run_oracle(orc, w, sweeps=sweeps, k=32, events=w.events, commit=False, seed=23,
                                         threads=min(16, os.cpu_count() or 1))
    assert len(tr) == len(otr)
    for key in ("sweep", "cell", "step", "type", "n_before"):
        assert np.array_equal(tr[key], otr[key]), key
    assert np.count_nonzero(tr["evaluated"] != otr["evaluated"]) <= max(2, len(tr) // 10000)
    ev_ = (otr["evaluated"] == 1) & (tr["evaluated"] == 1)
    d32, d64 = tr["dll"][ev_], otr["dll"][ev_]
    err = np.abs(d32 - d64) / np.maximum(np.abs(d64), 1.0)
    with np.errstate(divide="ignore", invalid="ignore"):
        rel = np.abs(d32 - d64) / np.abs(d64)
    rel = rel[np.isfinite(rel)]
    rec = {"workload": "1000x1000 km world at the density of the 4000 km / 24 h workload: 100 stations x "
                       "864000 f32 samples, ~%d events, dry run from the ground truth, %d sweeps, k=32"
                       % (len(w.events), sweeps),
           "n": int(err.size), "median": float(np.median(err)), "p99": float(np.quantile(err, 0.99)),
           "p999": float(np.quantile(err, 0.999)), "max": float(err.max()),
           "pure_relative_max": float(rel.max()), "bound": 1e-4,
           "decisions_differing": int(np.count_nonzero(tr["accepted"][ev_] != otr["accepted"][ev_]))}
    import bench
    rec["kernel_sha256"] = bench._kernel_digest()
    rec["command"] = ("python -m pytest tests/test_gpu_parity.py -m gpu -s "
                      "-k test_fp32_precision_at_scale_density")
    print("FP32_ERROR " + json.dumps(rec))
    assert err.size >= 100000
    assert err.max() <= 1e-4
    assert rec["decisions_differing"] <= max(2, err.size // 10000)
    m.destroy()


def test_fp32_bench_workload_at_full_size(cm, orc):
    """The bench workload at its full size (4000 x 4000 km, 24 h, 1600
    stations x 864,000 float32 samples, ~1e4 events, 40 x 40 regions,
    k = 32), in the launch configuration bench.py times (signals on the
    device, one persistent launch per sweep), dry run (commit off) from the
    ground truth for 3 sweeps: every step's type, validity and event count
    equal the oracle's, and every evaluated change of the log-likelihood
    (~150,000) is within 1e-4 (to max(|x|, 1)) of the oracle's float64 change
    for the same (state, candidate)."""
    w = worldgen.config_scale(seed=1000)
    sweeps = 3
    m, ev, ids, logp, stats, tr = run_gpu(cm, w, sweeps=sweeps, k=32, events=w.events, commit=False, seed=29,
                                          on_device=True)
    o, oev, oids, otr, odlp = run_oracle(orc, w, sweeps=sweeps, k=32, events=w.events, commit=False, seed=29,
                                         threads=os.cpu_count() or 1)
    assert len(tr) == len(otr) > 150000
    for key in ("sweep", "cell", "step", "type", "n_before", "evaluated"):
        assert np.array_equal(tr[key], otr[key]), key
    ev_ = otr["evaluated"] == 1
    d32, d64 = tr["dll"][ev_], otr["dll"][ev_]
    err = np.abs(d32 - d64) / np.maximum(np.abs(d64), 1.0)
    print("full size: %d evaluated, error median %.3g p99 %.3g max %.3g, %d decisions differ"
          % (err.size, np.median(err), np.quantile(err, 0.99), err.max(),
             np.count_nonzero(tr["accepted"][ev_] != otr["accepted"][ev_])))
    assert err.size > 140000
    assert err.max() <= 1e-4
    assert np.count_nonzero(tr["accepted"][ev_] != otr["accepted"][ev_]) <= max(2, err.size // 10000)
    assert np.array_equal(ids, oids) and np.array_equal(ev, oev)
    m.destroy()


@pytest.mark.parametrize("init", ["empty", "truth"])
def test_fp32_chain_tracks_recomputed_log_density(cm, orc, init):
    """float32 chain with commits: the running log-density (float64 sum of
    accepted changes) agrees with the oracle's log-density of the final event
    set, summed from scratch in float64, and with the GPU's own
    recomputation, so the variance re-synthesised on every accept stays
    consistent with the events."""
    w = small_world(seed=17, W=1000.0, T=3600.0, Lambda=500.0, n_side=10, dtype=np.float32)
    ev0 = w.events if init == "truth" else None
    m, ev, ids, logp, stats, tr = run_gpu(cm, w, sweeps=30, k=32, events=ev0, seed=5)
    assert sum(stats["accepted"]) > 1000
    want = orc.World(w).log_density(ev)
    print("running %.6f oracle %.6f rel %.3g" % (logp, want, abs(logp - want) / abs(want)))
    assert logp == pytest.approx(want, rel=1e-6)
    assert logp == pytest.approx(m.log_density(), rel=2e-7, abs=1.0)
    assert len(np.unique(ids)) == len(ids)
    assert np.all((ev[:, 0] >= 0) & (ev[:, 0] < w.params.W) & (ev[:, 2] >= 0) & (ev[:, 2] < w.params.T))
    assert np.all(ev[:, 3] >= 2.0)
    m.destroy()


@pytest.mark.parametrize("likelihood", ["variance", "mean"])
def test_fp32_staging_modes_agree(cm, likelihood):
    """Station windows staged in shared memory by bulk copies (automatic
    size), staged only where they fit in 64 samples, or read from global
    memory (the default): the same arithmetic on the same values, so the
    chains agree bit for bit."""
    w = small_world(seed=18, W=1000.0, T=3600.0, Lambda=500.0, n_side=10, dtype=np.float32,
                    likelihood=likelihood)
    runs = []
    for stage in (-1, 64, 0):
        m, ev, ids, logp, stats, tr = run_gpu(cm, w, sweeps=6, k=32, events=w.events, seed=9, stage_samples=stage)
        runs.append((ev, ids, logp, tr, stats))
        m.destroy()
    assert sum(runs[0][4]["accepted"]) > 100
    for ev, ids, logp, tr, _ in runs[1:]:
        assert np.array_equal(ev, runs[0][0]) and np.array_equal(ids, runs[0][1])
        assert logp == runs[0][2]
        assert np.array_equal(tr, runs[0][3])


@pytest.mark.parametrize("likelihood", ["variance", "mean"])
def test_fp32_persistent_sweep_matches_colour_by_colour(cm, likelihood):
    """One persistent launch per sweep, each region waiting only for its
    lower-colour neighbours, gives the chain of the colour-by-colour
    schedule bit for bit (the same steps see the same neighbour states)."""
    w = small_world(seed=19, W=1000.0, T=3600.0, Lambda=500.0, n_side=10, dtype=np.float32,
                    likelihood=likelihood)
    runs = []
    for schedule in (0, 1):
        m, ev, ids, logp, stats, tr = run_gpu(cm, w, sweeps=8, k=32, events=w.events, seed=13, schedule=schedule)
        runs.append((ev, ids, logp, tr, stats))
        m.destroy()
    assert sum(runs[0][4]["accepted"]) > 100
    assert runs[0][4]["kernel_launches"] < runs[1][4]["kernel_launches"]
    assert np.array_equal(runs[0][0], runs[1][0]) and np.array_equal(runs[0][1], runs[1][1])
    assert runs[0][2] == runs[1][2]
    assert np.array_equal(runs[0][3], runs[1][3])


def test_autotune_restores_the_chain(cm):
    """The autotuner's trial sweeps run from a checkpoint that is restored:
    the chain afterwards is the one without tuning."""
    w = small_world(seed=20, W=800.0, T=1800.0, Lambda=200.0, n_side=8, dtype=np.float32)
    out = []
    for tune in (True, False):
        m = cm.create_model(w.events, w.stations, w.signals,
                            cm.make_params(w.params, k_per_phase=32, seed=3, dtype=cm.F32))
        m.partition_and_color(w.params.L, 1)
        m.run_sweeps(3)
        if tune:
            t = m.autotune(2)
            assert t["ms_per_sweep"] > 0 and len(t["tried"]) == 6
            assert any(r["ms_per_sweep"] == t["ms_per_sweep"] for r in t["tried"])
        m.run_sweeps(5)
        ev, ids, lp, st = m.read_state()
        out.append((ev, ids, lp, st["proposed"], st["sweeps"]))
        m.destroy()
    (ea, ia, la, pa, sa), (eb, ib, lb, pb, sb) = out
    # restoring re-synthesises V from the events, which may change its last
    # bits (summation order): the log-density agrees to rounding
    assert np.array_equal(ia, ib) and np.array_equal(ea, eb) and pa == pb and sa == sb == 8
    assert la == pytest.approx(lb, rel=1e-11)


def _table_for(w, nx=40, nt=36, seed=3):
    """A learned-looking birth table: a smooth floor plus weight around the
    generated events' pixels and time bins."""
    rng = np.random.default_rng(seed)
    tab = (0.2 + rng.random((nx, nx, nt))).astype(np.float32)
    p = w.params
    for x, y, t, m in w.events:
        ix, iy, b = int(x / p.W * nx), int(y / p.W * nx), int(t / p.T * nt)
        tab[max(0, iy - 1):iy + 2, max(0, ix - 1):ix + 2, max(0, b - 1):b + 2] += 40.0
    return tab


@pytest.mark.parametrize("magnitudes,likelihood", [(False, "variance"), (True, "variance"), (True, "mean")])
def test_fp32_dry_run_with_learned_birth_table(cm, orc, magnitudes, likelihood):
    """Birth proposals from the mixture with a table: the same candidates on
    both sides (the table draw runs in explicitly rounded float64), Δℓ within
    1e-4 and log α (which now carries the mixture density) likewise.  With
    learned magnitudes the table births draw m from their entry's window
    (float64 on both sides), and the density carries the window."""
    w = small_world(seed=16, W=1000.0, T=3600.0, Lambda=500.0, n_side=10, dtype=np.float32,
                    likelihood=likelihood)
    tab = _table_for(w)
    params = cm.make_params(w.params, k_per_phase=32, seed=21, dtype=cm.F32, commit=False)
    m = cm.create_model(w.events, w.stations, w.signals, params)
    m.set_birth_table(tab, 0.5)
    centre = (2.2 + 2.0 * np.random.default_rng(5).random(tab.shape)).astype(np.float32)
    if magnitudes:
        m.set_birth_magnitude(centre, 0.3)
    m.partition_and_color(w.params.L, 1)
    ncx = int(np.floor(w.params.W / w.params.L)) + 2
    m.set_trace(4 * ncx * ncx * 32)
    m.run_sweeps(4)
    from gpu_helpers import TRACE_KEYS
    tr = np.sort(m.read_trace(), order=TRACE_KEYS)
    o = orc.World(w, k_per_phase=32, seed=21, commit=False)
    o.set_birth_table(tab, 0.5)
    if magnitudes:
        o.set_birth_magnitude(centre, 0.3)
    _, _, otr, _ = o.run_chromatic(w.events, 4, trace_cap=200000, threads=min(16, os.cpu_count() or 1))
    otr = np.sort(otr, order=TRACE_KEYS)
    assert len(tr) == len(otr)
    for key in ("sweep", "cell", "step", "type", "n_before"):
        assert np.array_equal(tr[key], otr[key]), key
    assert np.count_nonzero(tr["evaluated"] != otr["evaluated"]) <= max(2, len(tr) // 10000)
    ev_ = (otr["evaluated"] == 1) & (tr["evaluated"] == 1)
    births = ev_ & (otr["type"] == 0)
    assert births.sum() > 500
    err = np.abs(tr["dll"][ev_] - otr["dll"][ev_]) / np.maximum(np.abs(otr["dll"][ev_]), 1.0)
    assert err.max() <= 1e-4
    la_err = np.abs(tr["log_alpha"][ev_] - otr["log_alpha"][ev_]) / np.maximum(np.abs(otr["log_alpha"][ev_]), 1.0)
    assert la_err.max() <= 1e-4
    assert np.count_nonzero(tr["accepted"][ev_] != otr["accepted"][ev_]) <= max(2, ev_.sum() // 10000)
    m.destroy()


def test_nine_colour_geometry_replay_bit_exact(cm, orc):
    """R_max = L (events reach two regions away): 9 colours of period 3, the
    5 x 5 neighbourhood in the region prologue; float64 replay bit-exact."""
    w = small_world(seed=23, W=500.0, Lambda=80.0, R_max=100.0)
    params = cm.make_params(w.params, k_per_phase=16, seed=11, dtype=cm.F64)
    m = cm.create_model(None, w.stations, w.signals, params)
    assert m.partition_and_color(w.params.L, shift_mode=1) == 9
    m.destroy()
    m, ev, ids, logp, stats, tr = run_gpu(cm, w, sweeps=5)
    o, oev, oids, otr, odlp = run_oracle(orc, w, sweeps=5)
    assert_traces_match(tr, otr)
    assert np.array_equal(ids, oids)
    assert np.array_equal(ev[:, :3], oev[:, :3])
    m.destroy()


def test_nine_colour_geometry_fp32_deltas(cm, orc):
    w = small_world(seed=24, W=600.0, T=1800.0, Lambda=150.0, n_side=6, R_max=100.0, dtype=np.float32)
    m, ev, ids, logp, stats, tr = run_gpu(cm, w, sweeps=3, k=32, events=w.events, commit=False, seed=9)
    o, oev, oids, otr, odlp = run_oracle(orc, w, sweeps=3, k=32, events=w.events, commit=False, seed=9,
                                         threads=min(16, os.cpu_count() or 1))
    assert len(tr) == len(otr)
    for key in ("sweep", "cell", "step", "type", "n_before"):
        assert np.array_equal(tr[key], otr[key]), key
    ev_ = (otr["evaluated"] == 1) & (tr["evaluated"] == 1)
    assert ev_.sum() > 200
    err = np.abs(tr["dll"][ev_] - otr["dll"][ev_]) / np.maximum(np.abs(otr["dll"][ev_]), 1.0)
    assert err.max() <= 1e-4
    m.destroy()


# ---- the additive-mean reading (arrivals add to the sample mean) ------------
def _mean_world(seed):
    return small_world(seed=seed, W=1000.0, T=3600.0, Lambda=500.0, n_side=10, dtype=np.float32,
                       likelihood="mean")


def test_mean_reading_fp32_deltas(cm, orc):
    """The float32 per-sample term of the additive reading, (d (s - mu) -
    d^2/2) / noise over the touched windows, against the oracle's float64
    difference of log-densities on the same proposals (commit off)."""
    w = _mean_world(26)
    m, ev, ids, logp, stats, tr = run_gpu(cm, w, sweeps=3, k=32, events=w.events, commit=False, seed=3)
    o, oev, oids, otr, odlp = run_oracle(orc, w, sweeps=3, k=32, events=w.events, commit=False, seed=3,
                                         threads=min(16, os.cpu_count() or 1))
    assert len(tr) == len(otr)
    for key in ("sweep", "cell", "step", "type", "n_before"):
        assert np.array_equal(tr[key], otr[key]), key
    ev_ = (otr["evaluated"] == 1) & (tr["evaluated"] == 1)
    assert ev_.sum() > 1000
    err = np.abs(tr["dll"][ev_] - otr["dll"][ev_]) / np.maximum(np.abs(otr["dll"][ev_]), 1.0)
    print("mean reading fp32 dll rel err: median %.2e max %.2e" % (np.median(err), err.max()))
    assert err.max() <= 1e-4
    assert np.count_nonzero(tr["accepted"][ev_] != otr["accepted"][ev_]) <= max(2, ev_.sum() // 10000)
    m.destroy()


def test_mean_reading_chain_tracks_recomputed_log_density(cm, orc):
    """With commits the mean buffer is re-synthesised on every accept; the
    running log-density equals a recomputation, and the initial one equals
    the oracle's log-density of the starting state."""
    w = _mean_world(27)
    m, ev, ids, logp, stats, tr = run_gpu(cm, w, sweeps=20, k=32, events=None, seed=8)
    assert sum(stats["accepted"]) > 500
    assert logp == pytest.approx(m.log_density(), rel=2e-7, abs=1.0)
    o = orc.World(w)
    assert o.log_density(ev) == pytest.approx(m.log_density(), rel=1e-6)
    m.destroy()


def test_mean_reading_needs_float32(cm):
    w = small_world(seed=28, likelihood="mean")
    with pytest.raises(cm.ChromhError) as ei:
        cm.create_model(None, w.stations, w.signals, cm.make_params(w.params, dtype=cm.F64))
    assert ei.value.code == -1


def test_async_state_reads_equal_synchronous_ones(cm):
    """Double-buffered asynchronous reads taken after each sweep, fetched one
    sweep later, equal a second model's synchronous reads after the same
    sweeps (same chain)."""
    w = small_world(seed=29, W=1000.0, T=1800.0, Lambda=250.0, n_side=10, dtype=np.float32)
    params = cm.make_params(w.params, k_per_phase=16, seed=6, dtype=cm.F32)
    a = cm.create_model(None, w.stations, w.signals, params)
    b = cm.create_model(None, w.stations, w.signals, params)
    for m in (a, b):
        m.partition_and_color(w.params.L, 1)
    with pytest.raises(cm.ChromhError):
        a.read_state_fetch(0)   # nothing requested yet
    ref, got = [], []
    for i in range(6):
        a.run_sweeps(1)
        a.read_state_async(i % 2)
        if i > 0:
            got.append(a.read_state_fetch((i - 1) % 2))
        b.run_sweeps(1)
        ref.append(b.read_state())
    got.append(a.read_state_fetch(5 % 2))
    for (e0, i0, l0, s0), (e1, i1, l1, s1) in zip(ref, got):
        assert np.array_equal(e0, e1) and np.array_equal(i0, i1) and l0 == l1
        assert s0["accepted"] == s1["accepted"] and s0["sweeps"] == s1["sweeps"]
    assert len(got[-1][0]) > 0
    a.destroy()
    b.destroy()
