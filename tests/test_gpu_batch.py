"""A batch of independent models swept in one persistent launch per sweep
gives every model the chain cmh_run_sweeps gives it alone (bit for bit)."""
import numpy as np
import pytest

import worldgen
from gpu_helpers import lib

pytestmark = pytest.mark.gpu


def _worlds():
    rng = np.random.default_rng(77)
    out = []
    for i in range(7):
        side = float(100 * rng.integers(2, 7))
        T = float(rng.choice([600.0, 900.0, 1234.5]))
        lam = float(rng.uniform(5, 60)) * (side / 400.0) ** 2
        p = worldgen.ModelParams(W=side, T=T, Lambda=lam)
        n_st = int(rng.integers(3, 30))
        st = worldgen.uniform_stations(n_st, side, 300 + i)
        out.append(worldgen.make_world(p, st, 400 + i, np.float32))
    return out


def _model(cm, w, seed, start_truth, ev_capacity=0):
    m = cm.create_model(w.events if start_truth else None, w.stations, w.signals,
                        cm.make_params(w.params, k_per_phase=24, seed=seed, dtype=cm.F32, ev_capacity=ev_capacity))
    m.partition_and_color(w.params.L, shift_mode=1)
    return m


def test_batch_equals_models_run_alone():
    cm = lib()
    worlds = _worlds()
    # larger event capacities need more shared memory per region: the batch
    # puts those models in groups with fewer resident CTAs per SM
    caps = [0, 512, 0, 320, 0, 512, 0]
    alone = [_model(cm, w, 10 + i, i % 2 == 0, caps[i]) for i, w in enumerate(worlds)]
    batched = [_model(cm, w, 10 + i, i % 2 == 0, caps[i]) for i, w in enumerate(worlds)]
    for m in alone:
        m.run_sweeps(12)
    b = cm.create_batch(batched)
    assert len(b.groups()) >= 2 and sum(g[0] for g in b.groups()) == len(worlds)
    b.run_sweeps(5)
    b.run_sweeps(7)
    b.sync()
    for i, (a, c) in enumerate(zip(alone, batched)):
        ea, ia, la, sa = a.read_state()
        ec, ic, lc, sc = c.read_state()
        assert np.array_equal(ia, ic) and np.array_equal(ea, ec), i
        assert la == lc, i
        assert sa["proposed"] == sc["proposed"] and sa["accepted"] == sc["accepted"], i
        assert sc["sweeps"] == 12
    # a model swept alone after the batch continues the same chain
    alone[0].run_sweeps(3)
    batched[0].run_sweeps(3)
    assert np.array_equal(alone[0].read_state()[1], batched[0].read_state()[1])
    b.destroy()
    for m in alone + batched:
        m.destroy()


def test_batch_rejects_unsuitable_models():
    cm = lib()
    w = _worlds()[0]
    m = _model(cm, w, 1, True)
    with pytest.raises(cm.ChromhError):
        cm.create_batch([m, m])
    f64 = cm.create_model(w.events, w.stations, w.signals.astype(np.float64),
                          cm.make_params(w.params, k_per_phase=8, seed=1, dtype=cm.F64))
    f64.partition_and_color(w.params.L, 1)
    with pytest.raises(cm.ChromhError):
        cm.create_batch([m, f64])
    b = cm.create_batch([m])
    m.partition_and_color(w.params.L, 1)   # a new partition: the batch no longer applies
    with pytest.raises(cm.ChromhError) as ei:
        b.run_sweeps(1)
    assert ei.value.code == -8
    b.sync()
    b.destroy()
    m.destroy()
    f64.destroy()


def test_mean_reading_batch_equals_each_model_alone():
    """The batch kernel of the additive reading: a batch of such models gives
    each model's own chain bit for bit; a batch mixing readings is refused."""
    cm = lib()
    import worldgen
    ws = [worldgen.config_scale(seed=s, side_regions=3, T=900.0, likelihood="mean") for s in (3, 4)]
    def make(i, w):
        m = cm.create_model(w.events, w.stations, w.signals,
                            cm.make_params(w.params, k_per_phase=16, seed=60 + i, dtype=cm.F32))
        m.partition_and_color(w.params.L, 1)
        return m
    alone = [make(i, w) for i, w in enumerate(ws)]
    for m in alone:
        m.run_sweeps(5)
    ref = [m.read_state() for m in alone]
    batched = [make(i, w) for i, w in enumerate(ws)]
    b = cm.create_batch(batched)
    b.run_sweeps(5)
    b.sync()
    for (e0, i0, l0, _), m in zip(ref, batched):
        e1, i1, l1, _ = m.read_state()
        assert np.array_equal(e0, e1) and np.array_equal(i0, i1) and l0 == l1
    b.destroy()
    wv = worldgen.config_scale(seed=5, side_regions=3, T=900.0)
    mv = cm.create_model(wv.events, wv.stations, wv.signals,
                         cm.make_params(wv.params, k_per_phase=16, seed=1, dtype=cm.F32))
    mv.partition_and_color(wv.params.L, 1)
    with pytest.raises(cm.ChromhError):
        cm.create_batch([batched[0], mv])
    for m in alone + batched + [mv]:
        m.destroy()


def test_batched_instances_match_oracle():
    """Each instance of a batch, dry run (commit off) from its ground truth,
    against the oracle on the same world and seed: the same steps with the
    same move types and event counts, every float32 change of the
    log-likelihood within 1e-4 (to max(|x|, 1)) of the oracle's.  Instances of
    the batched workload's kind (uniform stations, uneven sizes), plus one
    whose regions spill their lists to global memory (256 stations on
    300 x 300 km)."""
    import os
    import oracle
    from gpu_helpers import TRACE_KEYS
    from test_gpu_dense import dense_world
    cm = lib()
    oracle.build()
    rng = np.random.default_rng(91)
    worlds = []
    for i in range(4):
        side = float(100 * rng.integers(3, 9))
        p = worldgen.ModelParams(W=side, T=float(rng.choice([900.0, 1800.0, 2400.5])),
                                 Lambda=float(rng.uniform(20, 200)) * (side / 500.0) ** 2)
        st = worldgen.uniform_stations(int(rng.integers(16, 96)), side, 500 + i)
        worlds.append(worldgen.make_world(p, st, 600 + i, np.float32))
    worlds.append(dense_world(33))
    k, sweeps = 16, 3
    models = []
    for i, w in enumerate(worlds):
        m = cm.create_model(w.events, w.stations, w.signals,
                            cm.make_params(w.params, k_per_phase=k, seed=70 + i, dtype=cm.F32, commit=False))
        m.partition_and_color(w.params.L, shift_mode=1)
        ncx = int(np.floor(w.params.W / w.params.L)) + 2
        m.set_trace(sweeps * ncx * ncx * k)
        models.append(m)
    assert models[-1].read_state(cap=0)[3]["spill_bytes"] > 0
    b = cm.create_batch(models)
    b.run_sweeps(sweeps)
    b.sync()
    threads = min(16, os.cpu_count() or 1)
    for i, (w, m) in enumerate(zip(worlds, models)):
        tr = np.sort(m.read_trace(), order=TRACE_KEYS)
        o = oracle.World(w, k_per_phase=k, seed=70 + i, commit=False)
        _, _, otr, _ = o.run_chromatic(w.events, sweeps, trace_cap=len(tr) + 16, threads=threads)
        otr = np.sort(otr, order=TRACE_KEYS)
        assert len(tr) == len(otr) > 0, i
        for key in ("sweep", "cell", "step", "type", "n_before", "evaluated"):
            assert np.array_equal(tr[key], otr[key]), (i, key)
        ev_ = otr["evaluated"] == 1
        err = np.abs(tr["dll"][ev_] - otr["dll"][ev_]) / np.maximum(np.abs(otr["dll"][ev_]), 1.0)
        assert ev_.sum() > 50 and err.max() <= 1e-4, (i, err.max())
    b.destroy()
    for m in models:
        m.destroy()


def test_batched_workload_at_full_size():
    """All 256 instances of the batched workload (the sizes and worlds
    bench.py draws, its capacities and its batched persistent launch, k = 32),
    dry run (commit off) from each instance's ground truth for one sweep:
    every instance's steps equal the oracle's (move type, validity, event
    count), and every float32 change of the log-likelihood (~390,000) is
    within 1e-4 (to max(|x|, 1)) of the oracle's on the same world and
    seed."""
    import os
    import sys
    import oracle
    from gpu_helpers import TRACE_KEYS
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    import bench
    cm = lib()
    oracle.build()
    worlds = worldgen.config_batched(256, seed=2000)
    k = bench.K_PER_PHASE
    models = []
    for i, w in enumerate(worlds):
        ev_cap, frz_cap = bench.instance_capacities(w.params)
        m = cm.create_model(w.events, w.stations, w.signals,
                            cm.make_params(w.params, k_per_phase=k, seed=bench.CHAIN_SEED + i, dtype=cm.F32,
                                           commit=False, ev_capacity=ev_cap, frozen_capacity=frz_cap))
        m.partition_and_color(w.params.L, shift_mode=1)
        ncx = int(np.floor(w.params.W / w.params.L)) + 2
        m.set_trace(ncx * ncx * k)
        models.append(m)
    b = cm.create_batch(models)
    b.run_sweeps(1)
    b.sync()
    threads = os.cpu_count() or 1
    errs, n_dec = [], 0
    for i, (w, m) in enumerate(zip(worlds, models)):
        tr = np.sort(m.read_trace(), order=TRACE_KEYS)
        o = oracle.World(w, k_per_phase=k, seed=bench.CHAIN_SEED + i, commit=False)
        _, _, otr, _ = o.run_chromatic(w.events, 1, trace_cap=len(tr) + 16, threads=threads)
        otr = np.sort(otr, order=TRACE_KEYS)
        assert len(tr) == len(otr), i
        for key in ("sweep", "cell", "step", "type", "n_before", "evaluated"):
            assert np.array_equal(tr[key], otr[key]), (i, key)
        ev_ = otr["evaluated"] == 1
        errs.append(np.abs(tr["dll"][ev_] - otr["dll"][ev_]) / np.maximum(np.abs(otr["dll"][ev_]), 1.0))
        n_dec += int(np.count_nonzero(tr["accepted"][ev_] != otr["accepted"][ev_]))
    b.destroy()
    for m in models:
        m.destroy()
    err = np.concatenate(errs)
    print("batched, full size: %d evaluated, error median %.3g p99 %.3g max %.3g, %d decisions differ"
          % (err.size, np.median(err), np.quantile(err, 0.99), err.max(), n_dec))
    assert err.size > 300000
    assert err.max() <= 1e-4
    assert n_dec <= max(2, err.size // 10000)
