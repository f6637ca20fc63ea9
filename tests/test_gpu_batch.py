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
