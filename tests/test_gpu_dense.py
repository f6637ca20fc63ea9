"""Regions too large for shared memory (dense stations): their arrival caches
and station lists live in a global slot per CTA.  The float32 sweep there
prices the same Δℓ as the oracle, and such a model runs in a batch exactly as
alone."""
import os

import numpy as np
import pytest

import worldgen
from gpu_helpers import TRACE_KEYS, lib

pytestmark = pytest.mark.gpu


def dense_world(seed=31):
    """300 x 300 km, 10 min, Lambda 200, 256 uniform stations: ~130 stations
    in a region's blanket, ~40 within R_max of a point."""
    p = worldgen.ModelParams(W=300.0, T=600.0, Lambda=200.0)
    return worldgen.make_world(p, worldgen.uniform_stations(256, p.W, seed), seed, np.float32)


@pytest.fixture(scope="module")
def cm():
    return lib()


@pytest.fixture(scope="module")
def orc():
    import oracle
    return oracle


def test_dense_dry_run_matches_oracle(cm, orc):
    w = dense_world()
    params = cm.make_params(w.params, k_per_phase=32, seed=5, dtype=cm.F32, commit=False)
    m = cm.create_model(w.events, w.stations, w.signals, params)
    m.partition_and_color(w.params.L, 1)
    assert m.read_state(cap=0)[3]["spill_bytes"] > 0
    ncx = int(np.floor(w.params.W / w.params.L)) + 2
    m.set_trace(3 * ncx * ncx * 32)
    m.run_sweeps(3)
    tr = np.sort(m.read_trace(), order=TRACE_KEYS)
    o = orc.World(w, k_per_phase=32, seed=5, commit=False)
    _, _, otr, _ = o.run_chromatic(w.events, 3, trace_cap=100000, threads=min(16, os.cpu_count() or 1))
    otr = np.sort(otr, order=TRACE_KEYS)
    assert len(tr) == len(otr)
    for key in ("sweep", "cell", "step", "type", "n_before"):
        assert np.array_equal(tr[key], otr[key]), key
    ev_ = (otr["evaluated"] == 1) & (tr["evaluated"] == 1)
    assert ev_.sum() > 500
    err = np.abs(tr["dll"][ev_] - otr["dll"][ev_]) / np.maximum(np.abs(otr["dll"][ev_]), 1.0)
    assert err.max() <= 1e-4
    m.destroy()


def test_dense_model_in_a_batch_equals_alone(cm):
    worlds = [dense_world(31), worldgen.config_scale(seed=7, side_regions=4, T=1200.0)]
    def make():
        ms = []
        for i, w in enumerate(worlds):
            m = cm.create_model(w.events, w.stations, w.signals,
                                cm.make_params(w.params, k_per_phase=16, seed=40 + i, dtype=cm.F32))
            m.partition_and_color(w.params.L, 1)
            ms.append(m)
        return ms
    alone = make()
    for m in alone:
        m.run_sweeps(4)
    ref = [m.read_state() for m in alone]
    batched = make()
    b = cm.create_batch(batched)
    b.run_sweeps(4)
    b.sync()
    got = [m.read_state() for m in batched]
    for (e0, i0, l0, _), (e1, i1, l1, _) in zip(ref, got):
        assert np.array_equal(e0, e1) and np.array_equal(i0, i1) and l0 == l1
    b.destroy()
    for m in alone + batched:
        m.destroy()
