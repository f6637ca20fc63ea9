"""Chain summaries: the float32 GPU sampler and the float64 oracle sample the
same posterior.  R independent chains per side (different seeds) start from
the generated ground truth; each chain's precision, recall, F1 and mean
location error against the ground truth (detectable zone) and its event
count are averaged over the second half of its sweeps, and the GPU mean
over chains must lie within 4 combined standard errors of the oracle mean.
"""
import os

import numpy as np
import pytest

from gpu_helpers import lib, small_world
from oracle import metrics as om

pytestmark = pytest.mark.gpu

R = 10
SWEEPS, EVERY, K = 160, 8, 32
KEYS = ("n_events", "precision", "recall", "f1", "loc_err")


def _summary(world, ev):
    s = om.scores(world.events, ev, world.params.L, world.params.tau, stations=world.stations,
                  R_max=world.params.R_max)
    return [float(len(ev)), s["precision"], s["recall"], s["f1"], s["loc_err"] if s["matched"] else 0.0]


def _gpu_chain(cm, world, seed):
    m = cm.create_model(world.events, world.stations, world.signals,
                        cm.make_params(world.params, k_per_phase=K, seed=seed, dtype=cm.F32))
    m.partition_and_color(world.params.L, shift_mode=1)
    out = []
    for s in range(0, SWEEPS, EVERY):
        m.run_sweeps(EVERY)
        if s + EVERY > SWEEPS // 2:
            ev, _, _, _ = m.read_state()
            out.append(_summary(world, ev))
    m.destroy()
    return np.mean(out, axis=0)


def _oracle_chain(orc, world, seed, threads):
    o = orc.World(world, k_per_phase=K, seed=seed)
    ev, ids = world.events, None
    out = []
    for s in range(0, SWEEPS, EVERY):
        ev, ids, _, _ = o.run_chromatic(ev, EVERY, ids=ids, sweep0=s, threads=threads)
        if s + EVERY > SWEEPS // 2:
            out.append(_summary(world, ev))
    return np.mean(out, axis=0)


def test_fp32_chain_summaries_match_oracle_within_mc_error(orc):
    cm = lib()
    w = small_world(seed=31, W=400.0, T=1200.0, Lambda=30.0, n_side=4, dtype=np.float32)
    threads = min(16, os.cpu_count() or 1)
    g = np.array([_gpu_chain(cm, w, 500 + r) for r in range(R)])
    o = np.array([_oracle_chain(orc, w, 900 + r, threads) for r in range(R)])
    mg, mo = g.mean(axis=0), o.mean(axis=0)
    se = np.sqrt(g.var(axis=0, ddof=1) / R + o.var(axis=0, ddof=1) / R)
    for i, key in enumerate(KEYS):
        print("%-10s gpu %.4f  oracle %.4f  se %.4f" % (key, mg[i], mo[i], se[i]))
    # the sampler does something: it keeps most of the true detectable events
    assert mo[KEYS.index("recall")] > 0.5
    for i, key in enumerate(KEYS):
        assert abs(mg[i] - mo[i]) <= 4.0 * se[i] + 1e-9, key
