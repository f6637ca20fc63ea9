"""Shared helpers of the GPU tests: run the CUDA path and the oracle on the same
seeded world and line their per-step traces up by (sweep, cell, step)."""
import numpy as np

import worldgen

TRACE_KEYS = ["sweep", "cell", "step"]


def lib():
    import __graft_entry__
    __graft_entry__.build()
    import paper_1612_00595_gb300 as cm
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    return cm


def small_world(seed=5, W=500.0, T=1200.0, Lambda=60.0, n_side=5, dtype=np.float64, **kw):
    p = worldgen.ModelParams(W=W, T=T, Lambda=Lambda, **kw)
    return worldgen.make_world(p, worldgen.jittered_grid_stations(n_side, W, seed), seed, dtype)


def run_gpu(cm, world, *, sweeps, k=16, seed=11, dtype=None, shift_mode=1, sx=0.0, sy=0.0, events=None,
            commit=True, trace=True, on_device=False, **pkw):
    if dtype is None:
        dtype = cm.F32 if world.signals.dtype == np.float32 else cm.F64
    params = cm.make_params(world.params, k_per_phase=k, seed=seed, dtype=dtype, commit=commit, **pkw)
    sig = world.signals
    if on_device:
        import torch
        sig = torch.from_numpy(np.ascontiguousarray(sig)).cuda()
    m = cm.create_model(events, world.stations, sig, params)
    m.partition_and_color(world.params.L, shift_mode=shift_mode, sx=sx, sy=sy)
    ncx = int(np.floor(world.params.W / world.params.L)) + 2
    if trace:
        m.set_trace(sweeps * ncx * ncx * k)
    m.run_sweeps(sweeps)
    ev, ids, logp, stats = m.read_state()
    tr = np.sort(m.read_trace(), order=TRACE_KEYS) if trace else None
    return m, ev, ids, logp, stats, tr


def run_oracle(orc, world, *, sweeps, k=16, seed=11, shift_mode=1, sx=0.0, sy=0.0, events=None, commit=True,
               threads=1, **okw):
    o = orc.World(world, k_per_phase=k, seed=seed, commit=commit, **okw)
    ev0 = np.zeros((0, 4)) if events is None else events
    ncx = int(np.floor(world.params.W / world.params.L)) + 2
    ev, ids, tr, dlp = o.run_chromatic(ev0, sweeps, shift_mode=shift_mode, sx=sx, sy=sy,
                                       trace_cap=sweeps * ncx * ncx * k + 16, threads=threads)
    return o, ev, ids, np.sort(tr, order=TRACE_KEYS), dlp


def assert_traces_match(tr, otr, rtol=1e-9):
    assert len(tr) == len(otr) > 0, (len(tr), len(otr))
    for key in ("sweep", "cell", "step", "type", "evaluated", "n_before"):
        assert np.array_equal(tr[key], otr[key]), key
    bad = np.nonzero(tr["accepted"] != otr["accepted"])[0]
    assert len(bad) == 0, "accept decisions differ at %s" % bad[:5]
    ev = otr["evaluated"] == 1
    # relative to max(|dll|, 1): a change below 1 in magnitude is a sum of
    # per-sample terms of either sign, each of order 1 and rounded at that
    # scale, so below 1 the bound is absolute; the pure relative error is
    # printed beside it
    scale = np.maximum(np.abs(otr["dll"][ev]), 1.0)
    err = np.abs(tr["dll"][ev] - otr["dll"][ev]) / scale
    with np.errstate(divide="ignore", invalid="ignore"):
        rel = np.abs(tr["dll"][ev] - otr["dll"][ev]) / np.abs(otr["dll"][ev])
    rel = rel[np.isfinite(rel)]
    print("dll: %d evaluated, max err %.3g (scale max(|x|,1)), max pure relative %.3g, %d with |dll| < 1"
          % (int(ev.sum()), err.max(initial=0.0), rel.max(initial=0.0), int((np.abs(otr["dll"][ev]) < 1).sum())))
    assert err.max(initial=0.0) <= rtol, err.max()
    la_err = np.abs(tr["log_alpha"][ev] - otr["log_alpha"][ev]) / np.maximum(np.abs(otr["log_alpha"][ev]), 1.0)
    assert la_err.max(initial=0.0) <= rtol, la_err.max()
    assert np.all(np.isneginf(tr["log_alpha"][~ev])) and np.all(np.isneginf(otr["log_alpha"][~ev]))
