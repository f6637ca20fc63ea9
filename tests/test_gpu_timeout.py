"""A bounded device wait that runs out.

The persistent float32 sweep lets a region start only after its neighbouring
regions of lower colours have announced the end of their phase; each poll of
such an announcement is bounded.  cmh_test_hold_region makes one region never
announce (a flag that nothing sets), so its higher-colour neighbours' waits
run out: the sweep latches CMH_ERR_TIMEOUT, the model refuses further work,
and the GPU stays usable -- a fresh model on it runs and agrees with a model
run before the failure.  No GPU fault is involved."""
import numpy as np
import pytest

from gpu_helpers import lib, small_world

pytestmark = pytest.mark.gpu


def _model(cm, w, seed=5):
    m = cm.create_model(w.events, w.stations, w.signals,
                        cm.make_params(w.params, k_per_phase=8, seed=seed, dtype=cm.F32))
    m.partition_and_color(w.params.L, 1)
    return m


def test_neighbour_wait_runs_out_and_latches_timeout():
    cm = lib()
    w = small_world(seed=51, W=1000.0, T=1800.0, Lambda=250.0, n_side=10, dtype=np.float32)
    ref = _model(cm, w)
    ref.run_sweeps(3)
    ev_ref, ids_ref, lp_ref, _ = ref.read_state()
    ref.destroy()

    m = _model(cm, w)
    m.run_sweeps(1)
    m.sync()
    # cell (2, 2) of the 12 x 12 grid: colour 0, inside the domain, with
    # live neighbours of the three other colours
    ncx = int(np.floor(w.params.W / w.params.L)) + 2
    m.test_hold_region(2 * ncx + 2, wait_limit=256)
    m.run_sweeps(1)
    with pytest.raises(cm.ChromhError) as ei:
        m.sync()
    assert ei.value.code == -6   # CMH_ERR_TIMEOUT
    with pytest.raises(cm.ChromhError) as ei:
        m.run_sweeps(1)
    assert ei.value.code == -8   # CMH_ERR_STATE
    m.destroy()

    # the GPU is still usable: a fresh model gives the same chain as before
    m2 = _model(cm, w)
    m2.run_sweeps(3)
    ev, ids, lp, _ = m2.read_state()
    assert np.array_equal(ids, ids_ref) and np.array_equal(ev, ev_ref) and lp == lp_ref
    m2.destroy()


def test_hold_hook_off_leaves_the_chain_unchanged():
    """Turning the hook on and off again (cell -1) changes nothing."""
    cm = lib()
    w = small_world(seed=52, W=1000.0, T=1800.0, Lambda=250.0, n_side=10, dtype=np.float32)
    a, b = _model(cm, w, seed=9), _model(cm, w, seed=9)
    b.test_hold_region(-1, wait_limit=1 << 20)
    for m in (a, b):
        m.run_sweeps(4)
    ea, ia, la, _ = a.read_state()
    eb, ib, lb, _ = b.read_state()
    assert np.array_equal(ia, ib) and np.array_equal(ea, eb) and la == lb
    a.destroy()
    b.destroy()
