"""The C-ABI library loads and exports every call include/chromh.h declares,
and its host-side argument checks answer without touching a GPU."""
import ctypes as C
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def cm():
    import __graft_entry__
    __graft_entry__.build()
    import paper_1612_00595_gb300 as cm
    return cm


def _declared():
    hdr = open(os.path.join(ROOT, "include", "chromh.h")).read()
    hdr = re.sub(r"/\*.*?\*/", "", hdr, flags=re.S)
    return sorted(set(re.findall(r"\b(cmh_[a-z0-9_]+)\s*\(", hdr)))


def test_every_declared_symbol_is_exported(cm):
    names = _declared()
    assert "cmh_create_model" in names and "cmh_run_sweeps" in names
    for n in names:
        assert hasattr(cm.lib, n), n
    assert sorted(cm.EXPORTS) == names


def test_strerror(cm):
    for code in range(0, -9, -1):
        assert cm.strerror(code)
    assert cm.strerror(-8) == "call out of order or error latched"


def _params(cm, **kw):
    import worldgen
    return cm.make_params(worldgen.ModelParams(W=200.0, T=60.0, Lambda=5.0), **kw)


@pytest.mark.parametrize("bad", [
    dict(p_birth=0.6, p_death=0.5),
    dict(k_per_phase=0),
    dict(k_per_phase=5000),
    dict(block_threads=100),
    dict(stage_samples=-2),
    dict(schedule=2),
    dict(ctas_per_sm=4),
    dict(dtype=7),
    dict(likelihood=2),
    dict(likelihood=1, dtype=0),   # the additive-mean reading is float32 only
    dict(p_pair=-0.1),
    dict(p_pair=0.6),              # p_birth + p_death + p_pair > 1
    dict(p_pair=0.2, dtype=1, stage_samples=-1),   # joint moves read windows from global memory
    dict(p_pair=0.2, dtype=1, likelihood=1),        # joint moves under the variance reading
    dict(sig_a=-1.0),
    dict(sig_a=2.0, dtype=1, stage_samples=-1),   # float32 latent arrivals read windows from global memory
    dict(sig_a=2.0, dtype=1, likelihood=1),        # latent arrivals under the variance reading
    dict(p_arr=0.1),               # the arrival-time move needs latent arrivals
    dict(sig_a=2.0, p_arr=0.1, sig_da=0.0),
    dict(sig_a=2.0, p_pair=0.3, p_arr=0.3),   # p_birth + p_death + p_pair + p_arr > 1
])
def test_create_model_rejects_bad_params_on_host(cm, bad):
    lik = bad.pop("likelihood", None)
    p = _params(cm, **bad)
    if lik is not None:
        p.likelihood = lik
    h = C.c_void_p()
    st = np.zeros((1, 2))
    sig = np.zeros((1, 10))
    rc = cm.lib.cmh_create_model(
        None, 0, C.c_void_p(st.ctypes.data), 1, C.c_void_p(sig.ctypes.data), 10, 10, 1, 0, C.byref(p), None,
        C.byref(h))
    assert rc == -1 and not h.value


def test_create_model_rejects_bad_events_on_host(cm):
    p = _params(cm)
    st = np.zeros((1, 2))
    sig = np.zeros((1, 10))
    h = C.c_void_p()
    for ev, code in [([[np.nan, 1.0, 1.0, 3.0]], -3), ([[250.0, 1.0, 1.0, 3.0]], -1),
                     ([[10.0, 1.0, 1.0, 1.5]], -1)]:
        e = np.array(ev, dtype=np.float64)
        rc = cm.lib.cmh_create_model(C.c_void_p(e.ctypes.data), 1, C.c_void_p(st.ctypes.data), 1,
                                     C.c_void_p(sig.ctypes.data), 10, 10, 1, 0, C.byref(p), None, C.byref(h))
        assert rc == code
    # sizes
    rc = cm.lib.cmh_create_model(None, 0, C.c_void_p(st.ctypes.data), 1, C.c_void_p(sig.ctypes.data), 10, 5, 1,
                                 0, C.byref(p), None, C.byref(h))
    assert rc == -1
    rc = cm.lib.cmh_create_model(None, 0, None, 1, None, 10, 10, 1, 0, C.byref(p), None, C.byref(h))
    assert rc == -1


def test_null_handles(cm):
    assert cm.lib.cmh_run_sweeps(None, 1) == -1
    assert cm.lib.cmh_sync(None) == -1
    assert cm.lib.cmh_read_state(None, None, None, 0, None, None, None) == -1
    assert cm.lib.cmh_philox4x64(None, None, None, -1) == -1
    cm.lib.cmh_destroy(None)
    h = C.c_void_p()
    assert cm.lib.cmh_batch_create(None, 0, None, C.byref(h)) == -1 and not h.value
    arr = (C.c_void_p * 1)(None)
    assert cm.lib.cmh_batch_create(arr, 1, None, C.byref(h)) == -1 and not h.value
    assert cm.lib.cmh_batch_run_sweeps(None, 1) == -1
    cm.lib.cmh_batch_destroy(None)
    n = C.c_int64()
    assert cm.lib.cmh_set_arrival_offsets(None, None, 0, 0) == -1
    assert cm.lib.cmh_read_arrival_offsets(None, None, 0, C.byref(n)) == -1


def test_null_handles_of_the_learned_proposal_and_async_reads(cm):
    f = np.zeros(4, dtype=np.float32)
    assert cm.lib.cmh_set_birth_table(None, None, 0, 0, 0, 0.0) == -1
    assert cm.lib.cmh_set_birth_magnitude(None, None, 0.0) == -1
    assert cm.lib.cmh_read_state_async(None, 0) == -1
    assert cm.lib.cmh_read_state_fetch(None, 0, None, None, 0, None, None, None) == -1
    assert cm.lib.cmh_autotune(None, 1, None) == -1
    assert cm.lib.cmh_batch_sync(None) == -1
    h = C.c_void_p()
    assert cm.lib.cmh_net_create(0, 1, None, C.byref(h)) == -1 and not h.value
    assert cm.lib.cmh_net_create(4097, 1, None, C.byref(h)) == -1 and not h.value
    assert cm.lib.cmh_net_forward(None, C.c_void_p(f.ctypes.data), 1, C.c_void_p(f.ctypes.data)) == -1
    assert cm.lib.cmh_net_train(None, None, 1, 1, 1e-3, None) == -1
    assert cm.lib.cmh_net_get_params(None, C.c_void_p(f.ctypes.data)) == -1
    assert cm.lib.cmh_net_birth_table(None, None, None, None, 1, 1, 1, 1, 1.0, None, None) == -1
    assert cm.lib.cmh_net_param_count() > 2_000_000
    cm.lib.cmh_net_destroy(None)


def test_alu_peaks_rejects_null_pointers(cm):
    out = C.c_double()
    assert cm.lib.cmh_measure_alu_peaks(None, C.byref(out), None) == -1
    assert cm.lib.cmh_measure_alu_peaks(C.byref(out), None, None) == -1
