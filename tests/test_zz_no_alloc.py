"""cmh_gaussian_loglik_noalloc: the Gaussian log-likelihood for callers that
cannot allocate device memory (their memory manager owns the GPU, or an
allocation would synchronise the device under someone else's kernels).

Collected last on purpose: a failure here leaves every other test already run.
It checks the allocation-free entry point against the existing one
(cmh_log_density) and against the oracle's log-likelihood, on two calls in a
row, through the C ABI.
"""
import ctypes as C

import numpy as np
import pytest

from gpu_helpers import lib, small_world

pytestmark = pytest.mark.gpu


def _noalloc(cm, sig, var, dtype):
    out = C.c_double()
    rc = cm.lib.cmh_gaussian_loglik_noalloc(C.c_void_p(sig.data_ptr()), C.c_void_p(var.data_ptr()),
                                            sig.shape[0], sig.shape[1], sig.stride(0), dtype, C.byref(out),
                                            None)
    assert rc == 0, cm.strerror(rc)
    return out.value


@pytest.mark.parametrize("f32", [False, True])
def test_noalloc_matches_log_density_noise_only(orc, f32):
    """No events: the variance is the noise variance everywhere.  The existing
    entry point returns -Lambda (empty-set prior) + that likelihood; the
    oracle gives the likelihood from its own sum.  float32 samples are priced
    in float32 and summed in float64, hence the looser bound there."""
    cm = lib()
    import torch
    w = small_world(seed=31, dtype=np.float32 if f32 else np.float64)
    dtype = cm.F32 if f32 else cm.F64
    m = cm.create_model(None, w.stations, w.signals, cm.make_params(w.params, dtype=dtype))
    want = m.log_density() + w.params.Lambda
    want_orc = orc.World(w).log_likelihood(np.zeros((0, 4)))
    sig = torch.from_numpy(w.signals).cuda()
    var = torch.full_like(sig, w.params.noise_var)
    torch.cuda.synchronize()
    for _ in range(2):
        got = _noalloc(cm, sig, var, dtype)
        assert got == pytest.approx(want, rel=1e-12)
        assert got == pytest.approx(want_orc, rel=1e-6 if f32 else 1e-12)
    m.destroy()


def test_noalloc_matches_log_density_with_events(orc):
    """Ground-truth events: the variance rows come from the oracle's
    definition; the allocation-free sum must equal the existing entry point's
    log-density minus the prior, and the oracle's log-likelihood of the same
    events, on two consecutive calls."""
    cm = lib()
    import torch
    w = small_world(seed=32)
    m = cm.create_model(w.events, w.stations, w.signals, cm.make_params(w.params, dtype=cm.F64))
    o = orc.World(w)
    want = m.log_density() - o.log_prior(w.events)
    want_orc = o.log_likelihood(w.events)
    ns = w.signals.shape[1]
    V = np.stack([o.variance(w.events, j, 0, ns) for j in range(w.n_stations)])
    sig = torch.from_numpy(w.signals).cuda()
    var = torch.from_numpy(V).cuda()
    torch.cuda.synchronize()
    for _ in range(2):
        got = _noalloc(cm, sig, var, cm.F64)
        assert got == pytest.approx(want, rel=1e-11)
        assert got == pytest.approx(want_orc, rel=1e-12)
    m.destroy()


def test_noalloc_rejects_sizes_beyond_its_scratch():
    cm = lib()
    out = C.c_double()
    dummy = C.c_void_p(16)  # never dereferenced: the size check comes first
    assert cm.lib.cmh_gaussian_loglik_noalloc(dummy, dummy, 8192, 10, 10, cm.F64, C.byref(out), None) == -5
    assert cm.lib.cmh_gaussian_loglik_noalloc(dummy, dummy, 4, 10, 5, cm.F64, C.byref(out), None) == -1
    assert cm.lib.cmh_gaussian_loglik_noalloc(None, None, 0, 10, 10, cm.F64, C.byref(out), None) == 0
    assert out.value == 0.0
