"""The measurements bench.py builds its roofline from: the device's MUFU and
float32 FMA throughput, and the count of unique window samples a region
phase touches."""
import numpy as np
import pytest

from gpu_helpers import lib, small_world

pytestmark = pytest.mark.gpu


def test_alu_peaks_are_plausible():
    cm = lib()
    mufu, fma = cm.measure_alu_peaks()
    print("MUFU %.3g ops/s, FMA %.3g flop/s" % (mufu, fma))
    # a GB300 (152 SMs, ~2 GHz) does on the order of 5e12 special-function
    # operations and 8e13 float32 flops per second
    assert 1e12 < mufu < 1e14
    assert 1e13 < fma < 5e14
    assert fma > 4 * mufu


@pytest.mark.parametrize("k", [1, 16])
def test_unique_samples_counted_only_while_timing(k):
    """With one step per region phase the union of the priced windows is the
    priced width itself; with more steps it is at most that.  Untimed sweeps
    count nothing."""
    cm = lib()
    w = small_world(seed=41, W=1000.0, T=3600.0, Lambda=500.0, n_side=10, dtype=np.float32)
    m = cm.create_model(w.events, w.stations, w.signals, cm.make_params(w.params, k_per_phase=k, seed=3,
                                                                       dtype=cm.F32))
    m.partition_and_color(w.params.L, 1)
    m.run_sweeps(2)
    _, _, _, s0 = m.read_state(cap=0)
    assert s0["unique_samples"] == 0
    m.set_timing(True)
    m.run_sweeps(4)
    m.set_timing(False)
    _, _, _, s1 = m.read_state(cap=0)
    priced = s1["priced_samples"] - s0["priced_samples"]
    unique = s1["unique_samples"]
    assert priced > 0
    if k == 1:
        assert unique == priced
    else:
        assert 0 < unique < priced
    m.run_sweeps(2)
    _, _, _, s2 = m.read_state(cap=0)
    assert s2["unique_samples"] == unique
    m.destroy()
