"""The learned-proposal network on the GPU: its BF16 tensor-core forward and
backward against the float64 numpy network of the oracle, and what training
on simulated windows gains."""
import numpy as np
import pytest

import worldgen
from gpu_helpers import lib, small_world
from oracle import net as onet

pytestmark = pytest.mark.gpu


def bf16(a):
    """Round to the nearest bfloat16 (ties to even), as float64."""
    b = np.ascontiguousarray(a, dtype=np.float32).view(np.uint32).astype(np.uint64)
    b = ((b + 0x7FFF + ((b >> 16) & 1)) >> 16) << 16
    return b.astype(np.uint32).view(np.float32).astype(np.float64)


def bf16_rounded_gradients(p, X, label, tl, ml):
    """The gradient with BF16 rounding where the kernels store a product
    operand in BF16 (parameters, input, every layer's activation, the output
    gradient, the hidden and convolution gradients), everything else in
    float64.  Test-only model of the kernels' precision, to separate rounding
    from a wrong index: it shares the float64 definition's building blocks."""
    sl = onet.block_slices()
    q = onet.unpack(bf16(p))
    x = bf16(X)
    B = len(X)
    cache = []
    for l in range(4):
        A = onet.im2col(x)
        y = np.maximum(A @ q["W%d" % l].T + p[sl["b%d" % l]], 0.0)
        cache.append((A, y))
        x = bf16(y)
    x4 = x.reshape(B, onet.F1IN)
    h = np.maximum(x4 @ q["F1"].T + p[sl["fb1"]], 0.0)
    hb = bf16(h)
    o = hb @ q["F2"].T + p[sl["fb2"]]
    # the output gradient is the definition's, taken at these outputs
    z = o[:, :onet.NPIX + 1]
    e = np.exp(z - z.max(axis=1, keepdims=True))
    dO = np.zeros_like(o)
    dO[:, :onet.NPIX + 1] = e / e.sum(axis=1, keepdims=True)
    dO[np.arange(B), label] -= 1.0
    for b in range(B):
        if label[b] >= onet.NPIX:
            continue
        for j, yv in enumerate((tl[b], ml[b])):
            mu, raw = o[b, onet.NPIX + 1 + 2 * j], o[b, onet.NPIX + 2 + 2 * j]
            iv = np.exp(-2.0 * min(max(raw, -4.0), 6.0))
            r = yv - mu
            dO[b, onet.NPIX + 1 + 2 * j] = -r * iv
            dO[b, onet.NPIX + 2 + 2 * j] = (1.0 - r * r * iv) if -4.0 < raw < 6.0 else 0.0
    dOb = bf16(dO / B)
    g = {"F2": dOb.T @ hb, "fb2": dOb.sum(axis=0)}
    dhb = bf16((dOb @ q["F2"]) * (h > 0))
    g["F1"], g["fb1"] = dhb.T @ x4, dhb.sum(axis=0)
    dy = (dhb @ q["F1"]).reshape(B, 16, onet.C)
    L = [256, 128, 64, 32, 16]
    for l in range(3, -1, -1):
        A, y = cache[l]
        dy = bf16(dy * (y > 0))
        g["W%d" % l], g["b%d" % l] = np.einsum("bto,btk->ok", dy, A), dy.sum(axis=(0, 1))
        if l > 0:
            dy = onet.col2im(dy @ q["W%d" % l], L[l])
    return g


def test_forward_and_gradients_match_float64_oracle():
    """Forward within 3e-2 of the float64 network.  Gradients: within 2e-2 of
    the same definition with the kernels' BF16 operand roundings, and within
    twice that rounding's own distance from float64 (+2e-2) of the float64
    gradient -- at batch 4 BF16 alone moves the deepest blocks by ~8%, while
    a wrong index or transposition moves a block by ~100%."""
    cm = lib()
    net = cm.Net(max_batch=8, seed=5)
    p = net.params()
    rng = np.random.default_rng(3)
    X = np.log1p(rng.normal(0.0, 1.5, size=(4, 256, 64)) ** 2).astype(np.float32)
    label = np.array([100, 4096, 2500, 7], dtype=np.int32)
    tl = np.array([3.0, 0.0, -7.5, 20.0], dtype=np.float32)
    ml = np.array([2.7, 0.0, 3.3, 2.1], dtype=np.float32)
    o_gpu = net.forward(X)
    o_orc, _ = onet.forward(bf16(p), bf16(X))
    rel = np.linalg.norm(o_gpu - o_orc) / np.linalg.norm(o_orc)
    print("forward rel err %.2e" % rel)
    assert rel < 3e-2
    g_gpu, l_gpu = net.gradients(X, label, tl, ml)
    l_orc, g_orc = onet.loss_and_grad(bf16(p), bf16(X), label, tl, ml)
    print("loss gpu %.5f oracle %.5f" % (l_gpu, l_orc))
    assert abs(l_gpu - l_orc) <= 2e-2 * max(1.0, abs(l_orc))
    g_bf = bf16_rounded_gradients(p.astype(np.float64), X.astype(np.float64), label, tl.astype(np.float64),
                                  ml.astype(np.float64))
    for name, s in onet.block_slices().items():
        ref = max(np.linalg.norm(g_orc[s]), 1e-12)
        e64 = np.linalg.norm(g_gpu[s] - g_orc[s]) / ref
        ebf = np.linalg.norm(g_gpu[s] - g_bf[name].ravel()) / max(np.linalg.norm(g_bf[name]), 1e-12)
        eround = np.linalg.norm(g_bf[name].ravel() - g_orc[s]) / ref
        print("grad %-4s vs float64 %.2e  vs BF16-rounded %.2e  (rounding alone %.2e)" % (name, e64, ebf, eround))
        assert ebf < 2e-2, name
        assert e64 < 2.0 * eround + 2e-2, name
    net.destroy()


@pytest.fixture(scope="module")
def trained():
    """A network trained on 512k simulated windows and the birth table (with
    magnitude centres) it makes from the signals of the 1000 km, 1 h,
    100-station float32 world."""
    cm = lib()
    w = worldgen.config_learned(seed=1000)
    m = cm.create_model(None, w.stations, w.signals,
                        cm.make_params(w.params, k_per_phase=32, seed=1, dtype=cm.F32))
    net = cm.Net(max_batch=256, seed=7)
    l0 = net.train(m, 1, 256, 1e-3)
    l1 = net.train(m, 2000, 256, 3e-4)
    tiles, origins = cm.grid_tiles(10, 100.0)
    tab, centre = net.birth_table(m, tiles, origins, 80, 80, 360, hop_s=12.8, magnitudes=True)
    yield cm, w, (l0, l1), (tab, centre)
    net.destroy()
    m.destroy()


def test_training_concentrates_the_birth_table_on_events(trained):
    cm, w, (l0, l1), (tab, centre) = trained
    print("loss %.3f -> %.3f" % (l0, l1))
    assert l1 < l0 - 2.0
    tab = tab.astype(np.float64)
    assert np.all(np.isfinite(tab)) and tab.sum() > 0
    nx, nt = tab.shape[1], tab.shape[2]
    dens = tab / tab.sum()
    det = np.array([np.min(np.hypot(w.stations[:, 0] - e[0], w.stations[:, 1] - e[1])) < w.params.R_max
                    for e in w.events])
    vals = []
    for x, y, t, mag in w.events[det]:
        ix, iy, b = int(x / w.params.W * nx), int(y / w.params.W * nx), int(t / w.params.T * nt)
        vals.append(dens[max(0, iy - 2):iy + 3, max(0, ix - 2):ix + 3, max(0, b - 1):b + 2].mean())
    gain = np.mean(vals) / dens.mean()
    print("table density near detectable events / mean density: %.1f" % gain)
    assert gain > 4.0
    assert np.all(np.isfinite(centre)) and centre.min() > 0.0


def test_learned_proposal_reaches_f1_sooner(trained):
    """What the network gains: from the empty hypothesis, the 50/50 mixture
    with the network's table and magnitudes (window half-width 0.3) finds the
    detectable events sooner and sheds the spurious ones sooner than the
    plain sampler.  Over 4 chains each: mean recall after 5 sweeps, and the
    sweeps to F1 >= 0.9 (detectable zone, checked every 5 sweeps; measured
    30-40 against 165-235)."""
    cm, w, _, (tab, centre) = trained
    from paper_1612_00595_gb300 import metrics
    P = w.params
    rec = {"plain": [], "learned": []}
    hit = {"plain": [], "learned": []}
    for seed in (7, 8, 9, 10):
        for kind in rec:
            m = cm.create_model(None, w.stations, w.signals,
                                cm.make_params(P, k_per_phase=32, seed=seed, dtype=cm.F32))
            m.partition_and_color(P.L)
            if kind == "learned":
                m.set_birth_table(tab, 0.5)
                m.set_birth_magnitude(centre, 0.3)
            first = 400
            for done in range(5, 405, 5):
                m.run_sweeps(5)
                sc = metrics.scores(w.events, m.read_state()[0], P.L, P.tau, w.stations, P.R_max)
                if done == 5:
                    rec[kind].append(sc["recall"])
                if sc["f1"] >= 0.9:
                    first = done
                    break
            hit[kind].append(first)
            m.destroy()
    print("recall after 5 sweeps: plain %s learned %s" % (np.round(rec["plain"], 3), np.round(rec["learned"], 3)))
    print("sweeps to F1 >= 0.9: plain %s learned %s" % (hit["plain"], hit["learned"]))
    assert np.mean(rec["learned"]) > np.mean(rec["plain"]) + 0.1
    assert max(hit["learned"]) < min(hit["plain"])


def test_training_on_the_additive_reading():
    """The window simulator follows the model's reading (arrivals add to the
    sample mean here): after training on such windows, the table made from a
    world of that reading concentrates on its detectable events."""
    cm = lib()
    w = small_world(seed=43, W=1000.0, T=1800.0, Lambda=250.0, n_side=10, dtype=np.float32, likelihood="mean")
    m = cm.create_model(None, w.stations, w.signals, cm.make_params(w.params, k_per_phase=32, seed=1, dtype=cm.F32))
    net = cm.Net(max_batch=256, seed=9)
    l0 = net.train(m, 1, 256, 3e-4)
    l1 = net.train(m, 2000, 256, 3e-4)
    tab = net.birth_table(m, *cm.grid_tiles(10, 100.0), 80, 80, 180, hop_s=12.8).astype(np.float64)
    dens = tab / tab.sum()
    det = np.array([np.min(np.hypot(w.stations[:, 0] - e[0], w.stations[:, 1] - e[1])) < w.params.R_max
                    for e in w.events])
    vals = [dens[max(0, iy - 2):iy + 3, max(0, ix - 2):ix + 3, max(0, b - 1):b + 2].mean()
            for ix, iy, b in ((int(x / w.params.W * 80), int(y / w.params.W * 80), int(t / w.params.T * 180))
                              for x, y, t, _ in w.events[det])]
    gain = np.mean(vals) / dens.mean()
    print("loss %.3f -> %.3f, table density near detectable events / mean: %.1f" % (l0, l1, gain))
    assert np.isfinite(l1) and l1 < l0
    assert gain > 4.0
    net.destroy()
    m.destroy()
