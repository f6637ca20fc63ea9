"""The learned-proposal network in plain float64 numpy (TEST INFRASTRUCTURE ONLY).

Only ``tests/`` may import this module; it shares no code with the CUDA
kernels.  It restates the network and its loss from their definitions:

  input   X[b, t, s]: 256 samples x 64 stations (channels)
  conv l = 1..4: y[b, t, o] = relu(b_l[o] + sum_{k<5, c<64} W_l[o, k*64 + c] x[b, 2t - 2 + k, c])
          (x = 0 outside [0, L_in)), 256 -> 128 -> 64 -> 32 -> 16 samples
  fc1     h = relu(F1 flat(y4) + fb1),  flat index t*64 + c
  fc2     o = F2 h + fb2, 4101 outputs: 4096 pixel logits, "no event",
          (mu_t, ls_t), (mu_m, ls_m)
  loss    mean over the batch of  -log softmax(o[:4097])[label]
          + [label < 4096] * sum over (t, m) of  ls + (y - mu)^2 / (2 e^{2 ls}),
          ls = clip(o, -4, 6) (no gradient where clipped)

Parameters are one flat vector in the order W1 b1 W2 b2 W3 b3 W4 b4 F1 fb1
F2 fb2.  Backward is the chain rule written out by hand.
"""
from __future__ import annotations

import numpy as np

C, KW, NPIX, NOUT, F1IN, F1OUT = 64, 5, 4096, 4101, 1024, 512
KC = C * KW


def unpack(p):
    p = np.asarray(p, dtype=np.float64)
    out, o = {}, 0
    for l in range(4):
        out["W%d" % l] = p[o:o + C * KC].reshape(C, KC); o += C * KC
        out["b%d" % l] = p[o:o + C]; o += C
    out["F1"] = p[o:o + F1OUT * F1IN].reshape(F1OUT, F1IN); o += F1OUT * F1IN
    out["fb1"] = p[o:o + F1OUT]; o += F1OUT
    out["F2"] = p[o:o + NOUT * F1OUT].reshape(NOUT, F1OUT); o += NOUT * F1OUT
    out["fb2"] = p[o:o + NOUT]; o += NOUT
    assert o == p.size
    return out


def im2col(x):
    """[B, L, 64] -> [B, L/2, 320]: column k*64 + c of row t is x[2t - 2 + k, c]."""
    B, L, _ = x.shape
    Lo = L // 2
    A = np.zeros((B, Lo, KC))
    for t in range(Lo):
        for k in range(KW):
            s = 2 * t - 2 + k
            if 0 <= s < L:
                A[:, t, k * C:(k + 1) * C] = x[:, s, :]
    return A


def col2im(dA, L):
    """Adjoint of im2col: [B, L/2, 320] -> [B, L, 64]."""
    B, Lo, _ = dA.shape
    dx = np.zeros((B, L, C))
    for t in range(Lo):
        for k in range(KW):
            s = 2 * t - 2 + k
            if 0 <= s < L:
                dx[:, s, :] += dA[:, t, k * C:(k + 1) * C]
    return dx


def forward(p, X):
    q = unpack(p)
    x = np.asarray(X, dtype=np.float64)
    cache = []
    for l in range(4):
        A = im2col(x)
        y = np.maximum(A @ q["W%d" % l].T + q["b%d" % l], 0.0)
        cache.append((A, y))
        x = y
    x4 = x.reshape(x.shape[0], F1IN)
    h = np.maximum(x4 @ q["F1"].T + q["fb1"], 0.0)
    o = h @ q["F2"].T + q["fb2"]
    return o, (q, cache, x4, h)


def loss_and_grad(p, X, label, t_label, m_label):
    o, (q, cache, x4, h) = forward(p, X)
    B = o.shape[0]
    label = np.asarray(label)
    z = o[:, :NPIX + 1]
    zmax = z.max(axis=1, keepdims=True)
    e = np.exp(z - zmax)
    sm = e / e.sum(axis=1, keepdims=True)
    lse = (zmax[:, 0] + np.log(e.sum(axis=1)))
    loss = lse - z[np.arange(B), label]
    dO = np.zeros_like(o)
    dO[:, :NPIX + 1] = sm
    dO[np.arange(B), label] -= 1.0
    for b in range(B):
        if label[b] >= NPIX:
            continue
        for j, y in enumerate((t_label[b], m_label[b])):
            mu, raw = o[b, NPIX + 1 + 2 * j], o[b, NPIX + 2 + 2 * j]
            ls = min(max(raw, -4.0), 6.0)
            iv = np.exp(-2.0 * ls)
            r = y - mu
            loss[b] += ls + 0.5 * r * r * iv
            dO[b, NPIX + 1 + 2 * j] = -r * iv
            dO[b, NPIX + 2 + 2 * j] = (1.0 - r * r * iv) if -4.0 < raw < 6.0 else 0.0
    dO /= B
    g = {}
    g["F2"] = dO.T @ h
    g["fb2"] = dO.sum(axis=0)
    dh = (dO @ q["F2"]) * (h > 0)
    g["F1"] = dh.T @ x4
    g["fb1"] = dh.sum(axis=0)
    dy = (dh @ q["F1"]).reshape(B, 16, C)
    L = [256, 128, 64, 32, 16]
    for l in range(3, -1, -1):
        A, y = cache[l]
        dy = dy * (y > 0)
        g["W%d" % l] = np.einsum("bto,btk->ok", dy, A)
        g["b%d" % l] = dy.sum(axis=(0, 1))
        if l > 0:
            dy = col2im(dy @ q["W%d" % l], L[l])
    flat = []
    for l in range(4):
        flat += [g["W%d" % l].ravel(), g["b%d" % l]]
    flat += [g["F1"].ravel(), g["fb1"], g["F2"].ravel(), g["fb2"]]
    return float(loss.mean()), np.concatenate(flat)


BLOCKS = ["W0", "b0", "W1", "b1", "W2", "b2", "W3", "b3", "F1", "fb1", "F2", "fb2"]


def block_slices():
    sizes = [C * KC, C] * 4 + [F1OUT * F1IN, F1OUT, NOUT * F1OUT, NOUT]
    out, o = {}, 0
    for name, n in zip(BLOCKS, sizes):
        out[name] = slice(o, o + n)
        o += n
    return out
