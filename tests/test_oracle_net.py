"""The float64 network of oracle/net.py (the reference for the GPU's
gradients) pinned by finite differences and by the adjointness of its
im2col / col2im pair."""
import numpy as np

from oracle import net as onet


def _params(rng, scale=0.05):
    n = sum(s.stop - s.start for s in onet.block_slices().values())
    return rng.normal(0.0, scale, n)


def test_im2col_col2im_adjoint():
    rng = np.random.default_rng(1)
    x = rng.normal(size=(2, 32, 64))
    y = rng.normal(size=(2, 16, 320))
    assert abs(np.sum(onet.im2col(x) * y) - np.sum(x * onet.col2im(y, 32))) < 1e-9


def test_backward_matches_finite_differences():
    rng = np.random.default_rng(2)
    p = _params(rng)
    X = rng.normal(0.5, 1.0, size=(3, 256, 64))
    label = np.array([17, 4096, 2000])
    tl = np.array([3.0, 0.0, -7.5])
    ml = np.array([2.7, 0.0, 3.3])
    loss, g = onet.loss_and_grad(p, X, label, tl, ml)
    sl = onet.block_slices()
    h = 1e-6
    for name, s in sl.items():
        for i in rng.choice(np.arange(s.start, s.stop), size=3, replace=False):
            pp, pm = p.copy(), p.copy()
            pp[i] += h
            pm[i] -= h
            fd = (onet.loss_and_grad(pp, X, label, tl, ml)[0] - onet.loss_and_grad(pm, X, label, tl, ml)[0]) / (2 * h)
            assert abs(fd - g[i]) <= 1e-5 * max(1.0, abs(fd)), (name, i, fd, g[i])
