"""Invariants of the spatial partition (§Partitioning the World).

* Binning is a partition: every point of the domain lands in exactly one live
  cell, whose rectangle contains it.
* Every station an event can reach (distance < R_max) is in the blanket of the
  event's cell: the footprint of any event lies inside its region's blanket.
* Same-colour regions have disjoint blankets, for the 4-colour pattern at
  R_max = L/2 and the 9-colour pattern at R_max = L, under random shifts.
  Together with the previous item this is the conditional independence that
  lets same-colour regions run in parallel.
* Cells of one colour never touch (8-neighbourhood).
"""
import numpy as np
import pytest

import worldgen


def _world(R_max, n_st=300, W=1000.0, seed=0):
    p = worldgen.ModelParams(W=W, T=100.0, Lambda=1.0, R_max=R_max, L=100.0)
    st = worldgen.uniform_stations(n_st, W, seed)
    return worldgen.World(params=p, stations=st, signals=np.zeros((n_st, 0)), events=np.zeros((0, 4)))


@pytest.mark.parametrize("R_max,period", [(50.0, 2), (100.0, 3), (30.0, 2)])
def test_period(orc, R_max, period):
    assert orc.World(_world(R_max)).period() == period


@pytest.mark.parametrize("R_max", [50.0, 100.0])
def test_blankets_disjoint_and_cover_footprints(orc, R_max):
    w = _world(R_max)
    o = orc.World(w)
    rng = np.random.default_rng(1)
    ncx, ncy = o.grid_dims()
    st = w.stations
    for trial in range(12):
        sx, sy = (0.0, 0.0) if trial == 0 else tuple(rng.uniform(0, 100.0, 2))
        B = o.blankets(sx, sy).astype(bool)
        col = np.array([o.colour_of(c) for c in range(ncx * ncy)])
        for c in range(o.period() ** 2):
            # at most one region of each colour per station
            assert B[col == c].sum(axis=0).max() <= 1
        # footprints of random events lie inside their cell's blanket
        pts = rng.uniform(0, w.params.W, size=(400, 2))
        for x, y in pts:
            cell = o.cell_of(sx, sy, x, y)
            r = o.cell_rect(sx, sy, cell)
            assert r[0] <= x < r[1] and r[2] <= y < r[3]
            reach = np.hypot(st[:, 0] - x, st[:, 1] - y) < R_max
            assert not np.any(reach & ~B[cell])


def test_binning_partitions_domain(orc):
    w = _world(50.0, n_st=0)
    o = orc.World(w)
    rng = np.random.default_rng(2)
    ncx, ncy = o.grid_dims()
    for _ in range(10):
        sx, sy = rng.uniform(0, 100.0, 2)
        rects = np.array([o.cell_rect(sx, sy, c) for c in range(ncx * ncy)])
        live = (rects[:, 1] > rects[:, 0]) & (rects[:, 3] > rects[:, 2])
        area = ((rects[:, 1] - rects[:, 0]) * (rects[:, 3] - rects[:, 2]))[live].sum()
        assert area == pytest.approx(w.params.W ** 2, rel=1e-12)
        pts = rng.uniform(0, w.params.W, size=(2000, 2))
        for x, y in pts:
            c = o.cell_of(sx, sy, x, y)
            inside = ((rects[:, 0] <= x) & (x < rects[:, 1]) & (rects[:, 2] <= y) & (y < rects[:, 3]))
            assert live[c] and inside[c] and inside.sum() == 1


def test_same_colour_cells_never_touch(orc):
    o = orc.World(_world(50.0, n_st=0))
    ncx, ncy = o.grid_dims()
    for c in range(ncx * ncy):
        ix, iy = c % ncx, c // ncx
        for dx in (-1, 0, 1):
            for dy in (-1, 0, 1):
                jx, jy = ix + dx, iy + dy
                if (dx, dy) != (0, 0) and 0 <= jx < ncx and 0 <= jy < ncy:
                    assert o.colour_of(jy * ncx + jx) != o.colour_of(c)


def test_dynamic_shift_is_uniform(orc):
    o = orc.World(_world(50.0, n_st=0), seed=5)
    s = np.array([o.shift(k) for k in range(4000)])
    assert s.min() >= 0.0 and s.max() < 100.0
    h, _ = np.histogram(s[:, 0], bins=10, range=(0, 100))
    assert np.max(np.abs(h / 4000.0 - 0.1)) < 0.025
    assert abs(np.corrcoef(s[:, 0], s[:, 1])[0, 1]) < 0.05
