"""Pins of the oracle's MH samplers.

* Exact enumeration on a lattice world: the posterior over every multiset of
  at most two events is computed from the definition (Poisson process on a
  finite point set: independent Poisson counts, times the likelihood), and
  the transition matrix of the serial kernel and of every region-restricted
  kernel is assembled from the proposal probabilities and the oracle's
  acceptance ratios.  Each kernel must leave the posterior invariant and
  satisfy detailed balance to ~1e-12 (MH acceptance rule, §Background; the
  region kernels of Algorithm "Chromatic MH with Static Coloring").
* Long lattice chains (serial, static and dynamic chromatic) reproduce the
  enumerated marginals within batch-means error.
* Prior-only continuous chains (no stations) reproduce the prior: Poisson
  count, uniform locations (including edge regions cut by the domain),
  Exp(1) magnitudes.
* The joint move of a pair (§MH moves, "Joint Events Move": the exchange of
  two events' locations, or one common offset of both) enters the same
  enumerated kernels with probability PP; they must still balance, and the
  chains with it must reproduce the same marginals.
"""
import itertools
import math

import numpy as np
import pytest

import worldgen

PB, PD = 0.25, 0.25
PMV = 1.0 - PB - PD
PP = 0.2   # share of joint moves where a test turns them on


def _lattice_world(orc, shift_cells=False, likelihood="variance"):
    p = worldgen.ModelParams(W=200.0, T=60.0, Lambda=1.5, v=6.0, alpha=0.5, beta_att=0.01,
                             tau=5.0, t_s=10.0, f_hz=1.0, R_max=50.0, L=100.0, likelihood=likelihood)
    st = np.array([[50.0, 50.0], [150.0, 150.0], [60.0, 140.0]])
    truth = np.array([[75.0, 75.0, 10.0, 3.5], [125.0, 175.0, 30.0, 2.5]])
    w = worldgen.make_world(p, st, seed=77, events=truth)
    lat = orc.Lattice(nx=4, ny=4, nt=2, nm=2, nmax=2, x0=25.0, dx=50.0, y0=25.0, dy=50.0,
                      t0=10.0, dt=20.0, m0=2.5, dm=1.0)
    return w, lat


def _points(lat):
    pts = []
    for iy in range(lat.ny):
        for ix in range(lat.nx):
            for it in range(lat.nt):
                for im in range(lat.nm):
                    pts.append((lat.x0 + ix * lat.dx, lat.y0 + iy * lat.dy,
                                lat.t0 + it * lat.dt, lat.m0 + im * lat.dm))
    return np.array(pts)


def _enumerate(o, lat, p):
    pts = _points(lat)
    states = [()]
    for n in range(1, lat.nmax + 1):
        states += list(itertools.combinations_with_replacement(range(len(pts)), n))
    index = {s: i for i, s in enumerate(states)}
    # Poisson process on the finite set: beta_p = Lambda * 1/(nx ny) * 1/nt * w_m
    wm = np.exp(-(lat.m0 + np.arange(lat.nm) * lat.dm - 2.0))
    wm /= wm.sum()
    beta = np.array([p.Lambda / (lat.nx * lat.ny * lat.nt) * wm[int(round((q[3] - lat.m0) / lat.dm))]
                     for q in pts])
    logpi = np.empty(len(states))
    for i, s in enumerate(states):
        ev = pts[list(s)]
        counts = np.bincount(np.array(s, dtype=int), minlength=len(pts)) if s else np.zeros(1)
        logpi[i] = (-p.Lambda + np.log(beta[list(s)]).sum()
                    - sum(math.lgamma(c + 1) for c in counts)
                    + o.log_likelihood(ev))
    pi = np.exp(logpi - logpi.max())
    pi /= pi.sum()
    return pts, states, index, pi


def _add(P, i, j, prob, la_ok):
    la, ok = la_ok
    if not ok:
        P[i, i] += prob
        return
    a = min(1.0, math.exp(min(la, 0.0)))
    P[i, j] += prob * a
    P[i, i] += prob * (1 - a)


def _pair_moves(o, lat, s, ev, own, key, index, cell, sx, sy, P, i, pp):
    """Transitions of the joint move: an ordered pair of distinct own events
    (probability 1 / (n (n - 1))), then with probability 1/2 the exchange of
    their locations, else one of the 8 lattice steps applied to both."""
    if len(own) < 2:
        P[i, i] += pp
        return
    n_o = len(own)
    base = pp / (n_o * (n_o - 1))
    steps = (lat.dx, lat.dy, lat.dt, lat.dm)
    for ai, a in enumerate(own):
        for bi, b in enumerate(own):
            if ai == bi:
                continue
            cands = []
            c1, c2 = ev[a].copy(), ev[b].copy()
            c1[:2], c2[:2] = ev[b][:2], ev[a][:2]
            cands.append((0.5 * base, c1, c2))
            for d in range(8):
                off = np.zeros(4)
                off[d >> 1] = (-1.0 if d & 1 else 1.0) * steps[d >> 1]
                cands.append((0.5 * base / 8, ev[a] + off, ev[b] + off))
            for prob, c1, c2 in cands:
                la_ok = o.log_alpha_pair(sx, sy, cell, ev, ai, bi, c1, c2)
                j = i
                if la_ok[1]:
                    moved = list(s)
                    moved.remove(s[a])
                    moved.remove(s[b])
                    moved += [key[tuple(c1)], key[tuple(c2)]]
                    j = index[tuple(sorted(moved))]
                _add(P, i, j, prob, la_ok)


def _kernel(o, lat, pts, states, index, cell, sx, sy, pp=0.0):
    pmv = PMV if pp == 0.0 else 1.0 - PB - PD - pp
    n = len(states)
    P = np.zeros((n, n))
    key = {tuple(q): i for i, q in enumerate(pts)}

    def in_region(x, y):
        return cell < 0 or o.cell_of(sx, sy, x, y) == cell

    xy_pts = sorted({(q[0], q[1]) for q in pts if in_region(q[0], q[1])})
    n_r = len(xy_pts)
    for i, s in enumerate(states):
        ev = pts[list(s)]
        own = [q for q in range(len(s)) if in_region(ev[q, 0], ev[q, 1])]
        # births
        if n_r == 0:
            P[i, i] += PB
        else:
            prob = PB / (n_r * lat.nt * lat.nm)
            for (x, y) in xy_pts:
                for it in range(lat.nt):
                    for im in range(lat.nm):
                        c = np.array([x, y, lat.t0 + it * lat.dt, lat.m0 + im * lat.dm])
                        la, ok = o.log_alpha(sx, sy, cell, ev, 0, -1, c)
                        if not ok:
                            P[i, i] += prob
                            continue
                        a = min(1.0, math.exp(min(la, 0.0)))
                        j = index[tuple(sorted(s + (key[tuple(c)],)))]
                        P[i, j] += prob * a
                        P[i, i] += prob * (1 - a)
        if not own:
            P[i, i] += PD + pmv + pp
            continue
        if pp > 0.0:
            _pair_moves(o, lat, s, ev, own, key, index, cell, sx, sy, P, i, pp)
        for qi, q in enumerate(own):
            prob = PD / len(own)
            la, ok = o.log_alpha(sx, sy, cell, ev, 1, qi, None)
            assert ok
            a = min(1.0, math.exp(min(la, 0.0)))
            rest = list(s)
            rest.remove(s[q])
            j = index[tuple(sorted(rest))]
            P[i, j] += prob * a
            P[i, i] += prob * (1 - a)
            for d in range(8):
                prob = pmv / (len(own) * 8)
                c = ev[q].copy()
                step = -1.0 if d & 1 else 1.0
                c[d >> 1] += step * (lat.dx, lat.dy, lat.dt, lat.dm)[d >> 1]
                la, ok = o.log_alpha(sx, sy, cell, ev, 2, qi, c)
                if not ok:
                    P[i, i] += prob
                    continue
                a = min(1.0, math.exp(min(la, 0.0)))
                moved = list(s)
                moved.remove(s[q])
                moved.append(key[tuple(c)])
                j = index[tuple(sorted(moved))]
                P[i, j] += prob * a
                P[i, i] += prob * (1 - a)
    return P


@pytest.fixture(scope="module", params=["variance", "mean"])
def lattice_case(orc, request):
    """The lattice world under each likelihood reading: the exact posterior by
    enumeration, which every sampler must leave invariant."""
    w, lat = _lattice_world(orc, likelihood=request.param)
    o = orc.World(w, p_birth=PB, p_death=PD, k_per_phase=10, seed=3, lattice=lat)
    pts, states, index, pi = _enumerate(o, lat, w.params)
    return o, lat, pts, states, index, pi


@pytest.fixture(scope="module", params=["variance", "mean"])
def lattice_pair_case(orc, request):
    """The same lattice world with joint moves on (share PP)."""
    w, lat = _lattice_world(orc, likelihood=request.param)
    o = orc.World(w, p_birth=PB, p_death=PD, k_per_phase=10, seed=3, lattice=lat, p_pair=PP)
    pts, states, index, pi = _enumerate(o, lat, w.params)
    return o, lat, pts, states, index, pi


def _check_kernel(P, pi):
    assert np.allclose(P.sum(axis=1), 1.0, atol=1e-13)
    assert P.min() >= -1e-15
    flow = pi[:, None] * P
    assert np.max(np.abs(flow - flow.T)) < 1e-13 * pi.max()
    assert np.max(np.abs(pi @ P - pi)) < 1e-13 * pi.max()


def test_serial_kernel_detailed_balance(lattice_case):
    o, lat, pts, states, index, pi = lattice_case
    P = _kernel(o, lat, pts, states, index, -1, 0.0, 0.0)
    _check_kernel(P, pi)
    # the kernel moves: it is not the identity
    assert np.mean(np.diag(P)) < 0.95


@pytest.mark.parametrize("shift", [(0.0, 0.0), (30.0, 70.0)])
def test_region_kernels_detailed_balance(lattice_case, shift):
    o, lat, pts, states, index, pi = lattice_case
    sx, sy = shift
    ncx, ncy = o.grid_dims()
    live = [c for c in range(ncx * ncy)
            if (lambda r: r[1] > r[0] and r[3] > r[2])(o.cell_rect(sx, sy, c))]
    assert len(live) == (4 if shift == (0.0, 0.0) else 9)
    for c in live:
        _check_kernel(_kernel(o, lat, pts, states, index, c, sx, sy), pi)


def test_pair_kernels_detailed_balance(lattice_pair_case):
    o, lat, pts, states, index, pi = lattice_pair_case
    P = _kernel(o, lat, pts, states, index, -1, 0.0, 0.0, pp=PP)
    _check_kernel(P, pi)
    # the joint move changes states on its own: with the other moves taken
    # out, the kernel still leaves the two-event states
    two = [i for i, s in enumerate(states) if len(s) == 2]
    assert np.mean(np.diag(P)[two]) < 0.95
    for shift in [(0.0, 0.0), (30.0, 70.0)]:
        ncx, ncy = o.grid_dims()
        for c in range(ncx * ncy):
            r = o.cell_rect(*shift, c)
            if r[1] > r[0] and r[3] > r[2]:
                _check_kernel(_kernel(o, lat, pts, states, index, c, *shift, pp=PP), pi)


def _batch_se(x, nb=40):
    x = np.asarray(x, dtype=np.float64)
    m = len(x) // nb
    b = x[: m * nb].reshape(nb, m).mean(axis=1)
    return b.mean(), b.std(ddof=1) / math.sqrt(nb)


@pytest.mark.parametrize("mode", ["serial", "static", "dynamic"])
def test_lattice_chain_marginals(lattice_case, mode):
    o, lat, pts, states, index, pi = lattice_case
    # exact marginals: P(N = n) and the mean occupancy of every xy site
    pN = np.zeros(lat.nmax + 1)
    occ = np.zeros(lat.nx * lat.ny)
    for s, q in zip(states, pi):
        pN[len(s)] += q
        for a in s:
            x, y = pts[a][:2]
            occ[int(round((y - lat.y0) / lat.dy)) * lat.nx + int(round((x - lat.x0) / lat.dx))] += q
    ev = np.zeros((0, 4))
    ids = None
    n_samples = 6000
    Ns, O = [], []
    for it in range(n_samples):
        if mode == "serial":
            ev, ids, _, _ = o.run_serial(ev, 40, ids=ids, step0=it * 40)
        else:
            ev, ids, _, _ = o.run_chromatic(ev, 1, ids=ids, sweep0=it,
                                            shift_mode=1 if mode == "dynamic" else 0,
                                            sx=0.0, sy=0.0)
        Ns.append(len(ev))
        o_ = np.zeros(lat.nx * lat.ny)
        for e in ev:
            o_[int(round((e[1] - lat.y0) / lat.dy)) * lat.nx + int(round((e[0] - lat.x0) / lat.dx))] += 1
        O.append(o_)
    Ns = np.array(Ns)
    O = np.array(O)
    for n in range(lat.nmax + 1):
        m, se = _batch_se(Ns == n)
        assert abs(m - pN[n]) < 5 * se + 2e-3, (n, m, pN[n], se)
    for site in range(lat.nx * lat.ny):
        m, se = _batch_se(O[:, site])
        assert abs(m - occ[site]) < 5 * se + 2e-3, (site, m, occ[site], se)


def test_lattice_chain_marginals_with_pairs(lattice_pair_case):
    """Dynamic chromatic chains with joint moves reproduce the enumerated
    marginals."""
    test_lattice_chain_marginals(lattice_pair_case, "dynamic")


@pytest.mark.parametrize("mode,p_pair", [("serial", 0.0), ("static", 0.0), ("dynamic", 0.0),
                                         ("dynamic", 0.3)])
def test_prior_only_chain_recovers_prior(orc, mode, p_pair):
    p, Ns, frac, ms = _prior_only_chain(orc, mode, p_pair)
    m, se = _batch_se(Ns)
    assert abs(m - p.Lambda) < 5 * se, (m, se)
    v = np.var(Ns)
    assert abs(v / p.Lambda - 1.0) < 0.25
    # uniform location over the domain, edge regions included
    assert np.max(np.abs(frac - 0.1)) < 0.02, frac
    # Exp(1) magnitudes above 2
    assert abs(ms.mean() - 1.0) < 0.06
    assert abs(np.mean(ms > 1.0) - math.exp(-1.0)) < 0.03


def _prior_only_chain(orc, mode, p_pair, mutant=0, n_iter=3000, p_bd=0.25, sig_m=0.5):
    """A chain with no stations: its state must follow the prior.  Returns
    the params, the event counts, the location histogram (10 bins of x and y
    pooled) and the magnitudes above 2."""
    p = worldgen.ModelParams(W=200.0, T=100.0, Lambda=12.0, R_max=50.0, L=100.0)
    w = worldgen.World(params=p, stations=np.zeros((0, 2)), signals=np.zeros((0, 0)),
                       events=np.zeros((0, 4)))
    o = orc.World(w, k_per_phase=8, seed=11, sig_xy=20.0, sig_t=10.0, sig_m=sig_m, p_pair=p_pair,
                  mutant=mutant, p_birth=p_bd, p_death=p_bd)
    ev = np.zeros((0, 4))
    ids = None
    Ns, xs, ms = [], [], []
    for it in range(n_iter):
        if mode == "serial":
            ev, ids, _, _ = o.run_serial(ev, 40, ids=ids, step0=it * 40)
        else:
            ev, ids, _, _ = o.run_chromatic(ev, 1, ids=ids, sweep0=it,
                                            shift_mode=1 if mode == "dynamic" else 0,
                                            sx=37.0, sy=61.0)
        Ns.append(len(ev))
        if it % 5 == 0:
            xs.extend(ev[:, 0])
            xs.extend(ev[:, 1])
            ms.extend(ev[:, 3] - 2.0)
    h, _ = np.histogram(xs, bins=10, range=(0.0, p.W))
    return p, np.array(Ns), h / h.sum(), np.array(ms)


def test_threaded_chromatic_equals_sequential(orc):
    """Same-colour regions are independent (disjoint blankets), so running
    them on several threads gives bit-identical chains and traces."""
    p = worldgen.ModelParams(W=500.0, T=400.0, Lambda=40.0, f_hz=2.0)
    w = worldgen.make_world(p, worldgen.jittered_grid_stations(5, p.W, 3), seed=3)
    o = orc.World(w, k_per_phase=16, seed=21)
    a = o.run_chromatic(np.zeros((0, 4)), 6, trace_cap=100000, threads=1)
    b = o.run_chromatic(np.zeros((0, 4)), 6, trace_cap=100000, threads=4)
    assert np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[1])
    assert np.array_equal(a[2], b[2])
    assert a[3] == b[3]
    # the running log-density change equals a from-scratch recomputation
    empty = np.zeros((0, 4))
    assert a[3] == pytest.approx(o.log_density(a[0]) - o.log_density(empty), rel=1e-9)


def _hot_table():
    """8 x 8 pixels of 25 km over 200 km, 10 bins of 10 s: weight 1, and 200 in
    a 2 x 2 pixel block during two bins."""
    tab = np.ones((8, 8, 10), dtype=np.float32)
    tab[5:7, 1:3, 2:4] = 200.0
    return tab


def _prior_with_table(orc, mutant=0, n_sweeps=3000):
    p = worldgen.ModelParams(W=200.0, T=100.0, Lambda=12.0, R_max=50.0, L=100.0)
    w = worldgen.World(params=p, stations=np.zeros((0, 2)), signals=np.zeros((0, 0)),
                       events=np.zeros((0, 4)))
    o = orc.World(w, k_per_phase=8, seed=12, sig_xy=20.0, sig_t=10.0, sig_m=0.5, mutant=mutant)
    o.set_birth_table(_hot_table(), mix=0.5)
    ev, ids = np.zeros((0, 4)), None
    Ns, hot_xy, hot_t, n_seen = [], 0, 0, 0
    for it in range(n_sweeps):
        ev, ids, _, _ = o.run_chromatic(ev, 1, ids=ids, sweep0=it, shift_mode=1)
        Ns.append(len(ev))
        if it % 5 == 0 and len(ev):
            in_xy = (ev[:, 0] >= 25.0) & (ev[:, 0] < 75.0) & (ev[:, 1] >= 125.0) & (ev[:, 1] < 175.0)
            in_t = (ev[:, 2] >= 20.0) & (ev[:, 2] < 40.0)
            hot_xy += int(in_xy.sum())
            hot_t += int(in_t.sum())
            n_seen += len(ev)
    return p, np.array(Ns), hot_xy / n_seen, hot_t / n_seen


def test_learned_birth_mixture_keeps_the_prior(orc):
    """With no stations the posterior is the prior.  A birth proposal that
    prefers a small space-time block (the learned component of the mixture)
    must not pull the chain there: the Hastings term carries the mixture
    density.  Event count ~ Poisson(Lambda), positions and times uniform."""
    p, Ns, fxy, ft = _prior_with_table(orc)
    m, se = _batch_se(Ns)
    assert abs(m - p.Lambda) < 5 * se, (m, se)
    assert abs(fxy - 4.0 / 64.0) < 0.012, fxy
    assert abs(ft - 0.2) < 0.025, ft


def _prior_with_magnitudes(orc, mutant=0, n_sweeps=3000):
    """The hot table with learned magnitudes: window [3.75, 4.25) everywhere
    (centre 4, half-width 0.25).  Returns the mean of m - 2 over the chain's
    events and the fraction of them inside the window."""
    p = worldgen.ModelParams(W=200.0, T=100.0, Lambda=12.0, R_max=50.0, L=100.0)
    w = worldgen.World(params=p, stations=np.zeros((0, 2)), signals=np.zeros((0, 0)),
                       events=np.zeros((0, 4)))
    o = orc.World(w, k_per_phase=8, seed=13, sig_xy=20.0, sig_t=10.0, sig_m=0.5, mutant=mutant)
    tab = _hot_table()
    o.set_birth_table(tab, mix=0.5)
    o.set_birth_magnitude(np.full(tab.shape, 4.0, dtype=np.float32), 0.25)
    ev, ids = np.zeros((0, 4)), None
    ms, means = [], []
    for it in range(n_sweeps):
        ev, ids, _, _ = o.run_chromatic(ev, 1, ids=ids, sweep0=it, shift_mode=1)
        if it % 5 == 0 and len(ev):
            ms.append(ev[:, 3].copy())
            means.append(ev[:, 3].mean() - 2.0)
    m = np.concatenate(ms)
    return m.mean() - 2.0, np.mean((m >= 3.75) & (m < 4.25)), np.array(means)


def test_learned_magnitudes_keep_the_prior(orc):
    """Table births that draw the magnitude from a narrow window must leave
    the magnitude law of the prior (m - 2 ~ Exp(1)): the Hastings terms carry
    the window density.  Prior mass of the window: e^-1.75 - e^-2.25."""
    mean, frac, per = _prior_with_magnitudes(orc)
    _, se = _batch_se(per)
    assert abs(mean - 1.0) < max(5 * se, 0.05), (mean, se)
    assert abs(frac - (np.exp(-1.75) - np.exp(-2.25))) < 0.02, frac
