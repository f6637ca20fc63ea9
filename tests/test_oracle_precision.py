"""Precision pin of the oracle's log-likelihood change of one proposal.

The change is, by definition (§Generative Model, Observed Signals: each
sample is a zero-mean Gaussian whose variance is the noise variance plus the
arriving events' envelope variances; or, in the additive-mean reading, a
Gaussian around the summed envelopes), the sum over the changed samples of the
difference of two Gaussian log-densities.  Here that definition is evaluated
exactly enough to judge the oracle: Python's ``decimal`` at 50 significant
digits, every quantity (distance, arrival time, amplitude, envelope, the two
log-densities) from the event coordinates and the recorded samples, the two
log-densities subtracted as they stand.

The cases are built to be ill-conditioned in float64: a large arrival that
the hypothesis does not explain (s^2 / 2V above 1e7) under a small event that
is moved a very little, moved, born or killed.  Subtracting the two rounded
log-densities of each sample there loses the digits a small change needs;
mutant 10 of oracle.c does exactly that, and the pin catches it.
"""
import decimal

import numpy as np
import pytest

import worldgen

D = decimal.Decimal
CTX = decimal.Context(prec=50)


def _world(likelihood="variance"):
    p = worldgen.ModelParams(W=200.0, T=600.0, Lambda=10.0, likelihood=likelihood)
    st = np.array([[100.0, 100.0], [150.0, 60.0]])
    # a large event (m = 9) 8 km from station 0 that the hypotheses leave
    # unexplained, and a small one (m = 2.5) they hold, 20 km away, arriving
    # inside the large one's window
    truth = np.array([[104.0, 93.0, 100.0, 9.0], [112.0, 116.0, 104.0, 2.5]])
    return worldgen.make_world(p, st, seed=77, events=truth)


def _exact_delta(world, state, old_idx, cand):
    """Exact change of the log-likelihood when state[old_idx] (or nothing) is
    replaced by cand (or nothing)."""
    p = world.params
    f, tau, v = D(p.f_hz), D(p.tau), D(p.v)
    with decimal.localcontext(CTX):
        def arrival(e, j):
            dx = D(e[0]) - D(world.stations[j, 0])
            dy = D(e[1]) - D(world.stations[j, 1])
            d = (dx * dx + dy * dy).sqrt()
            if not d < D(p.R_max):
                return None
            a = D(e[2]) + d / v
            k0 = int((a * f).to_integral_value(rounding=decimal.ROUND_CEILING))
            amp = (D(p.alpha) * D(e[3]) - D(p.beta_att) * d).exp()
            return k0, a, amp

        def contrib(arr, k):
            k0, a, amp = arr
            if k < k0 or k >= k0 + p.n_w:
                return D(0)
            sd = amp * (-(D(k) / f - a) / tau).exp()
            return sd if p.likelihood == "mean" else sd * sd

        def log_n(s, P):
            if p.likelihood == "mean":
                r = s - P
                return -r * r / (2 * D(p.noise_var))   # the 2 pi sigma^2 term cancels
            return -P.ln() / 2 - s * s / (2 * P)         # the 2 pi term cancels

        base_noise = D(0) if p.likelihood == "mean" else D(p.noise_var)
        total = D(0)
        keep = [e for i, e in enumerate(state) if i != old_idx]
        for j in range(world.n_stations):
            ao = arrival(state[old_idx], j) if old_idx >= 0 else None
            an = arrival(cand, j) if cand is not None else None
            if ao is None and an is None:
                continue
            lo = min(a[0] for a in (ao, an) if a is not None)
            hi = max(a[0] + p.n_w for a in (ao, an) if a is not None)
            lo, hi = max(lo, 0), min(hi, p.n_samples)
            others = [a for a in (arrival(e, j) for e in keep) if a is not None]
            for k in range(lo, hi):
                base = base_noise + sum((contrib(a, k) for a in others), D(0))
                P_old = base + (contrib(ao, k) if ao else D(0))
                P_new = base + (contrib(an, k) if an else D(0))
                s = D(float(world.signals[j, k]))
                total += log_n(s, P_new) - log_n(s, P_old)
        return float(total)


def _cases(world):
    e = world.events[1].copy()
    near = e + np.array([2e-5, -1e-5, 5e-6, 1e-6])       # a very small move
    step = e + np.array([3.1, -2.4, 1.7, 0.08])              # an ordinary walk step
    far = np.array([95.0, 120.0, 118.0, 2.6])                # a jump within the footprint
    small = np.array([97.0, 104.0, 103.0, 2.3])              # a newborn under the large arrival
    st = world.events[1:2].copy()
    return [
        ("move-near", st, 0, near),
        ("move-step", st, 0, step),
        ("move-far", st, 0, far),
        ("birth", st, -1, small),
        ("death", np.vstack([st, small]), 1, None),
    ]


@pytest.mark.parametrize("likelihood", ["variance", "mean"])
def test_delta_matches_exact_definition(orc, likelihood):
    w = _world(likelihood)
    o = orc.World(w)
    for name, state, idx, cand in _cases(w):
        exact = _exact_delta(w, state, idx, cand)
        got = o.delta_loglik(state, idx, cand)
        err = abs(got - exact) / max(abs(exact), 1.0)
        assert err < 1e-12, (name, got, exact, err)
    # the large arrival makes the case as ill-conditioned as intended: the
    # Gaussian terms per sample are far larger than the change they make
    assert np.max(w.signals[0] ** 2) > 1e7


@pytest.mark.parametrize("likelihood", ["variance", "mean"])
def test_mutant_subtracting_two_log_densities_is_caught(orc, likelihood):
    """Mutant 10 prices each sample as log N(new) - log N(old), the two
    rounded; under the unexplained arrival the very small move loses digits."""
    w = _world(likelihood)
    o = orc.World(w, mutant=10)
    errs = []
    for name, state, idx, cand in _cases(w):
        exact = _exact_delta(w, state, idx, cand)
        errs.append(abs(o.delta_loglik(state, idx, cand) - exact) / max(abs(exact), 1.0))
    assert max(errs) > 5e-11, errs
