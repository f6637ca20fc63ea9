"""The oracle's pins catch plausible mistakes.

Each mutant is the oracle rebuilt with one planted mistake (ORC_MUTANT in
oracle.c); the test asserts that the pin meant to catch it fails:
  1, 2, 4 (Hastings terms of birth, death, move) -> detailed balance on the
          enumerated lattice world;
  3 (an arrival adds its standard deviation, not its variance) -> Monte-Carlo
          of the generative story; detailed balance alone cannot see it,
          because the mutant is a self-consistent sampler of a wrong model;
  5 (the Hastings term of a birth ignores the learned component of the
          mixture proposal) -> a prior-only chain drifts to the table's hot
          block;
  6 (learned magnitudes priced with the prior law) -> magnitudes pile up in
          the learned window;
  7 (the joint move of a pair drops the prior ratio) -> detailed balance of
          the kernels with joint moves on (and magnitude drift in
          test_oracle_pair.py);
  8, 9 (the arrival-time move without its prior ratio; offsets of newly
          reached stations set to 0) -> offsets leave their prior in chains
          on signals without information (test_oracle_arrivals.py).
  10 (each sample's change priced as the difference of its two rounded
          log-densities) -> the exact decimal evaluation of the definition
          on an ill-conditioned case (test_oracle_precision.py).
"""
import math

import numpy as np
import pytest

import worldgen
from test_oracle_sampler import PB, PD, PP, _enumerate, _kernel, _lattice_world


def _max_imbalance(orc, mutant, shift=(0.0, 0.0), cell=-1, pp=0.0):
    w, lat = _lattice_world(orc)
    o = orc.World(w, p_birth=PB, p_death=PD, k_per_phase=10, seed=3, lattice=lat, mutant=mutant,
                  p_pair=pp)
    pts, states, index, pi = _enumerate(o, lat, w.params)
    P = _kernel(o, lat, pts, states, index, cell, *shift, pp=pp)
    flow = pi[:, None] * P
    return np.max(np.abs(flow - flow.T)) / pi.max()


def test_unmutated_oracle_balances(orc):
    assert _max_imbalance(orc, 0) < 1e-13
    assert _max_imbalance(orc, 0, pp=PP) < 1e-13


def test_pair_prior_mutant_breaks_detailed_balance(orc):
    assert _max_imbalance(orc, 7, pp=PP) > 1e-4
    assert _max_imbalance(orc, 7, shift=(30.0, 70.0), cell=5, pp=PP) > 1e-4
    # with joint moves off the mutant is the oracle
    assert _max_imbalance(orc, 7) < 1e-13


@pytest.mark.parametrize("mutant", [1, 2, 4])
def test_hastings_mutants_break_detailed_balance(orc, mutant):
    assert _max_imbalance(orc, mutant) > 1e-4
    # the region-restricted kernels see it too
    assert _max_imbalance(orc, mutant, shift=(30.0, 70.0), cell=5) > 1e-4


def _generative_ratio(orc, mutant):
    p = worldgen.ModelParams(W=100.0, T=40.0, Lambda=1.0, tau=4.0, t_s=20.0, f_hz=5.0, R_max=50.0,
                             alpha=1.0, beta_att=0.02)
    st = np.array([[40.0, 50.0]])
    ev = np.array([[55.0, 45.0, 3.3, 2.7]])
    sq = np.zeros(p.n_samples)
    n_rep = 1000
    for r in range(n_rep):
        sq += worldgen.make_world(p, st, seed=20_000 + r, events=ev).signals[0] ** 2
    sq /= n_rep
    o = orc.World(worldgen.World(params=p, stations=st, signals=np.zeros((1, p.n_samples)),
                                 events=ev), mutant=mutant)
    V = o.variance(ev, 0, 0, p.n_samples)
    return np.max(np.abs(sq / V - 1.0) / math.sqrt(2.0 / n_rep))


def test_variance_mutant_caught_by_generative_draws(orc):
    assert _generative_ratio(orc, 0) < 5.5
    assert _generative_ratio(orc, 3) > 20.0
    # ... while detailed balance is blind to it
    assert _max_imbalance(orc, 3) < 1e-13


def test_mixture_mutant_drifts_to_the_hot_block(orc):
    from test_oracle_sampler import _prior_with_table
    _, _, fxy, ft = _prior_with_table(orc, mutant=5, n_sweeps=1500)
    assert fxy > 0.1 and ft > 0.24, (fxy, ft)   # unmutated: 0.0625 and 0.2


def test_magnitude_mutant_piles_up_in_the_window(orc):
    from test_oracle_sampler import _prior_with_magnitudes
    mean, frac, _ = _prior_with_magnitudes(orc, mutant=6, n_sweeps=1500)
    assert frac > 0.12, (mean, frac)   # unmutated: 0.068
