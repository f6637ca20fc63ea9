"""The matching scores of §Experimental Results: the oracle's plain-loop
version pinned by hand-built cases, and the package's numpy version equal to
it on random event sets."""
import numpy as np
import pytest

from oracle import metrics as om


def ev(x, y, t, m=3.0):
    return (x, y, t, m)


def test_perfect_and_empty():
    T = [ev(10, 10, 5), ev(300, 40, 90)]
    s = om.scores(T, T, 100.0, 20.0)
    assert (s["precision"], s["recall"], s["f1"], s["loc_err"]) == (1.0, 1.0, 1.0, 0.0)
    s = om.scores(T, [], 100.0, 20.0)
    assert (s["precision"], s["recall"], s["f1"], s["matched"]) == (0.0, 0.0, 0.0, 0)
    s = om.scores([], T, 100.0, 20.0)
    assert (s["precision"], s["recall"], s["f1"]) == (0.0, 0.0, 0.0)


def test_earlier_true_event_takes_the_shared_candidate():
    # two true events near one inferred event: the earlier one (in time) wins
    T = [ev(0, 0, 30), ev(10, 0, 20)]
    I = [ev(5, 0, 25)]
    pairs = om.match(T, I, 100.0, 20.0)
    assert pairs == [(1, 0, 5.0)]
    s = om.scores(T, I, 100.0, 20.0)
    assert s["precision"] == 1.0 and s["recall"] == 0.5 and s["f1"] == pytest.approx(2 / 3)


def test_closest_candidate_and_strict_thresholds():
    T = [ev(0, 0, 0)]
    assert om.match(T, [ev(50, 0, 0), ev(30, 0, 0)], 100.0, 20.0) == [(0, 1, 30.0)]
    assert om.match(T, [ev(100, 0, 0)], 100.0, 20.0) == []       # distance must be < d_max
    assert om.match(T, [ev(0, 0, 20)], 100.0, 20.0) == []        # |dt| must be < t_max
    assert om.match(T, [ev(0, 0, -19.5)], 100.0, 20.0) == [(0, 0, 0.0)]
    # equal distances: the lower index
    assert om.match(T, [ev(0, 40, 0), ev(40, 0, 0)], 100.0, 20.0) == [(0, 0, 40.0)]


def test_detectable_zone_restriction():
    st = [(0.0, 0.0)]
    T = [ev(10, 0, 0), ev(500, 500, 0)]
    I = [ev(12, 0, 1)]
    s_all = om.scores(T, I, 100.0, 20.0)
    s_det = om.scores(T, I, 100.0, 20.0, stations=st, R_max=50.0)
    assert s_all["recall"] == 0.5 and s_det["recall"] == 1.0 and s_det["n_true"] == 1


@pytest.fixture(scope="module")
def pm():
    import __graft_entry__
    __graft_entry__.build()
    from paper_1612_00595_gb300 import metrics
    return metrics


def test_package_scores_equal_oracle(pm):
    rng = np.random.default_rng(5)
    st = rng.uniform(0, 1000, size=(20, 2))
    for trial in range(40):
        nt, ni = rng.integers(0, 40), rng.integers(0, 40)
        T = np.column_stack([rng.uniform(0, 1000, nt), rng.uniform(0, 1000, nt), rng.uniform(0, 600, nt),
                             2 + rng.exponential(1, nt)])
        # inferred: jittered copies of some true events plus clutter; some exact ties in time
        k = min(nt, ni)
        I = np.vstack([T[:k] + np.column_stack([rng.normal(0, 40, k), rng.normal(0, 40, k),
                                                  rng.normal(0, 10, k), np.zeros(k)]),
                       np.column_stack([rng.uniform(0, 1000, ni - k), rng.uniform(0, 1000, ni - k),
                                        rng.uniform(0, 600, ni - k), np.full(ni - k, 3.0)])])
        if nt > 3:
            T[1, 2] = T[2, 2]
        for kw in ({}, {"stations": st, "R_max": 50.0}):
            a = om.scores(T, I, 100.0, 20.0, **kw)
            b = pm.scores(T, I, 100.0, 20.0, **kw)
            for key in ("precision", "recall", "f1", "matched", "n_true", "n_inferred"):
                assert a[key] == b[key], (trial, key)
            assert (np.isnan(a["loc_err"]) and np.isnan(b["loc_err"])) or a["loc_err"] == pytest.approx(b["loc_err"])
