"""Detection scores of an inferred event set (§Experimental Results).

The true events are visited in origin-time order (ties by index); each is
paired with the closest unmatched inferred event within d_max in space and
t_max in time (ties by index), and both leave the pool.  Precision, recall,
F1 and the mean location error of the pairs follow; every ratio is 0 when
undefined.  ``stations`` and ``R_max`` restrict both sets to the detectable
zone (events within R_max of some station).  Host-side numpy; the sampler
itself never calls it.
"""
from __future__ import annotations

import numpy as np


def detectable(events: np.ndarray, stations: np.ndarray, R_max: float) -> np.ndarray:
    events = np.asarray(events, dtype=np.float64).reshape(-1, 4)
    stations = np.asarray(stations, dtype=np.float64).reshape(-1, 2)
    if len(events) == 0 or len(stations) == 0:
        return np.zeros(len(events), dtype=bool)
    d = np.hypot(events[:, None, 0] - stations[None, :, 0], events[:, None, 1] - stations[None, :, 1])
    return (d < R_max).any(axis=1)


def scores(true_events, inferred, d_max: float, t_max: float, stations=None, R_max=None) -> dict:
    te = np.asarray(true_events, dtype=np.float64).reshape(-1, 4)
    ie = np.asarray(inferred, dtype=np.float64).reshape(-1, 4)
    if stations is not None:
        te = te[detectable(te, stations, R_max)]
        ie = ie[detectable(ie, stations, R_max)]
    order = np.lexsort((np.arange(len(te)), te[:, 2]))
    free = np.ones(len(ie), dtype=bool)
    dists = []
    for i in order:
        d = np.hypot(ie[:, 0] - te[i, 0], ie[:, 1] - te[i, 1])
        ok = free & (d < d_max) & (np.abs(ie[:, 2] - te[i, 2]) < t_max)
        if not ok.any():
            continue
        j = int(np.flatnonzero(ok)[np.argmin(d[ok])])   # first index among equal distances
        free[j] = False
        dists.append(float(d[j]))
    n_m = len(dists)
    p = n_m / len(ie) if len(ie) else 0.0
    r = n_m / len(te) if len(te) else 0.0
    f1 = 2.0 * p * r / (p + r) if p + r > 0.0 else 0.0
    return {"precision": p, "recall": r, "f1": f1, "loc_err": float(np.mean(dists)) if n_m else float("nan"),
            "matched": n_m, "n_true": int(len(te)), "n_inferred": int(len(ie))}
