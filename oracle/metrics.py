"""Event matching and detection scores, plain loops (TEST INFRASTRUCTURE ONLY).

Only ``tests/``, ``__graft_entry__.smoke()`` and ``bench.py``'s CPU legs may
import this module; it shares no code with the package's own scorer.

§Experimental Results scores an inferred event set against the true one by
a greedy matching: the true events are visited one by one, each is paired
with the closest inferred event that lies within a distance and a time
threshold, and both leave the pool.  Readings taken here (the paper fixes
neither the visiting order nor the tie rule): true events in origin-time
order (ties by index); "closest" is the smallest spatial distance among the
unmatched inferred events with distance < d_max and |dt| < t_max (ties by
index).  Precision = matched / inferred, recall = matched / true,
F1 = 2PR / (P + R), each 0 when undefined.  Location error = mean spatial
distance of the matched pairs.  Scores can be restricted to the detectable
zone: events within R_max of at least one station (the only ones the
signals say anything about).
"""
from __future__ import annotations

import math


def detectable(events, stations, R_max):
    """For each event (x, y, ...): is some station closer than R_max."""
    out = []
    for e in events:
        hit = False
        for s in stations:
            if math.hypot(e[0] - s[0], e[1] - s[1]) < R_max:
                hit = True
                break
        out.append(hit)
    return out


def match(true_events, inferred, d_max, t_max):
    """Greedy matching; returns (i_true, j_inferred, distance) per pair."""
    order = sorted(range(len(true_events)), key=lambda i: (true_events[i][2], i))
    used = [False] * len(inferred)
    pairs = []
    for i in order:
        te = true_events[i]
        best, best_d = -1, 0.0
        for j, ie in enumerate(inferred):
            if used[j]:
                continue
            d = math.hypot(te[0] - ie[0], te[1] - ie[1])
            if d < d_max and abs(te[2] - ie[2]) < t_max and (best < 0 or d < best_d):
                best, best_d = j, d
        if best >= 0:
            used[best] = True
            pairs.append((i, best, best_d))
    return pairs


def scores(true_events, inferred, d_max, t_max, stations=None, R_max=None):
    """Precision, recall, F1, location error and counts; restricted to the
    detectable zone when stations and R_max are given."""
    true_events = [tuple(e) for e in true_events]
    inferred = [tuple(e) for e in inferred]
    if stations is not None:
        true_events = [e for e, k in zip(true_events, detectable(true_events, stations, R_max)) if k]
        inferred = [e for e, k in zip(inferred, detectable(inferred, stations, R_max)) if k]
    pairs = match(true_events, inferred, d_max, t_max)
    n_m = len(pairs)
    p = n_m / len(inferred) if inferred else 0.0
    r = n_m / len(true_events) if true_events else 0.0
    f1 = 2.0 * p * r / (p + r) if p + r > 0.0 else 0.0
    loc = sum(d for _, _, d in pairs) / n_m if n_m else float("nan")
    return {"precision": p, "recall": r, "f1": f1, "loc_err": loc, "matched": n_m,
            "n_true": len(true_events), "n_inferred": len(inferred)}
