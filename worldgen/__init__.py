"""Seeded synthetic worlds drawn from the toy seismic model's generative story.

This module is shared by the CPU oracle, the CUDA path's tests and ``bench.py``.
It only *samples* worlds, in the order the generative model states them
(§Generative Model of Seismic Signals): a Poisson number of events with uniform
space-time locations, arrival at each station after the travel time, an iid
Gaussian signal per arrival whose standard deviation follows the event's
amplitude envelope, and iid Gaussian background noise added on top; as in
§Experimental Results, the evaluation worlds are draws from the model
itself.  It evaluates no density, no proposal and
no acceptance ratio; those belong to the oracle and to the CUDA path, which
implement them independently.

World conventions (shared input format, not arithmetic of the method):
  * events: float64 array [n, 4] of (x km, y km, t s, magnitude m)
  * stations: float64 array [n_st, 2] of (x km, y km)
  * signals: array [n_st, n_samples] (float64 or float32); sample k is taken
    at time k / f_hz
"""
from __future__ import annotations

import concurrent.futures as _cf
import dataclasses
import math
import os
from typing import Optional

import numpy as np

__all__ = [
    "ModelParams",
    "World",
    "grid_stations",
    "jittered_grid_stations",
    "uniform_stations",
    "sample_events",
    "sample_signals",
    "make_world",
    "config_tiny",
    "config_replay",
    "config_scale",
    "config_batched",
    "batched_instances",
    "subworld",
]


@dataclasses.dataclass
class ModelParams:
    """Constants of the reconciled toy seismic model.

    Domain [0, W]^2 km x [0, T] s; Poisson event count with mean Lambda;
    magnitude m = 2 + Exp(1); travel speed v km/s; amplitude
    exp(alpha*m - beta_att*d); one-sided envelope exp(-u/tau) on 0 <= u < t_s;
    events reach only stations closer than R_max km; background noise variance
    noise_var; sample rate f_hz; spatial regions are squares of side L km.
    """

    W: float
    T: float
    Lambda: float
    v: float = 6.0
    alpha: float = 1.0
    beta_att: float = 0.01
    tau: float = 20.0
    t_s: float = 200.0
    noise_var: float = 1.0
    f_hz: float = 10.0
    R_max: float = 50.0
    L: float = 100.0
    n_samples: Optional[int] = None
    # "variance": each arrival adds (A e^{-u/tau})^2 to the variance of a
    # zero-mean sample; "mean": it adds A e^{-u/tau} to the mean of a sample
    # whose variance is the noise (the additive reading)
    likelihood: str = "variance"

    def __post_init__(self):
        if self.n_samples is None:
            self.n_samples = int(round(self.T * self.f_hz))

    @property
    def n_w(self) -> int:
        """Samples covered by one arrival: t_s * f_hz (an integer here)."""
        return int(round(self.t_s * self.f_hz))


@dataclasses.dataclass
class World:
    params: ModelParams
    stations: np.ndarray          # [n_st, 2] float64
    signals: np.ndarray           # [n_st, n_samples] float32 | float64
    events: np.ndarray            # [n, 4] float64 ground truth
    seed: int = 0
    # latent arrival offsets of the ground truth, dense [n, n_st] (0 where an
    # event does not reach a station); None: deterministic arrivals
    offsets: Optional[np.ndarray] = None

    @property
    def n_stations(self) -> int:
        return int(self.stations.shape[0])


# --------------------------------------------------------------------------
# station layouts
# --------------------------------------------------------------------------
def grid_stations(n_side: int, W: float) -> np.ndarray:
    """Stations at the centres of an n_side x n_side grid over [0, W]^2."""
    c = (np.arange(n_side, dtype=np.float64) + 0.5) * (W / n_side)
    xx, yy = np.meshgrid(c, c, indexing="xy")
    return np.stack([xx.ravel(), yy.ravel()], axis=1)


def jittered_grid_stations(n_side: int, W: float, seed: int, jitter_frac: float = 0.25) -> np.ndarray:
    """Grid centres moved by U(-j, j) per axis, j = jitter_frac * cell side."""
    base = grid_stations(n_side, W)
    rng = np.random.Generator(np.random.PCG64(np.random.SeedSequence([seed, 0x57A7])))
    j = jitter_frac * W / n_side
    return base + rng.uniform(-j, j, size=base.shape)


def uniform_stations(n: int, W: float, seed: int) -> np.ndarray:
    rng = np.random.Generator(np.random.PCG64(np.random.SeedSequence([seed, 0x57A8])))
    return rng.uniform(0.0, W, size=(n, 2))


# --------------------------------------------------------------------------
# events and signals
# --------------------------------------------------------------------------
def sample_events(p: ModelParams, seed: int) -> np.ndarray:
    """Poisson(Lambda) events, uniform (x, y, t), m = 2 + Exp(1); sorted by t."""
    rng = np.random.Generator(np.random.PCG64(np.random.SeedSequence([seed, 0xE7E7])))
    n = int(rng.poisson(p.Lambda))
    ev = np.empty((n, 4), dtype=np.float64)
    ev[:, 0] = rng.uniform(0.0, p.W, n)
    ev[:, 1] = rng.uniform(0.0, p.W, n)
    ev[:, 2] = rng.uniform(0.0, p.T, n)
    ev[:, 3] = 2.0 + rng.exponential(1.0, n)
    return ev[np.argsort(ev[:, 2], kind="stable")]


def _station_row(p: ModelParams, st: np.ndarray, events: np.ndarray, j: int,
                 seed: int, dtype, offsets: Optional[np.ndarray] = None) -> np.ndarray:
    """One station's record: background noise plus, per arrival, a Gaussian
    signal of that envelope (variance reading) or the envelope itself (mean
    reading)."""
    rng = np.random.Generator(np.random.PCG64(np.random.SeedSequence([seed, 0x5160, j])))
    ns = p.n_samples
    if dtype == np.float32:
        row = rng.standard_normal(ns, dtype=np.float32)
        row *= np.float32(math.sqrt(p.noise_var))
    else:
        row = rng.standard_normal(ns) * math.sqrt(p.noise_var)
    if events.shape[0] == 0:
        return row
    dist = np.hypot(events[:, 0] - st[0], events[:, 1] - st[1])
    nw = p.n_w
    for i in np.nonzero(dist < p.R_max)[0]:
        arrival = events[i, 2] + dist[i] / p.v
        if offsets is not None:
            arrival += offsets[i, j]
        k0 = math.ceil(arrival * p.f_hz)
        lo, hi = max(k0, 0), min(k0 + nw, ns)
        if lo >= hi:
            continue
        k = np.arange(lo, hi, dtype=np.float64)
        amp = math.exp(p.alpha * events[i, 3] - p.beta_att * dist[i])
        sd = amp * np.exp(-(k / p.f_hz - arrival) / p.tau)
        if p.likelihood == "mean":
            row[lo:hi] += sd.astype(row.dtype)
        else:
            row[lo:hi] += (sd * rng.standard_normal(hi - lo)).astype(row.dtype)
    return row


def sample_offsets(p: ModelParams, stations: np.ndarray, events: np.ndarray, seed: int,
                   sig_a: float) -> np.ndarray:
    """Latent arrival offsets (§Event Detections: the arrival is Gaussian
    around t + d/v): N(0, sig_a^2) for every (event, station within R_max),
    0 elsewhere, dense [n, n_st]."""
    rng = np.random.Generator(np.random.PCG64(np.random.SeedSequence([seed, 0xA771])))
    off = rng.normal(0.0, sig_a, size=(events.shape[0], stations.shape[0]))
    if events.shape[0]:
        d = np.hypot(events[:, None, 0] - stations[None, :, 0], events[:, None, 1] - stations[None, :, 1])
        off[d >= p.R_max] = 0.0
    return off


def sample_signals(p: ModelParams, stations: np.ndarray, events: np.ndarray, seed: int,
                   dtype=np.float64, threads: Optional[int] = None,
                   offsets: Optional[np.ndarray] = None) -> np.ndarray:
    """Signals [n_st, n_samples]; each station has its own seeded stream;
    ``offsets`` (dense [n, n_st]) shifts each arrival."""
    dtype = np.dtype(dtype).type
    n_st = stations.shape[0]
    out = np.empty((n_st, p.n_samples), dtype=dtype)

    def fill(j):
        out[j] = _station_row(p, stations[j], events, j, seed, dtype, offsets)

    threads = threads or min(16, os.cpu_count() or 1)
    if n_st * p.n_samples < 4_000_000 or threads <= 1:
        for j in range(n_st):
            fill(j)
    else:
        with _cf.ThreadPoolExecutor(threads) as ex:
            list(ex.map(fill, range(n_st)))
    return out


def make_world(p: ModelParams, stations: np.ndarray, seed: int, dtype=np.float64,
               events: Optional[np.ndarray] = None, sig_a: float = 0.0,
               offsets: Optional[np.ndarray] = None) -> World:
    """A seeded world; with ``sig_a`` > 0 (or explicit ``offsets``) the
    arrivals carry latent Gaussian offsets, returned in ``World.offsets``."""
    if events is None:
        events = sample_events(p, seed)
    stations = np.ascontiguousarray(stations, dtype=np.float64)
    if offsets is None and sig_a > 0.0:
        offsets = sample_offsets(p, stations, events, seed, sig_a)
    sig = sample_signals(p, stations, events, seed, dtype, offsets=offsets)
    return World(params=p, stations=stations, signals=sig, events=events, seed=seed, offsets=offsets)


def subworld(world: World, x0: float, x1: float, y0: float, y1: float) -> World:
    """Stations and true events inside [x0,x1) x [y0,y1), coordinates unchanged.

    The signals of the kept stations are the parent's rows, so a sub-world is a
    bounded sample of the same workload (used to time a slow CPU program).
    """
    st = world.stations
    keep = (st[:, 0] >= x0) & (st[:, 0] < x1) & (st[:, 1] >= y0) & (st[:, 1] < y1)
    ev = world.events
    kev = (ev[:, 0] >= x0) & (ev[:, 0] < x1) & (ev[:, 1] >= y0) & (ev[:, 1] < y1)
    off = None if world.offsets is None else world.offsets[kev][:, keep].copy()
    return World(params=world.params, stations=st[keep].copy(),
                 signals=world.signals[keep], events=ev[kev].copy(), seed=world.seed, offsets=off)


# --------------------------------------------------------------------------
# the workloads (sizes of the paper's toy world, scaled to the configurations)
# --------------------------------------------------------------------------
def config_tiny(seed: int = 1000) -> World:
    """200 x 200 km, 600 s, Lambda = 10, 4 stations on a 2 x 2 grid, 6000 f64 samples."""
    p = ModelParams(W=200.0, T=600.0, Lambda=10.0)
    return make_world(p, grid_stations(2, p.W), seed, np.float64)


def config_replay(seed: int = 1000, sig_a: float = 0.0) -> World:
    """1000 x 1000 km, 3600 s, Lambda = 500, 100 jittered stations, 36000 f64
    samples; with sig_a > 0 the arrivals carry latent Gaussian offsets."""
    p = ModelParams(W=1000.0, T=3600.0, Lambda=500.0)
    return make_world(p, jittered_grid_stations(10, p.W, seed), seed, np.float64, sig_a=sig_a)


def config_learned(seed: int = 1000) -> World:
    """The 1000 x 1000 km, 3600 s, Lambda = 500, 100-station world with float32
    signals, on which the learned birth proposal is compared with the plain one."""
    p = ModelParams(W=1000.0, T=3600.0, Lambda=500.0)
    return make_world(p, jittered_grid_stations(10, p.W, seed), seed, np.float32)


def config_scale(seed: int = 1000, dtype=np.float32, side_regions: int = 40,
                 T: float = 86400.0, likelihood: str = "variance", sig_a: float = 0.0) -> World:
    """4000 x 4000 km, 24 h, Lambda = 1e4, 1600 jittered stations, 864000 f32 samples.

    ``side_regions`` / ``T`` shrink the same density to a smaller world
    (Lambda scales with area x duration) for tests; ``sig_a`` > 0 gives the
    arrivals latent Gaussian offsets of that scale (seconds).
    """
    W = 100.0 * side_regions
    lam = 1.0e4 * (side_regions / 40.0) ** 2 * (T / 86400.0)
    p = ModelParams(W=W, T=T, Lambda=lam, likelihood=likelihood)
    return make_world(p, jittered_grid_stations(side_regions, W, seed), seed, dtype, sig_a=sig_a)


def batched_instances(n_instances: int = 256, seed: int = 2000):
    """The draws that size each instance of the batched workload, in order:
    (stations S, ModelParams) with S ~ logU[16,256], Lambda ~ logU[10,500],
    side ~ logU[200,2000] km (rounded to whole 100 km regions), T ~
    logU[600,7200] s.  Cheap: no signal is generated."""
    rng = np.random.Generator(np.random.PCG64(np.random.SeedSequence([seed, 0xBA7C])))
    out = []
    for i in range(n_instances):
        S = int(round(math.exp(rng.uniform(math.log(16), math.log(256)))))
        lam = math.exp(rng.uniform(math.log(10), math.log(500)))
        side = 100.0 * max(2, round(math.exp(rng.uniform(math.log(200), math.log(2000))) / 100.0))
        T = math.exp(rng.uniform(math.log(600), math.log(7200)))
        T = float(int(T * 10) / 10.0)
        out.append((S, ModelParams(W=side, T=T, Lambda=lam)))
    return out


def config_batched(n_instances: int = 256, seed: int = 2000, dtype=np.float32, indices=None):
    """Uneven independent instances (see batched_instances); ``indices``
    generates only those instances (the others are sized but not drawn), in
    the order given."""
    sizes = batched_instances(n_instances, seed)
    idx = range(n_instances) if indices is None else indices
    return [make_world(sizes[i][1], uniform_stations(sizes[i][0], sizes[i][1].W, seed + i), seed + 17 * i + 1, dtype)
            for i in idx]
