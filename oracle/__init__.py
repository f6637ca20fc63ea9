"""CPU oracle (TEST INFRASTRUCTURE ONLY).

Only ``tests/``, ``__graft_entry__.smoke()`` and ``bench.py``'s CPU-baseline leg
may import this package.  It wraps ``oracle.c`` (plain float64 C, compiled with
gcc) through ctypes and shares no code with the CUDA library.

Functions follow the paper's statement of the method:
  * ``log_prior`` / ``log_likelihood`` / ``log_density`` -- the joint density
    P(e, a, s) of §Generative Model of Seismic Signals (zero-jitter arrivals);
  * ``delta_loglik`` -- the change of the log-likelihood for one proposal;
  * ``log_alpha`` / ``log_alpha_pair`` -- the acceptance ratio of one explicit
    proposal (birth, death, move; the joint move of a pair);
  * ``run_serial`` -- Algorithm "Serial Metropolis Hastings";
  * ``run_chromatic`` -- Algorithm "Chromatic MH with Static Coloring" and the
    dynamic variant of §Chromatic MH with Dynamic Coloring (shift_mode=1);
  * ``cell_of`` / ``colour_of`` / ``blankets`` -- §Partitioning the World.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
from dataclasses import dataclass
from typing import Optional

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")


def _so_path(mutant: int = 0) -> str:
    return os.path.join(_HERE, "liboracle.so" if mutant == 0 else "liboracle_m%d.so" % mutant)


def build(force: bool = False, mutant: int = 0) -> str:
    """Compile liboracle.so with gcc (plain C, no FMA contraction).

    ``mutant`` > 0 builds a copy with a planted mistake (see ORC_MUTANT in
    oracle.c); only the pin tests use those.
    """
    so = _so_path(mutant)
    if force or not os.path.exists(so) or os.path.getmtime(so) < max(
            os.path.getmtime(_SRC), os.path.getmtime(os.path.join(_HERE, "oracle.h"))):
        tmp = so + ".tmp%d" % os.getpid()
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fopenmp", "-fPIC",
                               "-shared", "-DORC_MUTANT=%d" % mutant, "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, so)
    return so


class _Params(C.Structure):
    _fields_ = [(n, C.c_double) for n in
                ("W", "T", "Lambda", "v", "alpha", "beta_att", "tau", "t_s", "noise_var", "f_hz",
                 "R_max", "L", "p_birth", "p_death", "sig_xy", "sig_t", "sig_m")] + [
        ("n_w", C.c_int32), ("k_per_phase", C.c_int32), ("seed", C.c_uint64), ("commit", C.c_int32),
        ("lattice", C.c_int32), ("lat_nx", C.c_int32), ("lat_ny", C.c_int32), ("lat_nt", C.c_int32),
        ("lat_nm", C.c_int32), ("lat_nmax", C.c_int32), ("likelihood", C.c_int32)] + [
        (n, C.c_double) for n in ("lat_x0", "lat_dx", "lat_y0", "lat_dy", "lat_t0", "lat_dt",
                                  "lat_m0", "lat_dm", "p_pair", "sig_a", "p_arr", "sig_da")]


TRACE_DTYPE = np.dtype([("sweep", "<i4"), ("cell", "<i4"), ("step", "<i4"), ("type", "<i4"),
                        ("evaluated", "<i4"), ("accepted", "<i4"), ("n_before", "<i4"),
                        ("pad", "<i4"), ("dll", "<f8"), ("log_alpha", "<f8")])

_libs = {}


def lib(mutant: int = 0):
    if mutant not in _libs:
        L = C.CDLL(build(mutant=mutant))
        P = C.c_void_p
        d, i32, i64, u64 = C.c_double, C.c_int32, C.c_int64, C.c_uint64
        pd = C.POINTER(C.c_double)
        sig = {
            "orc_philox4x64": (None, [P, P, P]),
            "orc_world_new": (P, [C.POINTER(_Params), P, i32, P, i32, i64, i64]),
            "orc_world_free": (None, [P]),
            "orc_set_birth_table": (C.c_int, [P, P, i32, i32, i32, d]),
            "orc_set_birth_magnitude": (C.c_int, [P, P, d]),
            "orc_set_new": (P, [P, P, i64]),
            "orc_set_size": (i64, [P]),
            "orc_set_get": (None, [P, P, P]),
            "orc_set_free": (None, [P]),
            "orc_log_prior": (d, [P, P, i64]),
            "orc_log_likelihood": (d, [P, P, i64]),
            "orc_variance": (None, [P, P, i64, i32, i64, i64, P]),
            "orc_delta_loglik": (d, [P, P, i64, i64, P]),
            "orc_period": (i32, [P]),
            "orc_grid_dims": (None, [P, C.POINTER(i32), C.POINTER(i32)]),
            "orc_cell_of": (i32, [P, d, d, d, d]),
            "orc_cell_rect": (None, [P, d, d, i32, P]),
            "orc_colour_of": (i32, [P, i32]),
            "orc_shift": (None, [P, i64, pd, pd]),
            "orc_blankets": (None, [P, d, d, P]),
            "orc_log_alpha": (d, [P, d, d, i32, P, i64, i32, i64, P, C.POINTER(i32)]),
            "orc_log_alpha_pair": (d, [P, d, d, i32, P, i64, i64, i64, P, P, C.POINTER(i32)]),
            "orc_log_alpha_off": (d, [P, d, d, i32, P, P, i64, i32, i64, i32, P, P, C.POINTER(i32)]),
            "orc_log_prior_off": (d, [P, P, P, i64]),
            "orc_log_likelihood_off": (d, [P, P, P, i64]),
            "orc_set_new_w": (P, [P, P, P, P, i64]),
            "orc_set_offsets": (None, [P, P, P]),
            "orc_run_serial": (C.c_int, [P, P, i64, i64, P, i64, C.POINTER(i64), pd]),
            "orc_run_chromatic": (C.c_int, [P, P, i64, i64, i32, d, d, P, i64, C.POINTER(i64),
                                            i32, pd]),
        }
        for name, (res, args) in sig.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _libs[mutant] = L
    return _libs[mutant]


def _ptr(a: Optional[np.ndarray]):
    return None if a is None else a.ctypes.data_as(C.c_void_p)


def philox4x64(ctr, key) -> np.ndarray:
    c = np.ascontiguousarray(ctr, dtype=np.uint64)
    k = np.ascontiguousarray(key, dtype=np.uint64)
    out = np.zeros(4, dtype=np.uint64)
    lib().orc_philox4x64(_ptr(c), _ptr(k), _ptr(out))
    return out


@dataclass
class Lattice:
    """Finite coordinate grid for exact-enumeration worlds."""
    nx: int
    ny: int
    nt: int
    nm: int
    nmax: int
    x0: float
    dx: float
    y0: float
    dy: float
    t0: float
    dt: float
    m0: float
    dm: float


class World:
    """Oracle view of a worldgen.World plus the sampler's settings."""

    def __init__(self, world, p_birth=0.25, p_death=0.25, sig_xy=5.0, sig_t=2.0, sig_m=0.1,
                 k_per_phase=32, seed=1, commit=True, lattice: Optional[Lattice] = None,
                 mutant: int = 0, p_pair=0.0, sig_a=0.0, p_arr=0.0, sig_da=1.0):
        self._lib = lib(mutant)
        p = world.params
        self.world = world
        self.params = p
        prm = _Params()
        for n in ("W", "T", "Lambda", "v", "alpha", "beta_att", "tau", "t_s", "noise_var", "f_hz",
                  "R_max", "L"):
            setattr(prm, n, float(getattr(p, n)))
        prm.p_birth, prm.p_death, prm.p_pair = p_birth, p_death, p_pair
        prm.sig_a, prm.p_arr, prm.sig_da = sig_a, p_arr, sig_da
        self.latent = sig_a > 0.0
        prm.sig_xy, prm.sig_t, prm.sig_m = sig_xy, sig_t, sig_m
        prm.n_w = p.n_w
        prm.k_per_phase = k_per_phase
        prm.seed = seed
        prm.commit = 1 if commit else 0
        prm.likelihood = 1 if getattr(p, "likelihood", "variance") == "mean" else 0
        if lattice is not None:
            prm.lattice = 1
            for n in ("nx", "ny", "nt", "nm", "nmax"):
                setattr(prm, "lat_" + n, int(getattr(lattice, n)))
            for n in ("x0", "dx", "y0", "dy", "t0", "dt", "m0", "dm"):
                setattr(prm, "lat_" + n, float(getattr(lattice, n)))
        self._prm = prm
        self.k_per_phase = k_per_phase
        self._st = np.ascontiguousarray(world.stations, dtype=np.float64).reshape(-1, 2)
        sig = world.signals
        if sig.dtype not in (np.float32, np.float64):
            sig = sig.astype(np.float64)
        if sig.ndim != 2 or not sig.flags.c_contiguous:
            sig = np.ascontiguousarray(sig)
        self._sig = sig
        n_samp = sig.shape[1] if sig.ndim == 2 else 0
        self._h = self._lib.orc_world_new(C.byref(prm), _ptr(self._st), self._st.shape[0], _ptr(sig),
                                      1 if sig.dtype == np.float32 else 0, n_samp,
                                      sig.strides[0] // sig.itemsize if sig.shape[0] else n_samp)
        if not self._h:
            raise ValueError("oracle world rejected (with latent arrivals an event may reach at most 128 "
                             "stations)")

    def __del__(self):
        h = getattr(self, "_h", None)
        if h:
            self._lib.orc_world_free(h)
            self._h = None

    def set_birth_table(self, tab, mix=0.5):
        """Learned birth component: tab [ny, nx, nt] float32 weights over pixels
        of [0,W)^2 and time bins of [0,T), mixed with the uniform birth with
        weight mix; None removes it."""
        if tab is None:
            self._tab = None
            rc = self._lib.orc_set_birth_table(self._h, None, 0, 0, 0, 0.0)
        else:
            self._tab = np.ascontiguousarray(tab, dtype=np.float32)
            ny, nx, nt = self._tab.shape
            rc = self._lib.orc_set_birth_table(self._h, _ptr(self._tab), nx, ny, nt, float(mix))
        if rc != 0:
            raise ValueError("orc_set_birth_table rejected the table")

    def set_birth_magnitude(self, centre, half_width=0.25):
        """Magnitudes of the learned component: centre [ny, nx, nt] float32 (the
        table's shape); a table birth draws m uniform on [lo, lo + 2 h), lo =
        max(2, centre - h).  None returns to magnitudes from the prior."""
        if centre is None:
            self._mag = None
            rc = self._lib.orc_set_birth_magnitude(self._h, None, 0.0)
        else:
            self._mag = np.ascontiguousarray(centre, dtype=np.float32)
            rc = self._lib.orc_set_birth_magnitude(self._h, _ptr(self._mag), float(half_width))
        if rc != 0:
            raise ValueError("orc_set_birth_magnitude rejected the magnitudes")

    # ---- density -----------------------------------------------------------
    def _off(self, off, n):
        if off is None:
            return None
        off = np.ascontiguousarray(off, dtype=np.float64).reshape(n, self._st.shape[0])
        return off

    def log_prior(self, ev, off=None) -> float:
        """-Lambda + sum log beta(e), plus log N(delta; 0, sig_a^2) for every
        latent arrival offset (off: dense [n, n_st], None = 0)."""
        ev = np.ascontiguousarray(ev, dtype=np.float64).reshape(-1, 4)
        return self._lib.orc_log_prior_off(self._h, _ptr(ev), _ptr(self._off(off, ev.shape[0])), ev.shape[0])

    def log_likelihood(self, ev, off=None) -> float:
        ev = np.ascontiguousarray(ev, dtype=np.float64).reshape(-1, 4)
        return self._lib.orc_log_likelihood_off(self._h, _ptr(ev), _ptr(self._off(off, ev.shape[0])),
                                                ev.shape[0])

    def log_density(self, ev, off=None) -> float:
        return self.log_prior(ev, off) + self.log_likelihood(ev, off)

    def log_alpha_off(self, sx, sy, cell, ev, off, type_, idx=-1, station=-1, cand=None, cand_off=None):
        """Log acceptance ratio of one explicit proposal on a state with latent
        arrival offsets; type 4 moves the idx-th region event's offset at
        `station` to cand_off (a scalar)."""
        ev = np.ascontiguousarray(ev, dtype=np.float64).reshape(-1, 4)
        off = self._off(off, ev.shape[0])
        c = None if cand is None else np.ascontiguousarray(cand, dtype=np.float64)
        if cand_off is not None:
            cand_off = np.ascontiguousarray(np.atleast_1d(cand_off), dtype=np.float64)
        v = C.c_int32()
        la = self._lib.orc_log_alpha_off(self._h, sx, sy, int(cell), _ptr(ev), _ptr(off), ev.shape[0],
                                         int(type_), int(idx), int(station), _ptr(c), _ptr(cand_off),
                                         C.byref(v))
        return la, bool(v.value)

    def variance(self, ev, j, k0, k1) -> np.ndarray:
        ev = np.ascontiguousarray(ev, dtype=np.float64).reshape(-1, 4)
        out = np.empty(k1 - k0, dtype=np.float64)
        self._lib.orc_variance(self._h, _ptr(ev), ev.shape[0], int(j), int(k0), int(k1), _ptr(out))
        return out

    def delta_loglik(self, ev, old_idx: int = -1, cand=None) -> float:
        ev = np.ascontiguousarray(ev, dtype=np.float64).reshape(-1, 4)
        c = None if cand is None else np.ascontiguousarray(cand, dtype=np.float64)
        return self._lib.orc_delta_loglik(self._h, _ptr(ev), ev.shape[0], int(old_idx), _ptr(c))

    # ---- partition ---------------------------------------------------------
    def period(self) -> int:
        return self._lib.orc_period(self._h)

    def grid_dims(self):
        a, b = C.c_int32(), C.c_int32()
        self._lib.orc_grid_dims(self._h, C.byref(a), C.byref(b))
        return a.value, b.value

    def cell_of(self, sx, sy, x, y) -> int:
        return self._lib.orc_cell_of(self._h, sx, sy, x, y)

    def cell_rect(self, sx, sy, cell) -> np.ndarray:
        r = np.zeros(4)
        self._lib.orc_cell_rect(self._h, sx, sy, int(cell), _ptr(r))
        return r

    def colour_of(self, cell) -> int:
        return self._lib.orc_colour_of(self._h, int(cell))

    def shift(self, sweep):
        a, b = C.c_double(), C.c_double()
        self._lib.orc_shift(self._h, int(sweep), C.byref(a), C.byref(b))
        return a.value, b.value

    def blankets(self, sx, sy) -> np.ndarray:
        ncx, ncy = self.grid_dims()
        m = np.zeros((ncx * ncy, self._st.shape[0]), dtype=np.uint8)
        self._lib.orc_blankets(self._h, sx, sy, _ptr(m))
        return m

    def log_alpha(self, sx, sy, cell, ev, type_, idx=-1, cand=None):
        ev = np.ascontiguousarray(ev, dtype=np.float64).reshape(-1, 4)
        c = None if cand is None else np.ascontiguousarray(cand, dtype=np.float64)
        v = C.c_int32()
        la = self._lib.orc_log_alpha(self._h, sx, sy, int(cell), _ptr(ev), ev.shape[0], int(type_),
                                 int(idx), _ptr(c), C.byref(v))
        return la, bool(v.value)

    def log_alpha_pair(self, sx, sy, cell, ev, i, j, cand1, cand2):
        """Log acceptance ratio of the joint move of the region's i-th and j-th
        events to cand1 and cand2 (§MH moves, "Joint Events Move")."""
        ev = np.ascontiguousarray(ev, dtype=np.float64).reshape(-1, 4)
        c1 = np.ascontiguousarray(cand1, dtype=np.float64)
        c2 = np.ascontiguousarray(cand2, dtype=np.float64)
        v = C.c_int32()
        la = self._lib.orc_log_alpha_pair(self._h, sx, sy, int(cell), _ptr(ev), ev.shape[0], int(i),
                                          int(j), _ptr(c1), _ptr(c2), C.byref(v))
        return la, bool(v.value)

    # ---- samplers ----------------------------------------------------------
    def _set(self, ev, ids, off=None):
        ev = np.ascontiguousarray(ev, dtype=np.float64).reshape(-1, 4)
        if ids is None:
            ids = np.arange(ev.shape[0], dtype=np.uint64)
        ids = np.ascontiguousarray(ids, dtype=np.uint64)
        return self._lib.orc_set_new_w(self._h, _ptr(ev), _ptr(ids), _ptr(self._off(off, ev.shape[0])),
                                       ev.shape[0])

    def _get(self, h):
        n = self._lib.orc_set_size(h)
        ev = np.zeros((n, 4))
        ids = np.zeros(n, dtype=np.uint64)
        self._lib.orc_set_get(h, _ptr(ev), _ptr(ids))
        self.last_offsets = np.zeros((n, self._st.shape[0]))
        if n and self._st.shape[0]:
            self._lib.orc_set_offsets(self._h, h, _ptr(self.last_offsets))
        self._lib.orc_set_free(h)
        return ev, ids

    def run_serial(self, ev, n_steps, ids=None, step0=0, trace_cap=0, off=None):
        """Serial MH; with latent arrivals the final state's dense offsets
        are left in ``self.last_offsets`` (and ``off`` seeds the start's)."""
        h = self._set(ev, ids, off)
        tr = np.zeros(trace_cap, dtype=TRACE_DTYPE)
        nt = C.c_int64()
        dlp = C.c_double()
        rc = self._lib.orc_run_serial(self._h, h, step0, n_steps, _ptr(tr), trace_cap, C.byref(nt),
                                  C.byref(dlp))
        ev2, ids2 = self._get(h)
        if rc != 0:
            raise RuntimeError("orc_run_serial failed: %d" % rc)
        return ev2, ids2, tr[: min(nt.value, trace_cap)], dlp.value

    def run_chromatic(self, ev, n_sweeps, ids=None, sweep0=0, shift_mode=1, sx=0.0, sy=0.0,
                      trace_cap=0, threads=1, off=None):
        h = self._set(ev, ids, off)
        tr = np.zeros(trace_cap, dtype=TRACE_DTYPE)
        nt = C.c_int64()
        dlp = C.c_double()
        rc = self._lib.orc_run_chromatic(self._h, h, sweep0, n_sweeps, shift_mode, sx, sy, _ptr(tr),
                                     trace_cap, C.byref(nt), threads, C.byref(dlp))
        ev2, ids2 = self._get(h)
        if rc != 0:
            raise RuntimeError("orc_run_chromatic failed: %d" % rc)
        return ev2, ids2, tr[: min(nt.value, trace_cap)], dlp.value
