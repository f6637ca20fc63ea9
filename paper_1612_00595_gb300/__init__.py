"""Python binding of libchromh (include/chromh.h): argument marshalling only.

Every step of the sampler runs in the CUDA library; this module converts
numpy arrays / torch tensors into pointers and sizes and back.  Importing it
loads ``libchromh.so`` from this directory and raises if it is missing: there
is no fallback implementation.

Names follow the C ABI: ``create_model``, ``partition_and_color``,
``run_sweeps``, ``read_state`` (the calls of the paper's problem statement:
events, stations and signals in; the event hypothesis out), plus trace,
timing, checkpoint and test hooks.
"""
from __future__ import annotations

import ctypes as C
import os
from typing import Optional

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libchromh.so")

CMH_OK = 0
ERRORS = {
    -1: "CMH_ERR_ARG", -2: "CMH_ERR_GEOMETRY", -3: "CMH_ERR_NONFINITE", -4: "CMH_ERR_OOM",
    -5: "CMH_ERR_CAPACITY", -6: "CMH_ERR_TIMEOUT", -7: "CMH_ERR_CUDA", -8: "CMH_ERR_STATE",
}
F64, F32 = 0, 1


class ChromhError(RuntimeError):
    def __init__(self, code: int, what: str):
        self.code = code
        super().__init__("%s failed: %s (%d, %s)" % (what, ERRORS.get(code, "?"), code, strerror(code)))


class Params(C.Structure):
    _fields_ = [(n, C.c_double) for n in
                ("W", "T", "Lambda", "v", "alpha", "beta_att", "tau", "t_s", "noise_var", "f_hz",
                 "R_max", "p_birth", "p_death", "sig_xy", "sig_t", "sig_m")] + [
        ("k_per_phase", C.c_int32), ("commit", C.c_int32), ("seed", C.c_uint64), ("dtype", C.c_int32),
        ("ev_capacity", C.c_int32), ("frozen_capacity", C.c_int32), ("block_threads", C.c_int32),
        ("stage_samples", C.c_int32), ("schedule", C.c_int32), ("ctas_per_sm", C.c_int32),
        ("likelihood", C.c_int32), ("max_events", C.c_int64), ("p_pair", C.c_double),
        ("sig_a", C.c_double), ("p_arr", C.c_double), ("sig_da", C.c_double)]


class Tuning(C.Structure):
    _fields_ = [("schedule", C.c_int32), ("stage_samples", C.c_int32), ("ctas_per_sm", C.c_int32),
                ("ms_per_sweep", C.c_double), ("n_tried", C.c_int32), ("tried_schedule", C.c_int32 * 16),
                ("tried_stage", C.c_int32 * 16), ("tried_ctas", C.c_int32 * 16), ("tried_ms", C.c_double * 16)]

    def as_dict(self):
        n = self.n_tried
        return {"schedule": self.schedule, "stage_samples": self.stage_samples, "ctas_per_sm": self.ctas_per_sm,
                "ms_per_sweep": self.ms_per_sweep,
                "tried": [{"schedule": self.tried_schedule[i], "stage_samples": self.tried_stage[i],
                           "ctas_per_sm": self.tried_ctas[i], "ms_per_sweep": self.tried_ms[i]} for i in range(n)]}


class Grid(C.Structure):
    _fields_ = [("L", C.c_double)]


class Stats(C.Structure):
    _fields_ = [("proposed", C.c_uint64 * 3), ("evaluated", C.c_uint64 * 3), ("accepted", C.c_uint64 * 3),
                ("sweeps", C.c_int64), ("n_events", C.c_int64), ("phase_ms", C.c_double),
                ("phase_launches", C.c_int64), ("kernel_launches", C.c_int64),
                ("priced_samples", C.c_uint64), ("rewritten_samples", C.c_uint64), ("spill_bytes", C.c_int64),
                ("pair", C.c_uint64 * 3), ("arrival", C.c_uint64 * 3), ("unique_samples", C.c_uint64)]

    def as_dict(self):
        return {"proposed": list(self.proposed), "evaluated": list(self.evaluated),
                "accepted": list(self.accepted), "sweeps": self.sweeps, "n_events": self.n_events,
                "phase_ms": self.phase_ms, "phase_launches": self.phase_launches,
                "kernel_launches": self.kernel_launches, "priced_samples": self.priced_samples,
                "rewritten_samples": self.rewritten_samples, "spill_bytes": self.spill_bytes,
                "pair": list(self.pair), "arrival": list(self.arrival), "unique_samples": self.unique_samples}


TRACE_DTYPE = np.dtype([("sweep", "<i4"), ("cell", "<i4"), ("step", "<i4"), ("type", "<i4"),
                        ("evaluated", "<i4"), ("accepted", "<i4"), ("n_before", "<i4"),
                        ("written", "<i4"), ("dll", "<f8"), ("log_alpha", "<f8")])

EXPORTS = ["cmh_create_model", "cmh_partition_and_color", "cmh_run_sweeps", "cmh_read_state", "cmh_sync",
           "cmh_read_state_async", "cmh_read_state_fetch",
           "cmh_log_density", "cmh_set_trace", "cmh_read_trace", "cmh_set_timing", "cmh_read_shift",
           "cmh_checkpoint", "cmh_restore", "cmh_destroy", "cmh_strerror", "cmh_philox4x64",
           "cmh_gaussian_loglik_noalloc", "cmh_batch_create", "cmh_batch_run_sweeps", "cmh_batch_destroy",
           "cmh_autotune", "cmh_batch_sync", "cmh_batch_groups", "cmh_set_birth_table", "cmh_set_birth_magnitude",
           "cmh_net_param_count", "cmh_net_create", "cmh_net_destroy", "cmh_net_get_params", "cmh_net_set_params",
           "cmh_net_forward", "cmh_net_gradients", "cmh_net_train", "cmh_net_birth_table",
           "cmh_set_arrival_offsets", "cmh_read_arrival_offsets", "cmh_measure_alu_peaks",
           "cmh_test_hold_region"]


def _load():
    if not os.path.exists(LIB_PATH):
        raise ImportError("libchromh.so is not built (run __graft_entry__.build()); "
                          "the sampler has no CPU fallback")
    L = C.CDLL(LIB_PATH)
    P, i32, i64 = C.c_void_p, C.c_int32, C.c_int64
    sig = {
        "cmh_create_model": (C.c_int, [P, i64, P, i32, P, i64, i64, i32, i32, C.POINTER(Params), P,
                                       C.POINTER(P)]),
        "cmh_partition_and_color": (C.c_int, [P, C.POINTER(Grid), i32, C.c_double, C.c_double,
                                              C.POINTER(i32)]),
        "cmh_run_sweeps": (C.c_int, [P, i64]),
        "cmh_read_state_async": (C.c_int, [P, i32]),
        "cmh_read_state_fetch": (C.c_int, [P, i32, P, P, i64, C.POINTER(i64), C.POINTER(C.c_double), P]),
        "cmh_set_arrival_offsets": (C.c_int, [P, P, i64, i32]),
        "cmh_read_arrival_offsets": (C.c_int, [P, P, i64, C.POINTER(i64)]),
        "cmh_read_state": (C.c_int, [P, P, P, i64, C.POINTER(i64), C.POINTER(C.c_double),
                                     C.POINTER(Stats)]),
        "cmh_sync": (C.c_int, [P]),
        "cmh_log_density": (C.c_int, [P, C.POINTER(C.c_double)]),
        "cmh_set_trace": (C.c_int, [P, i64]),
        "cmh_read_trace": (C.c_int, [P, P, i64, C.POINTER(i64)]),
        "cmh_set_timing": (C.c_int, [P, i32]),
        "cmh_read_shift": (C.c_int, [P, C.POINTER(C.c_double), C.POINTER(C.c_double)]),
        "cmh_checkpoint": (C.c_int, [P, P, C.POINTER(C.c_size_t)]),
        "cmh_restore": (C.c_int, [P, P, C.c_size_t]),
        "cmh_destroy": (None, [P]),
        "cmh_strerror": (C.c_char_p, [C.c_int]),
        "cmh_philox4x64": (C.c_int, [P, P, P, i64]),
        "cmh_measure_alu_peaks": (C.c_int, [C.POINTER(C.c_double), C.POINTER(C.c_double), P]),
        "cmh_test_hold_region": (C.c_int, [P, i32, C.c_uint32]),
        "cmh_gaussian_loglik_noalloc": (C.c_int, [P, P, i32, i64, i64, i32, C.POINTER(C.c_double), P]),
        "cmh_batch_create": (C.c_int, [C.POINTER(P), i32, P, C.POINTER(P)]),
        "cmh_batch_run_sweeps": (C.c_int, [P, i64]),
        "cmh_batch_destroy": (None, [P]),
        "cmh_autotune": (C.c_int, [P, i32, C.POINTER(Tuning)]),
        "cmh_batch_sync": (C.c_int, [P]),
        "cmh_set_birth_table": (C.c_int, [P, P, i32, i32, i32, C.c_double]),
        "cmh_set_birth_magnitude": (C.c_int, [P, P, C.c_double]),
        "cmh_net_param_count": (i64, []),
        "cmh_net_create": (C.c_int, [i32, C.c_uint64, P, C.POINTER(P)]),
        "cmh_net_destroy": (None, [P]),
        "cmh_net_get_params": (C.c_int, [P, P]),
        "cmh_net_set_params": (C.c_int, [P, P]),
        "cmh_net_forward": (C.c_int, [P, P, i32, P]),
        "cmh_net_gradients": (C.c_int, [P, P, P, P, P, i32, P, C.POINTER(C.c_double)]),
        "cmh_net_train": (C.c_int, [P, P, i32, i32, C.c_double, C.POINTER(C.c_double)]),
        "cmh_net_birth_table": (C.c_int, [P, P, P, P, i32, i32, i32, i32, C.c_double, P, P]),
        "cmh_batch_groups": (C.c_int, [P, C.POINTER(i32), P, P, i32]),
    }
    for name, (res, args) in sig.items():
        f = getattr(L, name)
        f.restype = res
        f.argtypes = args
    return L


lib = _load()


def strerror(code: int) -> str:
    return lib.cmh_strerror(code).decode()


def _check(rc: int, what: str):
    if rc != CMH_OK:
        raise ChromhError(rc, what)


def _ptr(a):
    return None if a is None else C.c_void_p(a.ctypes.data)


def make_params(model_params, *, k_per_phase=32, seed=1, dtype=F64, p_birth=0.25, p_death=0.25,
                sig_xy=5.0, sig_t=2.0, sig_m=0.1, commit=True, ev_capacity=0, frozen_capacity=0,
                block_threads=0, stage_samples=0, schedule=0, ctas_per_sm=0, max_events=0,
                p_pair=0.0, sig_a=0.0, p_arr=0.0, sig_da=1.0) -> Params:
    """cmh_params from an object with the model fields (e.g. worldgen.ModelParams).
    ``p_pair`` > 0 turns on the joint move of a pair of events; ``sig_a`` > 0
    makes arrival times latent and ``p_arr`` the share of the arrival-time
    move of step ``sig_da`` (float32: the variance reading without staging)."""
    p = Params()
    for n in ("W", "T", "Lambda", "v", "alpha", "beta_att", "tau", "t_s", "noise_var", "f_hz", "R_max"):
        setattr(p, n, float(getattr(model_params, n)))
    p.p_birth, p.p_death = p_birth, p_death
    p.sig_xy, p.sig_t, p.sig_m = sig_xy, sig_t, sig_m
    p.k_per_phase = k_per_phase
    p.commit = 1 if commit else 0
    p.seed = seed
    p.dtype = dtype
    p.ev_capacity = ev_capacity
    p.frozen_capacity = frozen_capacity
    p.block_threads = block_threads
    p.stage_samples = stage_samples
    p.schedule = schedule
    p.ctas_per_sm = ctas_per_sm
    p.likelihood = 1 if getattr(model_params, "likelihood", "variance") == "mean" else 0
    p.max_events = max_events
    p.p_pair = p_pair
    p.sig_a, p.p_arr, p.sig_da = sig_a, p_arr, sig_da
    return p


class Model:
    """A cmh_model handle (see create_model)."""

    def __init__(self, handle, keep):
        self._h = handle
        self._keep = keep

    def __del__(self):
        self.destroy()

    def destroy(self):
        h = getattr(self, "_h", None)
        if h:
            lib.cmh_destroy(h)
            self._h = None

    @property
    def handle(self):
        return self._h

    # ---- the four calls of the problem statement -------------------------
    def partition_and_color(self, L: float, shift_mode: int = 1, sx: float = 0.0, sy: float = 0.0) -> int:
        n = C.c_int32()
        _check(lib.cmh_partition_and_color(self._h, C.byref(Grid(L)), shift_mode, sx, sy, C.byref(n)),
               "cmh_partition_and_color")
        return n.value

    def run_sweeps(self, n: int):
        _check(lib.cmh_run_sweeps(self._h, int(n)), "cmh_run_sweeps")

    def set_birth_table(self, tab, mix: float = 0.5):
        """Learned birth component: tab [ny, nx, nt] weights over pixels of
        [0,W)^2 and time bins of [0,T), mixed with the uniform birth with
        weight mix; None removes it."""
        if tab is None:
            _check(lib.cmh_set_birth_table(self._h, None, 0, 0, 0, 0.0), "cmh_set_birth_table")
            return
        t = np.ascontiguousarray(tab, dtype=np.float32)
        ny, nx, nt = t.shape
        _check(lib.cmh_set_birth_table(self._h, _ptr(t), nx, ny, nt, float(mix)), "cmh_set_birth_table")

    def set_birth_magnitude(self, centre, half_width: float = 0.25):
        """Learned magnitudes for the table births: centre [ny, nx, nt] (the
        table's shape); a table birth draws m uniform on [lo, lo + 2 h), lo =
        max(2, centre - h).  None returns to magnitudes from the prior."""
        if centre is None:
            _check(lib.cmh_set_birth_magnitude(self._h, None, 0.0), "cmh_set_birth_magnitude")
            return
        c = np.ascontiguousarray(centre, dtype=np.float32)
        _check(lib.cmh_set_birth_magnitude(self._h, _ptr(c), float(half_width)), "cmh_set_birth_magnitude")

    def autotune(self, trial_sweeps: int = 8) -> dict:
        """Time each launch configuration from a checkpoint, keep the fastest,
        restore the checkpoint (the chain is unchanged)."""
        t = Tuning()
        _check(lib.cmh_autotune(self._h, int(trial_sweeps), C.byref(t)), "cmh_autotune")
        return t.as_dict()

    def read_state(self, cap: Optional[int] = None):
        """(events [n,4] float64, ids [n] uint64, log_density, stats dict)."""
        n = C.c_int64()
        exact = cap is not None
        if cap is None:   # one call when the last count (plus room) suffices
            cap = getattr(self, "_last_n", 0) + 1024
        while True:
            ev = np.zeros((cap, 4), dtype=np.float64)
            ids = np.zeros(cap, dtype=np.uint64)
            lp = C.c_double()
            st = Stats()
            _check(lib.cmh_read_state(self._h, _ptr(ev), _ptr(ids), cap, C.byref(n), C.byref(lp), C.byref(st)),
                   "cmh_read_state")
            if exact or n.value <= cap:
                break
            cap = n.value
        self._last_n = n.value
        k = min(cap, n.value)
        return ev[:k], ids[:k], lp.value, st.as_dict()

    def set_arrival_offsets(self, off):
        """cmh_set_arrival_offsets: latent arrival offsets [n_events, n_stations]
        of the initial events (before partition_and_color)."""
        off = np.ascontiguousarray(off, dtype=np.float64)
        if off.ndim != 2:
            raise ValueError("offsets must be [n_events, n_stations]")
        _check(lib.cmh_set_arrival_offsets(self._h, _ptr(off), off.shape[0], off.shape[1]),
               "cmh_set_arrival_offsets")

    def read_arrival_offsets(self, n_stations: int):
        """cmh_read_arrival_offsets: [n, n_stations] offsets of the current
        events, rows in read_state's order (0 where an event does not reach)."""
        n = C.c_int64()
        _check(lib.cmh_read_arrival_offsets(self._h, None, 0, C.byref(n)), "cmh_read_arrival_offsets")
        out = np.zeros((n.value, n_stations), dtype=np.float64)
        _check(lib.cmh_read_arrival_offsets(self._h, _ptr(out), n.value, C.byref(n)), "cmh_read_arrival_offsets")
        return out

    def read_state_async(self, slot: int):
        """cmh_read_state_async: enqueue a copy of the state into slot 0 or 1."""
        _check(lib.cmh_read_state_async(self._h, int(slot)), "cmh_read_state_async")

    def read_state_fetch(self, slot: int):
        """cmh_read_state_fetch: the state of the slot's request, as read_state."""
        n = C.c_int64()
        _check(lib.cmh_read_state_fetch(self._h, int(slot), None, None, 0, C.byref(n), None, None),
               "cmh_read_state_fetch")
        cap = n.value
        ev = np.zeros((cap, 4), dtype=np.float64)
        ids = np.zeros(cap, dtype=np.uint64)
        lp = C.c_double()
        st = Stats()
        _check(lib.cmh_read_state_fetch(self._h, int(slot), _ptr(ev) if cap else None, _ptr(ids) if cap else None,
                                        cap, C.byref(n), C.byref(lp), C.byref(st)), "cmh_read_state_fetch")
        return ev, ids, lp.value, st.as_dict()

    # ---- extras -------------------------------------------------------------
    def sync(self):
        _check(lib.cmh_sync(self._h), "cmh_sync")

    def log_density(self) -> float:
        out = C.c_double()
        _check(lib.cmh_log_density(self._h, C.byref(out)), "cmh_log_density")
        return out.value

    def set_trace(self, capacity: int):
        _check(lib.cmh_set_trace(self._h, int(capacity)), "cmh_set_trace")

    def read_trace(self) -> np.ndarray:
        n = C.c_int64()
        _check(lib.cmh_read_trace(self._h, None, 0, C.byref(n)), "cmh_read_trace")
        out = np.zeros(n.value, dtype=TRACE_DTYPE)
        _check(lib.cmh_read_trace(self._h, _ptr(out), n.value, C.byref(n)), "cmh_read_trace")
        return out

    def test_hold_region(self, cell: int, wait_limit: int = 0):
        """cmh_test_hold_region: region `cell` never announces its phase, so
        its higher-colour neighbours' bounded waits run out (test hook)."""
        _check(lib.cmh_test_hold_region(self._h, int(cell), int(wait_limit)), "cmh_test_hold_region")

    def set_timing(self, enable: bool):
        _check(lib.cmh_set_timing(self._h, 1 if enable else 0), "cmh_set_timing")

    def read_shift(self):
        a, b = C.c_double(), C.c_double()
        _check(lib.cmh_read_shift(self._h, C.byref(a), C.byref(b)), "cmh_read_shift")
        return a.value, b.value

    def checkpoint(self) -> bytes:
        n = C.c_size_t()
        _check(lib.cmh_checkpoint(self._h, None, C.byref(n)), "cmh_checkpoint")
        buf = C.create_string_buffer(n.value)
        _check(lib.cmh_checkpoint(self._h, buf, C.byref(n)), "cmh_checkpoint")
        return buf.raw[: n.value]

    def restore(self, blob: bytes):
        buf = C.create_string_buffer(blob, len(blob))
        _check(lib.cmh_restore(self._h, buf, len(blob)), "cmh_restore")


def create_model(events, stations, signals, params: Params, stream=None) -> Model:
    """cmh_create_model.

    events   [n, 4] float64 (x, y, t, m) or None for the empty hypothesis
    stations [n_st, 2] float64
    signals  [n_st, n_samples]: numpy float32/float64 (host) or a CUDA torch
             tensor (device; its current stream orders the copy unless
             ``stream`` is given)
    stream   an int cudaStream_t or a torch.cuda.Stream; None lets the model
             create its own stream
    """
    ev = np.zeros((0, 4)) if events is None else np.ascontiguousarray(events, dtype=np.float64).reshape(-1, 4)
    st = np.ascontiguousarray(stations, dtype=np.float64).reshape(-1, 2)
    on_device = 0
    keep = [ev, st]
    if hasattr(signals, "data_ptr") and getattr(signals, "is_cuda", False):
        import torch
        if signals.dtype not in (torch.float32, torch.float64) or signals.dim() != 2 or signals.stride(1) != 1:
            raise ValueError("device signals must be a 2-D row-major float32/float64 tensor")
        sig_ptr = C.c_void_p(signals.data_ptr())
        n_st, n_samp = signals.shape
        pitch = signals.stride(0)
        sdt = F32 if signals.dtype == torch.float32 else F64
        on_device = 1
        if stream is None:
            stream = torch.cuda.current_stream(signals.device)
        keep.append(signals)
    else:
        sig = np.asarray(signals)
        if sig.dtype not in (np.float32, np.float64):
            sig = sig.astype(np.float64)
        if sig.ndim != 2:
            sig = sig.reshape(st.shape[0], -1)
        sig = np.ascontiguousarray(sig)
        n_st, n_samp = sig.shape
        pitch = n_samp
        sdt = F32 if sig.dtype == np.float32 else F64
        sig_ptr = _ptr(sig) if n_st else None
        keep.append(sig)
    if hasattr(stream, "cuda_stream"):
        stream = stream.cuda_stream
    h = C.c_void_p()
    _check(lib.cmh_create_model(_ptr(ev) if len(ev) else None, ev.shape[0], _ptr(st) if len(st) else None,
                                st.shape[0], sig_ptr, n_samp, pitch, sdt, on_device, C.byref(params),
                                C.c_void_p(stream) if stream else None, C.byref(h)),
           "cmh_create_model")
    return Model(h, keep[:0])


class Batch:
    """A cmh_batch: independent float32 models swept together (see create_batch)."""

    def __init__(self, handle, models):
        self._h = handle
        self._models = list(models)   # the batch refers to them: keep them alive

    def __del__(self):
        self.destroy()

    def destroy(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            lib.cmh_batch_destroy(self._h)
        self._h = None

    def run_sweeps(self, n: int):
        """Enqueue n sweeps of every model (asynchronous; see sync)."""
        _check(lib.cmh_batch_run_sweeps(self._h, n), "cmh_batch_run_sweeps")

    def sync(self):
        _check(lib.cmh_batch_sync(self._h), "cmh_batch_sync")

    def groups(self):
        """[(models, persistent-launch CTAs)] per shared-memory group."""
        n = C.c_int32()
        mp = (C.c_int32 * 3)()
        gp = (C.c_int32 * 3)()
        _check(lib.cmh_batch_groups(self._h, C.byref(n), mp, gp, 3), "cmh_batch_groups")
        return [(mp[i], gp[i]) for i in range(n.value)]


def create_batch(models, stream=None) -> Batch:
    """One persistent launch per sweep for every region of every model (each
    partitioned, float32, no staging); destroy the batch before the models."""
    arr = (C.c_void_p * len(models))(*[m._h.value for m in models])
    if hasattr(stream, "cuda_stream"):
        stream = stream.cuda_stream
    h = C.c_void_p()
    _check(lib.cmh_batch_create(arr, len(models), C.c_void_p(stream) if stream else None, C.byref(h)),
           "cmh_batch_create")
    return Batch(h, models)


NET_OUT = 4101        # 4096 tile pixels, "no event", time mean / log sd, magnitude mean / log sd
NET_WINDOW = 256      # samples per window
NET_STATIONS = 64     # stations per tile (8 x 8)


class Net:
    """The network behind the learned birth proposal (see cmh_net_* in the header)."""

    def __init__(self, max_batch: int = 256, seed: int = 1, stream=None):
        if hasattr(stream, "cuda_stream"):
            stream = stream.cuda_stream
        self._h = C.c_void_p()
        _check(lib.cmh_net_create(int(max_batch), int(seed), C.c_void_p(stream) if stream else None,
                                  C.byref(self._h)), "cmh_net_create")
        self.max_batch = max_batch
        self.n_params = int(lib.cmh_net_param_count())

    def __del__(self):
        self.destroy()

    def destroy(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            lib.cmh_net_destroy(self._h)
        self._h = None

    def params(self) -> np.ndarray:
        out = np.zeros(self.n_params, dtype=np.float32)
        _check(lib.cmh_net_get_params(self._h, _ptr(out)), "cmh_net_get_params")
        return out

    def set_params(self, p):
        p = np.ascontiguousarray(p, dtype=np.float32)
        assert p.size == self.n_params
        _check(lib.cmh_net_set_params(self._h, _ptr(p)), "cmh_net_set_params")

    def forward(self, features) -> np.ndarray:
        x = np.ascontiguousarray(features, dtype=np.float32)
        b = x.shape[0]
        out = np.zeros((b, NET_OUT), dtype=np.float32)
        _check(lib.cmh_net_forward(self._h, _ptr(x), b, _ptr(out)), "cmh_net_forward")
        return out

    def gradients(self, features, label, t_label, m_label):
        x = np.ascontiguousarray(features, dtype=np.float32)
        lab = np.ascontiguousarray(label, dtype=np.int32)
        tl = np.ascontiguousarray(t_label, dtype=np.float32)
        ml = np.ascontiguousarray(m_label, dtype=np.float32)
        g = np.zeros(self.n_params, dtype=np.float32)
        loss = C.c_double()
        _check(lib.cmh_net_gradients(self._h, _ptr(x), _ptr(lab), _ptr(tl), _ptr(ml), x.shape[0], _ptr(g),
                                     C.byref(loss)), "cmh_net_gradients")
        return g, loss.value

    def train(self, geometry: Model, steps: int, batch: int = 256, lr: float = 1e-3) -> float:
        loss = C.c_double()
        _check(lib.cmh_net_train(self._h, geometry._h, int(steps), int(batch), float(lr), C.byref(loss)),
               "cmh_net_train")
        return loss.value

    def birth_table(self, model: Model, tiles, origins, nx: int, ny: int, nt: int, hop_s: float = 12.8,
                    magnitudes: bool = False):
        """The birth table [ny, nx, nt] of the model's signals; with
        ``magnitudes`` also the window centres (weighted mean predicted
        magnitude per entry): returns (table, centres)."""
        t = np.ascontiguousarray(tiles, dtype=np.int32)
        o = np.ascontiguousarray(origins, dtype=np.float64)
        tab = np.zeros((ny, nx, nt), dtype=np.float32)
        mag = np.zeros((ny, nx, nt), dtype=np.float32) if magnitudes else None
        _check(lib.cmh_net_birth_table(self._h, model._h, _ptr(t), _ptr(o), t.shape[0], nx, ny, nt, float(hop_s),
                                       _ptr(tab), _ptr(mag) if magnitudes else None), "cmh_net_birth_table")
        return (tab, mag) if magnitudes else tab


def grid_tiles(n_side: int, spacing: float, tile: int = 8):
    """Tiles of tile x tile stations of a row-major n_side x n_side station grid
    (station r * n_side + c at cell (c, r) of side `spacing`): every tile origin
    (i0, j0) with i0, j0 in [0, n_side - tile]; returns (tiles [n][64], origins [n][2] km)."""
    tiles, origins = [], []
    for i0 in range(n_side - tile + 1):
        for j0 in range(n_side - tile + 1):
            tiles.append([(i0 + r) * n_side + (j0 + c) for r in range(tile) for c in range(tile)])
            origins.append([j0 * spacing, i0 * spacing])
    return np.array(tiles, dtype=np.int32), np.array(origins, dtype=np.float64)


def partition_and_color(model: Model, L: float, shift_mode: int = 1, sx: float = 0.0, sy: float = 0.0):
    return model.partition_and_color(L, shift_mode, sx, sy)


def run_sweeps(model: Model, n: int):
    return model.run_sweeps(n)


def read_state(model: Model, cap: Optional[int] = None):
    return model.read_state(cap)


def measure_alu_peaks(stream=None):
    """cmh_measure_alu_peaks: (MUFU operations/s, float32 flops/s) of the
    current device, each the best of three timed launches."""
    a, b = C.c_double(), C.c_double()
    st = None if stream is None else C.c_void_p(stream.cuda_stream)
    _check(lib.cmh_measure_alu_peaks(C.byref(a), C.byref(b), st), "cmh_measure_alu_peaks")
    return a.value, b.value


def philox4x64(ctr, key) -> np.ndarray:
    """Device Philox4x64-10 blocks for counters ctr [n, 4] and key [2]."""
    c = np.ascontiguousarray(ctr, dtype=np.uint64).reshape(-1, 4)
    k = np.ascontiguousarray(key, dtype=np.uint64).reshape(2)
    out = np.zeros_like(c)
    _check(lib.cmh_philox4x64(_ptr(c), _ptr(k), _ptr(out), c.shape[0]), "cmh_philox4x64")
    return out
