"""ctypes binding of the C ABI in ``include/pf.h`` (argument marshalling only).

Every function of the header is exposed under its own name; :class:`Filter` and
:class:`Batch` wrap the handles for numpy / torch callers.  All filter arithmetic runs
in the sm_103a library ``_build/libpf_gb300.so``; there is no fallback: if the library
is missing or cannot be loaded, every call raises.
"""
from __future__ import annotations

import ctypes
import os
import threading

import numpy as np

from . import build as _build

__all__ = [
    "PF_OK", "PF_ERR_ARG", "PF_ERR_OOM", "PF_ERR_CUDA", "PF_ERR_TIMEOUT", "PF_ERR_STATE",
    "PF_ERR_ADMISSION", "PF_REF64", "PF_F32", "PF_F16", "PF_BF16", "PF_FLAG_DEBUG_ARRAYS",
    "PF_FLAG_ACCUM32", "PF_FLAG_TUNED", "PF_RESAMPLE_SYSTEMATIC", "PF_RESAMPLE_STRATIFIED", "PF_RESAMPLE_MULTINOMIAL",
    "PF_RESAMPLE_GUMBEL", "PF_RESAMPLE_METROPOLIS", "PF_RESAMPLE_REJECTION",
    "RESAMPLERS", "PfTuning", "pf_autotune", "pf_autotune_batch", "pf_tuning_lookup",
    "pf_tuning_store", "pf_tuning_clear", "autotune", "autotune_batch", "PfConfig", "PfStateHeader", "PfError", "lib", "library_path",
    "pf_status_string", "pf_create", "pf_step_frame", "pf_run_frames", "pf_estimate",
    "pf_estimates", "pf_frames_done", "pf_get_counters", "pf_batch_get_counters", "PfCounters", "pf_reset", "pf_destroy", "pf_get_state", "pf_set_state", "pf_get_debug",
    "pf_debug_philox", "pf_debug_wait_timeout", "pf_batch_create", "pf_batch_step", "pf_batch_estimates",
    "pf_batch_set_videos", "pf_batch_run", "pf_batch_reset", "pf_step_frame_noalloc",
    "pf_batch_destroy", "Filter", "Batch", "PRECISIONS", "EXPORTED",
    "PfServerConfig", "PfServerStats", "PfTraceEvent", "Server", "pf_server_now", "pf_server_create",
    "pf_server_open", "pf_server_submit", "pf_server_tick", "pf_server_poll", "pf_server_drain",
    "pf_server_result", "pf_server_frames_done", "pf_server_close", "pf_server_get_stats",
    "pf_server_destroy", "pf_server_stream_bytes", "pf_server_replay",
    "pf_shard_partition", "pf_shard_create", "pf_shard_stats", "pf_shard_resample", "pf_shard_step",
    "pf_shard_frames_done", "pf_shard_destroy", "Shard",
]

PF_OK, PF_ERR_ARG, PF_ERR_OOM, PF_ERR_CUDA, PF_ERR_TIMEOUT, PF_ERR_STATE, PF_ERR_ADMISSION = range(7)
PF_REF64, PF_F32, PF_F16, PF_BF16 = range(4)
PF_FLAG_DEBUG_ARRAYS = 0x1
PF_FLAG_ACCUM32 = 0x2
PF_FLAG_TUNED = 0x4
PRECISIONS = {"ref64": PF_REF64, "f64": PF_REF64, "f32": PF_F32, "f16": PF_F16, "bf16": PF_BF16}
PF_RESAMPLE_SYSTEMATIC, PF_RESAMPLE_STRATIFIED, PF_RESAMPLE_MULTINOMIAL, PF_RESAMPLE_GUMBEL, \
    PF_RESAMPLE_METROPOLIS, PF_RESAMPLE_REJECTION = range(6)
RESAMPLERS = {"systematic": PF_RESAMPLE_SYSTEMATIC, "stratified": PF_RESAMPLE_STRATIFIED,
              "multinomial": PF_RESAMPLE_MULTINOMIAL, "gumbel": PF_RESAMPLE_GUMBEL,
              "metropolis": PF_RESAMPLE_METROPOLIS, "rejection": PF_RESAMPLE_REJECTION}
_POS_DTYPE = {PF_REF64: np.float64, PF_F32: np.float32, PF_F16: np.float16, PF_BF16: None}


class PfConfig(ctypes.Structure):
    _fields_ = [
        ("width", ctypes.c_int32), ("height", ctypes.c_int32),
        ("num_particles", ctypes.c_int64),
        ("disk_radius", ctypes.c_int32), ("precision", ctypes.c_int32),
        ("bg_level", ctypes.c_double), ("fg_level", ctypes.c_double),
        ("init_x", ctypes.c_double), ("init_y", ctypes.c_double),
        ("sigma_x", ctypes.c_double), ("sigma_y", ctypes.c_double),
        ("drift_x", ctypes.c_double), ("drift_y", ctypes.c_double),
        ("seed", ctypes.c_uint64), ("tracker_id", ctypes.c_uint32), ("flags", ctypes.c_uint32),
        ("est_capacity", ctypes.c_int32), ("resampler", ctypes.c_int32),
        ("resampler_steps", ctypes.c_int32), ("reserved", ctypes.c_int32),
    ]


class PfCounters(ctypes.Structure):
    _fields_ = [("frames", ctypes.c_int64), ("step_launches", ctypes.c_int64), ("kernel_launches", ctypes.c_int64),
                ("graph_launches", ctypes.c_int64), ("host_frame_bytes", ctypes.c_int64),
                ("status", ctypes.c_int32), ("reserved", ctypes.c_int32)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_ if k != "reserved"}


class PfStateHeader(ctypes.Structure):
    _fields_ = [
        ("magic", ctypes.c_uint32), ("precision", ctypes.c_int32),
        ("num_particles", ctypes.c_int64), ("t", ctypes.c_int64),
        ("max_l", ctypes.c_double), ("sum_e", ctypes.c_double),
        ("anchor_x", ctypes.c_double), ("anchor_y", ctypes.c_double),
        ("next_anchor_x", ctypes.c_double), ("next_anchor_y", ctypes.c_double),
        ("est_x", ctypes.c_double), ("est_y", ctypes.c_double),
    ]


class PfTuning(ctypes.Structure):
    _fields_ = [("tile", ctypes.c_int32), ("window", ctypes.c_int32), ("ctas_per_sm", ctypes.c_int32),
                ("reserved", ctypes.c_int32)]

    def as_dict(self):
        return {"tile": self.tile, "window": self.window, "ctas_per_sm": self.ctas_per_sm}


class PfServerConfig(ctypes.Structure):
    _fields_ = [
        ("hbm_budget_bytes", ctypes.c_int64), ("capacity", ctypes.c_double), ("headroom", ctypes.c_double),
        ("max_streams", ctypes.c_int32), ("queue_depth", ctypes.c_int32),
        ("max_in_flight", ctypes.c_int32), ("reserved", ctypes.c_int32),
    ]


class PfServerStats(ctypes.Structure):
    _fields_ = [
        ("streams_open", ctypes.c_int64), ("streams_admitted", ctypes.c_int64), ("streams_rejected", ctypes.c_int64),
        ("frames_submitted", ctypes.c_int64), ("frames_rejected", ctypes.c_int64), ("frames_done", ctypes.c_int64),
        ("launches", ctypes.c_int64), ("particle_steps", ctypes.c_double),
        ("latency_p50_ms", ctypes.c_double), ("latency_p99_ms", ctypes.c_double), ("latency_max_ms", ctypes.c_double),
        ("first_launch_s", ctypes.c_double), ("last_done_s", ctypes.c_double),
        ("hbm_in_use", ctypes.c_int64), ("hbm_peak", ctypes.c_int64), ("demand", ctypes.c_double),
    ]

    def as_dict(self):
        return {f: getattr(self, f) for f, _ in self._fields_}


class PfTraceEvent(ctypes.Structure):
    _fields_ = [
        ("time_s", ctypes.c_double), ("kind", ctypes.c_int32), ("stream", ctypes.c_int32),
        ("frame", ctypes.c_void_p), ("pitch_bytes", ctypes.c_int64),
        ("cfg", ctypes.POINTER(PfConfig)), ("fps", ctypes.c_double),
    ]


class PfError(RuntimeError):
    def __init__(self, status: int, what: str = ""):
        self.status = status
        super().__init__("%s: %s (status %d)" % (what, _status_name(status), status))


_P = ctypes.c_void_p
_I32 = ctypes.c_int32
_I64 = ctypes.c_int64
_SIG = {
    "pf_status_string": (ctypes.c_char_p, [ctypes.c_int]),
    "pf_create": (ctypes.c_int, [ctypes.POINTER(PfConfig), _P, ctypes.POINTER(_P)]),
    "pf_step_frame": (ctypes.c_int, [_P, _P, _I64, _I32]),
    "pf_run_frames": (ctypes.c_int, [_P, _P, _I64, _I64, _I32, _I32]),
    "pf_estimate": (ctypes.c_int, [_P, _I64, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_double)]),
    "pf_estimates": (ctypes.c_int, [_P, _I64, _I32, _P, _P]),
    "pf_frames_done": (_I64, [_P]),
    "pf_get_counters": (ctypes.c_int, [_P, ctypes.POINTER(PfCounters)]),
    "pf_batch_get_counters": (ctypes.c_int, [_P, ctypes.POINTER(PfCounters)]),
    "pf_reset": (ctypes.c_int, [_P]),
    "pf_destroy": (ctypes.c_int, [_P]),
    "pf_get_state": (ctypes.c_int, [_P, _P, ctypes.POINTER(ctypes.c_size_t)]),
    "pf_set_state": (ctypes.c_int, [_P, _P, ctypes.c_size_t]),
    "pf_get_debug": (ctypes.c_int, [_P, _I32, _P, ctypes.c_size_t]),
    "pf_debug_philox": (ctypes.c_int, [_P, _I64, ctypes.c_uint64, _P]),
    "pf_debug_wait_timeout": (ctypes.c_int, [ctypes.c_uint32, ctypes.POINTER(ctypes.c_uint32)]),
    "pf_batch_create": (ctypes.c_int, [ctypes.POINTER(PfConfig), _I32, _P, ctypes.POINTER(_P)]),
    "pf_batch_step": (ctypes.c_int, [_P, _P, _P, _P]),
    "pf_batch_estimates": (ctypes.c_int, [_P, _I64, _P]),
    "pf_batch_set_videos": (ctypes.c_int, [_P, _P, _P, _P]),
    "pf_batch_run": (ctypes.c_int, [_P, _I32]),
    "pf_batch_reset": (ctypes.c_int, [_P]),
    "pf_step_frame_noalloc": (ctypes.c_int, [ctypes.POINTER(PfConfig), _P, _P, _P, _P, _P, _I64,
                                             _P, _P, _P, _P, _P]),
    "pf_batch_destroy": (ctypes.c_int, [_P]),
    "pf_autotune": (ctypes.c_int, [ctypes.POINTER(PfConfig), _I32, _P, _I64, _I64, _I32, ctypes.POINTER(PfTuning),
                                   ctypes.POINTER(ctypes.c_double)]),
    "pf_autotune_batch": (ctypes.c_int, [ctypes.POINTER(PfConfig), _I32, _P, _P, _P, _I32, ctypes.POINTER(PfTuning),
                                         ctypes.POINTER(ctypes.c_double)]),
    "pf_tuning_lookup": (ctypes.c_int, [ctypes.POINTER(PfConfig), ctypes.POINTER(PfTuning)]),
    "pf_tuning_store": (ctypes.c_int, [ctypes.POINTER(PfConfig), ctypes.POINTER(PfTuning)]),
    "pf_tuning_clear": (ctypes.c_int, []),
    "pf_server_now": (ctypes.c_double, []),
    "pf_server_create": (ctypes.c_int, [ctypes.POINTER(PfServerConfig), ctypes.POINTER(_P)]),
    "pf_server_open": (ctypes.c_int, [_P, ctypes.POINTER(PfConfig), ctypes.c_double, _I32, ctypes.POINTER(_I32)]),
    "pf_server_submit": (ctypes.c_int, [_P, _I32, _P, _I64, _I32, ctypes.c_double]),
    "pf_server_tick": (ctypes.c_int, [_P, ctypes.POINTER(_I32)]),
    "pf_server_poll": (ctypes.c_int, [_P, ctypes.POINTER(_I32)]),
    "pf_server_drain": (ctypes.c_int, [_P]),
    "pf_server_result": (ctypes.c_int, [_P, _I32, _I64, ctypes.POINTER(ctypes.c_double),
                                        ctypes.POINTER(ctypes.c_double)]),
    "pf_server_frames_done": (_I64, [_P, _I32]),
    "pf_server_close": (ctypes.c_int, [_P, _I32]),
    "pf_server_get_stats": (ctypes.c_int, [_P, ctypes.POINTER(PfServerStats)]),
    "pf_server_destroy": (ctypes.c_int, [_P]),
    "pf_server_stream_bytes": (ctypes.c_int, [ctypes.POINTER(PfConfig), _I32, _I32, ctypes.POINTER(_I64)]),
    "pf_server_replay": (ctypes.c_int, [_P, ctypes.POINTER(PfTraceEvent), _I64, _I32, _I32]),
    "pf_shard_partition": (ctypes.c_int, [_I64, _I32, _I32, ctypes.POINTER(_I64), ctypes.POINTER(_I64)]),
    "pf_shard_create": (ctypes.c_int, [ctypes.POINTER(PfConfig), _I32, _I32, _P, ctypes.POINTER(_P)]),
    "pf_shard_stats": (ctypes.c_int, [_P, ctypes.POINTER(ctypes.c_double)]),
    "pf_shard_resample": (ctypes.c_int, [_P, ctypes.POINTER(ctypes.c_double), _I32, _P, _P, _I64,
                                         ctypes.POINTER(_I64)]),
    "pf_shard_step": (ctypes.c_int, [_P, _P, _P, _P, _I64, _I32]),
    "pf_shard_frames_done": (_I64, [_P]),
    "pf_shard_destroy": (ctypes.c_int, [_P]),
}
EXPORTED = tuple(_SIG)

_lock = threading.Lock()
_lib = None


def _study_threads():
    """Threads per CTA of a thread-block study build selected by the environment
    (PF_STEP_THREADS, one of 128, 256, 512, 1024), or None for the library."""
    v = os.environ.get("PF_STEP_THREADS")
    return int(v) if v else None


def _checked() -> bool:
    """The checked build (PF_CHECKED=1 in the environment)."""
    return os.environ.get("PF_CHECKED", "") not in ("", "0")


def _naive() -> bool:
    """The naive-resampling study build (PF_NAIVE=1 in the environment)."""
    return os.environ.get("PF_NAIVE", "") not in ("", "0")


def library_path() -> str:
    return _build.lib_path(_study_threads(), _checked(), _naive())


def lib(build_if_missing: bool = False):
    """The loaded library.  Raises if it is missing (no CPU fallback exists)."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        path = library_path()
        if not os.path.exists(path):
            if build_if_missing:
                _build.build(threads=_study_threads(), checked=_checked(), naive=_naive())
            else:
                raise RuntimeError("the CUDA library %s is not built; run "
                                   "`python -c 'import __graft_entry__ as g; g.build()'`" % path)
        handle = ctypes.CDLL(path)
        for name, (res, args) in _SIG.items():
            fn = getattr(handle, name)
            fn.restype = res
            fn.argtypes = args
        _lib = handle
        return _lib


def _status_name(status: int) -> str:
    names = {0: "ok", 1: "invalid argument", 2: "out of memory", 3: "CUDA error",
             4: "device wait timed out", 5: "failed or wrong state", 6: "admission refused"}
    return names.get(status, "unknown")


def _check(status: int, what: str):
    if status != PF_OK:
        raise PfError(status, what)


# ------------------------------------------------------------------ raw C ABI, same names
def pf_status_string(s: int) -> str:
    return lib().pf_status_string(s).decode()


def pf_create(cfg: PfConfig, stream=None):
    h = _P()
    _check(lib().pf_create(ctypes.byref(cfg), _P(stream or 0), ctypes.byref(h)), "pf_create")
    return h


def pf_step_frame(h, frame_ptr: int, pitch: int, on_device: int):
    return lib().pf_step_frame(h, _P(frame_ptr), pitch, on_device)


def pf_run_frames(h, frames_ptr: int, pitch: int, stride: int, count: int, on_device: int):
    return lib().pf_run_frames(h, _P(frames_ptr), pitch, stride, count, on_device)


def pf_estimate(h, t: int):
    x = ctypes.c_double()
    y = ctypes.c_double()
    _check(lib().pf_estimate(h, t, ctypes.byref(x), ctypes.byref(y)), "pf_estimate")
    return x.value, y.value


def pf_estimates(h, first: int, count: int, with_stats: bool = False):
    xy = np.empty((count, 2), np.float64)
    ms = np.empty((count, 2), np.float64) if with_stats else None
    _check(lib().pf_estimates(h, first, count, xy.ctypes.data_as(_P),
                              ms.ctypes.data_as(_P) if ms is not None else None), "pf_estimates")
    return (xy, ms) if with_stats else xy


def pf_reset(h):
    return lib().pf_reset(h)


def pf_frames_done(h) -> int:
    return int(lib().pf_frames_done(h))


def pf_get_counters(h) -> dict:
    c = PfCounters()
    _check(lib().pf_get_counters(h, ctypes.byref(c)), "pf_get_counters")
    return c.as_dict()


def pf_batch_get_counters(h) -> dict:
    c = PfCounters()
    _check(lib().pf_batch_get_counters(h, ctypes.byref(c)), "pf_batch_get_counters")
    return c.as_dict()


def pf_destroy(h):
    return lib().pf_destroy(h)


def pf_get_state(h) -> bytes:
    n = ctypes.c_size_t(0)
    _check(lib().pf_get_state(h, None, ctypes.byref(n)), "pf_get_state")
    buf = ctypes.create_string_buffer(n.value)
    _check(lib().pf_get_state(h, buf, ctypes.byref(n)), "pf_get_state")
    return buf.raw


def pf_set_state(h, blob: bytes):
    _check(lib().pf_set_state(h, blob, len(blob)), "pf_set_state")


def pf_get_debug(h, which: int, n: int, dtype):
    out = np.empty(n, dtype)
    _check(lib().pf_get_debug(h, which, out.ctypes.data_as(_P), out.nbytes), "pf_get_debug")
    return out


def pf_debug_philox(ctrs, seed: int) -> np.ndarray:
    c = np.ascontiguousarray(np.asarray(ctrs, np.uint32).reshape(-1, 4))
    out = np.empty_like(c)
    _check(lib().pf_debug_philox(c.ctypes.data_as(_P), c.shape[0], seed & 0xFFFFFFFFFFFFFFFF,
                                 out.ctypes.data_as(_P)), "pf_debug_philox")
    return out


def pf_debug_wait_timeout(spin_limit: int):
    """(status code, status bits) of a bounded wait on a flag nobody sets."""
    bits = ctypes.c_uint32(0)
    rc = lib().pf_debug_wait_timeout(spin_limit, ctypes.byref(bits))
    return rc, bits.value


def pf_batch_create(cfgs, stream=None):
    arr = (PfConfig * len(cfgs))(*cfgs)
    h = _P()
    _check(lib().pf_batch_create(arr, len(cfgs), _P(stream or 0), ctypes.byref(h)), "pf_batch_create")
    return h


def pf_batch_step(h, frame_ptrs, pitches, active=None):
    n = len(frame_ptrs)
    fp = (ctypes.c_void_p * n)(*[p or 0 for p in frame_ptrs])
    pp = (ctypes.c_int64 * n)(*pitches)
    am = (ctypes.c_uint8 * n)(*active) if active is not None else None
    return lib().pf_batch_step(h, fp, pp, am)


def pf_batch_estimates(h, n: int, t: int) -> np.ndarray:
    xy = np.empty((n, 2), np.float64)
    _check(lib().pf_batch_estimates(h, t, xy.ctypes.data_as(_P)), "pf_batch_estimates")
    return xy


def pf_batch_set_videos(h, video_ptrs, pitches, strides):
    n = len(video_ptrs)
    vp = (ctypes.c_void_p * n)(*video_ptrs)
    pp = (ctypes.c_int64 * n)(*pitches)
    sp = (ctypes.c_int64 * n)(*strides)
    return lib().pf_batch_set_videos(h, vp, pp, sp)


def pf_batch_run(h, count: int):
    return lib().pf_batch_run(h, count)


def pf_batch_reset(h):
    return lib().pf_batch_reset(h)


def pf_step_frame_noalloc(cfg: PfConfig, state_in: "PfStateHeader", x_in: int, y_in: int, l_in: int,
                          frame: int, pitch: int, x_out: int, y_out: int, l_out: int, stream=None):
    """Allocation-free frame step on caller-owned device buffers (pointers as ints).
    Returns the new frame's state header."""
    out = PfStateHeader()
    _check(lib().pf_step_frame_noalloc(ctypes.byref(cfg), ctypes.byref(state_in), _P(x_in), _P(y_in),
                                       _P(l_in), _P(frame), pitch, _P(x_out), _P(y_out), _P(l_out),
                                       ctypes.byref(out), _P(_stream_ptr(stream))), "pf_step_frame_noalloc")
    return out


def pf_batch_destroy(h):
    return lib().pf_batch_destroy(h)


# ------------------------------------------------------------------ one tracker on several GPUs
def pf_shard_partition(n_global: int, nranks: int, rank: int):
    """(first, count) of rank `rank`'s particles."""
    first, count = _I64(0), _I64(0)
    _check(lib().pf_shard_partition(n_global, nranks, rank, ctypes.byref(first), ctypes.byref(count)),
           "pf_shard_partition")
    return first.value, count.value


def pf_shard_create(cfg: "PfConfig", rank: int, nranks: int, stream=None):
    h = _P()
    _check(lib().pf_shard_create(ctypes.byref(cfg), rank, nranks, _P(_stream_ptr(stream)), ctypes.byref(h)),
           "pf_shard_create")
    return h


def pf_shard_stats(h):
    out = (ctypes.c_double * 4)()
    _check(lib().pf_shard_stats(h, out), "pf_shard_stats")
    return tuple(out)


def pf_shard_resample(h, global4, last: bool, send_x: int, send_y: int, capacity: int):
    g = (ctypes.c_double * 4)(*global4)
    run = (_I64 * 2)()
    _check(lib().pf_shard_resample(h, g, 1 if last else 0, _P(send_x), _P(send_y), capacity, run),
           "pf_shard_resample")
    return run[0], run[1]


def pf_shard_step(h, recv_x: int, recv_y: int, frame: int, pitch: int):
    _check(lib().pf_shard_step(h, _P(recv_x), _P(recv_y), _P(frame), pitch, 1), "pf_shard_step")


def pf_shard_frames_done(h) -> int:
    return lib().pf_shard_frames_done(h)


def pf_shard_destroy(h):
    return lib().pf_shard_destroy(h)


class Shard:
    """Rank `rank`'s shard of one tracker sharded by particles (pf_shard_*).  Positions
    travel between ranks as torch tensors on the shard's device (float64 for REF64, float32
    for F32); `paper_2308_00763_gb300.sharded.ShardedTracker` drives the exchanges."""

    def __init__(self, width, height, num_particles, disk_radius, precision="ref64", *, rank=0, nranks=1,
                 stream=None, **kw):
        import torch
        self.cfg = make_config(width, height, num_particles, disk_radius, precision, **kw)
        self.rank, self.nranks = rank, nranks
        self.first, self.count = pf_shard_partition(num_particles, nranks, rank)
        self.stream = stream
        self.dtype = torch.float64 if self.cfg.precision == PF_REF64 else torch.float32
        self.h = pf_shard_create(self.cfg, rank, nranks, stream)

    def stats(self):
        return pf_shard_stats(self.h)

    def resample(self, global4, last, send_x, send_y):
        return pf_shard_resample(self.h, global4, last, send_x.data_ptr(), send_y.data_ptr(), send_x.numel())

    def step(self, frame, recv_x=None, recv_y=None):
        pf_shard_step(self.h, recv_x.data_ptr() if recv_x is not None else 0,
                      recv_y.data_ptr() if recv_y is not None else 0, frame.data_ptr(), frame.stride(0))

    def frames_done(self):
        return pf_shard_frames_done(self.h)

    def close(self):
        if getattr(self, "h", None):
            pf_shard_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


# ------------------------------------------------------------------ convenience wrappers
def pf_autotune(cfg: PfConfig, copies: int, video_ptr: int, pitch: int, stride: int, n_frames: int):
    """(tuning, us per frame of the fastest candidate)."""
    t = PfTuning()
    us = ctypes.c_double(0.0)
    _check(lib().pf_autotune(ctypes.byref(cfg), copies, _P(video_ptr), pitch, stride, n_frames, ctypes.byref(t),
                             ctypes.byref(us)), "pf_autotune")
    return t, us.value


def pf_autotune_batch(cfgs, video_ptrs, pitches, strides, n_frames: int):
    """(tuning, us per frame of the fastest shape) over a whole batch."""
    n = len(cfgs)
    arr = (PfConfig * n)(*cfgs)
    vp = (ctypes.c_void_p * n)(*video_ptrs)
    pp = (ctypes.c_int64 * n)(*pitches)
    sp = (ctypes.c_int64 * n)(*strides)
    t = PfTuning()
    us = ctypes.c_double(0.0)
    _check(lib().pf_autotune_batch(arr, n, vp, pp, sp, n_frames, ctypes.byref(t), ctypes.byref(us)),
           "pf_autotune_batch")
    return t, us.value


def autotune_batch(cfgs, videos, n_frames=None):
    """Tune a batch's shape on its resident videos (CUDA uint8 tensors (T_i, H_i, W_i));
    returns (tuning dict, microseconds per frame of the fastest shape)."""
    n_frames = n_frames or min(v.shape[0] for v in videos)
    t, us = pf_autotune_batch(cfgs, [v.data_ptr() for v in videos], [v.stride(1) for v in videos],
                              [v.stride(0) for v in videos], n_frames)
    return t.as_dict(), us


def pf_tuning_lookup(cfg: PfConfig):
    """The cached tuning of cfg's shape bucket, or None."""
    t = PfTuning()
    rc = lib().pf_tuning_lookup(ctypes.byref(cfg), ctypes.byref(t))
    if rc == PF_ERR_STATE:
        return None
    _check(rc, "pf_tuning_lookup")
    return t


def pf_tuning_store(cfg: PfConfig, tile: int, window: int, ctas_per_sm: int):
    t = PfTuning(tile=tile, window=window, ctas_per_sm=ctas_per_sm, reserved=0)
    _check(lib().pf_tuning_store(ctypes.byref(cfg), ctypes.byref(t)), "pf_tuning_store")


def pf_tuning_clear():
    _check(lib().pf_tuning_clear(), "pf_tuning_clear")


def autotune(cfg: PfConfig, video, copies: int = 1):
    """Tune cfg's shape bucket on a resident video (CUDA uint8 tensor (T, H, W)); returns
    (tuning dict, microseconds per frame of the fastest shape)."""
    t, us = pf_autotune(cfg, copies, video.data_ptr(), video.stride(1), video.stride(0), video.shape[0])
    return t.as_dict(), us


def pf_server_now() -> float:
    return float(lib().pf_server_now())


def pf_server_create(cfg: PfServerConfig):
    h = _P()
    _check(lib().pf_server_create(ctypes.byref(cfg), ctypes.byref(h)), "pf_server_create")
    return h


def pf_server_open(h, cfg: PfConfig, fps: float, host_frames: int):
    """(status, stream id)."""
    sid = _I32(-1)
    rc = lib().pf_server_open(h, ctypes.byref(cfg), float(fps), int(host_frames), ctypes.byref(sid))
    return rc, sid.value


def pf_server_submit(h, sid: int, frame_ptr: int, pitch: int, on_device: int, arrival: float = -1.0):
    return lib().pf_server_submit(h, sid, _P(frame_ptr), pitch, on_device, float(arrival))


def pf_server_tick(h) -> int:
    n = _I32(0)
    _check(lib().pf_server_tick(h, ctypes.byref(n)), "pf_server_tick")
    return n.value


def pf_server_poll(h) -> int:
    n = _I32(0)
    _check(lib().pf_server_poll(h, ctypes.byref(n)), "pf_server_poll")
    return n.value


def pf_server_drain(h):
    _check(lib().pf_server_drain(h), "pf_server_drain")


def pf_server_result(h, sid: int, index: int):
    x = ctypes.c_double()
    y = ctypes.c_double()
    rc = lib().pf_server_result(h, sid, index, ctypes.byref(x), ctypes.byref(y))
    return rc, (x.value, y.value)


def pf_server_frames_done(h, sid: int) -> int:
    return int(lib().pf_server_frames_done(h, sid))


def pf_server_close(h, sid: int):
    _check(lib().pf_server_close(h, sid), "pf_server_close")


def pf_server_get_stats(h) -> dict:
    st = PfServerStats()
    _check(lib().pf_server_get_stats(h, ctypes.byref(st)), "pf_server_get_stats")
    return st.as_dict()


def pf_server_destroy(h):
    return lib().pf_server_destroy(h)


def pf_server_stream_bytes(cfg: PfConfig, host_frames: int, queue_depth: int) -> int:
    b = _I64(0)
    _check(lib().pf_server_stream_bytes(ctypes.byref(cfg), host_frames, queue_depth, ctypes.byref(b)),
           "pf_server_stream_bytes")
    return b.value


def pf_server_replay(h, events, n_streams: int, realtime: bool):
    arr = (PfTraceEvent * len(events))(*events)
    _check(lib().pf_server_replay(h, arr, len(events), n_streams, 1 if realtime else 0), "pf_server_replay")


def make_config(width, height, num_particles, disk_radius, precision="f32", *, init=(0.0, 0.0),
                sigma=(1.0, 1.0), drift=(0.0, 0.0), seed=1, tracker_id=0, bg=100.0, fg=228.0,
                flags=0, est_capacity=0, resampler="systematic", resampler_steps=0) -> PfConfig:
    prec = PRECISIONS[precision] if isinstance(precision, str) else int(precision)
    rs = RESAMPLERS[resampler] if isinstance(resampler, str) else int(resampler)
    return PfConfig(width=width, height=height, num_particles=num_particles, disk_radius=disk_radius,
                    precision=prec, bg_level=bg, fg_level=fg, init_x=init[0], init_y=init[1],
                    sigma_x=sigma[0], sigma_y=sigma[1], drift_x=drift[0], drift_y=drift[1],
                    seed=seed & 0xFFFFFFFFFFFFFFFF, tracker_id=tracker_id, flags=flags,
                    est_capacity=est_capacity, resampler=rs, resampler_steps=int(resampler_steps), reserved=0)


def _torch():
    import torch
    return torch


def _stream_ptr(stream):
    if stream is None:
        torch = _torch()
        if torch.cuda.is_available():
            return torch.cuda.current_stream().cuda_stream
        return 0
    return getattr(stream, "cuda_stream", stream)


def _frame_ptr(frame):
    """(pointer, pitch, on_device, keepalive) of a frame: torch CUDA tensor or host array."""
    if hasattr(frame, "data_ptr") and hasattr(frame, "is_cuda"):
        if frame.dtype.itemsize != 1 or frame.dim() < 2 or frame.stride(-1) != 1:
            raise ValueError("frame must be a uint8 tensor with unit column stride")
        if frame.is_cuda:
            return frame.data_ptr(), frame.stride(-2), 1, frame
        arr = frame.numpy()
    else:
        arr = frame
    arr = np.ascontiguousarray(arr, dtype=np.uint8)
    return arr.ctypes.data, arr.strides[-2], 0, arr


class Filter:
    """One tracker (pf_create / pf_step_frame / pf_estimate / pf_destroy)."""

    def __init__(self, width, height, num_particles, disk_radius, precision="f32", *, stream=None, **kw):
        self.cfg = make_config(width, height, num_particles, disk_radius, precision, **kw)
        self.precision = self.cfg.precision
        self.N = int(num_particles)
        self.h = pf_create(self.cfg, _stream_ptr(stream))

    # -- stepping
    def step(self, frame):
        ptr, pitch, dev, keep = _frame_ptr(frame)
        _check(pf_step_frame(self.h, ptr, pitch, dev), "pf_step_frame")
        return keep

    def run(self, frames):
        """Step every frame of a (T, H, W) uint8 array/tensor (host or CUDA)."""
        if hasattr(frames, "is_cuda") and frames.is_cuda:
            if frames.stride(-1) != 1:
                raise ValueError("frames must have unit column stride")
            _check(pf_run_frames(self.h, frames.data_ptr(), frames.stride(-2), frames.stride(0),
                                 frames.shape[0], 1), "pf_run_frames")
            return frames
        arr = np.ascontiguousarray(frames.numpy() if hasattr(frames, "numpy") else frames, np.uint8)
        _check(pf_run_frames(self.h, arr.ctypes.data, arr.strides[1], arr.strides[0], arr.shape[0], 0),
               "pf_run_frames")
        return arr

    # -- results
    def estimate(self, t):
        return pf_estimate(self.h, t)

    def estimates(self, first=0, count=None, with_stats=False):
        if count is None:
            count = self.frames_done - first
        return pf_estimates(self.h, first, count, with_stats)

    def reset(self):
        _check(pf_reset(self.h), "pf_reset")

    @property
    def frames_done(self):
        return pf_frames_done(self.h)

    def counters(self) -> dict:
        return pf_get_counters(self.h)

    # -- checkpoint
    def _pos_dtype(self):
        return _POS_DTYPE[self.precision]

    def get_state(self) -> dict:
        blob = pf_get_state(self.h)
        hdr = PfStateHeader.from_buffer_copy(blob[:ctypes.sizeof(PfStateHeader)])
        body = np.frombuffer(blob, dtype=np.uint8, offset=ctypes.sizeof(PfStateHeader))
        esz = {PF_REF64: 8, PF_F32: 4, PF_F16: 2, PF_BF16: 2}[self.precision]
        raw = body.reshape(3, self.N * esz)
        out = {k: getattr(hdr, k) for k, _ in PfStateHeader._fields_}
        for i, name in enumerate(("x", "y", "L")):
            out[name] = _decode(raw[i], self.precision)
        return out

    def set_state(self, st: dict):
        hdr = PfStateHeader(magic=0x31534650, precision=self.precision, num_particles=self.N)
        for k, _ in PfStateHeader._fields_:
            if k not in ("magic", "precision", "num_particles") and k in st:
                setattr(hdr, k, st[k])
        body = b"".join(_encode(np.asarray(st[n], np.float64), self.precision) for n in ("x", "y", "L"))
        pf_set_state(self.h, bytes(hdr) + body)

    def debug(self, which):
        if which == 0:
            return pf_get_debug(self.h, 0, self.N, np.int32)
        if which == 2:   # per-tile windows (x0, y0, width, height): rows of the tiles the step used
            w = np.full(4 * (-(-self.N // 1024)), -1, np.int32)
            _check(lib().pf_get_debug(self.h, 2, w.ctypes.data_as(_P), w.nbytes), "pf_get_debug")
            w = w.reshape(-1, 4)
            return w[w[:, 2] >= 0]
        return pf_get_debug(self.h, 1, self.N, np.float64 if self.precision == PF_REF64 else np.float32)

    def close(self):
        if getattr(self, "h", None):
            pf_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()


class Batch:
    """Many trackers stepped by one launch per frame (pf_batch_*)."""

    def __init__(self, cfgs, *, stream=None):
        self.cfgs = list(cfgs)
        self.n = len(self.cfgs)
        self.h = pf_batch_create(self.cfgs, _stream_ptr(stream))

    def step(self, frames, active=None):
        """frames: list of CUDA uint8 tensors (H_i, W_i) (None where inactive)."""
        ptrs = [f.data_ptr() if f is not None else 0 for f in frames]
        pitches = [f.stride(0) if f is not None else 0 for f in frames]
        _check(pf_batch_step(self.h, ptrs, pitches, active), "pf_batch_step")

    def set_videos(self, videos):
        """videos: list of CUDA uint8 tensors (T_i, H_i, W_i), resident for pf_batch_run."""
        self._videos = list(videos)
        _check(pf_batch_set_videos(self.h, [v.data_ptr() for v in videos], [v.stride(1) for v in videos],
                                   [v.stride(0) for v in videos]), "pf_batch_set_videos")

    def run(self, count):
        _check(pf_batch_run(self.h, count), "pf_batch_run")

    def reset(self):
        _check(pf_batch_reset(self.h), "pf_batch_reset")

    def estimates(self, t):
        return pf_batch_estimates(self.h, self.n, t)

    def counters(self) -> dict:
        return pf_batch_get_counters(self.h)

    def close(self):
        if getattr(self, "h", None):
            pf_batch_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Server:
    """Continuous batching over camera streams (pf_server_*)."""

    def __init__(self, hbm_budget_bytes, *, capacity=0.0, headroom=1.0, max_streams=64, queue_depth=4,
                 max_in_flight=2):
        self.cfg = PfServerConfig(hbm_budget_bytes=int(hbm_budget_bytes), capacity=float(capacity),
                                  headroom=float(headroom), max_streams=int(max_streams),
                                  queue_depth=int(queue_depth), max_in_flight=int(max_in_flight), reserved=0)
        self.h = pf_server_create(self.cfg)
        self._keep = {}

    def open(self, cfg: PfConfig, fps=30.0, host_frames=False):
        """Stream id, or None when admission refuses the stream."""
        rc, sid = pf_server_open(self.h, cfg, fps, 1 if host_frames else 0)
        if rc == PF_ERR_ADMISSION:
            return None
        _check(rc, "pf_server_open")
        return sid

    def submit(self, sid, frame, arrival=-1.0):
        """Queue a frame (CUDA tensor read in place, or host array copied); False when the
        stream's queue is full.  A CUDA frame is kept alive here until it completes."""
        ptr, pitch, on_dev, keep = _frame_ptr(frame)
        rc = pf_server_submit(self.h, sid, ptr, pitch, on_dev, arrival)
        if rc == PF_ERR_ADMISSION:
            return False
        _check(rc, "pf_server_submit")
        q = self._keep.setdefault(sid, [0, []])     # [frames submitted, [(index, tensor)]]
        if on_dev:
            q[1].append((q[0], keep))
        q[0] += 1
        done = pf_server_frames_done(self.h, sid)
        q[1] = [(i, t) for i, t in q[1] if i >= done]
        return True

    def tick(self):
        return pf_server_tick(self.h)

    def poll(self):
        return pf_server_poll(self.h)

    def drain(self):
        pf_server_drain(self.h)

    def result(self, sid, index):
        rc, xy = pf_server_result(self.h, sid, index)
        _check(rc, "pf_server_result")
        return xy

    def frames_done(self, sid):
        return pf_server_frames_done(self.h, sid)

    def close_stream(self, sid):
        pf_server_close(self.h, sid)
        self._keep.pop(sid, None)

    def stats(self):
        return pf_server_get_stats(self.h)

    def replay(self, events, n_streams, realtime=True):
        pf_server_replay(self.h, events, n_streams, realtime)

    def close(self):
        if getattr(self, "h", None):
            pf_server_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def _bf16_to_f64(u16: np.ndarray) -> np.ndarray:
    return (u16.astype(np.uint32) << 16).view(np.float32).astype(np.float64)


def _f64_to_bf16(x: np.ndarray) -> np.ndarray:
    f = np.asarray(x, np.float32)
    b = f.view(np.uint32).astype(np.uint64)
    # round to nearest even on the dropped 16 bits
    b = (b + 0x7FFF + ((b >> 16) & 1)) >> 16
    return b.astype(np.uint16)


def _decode(raw: np.ndarray, prec: int) -> np.ndarray:
    if prec == PF_REF64:
        return raw.view(np.float64).copy()
    if prec == PF_F32:
        return raw.view(np.float32).astype(np.float64)
    if prec == PF_F16:
        return raw.view(np.float16).astype(np.float64)
    return _bf16_to_f64(raw.view(np.uint16))


def _encode(x: np.ndarray, prec: int) -> bytes:
    if prec == PF_REF64:
        return np.ascontiguousarray(x, np.float64).tobytes()
    if prec == PF_F32:
        return np.ascontiguousarray(x, np.float32).tobytes()
    if prec == PF_F16:
        return np.ascontiguousarray(x, np.float16).tobytes()
    return _f64_to_bf16(x).tobytes()
