"""CPU FP64 oracle of the per-frame SIR particle-filter step (test infrastructure only).

The arithmetic lives in ``pf_oracle.c`` (plain C, FP64, no FMA contraction); this
module compiles it with gcc into ``oracle/_build/liborc.so`` and exposes numpy-level
wrappers.  Only the tests, ``__graft_entry__.smoke()`` and ``bench.py``'s CPU-baseline
leg import it.  It shares no code with the CUDA library.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading
from dataclasses import dataclass, field

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "pf_oracle.c")
_LIB = os.path.join(_HERE, "_build", "liborc.so")
_lock = threading.Lock()
_lib = None

_I64 = ctypes.c_int64
_U32 = ctypes.c_uint32
_U64 = ctypes.c_uint64
_D = ctypes.c_double
_P = ctypes.c_void_p


def build(force: bool = False) -> str:
    """Compile the oracle (plain C) if the library is missing or older than its source."""
    os.makedirs(os.path.dirname(_LIB), exist_ok=True)
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + ".tmp%d" % os.getpid()
        cmd = ["gcc", "-std=c11", "-O2", "-ffp-contract=off", "-fno-fast-math", "-fPIC",
               "-shared", "-o", tmp, _SRC, "-lm", "-lpthread"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        lib = ctypes.CDLL(build())
        sig = {
            "orc_philox_batch": (None, [_I64, _P, _U64, _P]),
            "orc_uniform_batch": (None, [_I64, _P, _P]),
            "orc_box_muller_batch": (None, [_I64, _P, _P, _P, _P]),
            "orc_round_pixel_batch": (None, [_I64, _P, _P]),
            "orc_resample_u0": (_D, [_U64, _U32, _U32]),
            "orc_normal2_batch": (None, [_U64, _U32, _U32, _I64, _I64, _P, _P]),
            "orc_disk_count": (ctypes.c_int, [ctypes.c_int]),
            "orc_likelihood_at": (_D, [_P, ctypes.c_int, ctypes.c_int, _I64, ctypes.c_int,
                                       _D, _D, _I64, _I64]),
            "orc_disk_sum": (_I64, [_P, ctypes.c_int, ctypes.c_int, _I64, ctypes.c_int,
                                    _I64, _I64]),
            "orc_propagate": (None, [_I64, _U32, _U64, _U32, _P, _P, _P, _D, _D, _D, _D,
                                     _D, _D, _P, _P, ctypes.c_int]),
            "orc_likelihood_all": (None, [_I64, _P, _P, _P, ctypes.c_int, ctypes.c_int, _I64,
                                          ctypes.c_int, _D, _D, _P, ctypes.c_int]),
            "orc_weights": (_D, [_I64, _P, _P]),
            "orc_normalise": (_D, [_I64, _P, _P, _P, _P, _P]),
            "orc_cdf": (None, [_I64, _P, _D, _P]),
            "orc_resample_f64": (None, [_I64, _P, _D, _P]),
            "orc_resample_f32": (None, [_I64, _P, ctypes.c_float, _P]),
            "orc_resample_div_f64": (None, [_I64, _P, _D, _P]),
            "orc_resample_div_f32": (None, [_I64, _P, ctypes.c_float, _P]),
            "orc_stratified_offsets": (None, [_U64, _U32, _U32, _I64, _P]),
            "orc_resample_strat_f64": (None, [_I64, _P, _P, _P]),
            "orc_resample_strat_f32": (None, [_I64, _P, _P, _P]),
            "orc_resample_multi_f64": (None, [_I64, _P, _P, _P]),
            "orc_resample_multi_f32": (None, [_I64, _P, _P, _P]),
            "orc_gumbel_f64": (None, [_U64, _U32, _U32, _I64, _P, _P]),
            "orc_gumbel_f32": (None, [_U64, _U32, _U32, _I64, _P, _P]),
            "orc_metropolis_f64": (None, [_U64, _U32, _U32, _I64, _P, ctypes.c_int, _P]),
            "orc_metropolis_f32": (None, [_U64, _U32, _U32, _I64, _P, ctypes.c_int, _P]),
            "orc_rejection_f64": (None, [_U64, _U32, _U32, _I64, _P, _D, ctypes.c_int, _P]),
            "orc_rejection_f32": (None, [_U64, _U32, _U32, _I64, _P, ctypes.c_float, ctypes.c_int, _P]),
            "orc_run": (ctypes.c_int, [_P, _I64, ctypes.c_int, ctypes.c_int, ctypes.c_int, _I64,
                                       _I64, ctypes.c_int, _D, _D, _D, _D, _D, _D, _D, _D,
                                       _U64, _U32, ctypes.c_int, ctypes.c_int, ctypes.c_int, _P, _P, _P]),
        }
        for name, (res, args) in sig.items():
            fn = getattr(lib, name)
            fn.restype = res
            fn.argtypes = args
        _lib = lib
        return lib


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


# --------------------------------------------------------------------------- RNG
def philox(ctrs, seed: int) -> np.ndarray:
    """Philox4x32-10 of each counter row (n, 4) under the 64-bit key ``seed``."""
    c = np.ascontiguousarray(np.asarray(ctrs, dtype=np.uint32).reshape(-1, 4))
    out = np.empty_like(c)
    _load().orc_philox_batch(c.shape[0], _ptr(c), seed & 0xFFFFFFFFFFFFFFFF, _ptr(out))
    return out


def uniform(words) -> np.ndarray:
    w = np.ascontiguousarray(np.asarray(words, dtype=np.uint32).ravel())
    u = np.empty(w.shape, dtype=np.float64)
    _load().orc_uniform_batch(w.size, _ptr(w), _ptr(u))
    return u


def box_muller(ua, ub):
    a = np.ascontiguousarray(np.asarray(ua, dtype=np.float64).ravel())
    b = np.ascontiguousarray(np.asarray(ub, dtype=np.float64).ravel())
    nx = np.empty_like(a)
    ny = np.empty_like(a)
    _load().orc_box_muller_batch(a.size, _ptr(a), _ptr(b), _ptr(nx), _ptr(ny))
    return nx, ny


def normals(seed: int, t: int, n: int, tracker: int = 0, start: int = 0):
    """The propagation draws (n_x, n_y) of particles start..start+n-1 at frame t."""
    nx = np.empty(n, np.float64)
    ny = np.empty(n, np.float64)
    _load().orc_normal2_batch(seed & 0xFFFFFFFFFFFFFFFF, t, tracker, start, n, _ptr(nx), _ptr(ny))
    return nx, ny


def resample_u0(seed: int, t: int, tracker: int = 0) -> float:
    return float(_load().orc_resample_u0(seed & 0xFFFFFFFFFFFFFFFF, t, tracker))


# --------------------------------------------------------------------------- template / pixels
def disk_count(r: int) -> int:
    return int(_load().orc_disk_count(r))


def round_pixel(v) -> np.ndarray:
    a = np.ascontiguousarray(np.asarray(v, dtype=np.float64).ravel())
    p = np.empty(a.shape, dtype=np.int64)
    _load().orc_round_pixel_batch(a.size, _ptr(a), _ptr(p))
    return p


def _frame_args(frame: np.ndarray):
    f = np.ascontiguousarray(frame, dtype=np.uint8)
    H, W = f.shape
    return f, W, H, W


def likelihood_at(frame: np.ndarray, r: int, px: int, py: int, bg=100.0, fg=228.0) -> float:
    f, W, H, pitch = _frame_args(frame)
    return float(_load().orc_likelihood_at(_ptr(f), W, H, pitch, r, bg, fg, px, py))


def disk_sum(frame: np.ndarray, r: int, px: int, py: int) -> int:
    f, W, H, pitch = _frame_args(frame)
    return int(_load().orc_disk_sum(_ptr(f), W, H, pitch, r, px, py))


# --------------------------------------------------------------------------- phases
def propagate(N, t, seed, xa, ya, anc, init=(0.0, 0.0), drift=(0.0, 0.0), sigma=(1.0, 1.0),
              tracker=0, nthreads=1):
    x = np.empty(N, np.float64)
    y = np.empty(N, np.float64)
    if anc is None:
        pa = pxa = pya = None
    else:
        xa = np.ascontiguousarray(xa, np.float64)
        ya = np.ascontiguousarray(ya, np.float64)
        anc = np.ascontiguousarray(anc, np.int64)
        pa, pxa, pya = _ptr(anc), _ptr(xa), _ptr(ya)
    _load().orc_propagate(N, t, seed & 0xFFFFFFFFFFFFFFFF, tracker, pxa, pya, pa,
                          init[0], init[1], drift[0], drift[1], sigma[0], sigma[1],
                          _ptr(x), _ptr(y), nthreads)
    return x, y


def likelihood_all(x, y, frame, r, bg=100.0, fg=228.0, nthreads=1):
    x = np.ascontiguousarray(x, np.float64)
    y = np.ascontiguousarray(y, np.float64)
    f, W, H, pitch = _frame_args(frame)
    L = np.empty(x.size, np.float64)
    _load().orc_likelihood_all(x.size, _ptr(x), _ptr(y), _ptr(f), W, H, pitch, r, bg, fg,
                               _ptr(L), nthreads)
    return L


# --------------------------------------------------------------------------- Eq. 4 in half precision
def round_half(v) -> np.ndarray:
    """binary16 round-to-nearest-even of float64 values (one rounding: numpy converts
    float64 to float16 directly)."""
    return np.asarray(v, np.float64).astype(np.float16).astype(np.float64)


def round_bf16(v) -> np.ndarray:
    """bfloat16 round-to-nearest-even of float64 values: 8 significant bits, the exponent
    range of binary32 (values here are far from its limits)."""
    v = np.asarray(v, np.float64)
    m, e = np.frexp(v)                       # v = m 2^e, 0.5 <= |m| < 1
    return np.ldexp(np.rint(np.ldexp(m, 8)), e - 8)


def round_f32(v) -> np.ndarray:
    return np.asarray(v, np.float64).astype(np.float32).astype(np.float64)


def half_terms(r: int, kind: str, bg=100.0, fg=228.0) -> np.ndarray:
    """The per-pixel term of Eq. 4 for every intensity 0..255 as the half filters form it
    (reading C10): kappa = 1 / sqrt(50 |D|) rounded to binary32 and then to the lane type;
    a = (I - bg) kappa and b = (I - fg) kappa, each one rounded product; term = a a - b b
    with b b rounded and a a - b b one fused (singly rounded) operation.  I - bg and
    I - fg are exact in both lane types.  kind: "f16" / "f16acc32" (binary16 lanes) or
    "bf16"."""
    rnd = round_bf16 if kind == "bf16" else round_half
    D = disk_count(r)
    kap = rnd(round_f32(1.0 / np.sqrt(50.0 * D)))
    I = np.arange(256, dtype=np.float64)
    a = rnd((I - bg) * kap)
    b = rnd((I - fg) * kap)
    return rnd(a * a - rnd(b * b))


def template_offsets(r: int):
    """(dx, dy) of the template D in row-major order: dy = -r..r, dx ascending (reading C2)."""
    out = []
    for dy in range(-r, r + 1):
        for dx in range(-r, r + 1):
            if dx * dx + dy * dy <= r * r:
                out.append((dx, dy))
    return np.array(out, dtype=np.int64).reshape(-1, 2)


def likelihood_half(x, y, frame, r: int, kind: str = "f16", bg=100.0, fg=228.0) -> np.ndarray:
    """L of Eq. 3 in the scaled per-pixel form of Eq. 4 evaluated in half precision as the
    half filters do (reading C10): the terms of half_terms at the template pixels of each
    particle's pixel (reading C3; template pixels clamped to the frame, reading C4); each
    template row (dy = -r..r) summed left to right (dx ascending), then the row sums added
    top to bottom -- in binary16 with one rounding per addition ("f16", the paper's half
    accumulation), or in binary32 and then rounded to the lane type ("f16acc32", "bf16").
    Every operation is emulated in FP64 with one correct rounding, so the result is the
    exact value of that sequence of operations."""
    f = np.ascontiguousarray(frame, dtype=np.uint8)
    H, W = f.shape
    px = round_pixel(x)
    py = round_pixel(y)
    tm = half_terms(r, kind, bg, fg)
    acc = np.zeros(px.size, np.float64)
    step = round_half if kind == "f16" else round_f32
    offs = template_offsets(r)
    for dy in range(-r, r + 1):
        row = np.zeros(px.size, np.float64)
        for dx in offs[offs[:, 1] == dy, 0]:
            I = f[np.clip(py + dy, 0, H - 1), np.clip(px + dx, 0, W - 1)]
            row = step(row + tm[I])
        acc = step(acc + row)
    return acc if kind == "f16" else (round_bf16(acc) if kind == "bf16" else round_half(acc))


def weights(L):
    L = np.ascontiguousarray(L, np.float64)
    e = np.empty_like(L)
    M = _load().orc_weights(L.size, _ptr(L), _ptr(e))
    return float(M), e


def normalise(e, x, y):
    e = np.ascontiguousarray(e, np.float64)
    x = np.ascontiguousarray(x, np.float64)
    y = np.ascontiguousarray(y, np.float64)
    xh = ctypes.c_double()
    yh = ctypes.c_double()
    S = _load().orc_normalise(e.size, _ptr(e), _ptr(x), _ptr(y), ctypes.byref(xh), ctypes.byref(yh))
    return float(S), float(xh.value), float(yh.value)


def cdf(e, S):
    e = np.ascontiguousarray(e, np.float64)
    C = np.empty_like(e)
    _load().orc_cdf(e.size, _ptr(e), float(S), _ptr(C))
    return C


def resample(C, u0, precision: str = "f64", divide: bool = False):
    """Systematic-resampling ancestors of CDF ``C`` with offset ``u0``, the decision taken
    in FP64 (``precision='f64'``) or FP32 (``'f32'``; C and u0 are rounded to FP32).  The
    stratum points are ``(j + u0) * (1/N)``, or ``(j + u0) / N`` with ``divide``."""
    L = _load()
    if precision == "f64":
        Cc = np.ascontiguousarray(C, np.float64)
        a = np.empty(Cc.size, np.int64)
        (L.orc_resample_div_f64 if divide else L.orc_resample_f64)(Cc.size, _ptr(Cc), float(u0), _ptr(a))
    elif precision == "f32":
        Cc = np.ascontiguousarray(C, np.float32)
        a = np.empty(Cc.size, np.int64)
        (L.orc_resample_div_f32 if divide else L.orc_resample_f32)(Cc.size, _ptr(Cc), float(np.float32(u0)), _ptr(a))
    else:
        raise ValueError(precision)
    return a


def stratified_offsets(seed: int, t: int, N: int, tracker: int = 0) -> np.ndarray:
    """Offsets v_j (j < N) of frame t's strata for stratified resampling."""
    v = np.empty(int(N), np.float64)
    _load().orc_stratified_offsets(seed & 0xFFFFFFFFFFFFFFFF, t, tracker, int(N), _ptr(v))
    return v


def resample_stratified(C, v, precision: str = "f64"):
    """Stratified-resampling ancestors of CDF ``C`` with offsets ``v`` (u_j = (j + v_j)/N),
    the decision taken in FP64 or FP32 (C and v rounded to FP32)."""
    if precision == "f64":
        Cc = np.ascontiguousarray(C, np.float64)
        vv = np.ascontiguousarray(v, np.float64)
        fn = _load().orc_resample_strat_f64
    elif precision == "f32":
        Cc = np.ascontiguousarray(C, np.float32)
        vv = np.ascontiguousarray(v, np.float32)
        fn = _load().orc_resample_strat_f32
    else:
        raise ValueError(precision)
    if vv.size != Cc.size:
        raise ValueError("one offset per stratum")
    a = np.empty(Cc.size, np.int64)
    fn(Cc.size, _ptr(Cc), _ptr(vv), _ptr(a))
    return a


def resample_multinomial(C, v, precision: str = "f64"):
    """Multinomial-resampling ancestors of CDF ``C`` from independent uniforms ``v``
    (a_j = min{k : C_k >= v_j}), decided in FP64 or FP32 (C and v rounded to FP32)."""
    if precision == "f64":
        Cc = np.ascontiguousarray(C, np.float64)
        vv = np.ascontiguousarray(v, np.float64)
        fn = _load().orc_resample_multi_f64
    elif precision == "f32":
        Cc = np.ascontiguousarray(C, np.float32)
        vv = np.ascontiguousarray(v, np.float32)
        fn = _load().orc_resample_multi_f32
    else:
        raise ValueError(precision)
    if vv.size != Cc.size:
        raise ValueError("one draw per offspring")
    a = np.empty(Cc.size, np.int64)
    fn(Cc.size, _ptr(Cc), _ptr(vv), _ptr(a))
    return a


def resample_gumbel(L, seed: int, t: int, tracker: int = 0, precision: str = "f64"):
    """Gumbel-max ancestors of frame t's unnormalised log weights ``L``:
    a_j = argmax_k (L_k - ln(-ln u_jk)), ties to the smallest k, decided in FP64 or FP32
    (L rounded to FP32, the variates from logf).  N^2 draws."""
    if precision == "f64":
        Lc = np.ascontiguousarray(L, np.float64)
        fn = _load().orc_gumbel_f64
    elif precision == "f32":
        Lc = np.ascontiguousarray(L, np.float32)
        fn = _load().orc_gumbel_f32
    else:
        raise ValueError(precision)
    a = np.empty(Lc.size, np.int64)
    fn(seed & 0xFFFFFFFFFFFFFFFF, t, tracker, Lc.size, _ptr(Lc), _ptr(a))
    return a


def gumbel_variates(seed: int, t: int, j: int, N: int, tracker: int = 0) -> np.ndarray:
    """The variates g_jk = -ln(-ln u_jk), k < N, of offspring j at frame t (FP64)."""
    k = np.arange(N)
    ctr = np.stack([k // 4, np.full(N, t), np.full(N, 4 + 256 * j), np.full(N, tracker)], axis=1)
    w = philox(ctr, seed)[k, k % 4]
    return -np.log(-np.log(uniform(w)))


METROPOLIS_STEPS = 64     # default chain length B


def resample_metropolis(L, B: int, seed: int, t: int, tracker: int = 0, precision: str = "f64"):
    """Metropolis ancestors of frame t's log weights ``L``: offspring j runs a B-step chain
    from k = j, proposals k' = floor(w N / 2^32) accepted when ln u <= L_k' - L_k, decided
    in FP64 or FP32 (L rounded to FP32, ln u from logf)."""
    if precision == "f64":
        Lc = np.ascontiguousarray(L, np.float64)
        fn = _load().orc_metropolis_f64
    elif precision == "f32":
        Lc = np.ascontiguousarray(L, np.float32)
        fn = _load().orc_metropolis_f32
    else:
        raise ValueError(precision)
    a = np.empty(Lc.size, np.int64)
    fn(seed & 0xFFFFFFFFFFFFFFFF, t, tracker, Lc.size, _ptr(Lc), int(B), _ptr(a))
    return a


def metropolis_chain(L, B: int, seed: int, t: int, j: int, tracker: int = 0):
    """Offspring j's chain in FP64, step by step: (states after each step, the margin
    |ln u - (L_k' - L_k)| of each acceptance test)."""
    L = np.asarray(L, np.float64)
    N = L.size
    k, states, margins = j, [], []
    for b in range(B):
        w = philox([[b // 2, t, 5 + 256 * j, tracker]], seed)[0]
        kp = (int(w[2 * (b % 2)]) * N) >> 32
        lu = float(np.log(uniform([w[2 * (b % 2) + 1]])[0]))
        d = L[kp] - L[k]
        margins.append(abs(lu - d))
        if lu <= d:
            k = kp
        states.append(k)
    return states, margins


REJECTION_TRIES = 4096    # tries per offspring before the last candidate is kept


def resample_rejection(L, M, seed: int, t: int, tracker: int = 0, precision: str = "f64",
                       tries: int = REJECTION_TRIES):
    """Rejection-resampling ancestors of frame t's log weights ``L`` with bound ``M``
    (max L): candidates j, then proposals k' = floor(w N / 2^32), the first passing
    ln u <= L_k - M kept (the last after ``tries``), decided in FP64 or FP32."""
    if precision == "f64":
        Lc = np.ascontiguousarray(L, np.float64)
        fn, Mc = _load().orc_rejection_f64, float(M)
    elif precision == "f32":
        Lc = np.ascontiguousarray(L, np.float32)
        fn, Mc = _load().orc_rejection_f32, float(np.float32(M))
    else:
        raise ValueError(precision)
    a = np.empty(Lc.size, np.int64)
    fn(seed & 0xFFFFFFFFFFFFFFFF, t, tracker, Lc.size, _ptr(Lc), Mc, int(tries), _ptr(a))
    return a


def rejection_trace(L, M, seed: int, t: int, j: int, tracker: int = 0, tries: int = REJECTION_TRIES):
    """Offspring j's tries in FP64 until acceptance: (candidates, margins |ln u - (L_k - M)|)."""
    L = np.asarray(L, np.float64)
    N = L.size
    k, cands, margins = j, [], []
    for i in range(tries):
        w = philox([[i // 2, t, 6 + 256 * j, tracker]], seed)[0]
        if i > 0:
            k = (int(w[2 * (i % 2)]) * N) >> 32
        lu = float(np.log(uniform([w[2 * (i % 2) + 1]])[0]))
        d = L[k] - M
        cands.append(k)
        margins.append(abs(lu - d))
        if lu <= d:
            break
    return cands, margins


RESAMPLERS = {"systematic": 0, "stratified": 1, "multinomial": 2, "gumbel": 3, "metropolis": 4, "rejection": 5}


def _iters(resampler, iters):
    """Chain length (Metropolis) or tries (rejection); None takes the library's default."""
    if iters is not None:
        return int(iters)
    return {"metropolis": METROPOLIS_STEPS, "rejection": REJECTION_TRIES}.get(resampler, 0)


# --------------------------------------------------------------------------- whole tracker
@dataclass
class FrameRecord:
    """What one frame of the oracle produced (all FP64)."""
    x: np.ndarray
    y: np.ndarray
    L: np.ndarray
    M: float
    S: float
    est: tuple
    C: np.ndarray
    u0: float
    anc: np.ndarray
    anc_in: np.ndarray | None = field(default=None)


def track_steps(frames: np.ndarray, N: int, r: int, *, init, sigma=(1.0, 1.0), drift=(0.0, 0.0),
                seed: int = 1, tracker: int = 0, bg=100.0, fg=228.0, nthreads=1, resampler="systematic",
                iters=None):
    """Run the tracker phase by phase (Fig. 1), yielding a FrameRecord per frame.
    Same arithmetic as :func:`track`, with every intermediate array exposed."""
    anc = None
    xa = ya = None
    for t in range(frames.shape[0]):
        x, y = propagate(N, t, seed, xa, ya, anc, init=init, drift=drift, sigma=sigma,
                         tracker=tracker, nthreads=nthreads)
        L = likelihood_all(x, y, frames[t], r, bg, fg, nthreads=nthreads)
        M, e = weights(L)
        S, xh, yh = normalise(e, x, y)
        C = cdf(e, S)
        u0 = resample_u0(seed, t, tracker)
        if resampler == "stratified":
            a = resample_stratified(C, stratified_offsets(seed, t, N, tracker), "f64")
        elif resampler == "multinomial":
            a = resample_multinomial(C, stratified_offsets(seed, t, N, tracker), "f64")
        elif resampler == "gumbel":
            a = resample_gumbel(L, seed, t, tracker, "f64")
        elif resampler == "metropolis":
            a = resample_metropolis(L, _iters(resampler, iters), seed, t, tracker, "f64")
        elif resampler == "rejection":
            a = resample_rejection(L, M, seed, t, tracker, "f64", _iters(resampler, iters))
        elif resampler == "systematic":
            a = resample(C, u0, "f64")
        else:
            raise ValueError(resampler)
        yield FrameRecord(x=x, y=y, L=L, M=M, S=S, est=(xh, yh), C=C, u0=u0, anc=a, anc_in=anc)
        xa, ya, anc = x, y, a


def track(frames: np.ndarray, N: int, r: int, *, init, sigma=(1.0, 1.0), drift=(0.0, 0.0),
          seed: int = 1, tracker: int = 0, bg=100.0, fg=228.0, nthreads=1, resampler="systematic",
          iters=None):
    """Whole FP64 track in C.  Returns (est (T,2), M (T,), S (T,))."""
    f = np.ascontiguousarray(frames, dtype=np.uint8)
    T, H, W = f.shape
    est = np.empty((T, 2), np.float64)
    M = np.empty(T, np.float64)
    S = np.empty(T, np.float64)
    rc = _load().orc_run(_ptr(f), H * W, T, W, H, W, N, r, bg, fg, init[0], init[1],
                         sigma[0], sigma[1], drift[0], drift[1], seed & 0xFFFFFFFFFFFFFFFF,
                         tracker, nthreads, RESAMPLERS[resampler], _iters(resampler, iters), _ptr(est), _ptr(M), _ptr(S))
    if rc != 0:
        raise MemoryError("oracle could not allocate its arrays")
    return est, M, S
