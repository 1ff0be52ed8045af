"""Seeded synthetic monochrome video: the tracking input of the particle filter.

The paper evaluates on a synthetic video in the style of the Rodinia particle-filter
application (Sec. V, "Verification & Accuracy Results"): one disk-shaped object of a
single foreground intensity on a background of a single intensity, Gaussian noise
added to every pixel, and the object bouncing specularly off the frame walls.  Neither
that generator nor its data is available, so this module stands in for it with the
same shapes: W x H uint8 frames, a disk of radius r, constant velocity v, intensity
levels 100 / 228 (the two constants of Eq. 3) and additive noise of std ``noise``.

This module is an *input generator only*.  It is shared by the CUDA path, the bench and
the CPU oracle, and it holds none of the filter's arithmetic: no random draw of the
method (those come from each side's own Philox4x32-10), no likelihood, no weighting,
no resampling.  Its noise comes from numpy's PCG64 stream, seeded per video.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np

__all__ = ["Video", "reflect", "centre_track", "make_video", "make_video_device", "batch_workload",
           "serving_workload"]


@dataclass
class Video:
    """T frames of H x W uint8 pixels plus the ground-truth disk centre of each frame."""

    frames: np.ndarray   # (T, H, W) uint8, C-contiguous, row-major (y = row, x = column)
    centres: np.ndarray  # (T, 2) float64, (x, y) of the disk centre in pixel units
    radius: int
    noise: float
    seed: int

    @property
    def T(self) -> int:
        return int(self.frames.shape[0])

    @property
    def H(self) -> int:
        return int(self.frames.shape[1])

    @property
    def W(self) -> int:
        return int(self.frames.shape[2])


def reflect(p: np.ndarray, lo: float, hi: float) -> np.ndarray:
    """Fold an unconstrained coordinate into [lo, hi] by specular reflection at both walls."""
    p = np.asarray(p, dtype=np.float64)
    span = hi - lo
    if span <= 0:
        return np.full_like(p, lo)
    q = np.mod(p - lo, 2.0 * span)
    q = np.where(q > span, 2.0 * span - q, q)
    return lo + q


def centre_track(W: int, H: int, T: int, r: int, v=(1.0, -2.0), c0=None,
                 bounce: bool = True) -> np.ndarray:
    """Centre of the disk in frames 0..T-1: c0 + t*v, folded into [r, W-1-r] x [r, H-1-r]."""
    if c0 is None:
        c0 = (W / 2.0, H / 2.0)
    t = np.arange(T, dtype=np.float64)
    cx = c0[0] + t * float(v[0])
    cy = c0[1] + t * float(v[1])
    if bounce:
        cx = reflect(cx, float(r), float(W - 1 - r))
        cy = reflect(cy, float(r), float(H - 1 - r))
    return np.stack([cx, cy], axis=1)


def make_video(W: int, H: int, T: int, r: int, *, v=(1.0, -2.0), c0=None,
               noise: float = 5.0, bg: int = 100, fg: int = 228, seed: int = 1,
               bounce: bool = True) -> Video:
    """Render T frames: bg everywhere, fg inside the disk (x-cx)^2 + (y-cy)^2 <= r^2,
    plus noise * N(0, 1) per pixel, rounded half up and clamped to [0, 255]."""
    centres = centre_track(W, H, T, r, v=v, c0=c0, bounce=bounce)
    rng = np.random.default_rng(seed)
    ys = np.arange(H, dtype=np.float64)[:, None]
    xs = np.arange(W, dtype=np.float64)[None, :]
    frames = np.empty((T, H, W), dtype=np.uint8)
    r2 = float(r) * float(r)
    for t in range(T):
        cx, cy = centres[t]
        inside = (xs - cx) ** 2 + (ys - cy) ** 2 <= r2
        img = np.where(inside, float(fg), float(bg))
        if noise > 0:
            img = img + noise * rng.standard_normal((H, W))
        frames[t] = np.clip(np.floor(img + 0.5), 0, 255).astype(np.uint8)
    return Video(frames=frames, centres=centres, radius=int(r), noise=float(noise), seed=int(seed))


def make_video_device(W: int, H: int, T: int, r: int, *, v=(1.0, -2.0), c0=None, noise: float = 5.0,
                      bg: int = 100, fg: int = 228, seed: int = 1, bounce: bool = True, device="cuda"):
    """The same recipe as :func:`make_video`, rendered on a torch device with torch's
    generator (so its noise differs from the numpy stream).  For inputs too large to render
    on the host, such as a batch of hundreds of videos.  Returns (frames (T, H, W) uint8
    tensor, centres (T, 2) numpy)."""
    import torch
    centres = centre_track(W, H, T, r, v=v, c0=c0, bounce=bounce)
    g = torch.Generator(device=device)
    g.manual_seed(int(seed))
    ys = torch.arange(H, dtype=torch.float32, device=device)[:, None]
    xs = torch.arange(W, dtype=torch.float32, device=device)[None, :]
    out = torch.empty((T, H, W), dtype=torch.uint8, device=device)
    r2 = float(r) * float(r)
    for t in range(T):
        cx, cy = float(centres[t, 0]), float(centres[t, 1])
        inside = (xs - cx) ** 2 + (ys - cy) ** 2 <= r2
        img = torch.where(inside, torch.tensor(float(fg), device=device), torch.tensor(float(bg), device=device))
        if noise > 0:
            img = img + noise * torch.randn((H, W), generator=g, device=device)
        out[t] = torch.clamp(torch.floor(img + 0.5), 0, 255).to(torch.uint8)
    return out, centres


def batch_workload(n: int = 256, T: int = 60, seed: int = 4):
    """Parameters of the batched-trackers workload: frame sizes uniform from
    {256^2, 512^2, 1024^2}, particle counts log-uniform in [1000, 262144], disk radius
    uniform in 3..12, constant velocity of uniform angle and speed in [0, 4) px/frame,
    noise 5, T frames; video i has seed 1000 + i."""
    rng = np.random.default_rng(seed)
    sizes = rng.choice([256, 512, 1024], size=n)
    N = np.floor(np.exp(rng.uniform(np.log(1000.0), np.log(262144.0), size=n))).astype(np.int64)
    r = rng.integers(3, 13, size=n)
    ang = rng.uniform(0.0, 2.0 * np.pi, size=n)
    spd = rng.uniform(0.0, 4.0, size=n)
    return [dict(W=int(sizes[i]), H=int(sizes[i]), T=T, r=int(r[i]), N=int(N[i]),
                 v=(float(spd[i] * np.cos(ang[i])), float(spd[i] * np.sin(ang[i]))),
                 noise=5.0, seed=1000 + i) for i in range(n)]


def serving_workload(n: int = 1024, seconds: float = 60.0, fps: float = 30.0, seed: int = 5):
    """Streams of the served multi-camera workload: stream i opens at U(0, 5/6 s) and stays
    open U(1/12 s, s) (clipped to the run of s seconds; s = 60 gives opens over the first
    50 s and lifetimes of 5-60 s), frames of 256^2, 512^2 or 1024^2 pixels, N log-uniform in
    [4096, 2^20], disk radius 3..12, FP16 or FP32 with probability 1/2 each, and frames
    arriving as a Poisson process of rate `fps` (exponential gaps) while it is open."""
    rng = np.random.default_rng(seed)
    out = []
    for i in range(n):
        size = int(rng.choice([256, 512, 1024]))
        N = int(np.floor(np.exp(rng.uniform(np.log(4096.0), np.log(float(1 << 20))))))
        t_open = float(rng.uniform(0.0, seconds * 5.0 / 6.0))
        t_close = min(seconds, t_open + float(rng.uniform(seconds / 12.0, seconds)))
        arrivals = []
        t = t_open + float(rng.exponential(1.0 / fps))
        while t < t_close:
            arrivals.append(t)
            t += float(rng.exponential(1.0 / fps))
        out.append(dict(W=size, H=size, N=N, r=int(rng.integers(3, 13)),
                        precision="f16" if rng.random() < 0.5 else "f32",
                        open=t_open, close=t_close, arrivals=arrivals, seed=2000 + i))
    return out
