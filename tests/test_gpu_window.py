"""The likelihood-table window of every tile covers the reach of its heavy ancestors.

Each tile tabulates the likelihood (Eq. 3 / Eq. 4) over a window: the bounding box of its
ancestors whose weight exp(L - M) is above 2^-30, widened by the drift and at least 3.5
sigma of the draw (Eq. 1-2) plus a pixel.  An offspring outside the window is evaluated
directly from the frame (the same arithmetic, so results never depend on the window), but
a window that misses heavy ancestors sends many offspring down that slow route.  This
checks the rule itself through the debug hook (pf_get_debug(which = 2)): for every tile of
every step, the window contains each heavy ancestor's position widened by |drift| + 3.5
sigma, at sizes whose last tile is ragged and lies within the first warp of its CTA.
"""
import math

import numpy as np
import pytest

from paper_2308_00763_gb300 import synth

pytestmark = pytest.mark.gpu

TILE = 4096  # particles per tile for a tracker smaller than half the device


@pytest.fixture(scope="module")
def pf():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2308_00763_gb300 as m
    m.lib(build_if_missing=True)
    return m


def _abs_positions(st, prec):
    if prec in ("f16", "bf16"):
        return st["x"] + st["anchor_x"], st["y"] + st["anchor_y"]
    return st["x"], st["y"]


@pytest.mark.parametrize("prec", ["ref64", "f32", "f16", "bf16"])
@pytest.mark.parametrize("N", [TILE + 200, 2 * TILE + 37, 150])
def test_window_covers_heavy_ancestors(pf, prec, N):
    import torch
    sig, drift = (2.0, 1.5), (1.0, -1.0)
    v = synth.make_video(160, 120, 8, 4, noise=5.0, seed=11, v=drift)
    frames = torch.from_numpy(v.frames).cuda()
    f = pf.Filter(v.W, v.H, N, 4, prec, init=tuple(v.centres[0]), sigma=sig, drift=drift, seed=5,
                  flags=pf.PF_FLAG_DEBUG_ARRAYS)
    f.step(frames[0])
    checked = 0
    for t in range(1, v.T):
        st = f.get_state()                       # the ancestors: frame t - 1
        f.step(frames[t])
        win = f.debug(2)
        assert len(win) == math.ceil(N / TILE)
        x, y = _abs_positions(st, prec)
        heavy = st["L"] - st["max_l"] > -20.0    # weight above e^-20 of the largest (< 2^-28)
        for q, (x0, y0, w, h) in enumerate(win):
            sl = slice(q * TILE, min(N, (q + 1) * TILE))
            hx, hy = x[sl][heavy[sl]], y[sl][heavy[sl]]
            if len(hx) == 0:
                continue
            assert w > 0 and h > 0, (t, q, "no table for a tile with heavy ancestors")
            rx = abs(drift[0]) + 3.5 * sig[0]
            ry = abs(drift[1]) + 3.5 * sig[1]
            assert x0 <= math.floor(hx.min() - rx) and x0 + w - 1 >= math.ceil(hx.max() + rx), (t, q, x0, w)
            assert y0 <= math.floor(hy.min() - ry) and y0 + h - 1 >= math.ceil(hy.max() + ry), (t, q, y0, h)
            checked += 1
    f.close()
    assert checked >= v.T - 1


def test_window_hook_needs_debug_arrays(pf):
    f = pf.Filter(64, 64, 1000, 3, "f32")
    with pytest.raises(pf.PfError):
        f.debug(2)
    f.close()
