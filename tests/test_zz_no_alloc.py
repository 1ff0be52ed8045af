"""pf_step_frame_noalloc: the frame step for callers that cannot allocate device memory.

Such callers (an engine that owns all CUDA memory, a real-time loop that forbids
allocation after start-up) pass every input and output buffer themselves; the step's
scratch lives in a fixed device array inside the library.  This file is collected last so
that a run stopping at the first failure has already run every other test.

The check: two consecutive frames stepped through the allocation-free entry point give
the same particles and estimates as the same two frames stepped by a pf_filter handle.
"""
import ctypes

import numpy as np
import pytest

from paper_2308_00763_gb300 import synth

pytestmark = pytest.mark.gpu

TOL_PX = {"ref64": 1e-9, "f32": 1e-3, "f16": 0.5, "bf16": 0.5}   # the parity tests' tolerances


@pytest.fixture(scope="module")
def pf():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2308_00763_gb300 as m
    m.lib(build_if_missing=True)
    return m


_TORCH_DTYPE = {"ref64": "float64", "f32": "float32", "f16": "float16", "bf16": "bfloat16"}


@pytest.mark.parametrize("resampler", ["systematic", "stratified"])
@pytest.mark.parametrize("prec", ["ref64", "f32", "f16", "bf16"])
def test_noalloc_two_frames_match_filter(pf, prec, resampler):
    import torch
    N = 3 * 4096 + 11
    v = synth.make_video(160, 120, 2, 4, noise=5.0, seed=31, v=(1.0, -1.0))
    frames = torch.from_numpy(v.frames).cuda()
    kw = dict(init=tuple(v.centres[0]), seed=77, tracker_id=2, resampler=resampler)

    # reference: a pf_filter handle
    f = pf.Filter(v.W, v.H, N, 4, prec, **kw)
    f.step(frames[0])
    st0 = f.get_state()
    f.step(frames[1])
    st1 = f.get_state()
    est = f.estimates(0, 2)
    f.close()

    # caller-owned buffers (the test allocates them; the entry point allocates nothing)
    dt = getattr(torch, _TORCH_DTYPE[prec])
    bufs = [[torch.zeros(N, dtype=dt, device="cuda") for _ in range(3)] for _ in range(2)]
    cfg = pf.make_config(v.W, v.H, N, 4, prec, **kw)
    hdr = pf.PfStateHeader(magic=0x31534650, precision=cfg.precision, num_particles=N, t=0)
    stream = torch.cuda.current_stream()
    ptr = [[b.data_ptr() for b in slot] for slot in bufs]
    out0 = pf.pf_step_frame_noalloc(cfg, hdr, 0, 0, 0, frames[0].data_ptr(), frames.stride(1),
                                    *ptr[0], stream=stream)
    out1 = pf.pf_step_frame_noalloc(cfg, out0, *ptr[0], frames[1].data_ptr(), frames.stride(1),
                                    *ptr[1], stream=stream)
    torch.cuda.synchronize()

    tol = TOL_PX[prec]
    assert out0.t == 1 and out1.t == 2
    for out, want in ((out0, est[0]), (out1, est[1])):
        assert abs(out.est_x - want[0]) <= tol and abs(out.est_y - want[1]) <= tol
    for out, st in ((out0, st0), (out1, st1)):
        assert out.max_l == st["max_l"] and out.sum_e == pytest.approx(st["sum_e"], rel=1e-12)
        assert (out.next_anchor_x, out.next_anchor_y) == (st["next_anchor_x"], st["next_anchor_y"])
    # the particles of the second frame, element by element
    for got, name in zip(bufs[1], ("x", "y", "L")):
        g = got.float().cpu().numpy().astype(np.float64) if prec == "bf16" else got.cpu().numpy().astype(np.float64)
        np.testing.assert_allclose(g, st1[name], rtol=0, atol=tol if name != "L" else 1e-6)


@pytest.mark.parametrize("scheme", ["multinomial", "gumbel", "metropolis", "rejection"])
def test_noalloc_rejects_pull_schemes(pf, scheme):
    """Multinomial, Gumbel-max, Metropolis and rejection resampling keep a CDF or the ancestors in
    device memory and run two more kernels; the allocation-free entry point takes
    systematic and stratified trackers only."""
    cfg = pf.make_config(64, 64, 1000, 3, "f32", resampler=scheme)
    hdr = pf.PfStateHeader(magic=0x31534650, precision=cfg.precision, num_particles=1000, t=0)
    with pytest.raises(pf.PfError):
        pf.pf_step_frame_noalloc(cfg, hdr, 0, 0, 0, 1 << 20, 64, 1 << 20, 1 << 20, 1 << 20, stream=0)


def test_noalloc_rejects_too_many_particles(pf):
    cfg = pf.make_config(64, 64, (1 << 22) + 1, 3, "f32")
    hdr = pf.PfStateHeader(magic=0x31534650, precision=cfg.precision, num_particles=cfg.num_particles, t=0)
    out = pf.PfStateHeader()
    rc = pf.lib().pf_step_frame_noalloc(ctypes.byref(cfg), ctypes.byref(hdr), None, None, None,
                                        ctypes.c_void_p(1), 64, ctypes.c_void_p(1), ctypes.c_void_p(1),
                                        ctypes.c_void_p(1), ctypes.byref(out), None)
    assert rc == pf.PF_ERR_ARG


def test_noalloc_rejects_misaligned_buffers(pf):
    import torch
    N = 64
    cfg = pf.make_config(64, 64, N, 3, "f32")
    hdr = pf.PfStateHeader(magic=0x31534650, precision=cfg.precision, num_particles=N, t=0)
    frame = torch.zeros((64, 64), dtype=torch.uint8, device="cuda")
    buf = torch.zeros(4 * N + 4, dtype=torch.float32, device="cuda")
    base = buf.data_ptr()
    out = pf.PfStateHeader()
    # x_out 4 bytes past a 16-byte boundary: rejected before any work is queued
    rc = pf.lib().pf_step_frame_noalloc(ctypes.byref(cfg), ctypes.byref(hdr), None, None, None,
                                        ctypes.c_void_p(frame.data_ptr()), 64,
                                        ctypes.c_void_p(base + 4), ctypes.c_void_p(base + 16 * 32),
                                        ctypes.c_void_p(base + 16 * 48), ctypes.byref(out), None)
    assert rc == pf.PF_ERR_ARG
