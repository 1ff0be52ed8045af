"""pf_step_frame_noalloc: the frame step for callers that cannot allocate device memory.

Such callers (an engine that owns all CUDA memory, a real-time loop that forbids
allocation after start-up) pass every input and output buffer themselves; the step's
scratch lives in a fixed device array inside the library.  This file is collected last so
that a run stopping at the first failure has already run every other test.

The check: two consecutive frames stepped through the allocation-free entry point give
the same particles and estimates, bit for bit, as the same two frames stepped by a
pf_filter handle (the same kernel with the same tiles): at a ragged size, at the 2^22
maximum (the scratch array's largest tile count), and after a larger call has left its
contents in the shared array.
"""
import ctypes

import numpy as np
import pytest

from paper_2308_00763_gb300 import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pf():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2308_00763_gb300 as m
    m.lib(build_if_missing=True)
    return m


_TORCH_DTYPE = {"ref64": "float64", "f32": "float32", "f16": "float16", "bf16": "bfloat16"}


def _two_frames(pf, prec, resampler, N, W=160, H=120):
    """Two frames through a pf_filter handle and through the allocation-free entry point:
    (the handle's states and estimates, the entry point's headers and second-frame buffers)."""
    import torch
    v = synth.make_video(W, H, 2, 4, noise=5.0, seed=31, v=(1.0, -1.0))
    frames = torch.from_numpy(v.frames).cuda()
    kw = dict(init=tuple(v.centres[0]), seed=77, tracker_id=2, resampler=resampler)
    f = pf.Filter(v.W, v.H, N, 4, prec, **kw)
    f.step(frames[0])
    st0 = f.get_state()
    f.step(frames[1])
    st1 = f.get_state()
    est = f.estimates(0, 2)
    f.close()
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
    return (st0, st1, est), (out0, out1, bufs[1])


def _assert_same(ref, got, prec):
    (st0, st1, est), (out0, out1, buf1) = ref, got
    assert out0.t == 1 and out1.t == 2
    for out, want in ((out0, est[0]), (out1, est[1])):
        assert (out.est_x, out.est_y) == (want[0], want[1])
    for out, st in ((out0, st0), (out1, st1)):
        assert out.max_l == st["max_l"] and out.sum_e == st["sum_e"]
        assert (out.next_anchor_x, out.next_anchor_y) == (st["next_anchor_x"], st["next_anchor_y"])
    for b, name in zip(buf1, ("x", "y", "L")):
        g = b.float().cpu().numpy().astype(np.float64) if prec == "bf16" else b.cpu().numpy().astype(np.float64)
        assert np.array_equal(g, st1[name]), (prec, name)


@pytest.mark.parametrize("prec", ["f32", "f16"])
def test_noalloc_largest_size_then_small_size(pf, prec):
    """At the 2^22-particle limit (the most tiles the scratch array holds), then a small
    tracker whose call finds the large one's descriptors and partials beyond its own tiles
    in the shared array: both equal a fresh pf_filter bit for bit."""
    _assert_same(*_two_frames(pf, prec, "systematic", 1 << 22, W=512, H=512), prec)
    _assert_same(*_two_frames(pf, prec, "systematic", 4096 + 3), prec)


def test_noalloc_rejects_overlapping_buffers_and_missing_state_out(pf):
    import torch
    N = 1000
    cfg = pf.make_config(64, 64, N, 3, "f32")
    hdr = pf.PfStateHeader(magic=0x31534650, precision=cfg.precision, num_particles=N, t=0)
    frame = torch.zeros((64, 64), dtype=torch.uint8, device="cuda")
    buf = torch.zeros(4 * N + 64, dtype=torch.float32, device="cuda")
    base = buf.data_ptr()
    out = pf.PfStateHeader()
    P = ctypes.c_void_p
    # y_out starts inside x_out
    rc = pf.lib().pf_step_frame_noalloc(ctypes.byref(cfg), ctypes.byref(hdr), None, None, None,
                                        P(frame.data_ptr()), 64, P(base), P(base + 16 * 100),
                                        P(base + 16 * 600), ctypes.byref(out), None)
    assert rc == pf.PF_ERR_ARG
    # distinct buffers but no state_out
    rc = pf.lib().pf_step_frame_noalloc(ctypes.byref(cfg), ctypes.byref(hdr), None, None, None,
                                        P(frame.data_ptr()), 64, P(base), P(base + 4 * 1008),
                                        P(base + 8 * 1008), None, None)
    assert rc == pf.PF_ERR_ARG
    # an input that is also an output (frame t > 0)
    hdr1 = pf.PfStateHeader(magic=0x31534650, precision=cfg.precision, num_particles=N, t=1, max_l=0.0, sum_e=1.0)
    other = torch.zeros(3 * N + 64, dtype=torch.float32, device="cuda").data_ptr()
    rc = pf.lib().pf_step_frame_noalloc(ctypes.byref(cfg), ctypes.byref(hdr1), P(base), P(other),
                                        P(other + 4 * 1008), P(frame.data_ptr()), 64, P(base),
                                        P(base + 4 * 1008), P(base + 8 * 1008), ctypes.byref(out), None)
    assert rc == pf.PF_ERR_ARG
    torch.cuda.synchronize()


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

    # the same kernel on the same tiles: the same bits
    _assert_same((st0, st1, est), (out0, out1, bufs[1]), prec)


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


def test_noalloc_rejects_stream_capture(pf):
    """The call waits for its step and reads the state back, so it refuses a capturing stream
    (before it touches the device) and the stream stays usable."""
    import torch
    N = 1000
    cfg = pf.make_config(64, 64, N, 3, "f32")
    hdr = pf.PfStateHeader(magic=0x31534650, precision=cfg.precision, num_particles=N, t=0)
    frame = torch.zeros((64, 64), dtype=torch.uint8, device="cuda")
    bufs = [torch.zeros(N + 16, dtype=torch.float32, device="cuda") for _ in range(3)]
    out = pf.PfStateHeader()
    P = ctypes.c_void_p
    s = torch.cuda.Stream()
    g = torch.cuda.CUDAGraph()
    torch.cuda.synchronize()
    with torch.cuda.graph(g, stream=s):
        rc = pf.lib().pf_step_frame_noalloc(ctypes.byref(cfg), ctypes.byref(hdr), None, None, None,
                                            P(frame.data_ptr()), 64, P(bufs[0].data_ptr()), P(bufs[1].data_ptr()),
                                            P(bufs[2].data_ptr()), ctypes.byref(out), P(s.cuda_stream))
        bufs[0].add_(1.0)    # something to capture
    assert rc == pf.PF_ERR_ARG
    rc = pf.lib().pf_step_frame_noalloc(ctypes.byref(cfg), ctypes.byref(hdr), None, None, None,
                                        P(frame.data_ptr()), 64, P(bufs[0].data_ptr()), P(bufs[1].data_ptr()),
                                        P(bufs[2].data_ptr()), ctypes.byref(out), P(s.cuda_stream))
    assert rc == pf.PF_OK and out.t == 1
    torch.cuda.synchronize()
