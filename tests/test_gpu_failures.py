"""Failure paths made on the host, with no GPU fault: an allocation the device cannot
satisfy, and checkpoint blobs that are corrupt.  Each call must return its error status,
leave no sticky CUDA error behind, and leave the library (and the handle, for a refused
checkpoint) usable: the runs after the failure give the same tracks as runs that never
saw it."""
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


def _video():
    return synth.make_video(120, 96, 6, 4, noise=5.0, seed=31, v=(1.0, 0.5))


def _track(pf, v, prec="f16", N=9000, seed=5):
    import torch
    f = pf.Filter(v.W, v.H, N, 4, prec, init=tuple(v.centres[0]), seed=seed)
    f.run(torch.from_numpy(v.frames).cuda())
    e = f.estimates(0, v.T)
    f.close()
    return e


def test_server_arena_beyond_device_memory_is_oom_and_recoverable(pf):
    """A server arena of 10 TB cannot be allocated: pf_server_create answers PF_ERR_OOM,
    hands back no handle, and filters and servers created afterwards run as before."""
    v = _video()
    before = _track(pf, v)
    with pytest.raises(pf.PfError) as ei:
        pf.Server(10 ** 13, max_streams=2, queue_depth=2)
    assert ei.value.status == pf.PF_ERR_OOM
    import torch
    torch.cuda.synchronize()                       # no sticky error left on the context
    assert np.array_equal(_track(pf, v), before)
    s = pf.Server(1 << 28, max_streams=2, queue_depth=2)
    sid = s.open(pf.make_config(v.W, v.H, 9000, 4, "f16", init=tuple(v.centres[0]), seed=5))
    fr = torch.from_numpy(v.frames).cuda()
    for t in range(v.T):
        assert s.submit(sid, fr[t])
        s.drain()
    served = np.array([s.result(sid, t) for t in range(v.T)])
    s.close()
    assert np.array_equal(served, before)


def _corruptions(pf, blob, prec_code, N):
    hsz = ctypes.sizeof(pf.PfStateHeader)
    hdr = pf.PfStateHeader.from_buffer_copy(blob[:hsz])

    def with_field(name, value):
        h = pf.PfStateHeader.from_buffer_copy(bytes(hdr))
        setattr(h, name, value)
        return bytes(h) + blob[hsz:]

    other_prec = pf.PF_F32 if prec_code != pf.PF_F32 else pf.PF_F16
    return {
        "truncated body": blob[:-1],
        "header only": blob[:hsz],
        "empty": b"",
        "bad magic": with_field("magic", 0x31534651),
        "other precision": with_field("precision", other_prec),
        "other particle count": with_field("num_particles", N + 1),
        "negative frame index": with_field("t", -1),
        "zero weight sum": with_field("sum_e", 0.0),
        "negative weight sum": with_field("sum_e", -1.0),
        "NaN weight sum": with_field("sum_e", float("nan")),
        "infinite max likelihood": with_field("max_l", float("inf")),
        "NaN max likelihood": with_field("max_l", float("nan")),
    }


@pytest.mark.parametrize("prec", ["ref64", "f32", "f16", "bf16"])
def test_corrupt_checkpoints_are_refused_and_the_filter_resumes(pf, prec):
    """Every corrupt blob is refused with PF_ERR_ARG before anything is written; the
    filter keeps its state, and restoring the good blob afterwards resumes the track
    exactly where an uninterrupted run goes."""
    import torch
    v = _video()
    fr = torch.from_numpy(v.frames).cuda()
    ref = pf.Filter(v.W, v.H, 9000, 4, prec, init=tuple(v.centres[0]), seed=5)
    ref.run(fr)
    want = ref.estimates(0, v.T)
    ref.close()

    f = pf.Filter(v.W, v.H, 9000, 4, prec, init=tuple(v.centres[0]), seed=5)
    f.run(fr[:3])
    good = pf.pf_get_state(f.h)
    for what, blob in _corruptions(pf, good, f.precision, 9000).items():
        with pytest.raises(pf.PfError) as ei:
            pf.pf_set_state(f.h, blob or b"\0")
        assert ei.value.status == pf.PF_ERR_ARG, what
        assert pf.pf_get_state(f.h) == good, what       # nothing was written
    # the refused calls did not disturb the run: it continues as if uninterrupted
    for t in range(3, v.T):
        f.step(fr[t])
    assert np.array_equal(f.estimates(0, v.T), want)
    # and the good blob restores frame 3's state into a fresh filter
    g = pf.Filter(v.W, v.H, 9000, 4, prec, init=tuple(v.centres[0]), seed=5)
    pf.pf_set_state(g.h, good)
    for t in range(3, v.T):
        g.step(fr[t])
    assert np.array_equal(g.estimates(3, v.T - 3), want[3:])
    f.close()
    g.close()
