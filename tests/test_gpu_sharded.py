"""One tracker sharded by particles, every shard on this GPU, driven by one process.

The shards are the library's (pf_shard_*); the exchange between them is
paper_2308_00763_gb300.sharded's host logic with the in-process communicator (slices of
the shards' device buffers; no kernel waits on another).  The sharded REF64 track equals
the unsharded oracle's within 1e-9 px; F32 matches it within 1e-3 px on frame 0 (before
any resampling decision) and within 0.05 px RMSE over the track (reading C15: FP32 CDF
rounding may flip a decision against the FP64 oracle's); the ranks' offspring runs tile
[0, N).
"""
import math

import numpy as np
import pytest

import oracle
from paper_2308_00763_gb300 import sharded, synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pf():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2308_00763_gb300 as m
    m.lib(build_if_missing=True)
    return m


class RecordingShard:
    """A library shard that records the offspring runs it produced."""

    def __init__(self, shard):
        self.s = shard
        self.rank, self.first, self.count, self.dtype = shard.rank, shard.first, shard.count, shard.dtype
        self.runs = []

    def stats(self):
        return self.s.stats()

    def resample(self, global4, last, sx, sy):
        run = self.s.resample(global4, last, sx, sy)
        self.runs.append(run)
        return run

    def step(self, frame, rx=None, ry=None):
        self.s.step(frame, rx, ry)


def _sharded_track(pf, v, N, prec, R, seed=1):
    import torch
    shards = [RecordingShard(pf.Shard(v.W, v.H, N, v.radius, prec, rank=q, nranks=R, init=tuple(v.centres[0]),
                                      seed=seed)) for q in range(R)]
    tr = sharded.ShardedTracker(shards, R, N, sharded.LocalComm())
    tr.run(torch.from_numpy(v.frames).cuda())
    est = tr.estimates()
    for f in range(v.T - 1):     # the runs of every resampled frame tile [0, N)
        runs = [s.runs[f] for s in shards]
        assert runs[0][0] == 0 and runs[-1][1] == N
        assert all(runs[q][1] == runs[q + 1][0] for q in range(R - 1))
    for s in shards:
        s.s.close()
    return est


@pytest.mark.parametrize("R,N", [(2, 1000), (3, 1001), (2, 6 * 4096 + 6), (4, 3 * 4096 + 2)])
def test_sharded_ref64_track_equals_oracle(pf, R, N):
    v = synth.make_video(128, 128, 10, 5, noise=5.0, seed=1)
    want, _, _ = oracle.track(v.frames, N, 5, init=tuple(v.centres[0]), seed=1)
    got = _sharded_track(pf, v, N, "ref64", R)
    assert np.abs(got - want).max() <= 1e-9


@pytest.mark.parametrize("R", [2, 3])
def test_sharded_f32_track(pf, R):
    v = synth.make_video(160, 120, 8, 4, noise=5.0, seed=7, v=(1.0, -1.0))
    N = 5 * 4096 + 14
    want, _, _ = oracle.track(v.frames, N, 4, init=tuple(v.centres[0]), seed=3)
    got = _sharded_track(pf, v, N, "f32", R, seed=3)
    assert np.abs(got[0] - want[0]).max() <= 1e-3
    assert math.sqrt(np.mean(np.sum((got - want) ** 2, axis=1))) <= 0.05


def test_shard_arguments(pf):
    with pytest.raises(pf.PfError):         # half precisions keep anchor offsets: not sharded
        pf.Shard(64, 64, 1000, 3, "f16", rank=0, nranks=2)
    with pytest.raises(pf.PfError):         # systematic resampling only
        pf.Shard(64, 64, 1000, 3, "ref64", rank=0, nranks=2, resampler="multinomial")
    with pytest.raises(pf.PfError):         # fewer than two particles per rank
        pf.Shard(64, 64, 5, 3, "ref64", rank=0, nranks=3)
    assert pf.pf_shard_partition(1001, 3, 2) == (664, 337)
