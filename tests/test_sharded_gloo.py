"""One tracker sharded by particles (paper_2308_00763_gb300.sharded) on CPU ranks.

The exchange logic -- the global M, S, estimate and per-rank prefixes from the gathered
statistics, the offspring runs of the ranks and the all-to-all that delivers every rank the
ancestors of its own slots -- is the library's own code (`ShardedTracker`, `TorchComm`)
running over gloo with 2 and 3 processes.  Each rank's compute is an FP64 stand-in built
from the oracle (test infrastructure: the GPU shards run the same exchange in
test_gpu_sharded.py): it propagates its slots with draws keyed by the global particle index
(Eq. 1-2), scores them (Eq. 3), and resamples its particles against the global CDF with the
global systematic strata (reading C8).  The sharded track must equal the unsharded oracle's
within 1e-9 px (the CDF is summed in another order, so only rounding differs).
"""
import math
import os
import socket

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

import oracle  # noqa: E402
from paper_2308_00763_gb300 import sharded, synth  # noqa: E402


class OracleShard:
    """Rank `rank`'s slots of an N-particle tracker, computed in FP64 with the oracle."""

    def __init__(self, N, r, rank, nranks, *, init, seed, sigma=(1.0, 1.0), drift=(0.0, 0.0)):
        self.N, self.r, self.rank = N, r, rank
        starts, counts = sharded.partition(N, nranks)
        self.first, self.count = starts[rank], counts[rank]
        self.init, self.seed, self.sigma, self.drift = init, seed, sigma, drift
        self.t = 0
        self.dtype = torch.float64

    def step(self, frame, recv_x=None, recv_y=None):
        N, sl = self.N, slice(self.first, self.first + self.count)
        if self.t == 0:
            x, y = oracle.propagate(N, 0, self.seed, None, None, None, init=self.init, drift=self.drift,
                                    sigma=self.sigma)
        else:
            xa = np.zeros(N)
            ya = np.zeros(N)
            xa[sl] = recv_x.numpy()
            ya[sl] = recv_y.numpy()
            x, y = oracle.propagate(N, self.t, self.seed, xa, ya, np.arange(N), init=self.init, drift=self.drift,
                                    sigma=self.sigma)
        self.x, self.y = x[sl], y[sl]
        self.L = oracle.likelihood_all(self.x, self.y, frame.numpy(), self.r)
        self.t += 1

    def stats(self):
        M, e = oracle.weights(self.L)
        S, ex, ey = oracle.normalise(e, self.x, self.y)
        return (M, S, ex, ey)

    def resample(self, global4, last, send_x, send_y):
        M, S, lo, hi = global4
        e = np.exp(self.L - M)
        P = lo + np.cumsum(e)
        P = np.minimum(P, hi)
        P[-1] = hi
        C = np.minimum(P / S, 1.0)
        if last:
            C[-1] = 1.0
        u0 = oracle.resample_u0(self.seed, self.t - 1)
        inv_n = 1.0 / self.N

        def count(c):   # strata points u_j = (j + u0) / N at or below c
            j = np.arange(self.N)
            return int(np.sum((j + u0) * inv_n <= c))

        j0 = count(min(lo / S, 1.0))
        j1 = count(C[-1])
        u = (np.arange(j0, j1) + u0) * inv_n
        a = np.searchsorted(C, u, side="left")           # first k with C_k >= u_j
        a = np.minimum(a, self.count - 1)
        send_x[:j1 - j0] = torch.from_numpy(self.x[a])
        send_y[:j1 - j0] = torch.from_numpy(self.y[a])
        return j0, j1


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, ws, port, N, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(ws))
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    try:
        v = synth.make_video(128, 128, 10, 5, noise=5.0, seed=1)
        shard = OracleShard(N, 5, rank, ws, init=tuple(v.centres[0]), seed=1)
        tr = sharded.ShardedTracker([shard], ws, N, sharded.TorchComm())
        tr.run(torch.from_numpy(v.frames))
        q.put((rank, tr.estimates().tolist()))
        dist.barrier()
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("ws,N", [(2, 1000), (3, 1001)])
def test_sharded_track_equals_unsharded_oracle(ws, N):
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, ws, port, N, q)) for r in range(ws)]
    for p in procs:
        p.start()
    out = dict(q.get(timeout=300) for _ in range(ws))
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    v = synth.make_video(128, 128, 10, 5, noise=5.0, seed=1)
    want, _, _ = oracle.track(v.frames, N, 5, init=tuple(v.centres[0]), seed=1)
    for rank in range(ws):
        got = np.array(out[rank])
        assert got.shape == want.shape
        assert np.abs(got - want).max() <= 1e-9, (rank, np.abs(got - want).max())


def test_partition_even_starts_and_cover():
    for N, R in [(1000, 2), (1001, 3), (2 ** 20, 8), (17, 4)]:
        starts, counts = sharded.partition(N, R)
        assert starts[0] == 0 and sum(counts) == N
        assert all(s % 2 == 0 for s in starts)
        assert all(starts[q] + counts[q] == starts[q + 1] for q in range(R - 1))
    with pytest.raises(ValueError):
        sharded.partition(5, 3)


def test_combine_equals_whole_arrays():
    """The rescaling merge of the ranks' (M_q, S_q, estimate_q) equals the whole cloud's
    log-sum-exp statistics and weighted mean, and P is the exclusive prefix."""
    rng = np.random.default_rng(3)
    L = rng.normal(0, 40, 5000)
    x = rng.normal(60, 3, 5000)
    y = rng.normal(40, 3, 5000)
    starts, counts = sharded.partition(5000, 3)
    stats = []
    for s, c in zip(starts, counts):
        M, e = oracle.weights(L[s:s + c])
        S, ex, ey = oracle.normalise(e, x[s:s + c], y[s:s + c])
        stats.append((M, S, ex, ey))
    g = sharded.combine(stats)
    M, e = oracle.weights(L)
    S, ex, ey = oracle.normalise(e, x, y)
    assert g.M == M
    assert g.S == pytest.approx(S, rel=1e-13)
    assert g.est_x == pytest.approx(ex, abs=1e-11) and g.est_y == pytest.approx(ey, abs=1e-11)
    for q, s in enumerate(starts):
        assert g.P[q] == pytest.approx(math.fsum(np.exp(L[:s] - M)), rel=1e-12, abs=1e-300)
    assert g.P[-1] == g.S


def test_splits_route_every_offspring_to_its_slot_owner():
    starts, counts = [0, 400, 800], [400, 400, 201]
    runs = [(0, 10), (10, 990), (990, 1001)]
    total_send = np.zeros(3, int)
    for q in range(3):
        send, recv = sharded.splits(runs, starts, counts, q)
        assert sum(send) == runs[q][1] - runs[q][0]
        assert sum(recv) == counts[q]
        total_send += np.array(send)
    assert list(total_send) == counts
    with pytest.raises(ValueError):
        sharded.splits([(0, 10), (11, 1001)], [0, 500], [500, 501], 0)
