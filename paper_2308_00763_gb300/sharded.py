"""One tracker sharded by particles across ranks (one GPU per rank).

The particle filter's per-frame step (Sec. IV, Fig. 1) couples every particle only through
three global quantities of the previous frame: the maximum log-likelihood M and the sum S
of exp(L - M) (Eq. 5 and the normalising kernel), the inclusive prefix of those weights
(the CDF the resampling kernel searches), and the resampled ancestors, which may live on
another rank.  Sharded, rank q holds the contiguous particles [k_q, k_q + n_q) and a frame
takes three exchanges (Sec. II notes that resampling is the step that resists
parallelisation; this is where the exchanges sit):

  1. an all-gather of each rank's (M_q, S_q, estimate_q) of the previous frame: every rank
     then forms the same global M, S, estimate and the exclusive prefix P_q of the rescaled
     totals S_q e^(M_q - M) in rank order (FP64 on the host, identical on every rank);
  2. each rank resamples its own particles against the global CDF (C_k = (P_q + local
     prefix) / S, pinned to P_q / S and P_(q+1) / S at its ends) with the global strata
     u_j = (j + u0) / N: its particles are the ancestors of the contiguous offspring run
     [J(P_q / S), J(P_(q+1) / S)), written as ancestor positions in offspring order;
  3. an all-to-all sends each slice of those runs to the rank that owns the offspring
     slots; every rank receives the ancestor positions of exactly its own slots, in order,
     and propagates them (draws keyed by the global particle index), so the sharded filter
     performs the unsharded filter's method.

This module holds the host logic (pure functions on plain numbers, the same on every rank)
and the driver `ShardedTracker`, which runs one shard per rank through the library's
pf_shard_* entry points and exchanges through a communicator: `TorchComm` over a
torch.distributed process group (NCCL between GPUs), or `LocalComm` for several shards
driven by one process (the exchange then moves slices between the shards' buffers; no
kernel waits on another).
"""
from __future__ import annotations

import math
from dataclasses import dataclass


def partition(N: int, nranks: int):
    """Contiguous particle ranges [k_q, k_q + n_q): n_q = N / nranks rounded to even counts
    (every rank's first particle has an even global index, so a pair of particles (2i, 2i+1),
    which shares one Philox block, never straddles two ranks); the last rank takes the rest."""
    if nranks < 1 or N < 2 * nranks:
        raise ValueError("need at least two particles per rank")
    base = (N // nranks) & ~1
    starts = [q * base for q in range(nranks)]
    counts = [base] * (nranks - 1) + [N - base * (nranks - 1)]
    return starts, counts


@dataclass
class GlobalFrame:
    """The global scalars of one frame, formed identically on every rank."""
    M: float               # max L over all particles
    S: float               # sum exp(L - M) over all particles
    est_x: float           # weighted mean position (the estimate)
    est_y: float
    P: list                # P[q]: sum of the rescaled totals of ranks < q (P[nranks] = S)


def combine(stats):
    """Global frame from per-rank (M_q, S_q, est_x_q, est_y_q), in rank order: the rescaling
    merge of log-sum-exp sums (Eq. 5), the weighted mean of the ranks' estimates, and the
    exclusive prefix of the rescaled totals."""
    M = max(s[0] for s in stats)
    scaled = [s[1] * math.exp(s[0] - M) for s in stats]
    P = [0.0]
    for v in scaled:
        P.append(P[-1] + v)
    S = P[-1]
    ex = sum(v * s[2] for v, s in zip(scaled, stats)) / S
    ey = sum(v * s[3] for v, s in zip(scaled, stats)) / S
    return GlobalFrame(M=M, S=S, est_x=ex, est_y=ey, P=P)


def splits(runs, starts, counts, rank):
    """All-to-all split sizes of `rank`: runs[q] = (jb, je) is rank q's offspring run
    (consecutive runs meet: runs[q][1] == runs[q+1][0], runs[0][0] == 0, runs[-1][1] == N);
    rank r owns slots [starts[r], starts[r] + counts[r]).  Returns (send, recv): send[r] =
    how many of this rank's offspring go to rank r, recv[q] = how many of this rank's slots
    come from rank q (both in rank order, which is offspring order)."""
    n = len(runs)
    for q in range(n - 1):
        if runs[q][1] != runs[q + 1][0]:
            raise ValueError("offspring runs do not meet between ranks %d and %d" % (q, q + 1))

    def overlap(a0, a1, b0, b1):
        return max(0, min(a1, b1) - max(a0, b0))

    jb, je = runs[rank]
    send = [overlap(jb, je, starts[r], starts[r] + counts[r]) for r in range(n)]
    lo, hi = starts[rank], starts[rank] + counts[rank]
    recv = [overlap(runs[q][0], runs[q][1], lo, hi) for q in range(n)]
    return send, recv


class LocalComm:
    """Every rank's shard in this process: the collectives are list operations over the
    shards (rank order); nothing waits on another kernel."""

    def all_gather(self, local):
        """local: this process's per-shard values (all ranks) -> every rank's value."""
        return list(local)

    def all_to_all(self, sends):
        """sends[i][r]: local shard i's tensor for rank r -> recv[i][q]: rank q's tensor for
        local shard i."""
        return [[sends[q][i] for q in range(len(sends))] for i in range(len(sends))]


class TorchComm:
    """One shard per process over a torch.distributed process group (NCCL between GPUs,
    gloo between CPU processes)."""

    def __init__(self, group=None):
        import torch.distributed as dist
        self.dist = dist
        self.group = group

    def all_gather(self, local):
        assert len(local) == 1, "one shard per process"
        out = [None] * self.dist.get_world_size(self.group)
        self.dist.all_gather_object(out, local[0], group=self.group)
        return out

    def all_to_all(self, sends):
        assert len(sends) == 1, "one shard per process"
        import torch
        send = sends[0]
        send_sizes = [int(t.numel()) for t in send]
        recv_sizes = self._sizes(send_sizes)
        recv = torch.empty(sum(recv_sizes), dtype=send[0].dtype, device=send[0].device)
        self.dist.all_to_all_single(recv, torch.cat(send).contiguous(), output_split_sizes=recv_sizes,
                                    input_split_sizes=send_sizes, group=self.group)
        return [list(torch.split(recv, recv_sizes))]

    def _sizes(self, mine):
        """What every rank sends this rank (an all-to-all of the counts)."""
        import torch
        dev = "cuda" if self.dist.get_backend(self.group) == "nccl" else "cpu"
        out = torch.empty(len(mine), dtype=torch.int64, device=dev)
        self.dist.all_to_all_single(out, torch.tensor(mine, dtype=torch.int64, device=dev), group=self.group)
        return [int(v) for v in out.tolist()]


class ShardedTracker:
    """One tracker sharded by particles: `shards` are this process's shards (one per rank
    under torch.distributed, all of them with LocalComm), each with rank, first, count,
    stats(), resample(global4, last, send_x, send_y) -> run, step(frame, recv_x, recv_y) and
    a torch dtype / device for the positions; `comm` carries the exchanges.  Estimates of
    every stepped frame are formed on the host from the gathered statistics (the same on
    every rank)."""

    def __init__(self, shards, nranks, num_particles, comm):
        self.shards = list(shards)
        self.nranks = nranks
        self.N = num_particles
        self.comm = comm
        self.starts, self.counts = partition(num_particles, nranks)
        self.t = 0
        self.est = []            # estimate of every frame whose statistics are combined
        self.frames = []         # the GlobalFrame of those frames
        self._send = {}

    def _buffers(self, s, device, dtype):
        import torch
        key = s.rank
        if key not in self._send:
            self._send[key] = (torch.empty(self.N, dtype=dtype, device=device),
                               torch.empty(self.N, dtype=dtype, device=device))
        return self._send[key]

    def _combine(self):
        """All-gather the shards' statistics of the last stepped frame; record its estimate."""
        stats = self.comm.all_gather([s.stats() for s in self.shards])
        g = combine(stats)
        self.frames.append(g)
        self.est.append((g.est_x, g.est_y))
        return g

    def step(self, frame):
        """Step every shard of this process on `frame` (a device tensor, rows contiguous)."""
        if self.t == 0:
            for s in self.shards:
                s.step(frame)
            self.t = 1
            return
        g = self._combine()
        runs_local, sends = [], []
        for s in self.shards:
            sx, sy = self._buffers(s, frame.device, s.dtype)
            q = s.rank
            run = s.resample((g.M, g.S, g.P[q], g.P[q + 1]), q == self.nranks - 1, sx, sy)
            runs_local.append(run)
        runs = self.comm.all_gather(runs_local)
        for s, run in zip(self.shards, runs_local):
            send, _ = splits(runs, self.starts, self.counts, s.rank)
            sx, sy = self._send[s.rank]
            chunks, at = [], 0
            for n in send:
                chunks.append((sx[at:at + n], sy[at:at + n]))
                at += n
            sends.append(chunks)
        xs = self.comm.all_to_all([[c[0] for c in ch] for ch in sends])
        ys = self.comm.all_to_all([[c[1] for c in ch] for ch in sends])
        import torch
        for s, rx, ry in zip(self.shards, xs, ys):
            s.step(frame, torch.cat(rx).contiguous(), torch.cat(ry).contiguous())
        self.t += 1

    def run(self, frames):
        for t in range(frames.shape[0]):
            self.step(frames[t])

    def estimates(self):
        """(frames stepped, 2) estimates; combines the last frame's statistics if needed."""
        import numpy as np
        if len(self.est) < self.t:
            self._combine()
        return np.array(self.est[:self.t])
