"""The multi-GPU form is replicas only: one independent tracker per rank, no collective
on the data path, and the whole-job throughput is the units of all ranks over the
slowest rank's time.  These world-size-2 runs exercise that aggregation on CPU (gloo)."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, ws, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(ws))
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    import importlib.util
    spec = importlib.util.spec_from_file_location("bench", os.path.join(os.path.dirname(__file__), "..", "bench.py"))
    bench = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(bench)
    # rank r took 100 + 50 r ms for 1e6 units
    value, ms = bench.replica_value(1.0e6, 100.0 + 50.0 * rank)
    q.put((rank, value, ms))
    dist.barrier()
    dist.destroy_process_group()


@pytest.mark.parametrize("ws", [2])
def test_replica_value_is_all_units_over_slowest_rank(ws):
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, ws, port, q)) for r in range(ws)]
    for p in procs:
        p.start()
    out = [q.get(timeout=120) for _ in range(ws)]
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    slowest = 100.0 + 50.0 * (ws - 1)
    for rank, value, ms in out:
        assert ms == slowest
        assert value == pytest.approx(1.0e6 * ws / (slowest * 1e-3))


def test_replica_value_single_process():
    import importlib.util
    spec = importlib.util.spec_from_file_location("bench", os.path.join(os.path.dirname(__file__), "..", "bench.py"))
    bench = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(bench)
    value, ms = bench.replica_value(5.0e5, 250.0)
    assert ms == 250.0 and value == pytest.approx(2.0e6)
