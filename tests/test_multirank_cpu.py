"""The N > 1 path of bench.py on CPU ranks (gloo, world size 2): the solve does not
shard (one independent replica per GPU), so what the ranks share is the timing
contract -- a barrier, the maximum of the ranks' times, and the whole-job value
(units of all ranks over the slowest rank's time) -- and the reference arm, which
only rank 0 runs."""
import os
import socket
import sys

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, ws, port, results):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(ws),
                      LOCAL_RANK=str(rank))
    sys.path.insert(0, ROOT)
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    try:
        assert bench.dist_env() == (ws, rank, rank)

        def reduce_max(x):
            t = torch.tensor([x], dtype=torch.float64)
            dist.all_reduce(t, op=dist.ReduceOp.MAX)
            return float(t.item())

        dist.barrier()
        # rank r took 1 + r seconds for 3 steps of 100 units
        value, t = bench.aggregate_over_ranks(1.0 + rank, 100.0, 3, ws, reduce_max)
        results[rank] = (value, t)
        # the reference arm: ranks other than 0 return without work or output
        if rank != 0:
            class A:  # only the fields run_reference reads before returning
                pass
            assert bench.run_reference(A()) == 0
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_take_the_slowest_time():
    ws = 2
    with mp.Manager() as m:
        results = m.dict()
        mp.spawn(_worker, args=(ws, _free_port(), results), nprocs=ws, join=True)
        res = dict(results)
    assert set(res) == {0, 1}
    for rank in range(ws):
        value, t = res[rank]
        assert t == 2.0  # the maximum over the ranks
        assert value == pytest.approx(100.0 * 3 * ws / 2.0)


def test_single_rank_needs_no_process_group():
    sys.path.insert(0, ROOT)
    import bench
    value, t = bench.aggregate_over_ranks(0.5, 10.0, 4, 1)
    assert t == 0.5 and value == pytest.approx(80.0)
