"""N > 1 replica path on CPU: two gloo ranks, each with its own replica
seed and elapsed time; whole-job throughput = all ranks' units / slowest
rank's time (the aggregation bench.py uses under torchrun)."""
import os
import socket

import pytest
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, q):
    os.environ.update(RANK=str(rank), WORLD_SIZE=str(world), LOCAL_RANK=str(rank),
                      MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    from paper_1412_8502_b300 import replicas
    replicas.init("gloo")
    r, w, lr = replicas.dist_env()
    replicas.barrier()
    ms = [100.0, 250.0][r]                 # rank 1 is the slowest
    units = 409600 * 10                     # nucleon-steps of this rank's replica
    rate = replicas.whole_job_rate(units, ms)
    q.put((r, w, lr, rate, replicas.max_over_ranks(ms), replicas.replica_seed(3, r)))
    replicas.finalize()


@pytest.mark.parametrize("world", [2])
def test_two_gloo_ranks_aggregate(world):
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    ps = [ctx.Process(target=_worker, args=(r, world, port, q)) for r in range(world)]
    for p in ps:
        p.start()
    out = [q.get(timeout=120) for _ in range(world)]
    for p in ps:
        p.join(timeout=60)
        assert p.exitcode == 0
    out.sort()
    for r, (rank, w, lr, rate, mx, seed) in enumerate(out):
        assert (rank, w, lr) == (r, world, r)
        assert mx == 250.0
        assert rate == pytest.approx(world * 409600 * 10 / 0.250)
    assert out[0][5] != out[1][5]


def test_single_rank_is_identity():
    from paper_1412_8502_b300 import replicas
    assert replicas.max_over_ranks(3.5) == 3.5
    assert replicas.whole_job_rate(1000.0, 500.0) == 2000.0
