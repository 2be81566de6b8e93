"""The N>1 path on CPU: two gloo ranks, distinct seeded batches, max-over-ranks timing."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, out):
    import sys
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    from paper_2402_18858_gb300 import sharding, workload as w
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    m = w.make_mechanism("h2_9", 0)
    seed = sharding.rank_state_seed(101, rank)
    st = w.make_states(m, 64, seed)
    # the slowest rank's time is what the job is charged
    tmax = sharding.max_over_ranks(0.5 + rank)
    dist.barrier()
    out[rank] = (seed, float(st.T[0]), tmax, sharding.job_throughput(64, world, tmax))
    dist.destroy_process_group()


def test_two_rank_weak_scaling_layout():
    world = 2
    mgr = mp.Manager()
    out = mgr.dict()
    mp.spawn(_worker, args=(world, _free_port(), out), nprocs=world, join=True)
    (s0, t0, m0, v0), (s1, t1, m1, v1) = out[0], out[1]
    assert s0 != s1 and t0 != t1          # independent batches
    assert m0 == m1 == 1.5                # max over ranks
    assert v0 == v1 == 64 * 2 / 1.5
