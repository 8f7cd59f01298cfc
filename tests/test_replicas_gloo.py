"""Replicas-only multi-GPU accounting of bench.py, exercised on CPU with two
gloo ranks: the job time is the slowest rank's and the rate counts every
rank's queries."""
import importlib.util
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _bench():
    spec = importlib.util.spec_from_file_location("bench_mod", os.path.join(ROOT, "bench.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    b = _bench()
    ws, r, local = b.dist_env()
    assert (ws, r, local) == (world, rank, rank)
    elapsed = 100.0 + 50.0 * rank            # rank 1 is the slower replica
    dist.barrier()
    job = b.replica_elapsed_ms(dist, elapsed)
    out[rank] = (job, b.replica_throughput(ws, 1024, job))
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_replicas_take_the_slowest_time():
    world = 2
    port = _free_port()
    ctx = mp.get_context("spawn")
    manager = ctx.Manager()
    out = manager.dict()
    procs = [ctx.Process(target=_rank, args=(r, world, port, out)) for r in range(world)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    for r in range(world):
        job, rate = out[r]
        assert job == 150.0
        assert rate == pytest.approx(2 * 1024 / 0.150)


def test_single_process_needs_no_collective():
    b = _bench()
    assert b.replica_elapsed_ms(None, 42.0) == 42.0
    assert b.replica_throughput(1, 10, 1000.0) == pytest.approx(10.0)
