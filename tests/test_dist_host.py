"""The multi-GPU path of bench.py is replicas only: every rank runs its own
reconstruction and rank 0 reports the slowest rank's time.  Its host-side
logic (barrier, max over ranks, summed throughput) is checked here with two
gloo ranks on the CPU."""
import os
import socket

import pytest
import torch.distributed as dist
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    import bench

    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        bench.barrier(world)
        slowest = bench.max_over_ranks(10.0 * (rank + 1), world)
        out[rank] = slowest
    finally:
        dist.destroy_process_group()


def test_max_over_ranks_gloo_world2():
    ctx = mp.get_context("spawn")
    with ctx.Manager() as m:
        out = m.dict()
        port = _free_port()
        procs = [ctx.Process(target=_worker, args=(r, 2, port, out)) for r in range(2)]
        for p in procs:
            p.start()
        for p in procs:
            p.join(timeout=120)
            assert p.exitcode == 0
        assert dict(out) == {0: 20.0, 1: 20.0}


def test_reference_arm_other_ranks_exit_quietly(monkeypatch, capsys):
    import bench

    monkeypatch.setenv("RANK", "1")
    monkeypatch.setenv("WORLD_SIZE", "1")
    args = type("A", (), dict(impl="reference", gpus=2, steps=1, warmup=0, workload="cfg1",
                              precision="fp32-kahan", ref_seconds=0.1))()
    assert bench.run_reference(args) == 0
    assert capsys.readouterr().out == ""
