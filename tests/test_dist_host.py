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


def _replica_worker(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    import time

    import bench
    import oracle.oracle as o
    from paper_1901_06503_gb300.inputs import add_noise, config

    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        # each rank reconstructs its own problem (its own seed): replicas
        w = config(1, n=12, seed=40 + rank)
        g = add_noise(o.forward(w.c, w.h, w.T, w.n_angles), w.noise, w.noise_rel)
        bench.barrier(world)
        t0 = time.perf_counter()
        h, _, k = o.fb(w.c, g, w.T, w.lam, 0.05, 2)
        ms = 1e3 * (time.perf_counter() - t0)
        nt, _ = o.time_steps(w.n, w.T, w.cfl, float(w.c.max()))
        units = 2.0 * nt * w.n ** 3  # voxel-steps of one FB iteration
        value, slowest = bench.replica_throughput(world, k, units, ms)
        out[rank] = dict(value=value, slowest=slowest, ms=ms, units=units, k=k,
                         h_norm=float((h * h).sum()) ** 0.5)
    finally:
        dist.destroy_process_group()


def test_two_replica_reconstructions_gloo_world2():
    """Two gloo ranks each run their own (CPU oracle) reconstruction; the
    reported throughput is both ranks' voxel-steps over the slowest rank's
    time, the same on every rank, and each rank's result is that of its own
    problem run alone."""
    import numpy as np

    import oracle.oracle as o
    from paper_1901_06503_gb300.inputs import add_noise, config

    ctx = mp.get_context("spawn")
    with ctx.Manager() as m:
        out = m.dict()
        port = _free_port()
        procs = [ctx.Process(target=_replica_worker, args=(r, 2, port, out)) for r in range(2)]
        for p in procs:
            p.start()
        for p in procs:
            p.join(timeout=300)
            assert p.exitcode == 0
        res = dict(out)
    slowest = max(res[0]["ms"], res[1]["ms"])
    want = (res[0]["k"] * res[0]["units"] + res[1]["k"] * res[1]["units"]) / (slowest / 1e3)
    for r in (0, 1):
        assert res[r]["slowest"] == slowest
        assert abs(res[r]["value"] - want) <= 1e-12 * want
        w = config(1, n=12, seed=40 + r)
        g = add_noise(o.forward(w.c, w.h, w.T, w.n_angles), w.noise, w.noise_rel)
        h, _, _ = o.fb(w.c, g, w.T, w.lam, 0.05, 2)
        assert abs(float(np.linalg.norm(h)) - res[r]["h_norm"]) <= 1e-12 * res[r]["h_norm"]


def test_reference_arm_other_ranks_exit_quietly(monkeypatch, capsys):
    import bench

    monkeypatch.setenv("RANK", "1")
    monkeypatch.setenv("WORLD_SIZE", "1")
    args = type("A", (), dict(impl="reference", gpus=2, steps=1, warmup=0, workload="cfg1",
                              precision="fp32-kahan", ref_seconds=0.1))()
    assert bench.run_reference(args) == 0
    assert capsys.readouterr().out == ""
