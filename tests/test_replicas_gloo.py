"""The bench's multi-rank path, on the CPU: two gloo ranks.

The solve does not shard (one solve is one GPU's work), so `bench.py --gpus N`
under torchrun runs N independent replicas with no data-path collective: a
barrier around the timed region, the slowest rank's time (max over ranks) and
a whole-job value of N x DOFs x steps over that time.  These tests run the
same host code (GpuContext.barrier / max_over_ranks, Workload.summary,
run_reference's rank filter) on two gloo ranks with CPU tensors; nothing here
touches a GPU.
"""
import os
import socket

import pytest


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank: int, world: int, port: int, out_dir: str):
    import torch
    import torch.distributed as dist

    import bench

    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        ctx = object.__new__(bench.GpuContext)  # the host side only: no device, no NCCL
        ctx.torch, ctx.dist, ctx.world, ctx.rank, ctx.local = torch, dist, world, rank, rank
        ctx.dev = torch.device("cpu")
        ctx.barrier()
        steps = 4
        # rank r was 100 + 50 r ms in all over its timed steps; the line uses the slowest
        local = {"fp32": 100.0 + 50.0 * rank, "fp64": 300.0 - 20.0 * rank}
        tot = {lab: ctx.max_over_ranks(v) for lab, v in local.items()}
        wl = object.__new__(bench.Workload)
        wl.ctx, wl.free_dofs = ctx, 1000
        info = (5, 5, 1e-9, 1.0, 2.0)  # iterations, total, residual, ms, compliance
        out = {lab: {"tot": t, "phases": {}, "infos": [info] * steps, "solve_ms": [1.0] * steps,
                     "ms": [t / steps] * steps} for lab, t in tot.items()}
        sm = wl.summary(out, ("fp32",), steps)
        with open(os.path.join(out_dir, f"rank{rank}.txt"), "w") as f:
            f.write(repr((tot["fp32"], tot["fp64"], sm["value"], sm["fp64_value"], sm["ms_per_step"])))
        # the reference arm: only rank 0 works and prints; the others return at once
        if rank != 0:
            bench.run_reference(None)
        ctx.barrier()
    finally:
        dist.destroy_process_group()


def test_two_gloo_replicas_take_the_slowest_rank(tmp_path):
    mp = pytest.importorskip("torch.multiprocessing")
    port = _free_port()
    mp.start_processes(_rank_main, args=(2, port, str(tmp_path)), nprocs=2, join=True, start_method="spawn")
    got = [eval(open(tmp_path / f"rank{r}.txt").read()) for r in range(2)]
    assert got[0] == got[1]  # every rank reports the same aggregate
    t32, t64, value, v64, ms = got[0]
    assert (t32, t64) == (150.0, 300.0)  # max over ranks
    assert value == pytest.approx(2 * 1000 * 4 / 0.150)  # all ranks' DOFs over the slowest time
    assert v64 == pytest.approx(2 * 1000 * 4 / 0.300)
    assert ms == pytest.approx(150.0 / 4)
