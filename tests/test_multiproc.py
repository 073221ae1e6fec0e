"""The multi-rank host logic of bench.py on CPU: two gloo ranks, each tracing
its own frames (weak scaling, no data-path collective), combined by the
max-over-ranks time and the sum-over-ranks ray count.  The oracle stands in
for the GPU here."""
import os
import socket

import numpy as np
import pytest
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out):
    import hashlib

    import torch
    import torch.distributed as dist

    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        import bench
        import oracle as O
        from paper_1910_01304_gb300.scenes import workloads as W
        s = W.small_scene(res=64)
        rays = np.concatenate([s.primary_rays(frame=bench.frame_index(f, rank)) for f in range(2)])
        hits, st = O.trace(s.tris, s.nodes, s.prim_index, s.root, rays, O.CLOSEST_HIT)
        digest = int(hashlib.sha1(rays.tobytes()).hexdigest()[:12], 16)
        got = [None] * world
        dist.all_gather_object(got, digest)
        total = bench.reduce_sum(float(len(rays)), dist, "cpu")
        slowest = bench.reduce_max(float(10 * (rank + 1)), dist, "cpu")
        hits_all = bench.reduce_sum(float(st["hits"]), dist, "cpu")
        out[rank] = dict(distinct=len(set(got)) == world, total=total, slowest=slowest, n=len(rays),
                         hits=hits_all, value=bench.job_mrays_per_s(total, slowest))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_weak_scaling():
    world = 2
    mgr = mp.get_context("spawn").Manager()
    out = mgr.dict()
    ctx = mp.get_context("spawn")
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, world, port, out)) for r in range(world)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    r0, r1 = out[0], out[1]
    assert r0["distinct"] and r1["distinct"]                  # each rank traced its own frames
    assert r0["total"] == r1["total"] == 2 * r0["n"]          # weak scaling: work grows with ranks
    assert r0["slowest"] == r1["slowest"] == 20.0             # the job takes its slowest rank's time
    assert r0["value"] == pytest.approx(2 * r0["n"] / 20e-3 / 1e6)
    assert r0["hits"] == r1["hits"] > 0


def test_single_process_reductions_are_identity():
    import bench
    assert bench.reduce_max(3.5, None, "cpu") == 3.5
    assert bench.reduce_sum(7.0, None, "cpu") == 7.0
    assert bench.frame_index(0, 0) != bench.frame_index(0, 1)
