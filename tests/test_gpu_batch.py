"""Batched traces (one persistent launch over many scenes and uneven ray
batches, replayed from a CUDA graph) against the oracle, item by item."""
import ctypes

import numpy as np
import pytest

import oracle as O
from gpu_util import assert_same_hits, assert_same_stats, hrpp_mod
from paper_1910_01304_gb300.scenes import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def H():
    return hrpp_mod()


def _table_spec(k):
    # None, then a rotation of table shapes, Go Up Levels and update modes
    specs = [None, (12, 1, 6, 0, 0), (13, 2, 5, 0, 0), (12, 4, 6, 1, 0), (14, 2, 6, 0, 1), (12, 2, 6, 2, 0)]
    return specs[k % len(specs)]


@pytest.mark.parametrize("width", [4, 2])
def test_batch_matches_oracle_per_item(H, width):
    import torch
    items = list(W.batched_workload(n_scenes=10, tris_range=(300, 30_000), rays_range=(40, 20_000), seed=5,
                                    width=width))
    scenes, tables, otables, rays_d, modes = [], [], [], [], []
    for k, (s, rays) in enumerate(items):
        g = H.Scene.from_workload(s)
        spec = _table_spec(k)
        mode = H.HRPP_CLOSEST_HIT if k % 2 == 0 else H.HRPP_ANY_HIT
        t = ot = None
        if spec is not None:
            log2e, ways, prec, go_up, online = spec
            t = H.Table(log2e, ways, prec, H.HRPP_UPDATE_ONLINE if online else H.HRPP_UPDATE_TWO_PHASE, go_up=go_up)
            if not online:
                ot = O.Table(log2e, ways, prec, O.TWO_PHASE, go_up=go_up)
        scenes.append(g)
        tables.append(t)
        otables.append(ot)
        rays_d.append(torch.from_numpy(rays).cuda())
        modes.append(mode)
    batch = H.Batch([(g, t, r, m) for g, t, r, m in zip(scenes, tables, rays_d, modes)], stats=True)
    for rep in range(2):
        batch.run()
        torch.cuda.synchronize()
        for k, (s, rays) in enumerate(items):
            online = _table_spec(k) is not None and _table_spec(k)[4] == 1
            gh = batch.hits[k].cpu().numpy()
            gst = batch.stats(k)
            if online:
                ph, _ = O.trace(s.tris, s.nodes, s.prim_index, s.root, rays, modes[k])
                if modes[k] == O.CLOSEST_HIT:
                    assert_same_hits(modes[k], gh, ph, f"item {k} online")
                else:
                    assert np.array_equal(gh.view(np.uint32) == O.NO_HIT, ph == O.NO_HIT)
                continue
            oh, ost = O.trace(s.tris, s.nodes, s.prim_index, s.root, rays, modes[k], otables[k])
            assert_same_hits(modes[k], gh, oh, f"run {rep} item {k}")
            assert_same_stats(gst, ost, msg=f"run {rep} item {k}")
            if tables[k] is not None:
                assert np.array_equal(tables[k].export(), otables[k].words), f"item {k} table"


@pytest.mark.parametrize("modes", ["closest", "any", "mixed"])
def test_batch_equals_single_calls(H, modes):
    """Batches of one query mode (one launch) and of both (two launches side
    by side) give exactly the hits of one hrpp_trace per item."""
    import torch
    items = list(W.batched_workload(n_scenes=4, tris_range=(1000, 8000), rays_range=(500, 3000), seed=8))
    gs = [H.Scene.from_workload(s) for s, _ in items]
    rs = [torch.from_numpy(r).cuda() for _, r in items]
    pick = {"closest": lambda k: H.HRPP_CLOSEST_HIT, "any": lambda k: H.HRPP_ANY_HIT,
            "mixed": lambda k: H.HRPP_ANY_HIT if k % 2 else H.HRPP_CLOSEST_HIT}[modes]
    ms = [pick(k) for k in range(len(items))]
    batch = H.Batch([(g, None, r, m) for g, r, m in zip(gs, rs, ms)])
    for _ in range(2):
        batch.run()
        for k in range(len(items)):
            single, _ = H.trace(gs[k], rs[k], ms[k])
            torch.cuda.synchronize()
            assert torch.equal(single.view(torch.int32), batch.hits[k].view(torch.int32)), (modes, k)


def test_batch_rejects_mixed_widths_and_shared_tables(H):
    import torch
    a, ra = W.batched_item("soup", 500, 64, 1, width=4)
    b, rb = W.batched_item("soup", 500, 64, 2, width=2)
    ga, gb = H.Scene.from_workload(a), H.Scene.from_workload(b)
    da, db = torch.from_numpy(ra).cuda(), torch.from_numpy(rb).cuda()
    with pytest.raises(H.HrppError) as e:
        H.Batch([(ga, None, da, H.HRPP_ANY_HIT), (gb, None, db, H.HRPP_ANY_HIT)])
    assert e.value.status == H.HRPP_ERR_INVALID_ARG
    c, rc = W.batched_item("soup", 500, 64, 3, width=4)
    gc = H.Scene.from_workload(c)
    t = H.Table(10, 1, 6)
    with pytest.raises(H.HrppError):
        H.Batch([(ga, t, da, H.HRPP_ANY_HIT), (gc, t, torch.from_numpy(rc).cuda(), H.HRPP_ANY_HIT)])
