"""Parity at the full terrain workload (2,313,248 triangles, 4-wide BVH,
1920x1080 primary rays, AO rays from their hits) in the launch configuration
bench.py times (128-thread blocks, 2^18-entry 2-way table, precision 6,
two-phase updates).

The oracle traces the whole primary batch (plain and HRPP: every hit, every
counter and every table word compared); AO rays are checked on a random
sample the oracle traces one by one, and on all rays through the invariant
that HRPP returns exactly what plain traversal returns.
"""
import numpy as np
import pytest

import oracle as O
from gpu_util import any_prims, as_words, assert_same_hits, assert_same_stats, gpu_trace, hrpp_mod
from paper_1910_01304_gb300.scenes import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def full():
    H = hrpp_mod()
    s = W.terrain_scene()
    return H, s, H.Scene.from_workload(s)


def test_full_terrain_primary_and_ao(full):
    H, s, g = full
    assert s.n_tris == 2_313_248
    prim = s.primary_rays(frame=1)
    assert len(prim) == 1920 * 1080
    # primary rays, plain: whole batch against the oracle
    oh, ost = O.trace(s.tris, s.nodes, s.prim_index, s.root, prim, O.CLOSEST_HIT)
    gh, gst = gpu_trace(H, g, prim, O.CLOSEST_HIT)
    assert_same_hits(O.CLOSEST_HIT, gh, oh, "full primary plain")
    assert_same_stats(gst, ost, msg="full primary plain")
    # primary rays, HRPP over two frames: hits, counters and table words
    tab = H.Table(18, 2, 6)
    otab = O.Table(18, 2, 6, O.TWO_PHASE)
    for frame in (1, 2):
        rays = prim if frame == 1 else s.primary_rays(frame=2)
        o2, os2 = O.trace(s.tris, s.nodes, s.prim_index, s.root, rays, O.CLOSEST_HIT, otab)
        g2, gs2 = gpu_trace(H, g, rays, O.CLOSEST_HIT, tab)
        assert_same_hits(O.CLOSEST_HIT, g2, o2, f"full primary hrpp frame {frame}")
        assert_same_stats(gs2, os2, msg=f"full primary hrpp frame {frame}")
        assert np.array_equal(tab.export(), otab.words)
    assert gs2["positives"] > 0
    # AO rays from the oracle's primary hits
    ao, _ = W.secondary_ao(s, prim, oh["t"], oh["prim"], frame=1)
    assert len(ao) > 4_000_000
    ga_plain, _ = gpu_trace(H, g, ao, O.ANY_HIT)
    tab_a = H.Table(18, 2, 6)
    for _ in range(2):
        ga_hrpp, sa = gpu_trace(H, g, ao, O.ANY_HIT, tab_a)
        # HRPP == plain on every ray (occlusion bit)
        assert np.array_equal(any_prims(ga_plain) == O.NO_HIT, any_prims(ga_hrpp) == O.NO_HIT)
    rng = np.random.default_rng(0)
    idx = np.sort(rng.choice(len(ao), 60000, replace=False))
    oa, _ = O.trace(s.tris, s.nodes, s.prim_index, s.root, ao[idx], O.ANY_HIT)
    assert np.array_equal(any_prims(ga_plain)[idx], oa)
    # closest-hit AO check of t on the same sample: the GPU's prim ids and t
    gc, _ = gpu_trace(H, g, ao[idx], O.CLOSEST_HIT)
    oc, _ = O.trace(s.tris, s.nodes, s.prim_index, s.root, ao[idx], O.CLOSEST_HIT)
    assert np.array_equal(as_words(gc), as_words(oc))


def test_full_batched_workload_sampled():
    """The 64-scene uneven batch at full size in one graph-replayed launch:
    every item checked against the oracle on a random sample of its rays."""
    import torch
    H = hrpp_mod()
    rng = np.random.default_rng(1)
    items, data = [], []
    for s, rays in W.batched_workload(n_scenes=64, seed=3):
        g = H.Scene.from_workload(s)
        d = torch.from_numpy(rays).cuda()
        items.append((g, H.Table(16, 2, 6), d, H.HRPP_CLOSEST_HIT))
        data.append((s, rays))
    batch = H.Batch(items)
    for _ in range(2):
        batch.run()
    torch.cuda.synchronize()
    for k, (s, rays) in enumerate(data):
        idx = np.sort(rng.choice(len(rays), min(len(rays), 300), replace=False))
        oh, _ = O.trace(s.tris, s.nodes, s.prim_index, s.root, rays[idx], O.CLOSEST_HIT)
        gh = batch.hits[k].cpu().numpy()[idx]
        assert np.array_equal(as_words(gh), as_words(oh)), f"item {k}"
