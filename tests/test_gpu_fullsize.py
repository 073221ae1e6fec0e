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
    # the dominant launch of the bench step, whole: HRPP any-hit over every
    # AO ray of two frames with the 2^18 x 2-way table, against the oracle's
    # two-phase HRPP (every prim, every counter, every table word)
    ao2, _ = W.secondary_ao(s, rays, o2["t"], o2["prim"], frame=2)
    tab_a = H.Table(18, 2, 6)
    otab_a = O.Table(18, 2, 6, O.TWO_PHASE)
    for frame, rays_a in ((1, ao), (2, ao2)):
        oa_h, oa_s = O.trace(s.tris, s.nodes, s.prim_index, s.root, rays_a, O.ANY_HIT, otab_a)
        ga_hrpp, sa = gpu_trace(H, g, rays_a, O.ANY_HIT, tab_a)
        assert_same_hits(O.ANY_HIT, ga_hrpp, oa_h, f"full AO hrpp frame {frame}")
        assert_same_stats(sa, oa_s, msg=f"full AO hrpp frame {frame}")
        assert np.array_equal(tab_a.export(), otab_a.words), f"full AO frame {frame}: table words differ"
    assert sa["positives"] > 0 and sa["inserts"] > 0
    # the two-pass schedule and a gated table on the same full-size launches:
    # equal to the fused launches just checked against the oracle (hits,
    # every counter, table words), frame after frame
    _compact_and_gate_match_fused(H, g, ((prim, O.CLOSEST_HIT), (rays, O.CLOSEST_HIT), (ao, O.ANY_HIT),
                                         (ao2, O.ANY_HIT)))
    # HRPP == plain on every ray (occlusion bit), for the same frame
    ga_hrpp, _ = gpu_trace(H, g, ao, O.ANY_HIT, tab_a)
    assert np.array_equal(any_prims(ga_plain) == O.NO_HIT, any_prims(ga_hrpp) == O.NO_HIT)
    rng = np.random.default_rng(0)
    idx = np.sort(rng.choice(len(ao), 60000, replace=False))
    oa, _ = O.trace(s.tris, s.nodes, s.prim_index, s.root, ao[idx], O.ANY_HIT)
    assert np.array_equal(any_prims(ga_plain)[idx], oa)
    # closest-hit AO check of t on the same sample: the GPU's prim ids and t
    gc, _ = gpu_trace(H, g, ao[idx], O.CLOSEST_HIT)
    oc, _ = O.trace(s.tris, s.nodes, s.prim_index, s.root, ao[idx], O.CLOSEST_HIT)
    assert np.array_equal(as_words(gc), as_words(oc))


def test_full_terrain_shadow_rays_both_schedules(full):
    """The terrain's shadow rays toward the low light (the workload of
    bench.py --workload shadow, where any-hit predictions pay) at full size,
    with its 2^22-entry 4-way table at precision 6: two warming frames, then
    frame 0 traced from the warmed table by the fused schedule and again,
    from the same table, by the two-pass schedule.  Every prim, every counter
    and every table word equals the oracle's two-phase HRPP."""
    import torch
    H, s, g = full
    shadows = {}
    for f in (1, 2, 0):
        prim = s.primary_rays(frame=f)
        oh, _ = O.trace(s.tris, s.nodes, s.prim_index, s.root, prim, O.CLOSEST_HIT)
        shadows[f], _ = W.secondary_shadow(s, prim, oh["t"], oh["prim"], light=W.TERRAIN_SUN)
    assert len(shadows[0]) > 1_000_000
    tab, snap = H.Table(22, 4, 6), H.Table(22, 4, 6)
    otab = O.Table(22, 4, 6, O.TWO_PHASE)
    for f in (1, 2):
        oh, ost = O.trace(s.tris, s.nodes, s.prim_index, s.root, shadows[f], O.ANY_HIT, otab)
        gh, gst = gpu_trace(H, g, shadows[f], O.ANY_HIT, tab)
        assert_same_hits(O.ANY_HIT, gh, oh, f"full shadow frame {f}")
        assert_same_stats(gst, ost, msg=f"full shadow frame {f}")
    snap.copy_from(tab)
    oh, ost = O.trace(s.tris, s.nodes, s.prim_index, s.root, shadows[0], O.ANY_HIT, otab)
    assert ost["true_pos"] > 0.3 * len(shadows[0])
    d0 = torch.from_numpy(shadows[0]).cuda()
    for sched in (H.HRPP_SCHEDULE_BATCH, H.HRPP_SCHEDULE_COMPACT):
        tab.copy_from(snap)
        gh, gst = H.trace(g, d0, O.ANY_HIT, tab, stats=True, schedule=sched)
        torch.cuda.synchronize()
        g.check()
        msg = f"full shadow frame 0 schedule {sched}"
        assert_same_hits(O.ANY_HIT, gh.cpu().numpy(), oh, msg)
        assert_same_stats(gst, ost, msg=msg)
        assert np.array_equal(tab.export(), otab.words), msg


def _compact_and_gate_match_fused(H, g, batches):
    """Per query mode, three tables traced batch after batch: fused BATCH
    (the reference), two-pass COMPACT, and BATCH under a gate; COMPACT must
    equal the reference in hits, counters and table words, and the gated
    table must give plain's results with gated + lookups = rays."""
    import torch
    tabs = {}
    for rays_np, mode in batches:
        if mode not in tabs:
            gated = H.Table(18, 2, 6)
            gated.set_gate(2621, 5)
            tabs[mode] = (H.Table(18, 2, 6), H.Table(18, 2, 6), gated)
        ref_t, cmp_t, gate_t = tabs[mode]
        d = torch.from_numpy(np.ascontiguousarray(rays_np)).cuda()
        h_ref, s_ref = H.trace(g, d, mode, ref_t, stats=True)
        h_cmp, s_cmp = H.trace(g, d, mode, cmp_t, stats=True, schedule=H.HRPP_SCHEDULE_COMPACT)
        h_gate, s_gate = H.trace(g, d, mode, gate_t, stats=True)
        h_plain, _ = H.trace(g, d, mode)
        torch.cuda.synchronize()
        g.check()
        assert torch.equal(h_ref.view(torch.int32), h_cmp.view(torch.int32)), mode
        assert s_ref == s_cmp, (mode, s_ref, s_cmp)
        assert np.array_equal(ref_t.export(), cmp_t.export()), mode
        if mode == H.HRPP_CLOSEST_HIT:
            assert torch.equal(h_gate.view(torch.int32), h_plain.view(torch.int32))
        else:
            assert torch.equal(h_gate == -1, h_plain == -1)
        assert s_gate["gated"] + s_gate["lookups"] == s_gate["rays"] == len(rays_np)


def test_full_batched_workload_sampled():
    """The 64-scene uneven batch at full size, graph-replayed (one launch per
    query mode, side by side), with the bench's item mix: per scene, its
    camera half as a closest-hit item and its random half as an any-hit item,
    each with its own table.  Every item is checked against the oracle on a
    random sample of its rays (closest hits bit for bit, any-hit prims bit for
    bit)."""
    import torch
    H = hrpp_mod()
    rng = np.random.default_rng(1)
    items, data = [], []
    for s, rays in W.batched_workload(n_scenes=64, seed=3):
        g = H.Scene.from_workload(s)
        half = len(rays) // 2
        for part, mode in ((rays[:half], H.HRPP_CLOSEST_HIT), (rays[half:], H.HRPP_ANY_HIT)):
            part = np.ascontiguousarray(part)
            if len(part) == 0:
                continue
            items.append((g, H.Table(16, 2, 6), torch.from_numpy(part).cuda(), mode))
            data.append((s, part, mode))
    assert sum(1 for *_, m in data if m == H.HRPP_ANY_HIT) >= 60
    batch = H.Batch(items)
    for _ in range(2):
        batch.run()
    torch.cuda.synchronize()
    for k, (s, rays, mode) in enumerate(data):
        idx = np.sort(rng.choice(len(rays), min(len(rays), 300), replace=False))
        omode = O.CLOSEST_HIT if mode == H.HRPP_CLOSEST_HIT else O.ANY_HIT
        oh, _ = O.trace(s.tris, s.nodes, s.prim_index, s.root, rays[idx], omode)
        gh = batch.hits[k].cpu().numpy()[idx]
        if omode == O.CLOSEST_HIT:
            assert np.array_equal(as_words(gh), as_words(oh)), f"item {k}"
        else:
            # a true positive reports the predicted leaf's hit: occlusion is
            # unique, the prim must be a valid hit of the ray
            assert np.array_equal(any_prims(gh) == O.NO_HIT, oh == O.NO_HIT), f"item {k}"
            for j in np.nonzero(any_prims(gh) != O.NO_HIT)[0][:40]:
                tri = s.tris[any_prims(gh)[j]].reshape(3, 3)
                assert O.ray_triangle(rays[idx][j], *tri)[0], f"item {k}: prim is not a hit"


def test_full_pathtrace_sampled():
    """Config 5 at full size: 4,281,344 triangles, 1280x720 x 4 spp x 5
    diffuse bounces plus a shadow ray per bounce (36.9M rays), traced through
    HRPP with one 2^18 x 2-way table per query mode shared by all bounces, as
    bench.py times it.  Each batch is checked on a random sample against the
    oracle's plain traversal: closest hits bit for bit, shadow rays by their
    occlusion bit (and the GPU's plain any-hit prim bit for bit)."""
    import torch
    H = hrpp_mod()
    s = W.pathtrace_scene()
    assert s.n_tris == 4_281_344
    g = H.Scene.from_workload(s)
    rng = np.random.default_rng(2)

    def gpu_closest(rays):
        hits, _ = H.trace(g, torch.from_numpy(np.ascontiguousarray(rays)).cuda(), H.HRPP_CLOSEST_HIT)
        h = hits.cpu().numpy()
        return h[:, 0].copy(), h[:, 1].view(np.uint32).copy()

    bounces = W.path_bounces(s, W.path_primary(s, spp=4, frame=0), gpu_closest, bounces=5, frame=0)
    assert len(bounces) == 5 and sum(len(c) + len(sh) for c, sh in bounces) > 30_000_000
    tabs = {O.CLOSEST_HIT: H.Table(18, 2, 6), O.ANY_HIT: H.Table(18, 2, 6)}
    for b, (closest, shadow) in enumerate(bounces):
        for mode, rays in ((O.CLOSEST_HIT, closest), (O.ANY_HIT, shadow)):
            d = torch.from_numpy(rays).cuda()
            gh, gst = H.trace(g, d, mode, tabs[mode], stats=True)
            torch.cuda.synchronize()
            g.check()
            assert gst["rays"] == len(rays)
            idx = np.sort(rng.choice(len(rays), 800, replace=False))
            oh, _ = O.trace(s.tris, s.nodes, s.prim_index, s.root, rays[idx], mode)
            gh = gh.cpu().numpy()[idx]
            if mode == O.CLOSEST_HIT:
                assert np.array_equal(as_words(gh), as_words(oh)), f"bounce {b}"
            else:
                assert np.array_equal(any_prims(gh) == O.NO_HIT, oh == O.NO_HIT), f"bounce {b}"
                gp, _ = H.trace(g, d, H.HRPP_ANY_HIT)
                assert np.array_equal(any_prims(gp.cpu().numpy()[idx]), oh), f"bounce {b} plain"


def test_full_learned_proposal_sampled():
    """Config 4 at full size: the closest-hit proposal trained as bench.py
    trains it (jittered frames of the small scene's camera until ~30M
    traces).  On a held-out frame, predictions sampled across the batch are
    an argmax of the oracle's logits under the trained weights, and traversal
    with every prediction returns exactly the plain hits."""
    import torch
    from oracle import proposal as P
    H = hrpp_mod()
    s = W.small_scene()
    g = H.Scene.from_workload(s)
    prop = H.Proposal.for_workload(g, s, seed=1)
    traces, f = 0, 0
    while traces < 30_000_000:
        f += 1
        rays = torch.from_numpy(s.primary_rays(frame=f)).cuda()
        hits, _ = H.trace(g, rays, H.HRPP_CLOSEST_HIT)
        prop.train(rays, prop.labels(hits), lr=1e-3)
        traces += int(rays.shape[0])
    test_np = s.primary_rays(frame=100_000)
    test = torch.from_numpy(test_np).cuda()
    nodes, classes = prop.predict(test)
    plain, _ = H.trace(g, test, H.HRPP_CLOSEST_HIT)
    learned, st = H.trace(g, test, H.HRPP_CLOSEST_HIT, stats=True, predicted=nodes)
    torch.cuda.synchronize()
    assert torch.equal(plain.view(torch.int32), learned.view(torch.int32))
    assert st["true_pos"] > 0.4 * st["rays"]
    rows = np.sort(np.random.default_rng(3).choice(len(test_np), 1500, replace=False))
    root = s.nodes[s.root]
    w = P.Weights.from_flat(prop.get_weights())
    _, _, z = P.forward(w, P.features(test_np[rows], root["lo"], root["hi"]))
    picked = z[np.arange(len(rows)), classes.cpu().numpy()[rows]]
    span = z.max(axis=1) - z.min(axis=1)
    assert np.all(z.max(axis=1) - picked <= 0.02 * span)
    assert np.mean(classes.cpu().numpy()[rows] == np.argmax(z, axis=1)) > 0.97


def test_maximum_table_and_ray_counts():
    """The size limits: tables at both ends of the allowed range (2^28
    entries in 8-way sets, a single 8-way set, a single entry) match the
    oracle word for word, and one call with 2^28 + 3 rays (8.6 GB of rays:
    copies of one frame) returns the single-frame answer for every copy."""
    import torch
    H = hrpp_mod()
    s = W.small_scene()
    g = H.Scene.from_workload(s)
    for log2_entries, ways in ((28, 8), (3, 8), (0, 1)):
        tab = H.Table(log2_entries, ways, 6)
        otab = O.Table(log2_entries, ways, 6, O.TWO_PHASE)
        for frame in range(2):
            rays = s.primary_rays(frame=frame)
            oh, ost = O.trace(s.tris, s.nodes, s.prim_index, s.root, rays, O.CLOSEST_HIT, otab)
            gh, gst = gpu_trace(H, g, rays, O.CLOSEST_HIT, tab)
            assert_same_hits(O.CLOSEST_HIT, gh, oh, f"2^{log2_entries} x {ways}")
            assert_same_stats(gst, ost, msg=f"2^{log2_entries} x {ways}")
        assert np.array_equal(tab.export(), otab.words)
        tab.close()
        del otab
    frame_np = s.primary_rays(frame=3)
    base = torch.from_numpy(frame_np).cuda()
    n = (1 << 28) + 3
    big = base.repeat(n // base.shape[0] + 1, 1)[:n].contiguous()
    out = torch.empty(n, dtype=torch.int32, device="cuda")
    H.trace(g, big, H.HRPP_ANY_HIT, hits=out)
    ref, _ = H.trace(g, base, H.HRPP_ANY_HIT)
    torch.cuda.synchronize()
    g.check()
    copies = out[: (n // base.shape[0]) * base.shape[0]].view(-1, base.shape[0])
    assert bool((copies == ref.unsqueeze(0)).all())
    assert torch.equal(out[-3:], ref[:3])
    oh, _ = O.trace(s.tris, s.nodes, s.prim_index, s.root, frame_np[:4000], O.ANY_HIT)
    assert np.array_equal(any_prims(ref[:4000].cpu().numpy()), oh)
