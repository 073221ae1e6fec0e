"""GPU parity: the CUDA path (through the C ABI) against the oracle.

Traversal arithmetic is the same IEEE-754 sequence on both sides, so hits
(t, prim, u, v bit patterns), any-hit prims, every statistics counter and,
in two-phase mode, the table words must be identical.  The acceptance
tolerances (prim ids exact except where the two nearest hits lie within 1e-6
relative t, t within 1e-5 relative) apply where the GPU is compared with brute
force instead of the oracle's traversal.
"""
import numpy as np
import pytest

import oracle as O
from gpu_util import (STAT_KEYS, any_prims, as_words, assert_same_hits, assert_same_stats, gpu_trace,
                      hrpp_mod)
from paper_1910_01304_gb300 import scenes as S
from paper_1910_01304_gb300.scenes import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def H():
    return hrpp_mod()


@pytest.fixture(scope="module")
def small_pair(H):
    s2, s4 = W.small_scene(width=2), W.small_scene(width=4)
    return (s2, H.Scene.from_workload(s2)), (s4, H.Scene.from_workload(s4))


def _oracle(s, rays, mode, table=None):
    return O.trace(s.tris, s.nodes, s.prim_index, s.root, rays, mode, table)


@pytest.mark.parametrize("width_idx", [0, 1])
@pytest.mark.parametrize("mode", [O.CLOSEST_HIT, O.ANY_HIT])
def test_plain_small_scene(H, small_pair, width_idx, mode):
    s, g = small_pair[width_idx]
    rays = s.primary_rays(frame=1)
    if mode == O.ANY_HIT:
        h, _ = _oracle(s, rays, O.CLOSEST_HIT)
        rays, _ = W.secondary_shadow(s, rays, h["t"], h["prim"])
    oh, ost = _oracle(s, rays, mode)
    gh, gst = gpu_trace(H, g, rays, mode)
    assert_same_hits(mode, gh, oh, "plain")
    assert_same_stats(gst, ost)


@pytest.mark.parametrize("ways", [1, 2, 4])
@pytest.mark.parametrize("width_idx", [0, 1])
def test_hrpp_small_scene_frames(H, small_pair, ways, width_idx):
    """Four jittered frames of primary (closest) and shadow (any) rays through
    one table per mode: hits, counters and table words match every frame."""
    s, g = small_pair[width_idx]
    tabs = {m: H.Table(12, ways, 6) for m in (O.CLOSEST_HIT, O.ANY_HIT)}
    otabs = {m: O.Table(12, ways, 6, O.TWO_PHASE) for m in (O.CLOSEST_HIT, O.ANY_HIT)}
    for frame in range(4):
        prim = s.primary_rays(frame=frame)
        ph, _ = _oracle(s, prim, O.CLOSEST_HIT)
        shadow, _ = W.secondary_shadow(s, prim, ph["t"], ph["prim"])
        for mode, rays in ((O.CLOSEST_HIT, prim), (O.ANY_HIT, shadow)):
            oh, ost = _oracle(s, rays, mode, otabs[mode])
            gh, gst = gpu_trace(H, g, rays, mode, tabs[mode])
            assert_same_hits(mode, gh, oh, f"frame {frame} mode {mode}")
            assert_same_stats(gst, ost, msg=f"frame {frame} mode {mode}")
            assert np.array_equal(tabs[mode].export(), otabs[mode].words), f"table words frame {frame}"
    # later frames predict something
    assert gst["positives"] > 0


@pytest.mark.parametrize("width", [2, 4])
def test_tiny_scenes_vs_brute_force(H, width):
    """Random soups, coplanar grids and degenerate triangles: GPU plain and HRPP
    against brute force under the acceptance tolerances (see the module
    docstring)."""
    rng = np.random.default_rng(width)
    for seed in range(40):
        n = int(rng.integers(1, 200))
        tris = S.soup(n, seed, -1, 1, 0.6) if seed % 2 else S.quad_grid(7, 5, -1, 1, -1, 1, 0.0)
        if seed % 5 == 0:
            tris[: max(1, n // 4), 3:6] = tris[: max(1, n // 4), 0:3]
        nodes, prim, root = S.build_bvh(tris, width=width)
        g = H.Scene(tris, nodes, prim, root, width)
        o = rng.uniform(-2, 2, (257, 3))
        d = rng.uniform(-1, 1, (257, 3)) - o
        d /= np.linalg.norm(d, axis=1, keepdims=True)
        rays = np.zeros((257, 8), np.float32)
        rays[:, :3], rays[:, 4:7], rays[:, 7] = o, d, np.inf
        rays[::9, 4:7] = [0, -1, 0]
        bc, tie = O.brute(rays, tris, O.CLOSEST_HIT)
        ba, _ = O.brute(rays, tris, O.ANY_HIT)
        tab_c, tab_a = H.Table(8, 2, 3), H.Table(8, 2, 3)
        for rep in range(2):
            for table in (None, "t"):
                gc, _ = gpu_trace(H, g, rays, O.CLOSEST_HIT, tab_c if table else None, stats=False)
                ga, _ = gpu_trace(H, g, rays, O.ANY_HIT, tab_a if table else None, stats=False)
                gw, bw = as_words(gc), as_words(bc)
                ok = ~tie
                assert np.array_equal(gw[ok, 1], bw[ok, 1]), seed           # prim ids
                tg, tb = gc[ok, 0], bc["t"][ok]
                fin = np.isfinite(tb)
                assert np.array_equal(np.isfinite(tg), fin)
                assert np.all(np.abs(tg[fin] - tb[fin]) <= 1e-5 * np.abs(tb[fin]))
                assert np.array_equal(any_prims(ga) == O.NO_HIT, ba == O.NO_HIT), seed


def test_edge_cases_ragged_and_degenerate(H, small_pair):
    s, g = small_pair[0]
    base = s.primary_rays()
    tab = H.Table(10, 1, 6)
    otab = O.Table(10, 1, 6, O.TWO_PHASE)
    for n in (0, 1, 31, 33, 1000, 4097):
        rays = base[:n].copy()
        if n > 10:
            rays[3, 3] = rays[3, 7] = 5.0            # tmin == tmax: empty interval
            rays[4, 4:7] = [0.0, -1.0, 0.0]          # exactly axis-aligned
            rays[5, 4:7] = [0.0, 0.0, -0.0]          # zero direction
            rays[6, 0:3] = [0.0, 1.0, 0.0]           # origin inside the sphere
            rays[7, 7] = 0.0                         # tmax 0
        for mode in (O.CLOSEST_HIT, O.ANY_HIT):
            oh, ost = _oracle(s, rays, mode, otab if mode == O.CLOSEST_HIT else None)
            gh, gst = gpu_trace(H, g, rays, mode, tab if mode == O.CLOSEST_HIT else None)
            if n:
                assert_same_hits(mode, gh, oh, f"n={n}")
            assert_same_stats(gst, ost, msg=f"n={n}")
        assert np.array_equal(tab.export(), otab.words)


def test_root_leaf_scene(H):
    tris = S.soup(3, 2, 0, 1, 0.5)
    nodes, prim, root = S.build_bvh(tris, trav_cost=0.0)  # 3 triangles: one leaf
    g = H.Scene(tris, nodes, prim, root, 2)
    assert g.info()["root_is_leaf"] == 1
    rays = S.sphere_rays(300, 1, -0.5, 1.5)
    for mode in (O.CLOSEST_HIT, O.ANY_HIT):
        oh, ost = O.trace(tris, nodes, prim, root, rays, mode)
        gh, gst = gpu_trace(H, g, rays, mode)
        assert_same_hits(mode, gh, oh)
        assert_same_stats(gst, ost)


@pytest.mark.parametrize("mode", [O.CLOSEST_HIT, O.ANY_HIT])
def test_online_mode_is_exact(H, small_pair, mode):
    s, g = small_pair[1]
    tab = H.Table(12, 2, 6, H.HRPP_UPDATE_ONLINE)
    for frame in range(3):
        rays = s.primary_rays(frame=frame)
        ph, _ = gpu_trace(H, g, rays, mode)
        hh, st = gpu_trace(H, g, rays, mode, tab)
        if mode == O.CLOSEST_HIT:
            assert np.array_equal(as_words(ph), as_words(hh))
        else:
            assert np.array_equal(any_prims(ph) == O.NO_HIT, any_prims(hh) == O.NO_HIT)
        assert st["positives"] + st["negatives"] == len(rays)
    assert st["true_pos"] > 0


def _one_ray_per_set(rays, p, log2_sets, batch):
    """Splits rays into batches in which no two rays share a table set (keys
    and sets from the oracle's Sec. 5 hash and index)."""
    sets = np.array([O.set_and_tag(O.ray_key(r, p), log2_sets)[0] for r in rays])
    out, cur, used = [], [], set()
    for i, st in enumerate(sets):
        if st in used:
            continue
        cur.append(i)
        used.add(st)
        if len(cur) == batch:
            out.append(rays[cur])
            cur, used = [], set()
    return out


@pytest.mark.parametrize("mode", [O.CLOSEST_HIT, O.ANY_HIT])
@pytest.mark.parametrize("width_idx", [0, 1])
def test_online_insert_matches_oracle_without_races(H, small_pair, mode, width_idx):
    """Online mode's compare-and-swap insert (the set's first empty way, else
    way ray mod W): in batches where no two rays share a set no insert races,
    so hits, every counter and every table word equal the oracle's online
    mode over batch after batch, through fills and evictions."""
    s, g = small_pair[width_idx]
    log2_entries, ways = 10, 4
    tab = H.Table(log2_entries, ways, 6, H.HRPP_UPDATE_ONLINE)
    otab = O.Table(log2_entries, ways, 6, O.ONLINE)
    pool = np.concatenate([s.primary_rays(frame=f)[::5] for f in range(3)])
    if mode == O.ANY_HIT:
        h, _ = _oracle(s, pool, O.CLOSEST_HIT)
        pool, _ = W.secondary_shadow(s, pool, h["t"], h["prim"])
    batches = _one_ray_per_set(pool, 6, log2_entries - 2, 200)[:30]
    assert len(batches) >= 8
    evictions = 0
    for k, rays in enumerate(batches):
        oh, ost = _oracle(s, rays, mode, otab)
        gh, gst = gpu_trace(H, g, rays, mode, tab)
        assert_same_hits(mode, gh, oh, f"batch {k}")
        assert_same_stats(gst, ost, msg=f"batch {k}")
        assert np.array_equal(tab.export(), otab.words), f"batch {k}: table words differ"
        evictions += gst["evictions"]
    assert evictions > 0


@pytest.mark.parametrize("schedule", [1, 2])
@pytest.mark.parametrize("mode", [O.CLOSEST_HIT, O.ANY_HIT])
@pytest.mark.parametrize("width_idx", [0, 1])
def test_gate_matches_oracle(H, small_pair, width_idx, mode, schedule):
    """The table gate against the oracle over frames that close and reopen
    it: hits, every counter (gated included), table words and the gate's
    state after every call, with both ray schedules."""
    s, g = small_pair[width_idx]
    # frame 0 on an empty table predicts nothing: the gate closes; the
    # sampled chunks of frames 1-2 predict and reopen it; the all-miss batch
    # closes it again, and frame 3 is traced through the closed gate
    tab = H.Table(12, 2, 6)
    tab.set_gate(40, 2)
    otab = O.Table(12, 2, 6, O.TWO_PHASE, gate_min_tp=40, gate_sample_log2=2)
    states = []
    for step in range(5):
        rays = s.primary_rays(frame=min(step, 3))
        if mode == O.ANY_HIT:
            h, _ = _oracle(s, rays, O.CLOSEST_HIT)
            rays, _ = W.secondary_shadow(s, rays, h["t"], h["prim"])
        if step == 3:
            rays = rays.copy()
            rays[:, 4:7] = [0.0, 1.0, 0.0]  # straight up: every ray misses
        oh, ost = _oracle(s, rays, mode, otab)
        d = __import__("torch").from_numpy(np.ascontiguousarray(rays)).cuda()
        gh, gst = H.trace(g, d, mode, tab, stats=True, schedule=schedule)
        __import__("torch").cuda.synchronize()
        assert_same_hits(mode, gh.cpu().numpy(), oh, f"step {step}")
        assert_same_stats(gst, ost, msg=f"step {step}")
        assert np.array_equal(tab.export(), otab.words), f"step {step}: table words differ"
        assert tab.gate_open() == otab.gate_open, f"step {step}: gate state differs"
        states.append((otab.gate_open, ost["gated"]))
    assert any(not o for o, _ in states) and any(o for o, _ in states[1:])
    assert any(gated > 0 for _, gated in states)


def test_gate_in_a_batch_matches_single_calls(H, small_pair):
    """A gated table in a batched launch: per item the hits, counters, table
    words and gate state equal those of hrpp_trace calls with the same gate,
    run after run."""
    import torch
    s, g = small_pair[1]
    rays = [torch.from_numpy(s.primary_rays(frame=f)).cuda() for f in range(3)]
    tb, tc = H.Table(12, 1, 6), H.Table(12, 1, 6)
    for t in (tb, tc):
        t.set_gate(3000, 3)
    buf = torch.empty_like(rays[0])
    batch = H.Batch([(g, tb, buf, H.HRPP_CLOSEST_HIT)], stats=True)
    for f in (0, 1, 2, 1):
        buf.copy_(rays[f])
        batch.run()
        ref, rst = H.trace(g, rays[f], H.HRPP_CLOSEST_HIT, tc, stats=True)
        torch.cuda.synchronize()
        assert torch.equal(batch.hits[0].view(torch.int32), ref.view(torch.int32))
        assert batch.stats(0) == rst
        assert np.array_equal(tb.export(), tc.export()) and tb.gate_open() == tc.gate_open()


def test_frozen_mode_never_writes(H, small_pair):
    s, g = small_pair[0]
    tab = H.Table(12, 1, 6)
    gpu_trace(H, g, s.primary_rays(), O.CLOSEST_HIT, tab)
    before = tab.export()
    tab.configure(6, H.HRPP_UPDATE_FROZEN)
    _, st = gpu_trace(H, g, s.primary_rays(frame=2), O.CLOSEST_HIT, tab)
    assert st["inserts"] == 0 and np.array_equal(tab.export(), before)


def test_host_buffers_match_device_path(H, small_pair):
    s, g = small_pair[0]
    rays = np.ascontiguousarray(s.primary_rays(frame=3))
    for mode in (O.CLOSEST_HIT, O.ANY_HIT):
        dev, _ = gpu_trace(H, g, rays, mode)
        host, st = H.trace(g, rays, mode, stats=True)
        assert isinstance(host, np.ndarray)
        if mode == O.CLOSEST_HIT:
            assert np.array_equal(as_words(dev), as_words(host))
        else:
            assert np.array_equal(any_prims(dev), any_prims(host))
        assert st["rays"] == len(rays)


def test_table_bound_to_its_scene_and_roundtrip(H, small_pair):
    (s2, g2), (s4, g4) = small_pair
    tab = H.Table(12, 1, 6)
    gpu_trace(H, g2, s2.primary_rays(), O.CLOSEST_HIT, tab)
    with pytest.raises(H.HrppError) as e:
        gpu_trace(H, g4, s4.primary_rays(), O.CLOSEST_HIT, tab)
    assert e.value.status == H.HRPP_ERR_INVALID_ARG
    words = tab.export()
    tab.reset()
    assert np.all(tab.export() == np.uint64(H.HRPP_EMPTY_WORD))
    gpu_trace(H, g4, s4.primary_rays(), O.CLOSEST_HIT, tab)   # rebinds after reset
    tab.reset()
    tab.import_(words)
    assert np.array_equal(tab.export(), words)


@pytest.mark.parametrize("width_idx", [0, 1])
def test_exponent_lsb_hash_matches_oracle(H, small_pair, width_idx):
    """The exponent-LSB hash variant: hits, counters and table words equal
    the oracle's over three frames of both query modes, at p = 3 (where the
    variants file rays differently)."""
    s, g = small_pair[width_idx]
    tabs = {m: H.Table(12, 2, 3, hash_variant=H.HRPP_HASH_EXP_LSB) for m in (O.CLOSEST_HIT, O.ANY_HIT)}
    otabs = {m: O.Table(12, 2, 3, O.TWO_PHASE, hash_variant=O.HASH_EXP_LSB) for m in (O.CLOSEST_HIT, O.ANY_HIT)}
    msb = O.Table(12, 2, 3, O.TWO_PHASE)
    for frame in range(3):
        prim = s.primary_rays(frame=frame)
        ph, _ = _oracle(s, prim, O.CLOSEST_HIT)
        shadow, _ = W.secondary_shadow(s, prim, ph["t"], ph["prim"])
        _oracle(s, prim, O.CLOSEST_HIT, msb)
        for mode, rays in ((O.CLOSEST_HIT, prim), (O.ANY_HIT, shadow)):
            oh, ost = _oracle(s, rays, mode, otabs[mode])
            gh, gst = gpu_trace(H, g, rays, mode, tabs[mode])
            assert_same_hits(mode, gh, oh, f"frame {frame}")
            assert_same_stats(gst, ost, msg=f"frame {frame}")
            assert np.array_equal(tabs[mode].export(), otabs[mode].words)
    assert not np.array_equal(otabs[O.CLOSEST_HIT].words, msb.words)
    with pytest.raises(H.HrppError):
        tabs[O.CLOSEST_HIT].set_hash(2)
    with pytest.raises(H.HrppError):
        H.Table(12, 2, 3).copy_from(tabs[O.CLOSEST_HIT])


def test_table_copy_restores_a_snapshot(H, small_pair):
    """hrpp_table_copy: a device snapshot of a warm table, restored after the
    table moved on, gives the words and the next batch's results, counters
    and words that the oracle gives from the same snapshot."""
    import torch
    s, g = small_pair[1]
    tab, snap = H.Table(12, 2, 6), H.Table(12, 2, 6)
    for f in (1, 2):
        H.trace(g, torch.from_numpy(s.primary_rays(frame=f)).cuda(), H.HRPP_CLOSEST_HIT, tab)
    snap.copy_from(tab)
    torch.cuda.synchronize()
    words = snap.export()
    assert np.array_equal(words, tab.export()) and (words != np.uint64(2**64 - 1)).any()
    H.trace(g, torch.from_numpy(s.primary_rays(frame=3)).cuda(), H.HRPP_CLOSEST_HIT, tab)
    assert not np.array_equal(tab.export(), words)
    tab.copy_from(snap)
    assert np.array_equal(tab.export(), words)
    rays = s.primary_rays(frame=4)
    otab = O.Table(12, 2, 6, O.TWO_PHASE)
    otab.words[:] = words
    oh, ost = _oracle(s, rays, O.CLOSEST_HIT, otab)
    gh, gst = gpu_trace(H, g, rays, O.CLOSEST_HIT, tab)
    assert_same_hits(O.CLOSEST_HIT, gh, oh)
    assert_same_stats(gst, ost)
    assert np.array_equal(tab.export(), otab.words)
    for bad in (H.Table(12, 4, 6), H.Table(12, 2, 5), H.Table(13, 2, 6), H.Table(12, 2, 6, go_up=1)):
        with pytest.raises(H.HrppError) as err:
            bad.copy_from(snap)
        assert err.value.status == H.HRPP_ERR_INVALID_ARG


@pytest.mark.parametrize("schedule", [1, 3])
@pytest.mark.parametrize("mode", [O.CLOSEST_HIT, O.ANY_HIT])
def test_staged_host_buffers_in_chunks_match_device_path(H, small_pair, mode, schedule):
    """Host ray and hit buffers above the staging chunk size (2 or 3 chunks
    with a ragged tail): pinned and pageable host memory give exactly the
    device path's hits, counters and table words over two calls, with a
    two-phase table whose gate samples by the call's ray index."""
    import torch
    s, g = small_pair[1]
    n = 10 * 65536 + 17
    frames = [np.concatenate([s.primary_rays(frame=f) for f in range(k, k + 11)])[:n] for k in (0, 11)]
    if mode == O.ANY_HIT:
        out = []
        for r in frames:
            h, _ = H.trace(g, torch.from_numpy(r).cuda(), H.HRPP_CLOSEST_HIT)
            hh = h.cpu().numpy()
            out.append(np.ascontiguousarray(W.secondary_shadow(s, r, hh[:, 0], hh[:, 1].view(np.uint32))[0]))
        frames = out
    for pinned in (True, False):
        t_dev, t_host = H.Table(14, 2, 6), H.Table(14, 2, 6)
        for t in (t_dev, t_host):
            t.set_gate(2000, 2)
        for rays in frames:
            ref, rst = H.trace(g, torch.from_numpy(rays).cuda(), mode, t_dev, stats=True, schedule=schedule)
            hr = torch.from_numpy(rays)
            hits = torch.empty(tuple(ref.shape), dtype=ref.dtype)
            if pinned:
                hr, hits = hr.pin_memory(), hits.pin_memory()
            got, gst = H.trace(g, hr, mode, t_host, hits=hits, stats=True, schedule=schedule)
            torch.cuda.synchronize()
            assert torch.equal(got.view(torch.int32), ref.cpu().view(torch.int32)), f"pinned={pinned}"
            assert gst == rst, f"pinned={pinned}"
            assert np.array_equal(t_dev.export(), t_host.export()) and t_dev.gate_open() == t_host.gate_open()
            assert rst["rays"] == len(rays) > 262144  # more than one staging chunk
            assert rst["gated"] > 0 or rst["lookups"] == len(rays)


def test_queued_host_async_calls_hold_bounded_staging(H, small_pair):
    """Twelve host_async calls queued without waiting (each with its own
    pinned buffers and a host_done event): every one returns the device
    path's hits, and the device memory they take stays within a few staging
    blocks, since at most 6 staged calls hold staging at once."""
    import torch
    s, g = small_pair[1]
    rays = np.concatenate([s.primary_rays(frame=f) for f in range(5)])
    ref, _ = H.trace(g, torch.from_numpy(rays).cuda(), H.HRPP_CLOSEST_HIT)
    block = len(rays) * (32 + 16)
    stream = torch.cuda.Stream()
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    calls = []
    for k in range(12):
        hr = torch.from_numpy(rays).pin_memory()
        hits = torch.full((len(rays), 4), 7.0).pin_memory()
        done = torch.cuda.Event()
        done.record(stream)  # creates the CUDA event; the library records it again
        H.trace(g, hr, H.HRPP_CLOSEST_HIT, None, hits=hits, stream=stream, host_async=True, host_done=done)
        calls.append((hr, hits, done))
    for hr, hits, done in calls:
        done.synchronize()
        assert torch.equal(hits.view(torch.int32), ref.cpu().view(torch.int32))
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert free0 - free1 <= 8 * (block + (2 << 20)), (free0 - free1, block)


def test_host_async_calls_match_device_path(H, small_pair):
    """hrpp_trace_opts.host_async: calls on pinned host buffers return before
    their work is done; several of them queued on two streams (one table
    each, three frames in a row) give, once the streams are synchronized,
    exactly the device path's hits and table words.  Pageable buffers are
    refused."""
    import torch
    s, g = small_pair[1]
    frames = [np.concatenate([s.primary_rays(frame=f) for f in range(k, k + 5)]) for k in (0, 5, 10)]
    tabs = [H.Table(14, 2, 6), H.Table(14, 2, 6)]
    refs = [H.Table(14, 2, 6), H.Table(14, 2, 6)]
    streams = [torch.cuda.Stream(), torch.cuda.Stream()]
    outs, want = [], []
    for k, rays in enumerate(frames):
        for j in range(2):  # table j traces every frame, with its own stream
            ref, _ = H.trace(g, torch.from_numpy(rays).cuda(), H.HRPP_CLOSEST_HIT, refs[j])
            want.append(ref)
            hr = torch.from_numpy(rays).pin_memory()
            hits = torch.full((len(rays), 4), 7.0).pin_memory()
            H.trace(g, hr, H.HRPP_CLOSEST_HIT, tabs[j], hits=hits, stream=streams[j], host_async=True)
            outs.append((hr, hits))
    torch.cuda.synchronize()
    for (hr, hits), ref in zip(outs, want):
        assert torch.equal(hits.view(torch.int32), ref.cpu().view(torch.int32))
    for t, r in zip(tabs, refs):
        assert np.array_equal(t.export(), r.export())
    g.check()
    # host_done: the event, not the stream, marks the hits in host memory
    for k, rays in enumerate(frames):
        hr = torch.from_numpy(rays).pin_memory()
        hits = torch.full((len(rays), 4), 7.0).pin_memory()
        done = torch.cuda.Event()
        done.record(streams[0])  # creates the CUDA event; the library records it again
        H.trace(g, hr, H.HRPP_CLOSEST_HIT, None, hits=hits, stream=streams[0], host_async=True, host_done=done,
                stage_chunks=k + 1)
        done.synchronize()
        ref, _ = H.trace(g, torch.from_numpy(rays).cuda(), H.HRPP_CLOSEST_HIT)
        assert torch.equal(hits.view(torch.int32), ref.cpu().view(torch.int32)), k
    with pytest.raises(H.HrppError) as err:
        H.trace(g, frames[0], H.HRPP_CLOSEST_HIT, host_async=True)  # numpy: pageable
    assert err.value.status == H.HRPP_ERR_INVALID_ARG


@pytest.mark.parametrize("n", [0, 1, 31, 33, 257])
def test_edge_sizes_through_every_path(H, small_pair, n):
    """Empty, single-ray and ragged batches through the two-pass schedule,
    a gated table, the staged host path (synchronous and host_async) and
    the device path: identical hits, counters and table words (zero counters
    and no work for an empty batch)."""
    import torch
    s, g = small_pair[0]
    rays = np.ascontiguousarray(s.primary_rays(frame=2)[:n])
    variants = [dict(), dict(schedule=H.HRPP_SCHEDULE_COMPACT), dict(host=True), dict(host=True, host_async=True)]
    out = []
    for v in variants:
        tab = H.Table(12, 2, 6)
        tab.set_gate(1000, 1)
        for frame in range(2):
            if v.get("host"):
                hr = torch.from_numpy(rays).pin_memory()
                hits = torch.full((n, 4), 7.0).pin_memory()
                h, st = H.trace(g, hr, H.HRPP_CLOSEST_HIT, tab, hits=hits, stats=True,
                                host_async=v.get("host_async", False))
            else:
                h, st = H.trace(g, torch.from_numpy(rays).cuda(), H.HRPP_CLOSEST_HIT, tab, stats=True,
                                schedule=v.get("schedule", 0))
            torch.cuda.synchronize()
        out.append((h.cpu().view(torch.int32).clone(), st, tab.export(), tab.gate_open()))
    ref = out[0]
    for v, o in zip(variants[1:], out[1:]):
        assert torch.equal(o[0], ref[0]), v
        assert o[1] == ref[1], (v, o[1], ref[1])
        assert np.array_equal(o[2], ref[2]) and o[3] == ref[3], v
    assert ref[1]["rays"] == n
    if n == 0:
        assert all(v == 0 for v in ref[1].values())


def test_block_sizes_give_identical_results(H, small_pair):
    s, g = small_pair[1]
    rays = s.primary_rays(frame=5)
    ref, rst = gpu_trace(H, g, rays, O.CLOSEST_HIT)
    for bt in (64, 256, 512):
        h, st = gpu_trace(H, g, rays, O.CLOSEST_HIT, block_threads=bt)
        assert np.array_equal(as_words(h), as_words(ref))
        assert_same_stats(st, rst)


def test_mid_terrain_bvh4_hrpp(H):
    """The terrain recipe at reduced size (BVH4, several ragged tiles of rays):
    primary closest-hit and ambient-occlusion any-hit rays over three frames."""
    s = W.terrain_scene(quads=96, n_spheres=6, subdiv=3, res=(200, 120))
    g = H.Scene.from_workload(s)
    tabs = {m: H.Table(14, 2, 6) for m in (O.CLOSEST_HIT, O.ANY_HIT)}
    otabs = {m: O.Table(14, 2, 6, O.TWO_PHASE) for m in (O.CLOSEST_HIT, O.ANY_HIT)}
    tp = {O.CLOSEST_HIT: 0, O.ANY_HIT: 0}
    for frame in range(3):
        prim = s.primary_rays(frame=frame)
        ph, _ = _oracle(s, prim, O.CLOSEST_HIT)
        ao, _ = W.secondary_ao(s, prim, ph["t"], ph["prim"], frame=frame)
        for mode, rays in ((O.CLOSEST_HIT, prim), (O.ANY_HIT, ao)):
            oh, ost = _oracle(s, rays, mode, otabs[mode])
            gh, gst = gpu_trace(H, g, rays, mode, tabs[mode])
            assert_same_hits(mode, gh, oh, f"frame {frame}")
            assert_same_stats(gst, ost, msg=f"frame {frame}")
            assert np.array_equal(tabs[mode].export(), otabs[mode].words)
            tp[mode] += gst["true_pos"]
    # primary rays of later frames find their leaves predicted
    assert tp[O.CLOSEST_HIT] > 0


@pytest.mark.parametrize("width_idx", [0, 1])
@pytest.mark.parametrize("mode", [O.CLOSEST_HIT, O.ANY_HIT])
def test_schedules_give_identical_results(H, small_pair, width_idx, mode):
    """Batch and refill schedules, any refill threshold and block size: the
    same hits, counters and table words as the oracle."""
    s, g = small_pair[width_idx]
    variants = [dict(schedule=H.HRPP_SCHEDULE_BATCH), dict(schedule=H.HRPP_SCHEDULE_REFILL, refill_min=1),
                dict(schedule=H.HRPP_SCHEDULE_REFILL, refill_min=8, block_threads=256),
                dict(schedule=H.HRPP_SCHEDULE_REFILL, refill_min=32, block_threads=64),
                dict(schedule=H.HRPP_SCHEDULE_COMPACT), dict(schedule=H.HRPP_SCHEDULE_COMPACT, block_threads=512)]
    prim = s.primary_rays(frame=2)
    ph, _ = _oracle(s, prim, O.CLOSEST_HIT)
    rays = prim if mode == O.CLOSEST_HIT else W.secondary_shadow(s, prim, ph["t"], ph["prim"])[0]
    otab = O.Table(12, 2, 6, O.TWO_PHASE)
    _oracle(s, s.primary_rays(frame=1), mode, otab)
    warm = otab.words.copy()
    oh, ost = _oracle(s, rays, mode, otab)
    import torch
    dr = torch.from_numpy(rays).cuda()
    for v in variants:
        tab = H.Table(12, 2, 6)
        tab.import_(warm)
        gh, gst = H.trace(g, dr, mode, tab, stats=True, **v)
        torch.cuda.synchronize()
        assert_same_hits(mode, gh.cpu().numpy(), oh, str(v))
        assert_same_stats(gst, ost, msg=str(v))
        assert np.array_equal(tab.export(), otab.words), str(v)


@pytest.mark.parametrize("verify", [0, 2])
@pytest.mark.parametrize("gated", [False, True])
def test_compact_schedule_matches_oracle(H, verify, gated):
    """The two-pass schedule (the ray pool of Sec. 4.1-4.2: lookups first,
    answered rays leave, the rest are queued and traversed) on the terrain
    recipe at reduced size, over frames whose any-hit AO rays and closest-hit
    primaries are partly predicted: hits, every counter, per-ray outcomes and
    box tests, table words and gate state equal the oracle's, with root
    verification (exact) and without (the paper's semantics).  The batches
    are ragged (not multiples of the 256-ray pass-1 block)."""
    import torch
    s = W.terrain_scene(quads=96, n_spheres=6, subdiv=3, res=(203, 117))
    g = H.Scene.from_workload(s)
    gate = (2500, 3) if gated else (0, 5)
    tabs = {m: H.Table(14, 2, 6) for m in (O.CLOSEST_HIT, O.ANY_HIT)}
    otabs = {m: O.Table(14, 2, 6, O.TWO_PHASE, gate_min_tp=gate[0], gate_sample_log2=gate[1])
             for m in (O.CLOSEST_HIT, O.ANY_HIT)}
    for t in tabs.values():
        t.set_gate(*gate)
    answered = 0
    for frame in range(4):
        prim = s.primary_rays(frame=frame % 3)
        ph, _ = _oracle(s, prim, O.CLOSEST_HIT)
        ao, _ = W.secondary_ao(s, prim, ph["t"], ph["prim"], frame=frame % 3)
        for mode, rays in ((O.CLOSEST_HIT, prim), (O.ANY_HIT, ao)):
            v = verify if mode == O.CLOSEST_HIT else 0
            oh, ost, ooc, obx = O.trace(s.tris, s.nodes, s.prim_index, s.root, rays, mode, otabs[mode],
                                        per_ray=True, verify=v)
            d = torch.from_numpy(rays).cuda()
            oc = torch.full((len(rays),), 255, dtype=torch.uint8, device="cuda")
            bx = torch.full((len(rays),), -1, dtype=torch.int32, device="cuda")
            gh, gst = H.trace(g, d, mode, tabs[mode], stats=True, schedule=H.HRPP_SCHEDULE_COMPACT, verify=v,
                              ray_outcome=oc, ray_box_tests=bx)
            torch.cuda.synchronize()
            g.check()
            msg = f"frame {frame} mode {mode}"
            assert_same_hits(mode, gh.cpu().numpy(), oh, msg)
            assert_same_stats(gst, ost, msg=msg)
            assert np.array_equal(oc.cpu().numpy(), ooc), msg
            assert np.array_equal(bx.cpu().numpy().view(np.uint32), obx), msg
            assert np.array_equal(tabs[mode].export(), otabs[mode].words), msg
            assert tabs[mode].gate_open() == otabs[mode].gate_open, msg
            if mode == O.ANY_HIT or verify == 2:
                answered += gst["true_pos"]
    assert answered > 0


@pytest.mark.parametrize("ways", [4, 8])
@pytest.mark.parametrize("schedule", ["batch", "compact"])
def test_many_predicted_leaves_per_ray_match_oracle(H, ways, schedule):
    """Lookups that find several predicted leaves: shadow rays toward a low
    light over the reduced terrain recipe (keys repeat across neighbouring
    hits and a key keeps several leaves), 4- and 8-way sets at p = 5, both
    schedules.  Every ray's candidates are tested in one loop over their
    triangles in way order (Sec. 4.2); hits, counters (predicted leaves and
    triangle tests up to an any-hit ray's first hit), per-ray outcomes and
    table words equal the oracle's, which tests leaf by leaf."""
    import torch
    s = W.terrain_scene(quads=96, n_spheres=6, subdiv=3, res=(203, 117))
    g = H.Scene.from_workload(s)
    sched = H.HRPP_SCHEDULE_COMPACT if schedule == "compact" else H.HRPP_SCHEDULE_BATCH
    tabs = {m: H.Table(12, ways, 5) for m in (O.CLOSEST_HIT, O.ANY_HIT)}
    otabs = {m: O.Table(12, ways, 5, O.TWO_PHASE) for m in (O.CLOSEST_HIT, O.ANY_HIT)}
    tot = {m: {"pred_leaves": 0, "positives": 0, "true_pos": 0} for m in tabs}
    for frame in range(4):
        prim = s.primary_rays(frame=frame % 3)
        ph, _ = _oracle(s, prim, O.CLOSEST_HIT)
        shadow, _ = W.secondary_shadow(s, prim, ph["t"], ph["prim"], light=W.TERRAIN_SUN)
        for mode, rays in ((O.CLOSEST_HIT, prim), (O.ANY_HIT, shadow)):
            oh, ost, ooc, _ = O.trace(s.tris, s.nodes, s.prim_index, s.root, rays, mode, otabs[mode], per_ray=True)
            d = torch.from_numpy(rays).cuda()
            oc = torch.full((len(rays),), 255, dtype=torch.uint8, device="cuda")
            gh, gst = H.trace(g, d, mode, tabs[mode], stats=True, schedule=sched, ray_outcome=oc)
            torch.cuda.synchronize()
            g.check()
            msg = f"frame {frame} mode {mode} ways {ways} {schedule}"
            assert_same_hits(mode, gh.cpu().numpy(), oh, msg)
            assert_same_stats(gst, ost, msg=msg)
            assert np.array_equal(oc.cpu().numpy(), ooc), msg
            assert np.array_equal(tabs[mode].export(), otabs[mode].words), msg
            for k in tot[mode]:
                tot[mode][k] += gst[k]
    # the case under test happened: positive rays with more than one
    # candidate leaf, and any-hit true positives
    for m in tabs:
        assert tot[m]["pred_leaves"] > tot[m]["positives"] > 0, (m, tot[m])
    assert tot[O.ANY_HIT]["true_pos"] > 0


@pytest.mark.parametrize("go_up", [1, 2, 5])
@pytest.mark.parametrize("width_idx", [0, 1])
def test_go_up_levels_match_oracle(H, small_pair, go_up, width_idx):
    """Go Up Level (Sec. 6.2): predicted subtrees, their counters and the
    ancestor words stored in the table, over three frames of both modes."""
    s, g = small_pair[width_idx]
    tabs = {m: H.Table(12, 2, 6, go_up=go_up) for m in (O.CLOSEST_HIT, O.ANY_HIT)}
    otabs = {m: O.Table(12, 2, 6, O.TWO_PHASE, go_up=go_up) for m in (O.CLOSEST_HIT, O.ANY_HIT)}
    pred = 0
    for frame in range(3):
        prim = s.primary_rays(frame=frame)
        ph, _ = _oracle(s, prim, O.CLOSEST_HIT)
        shadow, _ = W.secondary_shadow(s, prim, ph["t"], ph["prim"])
        for mode, rays in ((O.CLOSEST_HIT, prim), (O.ANY_HIT, shadow)):
            oh, ost = _oracle(s, rays, mode, otabs[mode])
            gh, gst = gpu_trace(H, g, rays, mode, tabs[mode])
            assert_same_hits(mode, gh, oh, f"frame {frame}")
            assert_same_stats(gst, ost, msg=f"frame {frame} go_up {go_up}")
            assert np.array_equal(tabs[mode].export(), otabs[mode].words)
            pred += gst["pred_interior_nodes"]
    assert pred > 0


def test_go_up_mid_terrain_bvh4(H):
    s = W.terrain_scene(quads=64, n_spheres=4, subdiv=2, res=(160, 96))
    g = H.Scene.from_workload(s)
    tab = H.Table(14, 4, 6, go_up=1)
    otab = O.Table(14, 4, 6, O.TWO_PHASE, go_up=1)
    for frame in range(2):
        prim = s.primary_rays(frame=frame)
        ph, _ = _oracle(s, prim, O.CLOSEST_HIT)
        ao, _ = W.secondary_ao(s, prim, ph["t"], ph["prim"], frame=frame)
        oh, ost = _oracle(s, ao, O.ANY_HIT, otab)
        gh, gst = gpu_trace(H, g, ao, O.ANY_HIT, tab)
        assert_same_hits(O.ANY_HIT, gh, oh)
        assert_same_stats(gst, ost)
        assert np.array_equal(tab.export(), otab.words)


@pytest.mark.parametrize("schedule", [1, 2])
@pytest.mark.parametrize("go_up", [0, 1])
@pytest.mark.parametrize("width_idx", [0, 1])
def test_bottom_up_verification_matches_oracle(H, small_pair, go_up, width_idx, schedule):
    """Closest-hit true positives verified by the bottom-up climb: hits,
    every counter and the table words equal the oracle's, over three frames,
    with both ray schedules."""
    s, g = small_pair[width_idx]
    tab = H.Table(12, 2, 6, go_up=go_up)
    otab = O.Table(12, 2, 6, O.TWO_PHASE, go_up=go_up)
    import torch
    tp = 0
    for frame in range(3):
        rays = s.primary_rays(frame=frame)
        oh, ost = O.trace(s.tris, s.nodes, s.prim_index, s.root, rays, O.CLOSEST_HIT, otab,
                          verify=O.VERIFY_BOTTOM_UP)
        gh, gst = H.trace(g, torch.from_numpy(rays).cuda(), H.HRPP_CLOSEST_HIT, tab, stats=True,
                          schedule=schedule, verify=H.HRPP_VERIFY_BOTTOM_UP)
        torch.cuda.synchronize()
        assert_same_hits(O.CLOSEST_HIT, gh.cpu().numpy(), oh, f"frame {frame}")
        assert_same_stats(gst, ost, msg=f"frame {frame}")
        assert np.array_equal(tab.export(), otab.words)
        tp += gst["true_pos"]
    assert tp > 0


@pytest.mark.parametrize("width", [2, 4])
def test_bottom_up_with_predicted_treelets(H, width):
    """Learned-style predictions (valid nodes, -1, out of range) verified by
    the climb: hits and counters equal the oracle's."""
    import torch
    s = W.small_scene(width=width)
    g = H.Scene.from_workload(s)
    rays = s.primary_rays(frame=5)
    rng = np.random.default_rng(11 + width)
    pred = rng.integers(-1, len(s.nodes) + 3, len(rays)).astype(np.int32)
    oh, ost = O.trace(s.tris, s.nodes, s.prim_index, s.root, rays, O.CLOSEST_HIT, predicted=pred,
                      verify=O.VERIFY_BOTTOM_UP)
    gh, gst = H.trace(g, torch.from_numpy(rays).cuda(), H.HRPP_CLOSEST_HIT, stats=True,
                      predicted=torch.from_numpy(pred).cuda(), verify=H.HRPP_VERIFY_BOTTOM_UP)
    torch.cuda.synchronize()
    assert_same_hits(O.CLOSEST_HIT, gh.cpu().numpy(), oh)
    assert_same_stats(gst, ost)
    assert gst["true_pos"] > 0


def test_bottom_up_mid_terrain_bvh4(H):
    """A deeper 4-wide tree: two frames of jittered primaries through a
    warm table, verified by the climb."""
    import torch
    s = W.terrain_scene(quads=64, n_spheres=4, subdiv=2, res=(160, 96))
    g = H.Scene.from_workload(s)
    tab = H.Table(14, 2, 6)
    otab = O.Table(14, 2, 6, O.TWO_PHASE)
    for frame in range(2):
        rays = s.primary_rays(frame=frame)
        oh, ost = O.trace(s.tris, s.nodes, s.prim_index, s.root, rays, O.CLOSEST_HIT, otab,
                          verify=O.VERIFY_BOTTOM_UP)
        gh, gst = H.trace(g, torch.from_numpy(rays).cuda(), H.HRPP_CLOSEST_HIT, tab, stats=True,
                          verify=H.HRPP_VERIFY_BOTTOM_UP)
        torch.cuda.synchronize()
        assert_same_hits(O.CLOSEST_HIT, gh.cpu().numpy(), oh)
        assert_same_stats(gst, ost)
        assert np.array_equal(tab.export(), otab.words)


@pytest.mark.parametrize("go_up", [0, 1])
@pytest.mark.parametrize("width_idx", [0, 1])
def test_unverified_mode_matches_oracle(H, small_pair, go_up, width_idx):
    """HRPP_VERIFY_NONE (the paper's semantics, not exact): hits, counters
    and table words equal the oracle's VERIFY_NONE over three frames, and
    some true positives do return another hit than plain traversal."""
    import torch
    s, g = small_pair[width_idx]
    tab = H.Table(12, 2, 6, go_up=go_up)
    otab = O.Table(12, 2, 6, O.TWO_PHASE, go_up=go_up)
    differ = 0
    for frame in range(3):
        rays = s.primary_rays(frame=frame)
        oh, ost = O.trace(s.tris, s.nodes, s.prim_index, s.root, rays, O.CLOSEST_HIT, otab, verify=O.VERIFY_NONE)
        gh, gst = H.trace(g, torch.from_numpy(rays).cuda(), H.HRPP_CLOSEST_HIT, tab, stats=True,
                          verify=H.HRPP_VERIFY_NONE)
        torch.cuda.synchronize()
        assert_same_hits(O.CLOSEST_HIT, gh.cpu().numpy(), oh, f"frame {frame}")
        assert_same_stats(gst, ost, msg=f"frame {frame}")
        assert np.array_equal(tab.export(), otab.words)
        ph, _ = _oracle(s, rays, O.CLOSEST_HIT)
        differ += int((as_words(oh) != as_words(ph)).any(axis=1).sum())
    assert differ > 0


def test_verify_mode_is_validated(H, small_pair):
    import torch
    s, g = small_pair[0]
    rays = torch.from_numpy(s.primary_rays()[:64]).cuda()
    with pytest.raises(H.HrppError) as err:
        H.trace(g, rays, H.HRPP_CLOSEST_HIT, verify=3)
    assert err.value.status == H.HRPP_ERR_INVALID_ARG


@pytest.mark.parametrize("width_idx", [0, 1])
def test_l2_persisting_window_changes_nothing(H, small_pair, width_idx):
    """An L2 access-policy window over the table or the interior nodes, with
    a persisting set-aside in force, leaves hits, counters and table words
    exactly as without it; an unknown window kind is rejected; releasing the
    set-aside leaves none."""
    import torch
    s, g = small_pair[width_idx]
    frames = [torch.from_numpy(s.primary_rays(frame=f)).cuda() for f in (1, 2)]
    try:
        granted = H.l2_set_aside(4 << 20)
    except H.HrppError as err:  # a device without persisting L2: the window is a no-op
        assert err.status == H.HRPP_ERR_CUDA
        granted = 0
    try:
        ref = H.Table(10, ways=2, precision=6)
        want = []
        for r in frames:
            h, st = H.trace(g, r, H.HRPP_CLOSEST_HIT, ref, stats=True)
            want.append((h.view(torch.int32).cpu(), st))
        for kind in (H.HRPP_L2_TABLE, H.HRPP_L2_NODES):
            t = H.Table(10, ways=2, precision=6)
            for r, (wh, wst) in zip(frames, want):
                h, st = H.trace(g, r, H.HRPP_CLOSEST_HIT, t, stats=True, l2_persist=kind)
                assert torch.equal(h.view(torch.int32).cpu(), wh) and st == wst
            assert np.array_equal(t.export(), ref.export())
            hp, _ = H.trace(g, frames[0], H.HRPP_ANY_HIT, None, l2_persist=kind)
            hq, _ = H.trace(g, frames[0], H.HRPP_ANY_HIT, None)
            assert torch.equal(hp, hq)
        with pytest.raises(H.HrppError) as err:
            H.trace(g, frames[0], H.HRPP_CLOSEST_HIT, ref, l2_persist=3)
        assert err.value.status == H.HRPP_ERR_INVALID_ARG
    finally:
        if granted:
            assert H.l2_set_aside(0) == 0


@pytest.mark.parametrize("width_idx", [0, 1])
def test_two_streams_two_tables_match_sequential(H, small_pair, width_idx):
    """A frame's primary and shadow batches traced side by side on two
    streams (one table each, one scene) give exactly the hits, counters and
    table words of the same calls in sequence, frame after frame."""
    import torch
    s, g = small_pair[width_idx]
    frames = []
    for f in range(3):
        prim = s.primary_rays(frame=f)
        ph, _ = _oracle(s, prim, O.CLOSEST_HIT)
        shadow, _ = W.secondary_shadow(s, prim, ph["t"], ph["prim"])
        frames.append((torch.from_numpy(prim).cuda(), torch.from_numpy(shadow).cuda()))
    seq = (H.Table(12, 2, 6), H.Table(12, 2, 6))
    par = (H.Table(12, 2, 6), H.Table(12, 2, 6))
    side = torch.cuda.Stream()
    main = torch.cuda.current_stream()
    for prim, shadow in frames:
        hc, sc = H.trace(g, prim, H.HRPP_CLOSEST_HIT, seq[0], stats=True)
        ha, sa = H.trace(g, shadow, H.HRPP_ANY_HIT, seq[1], stats=True)
        # side by side: device stats so that neither call waits
        st_c = torch.zeros(24, dtype=torch.int64, device="cuda")
        st_a = torch.zeros(24, dtype=torch.int64, device="cuda")
        oc = torch.empty_like(hc)
        oa = torch.empty_like(ha)
        fork = torch.cuda.Event()
        fork.record(main)
        side.wait_event(fork)
        H.hrpp_trace(g.handle, par[1].handle, H._ptr(shadow), int(shadow.shape[0]), H.HRPP_ANY_HIT, H._ptr(oa),
                     H._ptr(st_a), side.cuda_stream)
        H.hrpp_trace(g.handle, par[0].handle, H._ptr(prim), int(prim.shape[0]), H.HRPP_CLOSEST_HIT, H._ptr(oc),
                     H._ptr(st_c), main.cuda_stream)
        join = torch.cuda.Event()
        join.record(side)
        main.wait_event(join)
        torch.cuda.synchronize()
        assert torch.equal(oc.view(torch.int32), hc.view(torch.int32))
        assert torch.equal(oa, ha)
        names = H.STAT_NAMES
        assert [int(x) for x in st_c[:len(names)].cpu()] == [sc[n] for n in names]
        assert [int(x) for x in st_a[:len(names)].cpu()] == [sa[n] for n in names]
        assert np.array_equal(par[0].export(), seq[0].export())
        assert np.array_equal(par[1].export(), seq[1].export())


@pytest.mark.parametrize("width_idx", [0, 1])
def test_step_budget_reports_traversal_limit(H, small_pair, width_idx):
    """Failure detection without a fault: a per-traversal step budget far
    below what the rays need stops them early.  The kernel's bounded loop sets
    the scene's device flag; the host sees HRPP_ERR_TRAVERSAL_LIMIT (from
    hrpp_scene_check, or from the call itself when it synchronises for host
    stats), the flag is cleared, and the scene then traces exactly."""
    import torch
    s, g = small_pair[width_idx]
    rays_np = s.primary_rays(frame=1)
    rays = torch.from_numpy(rays_np).cuda()
    H.trace(g, rays, H.HRPP_CLOSEST_HIT, max_steps=2)
    with pytest.raises(H.HrppError) as err:
        g.check()
    assert err.value.status == H.HRPP_ERR_TRAVERSAL_LIMIT
    g.check()  # cleared
    with pytest.raises(H.HrppError) as err:
        H.trace(g, rays, H.HRPP_ANY_HIT, stats=True, max_steps=1)
    assert err.value.status == H.HRPP_ERR_TRAVERSAL_LIMIT
    g.check()
    # a budget the rays never reach changes nothing
    oh, ost = _oracle(s, rays_np, O.CLOSEST_HIT)
    gh, gst = H.trace(g, rays, H.HRPP_CLOSEST_HIT, stats=True, max_steps=1_000_000)
    torch.cuda.synchronize()
    assert_same_hits(O.CLOSEST_HIT, gh.cpu().numpy(), oh)
    assert_same_stats(gst, ost)


def test_injected_allocation_failures_return_oom(H, small_pair, monkeypatch):
    """Host-side fault injection (HRPP_FAIL_ALLOC_AFTER=N fails the device
    allocations after the first N): every creating entry point reports
    HRPP_ERR_OOM at each of its allocations, cleans up, and works again once
    the variable is gone."""
    import torch
    s, g = small_pair[0]
    rays = torch.from_numpy(s.primary_rays()[:256]).cuda()
    makers = {
        "scene": (6, lambda: H.Scene.from_workload(s)),
        "table": (2, lambda: H.Table(10, 2, 6)),
        "batch": (5, lambda: H.Batch([(g, None, rays, H.HRPP_CLOSEST_HIT)])),
    }
    for name, (n_allocs, make) in makers.items():
        for k in range(n_allocs):
            monkeypatch.setenv("HRPP_FAIL_ALLOC_AFTER", str(k))
            with pytest.raises(H.HrppError) as err:
                make()
            assert err.value.status == H.HRPP_ERR_OOM, (name, k)
            monkeypatch.delenv("HRPP_FAIL_ALLOC_AFTER")
        obj = make()  # nothing left behind: the next creation works
        obj.close()
    for k in (0, 7, 20):
        monkeypatch.setenv("HRPP_FAIL_ALLOC_AFTER", str(k))
        with pytest.raises(H.HrppError) as err:
            H.Proposal.for_workload(g, s, seed=1)
        assert err.value.status == H.HRPP_ERR_OOM
        monkeypatch.delenv("HRPP_FAIL_ALLOC_AFTER")
    prop = H.Proposal.for_workload(g, s, seed=1)
    monkeypatch.setenv("HRPP_FAIL_ALLOC_AFTER", "2")
    with pytest.raises(H.HrppError) as err:
        prop.predict(rays)
    assert err.value.status == H.HRPP_ERR_OOM
    monkeypatch.delenv("HRPP_FAIL_ALLOC_AFTER")
    nodes, _ = prop.predict(rays)  # the half-made buffers were released
    traced, _ = H.trace(g, rays, H.HRPP_CLOSEST_HIT, predicted=nodes)
    plain, _ = H.trace(g, rays, H.HRPP_CLOSEST_HIT)
    torch.cuda.synchronize()
    assert torch.equal(traced.view(torch.int32), plain.view(torch.int32))


@pytest.mark.parametrize("go_up", [0, 1])
@pytest.mark.parametrize("width_idx", [0, 1])
def test_per_ray_outcomes_and_box_tests_match_oracle(H, small_pair, go_up, width_idx):
    """Per-ray outputs of a statistics launch: the outcome class (Sec. 4.3)
    and the box tests of the traversal from the root, ray by ray, equal the
    oracle's, for plain traversal and for HRPP over three frames."""
    import torch
    s, g = small_pair[width_idx]
    tab = H.Table(12, 2, 6, go_up=go_up)
    otab = O.Table(12, 2, 6, O.TWO_PHASE, go_up=go_up)
    for frame in range(3):
        prim = s.primary_rays(frame=frame)
        ph, _ = _oracle(s, prim, O.CLOSEST_HIT)
        shadow, _ = W.secondary_shadow(s, prim, ph["t"], ph["prim"])
        for mode, rays in ((O.CLOSEST_HIT, prim), (O.ANY_HIT, shadow)):
            for use_table in (False, True):
                if use_table and mode == O.ANY_HIT:
                    continue  # one table, fed by the closest-hit rays
                d = torch.from_numpy(rays).cuda()
                oc = torch.full((len(rays),), 255, dtype=torch.uint8, device="cuda")
                bx = torch.zeros(len(rays), dtype=torch.int32, device="cuda")
                _, ost, ooc, obx = O.trace(s.tris, s.nodes, s.prim_index, s.root, rays, mode,
                                           otab if use_table else None, per_ray=True)
                _, gst = H.trace(g, d, mode, tab if use_table else None, stats=True, ray_outcome=oc,
                                 ray_box_tests=bx)
                torch.cuda.synchronize()
                assert_same_stats(gst, ost)
                assert np.array_equal(oc.cpu().numpy(), ooc), (frame, mode, use_table)
                assert np.array_equal(bx.cpu().numpy().view(np.uint32), obx), (frame, mode, use_table)
    # without statistics the per-ray buffers are left alone
    oc = torch.full((len(prim),), 255, dtype=torch.uint8, device="cuda")
    H.trace(g, torch.from_numpy(prim).cuda(), H.HRPP_CLOSEST_HIT, tab, ray_outcome=oc)
    torch.cuda.synchronize()
    assert bool((oc == 255).all())
