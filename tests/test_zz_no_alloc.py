"""hrpp_trace_noalloc against hrpp_trace.

hrpp_trace_noalloc exists for callers that cannot allocate device memory
during tracing: engines whose own allocator reserved all device memory up
front, or real-time loops that ban allocation calls because they can stall
or synchronise the device.  It must give exactly what hrpp_trace gives
(bit-identical hits, counters and table words; the same tolerance every
parity test here uses) and the same status, call after call, with its
scratch in the library's fixed device array.  This file is collected last on
purpose.
"""
import ctypes

import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def _setup():
    import torch
    from paper_1910_01304_gb300 import build
    build.build()
    from paper_1910_01304_gb300 import hrpp as H
    from paper_1910_01304_gb300.scenes import workloads as W
    return torch, H, W


def _stats_buffer(torch, H, where):
    """hrpp_stats in host memory (a ctypes struct) or device memory (20
    uint64 words in a torch tensor); returns (pointer, reader)."""
    if where == "host":
        st = H.hrpp_stats()
        return ctypes.byref(st), lambda: st.as_dict()
    dev = torch.full((20,), -1, dtype=torch.int64, device="cuda")

    def read():
        v = dev.cpu().numpy().view(np.uint64)
        return {k: int(v[i]) for i, k in enumerate(H.STAT_NAMES)}
    return dev.data_ptr(), read


def _call(H, fn, scene, table, rays, mode, hits, stats_ptr):
    return fn(scene.handle, table.handle if table is not None else None, H._ptr(rays), rays.shape[0], mode,
              H._ptr(hits), stats_ptr, None)


def _hits_like(torch, H, n, mode, fill):
    shape = (n, 4) if mode == H.HRPP_CLOSEST_HIT else (n,)
    dtype = torch.float32 if mode == H.HRPP_CLOSEST_HIT else torch.int32
    return torch.full(shape, fill, dtype=dtype, device="cuda")


@pytest.mark.parametrize("stats_where", ["host", "device"])
@pytest.mark.parametrize("width", [2, 4])
@pytest.mark.parametrize("mode_name", ["closest", "any"])
@pytest.mark.parametrize("with_table", [False, True, "gated"])
def test_noalloc_matches_trace_two_calls_in_a_row(mode_name, with_table, width, stats_where):
    torch, H, W = _setup()
    s = W.small_scene(width=width)
    g = H.Scene.from_workload(s)
    mode = H.HRPP_CLOSEST_HIT if mode_name == "closest" else H.HRPP_ANY_HIT
    t_ref = H.Table(12, 2, 6) if with_table else None
    t_new = H.Table(12, 2, 6) if with_table else None
    if with_table == "gated":  # a gate that closes after the first call
        t_ref.set_gate(65536, 2)
        t_new.set_gate(65536, 2)
    for frame in (1, 2):
        rays = torch.from_numpy(s.primary_rays(frame=frame)).cuda()
        h_ref = _hits_like(torch, H, rays.shape[0], mode, 0)
        h_new = _hits_like(torch, H, rays.shape[0], mode, 7)
        p_ref, read_ref = _stats_buffer(torch, H, stats_where)
        p_new, read_new = _stats_buffer(torch, H, stats_where)
        assert _call(H, H.hrpp_trace, g, t_ref, rays, mode, h_ref, p_ref) == H.HRPP_OK, H.hrpp_last_error()
        assert _call(H, H.hrpp_trace_noalloc, g, t_new, rays, mode, h_new, p_new) == H.HRPP_OK, H.hrpp_last_error()
        torch.cuda.synchronize()
        a = h_ref.cpu().numpy().view(np.uint32)
        b = h_new.cpu().numpy().view(np.uint32)
        assert np.array_equal(a, b), f"frame {frame}: hits differ"
        assert read_ref() == read_new(), f"frame {frame}: counters differ"
        if with_table:
            assert np.array_equal(t_ref.export(), t_new.export()), f"frame {frame}: table words differ"
            assert t_ref.gate_open() == t_new.gate_open()
    g.check()


def _scattered_rays(n, seed):
    """n rays from random points above the small scene's ground, each aimed at
    a random ground point: nearly every ray hits and nearly every ray has its
    own hash key, so nearly every ray of a call leaves an insert record."""
    rng = np.random.default_rng(seed)
    o = np.stack([rng.uniform(-3.9, 3.9, n), rng.uniform(2.2, 3.5, n), rng.uniform(-3.9, 3.9, n)], 1)
    tgt = np.stack([rng.uniform(-3.9, 3.9, n), np.zeros(n), rng.uniform(-3.9, 3.9, n)], 1)
    d = tgt - o
    d /= np.linalg.norm(d, axis=1, keepdims=True)
    rays = np.zeros((n, 8), np.float32)
    rays[:, 0:3] = o
    rays[:, 4:7] = d
    rays[:, 7] = np.inf
    return rays


@pytest.mark.parametrize("width", [2, 4])
def test_noalloc_at_its_maximum_batch_fills_the_record_array(width):
    """Two calls of exactly HRPP_NOALLOC_MAX_RAYS rays with a two-phase table:
    the insert records run to the end of the fixed array, and hits, counters
    and table words still equal hrpp_trace's."""
    torch, H, W = _setup()
    s = W.small_scene(width=width)
    g = H.Scene.from_workload(s)
    n = H.HRPP_NOALLOC_MAX_RAYS
    t_ref, t_new = H.Table(20, 1, 7), H.Table(20, 1, 7)
    for call in range(2):
        rays = torch.from_numpy(_scattered_rays(n, seed=100 + call)).cuda()
        h_ref = _hits_like(torch, H, n, H.HRPP_CLOSEST_HIT, 0)
        h_new = _hits_like(torch, H, n, H.HRPP_CLOSEST_HIT, 7)
        s_ref, s_new = H.hrpp_stats(), H.hrpp_stats()
        rc = _call(H, H.hrpp_trace, g, t_ref, rays, H.HRPP_CLOSEST_HIT, h_ref, ctypes.byref(s_ref))
        assert rc == H.HRPP_OK, H.hrpp_last_error()
        rc = _call(H, H.hrpp_trace_noalloc, g, t_new, rays, H.HRPP_CLOSEST_HIT, h_new, ctypes.byref(s_new))
        assert rc == H.HRPP_OK, H.hrpp_last_error()
        torch.cuda.synchronize()
        assert torch.equal(h_ref.view(torch.int32), h_new.view(torch.int32)), f"call {call}: hits differ"
        assert s_ref.as_dict() == s_new.as_dict(), f"call {call}: counters differ"
        assert np.array_equal(t_ref.export(), t_new.export()), f"call {call}: table words differ"
        # records: every insert that was not merged inside its warp; nearly
        # all rays insert here, so the array is filled nearly to its end
        assert s_new.rays == n
        assert s_new.inserts > 0.9 * n, s_new.as_dict()
    g.check()


def test_noalloc_allocates_nothing(monkeypatch):
    """With every device allocation refused (HRPP_FAIL_ALLOC_AFTER=0, the
    library's host-side fault injection), hrpp_trace cannot get its scratch
    and returns HRPP_ERR_OOM, while hrpp_trace_noalloc still returns HRPP_OK
    with exactly hrpp_trace's results, counters and table words."""
    torch, H, W = _setup()
    s = W.small_scene(width=4)
    g = H.Scene.from_workload(s)
    t_ref, t_new = H.Table(12, 2, 6), H.Table(12, 2, 6)
    rays = torch.from_numpy(s.primary_rays(frame=3)).cuda()
    n = rays.shape[0]
    for frame in range(2):
        h_ref = _hits_like(torch, H, n, H.HRPP_CLOSEST_HIT, 0)
        h_new = _hits_like(torch, H, n, H.HRPP_CLOSEST_HIT, 7)
        s_ref, s_new = H.hrpp_stats(), H.hrpp_stats()
        rc = _call(H, H.hrpp_trace, g, t_ref, rays, H.HRPP_CLOSEST_HIT, h_ref, ctypes.byref(s_ref))
        assert rc == H.HRPP_OK, H.hrpp_last_error()
        monkeypatch.setenv("HRPP_FAIL_ALLOC_AFTER", "0")
        try:
            rc = _call(H, H.hrpp_trace, g, t_new, rays, H.HRPP_CLOSEST_HIT, h_new, ctypes.byref(s_new))
            assert rc == H.HRPP_ERR_OOM, "hrpp_trace allocated scratch although every allocation was refused"
            rc = _call(H, H.hrpp_trace_noalloc, g, t_new, rays, H.HRPP_CLOSEST_HIT, h_new, ctypes.byref(s_new))
            assert rc == H.HRPP_OK, H.hrpp_last_error()
        finally:
            monkeypatch.delenv("HRPP_FAIL_ALLOC_AFTER")
        torch.cuda.synchronize()
        assert torch.equal(h_ref.view(torch.int32), h_new.view(torch.int32)), f"frame {frame}: hits differ"
        assert s_ref.as_dict() == s_new.as_dict(), f"frame {frame}: counters differ"
        assert np.array_equal(t_ref.export(), t_new.export()), f"frame {frame}: table words differ"
    g.check()


def test_noalloc_reports_a_stopped_ray_as_trace_does():
    """A ray stopped early leaves the scene's error flag set.  The next call
    that waits (host out_stats) reports HRPP_ERR_TRAVERSAL_LIMIT and clears
    the flag, for hrpp_trace and hrpp_trace_noalloc alike; a call that does
    not wait leaves the flag to hrpp_scene_check."""
    torch, H, W = _setup()
    s = W.small_scene(width=2)
    g = H.Scene.from_workload(s)
    rays = torch.from_numpy(s.primary_rays(frame=0)).cuda()
    n = rays.shape[0]
    for fn in (H.hrpp_trace, H.hrpp_trace_noalloc):
        H.trace(g, rays, H.HRPP_CLOSEST_HIT, max_steps=3)  # sets the flag, does not wait
        hits = _hits_like(torch, H, n, H.HRPP_CLOSEST_HIT, 0)
        st = H.hrpp_stats()
        rc = _call(H, fn, g, None, rays, H.HRPP_CLOSEST_HIT, hits, ctypes.byref(st))
        assert rc == H.HRPP_ERR_TRAVERSAL_LIMIT, (fn.__name__, rc)
        g.check()  # cleared by the call that reported it
        rc = _call(H, fn, g, None, rays, H.HRPP_CLOSEST_HIT, hits, ctypes.byref(st))
        assert rc == H.HRPP_OK, (fn.__name__, H.hrpp_last_error())
        # without host statistics the call does not wait: the flag waits for
        # hrpp_scene_check
        H.trace(g, rays, H.HRPP_CLOSEST_HIT, max_steps=3)
        assert _call(H, fn, g, None, rays, H.HRPP_CLOSEST_HIT, hits, None) == H.HRPP_OK
        with pytest.raises(H.HrppError) as err:
            g.check()
        assert err.value.status == H.HRPP_ERR_TRAVERSAL_LIMIT
        g.check()


def test_noalloc_rejects_batches_above_its_limit():
    torch, H, W = _setup()
    s = W.small_scene()
    g = H.Scene.from_workload(s)
    n = H.HRPP_NOALLOC_MAX_RAYS + 1
    rc = H.hrpp_trace_noalloc(g.handle, None, None, n, H.HRPP_CLOSEST_HIT, None, None, None)
    assert rc == H.HRPP_ERR_INVALID_ARG
    assert b"no-allocation limit" in H.hrpp_last_error()
    # host buffers would need staging: refused rather than allocated
    rays = np.ascontiguousarray(s.primary_rays()[:64])
    hits = np.empty((64, 4), np.float32)
    rc = H.hrpp_trace_noalloc(g.handle, None, H._ptr(rays), 64, H.HRPP_CLOSEST_HIT, H._ptr(hits), None, None)
    assert rc == H.HRPP_ERR_INVALID_ARG
