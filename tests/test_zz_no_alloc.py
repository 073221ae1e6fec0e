"""hrpp_trace_noalloc against hrpp_trace.

hrpp_trace_noalloc exists for callers that cannot allocate device memory
during tracing: engines whose own allocator reserved all device memory up
front, or real-time loops that ban allocation calls because they can stall
or synchronise the device.  It must give exactly what hrpp_trace gives
(bit-identical hits, counters and table words; the same tolerance every
parity test here uses), call after call, with its scratch in the library's
fixed device array.  This file is collected last on purpose.
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


def _call(H, fn, scene, table, rays, mode, hits, stats):
    rc = fn(scene.handle, table.handle if table is not None else None, H._ptr(rays), rays.shape[0], mode,
            H._ptr(hits), ctypes.byref(stats), None)
    assert rc == H.HRPP_OK, H.hrpp_last_error()


@pytest.mark.parametrize("mode_name", ["closest", "any"])
@pytest.mark.parametrize("with_table", [False, True])
def test_noalloc_matches_trace_two_calls_in_a_row(mode_name, with_table):
    torch, H, W = _setup()
    s = W.small_scene(width=4)
    g = H.Scene.from_workload(s)
    mode = H.HRPP_CLOSEST_HIT if mode_name == "closest" else H.HRPP_ANY_HIT
    t_ref = H.Table(12, 2, 6) if with_table else None
    t_new = H.Table(12, 2, 6) if with_table else None
    for frame in (1, 2):
        rays = torch.from_numpy(s.primary_rays(frame=frame)).cuda()
        shape = (rays.shape[0], 4) if mode == H.HRPP_CLOSEST_HIT else (rays.shape[0],)
        dtype = torch.float32 if mode == H.HRPP_CLOSEST_HIT else torch.int32
        h_ref = torch.empty(shape, dtype=dtype, device="cuda")
        h_new = torch.full(shape, 7, dtype=dtype, device="cuda")
        s_ref, s_new = H.hrpp_stats(), H.hrpp_stats()
        _call(H, H.hrpp_trace, g, t_ref, rays, mode, h_ref, s_ref)
        _call(H, H.hrpp_trace_noalloc, g, t_new, rays, mode, h_new, s_new)
        torch.cuda.synchronize()
        a = h_ref.cpu().numpy().view(np.uint32)
        b = h_new.cpu().numpy().view(np.uint32)
        assert np.array_equal(a, b), f"frame {frame}: hits differ"
        assert s_ref.as_dict() == s_new.as_dict(), f"frame {frame}: counters differ"
        if with_table:
            assert np.array_equal(t_ref.export(), t_new.export()), f"frame {frame}: table words differ"
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
