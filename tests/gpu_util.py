"""Helpers shared by the GPU tests: run the CUDA path through the C ABI and
compare with the oracle bit for bit."""
import numpy as np

import oracle as O

STAT_KEYS = ["rays", "hits", "lookups", "positives", "true_pos", "false_pos", "negatives", "tp_inexact",
             "inserts", "dup_inserts", "evictions", "interior_nodes", "box_tests", "leaves", "tri_tests",
             "pred_leaves", "pred_tri_tests", "pred_interior_nodes", "pred_box_tests", "gated"]


def hrpp_mod():
    from paper_1910_01304_gb300 import build
    build.build()
    from paper_1910_01304_gb300 import hrpp
    return hrpp


def gpu_trace(H, scene, rays_np, mode, table=None, stats=True, block_threads=0):
    import torch
    rays = torch.from_numpy(np.ascontiguousarray(rays_np, np.float32)).cuda()
    hits, st = H.trace(scene, rays, mode, table=table, stats=stats, block_threads=block_threads)
    torch.cuda.synchronize()
    scene.check()
    h = hits.cpu().numpy()
    return h, st


def as_words(closest_hits):
    """Closest-hit results as raw uint32 [n, 4] (t, prim, u, v) bit patterns."""
    if closest_hits.dtype == O.HIT_DTYPE:
        return closest_hits.view(np.uint32).reshape(-1, 4)
    return np.ascontiguousarray(closest_hits, np.float32).view(np.uint32).reshape(-1, 4)


def any_prims(h):
    return np.ascontiguousarray(h).view(np.uint32).reshape(-1)


def assert_same_hits(mode, gpu_hits, oracle_hits, msg=""):
    if mode == O.CLOSEST_HIT:
        g, o = as_words(gpu_hits), as_words(oracle_hits)
        bad = np.nonzero((g != o).any(axis=1))[0]
        assert len(bad) == 0, f"{msg}: {len(bad)} closest-hit rays differ, first {bad[:5]}: gpu {g[bad[:3]]} oracle {o[bad[:3]]}"
    else:
        g, o = any_prims(gpu_hits), any_prims(oracle_hits)
        bad = np.nonzero(g != o)[0]
        assert len(bad) == 0, f"{msg}: {len(bad)} any-hit rays differ, first {bad[:5]}: gpu {g[bad[:3]]} oracle {o[bad[:3]]}"


def assert_same_stats(gpu_stats, oracle_stats, keys=STAT_KEYS, msg=""):
    diff = {k: (gpu_stats[k], oracle_stats[k]) for k in keys if gpu_stats[k] != oracle_stats[k]}
    assert not diff, f"{msg}: counters differ (gpu, oracle): {diff}"


def oracle_table_like(t):
    return O.Table(t.log2_entries, t.ways, t.precision, O.TWO_PHASE, go_up=getattr(t, "go_up", 0))
