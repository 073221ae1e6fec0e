"""The autotuner returns a configuration and never changes a result (it
asserts bit-identical hits across every candidate it times)."""
import pytest

from gpu_util import hrpp_mod
from paper_1910_01304_gb300.scenes import workloads as W

pytestmark = pytest.mark.gpu


def test_autotune_small_scene():
    import numpy as np
    import torch
    H = hrpp_mod()
    from paper_1910_01304_gb300 import autotune
    s = W.small_scene(width=4)
    g = H.Scene.from_workload(s)
    warm = torch.from_numpy(s.primary_rays(frame=1)).cuda()
    ev = torch.from_numpy(s.primary_rays(frame=2)).cuda()
    grid = dict(log2_entries=(10, 12), ways=(1, 2), precision=(5, 6), go_up=(0, 1))
    r = autotune.tune(g, warm, ev, H.HRPP_CLOSEST_HIT, grid, reps=3,
                      launch_grid=[dict(block_threads=128, schedule=1), dict(block_threads=64, schedule=2)])
    assert r["rays"] == ev.shape[0] and r["plain_ms"] > 0 and r["best_ms"] > 0
    assert len(r["table_times"]) == 16
    if r["best_table"] is not None:
        assert r["best_ms"] <= r["plain_ms"]


def test_tune_batch_and_warm_snapshot_protocol():
    """The batched autotuner on a small uneven batch: it returns a
    configuration from its grid (every candidate gave identical results, or
    it would have raised), and a BatchSetup step with the tuned tables
    returns exactly the plain hits, step after step."""
    import numpy as np
    import torch
    H = hrpp_mod()
    from paper_1910_01304_gb300 import autotune
    items, frames = [], [[], [], []]
    for s, rays in W.batched_workload(n_scenes=6, tris_range=(2000, 20_000), rays_range=(2000, 20_000), seed=4):
        g = H.Scene.from_workload(s)
        half = len(rays) // 2
        per_frame = [rays] + [W.batched_rays(s, len(rays), f) for f in (1, 2)]
        for lo, hi, mode in ((0, half, H.HRPP_CLOSEST_HIT), (half, len(rays), H.HRPP_ANY_HIT)):
            items.append((g, mode))
            for f, r in enumerate(per_frame):
                frames[f].append(torch.from_numpy(np.ascontiguousarray(r[lo:hi])).cuda())
    grid = [None, dict(log2_entries=12, ways=1, precision=6), dict(log2_entries=14, ways=2, precision=5)]
    r = autotune.tune_batch(items, frames, table_grid=grid, block_grid=(128,), reps=2)
    assert r["block_threads"] == 128 and r["closest"] in grid and r["any"] in grid
    assert len(r["tried"]) == 1 + 2 * 2
    plain = autotune.BatchSetup(items, frames, None, None, 128)
    plain.step()
    cfg = grid[1]
    tuned = autotune.BatchSetup(items, frames, cfg, cfg, 128)
    for _ in range(2):
        tuned.step()
        torch.cuda.synchronize()
        for (_, mode), a, b in zip(items, plain.hits(), tuned.hits()):
            if mode == H.HRPP_CLOSEST_HIT:
                assert torch.equal(a.view(torch.int32), b.view(torch.int32))
            else:
                assert torch.equal(a == -1, b == -1)
    plain.close()
    tuned.close()
