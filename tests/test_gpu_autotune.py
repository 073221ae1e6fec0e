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
