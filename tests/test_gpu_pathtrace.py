"""Incoherent path tracing (the config-5 recipe at reduced size): five
diffuse bounces with a shadow ray per bounce, traced through one HRPP table
per query mode shared by all bounces, against the oracle bounce by bounce."""
import numpy as np
import pytest

import oracle as O
from gpu_util import assert_same_hits, assert_same_stats, gpu_trace, hrpp_mod
from paper_1910_01304_gb300.scenes import workloads as W

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("go_up", [0, 1])
def test_pathtrace_bounces_match_oracle(go_up):
    H = hrpp_mod()
    s = W.pathtrace_scene(quads=(96, 48), n_spheres=12, res=(128, 72), dome_subdiv=2)
    g = H.Scene.from_workload(s)
    tabs = {m: H.Table(14, 2, 6, go_up=go_up) for m in (O.CLOSEST_HIT, O.ANY_HIT)}
    otabs = {m: O.Table(14, 2, 6, O.TWO_PHASE, go_up=go_up) for m in (O.CLOSEST_HIT, O.ANY_HIT)}

    def oracle_closest(rays):
        h, _ = O.trace(s.tris, s.nodes, s.prim_index, s.root, rays, O.CLOSEST_HIT)
        return h["t"], h["prim"]

    for frame in range(2):
        bounces = W.path_bounces(s, W.path_primary(s, spp=2, frame=frame), oracle_closest, bounces=5, frame=frame)
        assert len(bounces) == 5
        for b, (closest, shadow) in enumerate(bounces):
            for mode, rays in ((O.CLOSEST_HIT, closest), (O.ANY_HIT, shadow)):
                oh, ost = O.trace(s.tris, s.nodes, s.prim_index, s.root, rays, mode, otabs[mode])
                gh, gst = gpu_trace(H, g, rays, mode, tabs[mode])
                assert_same_hits(mode, gh, oh, f"frame {frame} bounce {b}")
                assert_same_stats(gst, ost, msg=f"frame {frame} bounce {b} mode {mode}")
                assert np.array_equal(tabs[mode].export(), otabs[mode].words)
