"""Checks on the seeded input generators: sizes, determinism, BVH validity,
and PCG32 against its published reference sequence."""
import numpy as np
import pytest

from paper_1910_01304_gb300 import scenes as S
from paper_1910_01304_gb300.scenes import workloads as W


def test_pcg32_reference_sequence():
    # pcg32 demo (O'Neill): seed 42, sequence 54
    ref = [0xA15C02B7, 0x7B47F409, 0xBA1D3330, 0x83D2F293, 0xBFA4784B, 0xCBED606E]
    assert list(S.pcg32_stream(42, 54, 6)) == ref


def test_sizes():
    assert S.icosphere(3).shape == (1280, 9)
    assert S.icosphere(5).shape == (20480, 9)
    assert S.quad_grid(16, 16, -4, 4, -4, 4).shape == (512, 9)
    sph = S.icosphere(2, (1, 2, 3), 0.5)
    r = np.linalg.norm(sph.reshape(-1, 3) - np.array([1, 2, 3], np.float32), axis=1)
    assert np.allclose(r, 0.5, atol=1e-6)


def _validate(nodes, prim, n_tris, tris, width):
    seen = np.zeros(n_tris, np.int32)
    reached = np.zeros(len(nodes), np.int32)
    stack = [0]
    reached[0] = 1
    while stack:
        i = stack.pop()
        n = nodes[i]
        if n["count"] > 0:
            assert n["count"] <= 4
            ids = prim[n["first"]:n["first"] + n["count"]]
            seen[ids] += 1
            v = tris[ids].reshape(-1, 3)
            assert np.all(v >= n["lo"]) and np.all(v <= n["hi"])
            continue
        kids = [c for c in n["child"] if c >= 0]
        assert 1 <= len(kids) <= width
        for c in kids:
            assert np.all(nodes[c]["lo"] >= n["lo"]) and np.all(nodes[c]["hi"] <= n["hi"])
            reached[c] += 1
            stack.append(c)
    assert np.all(seen == 1)
    assert np.all(reached == 1)


@pytest.mark.parametrize("method,trav_cost", [("sah", 1.0), ("sah", 0.0), ("median", 0.0)])
@pytest.mark.parametrize("width", [2, 4])
def test_bvh_valid(width, method, trav_cost):
    for seed in range(5):
        tris = S.soup(300 + 37 * seed, seed)
        nodes, prim, root = S.build_bvh(tris, width=width, method=method, trav_cost=trav_cost)
        _validate(nodes, prim, len(tris), tris, width)
        if method == "sah" and trav_cost == 0.0:
            # without the leaf cost every node of <= 4 triangles is a leaf
            kids = nodes["child"][nodes["count"] == 0]
            sizes = [nodes["count"][c] for row in kids for c in row if c >= 0 and nodes["count"][c] > 0]
            assert min(sizes) >= 1
    s = W.small_scene(width=width)
    _validate(s.nodes, s.prim_index, s.n_tris, s.tris, width)


def test_boxes_are_padded():
    s = W.small_scene()
    leaf = s.nodes[s.nodes["count"] > 0]
    # ground leaves are flat in y; padding gives them thickness
    assert np.all(leaf["hi"][:, 1] > leaf["lo"][:, 1])


def test_deterministic():
    a = W.small_scene()
    b = W.small_scene()
    assert a.tris.tobytes() == b.tris.tobytes() and a.nodes.tobytes() == b.nodes.tobytes()
    assert a.primary_rays(frame=3).tobytes() == b.primary_rays(frame=3).tobytes()
    assert a.primary_rays(frame=0).tobytes() != a.primary_rays(frame=1).tobytes()


def test_secondary_rays():
    s = W.small_scene()
    rays = s.primary_rays()[:4096]
    import oracle as O
    h, _ = O.trace(s.tris, s.nodes, s.prim_index, 0, rays, O.CLOSEST_HIT)
    sh, src = W.secondary_shadow(s, rays, h["t"], h["prim"])
    assert len(sh) == int(np.count_nonzero(h["prim"] != O.NO_HIT))
    assert np.allclose(np.linalg.norm(sh[:, 4:7], axis=1), 1, atol=1e-6)
    ao, src2 = W.secondary_ao(s, rays, h["t"], h["prim"])
    assert len(ao) == 4 * len(sh) and np.all(ao[:, 7] == np.float32(0.5))


def test_sah_tree_is_cheaper_than_median():
    """The surface-area heuristic's own cost, summed over the interior nodes
    (area of each node over the root's), is lower for the SAH tree than for
    the median-split tree of the same scene, and both trees are equally
    deterministic.  Degenerate input (every centroid equal) still builds."""
    s = W.small_scene(width=2)

    def cost(nodes):
        a = nodes["hi"] - nodes["lo"]
        area = 2 * (a[:, 0] * a[:, 1] + a[:, 1] * a[:, 2] + a[:, 2] * a[:, 0])
        return float(area[nodes["count"] == 0].sum() / area[0])

    sah, _, _ = S.build_bvh(s.tris, width=2, method="sah")
    med, _, _ = S.build_bvh(s.tris, width=2, method="median")
    assert cost(sah) < cost(med)
    again, _, _ = S.build_bvh(s.tris, width=2, method="sah")
    assert again.tobytes() == sah.tobytes()
    same = np.tile(np.array([0, 0, 0, 1, 0, 0, 0, 1, 0], np.float32), (50, 1))
    nodes, prim, root = S.build_bvh(same, width=4)
    _validate(nodes, prim, len(same), same, 4)
    # the leaf cost splits small nodes only where that is cheaper: leaves get
    # smaller on average, never larger than max_leaf
    split, _, _ = S.build_bvh(s.tris, width=2, method="sah", trav_cost=1.0)
    fixed, _, _ = S.build_bvh(s.tris, width=2, method="sah", trav_cost=0.0)
    leaf = lambda n: n["count"][n["count"] > 0]
    assert leaf(split).max() <= 4 and leaf(split).mean() < leaf(fixed).mean()
    with pytest.raises(ValueError):
        S.build_bvh(s.tris, method="other")
