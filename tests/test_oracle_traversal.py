"""Pins for the oracle's BVH traversal: it must return what brute force over
all triangles returns (the result's plain definition), on tiny scenes of every
awkward kind, for binary and 4-wide BVHs."""
import numpy as np
import pytest

import oracle as O
from paper_1910_01304_gb300 import scenes as S


def _tiny_scene(seed):
    rng = np.random.default_rng(seed)
    kind = seed % 4
    n = int(rng.integers(1, 65))
    if kind == 0:     # random soup in the unit cube
        tris = S.soup(n, seed, 0.0, 1.0, 0.3)
    elif kind == 1:   # coplanar, axis-aligned ground pieces sharing edges
        g = int(max(1, np.sqrt(n / 2)))
        tris = S.quad_grid(g, g, -1, 1, -1, 1, 0.0)
    elif kind == 2:   # soup with degenerate triangles mixed in
        tris = S.soup(n, seed, -1.0, 1.0, 0.5)
        k = rng.integers(0, n, max(1, n // 5))
        tris[k, 3:6] = tris[k, 0:3]                    # zero area
    else:             # a sphere piece plus stacked coincident planes
        tris = np.concatenate([S.icosphere(1, (0, 0, 0), 0.7)[: max(1, n // 2)],
                               S.quad_grid(2, 2, -1, 1, -1, 1, 0.1), S.quad_grid(2, 2, -1, 1, -1, 1, 0.1)])
    return np.ascontiguousarray(tris, np.float32)


def _rays(seed, n=96):
    rng = np.random.default_rng(1000 + seed)
    o = rng.uniform(-2, 2, (n, 3))
    tgt = rng.uniform(-1, 1, (n, 3))
    d = tgt - o
    d /= np.linalg.norm(d, axis=1, keepdims=True)
    r = np.zeros((n, 8), np.float32)
    r[:, 0:3], r[:, 4:7] = o, d
    r[:, 7] = np.inf
    # a few axis-parallel rays with exactly-zero components, and short rays
    r[::7, 4:7] = [0, -1, 0]
    r[1::11, 4:7] = [1, 0, 0]
    r[2::5, 7] = rng.uniform(0.1, 3.0, len(r[2::5]))
    return r


@pytest.mark.parametrize("method", ["sah", "median"])
@pytest.mark.parametrize("width", [2, 4])
def test_traversal_equals_brute_force(width, method):
    n_cmp = 0
    for seed in range(240):
        tris = _tiny_scene(seed)
        nodes, prim, root = S.build_bvh(tris, width=width, method=method)
        rays = _rays(seed)
        hc, _ = O.trace(tris, nodes, prim, root, rays, O.CLOSEST_HIT)
        bc, tie = O.brute(rays, tris, O.CLOSEST_HIT)
        ok = ~tie
        assert np.array_equal(hc["prim"][ok], bc["prim"][ok]), seed
        assert np.array_equal(hc["t"][ok], bc["t"][ok]), seed
        assert np.array_equal(hc["u"][ok], bc["u"][ok]) and np.array_equal(hc["v"][ok], bc["v"][ok])
        ha, _ = O.trace(tris, nodes, prim, root, rays, O.ANY_HIT)
        ba, _ = O.brute(rays, tris, O.ANY_HIT)
        assert np.array_equal(ha == O.NO_HIT, ba == O.NO_HIT), seed
        # the any-hit prim reported is a real hit of that ray
        for i in np.nonzero(ha != O.NO_HIT)[0]:
            tr = tris[ha[i]]
            assert O.ray_triangle(rays[i], tr[0:3], tr[3:6], tr[6:9])[0]
        n_cmp += int(ok.sum())
    assert n_cmp > 20000


def test_traversal_small_scene_vs_brute(small):
    rays = small.primary_rays()[::8]
    h, st = O.trace(small.tris, small.nodes, small.prim_index, small.root, rays, O.CLOSEST_HIT)
    b, tie = O.brute(rays, small.tris, O.CLOSEST_HIT)
    ok = ~tie
    assert np.array_equal(h[ok], b[ok])
    assert st["rays"] == len(rays) and st["hits"] == int(np.count_nonzero(h["prim"] != O.NO_HIT))
    # interior nodes each test two boxes in a binary BVH
    assert st["box_tests"] == 2 * st["interior_nodes"]
    assert st["lookups"] == 0 and st["positives"] == 0


def test_traversal_counts_binary_vs_wide(small, small4):
    rays = small.primary_rays()[::4]
    h2, s2 = O.trace(small.tris, small.nodes, small.prim_index, 0, rays, O.CLOSEST_HIT)
    h4, s4 = O.trace(small4.tris, small4.nodes, small4.prim_index, 0, rays, O.CLOSEST_HIT)
    assert np.array_equal(h2, h4)
    assert s4["interior_nodes"] < s2["interior_nodes"]
    assert s4["box_tests"] <= 4 * s4["interior_nodes"]


def test_root_leaf_scene():
    tris = S.soup(3, 1, 0, 1, 0.4)
    nodes, prim, root = S.build_bvh(tris, width=2, trav_cost=0.0)  # 3 triangles: one leaf
    assert len(nodes) == 1 and nodes[0]["count"] == 3
    rays = _rays(3, 64)
    h, st = O.trace(tris, nodes, prim, root, rays, O.CLOSEST_HIT)
    b, tie = O.brute(rays, tris, O.CLOSEST_HIT)
    assert np.array_equal(h[~tie], b[~tie])
    assert st["interior_nodes"] == 0 and st["leaves"] == len(rays)


def _hand_bvh():
    """Root -> A (two triangles at z = 0) and B (two at z = -5); each child
    holds two one-triangle leaves.  Boxes are exact, padded by 1e-3."""
    tris = np.array([[0, 0, 0, 1, 0, 0, 0, 1, 0],
                     [2, 0, 0, 3, 0, 0, 2, 1, 0],
                     [0, 0, -5, 1, 0, -5, 0, 1, -5],
                     [2, 0, -5, 3, 0, -5, 2, 1, -5]], np.float32)
    nodes = np.zeros(7, S.NODE_DTYPE)

    def box(ids):
        v = tris[ids].reshape(-1, 3)
        return v.min(0) - 1e-3, v.max(0) + 1e-3

    layout = {0: ([1, 2], [0, 1, 2, 3]), 1: ([3, 4], [0, 1]), 2: ([5, 6], [2, 3])}
    for i, (kids, ids) in layout.items():
        nodes[i]["lo"], nodes[i]["hi"] = box(ids)
        nodes[i]["child"] = kids + [-1, -1]
    for i, t in zip(range(3, 7), range(4)):
        nodes[i]["lo"], nodes[i]["hi"] = box([t])
        nodes[i]["child"] = [-1] * 4
        nodes[i]["first"], nodes[i]["count"] = t, 1
    return tris, nodes, np.arange(4, dtype=np.uint32)


def test_children_visited_nearest_first():
    tris, nodes, prim = _hand_bvh()
    r = np.array([[0.25, 0.25, 1.0, 0.0, 0.0, 0.0, -1.0, np.inf]], np.float32)
    h, st = O.trace(tris, nodes, prim, 0, r, O.CLOSEST_HIT)
    assert h["prim"][0] == 0 and h["t"][0] == 1.0
    # root, A, then B whose leaves lie beyond the hit: 3 interior nodes, 6 box
    # tests, only the near leaf entered
    assert (st["interior_nodes"], st["box_tests"], st["leaves"], st["tri_tests"]) == (3, 6, 1, 1)
    # any-hit stops at the first hit in the same nearest-first order
    a, sa = O.trace(tris, nodes, prim, 0, r, O.ANY_HIT)
    assert a[0] == 0 and (sa["interior_nodes"], sa["leaves"]) == (2, 1)
    # reversed ray: B is nearer now
    r2 = np.array([[0.25, 0.25, -6.0, 0.0, 0.0, 0.0, 1.0, np.inf]], np.float32)
    a2, _ = O.trace(tris, nodes, prim, 0, r2, O.ANY_HIT)
    assert a2[0] == 2


def test_exact_ties_go_to_the_lower_prim_id():
    base = S.soup(40, 9, 0, 1, 0.3)
    tris = np.ascontiguousarray(np.concatenate([base, base[::-1]]), np.float32)  # every triangle twice
    n = len(base)
    for width in (2, 4):
        nodes, prim, root = S.build_bvh(tris, width=width)
        rays = _rays(9, 200)
        h, _ = O.trace(tris, nodes, prim, root, rays, O.CLOSEST_HIT)
        b, tie = O.brute(rays, tris, O.CLOSEST_HIT)
        hit = h["prim"] != O.NO_HIT
        assert hit.sum() > 20 and tie[hit].all()
        # the duplicate of base[i] is prim 2n-1-i: the lower id is always < n
        assert np.all(h["prim"][hit] < n)
        assert np.array_equal(h["prim"], b["prim"]) and np.array_equal(h["t"], b["t"])


def test_equal_entry_children_visited_in_slot_order():
    """Two leaves with identical boxes: the one in the lower slot goes first."""
    tri = np.array([0, 0, 0, 1, 0, 0, 0, 1, 0], np.float32)
    tris = np.stack([tri, tri])
    nodes = np.zeros(3, S.NODE_DTYPE)
    lo, hi = np.array([-1e-3, -1e-3, -1e-3]), np.array([1.001, 1.001, 1e-3])
    for i in range(3):
        nodes[i]["lo"], nodes[i]["hi"] = lo, hi
        nodes[i]["child"] = [-1] * 4
    nodes[0]["child"] = [1, 2, -1, -1]
    nodes[1]["first"], nodes[1]["count"] = 0, 1   # slot 0 -> prim_index[0] = prim 1
    nodes[2]["first"], nodes[2]["count"] = 1, 1   # slot 1 -> prim_index[1] = prim 0
    prim = np.array([1, 0], np.uint32)
    r = np.array([[0.25, 0.25, 1.0, 0.0, 0.0, 0.0, -1.0, np.inf]], np.float32)
    a, sa = O.trace(tris, nodes, prim, 0, r, O.ANY_HIT)
    assert a[0] == 1 and sa["leaves"] == 1
    h, sc = O.trace(tris, nodes, prim, 0, r, O.CLOSEST_HIT)
    assert h["prim"][0] == 0 and sc["leaves"] == 2
