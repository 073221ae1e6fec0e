"""Pins for the oracle's ray-triangle and ray-box tests.

Pinned against closed forms (hand-placed triangles and boxes), and against an
independent double-precision solution (numpy.linalg.solve of o + t d = v0 + u
e1 + v e2; a slab test in float64) on random cases away from the boundaries.
"""
import numpy as np
import pytest

import oracle as O

V0, V1, V2 = (0.0, 0.0, 0.0), (1.0, 0.0, 0.0), (0.0, 1.0, 0.0)


def ray(o, d, tmin=0.0, tmax=np.inf):
    return np.array([*o, tmin, *d, tmax], np.float32)


def test_triangle_closed_form_barycentrics():
    hit, t, u, v = O.ray_triangle(ray((0.25, 0.5, 2.0), (0, 0, -1)), V0, V1, V2)
    assert hit and t == 2.0 and u == 0.25 and v == 0.5
    # u weights v1 (the x axis here), v weights v2: swapping the vertices swaps them
    hit, t, u, v = O.ray_triangle(ray((0.25, 0.5, 2.0), (0, 0, -1)), V0, V2, V1)
    assert hit and u == 0.5 and v == 0.25
    # oblique ray: o + t d = (0.125, 0.25, 0) at t = 4
    d = np.array([0.125 - 1.125, 0.25 - 0.25, -4.0]) / 4.0
    hit, t, u, v = O.ray_triangle(ray((1.125, 0.25, 4.0), d), V0, V1, V2)
    assert hit and abs(t - 4.0) < 1e-6 and abs(u - 0.125) < 1e-6 and abs(v - 0.25) < 1e-6


def test_triangle_two_sided_and_translation():
    hit, t, *_ = O.ray_triangle(ray((0.2, 0.2, -3.0), (0, 0, 1)), V0, V1, V2)
    assert hit and t == 3.0
    off = np.array([10.0, -4.0, 2.0])
    hit, t, u, v = O.ray_triangle(ray(off + (0.25, 0.5, 2.0), (0, 0, -1)), off + V0, off + V1, off + V2)
    assert hit and t == 2.0 and u == 0.25 and v == 0.5


def test_triangle_edges_inclusive():
    for o in [(0.0, 0.5), (0.5, 0.0), (0.5, 0.5), (0.0, 0.0), (1.0, 0.0), (0.0, 1.0)]:
        hit, *_ = O.ray_triangle(ray((o[0], o[1], 1.0), (0, 0, -1)), V0, V1, V2)
        assert hit, o
    for o in [(-1e-6, 0.5), (0.5, -1e-6), (0.5 + 1e-6, 0.5), (1.0, 1e-6)]:
        hit, *_ = O.ray_triangle(ray((o[0], o[1], 1.0), (0, 0, -1)), V0, V1, V2)
        assert not hit, o


def test_triangle_interval_is_open():
    r = ray((0.2, 0.2, 1.0), (0, 0, -1), tmin=0.0, tmax=1.0)
    assert not O.ray_triangle(r, V0, V1, V2)[0]          # t == tmax
    r = ray((0.2, 0.2, 1.0), (0, 0, -1), tmin=1.0, tmax=5.0)
    assert not O.ray_triangle(r, V0, V1, V2)[0]          # t == tmin
    r = ray((0.2, 0.2, 1.0), (0, 0, -1), tmin=0.0, tmax=np.nextafter(np.float32(1.0), np.float32(2.0)))
    assert O.ray_triangle(r, V0, V1, V2)[0]
    r = ray((0.2, 0.2, 1.0), (0, 0, 1))                   # behind the origin
    assert not O.ray_triangle(r, V0, V1, V2)[0]


def test_triangle_parallel_and_degenerate():
    assert not O.ray_triangle(ray((0.2, 0.2, 0.0), (1, 0, 0)), V0, V1, V2)[0]   # in-plane: det == 0
    assert not O.ray_triangle(ray((0.2, 0.2, 1.0), (1, 0, 0)), V0, V1, V2)[0]   # parallel above
    assert not O.ray_triangle(ray((0.2, 0.2, 1.0), (0, 0, -1)), V0, V0, V2)[0]  # zero area


def test_triangle_against_float64_solve():
    rng = np.random.default_rng(11)
    agree = 0
    for _ in range(3000):
        v = rng.normal(size=(3, 3)).astype(np.float32)
        o = rng.normal(size=3).astype(np.float32) * 3
        d = rng.normal(size=3).astype(np.float32)
        d /= np.linalg.norm(d)
        d = d.astype(np.float32)
        e1, e2 = v[1].astype(np.float64) - v[0], v[2].astype(np.float64) - v[0]
        A = np.stack([-d.astype(np.float64), e1, e2], axis=1)
        if abs(np.linalg.det(A)) < 1e-3:
            continue
        t, u, w = np.linalg.solve(A, o.astype(np.float64) - v[0])
        margin = min(u, w, 1 - u - w, t)
        hit, tf, uf, vf = O.ray_triangle(ray(o, d), v[0], v[1], v[2])
        if abs(margin) < 1e-4:
            continue
        assert hit == (margin > 0), (u, w, t)
        if hit:
            assert abs(tf - t) <= 1e-4 * max(1.0, abs(t))
            assert abs(uf - u) <= 1e-4 and abs(vf - w) <= 1e-4
        agree += 1
    assert agree > 2500


def test_box_closed_forms():
    lo, hi = (0, 0, 0), (1, 1, 1)
    hit, tn = O.ray_box(ray((0.5, 0.5, -1.0), (0, 0, 1)), lo, hi)
    assert hit and tn == 1.0
    hit, tn = O.ray_box(ray((0.5, 0.5, 0.5), (0, 0, 1)), lo, hi)       # origin inside: tn = tmin
    assert hit and tn == 0.0
    assert not O.ray_box(ray((0.5, 0.5, -1.0), (0, 0, -1)), lo, hi)[0]  # pointing away
    assert not O.ray_box(ray((1.5, 0.5, -1.0), (0, 0, 1)), lo, hi)[0]   # parallel, outside the x slab
    assert not O.ray_box(ray((0.5, 0.5, -1.0), (0, 0, 1)), lo, hi, tcur=0.5)[0]  # bound before entry
    assert O.ray_box(ray((0.5, 0.5, -1.0), (0, 0, 1)), lo, hi, tcur=1.0)[0]      # bound at entry: inclusive
    # on the lower face plane of x, moving inside it
    assert O.ray_box(ray((0.0, 0.5, -1.0), (0, 0, 1)), lo, hi)[0]
    # zero-thickness box (a flat ground) hit head-on
    hit, tn = O.ray_box(ray((0.5, 1.0, 0.5), (0, -1, 0)), (0, 0, 0), (1, 0, 1))
    assert hit and tn == 1.0
    # diagonal entry through an edge
    d = np.array([1, 1, 0], np.float32) / np.sqrt(np.float32(2))
    hit, tn = O.ray_box(ray((-1.0, -1.0, 0.5), d), lo, hi)
    assert hit and abs(tn - np.sqrt(2)) < 1e-6


def test_box_against_float64_slabs():
    rng = np.random.default_rng(5)
    n_checked = 0
    for _ in range(5000):
        c = rng.normal(size=3)
        ext = np.abs(rng.normal(size=3)) + 0.01
        lo, hi = (c - ext).astype(np.float32), (c + ext).astype(np.float32)
        o = (rng.normal(size=3) * 3).astype(np.float32)
        d = rng.normal(size=3)
        d = (d / np.linalg.norm(d)).astype(np.float32)
        with np.errstate(divide="ignore", invalid="ignore"):
            inv = 1.0 / d.astype(np.float64)
            t0 = (lo.astype(np.float64) - o) * inv
            t1 = (hi.astype(np.float64) - o) * inv
        tn = max(np.max(np.minimum(t0, t1)), 0.0)
        tf = np.min(np.maximum(t0, t1))
        if abs(tn - tf) < 1e-5 * max(1.0, abs(tn)):
            continue
        hit, tn32 = O.ray_box(ray(o, d), lo, hi)
        assert hit == (tn <= tf)
        if hit:
            assert abs(tn32 - tn) <= 1e-5 * max(1.0, abs(tn))
        n_checked += 1
    assert n_checked > 4900


def test_brute_closest_and_any():
    tris = np.array([[0, 0, 0, 1, 0, 0, 0, 1, 0],
                     [0, 0, -1, 1, 0, -1, 0, 1, -1],
                     [0, 0, -2, 1, 0, -2, 0, 1, -2]], np.float32)
    r = np.stack([ray((0.2, 0.2, 1.0), (0, 0, -1)), ray((0.2, 0.2, -1.5), (0, 0, 1)),
                  ray((5, 5, 1.0), (0, 0, -1))])
    h, tie = O.brute(r, tris, O.CLOSEST_HIT)
    assert list(h["prim"]) == [0, 1, O.NO_HIT] and h["t"][0] == 1.0 and h["t"][1] == 0.5
    assert np.isinf(h["t"][2]) and not tie.any()
    a, _ = O.brute(r, tris, O.ANY_HIT)
    assert list(a) == [0, 0, O.NO_HIT]
    # two coincident triangles: the lower prim id wins the tie and it is flagged
    tris2 = np.concatenate([tris[:1], tris[:1]])
    h, tie = O.brute(r[:1], tris2, O.CLOSEST_HIT)
    assert h["prim"][0] == 0 and tie[0]
