"""The C ABI library loads and exports every entry point include/hrpp.h
declares; host-side validation rejects corrupt scenes and bad arguments
(fault injection on the host: no GPU is touched)."""
import ctypes
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def H():
    from paper_1910_01304_gb300 import build
    build.build()
    from paper_1910_01304_gb300 import hrpp
    return hrpp


def _declared():
    text = open(os.path.join(ROOT, "include", "hrpp.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(hrpp_[a-z0-9_]+)\s*\(", text)))


def test_every_declared_symbol_is_exported(H):
    names = _declared()
    assert "hrpp_trace" in names and "hrpp_scene_create" in names and "hrpp_table_create" in names
    lib = ctypes.CDLL(H.LIB_PATH)
    for n in names:
        assert hasattr(lib, n), n


def test_version_and_status_strings(H):
    assert H.hrpp_version() == 1
    assert H.hrpp_status_string(H.HRPP_ERR_INVALID_BVH) == b"HRPP_ERR_INVALID_BVH"


def _scene():
    from paper_1910_01304_gb300 import scenes as S
    tris = S.soup(200, 4)
    nodes, prim, root = S.build_bvh(tris, width=2)
    return tris, nodes, prim, root


def _validate(H, tris, nodes, prim, root=0, width=2):
    return H.hrpp_scene_validate(H._ptr(np.ascontiguousarray(tris)), tris.shape[0], H._ptr(np.ascontiguousarray(nodes)),
                                 nodes.shape[0], root, H._ptr(np.ascontiguousarray(prim)), prim.shape[0], width, None)


def test_validate_accepts_generated_scenes(H):
    tris, nodes, prim, root = _scene()
    info = H.validate_scene(tris, nodes, prim, root, 2)
    assert info["n_tris"] == 200 and info["n_leaves"] == int((nodes["count"] > 0).sum())
    from paper_1910_01304_gb300 import scenes as S
    n4, p4, r4 = S.build_bvh(tris, width=4)
    assert H.validate_scene(tris, n4, p4, r4, 4)["n_interior"] < info["n_interior"]
    # a binary BVH is also a valid 4-wide input; a 4-wide one is not binary
    assert _validate(H, tris, nodes, prim, 0, 4) == H.HRPP_OK
    assert _validate(H, tris, n4, p4, 0, 2) == H.HRPP_ERR_INVALID_BVH


def _expect(H, code, tris, nodes, prim, **kw):
    rc = _validate(H, tris, nodes, prim, **kw)
    assert rc == code, (rc, H.hrpp_last_error())


def test_validate_rejects_corrupt_bvhs(H):
    tris, nodes, prim, root = _scene()
    interior = np.nonzero(nodes["count"] == 0)[0]
    leaves = np.nonzero(nodes["count"] > 0)[0]
    # cycle: a child pointing back at the root
    n = nodes.copy(); n[interior[-1]]["child"][0] = 0
    _expect(H, H.HRPP_ERR_INVALID_BVH, tris, n, prim)
    # child out of range
    n = nodes.copy(); n[interior[3]]["child"][1] = len(nodes) + 5
    _expect(H, H.HRPP_ERR_INVALID_BVH, tris, n, prim)
    # shared child (node reached twice)
    n = nodes.copy(); n[interior[2]]["child"][1] = n[interior[3]]["child"][0]
    _expect(H, H.HRPP_ERR_INVALID_BVH, tris, n, prim)
    # prim listed twice in prim_index
    p = prim.copy(); p[5] = p[6]
    _expect(H, H.HRPP_ERR_INVALID_BVH, tris, nodes, p)
    # two leaves covering the same slots (and a slot left uncovered)
    n = nodes.copy(); n[leaves[1]]["first"] = n[leaves[0]]["first"]
    _expect(H, H.HRPP_ERR_INVALID_BVH, tris, n, prim)
    # child box outside its parent
    n = nodes.copy(); n[interior[1]]["hi"][0] += 10.0
    _expect(H, H.HRPP_ERR_INVALID_BVH, tris, n, prim)
    # leaf box that misses its triangles
    n = nodes.copy(); n[leaves[0]]["lo"][:] = n[leaves[0]]["hi"]
    _expect(H, H.HRPP_ERR_INVALID_BVH, tris, n, prim)
    # NaN box
    n = nodes.copy(); n[interior[1]]["lo"][2] = np.nan
    _expect(H, H.HRPP_ERR_INVALID_BVH, tris, n, prim)
    # interior node without children
    n = nodes.copy(); n[interior[1]]["child"][:] = -1
    _expect(H, H.HRPP_ERR_INVALID_BVH, tris, n, prim)


def test_validate_limits_and_arguments(H):
    tris, nodes, prim, root = _scene()
    # a leaf with 5 triangles exceeds HRPP_MAX_LEAF_TRIS
    from paper_1910_01304_gb300 import scenes as S
    n5, p5, _ = S.build_bvh(tris, width=2, max_leaf=5, trav_cost=0.0)
    if (n5["count"] > 4).any():
        _expect(H, H.HRPP_ERR_UNSUPPORTED, tris, n5, p5)
    _expect(H, H.HRPP_ERR_INVALID_ARG, tris, nodes, prim, width=3)
    _expect(H, H.HRPP_ERR_INVALID_ARG, tris, nodes, prim, root=len(nodes))
    t = tris.copy(); t[3, 4] = np.inf
    _expect(H, H.HRPP_ERR_INVALID_ARG, t, nodes, prim)
    assert _validate(H, tris, nodes, prim[:-1]) == H.HRPP_ERR_INVALID_ARG
    rc = H.hrpp_scene_validate(None, 0, None, 0, 0, None, 0, 2, None)
    assert rc == H.HRPP_ERR_INVALID_ARG
    assert b"n_tris" in H.hrpp_last_error()


def test_argument_errors_before_any_cuda_call(H):
    h = ctypes.c_void_p()
    assert H.hrpp_table_create(12, 3, ctypes.byref(h)) == H.HRPP_ERR_INVALID_ARG
    assert H.hrpp_table_create(40, 1, ctypes.byref(h)) == H.HRPP_ERR_INVALID_ARG
    assert H.hrpp_table_create(1, 4, ctypes.byref(h)) == H.HRPP_ERR_INVALID_ARG
    assert H.hrpp_trace(None, None, None, 0, 1, None, None, None) == H.HRPP_ERR_INVALID_ARG
    assert H.hrpp_table_configure(None, 6, 0) == H.HRPP_ERR_INVALID_ARG
    H.hrpp_scene_destroy(None)
    H.hrpp_table_destroy(None)
