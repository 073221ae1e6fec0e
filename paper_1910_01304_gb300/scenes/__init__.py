"""Seeded synthetic inputs: scenes, BVHs and rays (numpy wrappers over scenegen.c).

This module holds none of the HRPP arithmetic (no hash, no table, no ray-box or
ray-triangle test, no traversal).  It is the only code the CPU oracle and the
CUDA path share: both trace exactly the arrays made here.

Array formats (the canonical formats of the C ABI):
  tris        float32 [n, 9]   v0.xyz, v1.xyz, v2.xyz per triangle
  nodes       NODE_DTYPE [m]   lo[3], hi[3], child[4] (-1 none), first, count
  prim_index  uint32 [n]       leaf `first..first+count` index into it
  rays        float32 [n, 8]   ox, oy, oz, tmin, dx, dy, dz, tmax
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "scenegen.c")
_LIB_PATH = os.path.join(_HERE, "libscenegen.so")
_lock = threading.Lock()
_lib = None

NODE_DTYPE = np.dtype(
    [("lo", "<f4", (3,)), ("hi", "<f4", (3,)), ("child", "<i4", (4,)), ("first", "<u4"), ("count", "<u4")]
)
assert NODE_DTYPE.itemsize == 48
NO_HIT = 0xFFFFFFFF


def build(force: bool = False) -> str:
    """Compiles scenegen.c into libscenegen.so beside it (gcc, portable flags)."""
    if force or not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC):
        tmp = _LIB_PATH + f".tmp{os.getpid()}"
        subprocess.check_call(
            ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-ffp-contract=off", _SRC, "-o", tmp, "-lm"]
        )
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _L():
    global _lib
    with _lock:
        if _lib is None:
            build()
            lib = ctypes.CDLL(_LIB_PATH)
            P = ctypes.c_void_p
            u32, i32, u64, f32, f64 = ctypes.c_uint32, ctypes.c_int, ctypes.c_uint64, ctypes.c_float, ctypes.c_double
            sig = {
                "sg_splitmix64": (u64, [u64]),
                "sg_pcg32_stream": (None, [u64, u64, u32, P]),
                "sg_icosphere": (u32, [i32, f32, f32, f32, f32, P]),
                "sg_terrain_height": (f64, [u64, i32, f64, f64, f64, f64]),
                "sg_grid": (u32, [i32, i32, f32, f32, f32, f32, f32, u64, i32, f32, f32, P]),
                "sg_soup": (u32, [u32, u64, f32, f32, f32, P]),
                "sg_place_spheres": (None, [u32, u64, f32, f32, f32, f32, f32, f32, u64, i32, f32, f32, P]),
                "sg_build_bvh2": (i32, [P, u32, i32, P, P, P]),
                "sg_build_bvh2_sah": (i32, [P, u32, i32, f64, P, P, P]),
                "sg_collapse_bvh4": (i32, [P, u32, P, P]),
                "sg_pinhole": (None, [P, P, f32, u32, u32, u64, u32, u32, u32, P]),
                "sg_shadow_rays": (u32, [P, P, P, u32, P, P, P, P]),
                "sg_ao_rays": (u32, [P, P, P, u32, P, u32, f32, u64, u32, P, P]),
                "sg_sphere_rays": (None, [u32, u64, f32, f32, f32, P]),
            }
            for name, (res, args) in sig.items():
                fn = getattr(lib, name)
                fn.restype = res
                fn.argtypes = args
            _lib = lib
    return _lib


def _p(a: np.ndarray):
    assert a.flags["C_CONTIGUOUS"]
    return a.ctypes.data_as(ctypes.c_void_p)


def _f3(v):
    return np.ascontiguousarray(np.asarray(v, dtype=np.float32).reshape(3))


# ------------------------------------------------------------------ RNG --


def splitmix64(x: int) -> int:
    return int(_L().sg_splitmix64(x & 0xFFFFFFFFFFFFFFFF))


def pcg32_stream(initstate: int, initseq: int, n: int) -> np.ndarray:
    out = np.empty(n, np.uint32)
    _L().sg_pcg32_stream(initstate, initseq, n, _p(out))
    return out


# ------------------------------------------------------------- geometry --


def icosphere(subdiv: int, center=(0.0, 0.0, 0.0), radius: float = 1.0) -> np.ndarray:
    L = _L()
    n = L.sg_icosphere(subdiv, *map(float, center), float(radius), None)
    out = np.empty((n, 9), np.float32)
    L.sg_icosphere(subdiv, *map(float, center), float(radius), _p(out))
    return out


def quad_grid(nx: int, nz: int, x0: float, x1: float, z0: float, z1: float, y: float = 0.0) -> np.ndarray:
    out = np.empty((2 * nx * nz, 9), np.float32)
    _L().sg_grid(nx, nz, x0, x1, z0, z1, y, 0, 0, 0.0, 0.0, _p(out))
    return out


def terrain(nx: int, nz: int, x0: float, x1: float, z0: float, z1: float, seed: int, octaves: int = 4,
            amp: float = 8.0, freq: float = 1.0 / 16.0) -> np.ndarray:
    out = np.empty((2 * nx * nz, 9), np.float32)
    _L().sg_grid(nx, nz, x0, x1, z0, z1, 0.0, seed, octaves, amp, freq, _p(out))
    return out


def terrain_height(seed: int, x: float, z: float, octaves: int = 4, amp: float = 8.0, freq: float = 1.0 / 16.0) -> float:
    return float(_L().sg_terrain_height(seed, octaves, amp, freq, x, z))


def soup(n: int, seed: int, lo: float = 0.0, hi: float = 1.0, extent: float | None = None) -> np.ndarray:
    if extent is None:
        extent = 0.5 * (hi - lo) * max(n, 1) ** (-1.0 / 3.0)
    out = np.empty((n, 9), np.float32)
    _L().sg_soup(n, seed, lo, hi, extent, _p(out))
    return out


def place_spheres(count: int, seed: int, rmin: float, rmax: float, x0: float, x1: float, z0: float, z1: float,
                  terrain_seed: int, octaves: int = 4, amp: float = 8.0, freq: float = 1.0 / 16.0) -> np.ndarray:
    out = np.empty((count, 4), np.float32)
    _L().sg_place_spheres(count, seed, rmin, rmax, x0, x1, z0, z1, terrain_seed, octaves, amp, freq, _p(out))
    return out


# ------------------------------------------------------------------ BVH --


def build_bvh(tris: np.ndarray, width: int = 2, max_leaf: int = 4, method: str = "sah", trav_cost: float = 1.0):
    """Deterministic binary BVH, binned surface-area heuristic ("sah", the
    default) or median split ("median"); width 2 (binary) or 4 (collapsed).
    Leaves hold at most max_leaf triangles.  SAH: a node of up to max_leaf
    triangles still splits when trav_cost x its area plus its children's
    area x count is below its own area x count (one triangle test costing 1;
    trav_cost = 0 makes every such node a leaf).

    Returns (nodes, prim_index, root) in the canonical format; root is 0.
    """
    if method not in ("sah", "median"):
        raise ValueError("method must be 'sah' or 'median'")
    tris = np.ascontiguousarray(tris, dtype=np.float32).reshape(-1, 9)
    n = tris.shape[0]
    if n == 0:
        raise ValueError("empty scene")
    nodes2 = np.zeros(2 * n, NODE_DTYPE)
    prim = np.empty(n, np.uint32)
    cnt = ctypes.c_uint32(0)
    if method == "sah":
        rc = _L().sg_build_bvh2_sah(_p(tris), n, max_leaf, trav_cost, _p(nodes2), ctypes.byref(cnt), _p(prim))
    else:
        rc = _L().sg_build_bvh2(_p(tris), n, max_leaf, _p(nodes2), ctypes.byref(cnt), _p(prim))
    if rc != 0:
        raise RuntimeError(f"BVH build failed ({rc})")
    nodes2 = nodes2[: cnt.value].copy()
    if width == 2:
        return nodes2, prim, 0
    if width != 4:
        raise ValueError("width must be 2 or 4")
    nodes4 = np.zeros(cnt.value, NODE_DTYPE)
    c4 = ctypes.c_uint32(0)
    rc = _L().sg_collapse_bvh4(_p(nodes2), cnt.value, _p(nodes4), ctypes.byref(c4))
    if rc != 0:
        raise RuntimeError(f"sg_collapse_bvh4 failed ({rc})")
    return nodes4[: c4.value].copy(), prim, 0


# ----------------------------------------------------------------- rays --


def pinhole_rays(eye, target, vfov_deg: float, width: int, height: int, seed: int = 0, frame: int = 0,
                 tile=(8, 4)) -> np.ndarray:
    out = np.empty((width * height, 8), np.float32)
    _L().sg_pinhole(_p(_f3(eye)), _p(_f3(target)), vfov_deg, width, height, seed, frame, tile[0], tile[1], _p(out))
    return out


def _hit_arrays(hit_t, hit_prim, n):
    t = np.ascontiguousarray(np.asarray(hit_t, np.float32).reshape(n))
    p = np.ascontiguousarray(np.asarray(hit_prim, np.uint32).reshape(n))
    return t, p


def shadow_rays(rays: np.ndarray, hit_t, hit_prim, tris: np.ndarray, light):
    rays = np.ascontiguousarray(rays, np.float32)
    n = rays.shape[0]
    t, p = _hit_arrays(hit_t, hit_prim, n)
    out = np.empty((n, 8), np.float32)
    src = np.empty(n, np.uint32)
    k = _L().sg_shadow_rays(_p(rays), _p(t), _p(p), n, _p(np.ascontiguousarray(tris, np.float32)),
                            _p(_f3(light)), _p(out), _p(src))
    return out[:k].copy(), src[:k].copy()


def ao_rays(rays: np.ndarray, hit_t, hit_prim, tris: np.ndarray, per_hit: int = 4, tmax: float = 0.5,
            seed: int = 0, frame: int = 0):
    rays = np.ascontiguousarray(rays, np.float32)
    n = rays.shape[0]
    t, p = _hit_arrays(hit_t, hit_prim, n)
    n_hit = int(np.count_nonzero(p != NO_HIT))
    out = np.empty((max(n_hit * per_hit, 1), 8), np.float32)
    src = np.empty(max(n_hit * per_hit, 1), np.uint32)
    k = _L().sg_ao_rays(_p(rays), _p(t), _p(p), n, _p(np.ascontiguousarray(tris, np.float32)), per_hit, tmax,
                        seed, frame, _p(out), _p(src))
    return out[:k].copy(), src[:k].copy()


def sphere_rays(n: int, seed: int, lo: float, hi: float, tmax: float = float("inf")) -> np.ndarray:
    out = np.empty((n, 8), np.float32)
    _L().sg_sphere_rays(n, seed, lo, hi, tmax, _p(out))
    return out
