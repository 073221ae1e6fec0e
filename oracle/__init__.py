"""HRPP oracle: ctypes wrapper over oracle.c -- TEST INFRASTRUCTURE ONLY.

Plain, slow, single-threaded CPU restatement of the HRPP hot path (hash,
predictor table, predicted-leaf test, BVH traversal, ray-box and ray-triangle
tests).  Only tests/, __graft_entry__.smoke() and bench.py's CPU-baseline leg
and reference arm may import this package; the library's product path never
does.  It shares no code with the CUDA path.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_LIB_PATH = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None

ANY_HIT, CLOSEST_HIT = 0, 1
TWO_PHASE, SEQUENTIAL, UNBOUNDED, ONLINE = 0, 1, 2, 3
VERIFY_ROOT, VERIFY_BOTTOM_UP, VERIFY_NONE = 0, 1, 2
HASH_EXP_MSB, HASH_EXP_LSB = 0, 1
NO_HIT = 0xFFFFFFFF
EMPTY_WORD = 0xFFFFFFFFFFFFFFFF
TAG_BITS, LEAF_BITS = 36, 28
HIT_DTYPE = np.dtype([("t", "<f4"), ("prim", "<u4"), ("u", "<f4"), ("v", "<f4")])
OUTCOME = {0: "plain", 1: "negative", 2: "false_pos", 3: "true_pos"}
STAT_NAMES = ["rays", "hits", "lookups", "positives", "true_pos", "false_pos", "negatives", "tp_inexact",
              "inserts", "dup_inserts", "evictions", "interior_nodes", "box_tests", "leaves", "tri_tests",
              "pred_leaves", "pred_tri_tests", "pred_interior_nodes", "pred_box_tests", "gated"]
N_STATS = 20


def build(force: bool = False) -> str:
    """Compiles oracle.c (gcc -O2 -ffp-contract=off; no fast-math)."""
    if force or not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC):
        tmp = _LIB_PATH + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-std=gnu11", "-fPIC", "-shared", "-ffp-contract=off",
                               "-fno-fast-math", _SRC, "-o", tmp, "-lm"])
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


class _Scene(ctypes.Structure):
    _fields_ = [("tris", ctypes.c_void_p), ("n_tris", ctypes.c_uint32), ("nodes", ctypes.c_void_p),
                ("n_nodes", ctypes.c_uint32), ("root", ctypes.c_uint32), ("prim_index", ctypes.c_void_p),
                ("n_prim_index", ctypes.c_uint32)]


class _Table(ctypes.Structure):
    _fields_ = [("words", ctypes.c_void_p), ("log2_sets", ctypes.c_int), ("log2_ways", ctypes.c_int),
                ("precision", ctypes.c_int), ("update_mode", ctypes.c_int), ("unbounded", ctypes.c_void_p),
                ("go_up", ctypes.c_int), ("hash_variant", ctypes.c_int), ("gate_min_tp", ctypes.c_uint32),
                ("gate_sample_log2", ctypes.c_int), ("gate_open", ctypes.c_int)]


def _L():
    global _lib
    with _lock:
        if _lib is None:
            build()
            lib = ctypes.CDLL(_LIB_PATH)
            P, u32, u64, i32, f32 = ctypes.c_void_p, ctypes.c_uint32, ctypes.c_uint64, ctypes.c_int, ctypes.c_float
            sig = {
                "orc_hash_float": (u32, [f32, i32]),
                "orc_hash_float_variant": (u32, [f32, i32, i32]),
                "orc_ray_key": (u64, [P, i32]),
                "orc_ray_key_variant": (u64, [P, i32, i32]),
                "orc_mix48": (u64, [u64]),
                "orc_ray_triangle": (i32, [P, P, P, P, P, P, P]),
                "orc_ray_inverse": (None, [P, P, P]),
                "orc_ray_box": (i32, [P, P, f32, f32, P, P, P]),
                "orc_brute": (None, [P, u32, P, u32, i32, P, P]),
                "orc_trace": (i32, [ctypes.POINTER(_Scene), P, u32, i32, ctypes.POINTER(_Table), P, P, P, P, P, i32]),
                "orc_unbounded_size": (None, [ctypes.POINTER(_Table), P, P]),
                "orc_unbounded_free": (None, [ctypes.POINTER(_Table)]),
            }
            for name, (res, args) in sig.items():
                fn = getattr(lib, name)
                fn.restype = res
                fn.argtypes = args
            _lib = lib
    return _lib


def _p(a):
    if a is None:
        return None
    assert a.flags["C_CONTIGUOUS"], "array must be C-contiguous"
    return a.ctypes.data_as(ctypes.c_void_p)


def _f(a, n=None):
    a = np.ascontiguousarray(a, dtype=np.float32)
    if n is not None:
        a = a.reshape(n)
    return a


# ------------------------------------------------------------- hashing --

def hash_float(f: float, p: int) -> int:
    return int(_L().orc_hash_float(ctypes.c_float(f), p))


def ray_key(ray, p: int, variant: int = 0) -> int:
    if variant:
        return int(_L().orc_ray_key_variant(_p(_f(ray, 8)), p, variant))
    return int(_L().orc_ray_key(_p(_f(ray, 8)), p))


def hash_float_variant(f: float, p: int, variant: int) -> int:
    return int(_L().orc_hash_float_variant(ctypes.c_float(f), p, variant))


def ray_keys(rays: np.ndarray, p: int) -> np.ndarray:
    rays = _f(rays).reshape(-1, 8)
    return np.array([ray_key(r, p) for r in rays], dtype=np.uint64)


def mix48(k: int) -> int:
    return int(_L().orc_mix48(k & 0xFFFFFFFFFFFF))


def set_and_tag(key: int, log2_sets: int):
    m = mix48(key)
    return m & ((1 << log2_sets) - 1), (m >> log2_sets) & ((1 << TAG_BITS) - 1)


def way_of(leaf: int, log2_ways: int) -> int:
    if log2_ways == 0:
        return 0
    return ((leaf * 0x9E3779B1) & 0xFFFFFFFF) >> (32 - log2_ways)


# ------------------------------------------------------------ geometry --

def ray_triangle(ray, v0, v1, v2):
    """(hit, t, u, v) of the Moller-Trumbore test as the oracle defines it."""
    t, u, v = ctypes.c_float(), ctypes.c_float(), ctypes.c_float()
    hit = _L().orc_ray_triangle(_p(_f(ray, 8)), _p(_f(v0, 3)), _p(_f(v1, 3)), _p(_f(v2, 3)),
                                ctypes.byref(t), ctypes.byref(u), ctypes.byref(v))
    return bool(hit), t.value, u.value, v.value


def ray_box(ray, lo, hi, tcur=None):
    """(hit, tn) of the slab test; tcur defaults to the ray's tmax."""
    ray = _f(ray, 8)
    inv, oinv = np.empty(3, np.float32), np.empty(3, np.float32)
    _L().orc_ray_inverse(_p(ray), _p(inv), _p(oinv))
    tn = ctypes.c_float()
    tcur = float(ray[7]) if tcur is None else tcur
    hit = _L().orc_ray_box(_p(inv), _p(oinv), ctypes.c_float(ray[3]), ctypes.c_float(tcur), _p(_f(lo, 3)),
                           _p(_f(hi, 3)), ctypes.byref(tn))
    return bool(hit), tn.value


def brute(rays: np.ndarray, tris: np.ndarray, mode: int):
    """Brute force over all triangles.  closest -> (HIT_DTYPE hits, near_tie);
    any -> (uint32 prim-or-NO_HIT, None)."""
    rays = _f(rays).reshape(-1, 8)
    tris = _f(tris).reshape(-1, 9)
    n = rays.shape[0]
    if mode == CLOSEST_HIT:
        out = np.empty(n, HIT_DTYPE)
        tie = np.zeros(n, np.uint8)
        _L().orc_brute(_p(rays), n, _p(tris), tris.shape[0], mode, _p(out), _p(tie))
        return out, tie.astype(bool)
    out = np.empty(n, np.uint32)
    _L().orc_brute(_p(rays), n, _p(tris), tris.shape[0], mode, _p(out), None)
    return out, None


# ---------------------------------------------------------------- table --

class Table:
    """Predictor table state held by the oracle (bounded modes: numpy words)."""

    def __init__(self, log2_entries: int, ways: int = 1, precision: int = 6, update_mode: int = TWO_PHASE,
                 go_up: int = 0, hash_variant: int = 0, gate_min_tp: int = 0, gate_sample_log2: int = 5):
        log2_ways = {1: 0, 2: 1, 4: 2, 8: 3}[ways]
        if log2_entries - log2_ways < 0:
            raise ValueError("fewer entries than ways")
        self.log2_sets = log2_entries - log2_ways
        self.log2_ways = log2_ways
        self.ways = ways
        self.precision = precision
        self.update_mode = update_mode
        n_words = 1 << log2_entries if update_mode != UNBOUNDED else 1
        self.words = np.full(n_words, EMPTY_WORD, np.uint64)
        self.go_up = go_up
        self.hash_variant = hash_variant
        self._c = _Table(self.words.ctypes.data, self.log2_sets, self.log2_ways, precision, update_mode, None, go_up,
                         hash_variant, gate_min_tp, gate_sample_log2, 1)

    @property
    def gate_open(self) -> bool:
        return bool(self._c.gate_open)

    def reset(self):
        self.words[:] = EMPTY_WORD
        if self._c.unbounded:
            _L().orc_unbounded_free(ctypes.byref(self._c))

    def unbounded_size(self):
        keys, leaves = ctypes.c_uint64(), ctypes.c_uint64()
        _L().orc_unbounded_size(ctypes.byref(self._c), ctypes.byref(keys), ctypes.byref(leaves))
        return keys.value, leaves.value

    def __del__(self):
        try:
            if self._c.unbounded:
                _L().orc_unbounded_free(ctypes.byref(self._c))
        except Exception:
            pass


# ---------------------------------------------------------------- trace --

def trace(tris, nodes, prim_index, root, rays, mode: int, table: Table | None = None, per_ray: bool = False,
          predicted=None, verify: int = 0):
    """Plain traversal (table None) or HRPP against `table` (mutated).
    predicted: optional int32 [n] canonical node per ray whose subtree is
    traversed first (learned proposal; -1 = none).
    verify: how closest-hit true positives are verified, VERIFY_ROOT (a
    traversal from the root bounded by the predicted hit), VERIFY_BOTTOM_UP
    (a climb from the predicted hit's leaf through its ancestors' siblings) or
    VERIFY_NONE (the paper's semantics: the predicted hit is returned).

    Returns (hits, stats dict[, outcome uint8[n], box_tests uint32[n]])."""
    tris = _f(tris).reshape(-1, 9)
    nodes = np.ascontiguousarray(nodes)
    assert nodes.dtype.itemsize == 48
    prim_index = np.ascontiguousarray(prim_index, np.uint32)
    rays = _f(rays).reshape(-1, 8)
    n = rays.shape[0]
    sc = _Scene(tris.ctypes.data, tris.shape[0], nodes.ctypes.data, nodes.shape[0], int(root),
                prim_index.ctypes.data, prim_index.shape[0])
    out = np.empty(n, HIT_DTYPE) if mode == CLOSEST_HIT else np.empty(n, np.uint32)
    stats = np.zeros(N_STATS, np.uint64)
    outcome = np.zeros(n, np.uint8) if per_ray else None
    boxes = np.zeros(n, np.uint32) if per_ray else None
    tptr = ctypes.byref(table._c) if table is not None else None
    pred = None if predicted is None else np.ascontiguousarray(predicted, np.int32)
    rc = _L().orc_trace(ctypes.byref(sc), _p(rays), n, mode, tptr, _p(out), _p(stats), _p(outcome), _p(boxes),
                        _p(pred), int(verify))
    if rc != 0:
        raise RuntimeError("orc_trace failed")
    sd = {k: int(stats[i]) for i, k in enumerate(STAT_NAMES)}
    if per_ray:
        return out, sd, outcome, boxes
    return out, sd
