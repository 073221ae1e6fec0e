"""Python binding of the HRPP C ABI (include/hrpp.h), via ctypes.

The functions named hrpp_* mirror the C entry points one to one and only
marshal arguments.  `Scene`, `Table` and `trace` are thin conveniences over
them that accept numpy arrays (host) and torch tensors (device or host) and
turn non-OK statuses into HrppError.  All computation happens in libhrpp.so;
there is no fallback: if the library is missing, importing fails loudly.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libhrpp.so")

HRPP_OK, HRPP_ERR_INVALID_ARG, HRPP_ERR_INVALID_BVH, HRPP_ERR_OOM = 0, 1, 2, 3
HRPP_ERR_CUDA, HRPP_ERR_TRAVERSAL_LIMIT, HRPP_ERR_UNSUPPORTED = 4, 5, 6
HRPP_ANY_HIT, HRPP_CLOSEST_HIT = 0, 1
HRPP_UPDATE_TWO_PHASE, HRPP_UPDATE_ONLINE, HRPP_UPDATE_FROZEN = 0, 1, 2
HRPP_NO_HIT = 0xFFFFFFFF
HRPP_NOALLOC_MAX_RAYS = 1 << 20
HRPP_PROPOSAL_PARAMS = 256 * 96 + 256 + 256 * 256 + 256 + 4096 * 256 + 4096
HRPP_EMPTY_WORD = 0xFFFFFFFFFFFFFFFF
STAT_NAMES = ["rays", "hits", "lookups", "positives", "true_pos", "false_pos", "negatives", "tp_inexact",
              "inserts", "dup_inserts", "evictions", "interior_nodes", "box_tests", "leaves", "tri_tests",
              "pred_leaves", "pred_tri_tests", "pred_interior_nodes", "pred_box_tests", "gated"]


class hrpp_stats(ctypes.Structure):
    _fields_ = [(n, ctypes.c_uint64) for n in STAT_NAMES]

    def as_dict(self):
        return {n: int(getattr(self, n)) for n in STAT_NAMES}


class hrpp_scene_info(ctypes.Structure):
    _fields_ = [("n_tris", ctypes.c_uint32), ("n_interior", ctypes.c_uint32), ("n_leaves", ctypes.c_uint32),
                ("max_depth", ctypes.c_uint32), ("width", ctypes.c_uint32), ("root_is_leaf", ctypes.c_uint32),
                ("device_bytes", ctypes.c_uint64)]


class hrpp_trace_opts(ctypes.Structure):
    _fields_ = [("kernel_start", ctypes.c_void_p), ("kernel_stop", ctypes.c_void_p),
                ("predicted_nodes", ctypes.c_void_p), ("block_threads", ctypes.c_uint32),
                ("schedule", ctypes.c_uint32), ("refill_min", ctypes.c_uint32), ("max_steps", ctypes.c_uint32),
                ("verify", ctypes.c_uint32), ("l2_persist", ctypes.c_uint32),
                ("ray_outcome", ctypes.c_void_p), ("ray_box_tests", ctypes.c_void_p), ("host_async", ctypes.c_uint32),
                ("host_done", ctypes.c_void_p), ("stage_chunks", ctypes.c_uint32)]


HRPP_SCHEDULE_DEFAULT, HRPP_SCHEDULE_BATCH, HRPP_SCHEDULE_REFILL, HRPP_SCHEDULE_COMPACT = 0, 1, 2, 3
HRPP_VERIFY_ROOT, HRPP_VERIFY_BOTTOM_UP, HRPP_VERIFY_NONE = 0, 1, 2
HRPP_HASH_EXP_MSB, HRPP_HASH_EXP_LSB = 0, 1
HRPP_GEMM_A_MN_MAJOR, HRPP_GEMM_B_MN_MAJOR = 1, 2
HRPP_L2_NONE, HRPP_L2_TABLE, HRPP_L2_NODES = 0, 1, 2
HRPP_OUTCOME_PLAIN, HRPP_OUTCOME_NEGATIVE, HRPP_OUTCOME_FALSE_POS, HRPP_OUTCOME_TRUE_POS = 0, 1, 2, 3


class hrpp_batch_item(ctypes.Structure):
    _fields_ = [("scene", ctypes.c_void_p), ("table", ctypes.c_void_p), ("rays", ctypes.c_void_p),
                ("n_rays", ctypes.c_uint32), ("mode", ctypes.c_int), ("out_hits", ctypes.c_void_p)]


class HrppError(RuntimeError):
    def __init__(self, status: int, message: str):
        super().__init__(message)
        self.status = status


def _load():
    if not os.path.exists(LIB_PATH):
        raise ImportError(f"{LIB_PATH} is not built; run paper_1910_01304_gb300.build.build()")
    lib = ctypes.CDLL(LIB_PATH)
    P, u32, i32, sz = ctypes.c_void_p, ctypes.c_uint32, ctypes.c_int, ctypes.c_size_t
    st = ctypes.c_int
    sig = {
        "hrpp_scene_validate": (st, [P, u32, P, u32, u32, P, u32, i32, P]),
        "hrpp_scene_create": (st, [P, u32, P, u32, u32, P, u32, i32, P]),
        "hrpp_scene_get_info": (st, [P, P]),
        "hrpp_scene_check": (st, [P, P]),
        "hrpp_scene_destroy": (None, [P]),
        "hrpp_table_create": (st, [i32, i32, P]),
        "hrpp_table_configure": (st, [P, i32, i32]),
        "hrpp_table_set_go_up": (st, [P, i32]),
        "hrpp_table_set_hash": (st, [P, i32]),
        "hrpp_table_set_gate": (st, [P, u32, i32]),
        "hrpp_table_get_gate": (st, [P, P]),
        "hrpp_table_reset": (st, [P, P]),
        "hrpp_table_export": (st, [P, P, sz]),
        "hrpp_table_import": (st, [P, P, sz]),
        "hrpp_table_copy": (st, [P, P, P]),
        "hrpp_table_get_config": (st, [P, P, P, P, P]),
        "hrpp_table_destroy": (None, [P]),
        "hrpp_trace": (st, [P, P, P, u32, i32, P, P, P]),
        "hrpp_trace_ex": (st, [P, P, P, u32, i32, P, P, P, P]),
        "hrpp_trace_noalloc": (st, [P, P, P, u32, i32, P, P, P]),
        "hrpp_l2_set_aside": (st, [sz, P]),
        "hrpp_batch_create": (st, [P, u32, i32, u32, P]),
        "hrpp_batch_run": (st, [P, P]),
        "hrpp_batch_get_stats": (st, [P, u32, P]),
        "hrpp_batch_destroy": (None, [P]),
        "hrpp_gemm_bf16": (st, [P, P, P, i32, i32, i32, P]),
        "hrpp_gemm_bf16_ex": (st, [P, P, P, i32, i32, i32, i32, P]),
        "hrpp_proposal_create": (st, [P, P, u32, u32, P, u32, ctypes.c_uint64, P]),
        "hrpp_proposal_features": (st, [P, P, u32, P, P]),
        "hrpp_proposal_labels": (st, [P, P, u32, P, P]),
        "hrpp_proposal_train": (st, [P, P, P, u32, ctypes.c_float, P, P]),
        "hrpp_proposal_gradients": (st, [P, P, P, u32, P, P]),
        "hrpp_proposal_predict": (st, [P, P, u32, P, P, P]),
        "hrpp_proposal_get_weights": (st, [P, P, sz]),
        "hrpp_proposal_set_weights": (st, [P, P, sz]),
        "hrpp_proposal_class_nodes": (st, [P, P]),
        "hrpp_proposal_destroy": (None, [P]),
        "hrpp_last_error": (ctypes.c_char_p, []),
        "hrpp_status_string": (ctypes.c_char_p, [st]),
        "hrpp_version": (i32, []),
    }
    for name, (res, args) in sig.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    return lib


_lib = _load()

# ------------------------------------------------ one-to-one C entry points --

hrpp_scene_validate = _lib.hrpp_scene_validate
hrpp_scene_create = _lib.hrpp_scene_create
hrpp_scene_get_info = _lib.hrpp_scene_get_info
hrpp_scene_check = _lib.hrpp_scene_check
hrpp_scene_destroy = _lib.hrpp_scene_destroy
hrpp_table_create = _lib.hrpp_table_create
hrpp_table_configure = _lib.hrpp_table_configure
hrpp_table_set_go_up = _lib.hrpp_table_set_go_up
hrpp_table_set_hash = _lib.hrpp_table_set_hash
hrpp_table_set_gate = _lib.hrpp_table_set_gate
hrpp_table_get_gate = _lib.hrpp_table_get_gate
hrpp_table_reset = _lib.hrpp_table_reset
hrpp_table_export = _lib.hrpp_table_export
hrpp_table_import = _lib.hrpp_table_import
hrpp_table_copy = _lib.hrpp_table_copy
hrpp_table_get_config = _lib.hrpp_table_get_config
hrpp_table_destroy = _lib.hrpp_table_destroy
hrpp_trace = _lib.hrpp_trace
hrpp_trace_ex = _lib.hrpp_trace_ex
hrpp_trace_noalloc = _lib.hrpp_trace_noalloc
hrpp_l2_set_aside = _lib.hrpp_l2_set_aside
hrpp_batch_create = _lib.hrpp_batch_create
hrpp_batch_run = _lib.hrpp_batch_run
hrpp_batch_get_stats = _lib.hrpp_batch_get_stats
hrpp_batch_destroy = _lib.hrpp_batch_destroy
hrpp_gemm_bf16 = _lib.hrpp_gemm_bf16
hrpp_gemm_bf16_ex = _lib.hrpp_gemm_bf16_ex
hrpp_proposal_create = _lib.hrpp_proposal_create
hrpp_proposal_features = _lib.hrpp_proposal_features
hrpp_proposal_labels = _lib.hrpp_proposal_labels
hrpp_proposal_train = _lib.hrpp_proposal_train
hrpp_proposal_gradients = _lib.hrpp_proposal_gradients
hrpp_proposal_predict = _lib.hrpp_proposal_predict
hrpp_proposal_get_weights = _lib.hrpp_proposal_get_weights
hrpp_proposal_set_weights = _lib.hrpp_proposal_set_weights
hrpp_proposal_class_nodes = _lib.hrpp_proposal_class_nodes
hrpp_proposal_destroy = _lib.hrpp_proposal_destroy
hrpp_last_error = _lib.hrpp_last_error
hrpp_status_string = _lib.hrpp_status_string
hrpp_version = _lib.hrpp_version


def check(status: int):
    if status != HRPP_OK:
        raise HrppError(status, (hrpp_last_error() or b"").decode())


# --------------------------------------------------------- conveniences --

def _ptr(x):
    """Address of a numpy array or torch tensor (contiguous)."""
    if x is None:
        return None
    if isinstance(x, np.ndarray):
        assert x.flags["C_CONTIGUOUS"]
        return x.ctypes.data
    assert x.is_contiguous()
    return x.data_ptr()


def _stream_handle(stream):
    if stream is None:
        try:
            import torch
            if torch.cuda.is_available():
                return torch.cuda.current_stream().cuda_stream
        except ImportError:
            pass
        return None
    if isinstance(stream, int):
        return stream
    return stream.cuda_stream


def validate_scene(tris, nodes, prim_index, root: int, width: int) -> dict:
    tris = np.ascontiguousarray(tris, np.float32).reshape(-1, 9)
    nodes = np.ascontiguousarray(nodes)
    prim_index = np.ascontiguousarray(prim_index, np.uint32)
    info = hrpp_scene_info()
    check(hrpp_scene_validate(_ptr(tris), tris.shape[0], _ptr(nodes), nodes.shape[0], root, _ptr(prim_index),
                              prim_index.shape[0], width, ctypes.byref(info)))
    return {f: getattr(info, f) for f, _ in info._fields_}


class Scene:
    """Device-resident scene (hrpp_scene_create)."""

    def __init__(self, tris, nodes, prim_index, root: int = 0, width: int = 2):
        tris = np.ascontiguousarray(tris, np.float32).reshape(-1, 9)
        nodes = np.ascontiguousarray(nodes)
        assert nodes.dtype.itemsize == 48
        prim_index = np.ascontiguousarray(prim_index, np.uint32)
        h = ctypes.c_void_p()
        check(hrpp_scene_create(_ptr(tris), tris.shape[0], _ptr(nodes), nodes.shape[0], root, _ptr(prim_index),
                                prim_index.shape[0], width, ctypes.byref(h)))
        self.handle = h
        self.width = width
        self.n_tris = tris.shape[0]

    @classmethod
    def from_workload(cls, s):
        return cls(s.tris, s.nodes, s.prim_index, s.root, s.width)

    def info(self) -> dict:
        info = hrpp_scene_info()
        check(hrpp_scene_get_info(self.handle, ctypes.byref(info)))
        return {f: getattr(info, f) for f, _ in info._fields_}

    def check(self, stream=None):
        check(hrpp_scene_check(self.handle, _stream_handle(stream)))

    def close(self):
        if getattr(self, "handle", None):
            hrpp_scene_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Table:
    """Predictor table (hrpp_table_create / hrpp_table_configure)."""

    def __init__(self, log2_entries: int, ways: int = 1, precision: int = 6, update_mode: int = HRPP_UPDATE_TWO_PHASE,
                 go_up: int = 0, hash_variant: int = HRPP_HASH_EXP_MSB):
        h = ctypes.c_void_p()
        check(hrpp_table_create(log2_entries, ways, ctypes.byref(h)))
        self.handle = h
        self.log2_entries = log2_entries
        self.ways = ways
        self.configure(precision, update_mode)
        self.set_go_up(go_up)
        self.set_hash(hash_variant)

    def set_go_up(self, go_up: int):
        check(hrpp_table_set_go_up(self.handle, go_up))
        self.go_up = go_up

    def set_hash(self, hash_variant: int):
        check(hrpp_table_set_hash(self.handle, hash_variant))
        self.hash_variant = hash_variant

    def set_gate(self, min_tp_per_65536: int, sample_log2: int = 5):
        """hrpp_table_set_gate: 0 turns the gate off."""
        check(hrpp_table_set_gate(self.handle, int(min_tp_per_65536), int(sample_log2)))
        self.gate = (int(min_tp_per_65536), int(sample_log2))

    def gate_open(self) -> bool:
        v = ctypes.c_int()
        check(hrpp_table_get_gate(self.handle, ctypes.byref(v)))
        return bool(v.value)

    def configure(self, precision: int, update_mode: int):
        check(hrpp_table_configure(self.handle, precision, update_mode))
        self.precision = precision
        self.update_mode = update_mode

    def reset(self, stream=None):
        check(hrpp_table_reset(self.handle, _stream_handle(stream)))

    def export(self) -> np.ndarray:
        out = np.empty(1 << self.log2_entries, np.uint64)
        check(hrpp_table_export(self.handle, _ptr(out), out.shape[0]))
        return out

    def import_(self, words: np.ndarray):
        words = np.ascontiguousarray(words, np.uint64)
        check(hrpp_table_import(self.handle, _ptr(words), words.shape[0]))

    def copy_from(self, src: "Table", stream=None):
        """Device-to-device copy of src's words (hrpp_table_copy)."""
        check(hrpp_table_copy(self.handle, src.handle, _stream_handle(stream)))

    def close(self):
        if getattr(self, "handle", None):
            hrpp_table_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def trace(scene: Scene, rays, mode: int, table: Table | None = None, hits=None, stats: bool = False,
          stream=None, kernel_events=None, block_threads: int = 0, schedule: int = 0, refill_min: int = 0,
          predicted=None, max_steps: int = 0, verify: int = 0, ray_outcome=None, ray_box_tests=None,
          l2_persist: int = 0, host_async: bool = False, stage_chunks: int = 0, host_done=None):
    """Traces rays ([n, 8] float32 torch tensor on the GPU, or a host numpy
    array / torch tensor).  Returns (hits, stats dict or None).

    closest-hit hits: [n, 4] float32 (t, prim bits, u, v); any-hit: [n] int32
    (prim or -1).  Device rays give device hits unless `hits` is passed."""
    is_np = isinstance(rays, np.ndarray)
    n = int(rays.shape[0])
    if hits is None:
        if is_np:
            hits = np.empty((n, 4), np.float32) if mode == HRPP_CLOSEST_HIT else np.empty(n, np.int32)
        else:
            import torch
            shape = (n, 4) if mode == HRPP_CLOSEST_HIT else (n,)
            dtype = torch.float32 if mode == HRPP_CLOSEST_HIT else torch.int32
            hits = torch.empty(shape, dtype=dtype, device=rays.device)
    st = hrpp_stats() if stats else None
    opts = None
    if (kernel_events is not None or block_threads or schedule or refill_min or max_steps or verify or l2_persist
            or predicted is not None or ray_outcome is not None or ray_box_tests is not None or host_async
            or stage_chunks or host_done is not None):
        opts = hrpp_trace_opts()
        if predicted is not None:
            opts.predicted_nodes = _ptr(predicted)
        if kernel_events is not None:
            opts.kernel_start = kernel_events[0].cuda_event
            opts.kernel_stop = kernel_events[1].cuda_event
        opts.block_threads = block_threads
        opts.schedule = schedule
        opts.refill_min = refill_min
        opts.max_steps = max_steps
        opts.verify = verify
        opts.l2_persist = l2_persist
        opts.host_async = 1 if host_async else 0
        opts.stage_chunks = stage_chunks
        if host_done is not None:
            opts.host_done = host_done.cuda_event
        if ray_outcome is not None:
            opts.ray_outcome = _ptr(ray_outcome)
        if ray_box_tests is not None:
            opts.ray_box_tests = _ptr(ray_box_tests)
    check(hrpp_trace_ex(scene.handle, table.handle if table is not None else None, _ptr(rays), n, mode, _ptr(hits),
                        ctypes.byref(st) if st is not None else None, _stream_handle(stream),
                        ctypes.byref(opts) if opts is not None else None))
    return hits, (st.as_dict() if st is not None else None)


def l2_set_aside(nbytes: int) -> int:
    """Sets the current device's persisting-L2 set-aside (0 releases it);
    returns the size in force."""
    got = ctypes.c_size_t(0)
    check(hrpp_l2_set_aside(int(nbytes), ctypes.byref(got)))
    return int(got.value)


def closest_fields(hits):
    """Splits closest-hit output [n, 4] into (t, prim uint32, u, v) numpy arrays."""
    if not isinstance(hits, np.ndarray):
        hits = hits.cpu().numpy()
    h = np.ascontiguousarray(hits, np.float32)
    return h[:, 0].copy(), h[:, 1].view(np.uint32).copy(), h[:, 2].copy(), h[:, 3].copy()


class Batch:
    """Many (scene, table, rays) items traced by one persistent launch replayed
    from a CUDA graph (hrpp_batch_create / hrpp_batch_run).

    items: sequence of (Scene, Table or None, rays [n, 8] device tensor, mode).
    Output tensors are allocated here and refilled by every run()."""

    def __init__(self, items, stats: bool = False, block_threads: int = 0):
        import torch
        self.items = list(items)
        self.hits = []
        arr = (hrpp_batch_item * len(self.items))()
        for k, (scene, table, rays, mode) in enumerate(self.items):
            n = int(rays.shape[0])
            if mode == HRPP_CLOSEST_HIT:
                out = torch.empty((n, 4), dtype=torch.float32, device=rays.device)
            else:
                out = torch.empty((n,), dtype=torch.int32, device=rays.device)
            self.hits.append(out)
            arr[k] = hrpp_batch_item(scene.handle.value, table.handle.value if table is not None else None,
                                     _ptr(rays), n, mode, _ptr(out))
        h = ctypes.c_void_p()
        check(hrpp_batch_create(arr, len(self.items), 1 if stats else 0, block_threads, ctypes.byref(h)))
        self.handle = h

    def run(self, stream=None):
        check(hrpp_batch_run(self.handle, _stream_handle(stream)))

    def stats(self, k: int) -> dict:
        st = hrpp_stats()
        check(hrpp_batch_get_stats(self.handle, k, ctypes.byref(st)))
        return st.as_dict()

    def close(self):
        if getattr(self, "handle", None):
            hrpp_batch_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Proposal:
    """Learned treelet proposal (hrpp_proposal_*): a BF16 MLP on the tensor
    cores that predicts, per ray, a BVH node whose subtree is traversed first."""

    def __init__(self, scene: Scene, nodes, prim_index, root: int = 0, seed: int = 0):
        nodes = np.ascontiguousarray(nodes)
        prim_index = np.ascontiguousarray(prim_index, np.uint32)
        h = ctypes.c_void_p()
        check(hrpp_proposal_create(scene.handle, _ptr(nodes), nodes.shape[0], root, _ptr(prim_index),
                                   prim_index.shape[0], seed, ctypes.byref(h)))
        self.handle = h

    @classmethod
    def for_workload(cls, scene: Scene, s, seed: int = 0):
        return cls(scene, s.nodes, s.prim_index, s.root, seed)

    def features(self, rays, stream=None):
        import torch
        out = torch.empty((int(rays.shape[0]), 128), dtype=torch.bfloat16, device=rays.device)
        check(hrpp_proposal_features(self.handle, _ptr(rays), int(rays.shape[0]), _ptr(out), _stream_handle(stream)))
        return out

    def labels(self, closest_hits, stream=None):
        import torch
        out = torch.empty((int(closest_hits.shape[0]),), dtype=torch.int32, device=closest_hits.device)
        check(hrpp_proposal_labels(self.handle, _ptr(closest_hits), int(closest_hits.shape[0]), _ptr(out),
                                   _stream_handle(stream)))
        return out

    def train(self, rays, labels, lr: float = 1e-3, want_loss: bool = False, stream=None):
        loss = ctypes.c_float()
        check(hrpp_proposal_train(self.handle, _ptr(rays), _ptr(labels), int(rays.shape[0]), lr,
                                  ctypes.byref(loss) if want_loss else None, _stream_handle(stream)))
        return loss.value if want_loss else None

    def gradients(self, rays, labels):
        g = np.empty(HRPP_PROPOSAL_PARAMS, np.float32)
        loss = ctypes.c_float()
        check(hrpp_proposal_gradients(self.handle, _ptr(rays), _ptr(labels), int(rays.shape[0]), _ptr(g),
                                      ctypes.byref(loss)))
        return loss.value, g

    def predict(self, rays, stream=None):
        import torch
        n = int(rays.shape[0])
        nodes = torch.empty((n,), dtype=torch.int32, device=rays.device)
        classes = torch.empty((n,), dtype=torch.int32, device=rays.device)
        check(hrpp_proposal_predict(self.handle, _ptr(rays), n, _ptr(nodes), _ptr(classes), _stream_handle(stream)))
        return nodes, classes

    def get_weights(self) -> np.ndarray:
        w = np.empty(HRPP_PROPOSAL_PARAMS, np.float32)
        check(hrpp_proposal_get_weights(self.handle, _ptr(w), w.shape[0]))
        return w

    def set_weights(self, w: np.ndarray):
        w = np.ascontiguousarray(w, np.float32)
        check(hrpp_proposal_set_weights(self.handle, _ptr(w), w.shape[0]))

    def class_nodes(self) -> np.ndarray:
        out = np.empty(4096, np.int32)
        check(hrpp_proposal_class_nodes(self.handle, _ptr(out)))
        return out

    def close(self):
        if getattr(self, "handle", None):
            hrpp_proposal_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
