"""HRPP throughput benchmark on GB300.

One step = one frame of the terrain workload through the whole hot path:
1920x1080 primary closest-hit rays and 4 cosine-weighted ambient-occlusion
any-hit rays per primary hit (tmax 0.5), each batch traced by HRPP against its
own predictor table (two-phase updates included); the two batches are
independent and run side by side on two streams.  Scene: value-noise terrain
of 708x708 quads plus 64 icospheres, 2,313,248 triangles, 4-wide BVH.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl hrpp|reference]

Prints one JSON line (rank 0).  `value` is HRPP Mrays/s over all ranks with
the rays already resident on the GPU; `e2e` is the same through hrpp_trace on
pinned host buffers, every step's rays uploaded and hits downloaded inside the
timed region (the library stages each batch in chunks whose copies overlap
its traces; `e2e.torch_pipeline` is a device-buffer frame loop with its own
copy streams); `plain` gives the same library with no table on the same rays;
`gated` the same tables under a gate policy; `configs` the small-scene and
path-tracing workloads (configs 1 and 5) with their own rooflines.  The
reference arm times the CPU oracle on a bounded sample of the same workload.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "Mrays/s (any-hit, closest-hit) HRPP vs plain BVH on 1 GB300; % nodes skipped; HBM GB/s"
WORKLOAD = ("terrain 708x708 quads + 64 icospheres (2,313,248 tris), 4-wide BVH; 1920x1080 primary closest-hit "
            "rays + 4 cosine AO any-hit rays per hit (tmax 0.5); HRPP table per mode")


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=60)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="hrpp", choices=["hrpp", "reference"])
    ap.add_argument("--frames", type=int, default=4)
    ap.add_argument("--log2-entries", type=int, default=18)
    ap.add_argument("--ways", type=int, default=2)
    ap.add_argument("--precision", type=int, default=6)
    ap.add_argument("--update", default="two_phase", choices=["two_phase", "online"])
    ap.add_argument("--verify", default="root", choices=["root", "bottom_up", "none"],
                    help="how closest-hit true positives are verified (none: the paper's semantics, not exact)")
    ap.add_argument("--schedule", default="batch", choices=["batch", "compact"],
                    help="terrain: the HRPP launches' schedule (compact: the two-pass ray pool)")
    ap.add_argument("--quads", type=int, default=708)
    ap.add_argument("--spheres", type=int, default=64)
    ap.add_argument("--res", default="1920x1080")
    ap.add_argument("--l2", default="none", choices=["none", "table", "nodes"],
                    help="terrain: persisting-L2 window of the timed HRPP traces (with a set-aside)")
    ap.add_argument("--l2-set-aside-mb", type=int, default=64)
    ap.add_argument("--cpu-seconds", type=float, default=15.0)
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--traces", type=int, default=50_000_000, help="learned workload: training traces")
    ap.add_argument("--workload", default="terrain",
                    choices=["terrain", "small", "batched", "pathtrace", "learned", "shadow"],
                    help="terrain: the headline step; batched: the 64-scene uneven mix in one graph-replayed launch")
    ap.add_argument("--scenes", type=int, default=64)
    ap.add_argument("--no-learned", action="store_true", help="pathtrace: skip the learned proposal")
    ap.add_argument("--no-configs", action="store_true",
                    help="terrain: leave out the small-scene and path-tracing sub-results")
    ap.add_argument("--l2-variants", action="store_true",
                    help="terrain: also time the step with persisting-L2 windows over the table and the nodes")
    return ap.parse_args()


# ------------------------------------------------------------- helpers --

def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def frame_index(f: int, rank: int) -> int:
    """Jitter frame of local frame f on `rank`: every rank renders its own
    frames (weak scaling: per-rank work is fixed as ranks are added)."""
    return 1 + f + 1000 * rank


def reduce_max(x: float, dist, device) -> float:
    """Max over ranks (the job's time is its slowest rank's); identity alone."""
    if dist is None:
        return x
    import torch
    t = torch.tensor([x], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def reduce_sum(x: float, dist, device) -> float:
    """Sum over ranks (rays processed by the whole job); identity alone."""
    if dist is None:
        return x
    import torch
    t = torch.tensor([x], dtype=torch.float64, device=device)
    dist.all_reduce(t)
    return float(t.item())


def job_mrays_per_s(total_rays: float, max_ms: float) -> float:
    return total_rays / (max_ms * 1e-3) / 1e6


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 100 ms; stop()
    summarises the samples taken between mark(True) and mark(False) (plus one
    interval on each side)."""
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device_index: str):
        self.rows = []
        self.proc = None
        self.t0 = self.t1 = None
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                                          "-lms", "100", "-i", device_index], stdout=subprocess.PIPE,
                                         stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except (OSError, ValueError):
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.rows.append((time.time(), [x.strip() for x in line.split(",")]))

    def mark(self, start: bool):
        if start:
            self.t0 = time.time()
        else:
            self.t1 = time.time()

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"], "samples": 0}
        time.sleep(0.25)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        rows = [r for t, r in self.rows if self.t0 is not None and self.t0 - 0.1 <= t <= (self.t1 or t) + 0.1]
        if not rows:
            rows = [r for _, r in self.rows][-3:]
        sm, smax, power, reasons = [], [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            try:
                sm.append(float(r[1]))
                smax.append(float(r[2]))
                power.append(float(r[3]))
            except (ValueError, IndexError):
                continue
            for k, name in enumerate(names):
                if len(r) > 5 + k and r[5 + k].lower() == "active":
                    reasons.add(name)
        return {"sm_mhz": float(np.median(sm)) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm), "power_w_max": max(power) if power else None}


def kernel_source_hash():
    """Hash of what a recorded ncu figure depends on: the sources the recorded
    traversal kernels compile from and the generator of the scenes and BVHs
    they ran on."""
    h = hashlib.sha256()
    for f in ("csrc/trace_kernel.cuh", "csrc/device.cuh", "scenes/scenegen.c"):
        with open(os.path.join(ROOT, "paper_1910_01304_gb300", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def recorded_traffic(kernel: str, what: str = "traffic"):
    """A per-launch ncu figure from the committed summary ("traffic": DRAM
    bytes, "inst": warp instructions), if it was taken on the current kernel
    source.  Returns (value or None, source hash of the record)."""
    path = os.path.join(ROOT, "profiles", "traffic.txt")
    if not os.path.exists(path):
        return None, None
    src = kernel_source_hash()
    with open(path) as fh:
        for line in fh:
            parts = line.split()
            if len(parts) >= 4 and parts[0] == what and parts[1] == kernel:
                if parts[3] == src:
                    return float(parts[2]), parts[3]
                return None, parts[3]
    return None, None


def table_occupancy(words: np.ndarray, ways: int) -> dict:
    """Fill of a bounded table after a step: the share of valid words and the
    mean number of nodes per used set (the paper's leaves per entry)."""
    valid = words != np.uint64(0xFFFFFFFFFFFFFFFF)
    per_set = valid.reshape(-1, ways).sum(axis=1)
    used = per_set > 0
    return {"valid_words": int(valid.sum()), "words": int(words.size), "fill": float(valid.mean()),
            "nodes_per_used_set": float(per_set[used].mean()) if used.any() else 0.0}


def algorithmic_bytes(st: dict, mode_closest: bool, width: int, ways: int) -> float:
    """Bytes the method must move for one batch: rays, results, table sets,
    interior nodes, triangles (traversal and predicted leaves), insert records."""
    node_b = 64 if width == 2 else 128
    return (st["rays"] * (32 + (16 if mode_closest else 4)) + st["lookups"] * 8 * ways
            + (st["interior_nodes"] + st.get("pred_interior_nodes", 0)) * node_b
            + (st["tri_tests"] + st["pred_tri_tests"]) * 48 + st["inserts"] * 16)


def roofline_block(kernel_key: str, kname: str, ms: float, algo_bytes: float, st: dict, peak: float,
                   peak_kind: str, sm_mhz, n_sm: int) -> dict:
    """The dominant traversal launch against its bounds.  Its scene and table
    sit mostly in L1/L2, so it is bound by instruction issue (divergent SIMT
    traversal), not by HBM: `frac` is its DRAM traffic (ncu, recorded per
    kernel source in profiles/traffic.txt) over its CUDA-event time against
    the measured HBM copy bandwidth; `issue` is its warp instructions (same
    record) against one per cycle per SM sub-partition; `l2_frac` is ncu's L2
    throughput share; `effective_gbs` is the algorithmic bytes, most of which
    are L1/L2 hits."""
    sec = ms * 1e-3
    traffic, src = recorded_traffic(kernel_key)
    inst, _ = recorded_traffic(kernel_key, "inst")
    l2pct, _ = recorded_traffic(kernel_key, "l2pct")
    dram = traffic / sec / 1e9 if traffic is not None else None
    issue = None
    if inst is not None and sm_mhz:
        peak_issue = n_sm * 4 * sm_mhz * 1e6
        issue = {"warp_inst_per_launch": inst, "achieved": inst / sec, "peak": peak_issue, "unit": "warp inst/s",
                 "frac": inst / sec / peak_issue,
                 "peak_basis": f"{n_sm} SMs x 4 sub-partitions x 1 warp instruction per cycle at the sampled "
                               f"{sm_mhz:.0f} MHz"}
    return {"bound": "issue", "kernel": kname, "achieved": dram, "peak": peak, "unit": "GB/s",
            "frac": dram / peak if dram is not None else None, "peak_kind": peak_kind, "traffic": traffic,
            "what": "achieved = DRAM bytes per launch (ncu dram__bytes_read.sum + dram__bytes_write.sum on this "
                    "kernel source) / CUDA-event launch time, against the measured HBM copy bandwidth; the launch "
                    "is bound by instruction issue (issue.frac), not by HBM",
            "kernel_ms": ms, "issue": issue, "l2_frac": l2pct / 100.0 if l2pct is not None else None,
            "effective_gbs": {"value": algo_bytes / sec / 1e9, "of_hbm_peak": algo_bytes / sec / 1e9 / peak,
                              "algorithmic_bytes_per_launch": algo_bytes,
                              "note": "rays, results, table sets, nodes, triangles and insert records the method "
                                      "touches, per launch / launch time; most node and triangle bytes are L1/L2 "
                                      "hits, so this is not DRAM bandwidth"},
            "node_tests_per_s": {"box": (st["box_tests"] + st["pred_box_tests"]) / sec,
                                 "triangle": (st["tri_tests"] + st["pred_tri_tests"]) / sec},
            "traffic_source_hash": src, "kernel_source_hash": kernel_source_hash()}


def load_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as fh:
            d = json.load(fh)
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


# ----------------------------------------------------------- workload --

def make_frames(args, rank, scene_w, H, g, torch):
    """Primary rays per frame (jittered), their plain closest hits on the GPU,
    and the ambient-occlusion rays generated from those hits on the host."""
    from paper_1910_01304_gb300.scenes import workloads as W
    frames = []
    for f in range(args.frames):
        prim = scene_w.primary_rays(frame=frame_index(f, rank))
        dprim = torch.from_numpy(prim).cuda()
        hits, _ = H.trace(g, dprim, H.HRPP_CLOSEST_HIT)
        hh = hits.cpu().numpy()
        t, p = hh[:, 0], hh[:, 1].view(np.uint32)
        ao, _ = W.secondary_ao(scene_w, prim, t, p, frame=frame_index(f, rank))
        frames.append({"prim": dprim, "ao": torch.from_numpy(ao).cuda(), "prim_h": prim, "ao_h": ao})
    return frames


def host_threads():
    """Host cores this process may run on."""
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count() or 1


class OracleThreads:
    """The oracle's trace, unchanged, run ray-parallel across the host cores.
    Thread i takes rays i, i+k, i+2k, ... of each batch (a static
    partition that spreads sky and terrain rays evenly) and, for HRPP, its own
    pair of tables; the ctypes call releases the interpreter lock, so the k
    calls run concurrently.  Chunk copies and result gathering sit outside
    the timed calls."""

    def __init__(self, O, sw, k: int, table_args=None):
        from concurrent.futures import ThreadPoolExecutor
        self.O, self.sw, self.k = O, sw, k
        self.pool = ThreadPoolExecutor(k)
        self.tables = None
        if table_args is not None:
            self.tables = {m: [O.Table(*table_args) for _ in range(k)] for m in (O.CLOSEST_HIT, O.ANY_HIT)}

    def split(self, rays):
        return [np.ascontiguousarray(rays[i::self.k]) for i in range(self.k)]

    def trace(self, chunks, mode):
        """Traces prepared chunks; returns (per-chunk hits, seconds)."""
        O, sw = self.O, self.sw
        tabs = self.tables[mode] if self.tables is not None else [None] * self.k
        t0 = time.perf_counter()
        futs = [self.pool.submit(O.trace, sw.tris, sw.nodes, sw.prim_index, sw.root, c, mode, tb)
                for c, tb in zip(chunks, tabs) if len(c)]
        res = [f.result()[0] for f in futs]
        return res, time.perf_counter() - t0

    def gather(self, res, n, dtype):
        out = np.empty(n, dtype)
        for i, r in enumerate(res):
            out[i::self.k] = r
        return out

    def close(self):
        self.pool.shutdown()


def run_reference(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return 0
    import oracle as O
    from paper_1910_01304_gb300.scenes import workloads as W
    w, h = map(int, args.res.split("x"))
    sw = W.terrain_scene(quads=args.quads, n_spheres=args.spheres, res=(w, h))
    prim = sw.primary_rays(frame=1)
    k = host_threads()
    ot = OracleThreads(O, sw, k, (args.log2_entries, args.ways, args.precision, O.TWO_PHASE))
    # each step: a bounded sample of the step's work: 16 whole image rows per
    # host thread, spread evenly down the frame (sky and near terrain in the
    # frame's proportions), traced as primary closest-hit rays, then the AO
    # any-hit rays of their hits; each thread keeps its own tables across
    # steps
    n_rows = min(h, 16 * k)
    band = n_rows * w

    def step(j):
        """Returns (rays traced, seconds spent tracing)."""
        rows = [(j + r * (h // n_rows)) % h for r in range(n_rows)]
        sp = np.ascontiguousarray(np.concatenate([prim[r * w:(r + 1) * w] for r in rows]))
        res, t_p = ot.trace(ot.split(sp), O.CLOSEST_HIT)
        ph = ot.gather(res, len(sp), O.HIT_DTYPE)
        sa, _ = W.secondary_ao(sw, sp, ph["t"], ph["prim"], frame=1)
        _, t_a = ot.trace(ot.split(sa), O.ANY_HIT)
        return len(sp) + len(sa), t_p + t_a

    for j in range(args.warmup):
        step(j * 7)
    rays, dt = 0, 0.0
    for j in range(args.steps):
        r, t = step((args.warmup + j) * 7)
        rays += r
        dt += t
    ot.close()
    v = rays / dt / 1e6
    sample = (f"per step: {n_rows} whole rows spread evenly down a {w}x{h} frame ({band} primary closest-hit rays) and "
              f"the AO any-hit rays of their hits, oracle HRPP two-phase on {k} host threads (thread i takes rays "
              "i, i+k, ... with its own tables); the AO generation between the two traces is not timed")
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": "Mrays/s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": dt / args.steps * 1e3,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": WORKLOAD, "sample": sample},
            "cpu_baseline": {"value": v, "unit": "Mrays/s", "cores": k, "kind": "oracle", "sample": sample},
            "e2e": {"value": v, "unit": "Mrays/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def cpu_baseline(args, sw, frames):
    """The oracle, as it stands, on the host cores.

    value: HRPP (two-phase) over all of frame 0 on every host core, each
    thread with its own tables warmed by its share of the other frames (the
    GPU step's protocol, per thread); plain: the same rays without tables;
    single_core: HRPP on one core over a sample of frame 0 with cold tables."""
    import oracle as O
    k = host_threads()
    ta = (args.log2_entries, args.ways, args.precision, O.TWO_PHASE)
    ot = OracleThreads(O, sw, k, ta)
    for f in range(1, len(frames)):
        ot.trace(ot.split(frames[f]["prim_h"]), O.CLOSEST_HIT)
        ot.trace(ot.split(frames[f]["ao_h"]), O.ANY_HIT)
    cp, ca = ot.split(frames[0]["prim_h"]), ot.split(frames[0]["ao_h"])
    n0 = len(frames[0]["prim_h"]) + len(frames[0]["ao_h"])
    _, t_p = ot.trace(cp, O.CLOSEST_HIT)
    _, t_a = ot.trace(ca, O.ANY_HIT)
    ot.close()
    v_hrpp = n0 / (t_p + t_a) / 1e6
    plain = OracleThreads(O, sw, k)
    _, u_p = plain.trace(cp, O.CLOSEST_HIT)
    _, u_a = plain.trace(ca, O.ANY_HIT)
    plain.close()
    v_plain = n0 / (u_p + u_a) / 1e6
    single = cpu_single_core(args, sw, frames)
    return {"value": v_hrpp, "unit": "Mrays/s", "cores": k, "kind": "oracle",
            "sample": f"all of frame 0 ({len(frames[0]['prim_h'])} primary closest-hit + {len(frames[0]['ao_h'])} "
                      f"AO any-hit rays), oracle HRPP two-phase on {k} host threads (thread i takes rays i, i+k, ... "
                      f"with its own tables, warmed by its share of {len(frames) - 1} other frames), "
                      f"{t_p + t_a:.2f} s",
            "plain": {"value": v_plain, "unit": "Mrays/s", "cores": k, "seconds": u_p + u_a},
            "single_core": single}


def cpu_single_core(args, sw, frames):
    """The oracle, as it stands, on a bounded sample of frame 0 (one core)."""
    import oracle as O
    prim = frames[0]["prim_h"]
    ao = frames[0]["ao_h"]
    tc = O.Table(args.log2_entries, args.ways, args.precision, O.TWO_PHASE)
    ta = O.Table(args.log2_entries, args.ways, args.precision, O.TWO_PHASE)
    # calibrate the sample to about cpu_seconds of work
    probe_p, probe_a = prim[::512], ao[::512]
    t0 = time.perf_counter()
    O.trace(sw.tris, sw.nodes, sw.prim_index, sw.root, probe_p, O.CLOSEST_HIT, tc)
    O.trace(sw.tris, sw.nodes, sw.prim_index, sw.root, probe_a, O.ANY_HIT, ta)
    per = (time.perf_counter() - t0) / (len(probe_p) + len(probe_a))
    n_total = int(max(10000, min(len(prim) + len(ao), args.cpu_seconds / max(per, 1e-9))))
    frac = n_total / (len(prim) + len(ao))
    stride = max(1, int(round(1 / max(frac, 1e-9))))
    sp, sa = prim[::stride], ao[::stride]
    tc = O.Table(args.log2_entries, args.ways, args.precision, O.TWO_PHASE)
    ta = O.Table(args.log2_entries, args.ways, args.precision, O.TWO_PHASE)
    t0 = time.perf_counter()
    O.trace(sw.tris, sw.nodes, sw.prim_index, sw.root, sp, O.CLOSEST_HIT, tc)
    O.trace(sw.tris, sw.nodes, sw.prim_index, sw.root, sa, O.ANY_HIT, ta)
    dt = time.perf_counter() - t0
    return {"value": (len(sp) + len(sa)) / dt / 1e6, "unit": "Mrays/s", "cores": 1, "kind": "oracle",
            "sample": f"every {stride}th ray of frame 0: {len(sp)} primary closest-hit + {len(sa)} AO any-hit rays, "
                      f"HRPP two-phase, {dt:.1f} s on one host core"}


def batched_items(args):
    """The 64-scene uneven workload: per scene, its rays for args.frames
    frames, each split into camera rays (closest-hit) and random rays
    (any-hit)."""
    from paper_1910_01304_gb300.scenes import workloads as W
    out = []
    for s, rays in W.batched_workload(n_scenes=args.scenes, seed=3):
        n, half = len(rays), len(rays) // 2
        per_frame = [rays] + [W.batched_rays(s, n, f) for f in range(1, max(1, args.frames))]
        out.append((s, [(r[:half], r[half:]) for r in per_frame]))
    return out


def batched_roofline(step_ms: float, algo_bytes: float, peak: float, peak_kind: str) -> dict:
    """The batched step (two k_trace_batch launches side by side, then
    k_apply_batch) against HBM: DRAM bytes of its launches (ncu record per
    kernel source) over the step's CUDA-event time.  Like the single-scene
    launches it is bound by instruction issue; the algorithmic bytes, mostly
    L1/L2 hits, are reported as effective_gbs."""
    sec = step_ms * 1e-3
    traffic, _ = recorded_traffic("batched_step")  # all launches of one replay
    dram = traffic / sec / 1e9 if traffic is not None else None
    return {"bound": "issue", "kernel": "k_trace_batch<4, closest> || k_trace_batch<4, any> + k_apply_batch (graph)",
            "achieved": dram, "peak": peak, "unit": "GB/s", "frac": dram / peak if dram is not None else None,
            "peak_kind": peak_kind, "traffic": traffic,
            "what": "achieved = DRAM bytes of the step's launches (ncu, this kernel source) / step time",
            "effective_gbs": {"value": algo_bytes / sec / 1e9, "of_hbm_peak": algo_bytes / sec / 1e9 / peak,
                              "note": "algorithmic bytes per step / step time; mostly L1/L2 hits, not DRAM"},
            "kernel_source_hash": kernel_source_hash()}


def run_batched(args):
    """Config 3: the uneven 64-scene batch in one persistent launch replayed
    from a CUDA graph, with table and launch parameters picked by the
    autotuner.  Each step restores tables warmed by the other frames, then
    replays frame 0."""
    rank, world, local = dist_env()
    import torch
    torch.cuda.set_device(local)
    import __graft_entry__
    __graft_entry__.build()
    from paper_1910_01304_gb300 import autotune
    from paper_1910_01304_gb300 import hrpp as H
    t0 = time.time()
    work = batched_items(args)
    gen_s = time.time() - t0
    items, frames, n_tris = [], [[] for _ in range(max(1, args.frames))], 0
    for s, per_frame in work:
        g = H.Scene.from_workload(s)
        n_tris += s.n_tris
        for half, mode in ((0, H.HRPP_CLOSEST_HIT), (1, H.HRPP_ANY_HIT)):
            if len(per_frame[0][half]) == 0:
                continue
            items.append((g, mode))
            for f, pair in enumerate(per_frame):
                frames[f].append(torch.from_numpy(np.ascontiguousarray(pair[half])).cuda())
    n_rays = sum(int(r.shape[0]) for r in frames[0])
    stream = torch.cuda.current_stream()
    t0 = time.time()
    tuned = autotune.tune_batch(items, frames, reps=3)
    tune_s = time.time() - t0

    def timed(setup):
        for _ in range(args.warmup):
            setup.step()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(args.steps):
            setup.step()
        e1.record(stream)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / args.steps

    res = {}
    for name, cfg in (("hrpp", (tuned["closest"], tuned["any"])), ("plain", (None, None))):
        setup = autotune.BatchSetup(items, frames, cfg[0], cfg[1], tuned["block_threads"])
        res[name] = timed(setup)
        setup.close()
    # one replay of the tuned batch under an NVTX range (ncu --nvtx-include
    # profile_batched/: the step's launches, whose DRAM bytes the roofline reads)
    setup = autotune.BatchSetup(items, frames, tuned["closest"], tuned["any"], tuned["block_threads"])
    setup.step()
    torch.cuda.synchronize()
    torch.cuda.nvtx.range_push("profile_batched")
    setup.step()
    torch.cuda.synchronize()
    torch.cuda.nvtx.range_pop()
    setup.close()
    setup = autotune.BatchSetup(items, frames, tuned["closest"], tuned["any"], tuned["block_threads"], stats=True)
    setup.step()
    torch.cuda.synchronize()
    stats = [setup.batches[0].stats(k) for k in range(len(items))]
    setup.close()

    # the same frame-0 rays with one plain hrpp_trace launch per item, for
    # comparison with the single persistent launch
    outs = [torch.empty((r.shape[0], 4) if mode == H.HRPP_CLOSEST_HIT else (r.shape[0],),
                        dtype=torch.float32 if mode == H.HRPP_CLOSEST_HIT else torch.int32, device="cuda")
            for (g, mode), r in zip(items, frames[0])]

    class PerItem:
        def step(self):
            for (g, mode), r, o in zip(items, frames[0], outs):
                H.trace(g, r, mode, None, hits=o, block_threads=tuned["block_threads"])
    per_item_ms = timed(PerItem())

    def ways_of(mode):
        cfg = tuned["closest"] if mode == H.HRPP_CLOSEST_HIT else tuned["any"]
        return cfg["ways"] if cfg else 0

    hb = sum(algorithmic_bytes(st, items[k][1] == H.HRPP_CLOSEST_HIT, 4, ways_of(items[k][1]))
             for k, st in enumerate(stats))
    peak, peak_kind = load_peaks()
    tp = sum(st["true_pos"] for st in stats)
    lookups = sum(st["lookups"] for st in stats)
    n_tables = sum(1 for _, mode in items if (tuned["closest"] if mode == H.HRPP_CLOSEST_HIT else tuned["any"]))
    line = {"metric": METRIC, "value": n_rays / (res["hrpp"] * 1e-3) / 1e6, "unit": "Mrays/s", "n_gpus": 1,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": res["hrpp"], "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": f"batched: {len(work)} scenes (terrain / icosphere clusters / soup), log-uniform "
                                   f"10k-2M tris ({n_tris} total), log-uniform 4k-2M rays per scene ({n_rays} total), "
                                   "camera rays closest-hit + uniform-sphere rays any-hit, one persistent launch "
                                   "replayed from a CUDA graph", "items": len(items), "frames": args.frames,
                       "protocol": f"each step: restore the tables warmed by {args.frames - 1} other frames "
                                   "(jittered camera rays, re-drawn random rays), then replay frame 0",
                       "generation_s": gen_s},
            "autotune": {"closest": tuned["closest"], "any": tuned["any"], "block_threads": tuned["block_threads"],
                         "tuned_ms": tuned["ms"], "plain_ms": tuned["plain_ms"], "candidates": len(tuned["tried"]),
                         "seconds": tune_s, "items_with_a_table": n_tables},
            "plain": {"value": n_rays / (res["plain"] * 1e-3) / 1e6, "ms_per_step": res["plain"],
                      "speedup_hrpp_over_plain": res["plain"] / res["hrpp"]},
            "plain_per_item_launches": {"value": n_rays / (per_item_ms * 1e-3) / 1e6, "ms_per_step": per_item_ms,
                                        "launches": len(items)},
            "roofline": batched_roofline(res["hrpp"], hb, peak, peak_kind),
            "true_pos": tp, "lookups": lookups,
            "gpu_launches": (2 if n_tables else 1) * args.steps}
    print(json.dumps(line), flush=True)
    return 0


# Gate thresholds (true positives per 65536 lookups) of the "gated" variants:
# an any-hit true positive saves a whole traversal, and on these workloads a
# lookup costs about 4 % of one (the terrain AO launch: 1.108 against
# 1.066 ms), so hit-any tables keep predicting above 4 %; an exact closest-hit
# true positive still traverses, bounded by its hit, which saved at most
# 3.4 % of its box tests here -- less than the lookup costs -- so hit-all
# tables stay closed (100 %) and keep only their 1-in-32 sample.
GATE = {"closest": 65536, "any": 2621}
GATE_SAMPLE_LOG2 = 5


def make_tables(H, log2e, ways, precision, gated: bool, update=0):
    """(closest, any) tables, with the gate policy when gated."""
    out = []
    for name in ("closest", "any"):
        t = H.Table(log2e, ways, precision, update)
        if gated:
            t.set_gate(GATE[name], GATE_SAMPLE_LOG2)
        out.append(t)
    return tuple(out)


def summarize_config(line: dict) -> dict:
    """The part of a config's own bench line that the headline line carries."""
    keep = ("value", "unit", "ms_per_step", "plain", "gated", "per_mode_kernel_ms", "skipped", "roofline", "config",
            "sequential", "per_bounce")
    out = {k: line[k] for k in keep if k in line}
    out["speedup_hrpp_over_plain"] = line["plain"]["speedup_hrpp_over_plain"]
    return out


def limit_study() -> dict | None:
    """The paper's limit study on configs 1 and 2 (unbounded sequential table,
    8 jittered frames as 8 spp), computed by the oracle and stored by
    tests/golden/make_limit_study.py; None if it was not generated."""
    path = os.path.join(ROOT, "tests", "golden", "limit_study.json")
    if not os.path.exists(path):
        return None
    with open(path) as fh:
        d = json.load(fh)
    return {"what": d["what"],
            "entries": [{k: e[k] for k in ("workload", "query", "precision", "rays", "prediction_ratio",
                                           "skipped_limit_box_tests", "table_mb")} for e in d["entries"]]}


def max_sm_mhz():
    """The SM clock the issue-rate peak assumes when no clock was sampled:
    the maximum MEASURED_PEAKS.json records (2,070 MHz on GB300)."""
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as fh:
            return float(json.load(fh).get("sm_max_mhz", 2070.0))
    return 2070.0


def run_small(args, emit: bool = True, sm_mhz=None):
    """Config 1: the small scene (1,792 tris, binary BVH), 256x256 primary
    closest-hit rays and one shadow any-hit ray per hit, 2^12-entry
    direct-mapped tables.  Each step restores the tables warmed by the other
    frames and traces frame 0's two batches side by side; the step is
    captured into a CUDA graph (these launches are latency-bound) and
    replayed.  Returns the line (printed when emit)."""
    rank, world, local = dist_env()
    import torch
    torch.cuda.set_device(local)
    import __graft_entry__
    __graft_entry__.build()
    from paper_1910_01304_gb300 import hrpp as H
    from paper_1910_01304_gb300.scenes import workloads as W
    s = W.small_scene()
    g = H.Scene.from_workload(s)
    frames = []
    for f in range(max(2, args.frames)):
        prim = s.primary_rays(frame=frame_index(f, rank))
        hits, _ = H.trace(g, torch.from_numpy(prim).cuda(), H.HRPP_CLOSEST_HIT)
        hh = hits.cpu().numpy()
        shadow, _ = W.secondary_shadow(s, prim, hh[:, 0], hh[:, 1].view(np.uint32))
        frames.append((torch.from_numpy(prim).cuda(), torch.from_numpy(shadow).cuda()))

    def warm(gated):
        tabs = make_tables(H, 12, 1, 6, gated)
        for prim, shadow in frames[1:]:
            H.trace(g, prim, H.HRPP_CLOSEST_HIT, tabs[0])
            H.trace(g, shadow, H.HRPP_ANY_HIT, tabs[1])
        snaps = make_tables(H, 12, 1, 6, gated)
        snaps[0].copy_from(tabs[0])
        snaps[1].copy_from(tabs[1])
        return tabs, snaps

    prim, shadow = frames[0]
    out_c = torch.empty((prim.shape[0], 4), dtype=torch.float32, device="cuda")
    out_a = torch.empty((shadow.shape[0],), dtype=torch.int32, device="cuda")
    n_rays = int(prim.shape[0] + shadow.shape[0])

    fork_stream = torch.cuda.Stream()

    def step(tables, snaps):
        # the primary and shadow batches are independent inputs with one
        # table each: each branch restores its table and traces its batch,
        # side by side (fork and join, also under capture)
        cur = torch.cuda.current_stream()
        fork = torch.cuda.Event()
        fork.record(cur)
        fork_stream.wait_event(fork)
        if tables[0] is not None:
            tables[1].copy_from(snaps[1], stream=fork_stream)
            tables[0].copy_from(snaps[0])
        H.trace(g, shadow, H.HRPP_ANY_HIT, tables[1], hits=out_a, stream=fork_stream)
        H.trace(g, prim, H.HRPP_CLOSEST_HIT, tables[0], hits=out_c)
        join = torch.cuda.Event()
        join.record(fork_stream)
        cur.wait_event(join)

    def timed(tables, snaps):
        graph, replay = None, lambda: step(tables, snaps)
        try:
            side = torch.cuda.Stream()
            side.wait_stream(torch.cuda.current_stream())
            with torch.cuda.stream(side):
                for _ in range(3):
                    step(tables, snaps)
            torch.cuda.current_stream().wait_stream(side)
            graph = torch.cuda.CUDAGraph()
            with torch.cuda.graph(graph):
                step(tables, snaps)
            replay = graph.replay
        except Exception as exc:  # capture unsupported: time plain launches
            print(f"CUDA graph capture failed ({exc}); timing launches", file=sys.stderr)
            graph = None
        for _ in range(args.warmup):
            replay()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(args.steps):
            replay()
        e1.record()
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / args.steps, graph is not None

    tabs, snaps = warm(False)
    gtabs, gsnaps = warm(True)
    ms, graphed = timed(tabs, snaps)
    g_ms, _ = timed(gtabs, gsnaps)
    p_ms, p_graphed = timed((None, None), (None, None))

    # each launch alone (no graph), from the restored tables: the roofline's
    # kernel times, and the counters of one step
    def launch_ms(rays, mode, table, snap, hits, reps=20):
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(reps)]
        for a, b in ev:
            a.record(); b.record()
        for e in [None] * 3 + ev:
            if table is not None:
                table.copy_from(snap)
            H.trace(g, rays, mode, table, hits=hits, kernel_events=e)
        torch.cuda.synchronize()
        return float(np.median([a.elapsed_time(b) for a, b in ev]))
    kt = {"closest": launch_ms(prim, H.HRPP_CLOSEST_HIT, tabs[0], snaps[0], out_c),
          "any": launch_ms(shadow, H.HRPP_ANY_HIT, tabs[1], snaps[1], out_a)}
    # one restored step under an NVTX range (ncu --nvtx-include profile_small/)
    torch.cuda.nvtx.range_push("profile_small")
    for t, sn in zip(tabs, snaps):
        t.copy_from(sn)
    H.trace(g, prim, H.HRPP_CLOSEST_HIT, tabs[0], hits=out_c)
    H.trace(g, shadow, H.HRPP_ANY_HIT, tabs[1], hits=out_a)
    torch.cuda.synchronize()
    torch.cuda.nvtx.range_pop()
    for t, sn in zip(tabs, snaps):
        t.copy_from(sn)
    for t, sn in zip(gtabs, gsnaps):
        t.copy_from(sn)
    _, sc = H.trace(g, prim, H.HRPP_CLOSEST_HIT, tabs[0], stats=True)
    _, sa = H.trace(g, shadow, H.HRPP_ANY_HIT, tabs[1], stats=True)
    _, gc = H.trace(g, prim, H.HRPP_CLOSEST_HIT, gtabs[0], stats=True)
    _, ga = H.trace(g, shadow, H.HRPP_ANY_HIT, gtabs[1], stats=True)
    _, pc = H.trace(g, prim, H.HRPP_CLOSEST_HIT, None, stats=True)
    _, pa = H.trace(g, shadow, H.HRPP_ANY_HIT, None, stats=True)
    g.check()

    def skipped(h, p):
        return {"prediction_ratio": h["true_pos"] / max(1, h["rays"]),
                "skipped_exact_box_tests": 1.0 - h["box_tests"] / max(1, p["box_tests"]), "rays": h["rays"],
                "gated": h["gated"]}

    peak, peak_kind = load_peaks()
    dom = "any" if kt["any"] >= kt["closest"] else "closest"
    st_dom = sa if dom == "any" else sc
    n_sm = torch.cuda.get_device_properties(local).multi_processor_count
    roof = roofline_block(f"small_bvh2_{dom}", f"k_trace<2, {dom}, hrpp> (small scene)", kt[dom],
                          algorithmic_bytes(st_dom, dom == "closest", 2, 1), st_dom, peak, peak_kind,
                          sm_mhz or max_sm_mhz(), n_sm)
    value = job_mrays_per_s(n_rays, ms)
    line = {"metric": METRIC, "value": value, "unit": "Mrays/s", "n_gpus": 1, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": "small scene: icosphere (1,280 tris) on a 16x16-quad ground (512 tris), binary "
                                   "BVH; 256x256 primary closest-hit rays + 1 shadow any-hit ray per hit",
                       "rays_per_step": n_rays, "frames": max(2, args.frames),
                       "table": {"log2_entries": 12, "ways": 1, "precision": 6},
                       "protocol": "each step: restore the tables warmed by the other frames, trace frame 0 (primary and shadow "
                                    "batches side by side)",
                       "cuda_graph": graphed and p_graphed},
            "plain": {"value": job_mrays_per_s(n_rays, p_ms), "ms_per_step": p_ms, "speedup_hrpp_over_plain": p_ms / ms},
            "gated": {"value": job_mrays_per_s(n_rays, g_ms), "ms_per_step": g_ms, "speedup_over_plain": p_ms / g_ms,
                      "gate": {"min_tp_per_65536": GATE, "sample_log2": GATE_SAMPLE_LOG2},
                      "skipped": {"closest": skipped(gc, pc), "any": skipped(ga, pa)}},
            "per_mode_kernel_ms": kt,
            "skipped": {"closest": skipped(sc, pc), "any": skipped(sa, pa)},
            "roofline": roof,
            "gpu_launches": 4 * args.steps}
    if emit:
        print(json.dumps(line), flush=True)
    return line


def run_pathtrace(args, emit: bool = True, sm_mhz=None):
    """Config 5: 1280x720 x 4 spp x 5 diffuse bounces (+ one shadow ray per
    bounce) on the 4.28M-triangle closed terrain, HRPP vs plain per bounce.
    Each step restores the tables warmed by the other frames and traces frame
    0, the closest-hit and shadow chains side by side; a second pass in
    sequence times every launch alone.  Returns the line (printed when
    emit)."""
    rank, world, local = dist_env()
    import torch
    torch.cuda.set_device(local)
    import __graft_entry__
    __graft_entry__.build()
    from paper_1910_01304_gb300 import hrpp as H
    from paper_1910_01304_gb300.scenes import workloads as W
    s = W.pathtrace_scene()
    g = H.Scene.from_workload(s)

    def gpu_closest(rays):
        hits, _ = H.trace(g, torch.from_numpy(np.ascontiguousarray(rays)).cuda(), H.HRPP_CLOSEST_HIT)
        h = hits.cpu().numpy()
        return h[:, 0].copy(), h[:, 1].view(np.uint32).copy()

    frames = []
    for f in range(max(2, args.frames)):
        bs = W.path_bounces(s, W.path_primary(s, spp=4, frame=frame_index(f, rank)), gpu_closest, bounces=5,
                            frame=frame_index(f, rank))
        frames.append([(torch.from_numpy(c).cuda(), torch.from_numpy(sh).cuda()) for c, sh in bs])
    nb = len(frames[0])
    stream = torch.cuda.current_stream()
    side = torch.cuda.Stream()

    # the terrain protocol: the other frames warm the tables once, a device
    # snapshot is restored at the start of every step, which then traces
    # frame 0's bounces in order (no ray meets its own insert)
    def warm(gated):
        tabs = make_tables(H, args.log2_entries, args.ways, args.precision, gated)
        for fr in frames[1:]:
            for c, sh in fr:
                H.trace(g, c, H.HRPP_CLOSEST_HIT, tabs[0])
                H.trace(g, sh, H.HRPP_ANY_HIT, tabs[1])
        snaps = make_tables(H, args.log2_entries, args.ways, args.precision, gated)
        snaps[0].copy_from(tabs[0])
        snaps[1].copy_from(tabs[1])
        return tabs, snaps

    def step(tables, snaps, ev=None, concurrent=True):
        """Restore the tables, then trace frame 0's bounces.  concurrent: the
        closest-hit chain and the shadow chain (one table each, independent)
        run side by side; otherwise in sequence, each launch timed alone."""
        if tables[0] is not None:
            tables[0].copy_from(snaps[0])
            tables[1].copy_from(snaps[1])
        if concurrent:
            fork = torch.cuda.Event()
            fork.record(stream)
            side.wait_event(fork)
        for b, (c, sh) in enumerate(frames[0]):
            H.trace(g, c, H.HRPP_CLOSEST_HIT, tables[0], kernel_events=ev[b][0] if ev else None)
            H.trace(g, sh, H.HRPP_ANY_HIT, tables[1], kernel_events=ev[b][1] if ev else None,
                    stream=side if concurrent else None)
        if concurrent:
            join = torch.cuda.Event()
            join.record(side)
            stream.wait_event(join)

    def mk():
        e = torch.cuda.Event(enable_timing=True)
        e.record(stream)
        return e

    variants = {"hrpp": warm(False), "gated": warm(True), "plain": ((None, None), (None, None))}
    out = {}
    for name, (tables, snaps) in variants.items():
        res = []
        for conc in ((True, False) if name != "gated" else (True,)):
            for _ in range(args.warmup):
                step(tables, snaps, concurrent=conc)
            evs = None if conc else [[[(mk(), mk()), (mk(), mk())] for _ in range(nb)] for _ in range(args.steps)]
            torch.cuda.synchronize()
            e0, e1 = mk(), mk()
            e0.record(stream)
            for k in range(args.steps):
                step(tables, snaps, evs[k] if evs else None, concurrent=conc)
            e1.record(stream)
            torch.cuda.synchronize()
            res.append(e0.elapsed_time(e1) / args.steps)
        per_b = None
        if not conc:
            per_b = [[sum(evs[k][b][m][0].elapsed_time(evs[k][b][m][1]) for k in range(args.steps)) / args.steps
                      for m in range(2)] for b in range(nb)]
        out[name] = (res[0], per_b, res[1] if len(res) > 1 else None)
    rays_frame = sum(int(c.shape[0] + sh.shape[0]) for c, sh in frames[0])
    per_bounce = []
    (tab_c, tab_a), (snap_c, snap_a) = variants["hrpp"]
    # one restored step in sequence under an NVTX range (ncu --nvtx-include
    # profile_pathtrace/; its second closest-hit launch is bounce 1)
    torch.cuda.nvtx.range_push("profile_pathtrace")
    step((tab_c, tab_a), (snap_c, snap_a), concurrent=False)
    torch.cuda.synchronize()
    torch.cuda.nvtx.range_pop()
    tab_c.copy_from(snap_c)
    tab_a.copy_from(snap_a)
    stats_b = []
    for b, (c, sh) in enumerate(frames[0]):
        _, sc = H.trace(g, c, H.HRPP_CLOSEST_HIT, tab_c, stats=True)
        _, sa = H.trace(g, sh, H.HRPP_ANY_HIT, tab_a, stats=True)
        stats_b.append((sc, sa))
        hc, ha = out["hrpp"][1][b]
        pc, pa = out["plain"][1][b]
        per_bounce.append({"bounce": b, "closest_rays": int(c.shape[0]), "shadow_rays": int(sh.shape[0]),
                           "closest_mrays": {"hrpp": c.shape[0] / hc / 1e3, "plain": c.shape[0] / pc / 1e3},
                           "shadow_mrays": {"hrpp": sh.shape[0] / ha / 1e3, "plain": sh.shape[0] / pa / 1e3},
                           "prediction_ratio": {"closest": sc["true_pos"] / sc["rays"], "any": sa["true_pos"] / sa["rays"]}})
    g.check()
    # roofline: the bounce-1 closest-hit launch (incoherent rays over a scene
    # larger than L2)
    peak, peak_kind = load_peaks()
    n_sm = torch.cuda.get_device_properties(local).multi_processor_count
    b1 = min(1, nb - 1)
    roof = roofline_block("pt_bvh4_closest_b1", "k_trace<4, closest, hrpp> (path tracing, bounce 1)",
                          out["hrpp"][1][b1][0], algorithmic_bytes(stats_b[b1][0], True, 4, args.ways), stats_b[b1][0],
                          peak, peak_kind, sm_mhz or max_sm_mhz(), n_sm)
    learned = None if args.no_learned else pathtrace_learned(H, g, s, frames, per_bounce, stream)
    line = {"metric": METRIC, "value": rays_frame / (out["hrpp"][0] * 1e-3) / 1e6, "unit": "Mrays/s", "n_gpus": 1,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": out["hrpp"][0], "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": f"path tracing: {s.n_tris} tris (2048x1024-quad terrain, 256 icospheres, dome), "
                                   "1280x720 x 4 spp x 5 diffuse bounces + 1 shadow ray per bounce",
                       "rays_per_step": rays_frame, "frames": max(2, args.frames),
                       "protocol": f"each step: restore the tables warmed by {max(2, args.frames) - 1} other frame(s), "
                                   "then trace frame 0's bounces in order, the closest-hit chain and the shadow chain "
                                   "side by side (one table each)",
                       "table": {"log2_entries": args.log2_entries, "ways": args.ways, "precision": args.precision}},
            "plain": {"value": rays_frame / (out["plain"][0] * 1e-3) / 1e6, "ms_per_step": out["plain"][0],
                      "speedup_hrpp_over_plain": out["plain"][0] / out["hrpp"][0]},
            "gated": {"value": rays_frame / (out["gated"][0] * 1e-3) / 1e6, "ms_per_step": out["gated"][0],
                      "speedup_over_plain": out["plain"][0] / out["gated"][0],
                      "gate": {"min_tp_per_65536": GATE, "sample_log2": GATE_SAMPLE_LOG2}},
            "sequential": {"value": rays_frame / (out["hrpp"][2] * 1e-3) / 1e6,
                           "plain_value": rays_frame / (out["plain"][2] * 1e-3) / 1e6, "unit": "Mrays/s",
                           "how": "the same steps with every launch in sequence (per-bounce kernel times taken here)"},
            "per_bounce": per_bounce, "roofline": roof, "learned": learned, "gpu_launches": 4 * nb * args.steps}
    if emit:
        print(json.dumps(line), flush=True)
    return line


def run_shadow(args, emit: bool = True):
    """Hit-any locality on the terrain scene: its primary hits' shadow rays
    toward a low point light (workloads.TERRAIN_SUN, which shadows 86 % of
    the hits) instead of AO rays, the simple-lighting case in which the
    paper finds hit-any locality (Sec. 6.1).  Any-hit true positives are
    exact, so every skip is kept.  Each timed call restores a table warmed by
    3 other jittered frames and traces frame 0's shadow rays; the events
    bracket the whole call (traversal and table update).  Plain, the fused
    BATCH schedule and the two-pass COMPACT schedule, with config 2's table
    (2^18 x 2) and a larger one (2^22 x 4).  Not one of the five configs: a
    measurement of what exact HRPP gains where the rays have the locality the
    method needs."""
    rank, world, local = dist_env()
    import torch
    torch.cuda.set_device(local)
    import __graft_entry__
    __graft_entry__.build()
    from paper_1910_01304_gb300 import hrpp as H
    from paper_1910_01304_gb300.scenes import workloads as W
    s = W.terrain_scene()
    g = H.Scene.from_workload(s)
    frames = []
    for f in range(4):
        prim = s.primary_rays(frame=frame_index(f, rank))
        hits, _ = H.trace(g, torch.from_numpy(prim).cuda(), H.HRPP_CLOSEST_HIT)
        hh = hits.cpu().numpy()
        sh, _ = W.secondary_shadow(s, prim, hh[:, 0], hh[:, 1].view(np.uint32), light=W.TERRAIN_SUN)
        frames.append(torch.from_numpy(sh).cuda())
    rays0 = frames[0]
    n = int(rays0.shape[0])
    out = torch.empty((n,), dtype=torch.int32, device="cuda")
    stream = torch.cuda.current_stream()
    reps = max(5, args.steps)

    def call_ms(fn):
        """Median over reps of one call bracketed by events (setup() before)."""
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(reps)]
        for _ in range(max(3, args.warmup)):
            fn(None)
        torch.cuda.synchronize()
        for e in ev:
            fn(e)
        torch.cuda.synchronize()
        return float(np.median([a.elapsed_time(b) for a, b in ev]))

    def plain_call(e):
        if e:
            e[0].record(stream)
        H.trace(g, rays0, H.HRPP_ANY_HIT, None, hits=out)
        if e:
            e[1].record(stream)
    plain_ms = call_ms(plain_call)
    _, pst = H.trace(g, rays0, H.HRPP_ANY_HIT, None, stats=True)
    tables = {}
    for log2e, ways in ((18, 2), (22, 4)):
        tab, snap = H.Table(log2e, ways, 6), H.Table(log2e, ways, 6)
        for f in frames[1:]:
            H.trace(g, f, H.HRPP_ANY_HIT, tab)
        snap.copy_from(tab)
        row = {}
        for sched, name in ((H.HRPP_SCHEDULE_BATCH, "batch"), (H.HRPP_SCHEDULE_COMPACT, "compact")):
            def hrpp_call(e, sched=sched):
                tab.copy_from(snap)
                if e:
                    e[0].record(stream)
                H.trace(g, rays0, H.HRPP_ANY_HIT, tab, hits=out, schedule=sched)
                if e:
                    e[1].record(stream)
            ms = call_ms(hrpp_call)
            row[name] = {"ms": ms, "mrays": n / ms / 1e3, "speedup_over_plain": plain_ms / ms}
        tab.copy_from(snap)
        if log2e == 22:
            # one restored two-pass call under an NVTX range (ncu --nvtx-include profile_shadow/)
            torch.cuda.nvtx.range_push("profile_shadow")
            H.trace(g, rays0, H.HRPP_ANY_HIT, tab, hits=out, schedule=H.HRPP_SCHEDULE_COMPACT)
            torch.cuda.synchronize()
            torch.cuda.nvtx.range_pop()
            tab.copy_from(snap)
        hh, st = H.trace(g, rays0, H.HRPP_ANY_HIT, tab, stats=True)
        ph, _ = H.trace(g, rays0, H.HRPP_ANY_HIT)
        torch.cuda.synchronize()
        row["occlusion_checked"] = bool(torch.equal(hh == -1, ph == -1))
        row["prediction_ratio"] = st["true_pos"] / st["rays"]
        row["false_pos"] = st["false_pos"] / st["rays"]
        row["skipped_exact_box_tests"] = 1.0 - st["box_tests"] / pst["box_tests"]
        tables[f"2^{log2e}x{ways}"] = row
    g.check()
    best = max((r[k]["mrays"], name, k) for name, r in tables.items() for k in ("batch", "compact"))
    line = {"metric": METRIC, "value": best[0], "unit": "Mrays/s", "n_gpus": 1, "steps": reps,
            "warmup": max(3, args.warmup), "ms_per_step": n / best[0] / 1e3, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": f"terrain (2,313,248 tris) shadow rays toward a low point light "
                                   f"{W.TERRAIN_SUN} from frame 0's primary hits ({n} rays, "
                                   f"{pst['hits'] / n:.0%} occluded); not one of the five configs",
                       "best": {"table": best[1], "schedule": best[2]},
                       "protocol": "each call restores a table warmed by 3 other jittered frames; events bracket "
                                   "the whole call (traversal + table update); median of the calls"},
            "plain": {"value": n / plain_ms / 1e3, "ms": plain_ms, "speedup_hrpp_over_plain": plain_ms * best[0] * 1e3 / n},
            "tables": tables, "occluded": pst["hits"] / n}
    if emit:
        print(json.dumps(line), flush=True)
    return line


def pathtrace_learned(H, g, s, frames, per_bounce, stream):
    """The learned treelet proposal on the path-tracing workload: one model
    per query mode, trained on every bounce of the first frame (labels from
    closest-hit traces of the same rays), evaluated per bounce on the last
    frame beside the hash table and plain traversal (added to per_bounce)."""
    import torch

    def timed(fn):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        out = fn()
        e1.record(stream)
        e1.synchronize()
        return e0.elapsed_time(e1), out

    models = {"closest": H.Proposal.for_workload(g, s, seed=1), "any": H.Proposal.for_workload(g, s, seed=2)}
    t_train, traces = 0.0, 0
    for c, sh in frames[0]:
        for name, rays in (("closest", c), ("any", sh)):
            hits, _ = H.trace(g, rays, H.HRPP_CLOSEST_HIT)
            lab = models[name].labels(hits)
            ms, _ = timed(lambda: models[name].train(rays, lab, lr=1e-3))
            t_train += ms * 1e-3
            traces += int(rays.shape[0])
    eval_frame = frames[-1]
    for b, (c, sh) in enumerate(eval_frame):
        if b >= len(per_bounce):
            break
        entry = {}
        for name, mode, rays in (("closest", H.HRPP_CLOSEST_HIT, c), ("any", H.HRPP_ANY_HIT, sh)):
            # warm every timed call once (the first prediction allocates the
            # network's inference buffers)
            H.trace(g, rays, mode)
            warm_nodes, _ = models[name].predict(rays)
            H.trace(g, rays, mode, predicted=warm_nodes)
            ms_plain, _ = timed(lambda: H.trace(g, rays, mode))
            ms_pred, (nodes, _) = timed(lambda: models[name].predict(rays))
            ms_trace, _ = timed(lambda: H.trace(g, rays, mode, predicted=nodes))
            _, st = H.trace(g, rays, mode, stats=True, predicted=nodes)
            _, sp = H.trace(g, rays, mode, stats=True)
            n = int(rays.shape[0])
            entry[name] = {"rays": n, "plain_mrays": n / ms_plain / 1e3, "learned_mrays": n / ms_trace / 1e3,
                           "learned_incl_inference_mrays": n / (ms_trace + ms_pred) / 1e3,
                           "prediction_ratio": st["true_pos"] / max(1, st["rays"]),
                           "box_tests_vs_plain": (st["box_tests"] + st["pred_box_tests"]) / max(1, sp["box_tests"])}
        per_bounce[b]["learned"] = entry
    for m in models.values():
        m.close()
    gemm_flops_per_row = 2.0 * (128 * 256 + 256 * 256 + 256 * 4096) * 3.0
    return {"train_traces": traces, "train_seconds": t_train,
            "train_tflops": traces * gemm_flops_per_row / t_train / 1e12 if t_train else None,
            "trained_on": "frame 0, all bounces", "evaluated_on": f"frame {len(frames) - 1}"}


def run_learned(args):
    """Config 4: the learned treelet proposal trained on traversal traces of
    the small scene's camera, compared with the hash table on held-out
    primary (closest-hit) and shadow (any-hit) rays of that scene."""
    rank, world, local = dist_env()
    import torch
    torch.cuda.set_device(local)
    import __graft_entry__
    __graft_entry__.build()
    from paper_1910_01304_gb300 import hrpp as H
    from paper_1910_01304_gb300.scenes import workloads as W
    s = W.small_scene()
    g = H.Scene.from_workload(s)
    stream = torch.cuda.current_stream()
    models = {"closest": H.Proposal.for_workload(g, s, seed=1), "any": H.Proposal.for_workload(g, s, seed=2)}
    tables = {"closest": H.Table(12, 1, 6), "any": H.Table(12, 1, 6)}

    def frame_rays(f):
        prim = torch.from_numpy(s.primary_rays(frame=f)).cuda()
        hits, _ = H.trace(g, prim, H.HRPP_CLOSEST_HIT, tables["closest"])
        hh = hits.cpu().numpy()
        sh, _ = W.secondary_shadow(s, s.primary_rays(frame=f), hh[:, 0], hh[:, 1].view(np.uint32))
        shadow = torch.from_numpy(sh).cuda()
        H.trace(g, shadow, H.HRPP_ANY_HIT, tables["any"])
        sh_hits, _ = H.trace(g, shadow, H.HRPP_CLOSEST_HIT)
        return {"closest": (prim, hits), "any": (shadow, sh_hits)}

    t_train = 0.0
    traces = 0
    losses = {"closest": [], "any": []}
    gemm_flops_per_row = 2.0 * (128 * 256 + 256 * 256 + 256 * 4096) * 3.0
    f = 0
    while traces < args.traces:
        f += 1
        fr = frame_rays(f)
        last = traces + sum(int(fr[m][0].shape[0]) for m in fr) >= args.traces
        for mode in ("closest", "any"):
            rays, hits = fr[mode]
            lab = models[mode].labels(hits)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            loss = models[mode].train(rays, lab, lr=1e-3, want_loss=(f % 50 == 0 or f == 1 or last))
            e1.record(stream)
            e1.synchronize()
            t_train += e0.elapsed_time(e1) * 1e-3
            traces += int(rays.shape[0])
            if loss is not None:
                losses[mode].append(loss)
    n_train_frames = f
    train_tflops = traces * gemm_flops_per_row / t_train / 1e12 if t_train else None
    # evaluation on held-out frames: plain, hash table (frozen), learned treelets
    res = {}
    for mode_name, mode in (("closest", H.HRPP_CLOSEST_HIT), ("any", H.HRPP_ANY_HIT)):
        tables[mode_name].configure(6, H.HRPP_UPDATE_FROZEN)
        acc = {"plain": [0.0, None], "hash": [0.0, None], "learned": [0.0, None], "learned_incl_inference": [0.0, None]}
        rays_total = 0
        stats = {}
        for f in range(100000, 100000 + 4):
            fr = frame_rays(f)
            rays = fr[mode_name][0]
            rays_total += int(rays.shape[0])
            # warm every timed call: the first launch of each kernel loads it, and
            # the first prediction allocates the inference buffers (the table is
            # frozen, so the warm-up leaves it as it is)
            for _ in range(2):
                H.trace(g, rays, mode)
                H.trace(g, rays, mode, tables[mode_name])
                warm_nodes, _ = models[mode_name].predict(rays)
                H.trace(g, rays, mode, predicted=warm_nodes)
            def timed(fn):
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                out = fn()
                e1.record(stream)
                e1.synchronize()
                return e0.elapsed_time(e1), out
            ms, _ = timed(lambda: H.trace(g, rays, mode))
            acc["plain"][0] += ms
            ms, _ = timed(lambda: H.trace(g, rays, mode, tables[mode_name]))
            acc["hash"][0] += ms
            ms_pred, (nodes, _) = timed(lambda: models[mode_name].predict(rays))
            ms, _ = timed(lambda: H.trace(g, rays, mode, predicted=nodes))
            acc["learned"][0] += ms
            acc["learned_incl_inference"][0] += ms + ms_pred
            for name, kw in (("plain", {}), ("hash", {"table": tables[mode_name]}), ("learned", {"predicted": nodes})):
                _, st = H.trace(g, rays, mode, stats=True, **kw)
                for k, v in st.items():
                    stats.setdefault(name, {}).setdefault(k, 0)
                    stats[name][k] += v
        res[mode_name] = {
            "rays": rays_total,
            "mrays": {k: rays_total / (v[0] * 1e-3) / 1e6 for k, v in acc.items()},
            "prediction_ratio": {k: stats[k]["true_pos"] / stats[k]["rays"] for k in ("hash", "learned")},
            "box_tests_vs_plain": {k: (stats[k]["box_tests"] + stats[k]["pred_box_tests"]) / stats["plain"]["box_tests"]
                                   for k in ("hash", "learned")},
        }
    peak = None
    pk = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(pk):
        with open(pk) as fh:
            peak = float(json.load(fh)["bf16_tflops_sustained"])
    line = {"metric": METRIC, "value": res["any"]["mrays"]["learned"], "unit": "Mrays/s", "n_gpus": 1,
            "steps": 4, "warmup": 2, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "bf16 (MLP, fp32 accumulate) / f32 (traversal)", "data": "synthetic",
            "config": {"workload": "learned treelet proposal on the small scene (1,792 tris, BVH2): "
                                   "96-256-256-4096 BF16 MLP, one model per query mode",
                       "traces": traces, "frames": n_train_frames},
            "train": {"seconds_in_train_calls": t_train, "traces": traces, "loss_first_last": {
                k: (v[0], v[-1]) if v else None for k, v in losses.items()},
                "gemm_tflops": train_tflops, "tensor_peak_sustained_tflops": peak,
                "frac": (train_tflops / peak) if (train_tflops and peak) else None},
            "roofline": {"bound": "tensor", "kernel": "MLP training: tcgen05 GEMMs and the fused softmax cross-entropy "
                                                      "(train calls, forward + backward + Adam)",
                         "achieved": train_tflops, "peak": peak, "unit": "TFLOP/s",
                         "frac": (train_tflops / peak) if (train_tflops and peak) else None,
                         "peak_kind": "measured sustained bf16 (MEASURED_PEAKS.json)" if peak else None,
                         "what": "GEMM work of the train calls (3x the forward's 2.3 MFLOP per trace) over their "
                                 "CUDA-event time; the K = 256 layers are epilogue- and HBM-bound"},
            "eval": res}
    print(json.dumps(line), flush=True)
    return 0


def main():
    args = parse()
    if args.impl == "reference":
        return run_reference(args)
    if args.workload == "batched":
        return run_batched(args)
    if args.workload == "pathtrace":
        run_pathtrace(args)
        return 0
    if args.workload == "learned":
        return run_learned(args)
    if args.workload == "small":
        run_small(args)
        return 0
    if args.workload == "shadow":
        run_shadow(args)
        return 0
    rank, world, local = dist_env()
    import torch
    if not torch.cuda.is_available():
        raise SystemExit("bench.py needs a CUDA device")
    torch.cuda.set_device(local)
    pg = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
        pg = dist
    import __graft_entry__
    __graft_entry__.build()
    from paper_1910_01304_gb300 import hrpp as H
    from paper_1910_01304_gb300.scenes import workloads as W

    w, h = map(int, args.res.split("x"))
    sw = W.terrain_scene(quads=args.quads, n_spheres=args.spheres, res=(w, h))
    g = H.Scene.from_workload(sw)
    frames = make_frames(args, rank, sw, H, g, torch)
    upd = H.HRPP_UPDATE_TWO_PHASE if args.update == "two_phase" else H.HRPP_UPDATE_ONLINE
    tab_c = H.Table(args.log2_entries, args.ways, args.precision, upd)
    tab_a = H.Table(args.log2_entries, args.ways, args.precision, upd)
    stream = torch.cuda.current_stream()
    rays_per_frame = [int(f["prim"].shape[0] + f["ao"].shape[0]) for f in frames]
    out_c = torch.empty((frames[0]["prim"].shape[0], 4), dtype=torch.float32, device="cuda")
    out_a = torch.empty((frames[0]["ao"].shape[0],), dtype=torch.int32, device="cuda")

    def barrier():
        torch.cuda.synchronize()
        if pg is not None:
            pg.barrier()

    verify = {"root": H.HRPP_VERIFY_ROOT, "bottom_up": H.HRPP_VERIFY_BOTTOM_UP, "none": H.HRPP_VERIFY_NONE}[args.verify]
    sched = H.HRPP_SCHEDULE_COMPACT if args.schedule == "compact" else H.HRPP_SCHEDULE_BATCH
    l2_kinds = {"none": H.HRPP_L2_NONE, "table": H.HRPP_L2_TABLE, "nodes": H.HRPP_L2_NODES}
    l2_kind = [l2_kinds[args.l2]]
    if args.l2 != "none":
        H.l2_set_aside(args.l2_set_aside_mb << 20)

    # Warm tables: the other frames (1 .. F-1) go through HRPP once; device
    # snapshots of the tables they leave are restored at the start of every
    # step, which then traces frame 0 with full two-phase updates.  Every step
    # is the same work, and no ray is ever predicted from its own insert.
    for f in frames[1:]:
        H.trace(g, f["prim"], H.HRPP_CLOSEST_HIT, tab_c, verify=verify)
        H.trace(g, f["ao"], H.HRPP_ANY_HIT, tab_a)
    snap_c = H.Table(args.log2_entries, args.ways, args.precision, upd)
    snap_a = H.Table(args.log2_entries, args.ways, args.precision, upd)
    snap_c.copy_from(tab_c)
    snap_a.copy_from(tab_a)
    # the same tables under the gate policy (GATE), warmed the same way
    gtab_c, gtab_a = make_tables(H, args.log2_entries, args.ways, args.precision, True, upd)
    for f in frames[1:]:
        H.trace(g, f["prim"], H.HRPP_CLOSEST_HIT, gtab_c, verify=verify)
        H.trace(g, f["ao"], H.HRPP_ANY_HIT, gtab_a)
    gsnap_c, gsnap_a = make_tables(H, args.log2_entries, args.ways, args.precision, True, upd)
    gsnap_c.copy_from(gtab_c)
    gsnap_a.copy_from(gtab_a)
    snapshot_of = {id(tab_c): snap_c, id(tab_a): snap_a, id(gtab_c): gsnap_c, id(gtab_a): gsnap_a}
    f0 = frames[0]

    def restore(tables):
        for t in tables:
            if t is not None:
                t.copy_from(snapshot_of[id(t)])

    side = torch.cuda.Stream()

    def run(steps, warm, tables, events=None, offset=0, concurrent=True):
        """steps x (restore the tables, trace the primary and AO batches).
        concurrent: the two batches (independent; one table each) are traced
        side by side, the AO batch on a second stream, so that each launch's
        tail overlaps the other; otherwise one after the other (with kernel
        events, for timing each launch alone)."""
        total = 0
        for k in range(steps):
            ev = events[k] if events is not None else (None, None)
            restore(tables)
            if concurrent:
                fork = torch.cuda.Event()
                fork.record(stream)
                side.wait_event(fork)
                H.trace(g, f0["ao"], H.HRPP_ANY_HIT, tables[1], hits=out_a, stream=side, l2_persist=l2_kind[0],
                        schedule=sched)
                H.trace(g, f0["prim"], H.HRPP_CLOSEST_HIT, tables[0], hits=out_c, verify=verify,
                        l2_persist=l2_kind[0], schedule=sched)
                join = torch.cuda.Event()
                join.record(side)
                stream.wait_event(join)
            else:
                H.trace(g, f0["prim"], H.HRPP_CLOSEST_HIT, tables[0], hits=out_c,
                        kernel_events=ev[0] if ev[0] else None, verify=verify, l2_persist=l2_kind[0], schedule=sched)
                H.trace(g, f0["ao"], H.HRPP_ANY_HIT, tables[1], hits=out_a, kernel_events=ev[1] if ev[1] else None,
                        l2_persist=l2_kind[0], schedule=sched)
            total += rays_per_frame[0]
        return total

    def mk():
        # torch only reports elapsed_time for events it recorded itself; the
        # library re-records these on the same stream around the kernel, so a
        # first record here just marks them as recorded
        e = torch.cuda.Event(enable_timing=True)
        e.record(stream)
        return e

    def timed(tables, with_kernel_events):
        """Warm-up, then args.steps timed steps.  With kernel events the two
        batches run one after the other and each launch is timed alone;
        without, they run side by side (the step as measured)."""
        conc = not with_kernel_events
        run(args.warmup, True, tables, offset=0, concurrent=conc)
        events = [((mk(), mk()), (mk(), mk())) for _ in range(args.steps)] if with_kernel_events else None
        barrier()
        e0, e1 = mk(), mk()
        e0.record(stream)
        rays = run(args.steps, False, tables, events=events, offset=args.warmup, concurrent=conc)
        e1.record(stream)
        barrier()
        ms = e0.elapsed_time(e1)
        kt = None
        if events is not None:
            kt = {"closest": sum(a[0].elapsed_time(a[1]) for a, _ in events) / args.steps,
                  "any": sum(b[0].elapsed_time(b[1]) for _, b in events) / args.steps}
        return rays, ms, kt

    def max_over_ranks(x):
        return reduce_max(x, pg, "cuda")

    def sum_over_ranks(x):
        return reduce_sum(x, pg, "cuda")

    # --- HRPP, timed, with clocks sampled over the timed region
    try:
        dev_id = "GPU-" + str(torch.cuda.get_device_properties(local).uuid)
    except Exception:
        dev_id = str(local)
    clocks = ClockSampler(dev_id)
    run(args.warmup, True, (tab_c, tab_a))
    barrier()
    clocks.mark(True)
    rays, ms, _ = timed((tab_c, tab_a), False)
    ms_max = max_over_ranks(ms)
    total_rays = sum_over_ranks(rays)
    value = job_mrays_per_s(total_rays, ms_max)
    # each launch timed alone (the batches one after the other): the
    # roofline's kernel durations, and the sequential step for reference
    s_rays, s_ms, kt = timed((tab_c, tab_a), True)
    seq_value = sum_over_ranks(s_rays) / (max_over_ranks(s_ms) * 1e-3) / 1e6

    # --- plain traversal on the same rays
    p_rays, p_ms, _ = timed((None, None), False)
    p_value = sum_over_ranks(p_rays) / (max_over_ranks(p_ms) * 1e-3) / 1e6
    ps_rays, ps_ms, p_kt = timed((None, None), True)
    p_seq_value = sum_over_ranks(ps_rays) / (max_over_ranks(ps_ms) * 1e-3) / 1e6

    # --- the gate policy: tables that stop predicting while it does not pay
    g_rays, g_ms, _ = timed((gtab_c, gtab_a), False)
    g_value = sum_over_ranks(g_rays) / (max_over_ranks(g_ms) * 1e-3) / 1e6

    # --- the same HRPP step with a persisting-L2 window over the table words
    # or over the interior nodes (a set-aside only for these runs)
    l2_variants = None
    if args.l2 == "none" and args.l2_variants:
        try:
            granted = H.l2_set_aside(args.l2_set_aside_mb << 20)
        except H.HrppError:
            granted = 0
        # every rank runs the variants (they hold collectives) or none does
        if max_over_ranks(0.0 if granted else 1.0) > 0.0:
            if granted:
                H.l2_set_aside(0)
            granted = 0
        if granted:
            l2_variants = {"set_aside_bytes": granted}
            for name in ("table", "nodes"):
                l2_kind[0] = l2_kinds[name]
                v_rays, v_ms, _ = timed((tab_c, tab_a), False)
                l2_variants[name] = {"value": sum_over_ranks(v_rays) / (max_over_ranks(v_ms) * 1e-3) / 1e6}
            l2_kind[0] = H.HRPP_L2_NONE
            H.l2_set_aside(0)

    # --- one restored step under an NVTX range: the launches an ncu capture of
    # this workload selects (--nvtx --nvtx-include profile_terrain/)
    torch.cuda.nvtx.range_push("profile_terrain")
    restore((tab_c, tab_a))
    H.trace(g, f0["prim"], H.HRPP_CLOSEST_HIT, tab_c, hits=out_c, verify=verify, schedule=sched)
    H.trace(g, f0["ao"], H.HRPP_ANY_HIT, tab_a, hits=out_a, schedule=sched)
    torch.cuda.synchronize()
    torch.cuda.nvtx.range_pop()

    # --- counters of one step (from the restored warm tables), with per-ray
    # outcomes of HRPP and per-ray box tests of plain traversal
    restore((tab_c, tab_a))
    per_ray = {}
    for name, key in (("closest", "prim"), ("any", "ao")):
        n = int(f0[key].shape[0])
        per_ray[name] = (torch.empty(n, dtype=torch.uint8, device="cuda"), torch.empty(n, dtype=torch.int32, device="cuda"))
    _, sc = H.trace(g, f0["prim"], H.HRPP_CLOSEST_HIT, tab_c, stats=True, verify=verify,
                    ray_outcome=per_ray["closest"][0])
    _, sa = H.trace(g, f0["ao"], H.HRPP_ANY_HIT, tab_a, stats=True, ray_outcome=per_ray["any"][0])
    occupancy = {name: table_occupancy(t.export(), args.ways) for name, t in (("closest", tab_c), ("any", tab_a))}
    _, pc = H.trace(g, f0["prim"], H.HRPP_CLOSEST_HIT, None, stats=True, ray_box_tests=per_ray["closest"][1])
    _, pa = H.trace(g, f0["ao"], H.HRPP_ANY_HIT, None, stats=True, ray_box_tests=per_ray["any"][1])

    # --- the paper's own semantics (closest-hit true positives unverified; not
    # exact): kernel time from the restored table and the share of rays whose
    # hit differs from plain traversal
    def kernel_ms(fn, reps=10):
        ev = [(mk(), mk()) for _ in range(reps)]
        for e in ev:
            fn(e)
        torch.cuda.synchronize()
        return float(np.median([a.elapsed_time(b) for a, b in ev]))

    out_plain = torch.empty_like(out_c)
    H.trace(g, f0["prim"], H.HRPP_CLOSEST_HIT, None, hits=out_plain)

    def paper_step(e, schedule=0):
        restore((tab_c, tab_a))
        H.trace(g, f0["prim"], H.HRPP_CLOSEST_HIT, tab_c, hits=out_c, kernel_events=e, verify=H.HRPP_VERIFY_NONE,
                schedule=schedule)

    paper_ms = kernel_ms(paper_step)
    paper_wrong = float((out_c.view(torch.int32) != out_plain.view(torch.int32)).any(dim=1).double().mean())
    paper_compact_ms = kernel_ms(lambda e: paper_step(e, H.HRPP_SCHEDULE_COMPACT))
    plain_ms = kernel_ms(lambda e: H.trace(g, f0["prim"], H.HRPP_CLOSEST_HIT, None, hits=out_plain, kernel_events=e))

    def any_ms(schedule):
        def fn(e):
            restore((tab_c, tab_a))
            H.trace(g, f0["ao"], H.HRPP_ANY_HIT, tab_a, hits=out_a, kernel_events=e, schedule=schedule)
        return kernel_ms(fn)
    compact = {"closest_exact_ms": kernel_ms(lambda e: (restore((tab_c, tab_a)), H.trace(
                   g, f0["prim"], H.HRPP_CLOSEST_HIT, tab_c, hits=out_c, kernel_events=e, verify=verify,
                   schedule=H.HRPP_SCHEDULE_COMPACT))),
               "closest_exact_batch_ms": kernel_ms(lambda e: (restore((tab_c, tab_a)), H.trace(
                   g, f0["prim"], H.HRPP_CLOSEST_HIT, tab_c, hits=out_c, kernel_events=e, verify=verify))),
               "any_ms": any_ms(H.HRPP_SCHEDULE_COMPACT), "any_batch_ms": any_ms(H.HRPP_SCHEDULE_BATCH),
               "how": "HRPP_SCHEDULE_COMPACT (lookups first, answered rays leave, the rest queued and traversed) "
                      "against the fused BATCH schedule, kernel time of each launch from the restored tables"}
    paper_semantics = {"closest_mrays": f0["prim"].shape[0] / paper_ms / 1e3,
                       "closest_mrays_compact": f0["prim"].shape[0] / paper_compact_ms / 1e3,
                       "plain_closest_mrays": f0["prim"].shape[0] / plain_ms / 1e3,
                       "speedup_over_plain": plain_ms / paper_ms,
                       "speedup_over_plain_compact": plain_ms / paper_compact_ms, "rays_with_another_hit": paper_wrong,
                       "note": "not exact: true positives return the predicted hit unverified (Sec. 4.3)"}

    def skipped_limit(name):
        # the paper's semantics (its true positives skip traversal): the share
        # of plain box tests that belong to rays HRPP predicted correctly
        oc, bx = per_ray[name]
        bx = bx.double()
        return float(bx[oc == H.HRPP_OUTCOME_TRUE_POS].sum() / bx.sum().clamp(min=1))
    g.check()

    # --- end to end from pinned host memory, every step's rays uploaded and
    # its hits downloaded inside the timed region
    e2e = None
    if not args.no_e2e:
        hp = torch.from_numpy(f0["prim_h"]).pin_memory()
        ha = torch.from_numpy(f0["ao_h"]).pin_memory()
        n_step = hp.shape[0] + ha.shape[0]
        h2d, d2h = hp.numel() * 4 + ha.numel() * 4, out_c.numel() * 4 + out_a.numel() * 4

        def timed_loop(step):
            for k in range(args.warmup):
                step(k)
            barrier()
            t0 = time.perf_counter()
            for k in range(args.steps):
                step(args.warmup + k)
            barrier()
            return max_over_ranks(time.perf_counter() - t0)

        # (1) the library's own host path: hrpp_trace on pinned host buffers
        # with host_async, from one host thread.  Each call stages its batch
        # in chunks (uploads and downloads on copy streams of its own,
        # overlapping the chunks' traces) and returns at once; the two
        # batches of a step run side by side on two streams, and the next
        # step's uploads overlap this step's traces.  Streams and host hit
        # buffers alternate between steps; a step restores its tables after
        # the previous step's traces.
        lib_streams = [(torch.cuda.Stream(), torch.cuda.Stream()) for _ in range(2)]
        lib_hits = [(torch.empty((hp.shape[0], 4), dtype=torch.float32).pin_memory(),
                     torch.empty((ha.shape[0],), dtype=torch.int32).pin_memory()) for _ in range(2)]
        lib_done = [None]
        lib_host_done = [None, None]

        def library_step(k):
            b = k % 2
            sc_, sa_ = lib_streams[b]
            if lib_done[0] is not None:
                for e in lib_done[0]:
                    stream.wait_event(e)
            restore((tab_c, tab_a))
            ready = torch.cuda.Event()
            ready.record(stream)
            sc_.wait_event(ready)
            sa_.wait_event(ready)
            # host_done: the library records these once the hits are in host
            # memory, so the streams wait only for the traces and the next
            # step's traces overlap this step's downloads
            hd = (torch.cuda.Event(), torch.cuda.Event())
            for e in hd:
                e.record(stream)  # creates the CUDA event; the library records it again
            H.trace(g, ha, H.HRPP_ANY_HIT, tab_a, hits=lib_hits[b][1], stream=sa_, host_async=True, host_done=hd[1])
            H.trace(g, hp, H.HRPP_CLOSEST_HIT, tab_c, hits=lib_hits[b][0], verify=verify, stream=sc_,
                    host_async=True, host_done=hd[0])
            done = (torch.cuda.Event(), torch.cuda.Event())
            done[0].record(sc_)
            done[1].record(sa_)
            lib_done[0] = done
            lib_host_done[b] = hd
        dt_lib = timed_loop(library_step)
        for hd in lib_host_done:
            for e in hd or ():
                e.synchronize()
        torch.cuda.synchronize()
        lb = (args.warmup + args.steps - 1) % 2
        lib_same = bool(torch.equal(lib_hits[lb][0].view(torch.int32), out_plain.cpu().view(torch.int32))
                        and torch.equal(lib_hits[lb][1] == -1, out_a.cpu() == -1))
        oc, oa = lib_hits[0]

        # (2) one host thread, one stream: the same calls one after the other
        def serial_step(k):
            restore((tab_c, tab_a))
            H.trace(g, hp, H.HRPP_CLOSEST_HIT, tab_c, hits=oc, verify=verify)
            H.trace(g, ha, H.HRPP_ANY_HIT, tab_a, hits=oa)
        dt_serial = timed_loop(serial_step)

        # (3) a frame loop orchestrated around device buffers, as a renderer
        # with its own copy engine would run it: hrpp_trace on double-buffered
        # device buffers, uploads on one copy stream and downloads on another,
        # so that copies overlap the traces across steps (the AO upload under
        # the primary trace, the next step's uploads under this step's AO
        # trace, the downloads under the next step)
        comp = torch.cuda.current_stream()
        up, down, comp2 = torch.cuda.Stream(), torch.cuda.Stream(), torch.cuda.Stream()
        dp = [torch.empty_like(f0["prim"]) for _ in range(2)]
        da = [torch.empty_like(f0["ao"]) for _ in range(2)]
        dhc = [torch.empty_like(out_c) for _ in range(2)]
        dha = [torch.empty_like(out_a) for _ in range(2)]
        hoc = [torch.empty(tuple(out_c.shape), dtype=torch.float32).pin_memory() for _ in range(2)]
        hoa = [torch.empty(tuple(out_a.shape), dtype=torch.int32).pin_memory() for _ in range(2)]
        consumed, downloaded = [None, None], [None, None]

        def event(stream):
            e = torch.cuda.Event()
            e.record(stream)
            return e

        def pipe_step(k):
            b = k % 2
            with torch.cuda.stream(up):
                if consumed[b] is not None:      # step k-2's traces are done with these buffers
                    for e in consumed[b]:
                        up.wait_event(e)
                dp[b].copy_(hp, non_blocking=True)
                up_p = event(up)
                da[b].copy_(ha, non_blocking=True)
                up_a = event(up)
            if downloaded[b] is not None:        # step k-2's hits have left these buffers
                comp.wait_event(downloaded[b])
                comp2.wait_event(downloaded[b])
            restore((tab_c, tab_a))
            restored = event(comp)
            # the two batches side by side, as in the device-resident step
            comp2.wait_event(restored)
            comp2.wait_event(up_a)
            H.trace(g, da[b], H.HRPP_ANY_HIT, tab_a, hits=dha[b], stream=comp2)
            done_a = event(comp2)
            comp.wait_event(up_p)
            H.trace(g, dp[b], H.HRPP_CLOSEST_HIT, tab_c, hits=dhc[b], verify=verify)
            done_c = event(comp)
            comp.wait_event(done_a)              # the next restore rewrites the AO table
            consumed[b] = (done_c, done_a)
            with torch.cuda.stream(down):
                down.wait_event(done_c)
                hoc[b].copy_(dhc[b], non_blocking=True)
                down.wait_event(done_a)
                hoa[b].copy_(dha[b], non_blocking=True)
                downloaded[b] = event(down)
        dt_pipe = timed_loop(pipe_step)
        last = (args.warmup + args.steps - 1) % 2
        # closest hits bit for bit against plain traversal; any-hit rays by
        # whether they are occluded (any valid hit may be reported)
        pipe_same = bool(torch.equal(hoc[last].view(torch.int32), out_plain.cpu().view(torch.int32))
                         and torch.equal(hoa[last] == -1, out_a.cpu() == -1))
        mrays = lambda dt: sum_over_ranks(n_step * args.steps) / dt / 1e6
        e2e = {"value": mrays(dt_lib), "unit": "Mrays/s", "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h,
               "how": "hrpp_trace on pinned host buffers with host_async and a host_done event per call (the "
                      "library stages each batch in chunks whose uploads and downloads run on copy streams of its "
                      "own and returns at once; the streams wait only for the traces); one host thread, the two "
                      "batches side by side on two streams, streams and hit buffers alternating between steps; "
                      "every step's rays uploaded and hits downloaded",
               "hits_checked": lib_same,
               "serial": {"value": mrays(dt_serial), "unit": "Mrays/s",
                          "how": "hrpp_trace on host buffers, synchronous (each call returns with its hits), one "
                                 "call after the other"},
               "torch_pipeline": {"value": mrays(dt_pipe), "unit": "Mrays/s", "hits_checked": pipe_same,
                                  "how": "hrpp_trace on double-buffered device buffers, the two batches side by "
                                         "side; pinned-host uploads and downloads on two copy streams, overlapping "
                                         "the traces across steps"}}

    # --- configs 1 and 5 beside the headline (one GPU only: a sub-result per
    # config, each with its own kernel-event roofline)
    configs = locality_demo = None
    if world == 1 and not args.no_configs:
        configs = {}
        import copy
        a = copy.copy(args)
        a.steps, a.warmup, a.frames = max(5, min(args.steps, 20)), max(3, args.warmup), 4
        configs["small"] = summarize_config(run_small(a, emit=False))
        a = copy.copy(args)
        a.steps, a.warmup, a.frames, a.no_learned = max(3, min(args.steps, 5)), 3, 2, True
        a.log2_entries, a.ways, a.precision = 18, 2, 6
        configs["pathtrace"] = summarize_config(run_pathtrace(a, emit=False))
        a = copy.copy(args)
        a.steps, a.warmup = 11, 3
        demo = run_shadow(a, emit=False)
        locality_demo = {k: demo[k] for k in ("value", "unit", "config", "plain", "tables", "occluded")}

    # the clock record covers every timed GPU loop above (HRPP, plain, gated,
    # the end-to-end loops, the config sub-results)
    clocks.mark(False)
    clk = clocks.stop()

    if rank != 0:
        return 0
    # --- roofline of the dominant kernel
    peak, peak_kind = load_peaks()
    info = g.info()
    width = info["width"]
    dom = "any" if kt["any"] >= kt["closest"] else "closest"
    st_dom = sa if dom == "any" else sc
    bytes_launch = algorithmic_bytes(st_dom, dom == "closest", width, args.ways)
    kname = f"k_trace<{width}, {'closest' if dom == 'closest' else 'any'}, hrpp>"
    key = f"bvh{width}_{dom}"
    if args.schedule == "compact":  # both launches of the two-pass schedule; no record of its own
        kname, key = f"k_predict + k_trace_queue<{width}, {dom}> (two-pass)", f"compact_bvh{width}_{dom}"
    n_sm = torch.cuda.get_device_properties(local).multi_processor_count
    roof = roofline_block(key, kname, kt[dom], bytes_launch, st_dom, peak, peak_kind, clk.get("sm_mhz"), n_sm)

    def skipped(h, p, limit):
        return {"prediction_ratio": h["true_pos"] / max(1, h["rays"]),
                "skipped_exact_box_tests": 1.0 - h["box_tests"] / max(1, p["box_tests"]),
                "skipped_limit_box_tests": limit,
                "skipped_exact_interior_nodes": 1.0 - h["interior_nodes"] / max(1, p["interior_nodes"]),
                "positives": h["positives"], "true_pos": h["true_pos"], "false_pos": h["false_pos"],
                "tp_inexact": h["tp_inexact"], "rays": h["rays"]}

    cpu = None if args.no_cpu else cpu_baseline(args, sw, frames)
    launches_per_step = 2 + (2 if args.update == "two_phase" else 0)  # per batch: trace + k_apply
    line = {
        "metric": METRIC, "value": value, "unit": "Mrays/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_max / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": WORKLOAD, "tris": int(sw.n_tris), "bvh_width": width,
                   "rays_per_step": float(rays_per_frame[0]), "frames": args.frames,
                   "protocol": f"each step: restore the tables warmed by {args.frames - 1} other jittered frames, "
                               "then trace frame 0's closest-hit primaries and its AO rays (independent batches, one "
                               "table each) side by side on two streams, two-phase updates included",
                   "table": {"log2_entries": args.log2_entries, "ways": args.ways, "precision": args.precision,
                             "update": args.update, "verify": args.verify, "l2_window": args.l2},
                   "schedule": args.schedule,
                   "exact": args.verify != "none",
                   "l2": f"inputs larger than L2: {rays_per_frame[0] * 32 / 1e6:.0f} MB of rays per step; "
                         "scene resident"},
        "plain": {"value": p_value, "unit": "Mrays/s", "speedup_hrpp_over_plain": value / p_value,
                  "kernel_ms": p_kt},
        "sequential": {"value": seq_value, "plain_value": p_seq_value, "unit": "Mrays/s",
                       "how": "the same steps with the two batches one after the other (kernel times taken here)"},
        "per_mode_kernel_ms": kt,
        "l2_persist": l2_variants,
        "table_occupancy": occupancy,
        "gated": {"value": g_value, "unit": "Mrays/s", "speedup_over_plain": g_value / p_value,
                  "gate": {"min_tp_per_65536": GATE, "sample_log2": GATE_SAMPLE_LOG2},
                  "how": "the same step with each table's gate set: a table stops consulting (except every 32nd "
                         "32-ray chunk) after a call whose true positives fall below the threshold"},
        "compact_schedule": compact,
        "paper_semantics": paper_semantics,
        "skipped": {"closest": skipped(sc, pc, skipped_limit("closest")),
                    "any": skipped(sa, pa, skipped_limit("any")),
                    "limit_study": limit_study(),
                    "paper_context": "paper Table 1 (PBRT limit study, no hardware stated): 30-69% hit-all, "
                                     "<1-48% hit-any savings"},
        "configs": configs,
        "locality_demo": locality_demo,
        "roofline": roof,
        "cpu_baseline": cpu,
        "e2e": e2e,
        "gpu_launches": launches_per_step * args.steps,
        "clocks": clk,
    }
    print(json.dumps(line), flush=True)
    return 0


if __name__ == "__main__":
    sys.exit(main())
