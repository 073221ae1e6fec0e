"""Host legs of the benchmark: the oracle run ray-parallel across host
threads (the CPU baseline and the reference arm) gives exactly the
single-thread results, and the reference arm prints its JSON line."""
import json
import os
import subprocess
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_threaded_oracle_matches_one_thread():
    import bench
    import oracle as O
    from paper_1910_01304_gb300.scenes import workloads as W
    s = W.small_scene(width=4, res=64)
    rays = s.primary_rays(frame=1)
    want, _ = O.trace(s.tris, s.nodes, s.prim_index, s.root, rays, O.CLOSEST_HIT)
    for k in (1, 3, 8):
        plain = bench.OracleThreads(O, s, k)
        res, dt = plain.trace(plain.split(rays), O.CLOSEST_HIT)
        got = plain.gather(res, len(rays), O.HIT_DTYPE)
        plain.close()
        assert dt >= 0 and np.array_equal(got.view(np.uint8), want.view(np.uint8))
        # HRPP with one table pair per thread: the hits stay exact, frame after frame
        ot = bench.OracleThreads(O, s, k, (10, 2, 6, O.TWO_PHASE))
        for _ in range(2):
            res, _ = ot.trace(ot.split(rays), O.CLOSEST_HIT)
            got = ot.gather(res, len(rays), O.HIT_DTYPE)
            assert np.array_equal(got.view(np.uint8), want.view(np.uint8))
        ot.close()


def test_reference_arm_prints_its_line():
    out = subprocess.run([sys.executable, "bench.py", "--impl", "reference", "--steps", "2", "--warmup", "1",
                          "--quads", "48", "--spheres", "4", "--res", "160x90"],
                         cwd=ROOT, capture_output=True, text=True, timeout=600)
    assert out.returncode == 0, out.stderr[-2000:]
    line = json.loads(out.stdout.strip().splitlines()[-1])
    assert line["impl"] == "reference" and line["value"] > 0 and line["unit"] == "Mrays/s"
    assert line["cpu_baseline"]["kind"] == "oracle" and line["cpu_baseline"]["cores"] == bench_threads()
    assert line["e2e"]["h2d_bytes_per_step"] == 0 and line["e2e"]["value"] == line["value"]


def bench_threads():
    import bench
    return bench.host_threads()


def test_algorithmic_bytes_per_ray_formula():
    """32 B per ray + 16 (closest) or 4 (any) B of result + 8 B per way per
    lookup + one node per interior visit (predicted subtrees included) + 48 B
    per triangle test (predicted leaves included) + 16 B per insert."""
    import bench
    st = {"rays": 10, "lookups": 7, "interior_nodes": 100, "pred_interior_nodes": 5, "tri_tests": 40,
          "pred_tri_tests": 3, "inserts": 2}
    assert bench.algorithmic_bytes(st, True, 4, 2) == 10 * 48 + 7 * 16 + 105 * 128 + 43 * 48 + 2 * 16
    assert bench.algorithmic_bytes(st, False, 2, 1) == 10 * 36 + 7 * 8 + 105 * 64 + 43 * 48 + 2 * 16


def test_table_occupancy_counts_valid_words_per_set():
    import bench
    empty = np.uint64(0xFFFFFFFFFFFFFFFF)
    words = np.full(8, empty, np.uint64)          # 4 sets of 2 ways
    words[0] = words[1] = 5                        # set 0: 2 nodes
    words[4] = 9                                   # set 2: 1 node
    occ = bench.table_occupancy(words, 2)
    assert occ["valid_words"] == 3 and occ["words"] == 8 and occ["fill"] == 3 / 8
    assert occ["nodes_per_used_set"] == 1.5


def test_traffic_record_lists_both_launches():
    """profiles/traffic.txt holds DRAM bytes, warp instructions and the L2
    share per launch for the terrain, small-scene and path-tracing launches
    the bench's rooflines name, each with the kernel source hash it was
    taken on; a record on the current source is what the bench reads."""
    import re
    import bench
    path = os.path.join(ROOT, "profiles", "traffic.txt")
    rows = [line.split() for line in open(path) if line.strip() and not line.startswith("#")]
    keys = {(r[0], r[1]) for r in rows}
    for what in ("traffic", "inst", "l2pct"):
        for kernel in ("bvh4_any", "bvh4_closest", "small_bvh2_any", "small_bvh2_closest", "pt_bvh4_closest_b1"):
            assert (what, kernel) in keys
    for r in rows:
        assert float(r[2]) > 0 and re.fullmatch(r"[0-9a-f]{16}", r[3])
        if r[0] in ("traffic", "inst"):
            assert float(r[2]) == int(r[2])
        else:
            assert 0 < float(r[2]) <= 100
    value, src = bench.recorded_traffic("bvh4_any")
    if src == bench.kernel_source_hash():
        assert value is not None and value > 0


def test_frames_differ_across_ranks():
    import bench
    seen = {bench.frame_index(f, rank) for rank in range(8) for f in range(4)}
    assert len(seen) == 32
