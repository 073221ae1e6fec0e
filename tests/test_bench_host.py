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
