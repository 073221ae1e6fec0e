"""The paper's limit study (Sec. 6, Table 1) on this project's synthetic
scenes, computed by the oracle alone; writes tests/golden/limit_study.json.

Sec. 6 measures HRPP in software with an unbounded predictor table that has
no replacement and inserts each ray's leaf before the next ray is traced
(Sec. 4.3, Sec. 6), over 8 samples per pixel, with one predictor for
hit-all (closest-hit) and one for hit-any rays (Sec. 6.1), Go Up Level 0 and
hash precision 6 (Table 1 caption), and reports the share of traversal work
skipped.  The same is done here: each workload is traced as 8 jittered frames
(the analogue of 8 spp) through the oracle's unbounded, sequential table,
with true positives skipping their traversal (the paper's semantics: a
closest-hit true positive returns its predicted hit unverified).  For each
query type and precision it records

  prediction_ratio         true positives / rays
  skipped_limit_box_tests  plain box tests of the true-positive rays / all
                           plain box tests (the interior work they skip)
  table_mb                 8 bytes per key + 4 bytes per stored leaf, the
                           size of the unbounded map (Table 1's MB rows)

beside the bounded table's figures, which the GPU reports in bench.py.
Config 1 (small scene, shadow rays as hit-any) and config 2 (terrain, AO
rays as hit-any) at precision 6 and 5 (Sec. 5.1 finds the Buddha scene's
skipped work peaks at 5 bits); and, beside them, the terrain's shadow rays
toward a low point light (TERRAIN_SUN) as a hit-any workload with the
simple lighting in which the paper finds hit-any locality (Sec. 6.1).

Run: python tests/golden/make_limit_study.py [--only small]  (config 2 takes
a few minutes on one core per entry; entries run in parallel processes).
"""
from __future__ import annotations

import argparse
import json
import os
import sys
from concurrent.futures import ProcessPoolExecutor

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

OUT = os.path.join(HERE, "limit_study.json")
FRAMES = 8


def _scene(name):
    from paper_1910_01304_gb300.scenes import workloads as W
    return W.small_scene() if name == "small" else W.terrain_scene()


def _secondary(s, name, prim, h, f, W):
    if name == "small":
        return W.secondary_shadow(s, prim, h["t"], h["prim"])[0]
    if name == "terrain_shadow":  # shadow rays toward the low sun instead of AO rays
        return W.secondary_shadow(s, prim, h["t"], h["prim"], light=W.TERRAIN_SUN)[0]
    return W.secondary_ao(s, prim, h["t"], h["prim"], frame=f)[0]


def _frames(s, name, O):
    """Per jittered frame: primary rays and the secondary (hit-any) rays made
    from the oracle's plain primary hits."""
    from paper_1910_01304_gb300.scenes import workloads as W
    for f in range(FRAMES):
        prim = s.primary_rays(frame=f)
        h, _ = O.trace(s.tris, s.nodes, s.prim_index, s.root, prim, O.CLOSEST_HIT)
        yield prim, _secondary(s, name, prim, h, f, W)


def entry(name: str, query: str, precision: int) -> dict:
    """One (workload, query type, precision) cell of the study."""
    import oracle as O
    s = _scene(name)
    mode = O.CLOSEST_HIT if query == "hit_all" else O.ANY_HIT
    tab = O.Table(0, 1, precision, O.UNBOUNDED)
    rays_total = tp = 0
    box_all = box_tp = 0
    for prim, sec in _frames(s, name, O):
        rays = prim if mode == O.CLOSEST_HIT else sec
        _, _, _, plain_boxes = O.trace(s.tris, s.nodes, s.prim_index, s.root, rays, mode, per_ray=True)
        _, st, oc, _ = O.trace(s.tris, s.nodes, s.prim_index, s.root, rays, mode, tab, per_ray=True,
                               verify=O.VERIFY_NONE)
        is_tp = oc == 3
        rays_total += len(rays)
        tp += int(is_tp.sum())
        box_all += int(plain_boxes.astype(np.uint64).sum())
        box_tp += int(plain_boxes[is_tp].astype(np.uint64).sum())
    keys, leaves = tab.unbounded_size()
    return {"workload": name, "query": query, "precision": precision, "frames": FRAMES, "rays": rays_total,
            "true_pos": tp, "prediction_ratio": tp / max(1, rays_total),
            "skipped_limit_box_tests": box_tp / max(1, box_all), "keys": int(keys), "stored_leaves": int(leaves),
            "table_mb": (8 * keys + 4 * leaves) / 1e6}


def cells(only=None):
    names = ["small", "terrain", "terrain_shadow"] if only is None else [only]
    return [(n, q, p) for n in names for q in ("hit_all", "hit_any") for p in (6, 5)
            if not (n == "terrain_shadow" and q == "hit_all")]  # its hit-all rays are terrain's


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--only", choices=["small", "terrain", "terrain_shadow"])
    ap.add_argument("--jobs", type=int, default=min(8, os.cpu_count() or 1))
    args = ap.parse_args()
    todo = cells(args.only)
    with ProcessPoolExecutor(max_workers=args.jobs) as ex:
        res = list(ex.map(entry, *zip(*todo)))
    old = {}
    if os.path.exists(OUT):
        with open(OUT) as fh:
            old = {(e["workload"], e["query"], e["precision"]): e for e in json.load(fh)["entries"]}
    for e in res:
        old[(e["workload"], e["query"], e["precision"])] = e
    doc = {"what": "the paper's limit study (Sec. 6, Table 1: unbounded sequential table, true positives skip "
                   "traversal, 8 jittered frames as 8 spp, Go Up Level 0) on the synthetic configs 1 and 2, "
                   "computed by the oracle; written by tests/golden/make_limit_study.py",
           "entries": sorted(old.values(), key=lambda e: (e["workload"], e["query"], -e["precision"]))}
    with open(OUT, "w") as fh:
        json.dump(doc, fh, indent=1)
    for e in res:
        print(e["workload"], e["query"], e["precision"], f"ratio {e['prediction_ratio']:.3f}",
              f"skipped {e['skipped_limit_box_tests']:.3f}", f"{e['table_mb']:.1f} MB")


if __name__ == "__main__":
    main()
