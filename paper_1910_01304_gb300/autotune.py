"""Autotuner for HRPP launch and predictor-table parameters.

Nothing it picks can change a result: every candidate traces the same rays
and the tuner checks that all of them return the same results.  Closest-hit
hits are compared bit for bit; any-hit results by their occlusion bit, the only
part of them that is defined (a ray answered by a predicted node may report
another occluder than plain traversal finds first).  It times, with CUDA
events on the current stream:
  1. the traversal launch shape (threads per block, ray schedule) on plain
     traversal;
  2. predictor tables over a grid of sizes, associativities, hash precisions
     (Sec. 5.1's tight-vs-loose trade-off; p = 1..7), the exponent bits the
     hash keeps (most or least significant) and Go Up Levels (Sec. 6.2): each
     table is warmed on one ray set (a previous frame) and then frozen while
     a second ray set is timed, so the timing sees realistic prediction rates
     and no self-prediction.
It returns the fastest table (or none, when no table beats plain traversal)
with the timings it measured.

tune_batch does the same for a batched workload (one graph-replayed launch
over many scenes): block size on plain traversal, then a table
configuration for the closest-hit items and one for the any-hit items,
each timed from tables warmed by other frames and restored before every
replay.
"""
from __future__ import annotations

import hashlib
import itertools
import json

import numpy as np

from . import hrpp as H

LAUNCH_GRID = [dict(block_threads=b, schedule=s) for b in (64, 128, 256)
               for s in (H.HRPP_SCHEDULE_BATCH, H.HRPP_SCHEDULE_REFILL)]
TABLE_GRID = dict(log2_entries=(14, 16, 18, 20), ways=(1, 2, 4), precision=(1, 2, 3, 4, 5, 6, 7), go_up=(0, 1),
                  hash=(H.HRPP_HASH_EXP_MSB, H.HRPP_HASH_EXP_LSB))


def _time(fn, reps: int) -> float:
    import torch
    fn()
    ts = []
    for _ in range(reps):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        fn()
        e1.record()
        e1.synchronize()
        ts.append(e0.elapsed_time(e1))
    return float(np.median(ts))


def _digest(t, mode: int) -> str:
    """Closest-hit results bit for bit; any-hit results as the occlusion bit
    (a ray answered by a predicted node may report another occluder)."""
    a = t.cpu().numpy()
    if mode != H.HRPP_CLOSEST_HIT:
        a = a.view(np.uint32) != H.HRPP_NO_HIT
    return hashlib.sha1(a.tobytes()).hexdigest()


def tune(scene: H.Scene, rays_warm, rays_eval, mode: int, table_grid: dict | None = None, reps: int = 5,
         launch_grid: list | None = None) -> dict:
    """Tunes one (scene, mode) workload.  rays_*: [n, 8] device tensors."""
    import torch
    grid = TABLE_GRID if table_grid is None else table_grid
    launches = LAUNCH_GRID if launch_grid is None else launch_grid
    n = int(rays_eval.shape[0])
    shape = (n, 4) if mode == H.HRPP_CLOSEST_HIT else (n,)
    dtype = torch.float32 if mode == H.HRPP_CLOSEST_HIT else torch.int32
    out = torch.empty(shape, dtype=dtype, device=rays_eval.device)
    reference = None
    launch_times = []
    for cfg in launches:
        ms = _time(lambda: H.trace(scene, rays_eval, mode, None, hits=out, **cfg), reps)
        d = _digest(out, mode)
        reference = reference or d
        if d != reference:
            raise AssertionError(f"launch shape {cfg} changed the result")
        launch_times.append((ms, cfg))
    plain_ms, launch = min(launch_times, key=lambda x: x[0])
    best = dict(table=None, ms=plain_ms)
    table_times = []
    keys = list(grid)
    for values in itertools.product(*(grid[k] for k in keys)):
        tc = dict(zip(keys, values))
        t = H.Table(tc["log2_entries"], tc["ways"], tc["precision"], H.HRPP_UPDATE_TWO_PHASE, go_up=tc.get("go_up", 0),
                    hash_variant=tc.get("hash", H.HRPP_HASH_EXP_MSB))
        H.trace(scene, rays_warm, mode, t, **launch)
        t.configure(tc["precision"], H.HRPP_UPDATE_FROZEN)
        ms = _time(lambda: H.trace(scene, rays_eval, mode, t, hits=out, **launch), reps)
        if _digest(out, mode) != reference:
            raise AssertionError(f"table {tc} changed the result")
        table_times.append(dict(tc, ms=ms))
        if ms < best["ms"]:
            best = dict(table=tc, ms=ms)
        t.close()
    return dict(mode="closest" if mode == H.HRPP_CLOSEST_HIT else "any", rays=n, launch=launch, plain_ms=plain_ms,
                best_table=best["table"], best_ms=best["ms"], speedup_over_plain=plain_ms / best["ms"],
                launch_times=[dict(c, ms=m) for m, c in launch_times], table_times=table_times)


BATCH_TABLE_GRID = [None] + [dict(log2_entries=e, ways=w, precision=p, hash=h) for e in (14, 16) for w in (1, 2)
                              for p in (5, 6) for h in (H.HRPP_HASH_EXP_MSB, H.HRPP_HASH_EXP_LSB)]
BATCH_BLOCK_GRID = (128, 256)


class BatchSetup:
    """One candidate configuration of a batched workload: a table per item
    (or none), one graph-replayed Batch per frame, and device snapshots of the
    tables after frames 1.. have warmed them.  step() restores the snapshots
    and replays frame 0, so every step is the same work."""

    def __init__(self, items, frames, cfg_closest, cfg_any, block_threads: int, stats: bool = False):
        self.tables, self.snaps = [], []
        for scene, mode in items:
            cfg = cfg_closest if mode == H.HRPP_CLOSEST_HIT else cfg_any
            if cfg is None:
                self.tables.append(None)
                continue
            self.tables.append(H.Table(cfg["log2_entries"], cfg["ways"], cfg["precision"],
                                       hash_variant=cfg.get("hash", H.HRPP_HASH_EXP_MSB)))
        self.batches = [H.Batch([(sc, t, rays, mode) for (sc, mode), t, rays in zip(items, self.tables, fr)],
                                stats=stats and k == 0, block_threads=block_threads)
                        for k, fr in enumerate(frames)]
        for b in self.batches[1:]:
            b.run()
        for t in self.tables:
            if t is None:
                self.snaps.append(None)
                continue
            snap = H.Table(t.log2_entries, t.ways, t.precision, hash_variant=t.hash_variant)
            snap.copy_from(t)
            self.snaps.append(snap)

    def step(self, stream=None):
        for t, snap in zip(self.tables, self.snaps):
            if t is not None:
                t.copy_from(snap, stream)
        self.batches[0].run(stream)

    def hits(self):
        return self.batches[0].hits

    def close(self):
        for b in self.batches:
            b.close()
        for t in self.tables + self.snaps:
            if t is not None:
                t.close()


def _batch_digest(items, hits) -> str:
    """Closest-hit results bit for bit; any-hit results as the occlusion
    bit (the prim an any-hit ray reports may differ when a predicted leaf
    answers it)."""
    h = hashlib.sha1()
    for (_, mode), out in zip(items, hits):
        a = out.cpu().numpy()
        h.update(a.tobytes() if mode == H.HRPP_CLOSEST_HIT else (a.view(np.uint32) != H.HRPP_NO_HIT).tobytes())
    return h.hexdigest()


def tune_batch(items, frames, table_grid=None, block_grid=None, reps: int = 3) -> dict:
    """Tunes a batched workload.  items: [(Scene, mode)]; frames: per frame, a
    list of ray tensors, one per item (frame 0 is the one timed, the others
    warm the tables).  Picks the block size on plain traversal, then the
    table configuration (or none) of the closest-hit items and of the any-hit
    items in turn.  Every candidate must return the same results."""
    grid = BATCH_TABLE_GRID if table_grid is None else table_grid
    blocks = BATCH_BLOCK_GRID if block_grid is None else block_grid
    reference = None

    def measure(cfg_c, cfg_a, block):
        nonlocal reference
        setup = BatchSetup(items, frames, cfg_c, cfg_a, block)
        ms = _time(setup.step, reps)
        d = _batch_digest(items, setup.hits())
        setup.close()
        reference = reference or d
        if d != reference:
            raise AssertionError(f"configuration {cfg_c}, {cfg_a}, {block} changed the results")
        return ms

    tried = []
    block_ms = [(measure(None, None, b), b) for b in blocks]
    best_ms, block = min(block_ms)
    tried += [dict(closest=None, any=None, block_threads=b, ms=m) for m, b in block_ms]
    plain_ms = best_ms
    choice = {"closest": None, "any": None}
    for mode in ("closest", "any"):
        for cfg in grid:
            if cfg is None:
                continue
            trial = dict(choice, **{mode: cfg})
            ms = measure(trial["closest"], trial["any"], block)
            tried.append(dict(trial, block_threads=block, ms=ms))
            if ms < best_ms:
                best_ms, choice = ms, trial
    return dict(closest=choice["closest"], any=choice["any"], block_threads=block, ms=best_ms, plain_ms=plain_ms,
                tried=tried)


def main():
    import argparse

    import torch

    from .scenes import workloads as W
    ap = argparse.ArgumentParser(description="tune HRPP launch and table parameters on a workload")
    ap.add_argument("--workload", default="terrain", choices=["terrain", "small"])
    ap.add_argument("--quick", action="store_true", help="a reduced table grid")
    args = ap.parse_args()
    if args.workload == "terrain":
        s = W.terrain_scene()
    else:
        s = W.small_scene()
    g = H.Scene.from_workload(s)
    grid = dict(log2_entries=(16, 18), ways=(1, 2), precision=(5, 6), go_up=(0,)) if args.quick else None
    results = []
    prims = [torch.from_numpy(s.primary_rays(frame=f)).cuda() for f in (1, 2)]
    results.append(tune(g, prims[0], prims[1], H.HRPP_CLOSEST_HIT, grid))
    secondary = []
    for f, pr in zip((1, 2), prims):
        hits, _ = H.trace(g, pr, H.HRPP_CLOSEST_HIT)
        h = hits.cpu().numpy()
        rays_np = pr.cpu().numpy()
        if args.workload == "terrain":
            sec, _ = W.secondary_ao(s, rays_np, h[:, 0], h[:, 1].view(np.uint32), frame=f)
        else:
            sec, _ = W.secondary_shadow(s, rays_np, h[:, 0], h[:, 1].view(np.uint32))
        secondary.append(torch.from_numpy(sec).cuda())
    results.append(tune(g, secondary[0], secondary[1], H.HRPP_ANY_HIT, grid))
    for r in results:
        r.pop("table_times")
        print(json.dumps(r))


if __name__ == "__main__":
    main()
