"""The stored limit study (tests/golden/limit_study.json, the paper's Sec. 6
setting on configs 1 and 2) against a fresh oracle run of the small-scene
cells, and against what the paper's setting fixes: an unbounded table whose
true positives skip their traversal."""
import json
import os

import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
PATH = os.path.join(HERE, "golden", "limit_study.json")


def _stored():
    with open(PATH) as fh:
        return {(e["workload"], e["query"], e["precision"]): e for e in json.load(fh)["entries"]}


@pytest.mark.parametrize("query,precision", [("hit_any", 6), ("hit_all", 5)])
def test_small_scene_cells_reproduce(query, precision):
    import sys
    sys.path.insert(0, os.path.join(HERE, "golden"))
    from make_limit_study import entry
    fresh = entry("small", query, precision)
    assert _stored()[("small", query, precision)] == fresh


def test_limit_study_is_consistent_with_the_paper_setting():
    """Every cell covers all 8 frames' rays; hit-all predicts better than
    hit-any (Sec. 6.1 finds hit-all rays far more predictable); a true
    positive skips at most all of its plain box tests, so the skipped share
    is a share; and the coarser hash (p = 5) stores no more keys than p = 6
    on the same rays (Sec. 5.1: fewer bits, fewer distinct keys)."""
    st = _stored()
    for name in ("small", "terrain"):
        for q in ("hit_all", "hit_any"):
            for p in (6, 5):
                e = st[(name, q, p)]
                assert e["frames"] == 8 and e["rays"] > 0
                assert 0.0 <= e["skipped_limit_box_tests"] <= 1.0
                assert 0.0 <= e["prediction_ratio"] <= 1.0
            assert st[(name, q, 5)]["keys"] <= st[(name, q, 6)]["keys"]
        assert st[(name, "hit_all", 6)]["prediction_ratio"] > st[(name, "hit_any", 6)]["prediction_ratio"]
    # the terrain's shadow rays toward the low sun: hit-any rays with the
    # simple lighting of Sec. 6.1, far more predictable than its AO rays
    for p in (6, 5):
        e = st[("terrain_shadow", "hit_any", p)]
        assert e["frames"] == 8 and 0.0 <= e["skipped_limit_box_tests"] <= 1.0
        assert e["prediction_ratio"] > st[("terrain", "hit_any", p)]["prediction_ratio"]
    assert st[("terrain_shadow", "hit_any", 5)]["keys"] <= st[("terrain_shadow", "hit_any", 6)]["keys"]
