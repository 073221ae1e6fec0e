"""Pins for the oracle's HRPP simulation (Sec. 4.2-4.3, Sec. 5).

Pinned against the plain result (HRPP must return exactly what plain traversal
returns), against brute force restricted to the predicted leaf, and against
invariants the method fixes: an empty table predicts nothing; in the
unbounded limit-study table every ray that hit is, on a second pass, a
positive whose own leaf is predicted; any-hit true positives do no interior
work while every other ray does exactly its plain traversal.
"""
import numpy as np
import pytest

import oracle as O
from paper_1910_01304_gb300.scenes import workloads as W


def _leaf_of_prim(nodes, prim_index):
    m = {}
    for n in nodes:
        if n["count"] > 0:
            lid = (int(n["first"]) << 2) | (int(n["count"]) - 1)
            for j in range(int(n["count"])):
                m[int(prim_index[n["first"] + j])] = lid
    return m


def _check_identities(st, n):
    assert st["rays"] == n and st["lookups"] == n
    assert st["positives"] + st["negatives"] == n
    assert st["true_pos"] + st["false_pos"] == st["positives"]
    assert st["dup_inserts"] <= st["inserts"]


@pytest.mark.parametrize("mode", [O.CLOSEST_HIT, O.ANY_HIT])
def test_empty_table_is_plain_plus_one_lookup(small, mode):
    rays = small.primary_rays()[::3]
    hp, sp = O.trace(small.tris, small.nodes, small.prim_index, 0, rays, mode)
    tab = O.Table(16, 1, 6, O.TWO_PHASE)
    hh, sh = O.trace(small.tris, small.nodes, small.prim_index, 0, rays, mode, tab)
    assert np.array_equal(hp, hh)
    for k in ("interior_nodes", "box_tests", "leaves", "tri_tests", "hits"):
        assert sp[k] == sh[k]
    assert sh["negatives"] == len(rays) and sh["positives"] == 0
    assert sh["inserts"] == sp["hits"]
    _check_identities(sh, len(rays))


@pytest.mark.parametrize("mode", [O.CLOSEST_HIT, O.ANY_HIT])
@pytest.mark.parametrize("upd", [O.TWO_PHASE, O.SEQUENTIAL, O.UNBOUNDED])
@pytest.mark.parametrize("ways", [1, 4])
def test_results_equal_plain_over_frames(small, mode, upd, ways):
    tab = O.Table(10, ways, 6, upd)
    for frame in range(3):
        rays = small.primary_rays(frame=frame)[::2]
        hp, sp = O.trace(small.tris, small.nodes, small.prim_index, 0, rays, mode)
        hh, sh = O.trace(small.tris, small.nodes, small.prim_index, 0, rays, mode, tab)
        if mode == O.CLOSEST_HIT:
            assert np.array_equal(hp, hh), (frame, upd)
        else:
            # any-hit: the occlusion bit is unique; the prim reported need
            # only be a real hit of that ray
            assert np.array_equal(hp == O.NO_HIT, hh == O.NO_HIT), (frame, upd)
            for i in np.nonzero(hh != hp)[0]:
                tr = small.tris[hh[i]]
                assert O.ray_triangle(rays[i], tr[0:3], tr[3:6], tr[6:9])[0]
        _check_identities(sh, len(rays))
        assert sh["hits"] == sp["hits"]


def test_unbounded_second_pass_predicts_every_hit(small):
    rays = small.primary_rays()[::2]
    leaf_of = _leaf_of_prim(small.nodes, small.prim_index)
    for mode in (O.ANY_HIT, O.CLOSEST_HIT):
        tab = O.Table(0, 1, 6, O.UNBOUNDED)
        h1, s1 = O.trace(small.tris, small.nodes, small.prim_index, 0, rays, mode, tab)
        h2, s2, oc, _ = O.trace(small.tris, small.nodes, small.prim_index, 0, rays, mode, tab, per_ray=True)
        hit = (h2 if mode == O.ANY_HIT else h2["prim"]) != O.NO_HIT
        # every ray that hit has its own leaf under its key: a true positive
        assert np.all(oc[hit] == 3)
        assert s2["true_pos"] == int(hit.sum())
        assert s2["tp_inexact"] == 0 and s2["inserts"] == 0
        keys, leaves = tab.unbounded_size()
        # one key per distinct ray key that hit, each listing distinct leaves
        hit_rays = rays[hit]
        hk = {}
        prims = (h1 if mode == O.ANY_HIT else h1["prim"])[hit]
        for r, p in zip(hit_rays, prims):
            hk.setdefault(O.ray_key(r, 6), set()).add(leaf_of[int(p)])
        assert keys == len(hk)
        assert leaves == sum(len(v) for v in hk.values())


def test_any_hit_true_positives_skip_all_interior_work(small):
    rays = small.primary_rays()[::2]
    tab = O.Table(0, 1, 6, O.UNBOUNDED)
    O.trace(small.tris, small.nodes, small.prim_index, 0, small.primary_rays(frame=1)[::2], O.ANY_HIT, tab)
    _, sp, _, plain_boxes = O.trace(small.tris, small.nodes, small.prim_index, 0, rays, O.ANY_HIT, per_ray=True)
    _, sh, oc, hrpp_boxes = O.trace(small.tris, small.nodes, small.prim_index, 0, rays, O.ANY_HIT, tab,
                                    per_ray=True)
    tp = oc == 3
    assert tp.sum() > 1000
    assert np.all(hrpp_boxes[tp] == 0)
    assert np.array_equal(hrpp_boxes[~tp], plain_boxes[~tp])
    assert sh["box_tests"] == int(plain_boxes[~tp].sum())


def test_single_key_direct_mapped_winner_and_reuse(small):
    """All rays share one key: the highest-index hitting ray's leaf wins the
    slot; on the next pass exactly the rays that hit that leaf are true
    positives (brute force over the leaf's own triangles)."""
    rng = np.random.default_rng(0)
    n = 500
    o = np.array([0.0, 2.5, 6.0], np.float32)
    d = np.array([0.3, -0.55, -0.78]) + rng.uniform(-0.005, 0.005, (n, 3))
    d /= np.linalg.norm(d, axis=1, keepdims=True)
    rays = np.zeros((n, 8), np.float32)
    rays[:, 0:3], rays[:, 4:7], rays[:, 7] = o, d, np.inf
    p = 1
    keys = {O.ray_key(r, p) for r in rays}
    assert len(keys) == 1
    key = keys.pop()
    leaf_of = _leaf_of_prim(small.nodes, small.prim_index)
    tab = O.Table(8, 1, p, O.TWO_PHASE)
    s, tag = O.set_and_tag(key, 8)
    h1, s1 = O.trace(small.tris, small.nodes, small.prim_index, 0, rays, O.ANY_HIT, tab)
    hit_idx = np.nonzero(h1 != O.NO_HIT)[0]
    assert len(hit_idx) > 10
    last = int(hit_idx[-1])
    winner_leaf = leaf_of[int(h1[last])]
    assert int(tab.words[s]) == (tag << O.LEAF_BITS) | winner_leaf
    assert np.count_nonzero(tab.words != np.uint64(O.EMPTY_WORD)) == 1
    assert s1["inserts"] == len(hit_idx) and s1["dup_inserts"] == len(hit_idx) - 1
    # second pass: brute force over the winner leaf's triangles decides TP
    first, cnt = winner_leaf >> 2, (winner_leaf & 3) + 1
    leaf_prims = small.prim_index[first:first + cnt]
    expect_tp = np.array([any(O.ray_triangle(r, *np.split(small.tris[q], 3))[0] for q in leaf_prims)
                          for r in rays])
    _, s2, oc, _ = O.trace(small.tris, small.nodes, small.prim_index, 0, rays, O.ANY_HIT, tab, per_ray=True)
    assert np.array_equal(oc == 3, expect_tp)
    assert s2["positives"] == n and s2["pred_leaves"] == n


def _online_rays(small, n, seed):
    """Camera rays toward random points of the small scene: nearly all hit,
    and they spread over many leaves and keys."""
    rng = np.random.default_rng(seed)
    o = np.array([0.0, 2.5, 6.0])
    tgt = np.stack([rng.uniform(-3.5, 3.5, n), rng.uniform(0.0, 1.5, n), rng.uniform(-3.5, 3.5, n)], 1)
    d = tgt - o
    d /= np.linalg.norm(d, axis=1, keepdims=True)
    rays = np.zeros((n, 8), np.float32)
    rays[:, 0:3], rays[:, 4:7], rays[:, 7] = o, d, np.inf
    return rays


def _word_of(small, ray, p, log2_sets, leaf_of):
    """The table word ray `ray` inserts, from independent pieces: its key
    (Sec. 5 hash, pinned by worked values), the leaf holding its brute-force
    closest hit (found by walking the BVH's leaves) and the set/tag split."""
    key = O.ray_key(ray, p)
    _, tag = O.set_and_tag(key, log2_sets)
    hb, _ = O.brute(ray[None], small.tris, O.CLOSEST_HIT)
    prim = int(hb["prim"][0])
    return None if prim == O.NO_HIT else (tag << O.LEAF_BITS) | leaf_of[prim]


def test_online_fills_empty_ways_then_evicts(small):
    """Online mode, one set of four ways (every ray maps to it): inserts fill
    the empty ways first, every later insert evicts exactly one word, a set
    never holds a word twice (Sec. 5), and results are plain's."""
    tab = O.Table(2, 4, 6, O.ONLINE)
    rays = _online_rays(small, 300, seed=5)
    hp, _ = O.trace(small.tris, small.nodes, small.prim_index, 0, rays, O.CLOSEST_HIT)
    hh, st = O.trace(small.tris, small.nodes, small.prim_index, 0, rays, O.CLOSEST_HIT, tab)
    assert np.array_equal(hp, hh)
    assert st["inserts"] > 50
    assert st["evictions"] == st["inserts"] - 4
    assert st["dup_inserts"] == 0
    assert np.all(tab.words != np.uint64(O.EMPTY_WORD))
    assert len(set(tab.words.tolist())) == 4


def test_online_full_set_replaces_the_way_of_the_ray_index(small):
    """When a set is full, the insert of the call's ray i replaces way
    (i mod W): single-ray calls only ever rewrite way 0, and a four-ray call
    whose rays all insert leaves way k holding ray k's word, built from the
    ray's key and the leaf of its brute-force hit."""
    leaf_of = _leaf_of_prim(small.nodes, small.prim_index)
    tab = O.Table(2, 4, 6, O.ONLINE)
    rays = _online_rays(small, 400, seed=6)
    filled = None
    for k in range(200):
        _, st = O.trace(small.tris, small.nodes, small.prim_index, 0, rays[k:k + 1], O.CLOSEST_HIT, tab)
        if filled is None:
            if np.all(tab.words != np.uint64(O.EMPTY_WORD)):
                filled = tab.words.copy()
            continue
        assert np.array_equal(tab.words[1:], filled[1:]), k
    assert filled is not None
    # a batch of four inserting rays (distinct words, none already present)
    present = set(tab.words.tolist())
    batch, words = [], []
    for r in rays[200:]:
        w = _word_of(small, r, 6, 0, leaf_of)
        if w is not None and w not in present and w not in words:
            batch.append(r)
            words.append(w)
        if len(batch) == 4:
            break
    _, st = O.trace(small.tris, small.nodes, small.prim_index, 0, np.array(batch), O.CLOSEST_HIT, tab)
    assert st["inserts"] == 4 and st["evictions"] == 4
    assert tab.words.tolist() == words


def _sampled(n, sample_log2):
    i = np.arange(n)
    return ((i >> 5) & ((1 << sample_log2) - 1)) == 0


@pytest.mark.parametrize("mode", [O.CLOSEST_HIT, O.ANY_HIT])
def test_gate_off_changes_nothing(small, mode):
    """A gate threshold of 0 is no gate: hits, counters and table words equal
    a table without one, frame after frame."""
    a = O.Table(12, 2, 6, O.TWO_PHASE)
    b = O.Table(12, 2, 6, O.TWO_PHASE, gate_min_tp=0)
    for f in range(3):
        rays = small.primary_rays(frame=f)[::2]
        ha, sa = O.trace(small.tris, small.nodes, small.prim_index, 0, rays, mode, a)
        hb, sb = O.trace(small.tris, small.nodes, small.prim_index, 0, rays, mode, b)
        assert np.array_equal(ha, hb) and sa == sb and np.array_equal(a.words, b.words)
        assert sb["gated"] == 0


def test_closed_gate_leaves_the_table_to_the_sampled_chunks(small):
    """A threshold no call can reach (every lookup a true positive) closes the
    gate after the first call.  The next call: exactly the rays of every 8th
    32-ray chunk consult the table (a count fixed by the ray indices alone),
    every other ray is gated and does exactly its plain traversal with no
    insert, the results are plain's, and the table ends as it would after
    tracing only the sampled rays with an open gate."""
    s8 = 3
    tab = O.Table(12, 2, 6, O.TWO_PHASE, gate_min_tp=65536, gate_sample_log2=s8)
    ref = O.Table(12, 2, 6, O.TWO_PHASE)
    r1 = small.primary_rays(frame=1)
    _, st1 = O.trace(small.tris, small.nodes, small.prim_index, 0, r1, O.CLOSEST_HIT, tab)
    O.trace(small.tris, small.nodes, small.prim_index, 0, r1, O.CLOSEST_HIT, ref)
    assert st1["gated"] == 0 and st1["true_pos"] < st1["lookups"]
    assert not tab.gate_open
    r2 = small.primary_rays(frame=2)
    n = len(r2)
    smp = _sampled(n, s8)
    hp, _, _, plain_boxes = O.trace(small.tris, small.nodes, small.prim_index, 0, r2, O.CLOSEST_HIT, per_ray=True)
    hg, st2, oc, boxes = O.trace(small.tris, small.nodes, small.prim_index, 0, r2, O.CLOSEST_HIT, tab, per_ray=True)
    assert np.array_equal(hp, hg)
    assert st2["lookups"] == int(smp.sum()) and st2["gated"] == n - int(smp.sum())
    assert np.all(oc[~smp] == 0)
    assert np.array_equal(boxes[~smp], plain_boxes[~smp])
    O.trace(small.tris, small.nodes, small.prim_index, 0, np.ascontiguousarray(r2[smp]), O.CLOSEST_HIT, ref)
    assert np.array_equal(tab.words, ref.words)


def test_gate_reopens_when_the_sample_predicts(small):
    """The decision uses only the call's own consulting rays: with a
    threshold of one true positive per 65536 lookups a closed gate reopens
    after any call whose sampled rays hit a prediction, and a call whose
    sampled rays see none closes it again."""
    tab = O.Table(12, 1, 6, O.TWO_PHASE, gate_min_tp=1, gate_sample_log2=2)
    rays = small.primary_rays(frame=0)
    _, st = O.trace(small.tris, small.nodes, small.prim_index, 0, rays, O.CLOSEST_HIT, tab)
    assert st["true_pos"] == 0 and not tab.gate_open  # an empty table predicts nothing
    _, st = O.trace(small.tris, small.nodes, small.prim_index, 0, rays, O.CLOSEST_HIT, tab)
    assert st["gated"] > 0 and st["true_pos"] > 0 and tab.gate_open
    _, st = O.trace(small.tris, small.nodes, small.prim_index, 0, rays, O.CLOSEST_HIT, tab)
    assert st["gated"] == 0 and tab.gate_open
    # rays that all miss: no consulting ray predicts, the gate closes
    miss = rays.copy()
    miss[:, 4:7] = [0.0, 1.0, 0.0]
    _, st = O.trace(small.tris, small.nodes, small.prim_index, 0, miss, O.CLOSEST_HIT, tab)
    assert st["lookups"] == len(miss) and st["true_pos"] == 0 and not tab.gate_open


def test_two_phase_vs_sequential_within_a_batch(small):
    """Two-phase lookups see the table as it was at batch start; sequential
    lookups see earlier rays' inserts."""
    r = small.primary_rays()[::2]
    rays = np.concatenate([r, r])  # the second half repeats the first
    t2 = O.Table(16, 1, 6, O.TWO_PHASE)
    _, s2 = O.trace(small.tris, small.nodes, small.prim_index, 0, rays, O.ANY_HIT, t2)
    assert s2["positives"] == 0
    tseq = O.Table(16, 1, 6, O.SEQUENTIAL)
    _, sq = O.trace(small.tris, small.nodes, small.prim_index, 0, rays, O.ANY_HIT, tseq)
    assert sq["positives"] > 0 and sq["true_pos"] > 0


@pytest.mark.parametrize("ways", [2, 4, 8])
def test_ways_hold_distinct_leaves_of_one_key(small, ways):
    tab = O.Table(12, ways, 6, O.TWO_PHASE)
    for f in range(2):
        O.trace(small.tris, small.nodes, small.prim_index, 0, small.primary_rays(frame=f), O.CLOSEST_HIT, tab)
    w = tab.words.reshape(-1, ways)
    valid = w != np.uint64(O.EMPTY_WORD)
    leaves = (w & np.uint64((1 << O.LEAF_BITS) - 1)).astype(np.int64)
    tags = (w >> np.uint64(O.LEAF_BITS)).astype(np.int64)
    # a (tag, leaf) pair sits only in way way_of(leaf)
    for s, k in zip(*np.nonzero(valid)):
        assert O.way_of(int(leaves[s, k]), {2: 1, 4: 2, 8: 3}[ways]) == k
    # some set holds several leaves under one tag (several predictions per key)
    multi = 0
    for s in range(w.shape[0]):
        ts = tags[s][valid[s]]
        multi += len(ts) - len(set(ts.tolist()))
    assert multi > 0
    # every stored leaf is a real leaf of the BVH
    real = {(int(n["first"]) << 2) | (int(n["count"]) - 1) for n in small.nodes if n["count"] > 0}
    assert set(leaves[valid].tolist()) <= real


# ------------------------------------------------------------ Go Up Level --

def _preorder_and_parents(nodes, root=0):
    """Independent restatement: interior preorder ranks (children in slot
    order) and parent links of a canonical BVH."""
    rank, parent, stack = {}, {}, [root]
    while stack:
        i = stack.pop()
        if nodes[i]["count"] > 0:
            continue
        rank[i] = len(rank)
        for c in reversed([int(c) for c in nodes[i]["child"] if c >= 0]):
            parent[c] = i
            stack.append(c)
    return rank, parent


@pytest.mark.parametrize("go_up", [1, 2, 3])
@pytest.mark.parametrize("mode", [O.CLOSEST_HIT, O.ANY_HIT])
def test_go_up_results_equal_plain(small, go_up, mode):
    tab = O.Table(12, 2, 6, O.TWO_PHASE, go_up=go_up)
    for frame in range(3):
        rays = small.primary_rays(frame=frame)[::2]
        hp, _ = O.trace(small.tris, small.nodes, small.prim_index, 0, rays, mode)
        hh, sh = O.trace(small.tris, small.nodes, small.prim_index, 0, rays, mode, tab)
        if mode == O.CLOSEST_HIT:
            assert np.array_equal(hp, hh)
        else:
            assert np.array_equal(hp == O.NO_HIT, hh == O.NO_HIT)
        _check_identities(sh, len(rays))
    assert sh["true_pos"] > 0 and sh["pred_interior_nodes"] > 0


@pytest.mark.parametrize("go_up", [1, 2])
def test_go_up_table_holds_ancestors_of_hit_leaves(small, go_up):
    """Every stored node is the G-th ancestor (preorder rank) of a leaf that a
    ray of the batch hit; the insert goes to way way_of(rank)."""
    rank, parent = _preorder_and_parents(small.nodes)
    leaf_node = {int(n["first"]): i for i, n in enumerate(small.nodes) if n["count"] > 0}
    prim_leaf = {}
    for first, i in leaf_node.items():
        for j in range(int(small.nodes[i]["count"])):
            prim_leaf[int(small.prim_index[first + j])] = i
    rays = small.primary_rays()[::2]
    tab = O.Table(14, 2, 6, O.TWO_PHASE, go_up=go_up)
    h, _ = O.trace(small.tris, small.nodes, small.prim_index, 0, rays, O.CLOSEST_HIT, tab)
    expect = set()
    for p in h["prim"][h["prim"] != O.NO_HIT]:
        n = prim_leaf[int(p)]
        for _ in range(go_up):
            n = parent.get(n, n)
        expect.add(rank[n])
    w = tab.words.reshape(-1, 2)
    valid = w != np.uint64(O.EMPTY_WORD)
    stored = (w & np.uint64((1 << O.LEAF_BITS) - 1)).astype(np.int64)
    assert valid.sum() > 50
    assert set(stored[valid].tolist()) <= expect
    for s_, k in zip(*np.nonzero(valid)):
        assert O.way_of(int(stored[s_, k]), 1) == k


def test_go_up_past_the_root_predicts_the_whole_tree(small):
    """G larger than the tree's depth stores the root: a predicted ray then
    traverses the whole tree as its 'subtree', so a true positive's predicted
    work equals its plain traversal."""
    rays = small.primary_rays()[::4]
    tab = O.Table(16, 1, 6, O.UNBOUNDED, go_up=64)
    O.trace(small.tris, small.nodes, small.prim_index, 0, rays, O.ANY_HIT, tab)
    keys, nodes_stored = tab.unbounded_size()
    assert keys > 0 and nodes_stored == keys          # one node (the root) per key
    _, sp, _, plain_boxes = O.trace(small.tris, small.nodes, small.prim_index, 0, rays, O.ANY_HIT, per_ray=True)
    h, sh, oc, boxes = O.trace(small.tris, small.nodes, small.prim_index, 0, rays, O.ANY_HIT, tab, per_ray=True)
    tp = oc == 3
    hit = h != O.NO_HIT
    assert np.array_equal(tp, hit)                     # every ray that hits is a true positive
    assert np.all(boxes[tp] == 0)                      # no main traversal for them
    fp = oc == 2                                       # predicted but no hit: full subtree + full traversal
    assert sh["pred_box_tests"] == int(plain_boxes[tp].sum() + plain_boxes[fp].sum())


def test_go_up_unbounded_second_pass(small):
    rays = small.primary_rays()[::2]
    tab = O.Table(0, 1, 6, O.UNBOUNDED, go_up=1)
    h1, _ = O.trace(small.tris, small.nodes, small.prim_index, 0, rays, O.ANY_HIT, tab)
    keys1 = tab.unbounded_size()
    h2, s2, oc, _ = O.trace(small.tris, small.nodes, small.prim_index, 0, rays, O.ANY_HIT, tab, per_ray=True)
    hit = h2 != O.NO_HIT
    assert np.all(oc[hit] == 3) and s2["inserts"] == 0
    # go-up 1 needs no more nodes than go-up 0 (Sec. 6.2: fewer entries)
    tab0 = O.Table(0, 1, 6, O.UNBOUNDED, go_up=0)
    O.trace(small.tris, small.nodes, small.prim_index, 0, rays, O.ANY_HIT, tab0)
    assert keys1[1] <= tab0.unbounded_size()[1]


# ------------------------------------------------- predicted treelets --

def test_predicted_leaf_of_the_hit_is_a_true_positive(small):
    """A prediction naming the very leaf (or an ancestor) holding a ray's
    hit makes that ray a true positive; results never change."""
    rays = small.primary_rays()[::3]
    h, _ = O.trace(small.tris, small.nodes, small.prim_index, 0, rays, O.CLOSEST_HIT)
    leaf_node = {}
    for i, n in enumerate(small.nodes):
        if n["count"] > 0:
            for j in range(int(n["count"])):
                leaf_node[int(small.prim_index[n["first"] + j])] = i
    parent = {int(c): i for i, n in enumerate(small.nodes) for c in n["child"] if c >= 0}
    hit = h["prim"] != O.NO_HIT
    for lift in (0, 2):
        pred = np.full(len(rays), -1, np.int32)
        for k in np.nonzero(hit)[0]:
            n = leaf_node[int(h["prim"][k])]
            for _ in range(lift):
                n = parent.get(n, n)
            pred[k] = n
        for mode in (O.ANY_HIT, O.CLOSEST_HIT):
            hp, sp = O.trace(small.tris, small.nodes, small.prim_index, 0, rays, mode)
            hh, sh, oc, boxes = O.trace(small.tris, small.nodes, small.prim_index, 0, rays, mode, per_ray=True,
                                        predicted=pred)
            if mode == O.CLOSEST_HIT:
                assert np.array_equal(hp, hh)
            else:
                assert np.array_equal(hp == O.NO_HIT, hh == O.NO_HIT)
            assert np.array_equal(oc == 3, hit) and sh["inserts"] == 0
            assert sh["positives"] == int(hit.sum()) and sh["lookups"] == len(rays)
            if mode == O.ANY_HIT:
                assert np.all(boxes[hit] == 0)
    # out-of-range or unreachable predictions are ignored
    bad = np.full(len(rays), len(small.nodes) + 5, np.int32)
    _, sb = O.trace(small.tris, small.nodes, small.prim_index, 0, rays, O.ANY_HIT, predicted=bad)
    assert sb["positives"] == 0


# ---------------------------------------------- bottom-up verification --

def _tree(nodes, root):
    """Parent and depth of every node under root, from a walk of the node
    array written here (independent of the oracle's own tree walk)."""
    parent, depth = {}, {int(root): 0}
    stack = [int(root)]
    while stack:
        i = stack.pop()
        for c in nodes[i]["child"]:
            if c >= 0:
                parent[int(c)] = i
                depth[int(c)] = depth[i] + 1
                stack.append(int(c))
    return parent, depth


def _leaf_nodes(nodes, prim_index):
    m = {}
    for i, n in enumerate(nodes):
        if n["count"] > 0:
            for j in range(int(n["count"])):
                m[int(prim_index[n["first"] + j])] = i
    return m


_MOVED = ("interior_nodes", "box_tests", "leaves", "tri_tests")


@pytest.mark.parametrize("scene", ["small", "small4"])
def test_bottom_up_saves_exactly_the_climb_path(scene, request):
    """With the leaf of each ray's closest hit predicted, root verification
    and the climb visit the same sibling subtrees under the same bound: the
    climb makes one box test fewer per ancestor of the leaf (the child it came
    from), does not test the predicted leaf again, and visits the same
    interior nodes."""
    s = request.getfixturevalue(scene)
    rays = s.primary_rays()[::7]
    hp, _ = O.trace(s.tris, s.nodes, s.prim_index, s.root, rays, O.CLOSEST_HIT)
    leaf = _leaf_nodes(s.nodes, s.prim_index)
    _, depth = _tree(s.nodes, s.root)
    hit = np.nonzero(hp["prim"] != O.NO_HIT)[0]
    assert len(hit) > 100
    for k in hit[:160]:
        lf = leaf[int(hp["prim"][k])]
        pred = np.array([lf], np.int32)
        r = rays[k:k + 1]
        hr, sr = O.trace(s.tris, s.nodes, s.prim_index, s.root, r, O.CLOSEST_HIT, predicted=pred,
                         verify=O.VERIFY_ROOT)
        hb, sb = O.trace(s.tris, s.nodes, s.prim_index, s.root, r, O.CLOSEST_HIT, predicted=pred,
                         verify=O.VERIFY_BOTTOM_UP)
        assert hr.tobytes() == hb.tobytes() == hp[k:k + 1].tobytes()
        assert sb["true_pos"] == sr["true_pos"] == 1 and sb["tp_inexact"] == sr["tp_inexact"] == 0
        assert sr["interior_nodes"] == sb["interior_nodes"]
        assert sr["box_tests"] - sb["box_tests"] == depth[lf]
        assert sr["leaves"] - sb["leaves"] == 1
        assert sr["tri_tests"] - sb["tri_tests"] == int(s.nodes[lf]["count"])
        for key in sr:
            if key not in _MOVED:
                assert sr[key] == sb[key], key


@pytest.mark.parametrize("scene", ["small", "small4"])
@pytest.mark.parametrize("go_up", [0, 1])
@pytest.mark.parametrize("ways", [1, 4])
def test_bottom_up_keeps_results_and_table(scene, go_up, ways, request):
    """Over frames with a table, the climb returns exactly the plain hits and
    leaves the table and every predictor counter as root verification does
    (inserts depend only on the final hit); only traversal work moves, and
    it never grows."""
    s = request.getfixturevalue(scene)
    tr = O.Table(10, ways, 6, O.TWO_PHASE, go_up=go_up)
    tb = O.Table(10, ways, 6, O.TWO_PHASE, go_up=go_up)
    for frame in range(3):
        rays = s.primary_rays(frame=frame)[::2]
        hp, _ = O.trace(s.tris, s.nodes, s.prim_index, s.root, rays, O.CLOSEST_HIT)
        hr, sr = O.trace(s.tris, s.nodes, s.prim_index, s.root, rays, O.CLOSEST_HIT, tr, verify=O.VERIFY_ROOT)
        hb, sb = O.trace(s.tris, s.nodes, s.prim_index, s.root, rays, O.CLOSEST_HIT, tb,
                         verify=O.VERIFY_BOTTOM_UP)
        assert hp.tobytes() == hr.tobytes() == hb.tobytes()
        assert np.array_equal(tr.words, tb.words)
        for key in sr:
            if key not in _MOVED:
                assert sr[key] == sb[key], (frame, key)
        assert sb["box_tests"] <= sr["box_tests"]
        if frame > 0:
            assert sb["true_pos"] > 0 and sb["box_tests"] < sr["box_tests"]


def test_bottom_up_finds_a_closer_hit(small):
    """Predicting the leaf of a ray's second-nearest hit (a farther leaf):
    the climb must still return the nearest hit, and counts the ray as an
    inexact true positive, like root verification."""
    s = small
    rays = s.primary_rays()[::3]
    h1, _ = O.trace(s.tris, s.nodes, s.prim_index, s.root, rays, O.CLOSEST_HIT)
    beyond = rays.copy()
    beyond[:, 3] = h1["t"]                      # open interval: only hits past the first
    h2, _ = O.trace(s.tris, s.nodes, s.prim_index, s.root, beyond, O.CLOSEST_HIT)
    leaf = _leaf_nodes(s.nodes, s.prim_index)
    two = (h1["prim"] != O.NO_HIT) & (h2["prim"] != O.NO_HIT)
    pick = [k for k in np.nonzero(two)[0] if leaf[int(h1["prim"][k])] != leaf[int(h2["prim"][k])]]
    assert len(pick) > 50
    r = rays[pick]
    pred = np.array([leaf[int(h2["prim"][k])] for k in pick], np.int32)
    for verify in (O.VERIFY_ROOT, O.VERIFY_BOTTOM_UP):
        hh, st = O.trace(s.tris, s.nodes, s.prim_index, s.root, r, O.CLOSEST_HIT, predicted=pred, verify=verify)
        assert hh.tobytes() == h1[pick].tobytes()
        assert st["true_pos"] == len(pick) and st["tp_inexact"] == len(pick)


def test_bottom_up_on_a_root_leaf_scene():
    """A tree that is one leaf has nothing to climb: the predicted leaf's
    test is the whole answer."""
    from paper_1910_01304_gb300 import scenes as S
    tris = S.soup(3, 2, 0, 1, 0.5)
    nodes, prim, root = S.build_bvh(tris, trav_cost=0.0)  # 3 triangles: one leaf
    assert nodes[root]["count"] > 0
    rays = S.sphere_rays(300, 1, -0.5, 1.5)
    hp, _ = O.trace(tris, nodes, prim, root, rays, O.CLOSEST_HIT)
    pred = np.full(len(rays), root, np.int32)
    hb, sb = O.trace(tris, nodes, prim, root, rays, O.CLOSEST_HIT, predicted=pred, verify=O.VERIFY_BOTTOM_UP)
    assert hp.tobytes() == hb.tobytes()
    n_hit = int((hp["prim"] != O.NO_HIT).sum())
    assert n_hit > 0 and sb["true_pos"] == n_hit
    assert sb["box_tests"] == 0 and sb["interior_nodes"] == 0
    assert sb["leaves"] == len(rays) - n_hit      # only false positives traverse (the root leaf)


def test_exponent_lsb_hash_variant_keeps_results(small):
    """The exponent-LSB hash variant files rays under other keys (so other
    table words and predictions) but never changes a result."""
    tm = O.Table(12, 2, 6, O.TWO_PHASE)
    tl = O.Table(12, 2, 6, O.TWO_PHASE, hash_variant=O.HASH_EXP_LSB)
    tp = 0
    for frame in range(3):
        rays = small.primary_rays(frame=frame)[::2]
        hp, _ = O.trace(small.tris, small.nodes, small.prim_index, 0, rays, O.CLOSEST_HIT)
        hm, sm = O.trace(small.tris, small.nodes, small.prim_index, 0, rays, O.CLOSEST_HIT, tm)
        hl, sl = O.trace(small.tris, small.nodes, small.prim_index, 0, rays, O.CLOSEST_HIT, tl)
        assert hp.tobytes() == hm.tobytes() == hl.tobytes()
        tp += sl["true_pos"]
        _check_identities(sl, len(rays))
    assert tp > 0 and not np.array_equal(tm.words, tl.words)


# ------------------------------------------- qualitative trends (Sec. 5-6) --

def _unbounded_run(s, p, mode, warm_frames=3):
    """Warm an unbounded (limit-study) table with a few frames, then trace one
    more; returns (distinct keys, stored leaves, stats of the last frame)."""
    t = O.Table(12, 1, p, O.UNBOUNDED)

    def rays_of(f):
        pr = s.primary_rays(frame=f)[::2]
        if mode == O.CLOSEST_HIT:
            return pr
        ph, _ = O.trace(s.tris, s.nodes, s.prim_index, s.root, pr, O.CLOSEST_HIT)
        sh, _ = W.secondary_shadow(s, pr, ph["t"], ph["prim"])
        return sh

    for f in range(warm_frames):
        O.trace(s.tris, s.nodes, s.prim_index, s.root, rays_of(f), mode, t)
    keys, leaves = t.unbounded_size()
    _, st = O.trace(s.tris, s.nodes, s.prim_index, s.root, rays_of(warm_frames), mode, t)
    return keys, leaves, st


@pytest.mark.parametrize("mode", [O.CLOSEST_HIT, O.ANY_HIT])
def test_precision_trades_keys_for_false_positives(small, mode):
    """Sec. 5.1 / 6.1: looser hashing (fewer bits) files more rays under one
    key, so entries hold more leaves and predictions miss more often; tighter
    hashing needs more keys and more stored leaves."""
    runs = {p: _unbounded_run(small, p, mode) for p in (2, 4, 6)}
    keys = [runs[p][0] for p in (2, 4, 6)]
    leaves = [runs[p][1] for p in (2, 4, 6)]
    per_key = [l / k for k, l in zip(keys, leaves)]
    fps = [runs[p][2]["false_pos"] for p in (2, 4, 6)]
    assert keys[0] < keys[1] < keys[2]
    assert leaves[0] < leaves[1] < leaves[2]
    assert per_key[0] > per_key[1] > per_key[2]
    assert fps[0] > fps[1] > fps[2]


def test_hit_all_locality_exceeds_hit_any(small):
    """Sec. 6.1: closest-hit (hit-all) rays are predicted far more often than
    shadow (hit-any) rays with the same hash."""
    _, _, sc = _unbounded_run(small, 6, O.CLOSEST_HIT)
    _, _, sa = _unbounded_run(small, 6, O.ANY_HIT)
    assert sc["true_pos"] / sc["rays"] > 5 * sa["true_pos"] / sa["rays"]


# ------------------------------------ the paper's semantics (no verification) --

def test_unverified_true_positives_follow_the_paper(small):
    """VERIFY_NONE (Sec. 4.3 as the paper runs it): a closest-hit true
    positive returns the best hit among its predicted leaves and does no
    traversal and no insert; every other ray is exactly as with verification.
    Results can then differ from plain traversal only on true positives, and
    where they do, the returned hit is still a real hit of that ray."""
    s = small
    tv = O.Table(12, 2, 6, O.TWO_PHASE)
    tn = O.Table(12, 2, 6, O.TWO_PHASE)
    wrong_total = 0
    for frame in range(4):
        rays = s.primary_rays(frame=frame)[::2]
        hp, sp, _, bxp = O.trace(s.tris, s.nodes, s.prim_index, s.root, rays, O.CLOSEST_HIT, per_ray=True)
        hv, sv = O.trace(s.tris, s.nodes, s.prim_index, s.root, rays, O.CLOSEST_HIT, tv)
        hn, sn, ocn, bxn = O.trace(s.tris, s.nodes, s.prim_index, s.root, rays, O.CLOSEST_HIT, tn, per_ray=True,
                                   verify=O.VERIFY_NONE)
        assert hp.tobytes() == hv.tobytes()
        tp = ocn == 3
        assert np.all(bxn[tp] == 0) and sn["tp_inexact"] == 0
        # every other ray is answered and counted exactly as plain traversal
        assert hn[~tp].tobytes() == hp[~tp].tobytes() and np.array_equal(bxn[~tp], bxp[~tp])
        wrong = np.nonzero(hn["prim"] != hp["prim"])[0]
        assert np.all(tp[wrong])
        wrong_total += len(wrong)
        for k in wrong[:20]:   # a real hit of that ray, never closer than the true closest
            tri = np.asarray(s.tris, np.float32).reshape(-1, 9)[hn["prim"][k]]
            hit, t, _, _ = O.ray_triangle(rays[k], tri[0:3], tri[3:6], tri[6:9])
            assert hit and t == hn["t"][k] and hn["t"][k] >= hp["t"][k]
    assert wrong_total > 0
