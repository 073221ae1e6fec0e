"""Pins for the learned-proposal oracle (oracle/proposal.py): bf16 rounding,
the feature definition on hand-placed rays, gradients against finite
differences, the uniform-softmax loss, and the treelet class codes against
the BVH itself."""
import math

import numpy as np
import pytest

from oracle import proposal as P
from paper_1910_01304_gb300 import scenes as S


def test_bf16_rounding():
    one = np.float32(1.0)
    assert P.bf16(one) == one
    assert P.bf16(np.float32(1 + 2 ** -8)) == one                  # tie -> even
    assert P.bf16(np.float32(1 + 3 * 2 ** -8)) == np.float32(1 + 2 ** -6)  # tie, odd -> up
    assert P.bf16(np.float32(1 + 2 ** -7)) == np.float32(1 + 2 ** -7)  # representable
    assert P.bf16(np.float32(1 + 2 ** -8 + 2 ** -12)) == np.float32(1 + 2 ** -7)
    assert P.bf16(np.float32(-2.5)) == np.float32(-2.5)
    assert np.isnan(P.bf16(np.float32(np.nan)))


def test_sine_table_anchors():
    s = P.sine_table()
    assert s.shape == (65536,)
    assert s[0] == 0 and s[16384] == 1 and s[49152] == -1
    assert abs(s[32768]) < 1e-15
    assert s[8192] == P.bf16(np.float32(math.sqrt(0.5)))
    # every entry is a bf16 value
    assert np.array_equal(P.bf16(s), s)


def _ray(o, d):
    return np.array([[*o, 0.0, *d, np.inf]], np.float32)


def test_quantised_inputs_on_axes_and_box():
    lo, hi = (0.0, 0.0, 0.0), (2.0, 4.0, 8.0)
    q = P.quantised_inputs(_ray((1.0, 2.0, 4.0), (1, 0, 0)), lo, hi)[0]
    assert list(q[:3]) == [32767, 32767, 32767]              # box centre
    assert list(q[3:]) == [65535, 32767]                     # +x -> (1, 0)
    q = P.quantised_inputs(_ray((-5.0, 100.0, 0.0), (0, 0, 1)), lo, hi)[0]
    assert list(q) == [0, 65535, 0, 32767, 32767]            # clamped; +z -> (0, 0)
    q = P.quantised_inputs(_ray((0, 0, 0), (0, 0, -1)), lo, hi)[0]
    assert list(q[3:]) == [65535, 65535]                     # -z folds to (1, 1)
    q = P.quantised_inputs(_ray((0, 0, 0), (0, -1, 0)), lo, hi)[0]
    assert list(q[3:]) == [32767, 0]                         # -y -> (0, -1)
    q = P.quantised_inputs(_ray((0, 0, 0), (-1, 0, -1e-30)), lo, hi)[0]
    assert list(q[3:]) == [0, 32767]                          # -x just below the equator: the fold keeps (-1, 0)


def test_feature_layout():
    rays = np.concatenate([_ray((0.3, 0.7, 0.1), (0.2, -0.5, 0.8)), _ray((0.9, 0.2, 0.5), (-0.6, 0.1, -0.7))])
    f = P.features(rays, (0, 0, 0), (1, 1, 1))
    q = P.quantised_inputs(rays, (0, 0, 0), (1, 1, 1))
    s = P.sine_table()
    assert f.shape == (2, 96) and np.all(f[:, 95] == 1)
    for r in range(2):
        for i in range(5):
            assert f[r, i] == P.bf16(np.float32(q[r, i] / 32768.0 - 1.0))
            for k in range(9):
                ph = (int(q[r, i]) << k) & 0xFFFF
                assert f[r, 5 + 18 * i + 2 * k] == s[ph]
                assert f[r, 6 + 18 * i + 2 * k] == s[(ph + 16384) & 0xFFFF]
    # sin^2 + cos^2 = 1 within bf16 rounding
    sin = f[:, 5:95:2].astype(np.float64)
    cos = f[:, 6:95:2].astype(np.float64)
    assert np.allclose(sin ** 2 + cos ** 2, 1.0, atol=2e-2)


def test_uniform_logits_give_log_classes():
    w = P.Weights({k: np.zeros(s) for k, s in P.Weights.SHAPES})
    x = np.random.default_rng(0).normal(size=(5, 96))
    loss, g = P.loss_and_grads(w, x, np.array([0, 7, -1, 4095, 3]))
    assert loss == pytest.approx(math.log(4096))
    # dL/db3 = mean(p - onehot) over the four labelled rows
    expect = np.full(4096, 4 / 4096 / 4)
    for lab in (0, 7, 4095, 3):
        expect[lab] -= 1 / 4
    assert np.allclose(g["b3"], expect)


def test_gradients_match_finite_differences():
    rng = np.random.default_rng(1)
    w = P.Weights.random(3, scale=0.5)
    x = rng.normal(size=(6, 96))
    lab = np.array([5, 100, -1, 4000, 17, 2048])
    _, g = P.loss_and_grads(w, x, lab, round_bf16=False)
    h = 1e-6
    for key in ("W1", "b1", "W2", "b2", "W3", "b3"):
        a = w.a[key]
        flat = a.reshape(-1)
        for idx in rng.choice(flat.size, 6, replace=False):
            old = flat[idx]
            flat[idx] = old + h
            lp, _ = P.loss_and_grads(w, x, lab, round_bf16=False)
            flat[idx] = old - h
            lm, _ = P.loss_and_grads(w, x, lab, round_bf16=False)
            flat[idx] = old
            fd = (lp - lm) / (2 * h)
            an = g[key].reshape(-1)[idx]
            assert abs(fd - an) <= 1e-6 + 1e-4 * abs(fd), (key, idx, fd, an)


def test_predict_is_first_argmax():
    w = P.Weights({k: np.zeros(s) for k, s in P.Weights.SHAPES})
    w.a["b3"][[10, 20]] = 1.0
    assert list(P.predict(w, np.zeros((3, 96)))) == [10, 10, 10]


@pytest.mark.parametrize("width", [2, 4])
def test_class_codes_follow_the_tree(width):
    from paper_1910_01304_gb300.scenes import workloads as W
    s = W.small_scene(width=width)
    code_of, to_node = P.leaf_codes(s.nodes, s.root, width)
    leaves = [i for i, n in enumerate(s.nodes) if n["count"] > 0]
    assert set(code_of) == set(leaves)
    parent = {int(c): i for i, n in enumerate(s.nodes) for c in n["child"] if c >= 0}

    def depth(i):
        d = 0
        while i in parent:
            i, d = parent[i], d + 1
        return d

    levels = 12 if width == 2 else 6
    for i, c in code_of.items():
        a = i
        while depth(a) > levels:
            a = parent[a]
        # a leaf within the code's depth is its own treelet; a deeper one
        # belongs to its ancestor at the code's depth
        assert to_node[c] == a
    shallow = [i for i in leaves if depth(i) <= levels]
    assert len({code_of[i] for i in shallow}) == len(shallow)
    pc = P.prim_classes(s.nodes, s.prim_index, s.root, width)
    assert np.all(pc >= 0) and len(pc) == s.n_tris


def test_deep_leaves_share_their_depth_limit_ancestor():
    tris = S.soup(40000, 4)
    nodes, prim, root = S.build_bvh(tris, width=2)
    code_of, to_node = P.leaf_codes(nodes, root, 2)
    parent = {}
    for i, n in enumerate(nodes):
        for c in n["child"]:
            if c >= 0:
                parent[int(c)] = i

    def depth(i):
        d = 0
        while i in parent:
            i = parent[i]
            d += 1
        return d

    deep = [i for i in code_of if depth(i) > 12]
    assert deep
    for i in deep[:200]:
        a = i
        while depth(a) > 12:
            a = parent[a]
        assert to_node[code_of[i]] == a
