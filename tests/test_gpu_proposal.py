"""The learned treelet proposal on the GPU (tcgen05 MLP) against the oracle
(oracle/proposal.py, fp64) and against the hash predictor.

Tolerances: features, class tables and labels are integer or exact-bf16
work and must match bit for bit.  The network runs bf16 inputs with fp32
accumulation and rounds hidden activations and back-propagated gradients to
bf16 (relative step 2^-8); the oracle keeps the activations' bf16 rounding
but computes everything else in fp64.  Three such roundings on a gradient's
path bound its relative error by a few 2^-8, so gradients must agree to 3%
(relative L2 per tensor, cosine > 0.999) and predicted classes must be an
argmax of the oracle's logits within 2% of the logit range."""
import numpy as np
import pytest

import oracle as O
from gpu_util import any_prims, as_words, assert_same_hits, assert_same_stats, gpu_trace, hrpp_mod
from oracle import proposal as P
from paper_1910_01304_gb300.scenes import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    H = hrpp_mod()
    s = W.small_scene()
    g = H.Scene.from_workload(s)
    prop = H.Proposal.for_workload(g, s, seed=1)
    return H, s, g, prop


def _rays(s, n=4000, seed=0):
    rng = np.random.default_rng(seed)
    r = s.primary_rays(frame=3)[:n].copy()
    # awkward directions: axis-aligned, -z, zero components, tiny values
    r[0:6, 4:7] = [[1, 0, 0], [-1, 0, 0], [0, 1, 0], [0, -1, 0], [0, 0, 1], [0, 0, -1]]
    r[6, 4:7] = [-0.0, 0.6, -0.8]
    r[7, 4:7] = [1e-30, -1e-30, -1.0]
    r[8:40, 0:3] = rng.uniform(-10, 10, (32, 3))          # origins outside the box
    return np.ascontiguousarray(r)


def _box(s):
    root = s.nodes[s.root]
    return root["lo"], root["hi"]


@pytest.mark.parametrize("n", [4000, 4001, 129])
def test_features_bit_exact(env, n):
    """Ragged tails: 4000 = 31 blocks of 128 + 32, 4001 leaves a row count
    that is not a multiple of 8, 129 a single row in the last block."""
    import torch
    H, s, g, prop = env
    rays = _rays(s)[:n] if n <= 4000 else np.ascontiguousarray(np.concatenate([_rays(s), s.primary_rays(frame=5)[:1]]))
    f = prop.features(torch.from_numpy(rays).cuda()).cpu()
    gpu = f.view(torch.int16).numpy().view(np.uint16)
    lo, hi = _box(s)
    ref = np.zeros((len(rays), 128), np.float32)
    ref[:, :96] = P.features(rays, lo, hi)
    ref_bits = (ref.view(np.uint32) >> 16).astype(np.uint16)
    bad = np.nonzero((gpu != ref_bits).any(axis=1))[0]
    assert len(bad) == 0, f"rows {bad[:5]} differ"


def test_class_nodes_and_labels(env):
    import torch
    H, s, g, prop = env
    _, to_node = P.leaf_codes(s.nodes, s.root, s.width)
    assert np.array_equal(prop.class_nodes(), to_node)
    rays = s.primary_rays(frame=2)
    dr = torch.from_numpy(rays).cuda()
    hits, _ = H.trace(g, dr, H.HRPP_CLOSEST_HIT)
    lab = prop.labels(hits).cpu().numpy()
    oh, _ = O.trace(s.tris, s.nodes, s.prim_index, s.root, rays, O.CLOSEST_HIT)
    pc = P.prim_classes(s.nodes, s.prim_index, s.root, s.width)
    expect = np.where(oh["prim"] == O.NO_HIT, -1, pc[np.minimum(oh["prim"], len(pc) - 1)])
    assert np.array_equal(lab, expect)


def test_gradients_match_oracle(env):
    import torch
    H, s, g, prop = env
    w = P.Weights.random(7, scale=0.4)
    prop.set_weights(w.flat())
    rays = _rays(s, 600, seed=1)
    rng = np.random.default_rng(2)
    labels = rng.integers(0, 4096, len(rays)).astype(np.int32)
    labels[::7] = -1
    loss_g, grads = prop.gradients(torch.from_numpy(rays).cuda(), torch.from_numpy(labels).cuda())
    lo, hi = _box(s)
    x = P.features(rays, lo, hi)
    loss_o, go = P.loss_and_grads(P.Weights.from_flat(w.flat()), x, labels)
    assert loss_g == pytest.approx(loss_o, rel=2e-3)
    gg = P.Weights.from_flat(grads)
    for k, _ in P.Weights.SHAPES:
        a, b = gg.a[k].ravel(), go[k].ravel()
        rel = np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-30)
        cos = float(a @ b / (np.linalg.norm(a) * np.linalg.norm(b) + 1e-30))
        assert rel < 3e-2 and cos > 0.999, (k, rel, cos)
    # weights round-trip through the API layout
    assert np.array_equal(prop.get_weights(), w.flat())


def test_predictions_are_argmax_of_oracle_logits(env):
    import torch
    H, s, g, prop = env
    w = P.Weights.random(11, scale=1.5)
    prop.set_weights(w.flat())
    rays = _rays(s, 3000, seed=3)
    nodes, classes = prop.predict(torch.from_numpy(rays).cuda())
    classes = classes.cpu().numpy()
    lo, hi = _box(s)
    _, _, z = P.forward(P.Weights.from_flat(w.flat()), P.features(rays, lo, hi))
    zmax = z.max(axis=1)
    span = zmax - z.min(axis=1)
    picked = z[np.arange(len(rays)), classes]
    assert np.all(zmax - picked <= 0.02 * span)
    assert np.mean(classes == np.argmax(z, axis=1)) > 0.97
    _, to_node = P.leaf_codes(s.nodes, s.root, s.width)
    assert np.array_equal(nodes.cpu().numpy(), to_node[classes])


@pytest.mark.parametrize("width", [2, 4])
def test_trace_with_predicted_nodes_matches_oracle(width):
    """Predicted treelets given to both sides (valid nodes, -1 and
    out-of-range values): hits, counters and table words match."""
    import torch
    H = hrpp_mod()
    s = W.small_scene(width=width)
    g = H.Scene.from_workload(s)
    rng = np.random.default_rng(width)
    prim = s.primary_rays(frame=4)
    ph, _ = O.trace(s.tris, s.nodes, s.prim_index, s.root, prim, O.CLOSEST_HIT)
    shadow, _ = W.secondary_shadow(s, prim, ph["t"], ph["prim"])
    for mode, rays in ((O.CLOSEST_HIT, prim), (O.ANY_HIT, shadow)):
        pred = rng.integers(-1, len(s.nodes) + 3, len(rays)).astype(np.int32)
        dpred = torch.from_numpy(pred).cuda()
        for use_table in (False, True):
            t = H.Table(12, 2, 6) if use_table else None
            ot = O.Table(12, 2, 6, O.TWO_PHASE) if use_table else None
            oh, ost = O.trace(s.tris, s.nodes, s.prim_index, s.root, rays, mode, ot, predicted=pred)
            gh, gst = H.trace(g, torch.from_numpy(rays).cuda(), mode, t, stats=True, predicted=dpred)
            torch.cuda.synchronize()
            assert_same_hits(mode, gh.cpu().numpy(), oh)
            assert_same_stats(gst, ost)
            if use_table:
                assert np.array_equal(t.export(), ot.words)


def test_training_beats_the_hash_predictor():
    """Trained on traversal traces of the small scene's camera (jittered
    frames), the network predicts the treelet holding the closest hit for
    more held-out primary rays than the hash table does, and the traced
    results stay exactly those of plain traversal."""
    import torch
    H = hrpp_mod()
    s = W.small_scene()
    g = H.Scene.from_workload(s)
    prop = H.Proposal.for_workload(g, s, seed=5)
    tab = H.Table(12, 1, 6)
    losses = []
    for f in range(1, 25):
        r = torch.from_numpy(s.primary_rays(frame=f)).cuda()
        hits, _ = H.trace(g, r, H.HRPP_CLOSEST_HIT, tab)           # the hash table sees the same frames
        lab = prop.labels(hits)
        loss = prop.train(r, lab, lr=2e-3, want_loss=(f % 6 == 0))
        if loss is not None:
            losses.append(loss)
    assert losses[-1] < losses[0]
    test = torch.from_numpy(s.primary_rays(frame=100)).cuda()
    plain, _ = H.trace(g, test, H.HRPP_CLOSEST_HIT)
    nodes, _ = prop.predict(test)
    learned, sl = H.trace(g, test, H.HRPP_CLOSEST_HIT, stats=True, predicted=nodes)
    hashed, sh = H.trace(g, test, H.HRPP_CLOSEST_HIT, tab, stats=True)
    torch.cuda.synchronize()
    assert torch.equal(plain.view(torch.int32), learned.view(torch.int32))
    assert torch.equal(plain.view(torch.int32), hashed.view(torch.int32))
    assert sl["true_pos"] > 1.5 * sh["true_pos"], (sl["true_pos"], sh["true_pos"])


def _many_rays(s, n, seed):
    """n rays from jittered camera frames of the small scene, with random
    origins mixed in so that rows differ across chunk boundaries."""
    rng = np.random.default_rng(seed)
    out, f = [], 1
    while sum(len(r) for r in out) < n:
        out.append(s.primary_rays(frame=f))
        f += 1
    r = np.concatenate(out)[:n].copy()
    r[::5, 0:3] = rng.uniform(-6, 6, (len(r[::5]), 3))
    return np.ascontiguousarray(r)


def test_predictions_across_inference_chunks(env):
    """Prediction runs in chunks of 65,536 rows: 140,001 rays cover two
    full chunks and a ragged tail.  Rows sampled around every chunk and tile
    boundary are an argmax of the oracle's logits."""
    import torch
    H, s, g, prop = env
    w = P.Weights.random(13, scale=1.5)
    prop.set_weights(w.flat())
    n = 140_001
    rays = _many_rays(s, n, 4)
    nodes, classes = prop.predict(torch.from_numpy(rays).cuda())
    classes = classes.cpu().numpy()
    edges = [0, 127, 128, 65535, 65536, 65537, 131071, 131072, 131073, n - 2, n - 1]
    rng = np.random.default_rng(5)
    rows = np.unique(np.concatenate([edges, rng.integers(0, n, 1500)]))
    lo, hi = _box(s)
    _, _, z = P.forward(P.Weights.from_flat(w.flat()), P.features(rays[rows], lo, hi))
    zmax, span = z.max(axis=1), z.max(axis=1) - z.min(axis=1)
    picked = z[np.arange(len(rows)), classes[rows]]
    assert np.all(zmax - picked <= 0.02 * span)
    assert np.mean(classes[rows] == np.argmax(z, axis=1)) > 0.97
    _, to_node = P.leaf_codes(s.nodes, s.root, s.width)
    assert np.array_equal(nodes.cpu().numpy(), to_node[classes])


@pytest.mark.parametrize("n", [9000, 16384])
def test_gradients_of_a_ragged_batch(env, n):
    """9,000 rays (70 full 128-row tiles and a tail of 40), and a full
    16,384-row minibatch: the size at which the 4096-column bias gradient
    takes 256 rows per block and the weight gradients their full split-K
    grids."""
    import torch
    H, s, g, prop = env
    w = P.Weights.random(17, scale=0.4)
    prop.set_weights(w.flat())
    rays = _many_rays(s, n, 6)
    labels = np.random.default_rng(7).integers(-1, 4096, len(rays)).astype(np.int32)
    loss_g, grads = prop.gradients(torch.from_numpy(rays).cuda(), torch.from_numpy(labels).cuda())
    lo, hi = _box(s)
    loss_o, go = P.loss_and_grads(P.Weights.from_flat(w.flat()), P.features(rays, lo, hi), labels)
    assert loss_g == pytest.approx(loss_o, rel=2e-3)
    gg = P.Weights.from_flat(grads)
    for k, _ in P.Weights.SHAPES:
        a, b = gg.a[k].ravel(), go[k].ravel()
        rel = np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-30)
        cos = float(a @ b / (np.linalg.norm(a) * np.linalg.norm(b) + 1e-30))
        assert rel < 3e-2 and cos > 0.999, (k, rel, cos)


def test_gradients_reject_an_oversized_batch(env):
    import torch
    H, s, g, prop = env
    rays = torch.zeros((16385, 8), dtype=torch.float32, device="cuda")
    labels = torch.zeros(16385, dtype=torch.int32, device="cuda")
    with pytest.raises(RuntimeError):
        prop.gradients(rays, labels)


def test_train_loss_covers_every_minibatch(env):
    """A train call over 20,000 rays takes two minibatches (16,384 + 3,616).
    With a step far below bf16 resolution the weights do not move, so the
    reported loss is the oracle's mean loss over all labelled rays."""
    import torch
    H, s, g, prop = env
    w = P.Weights.random(19, scale=0.4)
    prop.set_weights(w.flat())
    rays = _many_rays(s, 20_000, 8)
    labels = np.random.default_rng(9).integers(-1, 4096, len(rays)).astype(np.int32)
    labels[16384:] = np.where(labels[16384:] >= 0, 7, -1)   # the second minibatch differs in loss
    loss = prop.train(torch.from_numpy(rays).cuda(), torch.from_numpy(labels).cuda(), lr=1e-20, want_loss=True)
    lo, hi = _box(s)
    wo = P.Weights.from_flat(w.flat())
    total, count = 0.0, 0
    for a in range(0, len(rays), 5000):
        lab = labels[a:a + 5000]
        l, _ = P.loss_and_grads(wo, P.features(rays[a:a + 5000], lo, hi), lab)
        k = int((lab >= 0).sum())
        total += l * k
        count += k
    assert loss == pytest.approx(total / count, rel=2e-3)


def test_adam_steps_follow_the_update_rule(env):
    """Two train calls of one minibatch each move every weight as Adam with
    bias correction does (beta1 0.9, beta2 0.999, eps 1e-8; Kingma and Ba's
    update) on the gradients that hrpp_proposal_gradients reports at the same
    weights.  The first step has a closed form, -lr g / (|g| + eps): lr against
    the sign of every gradient clear of zero.  Gradients are recomputed inside
    the train call with fp32 atomics in another order, so the check keeps to
    entries whose gradients are far from zero (relative noise ~1e-6); every
    other entry moves by no more than Adam's bound on a step."""
    import torch
    H, s, g, prop = env
    w0 = P.Weights.random(23, scale=0.4).flat()
    rays = torch.from_numpy(_rays(s, 3000, seed=5)).cuda()
    labels = torch.from_numpy(np.random.default_rng(6).integers(0, 4096, 3000).astype(np.int32)).cuda()
    lr = 1e-3
    prop.set_weights(w0)
    _, g1 = prop.gradients(rays, labels)
    prop.train(rays, labels, lr=lr)
    w1 = prop.get_weights()
    _, g2 = prop.gradients(rays, labels)
    prop.train(rays, labels, lr=lr)
    w2 = prop.get_weights()
    ga, gb = g1.astype(np.float64), g2.astype(np.float64)
    step1 = -lr * ga / (np.abs(ga) + 1e-8)
    m = 0.09 * ga + 0.1 * gb
    v = 0.999 * 0.001 * ga * ga + 0.001 * gb * gb
    step2 = -lr * (m / (1 - 0.9 ** 2)) / (np.sqrt(v / (1 - 0.999 ** 2)) + 1e-8)
    off = 0
    for k, shape in P.Weights.SHAPES:
        n = int(np.prod(shape))
        sl = slice(off, off + n)
        off += n
        big = lambda x: np.abs(x) > max(1e-4 * np.abs(x).max(), 1e-6)
        keep1, keep2 = big(ga[sl]), big(ga[sl]) & big(gb[sl])
        assert keep1.mean() > 0.25 and keep2.mean() > 0.25, (k, keep1.mean(), keep2.mean())
        d1 = w1[sl].astype(np.float64) - w0[sl]
        d2 = w2[sl].astype(np.float64) - w1[sl]
        tol = 1e-3 * lr + 1e-7
        assert np.abs(d1 - step1[sl])[keep1].max() < tol, k
        assert np.abs(d2 - step2[sl])[keep2].max() < tol, k
        # |m_hat| / sqrt(v_hat) <= 1 at step 1 and <= 1.0014 at step 2 (Cauchy-Schwarz)
        assert np.abs(d1).max() <= lr * 1.0001 + 1e-7 and np.abs(d2).max() <= lr * 1.002 + 1e-7, k
    assert off == len(w0)
