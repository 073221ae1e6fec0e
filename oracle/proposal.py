"""Oracle of the learned treelet proposal -- TEST INFRASTRUCTURE ONLY.

Plain numpy restatement (fp64 where the network computes, float32 where the
definition fixes float32 steps) of what the library's tensor-core MLP
computes.  Shares no code with the CUDA path.

Definition
----------
Input features (96 per ray) of a ray (o, d) in a scene box [lo, hi]:
  q0..q2  origin quantised to 16 bits: u = (o - lo) * (65535 / (hi - lo)),
          float32 steps, then 0 if u <= 0 (or NaN), 65535 if u >= 65535,
          else trunc(u)
  q3, q4  direction, octahedral encoding: p = d.xy / (|d.x| + |d.y| + |d.z|);
          for d.z < 0, p = ((1 - |p.y|) sgn p.x, (1 - |p.x|) sgn p.y) with
          sgn(0) = +1; u = (p + 1) * 32767.5, quantised as above
  f[0..4]            bf16(q_i / 32768 - 1)
  f[5 + 18i + 2k]    S[(q_i << k) mod 65536],  k = 0..8   (Fourier sine)
  f[6 + 18i + 2k]    S[((q_i << k) + 16384) mod 65536]    (Fourier cosine)
  f[95]              1
  S[j] = bf16(float32(sin(2 pi j / 65536)))  (round to float32, then bf16,
  each to nearest even).
Network: H1 = bf16(relu(X W1^T + b1)), H2 = bf16(relu(H1 W2^T + b2)),
Z = H2 W3^T + b3; weights used as bf16, biases fp32; 96 -> 256 -> 256 -> 4096.
Loss: mean softmax cross-entropy over rays with a label (label >= 0).
Prediction: argmax_j Z_j, the first index among equal maxima.
Classes: the 12-bit path code from the root (BVH2: one child-slot bit per
level, 12 levels; BVH4: two bits per level, 6 levels; leaves shallower than
that pad with zeros).  A class's treelet root is the node reached by
following its code from the root, stopping at a leaf or a missing child.
"""
from __future__ import annotations

import math

import numpy as np

N_FEATURES, HIDDEN, N_CLASSES = 96, 256, 4096
CODE_BITS = 12

# ---------------------------------------------------------------- bf16 --


def bf16(x) -> np.ndarray:
    """Round to the nearest bfloat16 (ties to even), through float32."""
    f = np.asarray(x, dtype=np.float32)
    b = f.view(np.uint32).astype(np.uint64)
    rounded = (b + 0x7FFF + ((b >> 16) & 1)) & 0xFFFF0000
    out = rounded.astype(np.uint32).view(np.float32)
    nan = np.isnan(f)
    if np.any(nan):
        out = np.where(nan, np.float32(np.nan), out)
    return out


_SIN = None


def sine_table() -> np.ndarray:
    global _SIN
    if _SIN is None:
        vals = np.array([math.sin(2.0 * math.pi * j / 65536.0) for j in range(65536)], np.float64)
        _SIN = bf16(vals.astype(np.float32))
    return _SIN


# ------------------------------------------------------------ features --


def _quantise(u: np.ndarray) -> np.ndarray:
    u = np.asarray(u, np.float32)
    q = np.zeros(u.shape, np.int64)
    big = u >= np.float32(65535.0)
    mid = (u > 0) & ~big
    q[mid] = u[mid].astype(np.int64)     # truncation toward zero
    q[big] = 65535
    return q


def quantised_inputs(rays: np.ndarray, lo, hi) -> np.ndarray:
    """[n, 5] int64: quantised origin (3) and octahedral direction (2)."""
    r = np.asarray(rays, np.float32).reshape(-1, 8)
    lo = np.asarray(lo, np.float32)
    hi = np.asarray(hi, np.float32)
    q = np.zeros((r.shape[0], 5), np.int64)
    with np.errstate(divide="ignore", invalid="ignore"):
        for a in range(3):
            s = np.float32(65535.0) / (hi[a] - lo[a])
            q[:, a] = _quantise((r[:, a] - lo[a]) * s)
        ax, ay, az = np.abs(r[:, 4]), np.abs(r[:, 5]), np.abs(r[:, 6])
        l1 = (ax + ay) + az
        px = r[:, 4] / l1
        py = r[:, 5] / l1
        sx = np.where(px >= 0, np.float32(1), np.float32(-1))
        sy = np.where(py >= 0, np.float32(1), np.float32(-1))
        fold = r[:, 6] < 0
        ux = np.where(fold, (np.float32(1) - np.abs(py)) * sx, px).astype(np.float32)
        uy = np.where(fold, (np.float32(1) - np.abs(px)) * sy, py).astype(np.float32)
        q[:, 3] = _quantise((ux + np.float32(1)) * np.float32(32767.5))
        q[:, 4] = _quantise((uy + np.float32(1)) * np.float32(32767.5))
    return q


def features(rays: np.ndarray, lo, hi) -> np.ndarray:
    """[n, 96] float32 (bf16 values) network inputs."""
    q = quantised_inputs(rays, lo, hi)
    S = sine_table()
    n = q.shape[0]
    f = np.zeros((n, N_FEATURES), np.float32)
    f[:, 0:5] = bf16(q.astype(np.float32) * np.float32(1.0 / 32768.0) - np.float32(1.0))
    for i in range(5):
        for k in range(9):
            ph = (q[:, i] << k) & 0xFFFF
            f[:, 5 + 18 * i + 2 * k] = S[ph]
            f[:, 6 + 18 * i + 2 * k] = S[(ph + 16384) & 0xFFFF]
    f[:, 95] = 1.0
    return f


# ------------------------------------------------------------- network --


class Weights:
    """W1 [256, 96], b1 [256], W2 [256, 256], b2 [256], W3 [4096, 256], b3 [4096]."""

    SHAPES = [("W1", (HIDDEN, N_FEATURES)), ("b1", (HIDDEN,)), ("W2", (HIDDEN, HIDDEN)), ("b2", (HIDDEN,)),
              ("W3", (N_CLASSES, HIDDEN)), ("b3", (N_CLASSES,))]

    def __init__(self, arrays: dict):
        self.a = {k: np.asarray(arrays[k], np.float64) for k, _ in self.SHAPES}

    @classmethod
    def random(cls, seed: int, scale: float = 1.0):
        rng = np.random.default_rng(seed)
        arr = {}
        for k, shp in cls.SHAPES:
            if k.startswith("W"):
                a = math.sqrt(6.0 / shp[1]) * scale
                arr[k] = rng.uniform(-a, a, shp)
            else:
                arr[k] = rng.uniform(-0.1, 0.1, shp) * scale
        return cls(arr)

    def flat(self) -> np.ndarray:
        return np.concatenate([self.a[k].ravel() for k, _ in self.SHAPES]).astype(np.float32)

    @classmethod
    def from_flat(cls, v: np.ndarray):
        v = np.asarray(v, np.float64)
        arr, off = {}, 0
        for k, shp in cls.SHAPES:
            n = int(np.prod(shp))
            arr[k] = v[off:off + n].reshape(shp)
            off += n
        return cls(arr)

    @classmethod
    def size(cls) -> int:
        return int(sum(np.prod(s) for _, s in cls.SHAPES))


def forward(w: Weights, x: np.ndarray, round_bf16: bool = True):
    """Returns (H1, H2, Z) in fp64.  round_bf16 applies the network's bf16
    rounding of weights and hidden activations (off only for derivative
    checks of the formulas)."""
    r = bf16 if round_bf16 else (lambda a: np.asarray(a, np.float64))
    W1, W2, W3 = (np.asarray(r(w.a[k]), np.float64) for k in ("W1", "W2", "W3"))
    x = np.asarray(x, np.float64)
    h1 = np.asarray(r(np.maximum(x @ W1.T + w.a["b1"], 0.0)), np.float64)
    h2 = np.asarray(r(np.maximum(h1 @ W2.T + w.a["b2"], 0.0)), np.float64)
    z = h2 @ W3.T + w.a["b3"]
    return h1, h2, z


def loss_and_grads(w: Weights, x: np.ndarray, labels: np.ndarray, round_bf16: bool = True):
    """Mean softmax cross-entropy over labelled rows, and its gradients with
    respect to every weight and bias (the bf16 roundings are differentiated
    as the identity)."""
    r = bf16 if round_bf16 else (lambda a: np.asarray(a, np.float64))
    W1, W2, W3 = (np.asarray(r(w.a[k]), np.float64) for k in ("W1", "W2", "W3"))
    x = np.asarray(x, np.float64)
    h1, h2, z = forward(w, x, round_bf16)
    lab = np.asarray(labels, np.int64)
    m = lab >= 0
    n_lab = int(m.sum())
    zs = z - z.max(axis=1, keepdims=True)
    p = np.exp(zs)
    p /= p.sum(axis=1, keepdims=True)
    loss = 0.0
    dz = np.zeros_like(z)
    if n_lab:
        idx = np.nonzero(m)[0]
        loss = float(-np.log(p[idx, lab[idx]]).sum() / n_lab)
        dz[idx] = p[idx]
        dz[idx, lab[idx]] -= 1.0
        dz /= n_lab
    g = {"W3": dz.T @ h2, "b3": dz.sum(0)}
    dh2 = dz @ W3
    dz2 = dh2 * (h2 > 0)
    g["W2"] = dz2.T @ h1
    g["b2"] = dz2.sum(0)
    dh1 = dz2 @ W2
    dz1 = dh1 * (h1 > 0)
    g["W1"] = dz1.T @ x
    g["b1"] = dz1.sum(0)
    return loss, g


def predict(w: Weights, x: np.ndarray) -> np.ndarray:
    _, _, z = forward(w, x)
    return np.argmax(z, axis=1)


# ------------------------------------------------------------- classes --


def leaf_codes(nodes: np.ndarray, root: int, width: int):
    """(class of each leaf node index, class -> treelet root node) for a
    canonical BVH."""
    bits_per = 1 if width == 2 else 2
    levels = CODE_BITS // bits_per
    code_of = {}
    stack = [(root, 0, 0)]
    while stack:
        i, code, depth = stack.pop()
        if nodes[i]["count"] > 0:
            code_of[i] = code << (bits_per * (levels - depth)) if depth <= levels else code
            continue
        for s, c in enumerate(nodes[i]["child"]):
            if c < 0:
                continue
            if depth < levels:
                stack.append((int(c), (code << bits_per) | s, depth + 1))
            else:
                stack.append((int(c), code, depth + 1))
    to_node = np.zeros(1 << CODE_BITS, np.int64)
    for cls in range(1 << CODE_BITS):
        n = root
        for lv in range(levels):
            if nodes[n]["count"] > 0:
                break
            s = (cls >> (bits_per * (levels - 1 - lv))) & ((1 << bits_per) - 1)
            c = int(nodes[n]["child"][s])
            if c < 0:
                break
            n = c
        to_node[cls] = n
    return code_of, to_node


def prim_classes(nodes: np.ndarray, prim_index: np.ndarray, root: int, width: int) -> np.ndarray:
    """Class of the leaf holding each primitive."""
    code_of, _ = leaf_codes(nodes, root, width)
    out = np.full(len(prim_index), -1, np.int64)
    for i, code in code_of.items():
        n = nodes[i]
        out[prim_index[n["first"]:n["first"] + n["count"]]] = code
    return out
