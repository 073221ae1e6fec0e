"""Pins for the oracle's ray hash (Sec. 5) and table index.

Pinned against: hand-worked values (tests/golden), and properties the paper's
definition fixes (bit budget 1 + 2p, sign in the top bit, kept vs dropped bits,
binade aliasing of the exponent's top bits, XOR swizzle of origin and
direction).  The 48-bit mixer is pinned by an independent inverse.
"""
import os
import struct

import numpy as np
import pytest

import oracle as O

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _bits(f):
    return struct.unpack("<I", struct.pack("<f", f))[0]


def _float(b):
    return struct.unpack("<f", struct.pack("<I", b & 0xFFFFFFFF))[0]


def _rows(name):
    with open(os.path.join(GOLDEN, name)) as fh:
        return [ln.split() for ln in fh if ln.strip() and not ln.startswith("#")]


def test_hash_worked_values():
    rows = _rows("hash_worked_values.txt")
    assert len(rows) == 7
    for row in rows:
        f = float(row[0])
        assert _bits(f) == int(row[1], 16), row
        for p in range(1, 8):
            assert O.hash_float(f, p) == int(row[1 + p]), (row, p)


def test_hash_exponent_lsb_variant_worked_values():
    """The tuning variant that keeps the exponent's least significant bits."""
    rows = _rows("hash_lsb_worked_values.txt")
    assert len(rows) == 6
    for row in rows:
        f = float(row[0])
        assert _bits(f) == int(row[1], 16), row
        for p in range(1, 8):
            assert O.hash_float_variant(f, p, O.HASH_EXP_LSB) == int(row[1 + p]), (row, p)
            assert O.hash_float_variant(f, p, O.HASH_EXP_MSB) == O.hash_float(f, p)


def test_hash_variants_split_binades_differently():
    """The Sec. 5 hash aliases neighbouring binades (1.0, 0.5, 0.25 share
    their top exponent bits); the LSB variant separates them but aliases
    binades 2^p apart instead."""
    p = 3
    msb = [O.hash_float(2.0 ** -k, p) for k in range(4)]
    lsb = [O.hash_float_variant(2.0 ** -k, p, O.HASH_EXP_LSB) for k in range(4)]
    assert len(set(msb)) == 1 and len(set(lsb)) == 4
    assert O.hash_float_variant(1.0, p, O.HASH_EXP_LSB) == O.hash_float_variant(2.0 ** -8, p, O.HASH_EXP_LSB)
    ray = [1.0, 0.5, 0.25, 0.0, 0.6, -0.8, 0.0, 1.0]
    assert O.ray_key(ray, p, O.HASH_EXP_LSB) != O.ray_key(ray, p)
    assert O.ray_key(ray, p, O.HASH_EXP_MSB) == O.ray_key(ray, p)


def test_ray_key_worked_values():
    for row in _rows("ray_key_worked_values.txt"):
        ox, oy, oz, dx, dy, dz = map(float, row[:6])
        p = int(row[6])
        ray = [ox, oy, oz, 0.0, dx, dy, dz, 1.0]
        assert O.ray_key(ray, p) == int(row[7], 16)


@pytest.mark.parametrize("p", range(1, 8))
def test_hash_bit_budget_and_sign(p):
    rng = np.random.default_rng(p)
    for b in rng.integers(0, 2**32, 2000, dtype=np.uint64):
        b = int(b)
        f = _float(b)
        h = O.hash_float(f, p)
        assert h < (1 << (1 + 2 * p))
        # the sign is the top bit of the 1+2p
        assert (h >> (2 * p)) == (b >> 31)
    # every kept bit set -> all 1+2p bits set
    assert O.hash_float(_float(0xFFFFFFFF), p) == (1 << (1 + 2 * p)) - 1


@pytest.mark.parametrize("p", range(1, 8))
def test_hash_keeps_msbs_and_drops_the_rest(p):
    """Flipping a dropped bit never changes h; flipping a kept bit always does."""
    kept = {31} | {30 - i for i in range(p)} | {22 - i for i in range(p)}
    rng = np.random.default_rng(100 + p)
    for b in rng.integers(0, 2**32, 300, dtype=np.uint64):
        b = int(b)
        h = O.hash_float(_float(b), p)
        for bit in range(32):
            flipped = b ^ (1 << bit)
            if (flipped >> 23) & 0xFF == 0xFF or (b >> 23) & 0xFF == 0xFF:
                continue  # keep clear of NaN payload canonicalisation in ctypes
            h2 = O.hash_float(_float(flipped), p)
            if bit in kept:
                assert h2 != h, (hex(b), bit)
            else:
                assert h2 == h, (hex(b), bit)


def test_hash_aliases_binades_through_exponent_msbs():
    # 1.0, 0.5, 0.25, 0.125 have exponents 127..124: equal top 6 bits
    for p in range(1, 7):
        assert O.hash_float(1.0, p) == O.hash_float(0.5, p) == O.hash_float(0.25, p) == O.hash_float(0.125, p)
    assert O.hash_float(1.0, 7) == O.hash_float(0.5, 7)
    assert O.hash_float(1.0, 7) != O.hash_float(0.25, 7)
    assert O.hash_float(0.0, 3) != O.hash_float(-0.0, 3)


@pytest.mark.parametrize("p", [2, 6])
def test_hash_monotone_within_binade(p):
    xs = np.sort(np.random.default_rng(p).uniform(1.0, 2.0, 500).astype(np.float32))
    hs = [O.hash_float(float(x), p) for x in xs]
    assert all(a <= b for a, b in zip(hs, hs[1:]))
    # exactly 2^p distinct values over a binade
    grid = [1.0 + k / 2**p for k in range(2**p)]
    assert len({O.hash_float(g, p) for g in grid}) == 2**p


def test_key_swizzle_pairs():
    """Sec. 5 pairs o_x with d_z, o_y with d_y and o_z with d_x by XOR."""
    rng = np.random.default_rng(7)
    for _ in range(200):
        o = rng.normal(size=3).astype(np.float32)
        d = rng.normal(size=3).astype(np.float32)
        ray = np.array([o[0], o[1], o[2], 0, d[0], d[1], d[2], 1], np.float32)
        k = O.ray_key(ray, 6)
        assert k < (1 << 48)
        # exchanging the members of a XOR pair leaves the key unchanged
        r2 = ray.copy(); r2[0], r2[6] = ray[6], ray[0]
        r3 = ray.copy(); r3[2], r3[4] = ray[4], ray[2]
        r4 = ray.copy(); r4[1], r4[5] = ray[5], ray[1]
        assert O.ray_key(r2, 6) == k and O.ray_key(r3, 6) == k and O.ray_key(r4, 6) == k
    # a ray whose swizzled pairs are equal has key 0
    ray = np.array([0.7, -3.0, 5.5, 0, 5.5, -3.0, 0.7, 1], np.float32)
    assert O.ray_key(ray, 6) == 0


def test_key_field_layout():
    # only o_x set (d = 0): h(o_x) lands in the low 16 bits
    for p in (2, 6, 7):
        h = O.hash_float(3.0, p)
        assert O.ray_key([3.0, 0, 0, 0, 0, 0, 0, 1], p) == h
        assert O.ray_key([0, 3.0, 0, 0, 0, 0, 0, 1], p) == h << 16
        assert O.ray_key([0, 0, 3.0, 0, 0, 0, 0, 1], p) == h << 32
        assert O.ray_key([0, 0, 0, 0, 3.0, 0, 0, 1], p) == h << 32   # d_x pairs with o_z
        assert O.ray_key([0, 0, 0, 0, 0, 0, 3.0, 1], p) == h         # d_z pairs with o_x


def _inv_xorshift(y, s, bits=48):
    x = y
    for _ in range(bits // s + 1):
        x = y ^ (x >> s)
    return x & ((1 << bits) - 1)


def _unmix48(m):
    M = (1 << 48) - 1
    m = _inv_xorshift(m, 21)
    m = (m * pow(0xC2B2AE3D27D5, -1, 1 << 48)) & M
    m = _inv_xorshift(m, 25)
    m = (m * pow(0x9E3779B97F4B, -1, 1 << 48)) & M
    m = _inv_xorshift(m, 23)
    return m


def test_mix48_is_a_bijection():
    rng = np.random.default_rng(3)
    keys = [int(k) for k in rng.integers(0, 1 << 48, 20000, dtype=np.uint64)] + list(range(256))
    for k in keys:
        m = O.mix48(k)
        assert m < (1 << 48)
        assert _unmix48(m) == k


def test_mix48_spreads_nearby_keys():
    # keys that differ in one low bit land in unrelated sets
    sets = [O.mix48(k) & 0xFFF for k in range(1 << 14)]
    counts = np.bincount(sets, minlength=4096)
    assert counts.max() <= 16  # 4 expected per set
    assert np.count_nonzero(counts) > 3900


def test_way_of_range():
    for lw in range(0, 4):
        ws = {O.way_of(leaf, lw) for leaf in range(0, 4096, 4)}
        assert ws == set(range(1 << lw))
