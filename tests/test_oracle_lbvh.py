"""Pins of the oracle's Morton codes, sort and LBVH (Sec. 3.1, R8, R10)."""
import math
import os

import numpy as np
import pytest

from paper_1912_09596_gb300 import synth

GOLD = os.path.join(os.path.dirname(__file__), "golden", "table1_lbvh.txt")


def _table1():
    rows = []
    for line in open(GOLD):
        if line.startswith("#") or not line.strip():
            continue
        f = line.split()
        rows.append(dict(name=f[0], dims=tuple(int(x) for x in f[1:4]), nodes=int(f[4]),
                         height=int(f[5]), garbled=len(f) > 6))
    return rows


def height_bound(grid):
    """Levels of a binary radix tree over 30-bit Morton codes of bricks with
    coordinates < g_a: one level per distinct key bit, plus the leaves."""
    return sum(int(math.ceil(math.log2(g))) if g > 1 else 0 for g in grid) + 1


def tree_height(left, right):
    if len(left) == 0:
        return 1
    h, stack = 0, [(0, 1)]
    while stack:
        node, d = stack.pop()
        for c in (left[node], right[node]):
            if c < 0:
                h = max(h, d + 1)
            else:
                stack.append((c, d + 1))
    return h


# ----------------------------------------------------------------- R10 Morton
def test_morton_vectors(ora):
    assert ora.morton30(1, 0, 0) == 1
    assert ora.morton30(0, 1, 0) == 2
    assert ora.morton30(0, 0, 1) == 4
    assert ora.morton30(1023, 1023, 1023) == 2 ** 30 - 1
    assert ora.morton30(2, 0, 0) == 8
    assert ora.morton30(0, 0, 512) == 1 << 29
    assert ora.morton30(3, 5, 6) == 0b110101011   # z2y2x2 z1y1x1 z0y0x0


def test_morton_keys_from_brick_ids(ora):
    gx, gy = 5, 7
    ids = np.array([0, 1, 5, 35, 36 + 5 + 1], dtype=np.uint32)
    keys = ora.morton_keys(ids, gx, gy)
    ref = [ora.morton30(int(b) % gx, (int(b) // gx) % gy, int(b) // (gx * gy)) for b in ids]
    assert keys.tolist() == ref


def test_sort_matches_numpy(ora):
    rng = np.random.default_rng(0)
    keys = rng.permutation(1 << 20)[:5000].astype(np.uint32)
    ids = np.arange(5000, dtype=np.uint32)
    k, v = ora.sort_pairs(keys, ids)
    order = np.argsort(keys, kind="stable")
    assert np.array_equal(k, keys[order]) and np.array_equal(v, ids[order])


# ------------------------------------------------------------------ topology
def _random_sorted_keys(rng, n, bits=30):
    return np.sort(rng.choice(1 << bits, size=n, replace=False)).astype(np.uint32)


@pytest.mark.parametrize("n", [2, 3, 4, 5, 17, 100, 1000, 4097])
def test_topdown_equals_karras(ora, n):
    """Two independent constructions of the radix tree (recursive split at the
    highest differing bit, and Karras' per-node search) agree exactly."""
    rng = np.random.default_rng(n)
    for bits in (30, 12):
        if n > (1 << bits):
            continue
        k = _random_sorted_keys(rng, n, bits)
        l1, r1, _ = ora.lbvh_topdown(k)
        l2, r2 = ora.lbvh_karras(k)
        assert np.array_equal(l1, l2) and np.array_equal(r1, r2)


@pytest.mark.parametrize("n", [2, 3, 9, 500])
def test_radix_tree_shape(ora, n):
    """n leaves, n - 1 inner nodes (2n - 1 in all); each node except the root
    is some node's child exactly once; every range splits at its top bit."""
    rng = np.random.default_rng(100 + n)
    k = _random_sorted_keys(rng, n)
    left, right, ranges = ora.lbvh_topdown(k)
    kids = np.concatenate([left, right])
    inner = np.sort(kids[kids >= 0])
    leaves = np.sort(-1 - kids[kids < 0])
    assert np.array_equal(inner, np.arange(1, n - 1))
    assert np.array_equal(leaves, np.arange(n))
    for i in range(n - 1):
        f, l = ranges[i]
        bit = 31 - (32 - int(k[f] ^ k[l]).bit_length())
        lk = ranges[left[i]] if left[i] >= 0 else (-1 - left[i],) * 2
        rk = ranges[right[i]] if right[i] >= 0 else (-1 - right[i],) * 2
        assert lk[0] == f and rk[1] == l and lk[1] + 1 == rk[0]
        assert all(((int(k[j]) >> bit) & 1) == 0 for j in range(lk[0], lk[1] + 1))
        assert all(((int(k[j]) >> bit) & 1) == 1 for j in range(rk[0], rk[1] + 1))


def test_table1_heights_obey_bound():
    """Table 1's LBVH heights never exceed (sum of Morton bits) + 1 and reach it
    for 10 of 11 data sets: this fixes the paper's height convention (levels,
    root and leaves included) used by the tests below.  Node counts are odd
    (2n - 1) except the row flagged as garbled."""
    rows = _table1()
    reached = 0
    for r in rows:
        grid = [-(-d // 8) for d in r["dims"]]
        assert r["height"] <= height_bound(grid), r
        reached += r["height"] == height_bound(grid)
        if not r["garbled"]:
            assert r["nodes"] % 2 == 1
    assert reached == 10


@pytest.mark.parametrize("g", [2, 4, 8, 16])
def test_full_occupancy_complete_tree(ora, g):
    """All g^3 bricks non-empty, g a power of two: the radix tree is complete,
    2 g^3 - 1 nodes and height 3 log2 g + 1 (the bound is attained)."""
    mask = np.ones(g ** 3, dtype=np.uint8)
    t = ora.lbvh_build(mask, (g, g, g))
    n = len(t["sorted_keys"])
    assert n == g ** 3 and len(t["left"]) == n - 1
    assert tree_height(t["left"], t["right"]) == 3 * int(math.log2(g)) + 1


@pytest.mark.parametrize("seed", range(6))
def test_lbvh_boxes_contain_and_separate(ora, seed):
    """Parent boxes contain child boxes; the two children of an inner node are
    separated by a plane on axis (top bit mod 3) (R8); the height obeys the
    Table 1 bound."""
    rng = np.random.default_rng(seed)
    grid = tuple(int(x) for x in rng.integers(2, 12, 3))
    mask = (rng.random(int(np.prod(grid))) < rng.uniform(0.05, 0.6)).astype(np.uint8)
    if mask.sum() < 2:
        mask[:2] = 1
    t = ora.lbvh_build(mask, grid)
    gx, gy, _ = grid
    left, right, boxes, sids, keys = t["left"], t["right"], t["boxes"], t["sorted_ids"], t["sorted_keys"]

    def box(c):
        if c >= 0:
            return boxes[c]
        b = int(sids[-1 - c])
        lo = np.array([b % gx, (b // gx) % gy, b // (gx * gy)])
        return np.concatenate([lo, lo + 1])

    for i in range(len(left)):
        P, L, R = box(i), box(left[i]), box(right[i])
        for C in (L, R):
            assert np.all(C[:3] >= P[:3]) and np.all(C[3:] <= P[3:])
        f, l = t["ranges"][i]
        bit = int(keys[f] ^ keys[l]).bit_length() - 1
        ax = bit % 3
        assert L[3 + ax] <= R[ax]
    assert tree_height(left, right) <= height_bound(grid)


def test_lbvh_single_and_empty(ora):
    t = ora.lbvh_build(np.zeros(27, np.uint8), (3, 3, 3))
    assert len(t["sorted_ids"]) == 0 and len(t["left"]) == 0
    m = np.zeros(27, np.uint8)
    m[13] = 1
    t = ora.lbvh_build(m, (3, 3, 3))
    assert t["sorted_ids"].tolist() == [13] and len(t["left"]) == 0
