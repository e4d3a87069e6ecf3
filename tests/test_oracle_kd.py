"""Pins of the oracle's k-d tree builder (Sec. 3.2, Sec. 4.3, R9): validity
invariants, a per-node brute-force check of the greedy choice, and the Table 1
entry "Menger Sponge, Shallow: 1 node, height 1".

The greedy topology itself has no printed value to compare with (Table 1 needs
the paper's data sets), so beyond these properties it is parity-unpinned."""
import numpy as np
import pytest

from paper_1912_09596_gb300 import synth


def vol_of(box, B, dims):
    v = 1
    for a in range(3):
        v *= min(box[3 + a] * B, dims[a]) - box[a] * B
    return v


def tight(m3, lo):
    """Tight brick box of the True cells of m3 (z, y, x) offset by lo (x, y, z)."""
    if not m3.any():
        return None
    out = []
    for a, axes in ((0, (0, 1)), (1, (0, 2)), (2, (1, 2))):
        proj = m3.any(axis=axes)
        idx = np.flatnonzero(proj)
        out.append((lo[a] + idx[0], lo[a] + idx[-1] + 1))
    return [out[0][0], out[1][0], out[2][0], out[0][1], out[1][1], out[2][1]]


def sub(mask3, box):
    return mask3[box[2]:box[5], box[1]:box[4], box[0]:box[3]]


def split_costs(mask3, box, B, dims, nbins):
    """All candidate (cost, axis, plane) of a node by direct enumeration."""
    res = []
    M = sub(mask3, box)
    for a in range(3):
        e = box[3 + a] - box[a]
        if e < 2:
            continue
        if nbins == 0:
            planes = list(range(box[a] + 1, box[3 + a]))
        else:
            planes = []
            for j in range(1, nbins):
                p = box[a] + (j * e) // nbins
                if box[a] < p < box[3 + a] and p not in planes:
                    planes.append(p)
        for p in planes:
            k = p - box[a]
            ax = 2 - a  # numpy axis of brick axis a
            L = np.take(M, np.arange(0, k), axis=ax)
            R = np.take(M, np.arange(k, e), axis=ax)
            lo_r = list(box[:3])
            lo_r[a] = p
            tl, tr = tight(L, box[:3]), tight(R, lo_r)
            if tl is None or tr is None:
                continue
            res.append((vol_of(tl, B, dims) + vol_of(tr, B, dims), a, p, tl, tr))
    return res


def check_tree(nodes, mask, grid, B, dims, nbins, halting, mls):
    gx, gy, gz = grid
    mask3 = mask.reshape(gz, gy, gx).astype(bool)
    if not mask3.any():
        assert len(nodes) == 0
        return
    root = tight(mask3, [0, 0, 0])
    assert nodes[0, :6].tolist() == root
    vroot = vol_of(root, B, dims)
    m = len(nodes)
    seen_child = np.zeros(m, dtype=int)
    last_child = 0
    for i in range(m):
        box = nodes[i, :6].tolist()
        axis, plane, fc = nodes[i, 6:9].tolist()
        assert tight(sub(mask3, box), box[:3]) == box, "node box not tight"
        V = vol_of(box, B, dims)
        allowed = (10 * V > vroot) if halting == 0 else (V > 512)
        cands = split_costs(mask3, box, B, dims, nbins) if allowed else []
        best = min(cands, key=lambda c: (c[0], c[1], c[2])) if cands else None
        if fc < 0:
            # leaf: halting stopped it, or no candidate beats V(X) and the
            # maximum leaf size does not force a middle split
            assert (not allowed) or ((best is None or best[0] >= V) and
                                     not (mls > 0 and V > mls ** 3 and
                                          any(box[3 + a] - box[a] >= 2 for a in range(3))))
            continue
        assert allowed
        assert fc > i and fc >= last_child and fc + 1 < m
        last_child = fc + 2
        seen_child[fc] += 1
        seen_child[fc + 1] += 1
        if best is not None and best[0] < V:
            assert (axis, plane) == (best[1], best[2]), "not the cheapest split"
        else:
            assert mls > 0 and V > mls ** 3
            exts = [(min(box[3 + a] * B, dims[a]) - box[a] * B if box[3 + a] - box[a] >= 2 else -1, -a)
                    for a in range(3)]
            a = -max(exts)[1]
            assert axis == a and plane == box[a] + (box[3 + a] - box[a]) // 2
        L, R = nodes[fc, :6].tolist(), nodes[fc + 1, :6].tolist()
        assert L[3 + axis] <= plane <= R[axis]
        for C in (L, R):
            assert all(C[a] >= box[a] and C[3 + a] <= box[3 + a] for a in range(3))
        lo_r = list(box[:3])
        lo_r[axis] = plane
        k = plane - box[axis]
        M = sub(mask3, box)
        assert L == tight(np.take(M, np.arange(0, k), axis=2 - axis), box[:3])
        assert R == tight(np.take(M, np.arange(k, box[3 + axis] - box[axis]), axis=2 - axis), lo_r)
    assert seen_child[0] == 0 and np.all(seen_child[1:] == 1)
    # leaves partition the non-empty bricks: each covered by exactly one leaf
    leaves = nodes[nodes[:, 8] < 0]
    cover = np.zeros(mask3.shape, dtype=int)
    for lf in leaves:
        cover[lf[2]:lf[5], lf[1]:lf[4], lf[0]:lf[3]] += 1
    assert np.all(cover[mask3] == 1)
    assert m % 2 == 1          # full binary tree: all k-d counts of Table 1 are odd


def _masks():
    rng = np.random.default_rng(0)
    for s in range(8):
        grid = tuple(int(x) for x in rng.integers(1, 9, 3))
        p = rng.uniform(0.02, 0.7)
        yield "rand%d" % s, (rng.random(int(np.prod(grid))) < p).astype(np.uint8), grid
    # two clusters far apart, one voxel-thin plane of bricks
    g = (12, 10, 9)
    m = np.zeros(g[::-1], np.uint8)
    m[1:3, 1:4, 1:3] = 1
    m[6:9, 6:10, 8:12] = 1
    m[4, :, :] = 1
    yield "clusters", m.ravel(), g
    yield "empty", np.zeros(27, np.uint8), (3, 3, 3)
    one = np.zeros(64, np.uint8)
    one[37] = 1
    yield "single", one, (4, 4, 4)


@pytest.mark.parametrize("case", list(_masks()), ids=lambda c: c[0])
@pytest.mark.parametrize("nbins", [0, 4])
@pytest.mark.parametrize("halting,mls", [(0, 0), (1, 0), (1, 16), (1, 32)])
@pytest.mark.parametrize("B", [4, 8])
def test_kd_definition_brute_force(ora, case, nbins, halting, mls, B):
    name, mask, grid = case
    dims = tuple(g * B - (1 if g > 1 else 0) for g in grid)   # partial last bricks
    nodes = ora.kd_build(mask, grid, B, dims, nbins=nbins, halting=halting, mls=mls)
    check_tree(nodes, mask, grid, B, dims, nbins, halting, mls)


@pytest.mark.parametrize("nbins", [0, 4])
@pytest.mark.parametrize("halting", [0, 1])
@pytest.mark.parametrize("n,B", [(81, 8), (81, 4), (243, 8)])
def test_menger_sponge_is_one_node(ora, nbins, halting, n, B):
    """Table 1: the Menger sponge's Shallow tree is a single node (height 1),
    for both the CPU (exhaustive) and the GPU (4 bins) builders.  The sponge
    keeps its 12 cube edges solid, so every plane leaves tight boxes that
    span the full extent and no split lowers the cost."""
    v = synth.menger_u8(n)
    vol = ora.OVolume(v, 0, 255)
    otf = ora.OTF(synth.tf_ramp(256, 100))
    mask = ora.build_mask(vol, otf, B)
    assert 0 < mask.sum() < mask.size
    nodes = ora.kd_build(mask, vol.grid(B), B, vol.dims, nbins=nbins, halting=halting, mls=0)
    assert len(nodes) == 1 and nodes[0, 8] == -1


def test_menger_sponge_max_leaf_size_splits(ora):
    """With a maximum leaf size the same sponge is split (Sec. 4.3): every
    leaf is at most mls^3 or can no longer be split."""
    v = synth.menger_u8(81)
    vol = ora.OVolume(v, 0, 255)
    otf = ora.OTF(synth.tf_ramp(256, 100))
    mask = ora.build_mask(vol, otf, 4)
    nodes = ora.kd_build(mask, vol.grid(4), 4, vol.dims, nbins=4, halting=1, mls=16)
    assert len(nodes) > 1
    check_tree(nodes, mask, vol.grid(4), 4, vol.dims, 4, 1, 16)


def test_shallow_halting_is_strict(ora):
    """Shallow halting splits only nodes *above* 10 % of the root volume: this
    mask yields a node of exactly 10 % whose cheapest split would lower the
    cost, and it stays a leaf."""
    grid, B = (6, 1, 10), 4
    dims = tuple(g * B for g in grid)
    mask = np.zeros(60, np.uint8)
    mask[[0, 7, 15, 16, 26, 29, 43, 45, 49, 54, 57]] = 1
    nodes = ora.kd_build(mask, grid, B, dims, nbins=0, halting=0)
    vroot = vol_of(nodes[0, :6].tolist(), B, dims)
    eq = [i for i in range(len(nodes)) if 10 * vol_of(nodes[i, :6].tolist(), B, dims) == vroot]
    assert eq and all(nodes[i, 8] == -1 for i in eq)
    check_tree(nodes, mask, grid, B, dims, 0, 0, 0)


@pytest.mark.parametrize("nbins", [0, 4])
def test_two_clusters_split_in_the_gap_by_hand(ora, nbins):
    """A hand-derived tree (R9, Sec. 3.2.1): two 2x2x2-brick clusters in
    opposite corners of an 8^3-brick grid.  Every plane inside the gap, on
    any axis, gives the two clusters' boxes as L and R (the least cost), so
    the tie rule picks axis x and the lowest such plane, 2 (a candidate with
    and without 4 bins).  A full 2x2x2 cube cannot lower its cost by any
    split (V(L) + V(R) = V), so both children are leaves: 3 nodes."""
    g = 8
    mask = np.zeros((g, g, g), dtype=np.uint8)       # [z][y][x]
    mask[:2, :2, :2] = 1
    mask[6:, 6:, 6:] = 1
    B = 8
    nodes = ora.kd_build(mask.reshape(-1), (g, g, g), B, (g * B,) * 3, nbins=nbins, halting=1, mls=0)
    want = np.array([[0, 0, 0, 8, 8, 8, 0, 2, 1],
                     [0, 0, 0, 2, 2, 2, -1, 0, -1],
                     [6, 6, 6, 8, 8, 8, -1, 0, -1]], dtype=np.int32)
    assert np.array_equal(nodes, want)


@pytest.mark.parametrize("nbins", [0, 4])
def test_full_cube_max_leaf_size_by_hand(ora, nbins):
    """A hand-derived tree for the maximum leaf size (Sec. 4.3, R9): a full
    8^3-brick cube (64^3 voxels) never lowers its cost by a split (L and R
    always fill V), so only the MLS 32 rule splits it: in the middle of the
    longest axis, the lower axis on ties, until the 32^3-voxel octants."""
    g, B = 8, 8
    mask = np.ones((g, g, g), dtype=np.uint8)
    nodes = ora.kd_build(mask.reshape(-1), (g, g, g), B, (g * B,) * 3, nbins=nbins, halting=1, mls=32)
    want = [[0, 0, 0, 8, 8, 8, 0, 4, 1],
            [0, 0, 0, 4, 8, 8, 1, 4, 3], [4, 0, 0, 8, 8, 8, 1, 4, 5],
            [0, 0, 0, 4, 4, 8, 2, 4, 7], [0, 4, 0, 4, 8, 8, 2, 4, 9],
            [4, 0, 0, 8, 4, 8, 2, 4, 11], [4, 4, 0, 8, 8, 8, 2, 4, 13]]
    for lo in [(0, 0, 0), (0, 0, 4), (0, 4, 0), (0, 4, 4), (4, 0, 0), (4, 0, 4), (4, 4, 0), (4, 4, 4)]:
        want.append([lo[0], lo[1], lo[2], lo[0] + 4, lo[1] + 4, lo[2] + 4, -1, 0, -1])
    assert np.array_equal(nodes, np.array(want, dtype=np.int32))
    # without the maximum leaf size the cube stays one leaf
    one = ora.kd_build(mask.reshape(-1), (g, g, g), B, (g * B,) * 3, nbins=nbins, halting=1, mls=0)
    assert np.array_equal(one, np.array([[0, 0, 0, 8, 8, 8, -1, 0, -1]], dtype=np.int32))
