"""Pins of the oracle's brick classifier (R3, R4, Sec. 3.1) and compaction:
brute-force point sampling on tiny volumes and library reductions."""
import numpy as np
import pytest

from paper_1912_09596_gb300 import synth


def _cases():
    yield "u8", synth.random_u8((13, 11, 9), seed=1, p_zero=0.9), (0, 255), \
        synth.tf_random_sparse(256, seed=2, p_zero=0.8)
    yield "u8_ramp", synth.blobs_u8((20, 18, 16), n_blobs=4, seed=5), (0, 255), synth.tf_ramp(256, 40)
    rng = np.random.default_rng(3)
    f = np.where(rng.random((10, 12, 14)) < 0.85, 0.0, rng.uniform(0, 1, (10, 12, 14)))
    yield "f32", f.astype(np.float32), (0.0, 1.0), synth.tf_random_sparse(1024, seed=6, p_zero=0.9)
    u = np.where(rng.random((9, 10, 11)) < 0.8, 0, rng.integers(0, 65536, (9, 10, 11)))
    yield "u16", u.astype(np.uint16), (0, 65535), synth.tf_random_sparse(300, seed=8, p_zero=0.9)
    # large magnitudes with a narrow TF window: one ulp spans many TF entries
    g = (1.0e6 + rng.integers(0, 4, (8, 8, 8)) * 0.0625).astype(np.float32)
    yield "f32_narrow", g, (1.0e6, 1.0e6 + 0.25), synth.tf_random_sparse(64, seed=9, p_zero=0.9)


def _points(dims, rng):
    nx, ny, nz = dims
    n = np.array(dims, dtype=np.float64)
    lat = np.stack(np.meshgrid(np.arange(nx + 1), np.arange(ny + 1),
                               np.arange(nz + 1), indexing="ij"), -1).reshape(-1, 3)
    half = lat + 0.5
    rnd = rng.uniform(-0.4, 1.0, size=(4000, 3)) * (n + 0.8)
    near = np.round(rng.uniform(0, 1, size=(2000, 3)) * n) + rng.uniform(-0.49, 0.49, (2000, 3))
    return np.concatenate([lat, half, rnd, near]).astype(np.float32)


@pytest.mark.parametrize("case", list(_cases()), ids=lambda c: c[0])
@pytest.mark.parametrize("B", [2, 4, 8])
def test_mask_is_conservative_brute_force(ora, case, B):
    """R3 + R4: any point whose classified alpha is > 0 lies only in
    non-empty bricks, even after dilating each brick's closed region by just
    under half a voxel (the margin the skipping renderer relies on)."""
    name, v, (lo, hi), tf = case
    vol, otf = ora.OVolume(v, lo, hi), ora.OTF(tf)
    gx, gy, gz = vol.grid(B)
    mask = ora.build_mask(vol, otf, B).reshape(gz, gy, gx)
    cells = ora.brick_mask_cells(vol, B, otf).reshape(gz, gy, gx)
    rng = np.random.default_rng(B)
    n = np.array(vol.dims)
    hits = 0
    for p in _points(vol.dims, rng):
        a = ora.point_rgba(vol, otf, p)[3]
        if not a > 0:
            continue
        hits += 1
        rng_b = []
        for ax in range(3):
            g = (gx, gy, gz)[ax]
            bs = [b for b in range(g)
                  if b * B - 0.5 < p[ax] < min((b + 1) * B, n[ax]) + 0.5]
            rng_b.append(bs)
        for bz in rng_b[2]:
            for by in rng_b[1]:
                for bx in rng_b[0]:
                    assert mask[bz, by, bx] == 1, (name, p, (bx, by, bz))
                    assert cells[bz, by, bx] == 1, (name, p, (bx, by, bz))
    assert hits > 0


@pytest.mark.parametrize("case", list(_cases()), ids=lambda c: c[0])
def test_cell_mask_within_minmax_mask(ora, case):
    """The per-cell test is at least as tight as the brick min/max test."""
    name, v, (lo, hi), tf = case
    vol, otf = ora.OVolume(v, lo, hi), ora.OTF(tf)
    for B in (2, 4, 8):
        mm = ora.build_mask(vol, otf, B)
        cm = ora.brick_mask_cells(vol, B, otf)
        assert np.all(cm <= mm)


@pytest.mark.parametrize("case", list(_cases()), ids=lambda c: c[0])
def test_cell_mask_equals_minmax_mask(ora, case):
    """...and in fact equal to it: the cells touching a brick cover its apron
    voxels, neighbouring cells share corner voxels, and the TF index interval
    of a range is monotone in its ends, so the cells' intervals overlap in a
    chain whose union is the brick's own interval; a non-zero entry of that
    interval lies in some cell's.  A cell range that starts one cell late
    (no cell c = bB - 1) makes the masks differ on most of these volumes and
    brick sizes."""
    name, v, (lo, hi), tf = case
    vol, otf = ora.OVolume(v, lo, hi), ora.OTF(tf)
    for B in (2, 3, 4, 5, 8):
        mm = ora.build_mask(vol, otf, B)
        cm = ora.brick_mask_cells(vol, B, otf)
        assert np.array_equal(cm, mm), (name, B)


@pytest.mark.parametrize("dtype", ["u8", "f32"])
@pytest.mark.parametrize("B", [3, 4, 8])
def test_minmax_matches_numpy(ora, dtype, B):
    """Brick min/max over the clamped apron range [bB-1, (b+1)B] (R3)."""
    rng = np.random.default_rng(B)
    shape = (11, 13, 10)
    v = (rng.integers(0, 256, shape).astype(np.uint8) if dtype == "u8"
         else rng.standard_normal(shape).astype(np.float32))
    vol = ora.OVolume(v, 0, 255)
    mn, mx = ora.brick_minmax(vol, B)
    gx, gy, gz = vol.grid(B)
    k = 0
    for bz in range(gz):
        for by in range(gy):
            for bx in range(gx):
                sl = v[max(0, bz * B - 1):min(shape[0], (bz + 1) * B + 1),
                       max(0, by * B - 1):min(shape[1], (by + 1) * B + 1),
                       max(0, bx * B - 1):min(shape[2], (bx + 1) * B + 1)]
                assert mn[k] == sl.min() and mx[k] == sl.max()
                k += 1


def test_mask_ramp_tf_exact_cases(ora):
    """u8, NT = 256, alpha 0 below 40: a brick whose apron stays below 39 is
    empty, one that reaches 40 is not."""
    tf = ora.OTF(synth.tf_ramp(256, 40))
    mn = np.array([0, 0, 10, 39, 40, 200], dtype=np.float32)
    mx = np.array([0, 38, 38, 39, 40, 255], dtype=np.float32)
    m = ora.brick_mask(mn, mx, tf, 0, 255)
    assert m.tolist() == [0, 0, 0, 1, 1, 1]


def test_compaction_is_sorted_nonzero(ora):
    rng = np.random.default_rng(0)
    for n in (0, 1, 7, 1000):
        m = (rng.random(n) < 0.3).astype(np.uint8)
        assert np.array_equal(ora.compact(m), np.flatnonzero(m).astype(np.uint32))


def test_lerp_never_leaves_corner_range(ora):
    """The lemma behind R4: a trilinear sample lies within [min, max] of its
    8 corner values, for mixed signs and magnitudes and f close to 1."""
    rng = np.random.default_rng(11)
    for it in range(40):
        v = (rng.uniform(-1, 1, (2, 2, 2)) * 10.0 ** rng.integers(-6, 7, (2, 2, 2))).astype(np.float32)
        vol = ora.OVolume(v, 0, 1)
        lo, hi = float(v.min()), float(v.max())
        fs = np.concatenate([rng.uniform(0, 1, 60), 1 - 2.0 ** -np.arange(18, 25)])
        for fx in fs[::3]:
            for fy in fs[1::5]:
                fz = fs[(it * 7) % len(fs)]
                p = np.float32([0.5 + fx, 0.5 + fy, 0.5 + fz])
                val = ora.sample_value(vol, p)
                assert lo <= val <= hi
