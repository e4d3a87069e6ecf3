"""GPU parity of the empty test, compaction, naive marcher and macrocell-grid
renderer against the CPU oracle, through the C ABI."""
import numpy as np
import pytest

from paper_1912_09596_gb300 import synth
from gpu_util import assert_image_parity, bits, render, upload

pytestmark = pytest.mark.gpu


def _volumes():
    yield "blobs64_u8", synth.blobs_u8((64, 64, 64), seed=0), (0, 255), synth.tf_ramp(256, 40)
    yield "ragged_u8", synth.blobs_u8((37, 29, 45), n_blobs=6, seed=4), (0, 255), \
        synth.tf_random_sparse(256, seed=5, p_zero=0.7)
    rng = np.random.default_rng(9)
    f = np.where(rng.random((33, 40, 27)) < 0.9, 0.0, rng.uniform(0, 1, (33, 40, 27)))
    yield "sparse_f32", f.astype(np.float32), (0.0, 1.0), synth.tf_random_sparse(1024, seed=6, p_zero=0.85)
    u = np.where(rng.random((30, 26, 34)) < 0.8, 0, rng.integers(0, 65536, (30, 26, 34)))
    yield "sparse_u16", u.astype(np.uint16), (0, 65535), synth.tf_random_sparse(700, seed=8, p_zero=0.8)


VOLS = list(_volumes())


@pytest.mark.parametrize("case", VOLS, ids=lambda c: c[0])
@pytest.mark.parametrize("B", [4, 8, 16, 32])
def test_minmax_mask_ids_bit_exact(gpu, ctx, ora, case, B):
    ess, torch = gpu
    name, v, (lo, hi), tf = case
    vol, t = upload(ess, torch, ctx, v, lo, hi, tf)
    ov, ot = ora.OVolume(v, lo, hi), ora.OTF(tf)
    for empty_test in (0, 1):
        st = ess.ess_build(ctx, vol, t, ess.GRID, ess.build_params(brick=B, empty_test=empty_test))
        mask = ess.ess_structure_read(ctx, st, ess.ARR_MASK)
        if empty_test == 0:
            mm = ess.ess_structure_read(ctx, st, ess.ARR_MINMAX).reshape(-1, 2)
            rmin, rmax = ora.brick_minmax(ov, B)
            assert np.array_equal(mm[:, 0], rmin) and np.array_equal(mm[:, 1], rmax)
            ref = ora.brick_mask(rmin, rmax, ot, lo, hi)
        else:
            ref = ora.brick_mask_cells(ov, B, ot)
        assert np.array_equal(mask, ref), (name, B, empty_test)
        ids = ess.ess_structure_read(ctx, st, ess.ARR_IDS)
        assert np.array_equal(ids, ora.compact(ref))
        info = ess.ess_structure_info_get(ctx, st)
        assert info["n_nonempty"] == int(ref.sum())
        assert (info["gx"], info["gy"], info["gz"]) == ov.grid(B)
        ess.ess_release(ctx, st)


def _vote_volumes():
    """Rows of whole bricks (nx a multiple of 8) but ragged in y and z, for the
    staged vote of 4^3 and 8^3 bricks: mostly-zero volumes whose few
    non-zero voxels decide the bricks, so a brick's first visible cell row
    can come in any of its rounds; the 96^3 case has more bricks than the
    kernel has warps, so that each warp takes several."""
    rng = np.random.default_rng(31)

    def sparse(shape, vals):
        return np.where(rng.random(shape) < 0.97, 0, vals(shape))

    yield "u8_40", sparse((19, 21, 40), lambda sh: rng.integers(1, 256, sh)).astype(np.uint8), \
        (0, 255), 256
    # rows of whole 16-byte blocks: the two-block row loads of 8-bit voxels
    yield "u8_48", sparse((19, 21, 48), lambda sh: rng.integers(1, 256, sh)).astype(np.uint8), \
        (0, 255), 256
    yield "u16_24", sparse((13, 30, 24), lambda sh: rng.integers(1, 65536, sh)).astype(np.uint16), \
        (0, 65535), 700
    yield "f32_16", sparse((22, 11, 16), lambda sh: rng.uniform(0, 1, sh)).astype(np.float32), \
        (0.0, 1.0), 1024
    yield "u8_96", synth.blobs_u8((96, 96, 96), n_blobs=12, seed=7), (0, 255), 256


@pytest.mark.parametrize("case", list(_vote_volumes()), ids=lambda c: c[0])
@pytest.mark.parametrize("B", [4, 8])
def test_vote_staged_bit_exact(gpu, ctx, ora, case, B):
    """The staged per-cell vote (rows of whole bricks) equals the oracle's per-cell
    mask bit for bit, under TFs whose first entries are transparent (cells of
    zeros are invisible) and under a TF that leaves them opaque."""
    ess, torch = gpu
    name, v, (lo, hi), nt = case
    ov = ora.OVolume(v, lo, hi)
    vol = ess.ess_volume_upload(ctx, torch.from_numpy(v).cuda(), lo, hi)
    for seed, clear_low in ((1, True), (2, True), (3, False)):
        tf = synth.tf_random_sparse(nt, seed=seed, p_zero=0.8)
        if clear_low:
            tf[:2, 3] = 0.0
        t = ess.ess_tf_set(ctx, torch.from_numpy(tf).cuda())
        ref = ora.brick_mask_cells(ov, B, ora.OTF(tf))
        st = ess.ess_build(ctx, vol, t, ess.GRID, ess.build_params(brick=B, empty_test=1))
        mask = ess.ess_structure_read(ctx, st, ess.ARR_MASK)
        assert np.array_equal(mask, ref), (name, B, seed)
        assert np.array_equal(ess.ess_structure_read(ctx, st, ess.ARR_IDS), ora.compact(ref))
        ess.ess_release(ctx, st)
        ess.ess_release(ctx, t)
    ess.ess_release(ctx, vol)


def _row_volumes():
    """Rows of whole 16-byte vectors, more than 32 vectors per row (two warps
    share a brick row) and, for the wide bricks, a ragged last brick in x."""
    rng = np.random.default_rng(21)
    yield "u8_528", rng.integers(0, 256, (19, 21, 528)).astype(np.uint8), (0, 255)
    yield "u16_264", rng.integers(0, 65536, (17, 23, 264)).astype(np.uint16), (0, 65535)
    yield "f32_136", rng.uniform(-3, 5, (18, 13, 136)).astype(np.float32), (-3.0, 5.0)
    yield "u8_64", synth.blobs_u8((9, 70, 64), n_blobs=5, seed=3), (0, 255)


@pytest.mark.parametrize("case", list(_row_volumes()), ids=lambda c: c[0])
@pytest.mark.parametrize("B", [2, 4, 8, 16, 32, 64, 6])
def test_minmax_vector_rows_and_rescan(gpu, ctx, ora, case, B):
    """The per-brick min/max over whole-vector rows, for every brick size
    (powers of two take the vectorised reduction, 6 the per-brick one), equals
    the oracle bit for bit, and recomputing it in every rebuild (rescan)
    gives the same min/max and mask."""
    ess, torch = gpu
    name, v, (lo, hi) = case
    tf = synth.tf_random_sparse(256, seed=B, p_zero=0.6)
    vol, t = upload(ess, torch, ctx, v, lo, hi, tf)
    ov, ot = ora.OVolume(v, lo, hi), ora.OTF(tf)
    rmin, rmax = ora.brick_minmax(ov, B)
    ref = ora.brick_mask(rmin, rmax, ot, lo, hi)
    for rescan in (1, 0, 1):
        st = ess.ess_build(ctx, vol, t, ess.GRID, ess.build_params(brick=B, rescan=rescan))
        ess.ess_tf_update(ctx, t, torch.from_numpy(tf).cuda())   # an edit: the pass runs again
        ess.ess_rebuild(ctx, st)
        mm = ess.ess_structure_read(ctx, st, ess.ARR_MINMAX).reshape(-1, 2)
        assert np.array_equal(bits(mm[:, 0]), bits(rmin)) and np.array_equal(bits(mm[:, 1]), bits(rmax))
        assert np.array_equal(ess.ess_structure_read(ctx, st, ess.ARR_MASK), ref)
        ess.ess_release(ctx, st)


@pytest.mark.parametrize("case", VOLS, ids=lambda c: c[0])
@pytest.mark.parametrize("ert", [2.0, 0.95])
def test_render_naive_and_grid_match_oracle(gpu, ctx, ora, case, ert):
    ess, torch = gpu
    name, v, (lo, hi), tf = case
    vol, t = upload(ess, torch, ctx, v, lo, hi, tf)
    ov, ot = ora.OVolume(v, lo, hi), ora.OTF(tf)
    rng = np.random.default_rng(len(name))
    naive = ess.ess_build(ctx, vol, t, ess.NONE)
    grids = {B: ess.ess_build(ctx, vol, t, ess.GRID, ess.build_params(brick=B)) for B in (4, 8, 16)}
    cams = [synth.random_camera(ov.dims, rng, ortho=False),
            synth.random_camera(ov.dims, rng, ortho=True),
            synth.axis_ortho_camera(ov.dims, axis=1)]
    for ci, cam in enumerate(cams):
        W, H = (53, 37) if ci == 0 else (40, 32)        # ragged tiles too
        ref, _ = ora.render_naive(ov, ot, cam, W, H, dt=0.5, ert=ert, bg=(0.1, 0.2, 0.3, 0.4))
        got = render(ess, torch, ctx, naive, cam, W, H, ert=ert, bg=(0.1, 0.2, 0.3, 0.4))
        assert_image_parity(got, ref, "%s naive cam%d" % (name, ci))
        for B, st in grids.items():
            g = render(ess, torch, ctx, st, cam, W, H, ert=ert, bg=(0.1, 0.2, 0.3, 0.4))
            assert_image_parity(g, ref, "%s grid B=%d cam%d" % (name, B, ci))
            assert np.array_equal(bits(g), bits(got)), "skipping changed the GPU image"


def test_grid_skips_samples(gpu, ctx, ora):
    ess, torch = gpu
    v = synth.blobs_u8((64, 64, 64), seed=0)
    vol, t = upload(ess, torch, ctx, v, 0, 255, synth.tf_ramp(256, 40))
    cam = synth.orbit_camera((64, 64, 64), 64, 64, 0.4)
    naive = ess.ess_build(ctx, vol, t, ess.NONE)
    grid = ess.ess_build(ctx, vol, t, ess.GRID, ess.build_params(brick=8))
    ess.ess_sample_count(ctx, reset=True)
    a = render(ess, torch, ctx, naive, cam, 64, 64)
    n_naive = ess.ess_sample_count(ctx, reset=True)
    b = render(ess, torch, ctx, grid, cam, 64, 64)
    n_grid = ess.ess_sample_count(ctx, reset=True)
    ov, ot = ora.OVolume(v, 0, 255), ora.OTF(synth.tf_ramp(256, 40))
    _, n_ref = ora.render_naive(ov, ot, cam, 64, 64)
    assert n_naive == n_ref
    assert 0 < n_grid < n_naive
    assert np.array_equal(bits(a), bits(b))


def test_empty_tf_and_tiny_volume(gpu, ctx, ora):
    ess, torch = gpu
    v = synth.random_u8((9, 7, 5), seed=1, p_zero=0.5)
    tf = synth.tf_random_sparse(256, seed=2)
    tf[:, 3] = 0.0
    vol, t = upload(ess, torch, ctx, v, 0, 255, tf, device=False)
    st = ess.ess_build(ctx, vol, t, ess.GRID, ess.build_params(brick=4))
    assert ess.ess_structure_info_get(ctx, st)["n_nonempty"] == 0
    cam = synth.orbit_camera((9, 7, 5), 16, 16, 1.0)
    img = render(ess, torch, ctx, st, cam, 16, 16, bg=(0.5, 0.25, 0.125, 1.0))
    assert np.all(img == np.float32([0.5, 0.25, 0.125, 1.0]))
    one = np.full((1, 1, 1), 200, np.uint8)
    vol1, t1 = upload(ess, torch, ctx, one, 0, 255, synth.tf_ramp(256, 40), device=False)
    st1 = ess.ess_build(ctx, vol1, t1, ess.GRID, ess.build_params(brick=2))
    cam1 = synth.orbit_camera((1, 1, 1), 8, 8, 0.2, dist=3.0)
    ov, ot = ora.OVolume(one, 0, 255), ora.OTF(synth.tf_ramp(256, 40))
    ref, _ = ora.render_naive(ov, ot, cam1, 8, 8)
    assert_image_parity(render(ess, torch, ctx, st1, cam1, 8, 8), ref, "1 voxel")


def test_tf_update_makes_structure_stale(gpu, ctx, ora):
    ess, torch = gpu
    v = synth.blobs_u8((32, 32, 32), n_blobs=4, seed=3)
    tf0, tf1 = synth.tf_ramp(256, 40), synth.tf_window(256, 120, 200)
    vol, t = upload(ess, torch, ctx, v, 0, 255, tf0)
    st = ess.ess_build(ctx, vol, t, ess.GRID, ess.build_params(brick=8))
    ess.ess_tf_update(ctx, t, tf1)                 # host table: staged copy
    cam = synth.orbit_camera((32, 32, 32), 24, 24, 0.9)
    with pytest.raises(ess.EssError) as e:
        render(ess, torch, ctx, st, cam, 24, 24)
    assert e.value.status == ess.ERR_STALE
    ess.ess_rebuild(ctx, st)
    ov = ora.OVolume(v, 0, 255)
    ref_mask = ora.build_mask(ov, ora.OTF(tf1), 8)
    assert np.array_equal(ess.ess_structure_read(ctx, st, ess.ARR_MASK), ref_mask)
    ref, _ = ora.render_naive(ov, ora.OTF(tf1), cam, 24, 24)
    assert_image_parity(render(ess, torch, ctx, st, cam, 24, 24), ref, "after rebuild")


def test_invalid_inputs_are_rejected(gpu, ctx):
    ess, torch = gpu
    bad = np.full((4, 4, 4), np.nan, dtype=np.float32)
    with pytest.raises(ess.EssError) as e:
        ess.ess_volume_upload(ctx, bad, 0.0, 1.0)
    assert e.value.status == ess.ERR_ARG
    with pytest.raises(ess.EssError):
        ess.ess_volume_upload(ctx, np.zeros((4, 4, 4), np.uint8), 1.0, 1.0)
    tf = np.zeros((16, 4), np.float32)
    tf[3, 3] = 1.5
    with pytest.raises(ess.EssError):
        ess.ess_tf_set(ctx, tf)
    vol = ess.ess_volume_upload(ctx, np.zeros((4, 4, 4), np.uint8), 0, 255)
    t = ess.ess_tf_set(ctx, np.zeros((16, 4), np.float32))
    with pytest.raises(ess.EssError):
        ess.ess_build(ctx, vol, t, ess.GRID, ess.build_params(brick=1))
    with pytest.raises(ess.EssError) as e:
        ess.ess_build(ctx, vol, 12345, ess.GRID)
    assert e.value.status == ess.ERR_HANDLE
    st = ess.ess_build(ctx, vol, t, ess.GRID, ess.build_params(brick=4))
    with pytest.raises(ess.EssError):
        ess.ess_release(ctx, vol)                  # still used by st
    ess.ess_release(ctx, st)
    ess.ess_release(ctx, vol)


@pytest.mark.parametrize("case", VOLS, ids=lambda c: c[0])
def test_dense_and_cell_samplers_agree(gpu, ctx, ora, case):
    """Dense voxel reads and the corner-replicated cell copy give the same
    bits, and both match the oracle."""
    ess, torch = gpu
    name, v, (lo, hi), tf = case
    vol, t = upload(ess, torch, ctx, v, lo, hi, tf)
    ov, ot = ora.OVolume(v, lo, hi), ora.OTF(tf)
    rng = np.random.default_rng(21)
    sts = [ess.ess_build(ctx, vol, t, k, ess.build_params(brick=8)) for k in ess.KINDS]
    for cam in (synth.random_camera(ov.dims, rng, ortho=False),
                synth.random_camera(ov.dims, rng, ortho=True)):
        ref, _ = ora.render_naive(ov, ot, cam, 45, 35, ert=0.97)
        imgs = []
        for cells in (1, 0, 1):
            ess.ess_volume_set_sampler(ctx, vol, cells)
            for st in sts:
                imgs.append(render(ess, torch, ctx, st, cam, 45, 35, ert=0.97))
        assert_image_parity(imgs[0], ref, name)
        for im in imgs[1:]:
            assert np.array_equal(bits(im), bits(imgs[0]))


def test_rescan_once_per_tf_edit(gpu, ctx, ora):
    """With rescan, the volume is read once per TF edit (Sec. 3.1 classifies
    after each edit), and the grid, LBVH and k-d rebuilt for that edit share
    the pass: one min/max launch per edit and brick size, none when nothing
    was edited, one more per further brick size; masks still equal the
    oracle's."""
    ess, torch = gpu
    v = synth.ct_like_u8((96, 80, 72), seed=2, n_vessels=5)
    tfs = synth.tf_set_ct()
    vol, t = upload(ess, torch, ctx, v, 0, 255, tfs[0])
    kd = dict(nbins=4, halting=1, mls=32)
    sts = [ess.ess_build(ctx, vol, t, k, ess.build_params(brick=8, rescan=1, **kd))
           for k in (ess.GRID, ess.LBVH, ess.KD)]
    other = ess.ess_build(ctx, vol, t, ess.GRID, ess.build_params(brick=16, rescan=1))
    ess.ess_sync(ctx)
    ess.ess_profile_reset(ctx)
    ess.ess_profile_enable(ctx, True)
    for ti in (1, 2, 3):
        ess.ess_tf_update(ctx, t, torch.from_numpy(tfs[ti]).cuda())
        for st in sts:
            ess.ess_rebuild(ctx, st)
    for st in sts:                     # no edit since: the last pass stands
        ess.ess_rebuild(ctx, st)
    ess.ess_rebuild(ctx, other)        # another brick size: its own pass
    ess.ess_rebuild_batch(ctx, sts)    # the batch finds this edit's pass done
    ess.ess_sync(ctx)
    ess.ess_profile_enable(ctx, False)
    assert ess.ess_profile_read(ctx)["brick_minmax"][0] == 4
    ov, ot = ora.OVolume(v, 0, 255), ora.OTF(tfs[3])
    for st, B in zip(sts + [other], (8, 8, 8, 16)):
        assert np.array_equal(ess.ess_structure_read(ctx, st, ess.ARR_MASK), ora.build_mask(ov, ot, B))
        ess.ess_release(ctx, st)
