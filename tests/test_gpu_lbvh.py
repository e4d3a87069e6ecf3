"""GPU parity of the LBVH build (Morton codes, onesweep radix sort, Karras
emission, bottom-up boxes) and of the LBVH renderer, against the oracle."""
import numpy as np
import pytest

from paper_1912_09596_gb300 import synth
from gpu_util import assert_image_parity, bits, render, upload

pytestmark = pytest.mark.gpu


def lbvh_case(gpu, ctx, ora, v, lo, hi, tf, B):
    ess, torch = gpu
    vol, t = upload(ess, torch, ctx, v, lo, hi, tf)
    st = ess.ess_build(ctx, vol, t, ess.LBVH, ess.build_params(brick=B))
    ov, ot = ora.OVolume(v, lo, hi), ora.OTF(tf)
    mask = ora.build_mask(ov, ot, B)
    ref = ora.lbvh_build(mask, ov.grid(B))
    return ess, st, ov, ot, ref


def check_lbvh(ess, ctx, st, ref):
    rd = lambda a: ess.ess_structure_read(ctx, st, a)
    assert np.array_equal(rd(ess.ARR_IDS), ref["ids"])
    assert np.array_equal(rd(ess.ARR_KEYS), ref["keys"])
    assert np.array_equal(rd(ess.ARR_SORTED_KEYS), ref["sorted_keys"])
    assert np.array_equal(rd(ess.ARR_SORTED_IDS), ref["sorted_ids"])
    assert np.array_equal(rd(ess.ARR_LBVH_LEFT), ref["left"])
    assert np.array_equal(rd(ess.ARR_LBVH_RIGHT), ref["right"])
    assert np.array_equal(rd(ess.ARR_LBVH_BOXES).reshape(-1, 6), ref["boxes"].reshape(-1, 6))
    info = ess.ess_structure_info_get(ctx, st)
    n = len(ref["ids"])
    assert info["n_nonempty"] == n and info["n_nodes"] == (2 * n - 1 if n else 0)
    return info


def oracle_height(ref):
    left, right = ref["left"], ref["right"]
    if len(ref["ids"]) == 0:
        return 0
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


@pytest.mark.parametrize("B", [4, 8, 16])
@pytest.mark.parametrize("seed", [0, 1])
def test_lbvh_build_bit_exact(gpu, ctx, ora, B, seed):
    v = synth.blobs_u8((72, 56, 64), n_blobs=8, seed=seed)
    tf = synth.tf_ramp(256, 40) if seed == 0 else synth.tf_random_sparse(256, seed=seed, p_zero=0.6)
    ess, st, ov, ot, ref = lbvh_case(gpu, ctx, ora, v, 0, 255, tf, B)
    info = check_lbvh(ess, ctx, st, ref)
    assert info["height"] == oracle_height(ref)


@pytest.mark.parametrize("dims,B,p_zero", [((256, 256, 256), 2, 0.0), ((300, 200, 260), 2, 0.3),
                                            ((512, 512, 512), 4, 0.0)])
def test_lbvh_large_multi_tile_sort(gpu, ctx, ora, dims, B, p_zero):
    """Up to 2M keys: hundreds of sort tiles, so the decoupled look-back runs."""
    rng = np.random.default_rng(B)
    nx, ny, nz = dims
    v = np.full((nz, ny, nx), 200, np.uint8)
    if p_zero > 0:
        # knock out random bricks entirely
        gx, gy, gz = -(-nx // B), -(-ny // B), -(-nz // B)
        dead = rng.random((gz, gy, gx)) < p_zero
        up = np.kron(dead, np.ones((B, B, B), bool))[:nz, :ny, :nx]
        v[up] = 0
    tf = synth.tf_ramp(256, 100)
    ess, st, ov, ot, ref = lbvh_case(gpu, ctx, ora, v, 0, 255, tf, B)
    assert len(ref["ids"]) > 100000
    check_lbvh(ess, ctx, st, ref)
    ess.ess_sync(ctx)


@pytest.mark.parametrize("nonempty", [0, 1, 2, 3])
def test_lbvh_tiny_counts(gpu, ctx, ora, nonempty):
    v = np.zeros((16, 16, 16), np.uint8)
    spots = [(1, 1, 1), (14, 14, 14), (2, 13, 7)]
    for (x, y, z) in spots[:nonempty]:
        v[z, y, x] = 250
    tf = synth.tf_ramp(256, 100)
    ess, st, ov, ot, ref = lbvh_case(gpu, ctx, ora, v, 0, 255, tf, 4)
    check_lbvh(ess, ctx, st, ref)
    cam = synth.orbit_camera(ov.dims, 40, 30, 0.5)
    refimg, _ = ora.render_naive(ov, ot, cam, 40, 30, bg=(0.2, 0.1, 0.0, 1.0))
    assert_image_parity(render(*ess_torch(gpu), ctx, st, cam, 40, 30, bg=(0.2, 0.1, 0.0, 1.0)),
                        refimg, "lbvh n=%d" % nonempty)


def ess_torch(gpu):
    return gpu


@pytest.mark.parametrize("ert", [2.0, 0.99])
def test_lbvh_render_matches_oracle_and_naive(gpu, ctx, ora, ert):
    ess, torch = gpu
    rng = np.random.default_rng(3)
    cases = [
        ("blobs", synth.blobs_u8((64, 48, 56), seed=2), (0, 255), synth.tf_ramp(256, 40)),
        ("f32", np.where(rng.random((40, 36, 44)) < 0.9, 0, rng.uniform(0, 1, (40, 36, 44)))
         .astype(np.float32), (0.0, 1.0), synth.tf_random_sparse(1024, seed=1, p_zero=0.85)),
        ("menger", synth.menger_u8(27), (0, 255), synth.tf_ramp(256, 100)),
    ]
    for name, v, (lo, hi), tf in cases:
        vol, t = upload(ess, torch, ctx, v, lo, hi, tf)
        naive = ess.ess_build(ctx, vol, t, ess.NONE)
        ov, ot = ora.OVolume(v, lo, hi), ora.OTF(tf)
        for B in (2, 4, 8):
            st = ess.ess_build(ctx, vol, t, ess.LBVH, ess.build_params(brick=B))
            for cam in (synth.random_camera(ov.dims, rng, ortho=False),
                        synth.random_camera(ov.dims, rng, ortho=True),
                        synth.axis_ortho_camera(ov.dims, axis=0, half=(B * 2.0, B * 2.0))):
                W, H = 37, 29
                ref, _ = ora.render_naive(ov, ot, cam, W, H, ert=ert)
                got = render(ess, torch, ctx, st, cam, W, H, ert=ert)
                assert_image_parity(got, ref, "%s lbvh B=%d" % (name, B))
                g0 = render(ess, torch, ctx, naive, cam, W, H, ert=ert)
                assert np.array_equal(bits(got), bits(g0))
            ess.ess_release(ctx, st)


def test_lbvh_rebuild_after_tf_edit(gpu, ctx, ora):
    ess, torch = gpu
    v = synth.ct_like_u8((96, 96, 96), seed=1, n_vessels=6)
    tfs = synth.tf_set_ct(256)
    vol, t = upload(ess, torch, ctx, v, 0, 255, tfs[0])
    st = ess.ess_build(ctx, vol, t, ess.LBVH, ess.build_params(brick=8))
    ov = ora.OVolume(v, 0, 255)
    cam = synth.orbit_camera(ov.dims, 48, 48, 1.2)
    for i, tf in enumerate(tfs):
        ess.ess_tf_update(ctx, t, torch.from_numpy(tf).cuda())
        ess.ess_rebuild(ctx, st)
        ot = ora.OTF(tf)
        ref = ora.lbvh_build(ora.build_mask(ov, ot, 8), ov.grid(8))
        check_lbvh(ess, ctx, st, ref)
        refimg, _ = ora.render_naive(ov, ot, cam, 48, 48, ert=0.99)
        assert_image_parity(render(ess, torch, ctx, st, cam, 48, 48, ert=0.99), refimg, "edit %d" % i)
