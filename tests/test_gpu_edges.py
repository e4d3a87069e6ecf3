"""Edge cases of the path at the limits the ABI allows: the largest TF table
(65536 entries), one-pixel and one-row images, a volume with the maximum of
1024 bricks along one axis (the 30-bit Morton code's limit), and the smallest
and largest brick sizes.  Structures bit-exact, images against the oracle."""
import numpy as np
import pytest

from paper_1912_09596_gb300 import synth
from gpu_util import assert_image_parity, upload
from test_gpu_kd import kd_height
from test_gpu_lbvh import check_lbvh

pytestmark = pytest.mark.gpu

KINDS = ("NONE", "GRID", "LBVH", "KD", "HYBRID")


def _render(ess, torch, ctx, st, cam, W, H, ert=0.99):
    out = torch.empty((H, W, 4), dtype=torch.float32, device="cuda")
    ess.ess_render(ctx, st, ess.camera_from(cam), ess.render_params(0.5, ert, (0.1, 0.2, 0.3, 0.4)),
                   W, H, out)
    ess.ess_sync(ctx)
    return out.cpu().numpy()


def _all_kinds(ess, ctx, vol, t, B):
    return {k: ess.ess_build(ctx, vol, t, getattr(ess, k),
                             ess.build_params(brick=B, halting=0 if k == "HYBRID" else 1))
            for k in KINDS}


def test_largest_tf_table(gpu, ctx, ora):
    """A 65536-entry TF over a u16 volume: every TF entry is addressable."""
    ess, torch = gpu
    v = synth.ct_like_u16((36, 40, 32), seed=5)
    tf = synth.tf_random_sparse(65536, seed=7, p_zero=0.7)
    vol, t = upload(ess, torch, ctx, v, 0, 65535, tf)
    ov, ot = ora.OVolume(v, 0, 65535), ora.OTF(tf)
    cam = synth.orbit_camera(v.shape[::-1], 40, 32, theta=1.3, phi=0.4)
    ref, _ = ora.render_naive(ov, ot, cam, 40, 32, dt=0.5, ert=0.99, bg=(0.1, 0.2, 0.3, 0.4))
    mask = ora.build_mask(ov, ot, 8)
    for k, st in _all_kinds(ess, ctx, vol, t, 8).items():
        if k != "NONE":
            assert np.array_equal(ess.ess_structure_read(ctx, st, ess.ARR_MASK), mask), k
        assert_image_parity(_render(ess, torch, ctx, st, cam, 40, 32), ref, "65536-entry TF " + k)


@pytest.mark.parametrize("W,H", [(1, 1), (1, 9), (13, 1), (3, 5), (33, 17)])
def test_tiny_and_ragged_images(gpu, ctx, ora, W, H):
    ess, torch = gpu
    v = synth.blobs_u8((30, 26, 22), n_blobs=5, seed=4)
    tf = synth.tf_ramp(256, 40)
    vol, t = upload(ess, torch, ctx, v, 0, 255, tf)
    cam = synth.orbit_camera(v.shape[::-1], W, H, theta=0.8, phi=0.2, dist=1.4)
    ref, _ = ora.render_naive(ora.OVolume(v, 0, 255), ora.OTF(tf), cam, W, H, dt=0.5, ert=0.99,
                              bg=(0.1, 0.2, 0.3, 0.4))
    for k, st in _all_kinds(ess, ctx, vol, t, 4).items():
        assert_image_parity(_render(ess, torch, ctx, st, cam, W, H), ref, "%dx%d %s" % (W, H, k))


@pytest.mark.parametrize("nx,B", [(8192, 8), (2048, 2)])
def test_1024_bricks_along_one_axis(gpu, ctx, ora, nx, B):
    """gx = 1024 bricks: Morton x coordinates up to 1023 (all 10 bits), the
    LBVH and k-d trees bit-exact, images against the oracle."""
    ess, torch = gpu
    rng = np.random.default_rng(nx + B)
    v = np.where(rng.random((3, 2, nx)) < 0.2, rng.integers(60, 256, (3, 2, nx)), 0).astype(np.uint8)
    tf = synth.tf_ramp(256, 40)
    vol, t = upload(ess, torch, ctx, v, 0, 255, tf)
    ov, ot = ora.OVolume(v, 0, 255), ora.OTF(tf)
    assert ov.grid(B)[0] == 1024
    mask = ora.build_mask(ov, ot, B)
    sts = _all_kinds(ess, ctx, vol, t, B)
    check_lbvh(ess, ctx, sts["LBVH"], ora.lbvh_build(mask, ov.grid(B)))
    ref_kd = ora.kd_build(mask, ov.grid(B), B, ov.dims, nbins=4, halting=1, mls=0)
    got_kd = ess.ess_structure_read(ctx, sts["KD"], ess.ARR_KD_NODES).reshape(-1, 9)
    assert np.array_equal(got_kd, ref_kd)
    assert ess.ess_structure_info_get(ctx, sts["KD"])["height"] == kd_height(ref_kd)
    # a view down the long axis and one across it
    cams = [synth.axis_ortho_camera(ov.dims, axis=0, half=(1.5, 1.0)),
            synth.axis_ortho_camera(ov.dims, axis=2, half=(nx / 2.0, 1.0))]
    for cam, (W, H) in zip(cams, [(6, 4), (256, 3)]):
        ref, _ = ora.render_naive(ov, ot, cam, W, H, dt=0.5, ert=0.99, bg=(0.1, 0.2, 0.3, 0.4))
        for k, st in sts.items():
            assert_image_parity(_render(ess, torch, ctx, st, cam, W, H), ref,
                                "%d long, B=%d, %s" % (nx, B, k))


@pytest.mark.parametrize("B", [2, 64])
def test_smallest_and_largest_bricks(gpu, ctx, ora, B):
    """B = 2 (many tiny bricks) and B = 64 (two partial bricks per axis)."""
    ess, torch = gpu
    v = synth.blobs_u8((70, 66, 74), n_blobs=8, seed=9)
    tf = synth.tf_ramp(256, 60)
    vol, t = upload(ess, torch, ctx, v, 0, 255, tf)
    ov, ot = ora.OVolume(v, 0, 255), ora.OTF(tf)
    mask = ora.build_mask(ov, ot, B)
    sts = _all_kinds(ess, ctx, vol, t, B)
    check_lbvh(ess, ctx, sts["LBVH"], ora.lbvh_build(mask, ov.grid(B)))
    ref_kd = ora.kd_build(mask, ov.grid(B), B, ov.dims, nbins=4, halting=1, mls=0)
    assert np.array_equal(ess.ess_structure_read(ctx, sts["KD"], ess.ARR_KD_NODES).reshape(-1, 9),
                          ref_kd)
    cam = synth.orbit_camera(v.shape[::-1], 48, 40, theta=2.1, phi=0.5)
    ref, _ = ora.render_naive(ov, ot, cam, 48, 40, dt=0.5, ert=0.99, bg=(0.1, 0.2, 0.3, 0.4))
    for k, st in sts.items():
        assert_image_parity(_render(ess, torch, ctx, st, cam, 48, 40), ref, "B=%d %s" % (B, k))


@pytest.mark.parametrize("dist,fov", [(1.6, 40.0), (1400.0, 0.08)])
def test_grid_crossings_near_and_far_camera(gpu, ctx, ora, dist, fov):
    """The grid walk advances its crossings by B |1/d| when the host bounds
    their drift below dt / 4, and recomputes them from plane positions
    otherwise: a camera 58,000 voxels away takes the second path.  Images
    against the oracle's naive march, sample counts against its enumeration
    of the non-empty bricks."""
    ess, torch = gpu
    v = synth.blobs_u8((48, 44, 52), n_blobs=7, seed=12)
    tf = synth.tf_ramp(256, 50)
    vol, t = upload(ess, torch, ctx, v, 0, 255, tf)
    ov, ot = ora.OVolume(v, 0, 255), ora.OTF(tf)
    W, H, B = 40, 36, 4
    cam = synth.orbit_camera(v.shape[::-1], W, H, theta=0.9, phi=0.3, dist=dist, fov_deg=fov)
    assert np.abs(cam.eye).max() < 60000.0
    ref, _ = ora.render_naive(ov, ot, cam, W, H, dt=0.5, ert=2.0, bg=(0.1, 0.2, 0.3, 0.4))
    mask = ora.build_mask(ov, ot, B)
    boxes = ora.brick_boxes(np.nonzero(mask)[0], ov.grid(B), B, ov.dims)
    _, n_ref = ora.render_boxes(ov, ot, cam, W, H, boxes, dt=0.5, ert=2.0)
    assert n_ref > 10000
    for k in ("GRID", "HYBRID"):
        st = ess.ess_build(ctx, vol, t, getattr(ess, k),
                           ess.build_params(brick=B, halting=0 if k == "HYBRID" else 1))
        ess.ess_sample_count(ctx, reset=True)
        img = _render(ess, torch, ctx, st, cam, W, H, ert=2.0)
        n_gpu = ess.ess_sample_count(ctx, reset=True)
        assert_image_parity(img, ref, "dist %g %s" % (dist, k))
        if k == "GRID":
            assert abs(n_gpu - n_ref) <= max(8, 0.002 * n_ref), (dist, n_gpu, n_ref)
        ess.ess_release(ctx, st)
