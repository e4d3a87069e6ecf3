"""Builds run on the context's build stream and are joined into the context
stream by the structure's users (render, batch render, reads, info, release,
TF updates, ess_sync).  These tests issue rebuilds and their users back to back
with no synchronisation in between, over several TF edits and several
structures at once, and check every result against naive marching (images:
bit-identical, Sec. 2) or the oracle (masks and k-d nodes, bit-exact)."""
import numpy as np
import pytest

from paper_1912_09596_gb300 import synth
from gpu_util import bits

pytestmark = pytest.mark.gpu

KINDS = ("GRID", "LBVH", "KD", "HYBRID")


def _scene(ess, torch, ctx):
    v = synth.ct_like_u8((112, 96, 80), seed=4, n_vessels=10)
    tfs = synth.tf_set_ct(256)
    vol = ess.ess_volume_upload(ctx, torch.from_numpy(v).cuda(), 0.0, 255.0)
    tf = ess.ess_tf_set(ctx, tfs[0])
    return v, tfs, vol, tf


def test_rebuilds_and_renders_back_to_back(gpu, ctx):
    """TF edit, rebuild of four structures, then their renders, with no sync:
    every frame equals the naive frame of the same edit bit for bit."""
    ess, torch = gpu
    v, tfs, vol, tf = _scene(ess, torch, ctx)
    naive = ess.ess_build(ctx, vol, tf, ess.NONE)
    sts = [ess.ess_build(ctx, vol, tf, getattr(ess, k),
                         ess.build_params(brick=8, halting=0 if k == "HYBRID" else 1))
           for k in KINDS]
    W, H = 96, 80
    rp = ess.render_params(0.5, 0.99)
    frames = []
    for i, table in enumerate(tfs):
        ess.ess_tf_update(ctx, tf, table)
        for st in sts + [naive]:
            ess.ess_rebuild(ctx, st)
        cam = ess.camera_from(synth.orbit_camera(v.shape[::-1], W, H, theta=0.7 * i, phi=0.3,
                                                 dist=1.7))
        outs = []
        for st in [naive] + sts[::-1]:  # render in another order than built
            out = torch.empty((H, W, 4), dtype=torch.float32, device="cuda")
            ess.ess_render(ctx, st, cam, rp, W, H, out)
            outs.append(out)
        frames.append(outs)
    ess.ess_sync(ctx)
    for i, outs in enumerate(frames):
        ref = bits(outs[0].cpu().numpy())
        assert ref.any()
        for k, o in zip(KINDS[::-1], outs[1:]):
            assert np.array_equal(bits(o.cpu().numpy()), ref), "edit %d, %s" % (i, k)


def test_reads_follow_their_rebuild(gpu, ctx, ora):
    """Reads of the mask and the k-d nodes right after each rebuild see that
    rebuild (oracle, bit-exact)."""
    ess, torch = gpu
    v, tfs, vol, tf = _scene(ess, torch, ctx)
    kd = ess.ess_build(ctx, vol, tf, ess.KD, ess.build_params(brick=8, nbins=4, halting=1, mls=32))
    grid = ess.ess_build(ctx, vol, tf, ess.GRID, ess.build_params(brick=8))
    ov = ora.OVolume(v, 0, 255)
    for table in tfs[:5]:
        ess.ess_tf_update(ctx, tf, table)
        ess.ess_rebuild(ctx, kd)
        ess.ess_rebuild(ctx, grid)
        ot = ora.OTF(table)
        mask = ora.build_mask(ov, ot, 8)
        ref = ora.kd_build(mask, ov.grid(8), 8, ov.dims, nbins=4, halting=1, mls=32)
        got = ess.ess_structure_read(ctx, kd, ess.ARR_KD_NODES).reshape(-1, 9)
        assert np.array_equal(got, ref)
        assert np.array_equal(ess.ess_structure_read(ctx, grid, ess.ARR_MASK), mask)
        info = ess.ess_structure_info_get(ctx, kd)
        assert info["n_nodes"] == len(ref) and info["n_nonempty"] == int(mask.sum())


def test_release_and_tf_update_after_pending_rebuild(gpu, ctx):
    """Releasing a structure, or editing the TF, while its rebuild may still
    run is safe: the context waits for the build first."""
    ess, torch = gpu
    v, tfs, vol, tf = _scene(ess, torch, ctx)
    for k in KINDS:
        st = ess.ess_build(ctx, vol, tf, getattr(ess, k), ess.build_params(brick=8))
        ess.ess_rebuild(ctx, st)
        ess.ess_release(ctx, st)
    st = ess.ess_build(ctx, vol, tf, ess.KD, ess.build_params(brick=8))
    for table in tfs[:4]:
        ess.ess_rebuild(ctx, st)
        ess.ess_tf_update(ctx, tf, table)
    ess.ess_rebuild(ctx, st)
    ess.ess_sync(ctx)
    naive = ess.ess_build(ctx, vol, tf, ess.NONE)
    W, H = 64, 64
    cam = ess.camera_from(synth.orbit_camera(v.shape[::-1], W, H, theta=1.1, phi=0.3, dist=1.7))
    rp = ess.render_params(0.5, 0.99)
    a = torch.empty((H, W, 4), dtype=torch.float32, device="cuda")
    b = torch.empty_like(a)
    ess.ess_render(ctx, st, cam, rp, W, H, a)
    ess.ess_render(ctx, naive, cam, rp, W, H, b)
    ess.ess_sync(ctx)
    assert np.array_equal(bits(a.cpu().numpy()), bits(b.cpu().numpy()))
