"""ess_rebuild_batch: many structures (one per TF) over one volume rebuilt
together, with one min/max rescan per volume and brick size and the build
chains spread over several streams.  Every structure equals its oracle build
and its single ess_rebuild (masks, LBVH and k-d nodes bit for bit), renders
right after the batch equal the naive image, and bad batches are refused."""
import numpy as np
import pytest

from paper_1912_09596_gb300 import synth
from gpu_util import assert_image_parity, bits

pytestmark = pytest.mark.gpu


def _setup(ess, torch, ctx, n_tf, kinds, rescan):
    v = synth.ct_like_u16((48, 44, 40), seed=6)
    vol = ess.ess_volume_upload(ctx, torch.from_numpy(v).cuda(), 0, 65535)
    tfs = [synth.tf_piecewise_random(1024, seed=50 + i) for i in range(n_tf)]
    tfh = [ess.ess_tf_set(ctx, t) for t in tfs]
    sts = []
    for i, t in enumerate(tfh):
        k = kinds[i % len(kinds)]
        sts.append((k, ess.ess_build(ctx, vol, t, k, ess.build_params(
            brick=8 if i % 2 == 0 else 4, rescan=rescan, halting=0 if k == ess.HYBRID else 1))))
    return v, tfs, tfh, vol, sts


@pytest.mark.parametrize("rescan", [1, 0])
def test_batch_equals_oracle_and_single_rebuilds(gpu, ctx, ora, rescan):
    ess, torch = gpu
    kinds = (ess.GRID, ess.LBVH, ess.KD, ess.HYBRID)
    v, tfs, tfh, vol, sts = _setup(ess, torch, ctx, 12, kinds, rescan)
    ov = ora.OVolume(v, 0, 65535)
    # edit every TF, then rebuild all at once
    new = [synth.tf_piecewise_random(1024, seed=90 + i) for i in range(len(tfh))]
    for t, table in zip(tfh, new):
        ess.ess_tf_update(ctx, t, table)
    ess.ess_rebuild_batch(ctx, [h for _, h in sts])
    reads = {}
    for i, ((k, h), table) in enumerate(zip(sts, new)):
        B = 8 if i % 2 == 0 else 4
        ot = ora.OTF(table)
        mask = ora.build_mask(ov, ot, B)
        got_mask = ess.ess_structure_read(ctx, h, ess.ARR_MASK)
        assert np.array_equal(got_mask, mask), (i, k)
        if k in (ess.KD, ess.HYBRID):
            ref = ora.kd_build(mask, ov.grid(B), B, ov.dims, nbins=4,
                               halting=0 if k == ess.HYBRID else 1, mls=0)
            got = ess.ess_structure_read(ctx, h, ess.ARR_KD_NODES).reshape(-1, 9)
            assert np.array_equal(got, ref), (i, k)
        if k == ess.LBVH:
            ref = ora.lbvh_build(mask, ov.grid(B))
            assert np.array_equal(ess.ess_structure_read(ctx, h, ess.ARR_LBVH_LEFT), ref["left"])
            assert np.array_equal(ess.ess_structure_read(ctx, h, ess.ARR_LBVH_BOXES).reshape(-1, 6),
                                  ref["boxes"].reshape(-1, 6))
        reads[i] = got_mask
    # the same structures rebuilt one by one give the same arrays
    for _, h in sts:
        ess.ess_rebuild(ctx, h)
    for i, (k, h) in enumerate(sts):
        assert np.array_equal(ess.ess_structure_read(ctx, h, ess.ARR_MASK), reads[i])


def test_renders_right_after_the_batch(gpu, ctx, ora):
    ess, torch = gpu
    kinds = (ess.GRID, ess.LBVH, ess.KD)
    v, tfs, tfh, vol, sts = _setup(ess, torch, ctx, 6, kinds, 1)
    new = [synth.tf_piecewise_random(1024, seed=120 + i) for i in range(len(tfh))]
    for t, table in zip(tfh, new):
        ess.ess_tf_update(ctx, t, table)
    ess.ess_rebuild_batch(ctx, [h for _, h in sts])
    cam = synth.orbit_camera(v.shape[::-1], 40, 32, theta=0.9, phi=0.3)
    outs = []
    for _, h in sts:
        out = torch.empty((32, 40, 4), dtype=torch.float32, device="cuda")
        ess.ess_render(ctx, h, ess.camera_from(cam), ess.render_params(0.5, 0.99), 40, 32, out)
        outs.append(out)
    ess.ess_sync(ctx)
    ov = ora.OVolume(v, 0, 65535)
    for out, table in zip(outs, new):
        ref, _ = ora.render_naive(ov, ora.OTF(table), cam, 40, 32, dt=0.5, ert=0.99)
        assert_image_parity(out.cpu().numpy(), ref, "after batch rebuild")


def test_bad_batches_are_refused(gpu, ctx):
    ess, torch = gpu
    v, tfs, tfh, vol, sts = _setup(ess, torch, ctx, 2, (ess.GRID,), 0)
    h = sts[0][1]
    with pytest.raises(ess.EssError) as e:
        ess.ess_rebuild_batch(ctx, [h, h])
    assert e.value.status == ess.ERR_ARG
    with pytest.raises(ess.EssError) as e:
        ess.ess_rebuild_batch(ctx, [h, 12345])
    assert e.value.status == ess.ERR_HANDLE
