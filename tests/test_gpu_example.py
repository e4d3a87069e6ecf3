"""The binding's usage example (the one the README shows) runs on a GB300:
upload, TF, k-d build, render, a TF edit with its rebuild, a shaded frame; the
frames are checked against the oracle's naive marching on sampled pixels."""
import numpy as np
import pytest

from gpu_util import TOL, bits

pytestmark = pytest.mark.gpu


def test_binding_example_runs(gpu, ora):
    import torch
    from paper_1912_09596_gb300 import ess, synth

    vol_np = synth.ct_like_u8((256, 256, 256))
    ctx = ess.ess_create(0, torch.cuda.current_stream())
    vol = ess.ess_volume_upload(ctx, torch.from_numpy(vol_np).cuda(), 0, 255)
    tf = ess.ess_tf_set(ctx, synth.tf_set_ct(256)[0])              # (NT, 4) float32 RGBA
    st = ess.ess_build(ctx, vol, tf, ess.KD, ess.build_params(brick=8, nbins=4, halting=1, mls=32))
    cam_py = synth.orbit_camera((256, 256, 256), 1024, 1024, theta=0.5)
    cam = ess.camera_from(cam_py)
    out = torch.empty((1024, 1024, 4), dtype=torch.float32, device="cuda")
    ess.ess_render(ctx, st, cam, ess.render_params(dt=0.5, ert=0.99), 1024, 1024, out)
    first = out.cpu().numpy()
    ess.ess_tf_update(ctx, tf, synth.tf_set_ct(256)[3])            # a TF edit ...
    ess.ess_rebuild(ctx, st)                                       # ... and the rebuild
    ess.ess_render(ctx, st, cam, ess.render_params(0.5, 0.99, shade=(0.25, 0.6, 0.3, 12)),
                   1024, 1024, out)                                # gradient-shaded frame
    ess.ess_sync(ctx)
    shaded = out.cpu().numpy()
    ess.ess_destroy(ctx)

    ov = ora.OVolume(vol_np, 0, 255)
    rng = np.random.default_rng(0)
    xy = np.stack([rng.integers(0, 1024, 64), rng.integers(0, 1024, 64)], axis=1).astype(np.int32)
    for img, t, shade in ((first, 0, None), (shaded, 3, (0.25, 0.6, 0.3, 12))):
        ref, _ = ora.render_pixels(ov, ora.OTF(synth.tf_set_ct(256)[t]), cam_py, 1024, 1024, xy,
                                   dt=0.5, ert=0.99, threads=8, shade=shade)
        got = img[xy[:, 1], xy[:, 0]]
        if not np.array_equal(bits(got), bits(ref)):
            assert float(np.abs(got.astype(np.float64) - ref).max()) <= TOL
