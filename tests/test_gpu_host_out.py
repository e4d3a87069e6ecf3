"""Host outputs of ess_render: a pinned buffer is written by the render kernel
itself over the host link, pageable memory through a staging buffer and a
copy; both give the device output's bits, and the oracle's image."""
import numpy as np
import pytest

from paper_1912_09596_gb300 import synth
from gpu_util import assert_image_parity, bits, upload

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("kind", ["GRID", "LBVH", "KD"])
def test_host_outputs_equal_device_output(gpu, ctx, ora, kind):
    ess, torch = gpu
    v = synth.blobs_u8((40, 36, 44), n_blobs=6, seed=13)
    tf = synth.tf_ramp(256, 45)
    vol, t = upload(ess, torch, ctx, v, 0, 255, tf)
    st = ess.ess_build(ctx, vol, t, getattr(ess, kind), ess.build_params(brick=4))
    W, H = 37, 29
    cam = synth.orbit_camera(v.shape[::-1], W, H, theta=1.1, phi=0.25)
    rp = ess.render_params(0.5, 0.99, (0.1, 0.2, 0.3, 0.4))
    dev = torch.empty((H, W, 4), dtype=torch.float32, device="cuda")
    ess.ess_render(ctx, st, ess.camera_from(cam), rp, W, H, dev)
    ess.ess_sync(ctx)
    ref_dev = dev.cpu().numpy()
    outs = []
    for _ in range(2):  # twice: the second call reuses the path's buffers
        pinned = torch.full((H, W, 4), -1.0, dtype=torch.float32).pin_memory()
        pageable = np.full((H, W, 4), -1.0, dtype=np.float32)
        ess.ess_render(ctx, st, ess.camera_from(cam), rp, W, H, pinned)
        ess.ess_render(ctx, st, ess.camera_from(cam), rp, W, H, pageable)
        outs += [pinned.numpy().copy(), pageable]
    for o in outs:
        assert np.array_equal(bits(o), bits(ref_dev))
    ref, _ = ora.render_naive(ora.OVolume(v, 0, 255), ora.OTF(tf), cam, W, H, dt=0.5, ert=0.99,
                              bg=(0.1, 0.2, 0.3, 0.4))
    assert_image_parity(outs[0], ref, "pinned host output " + kind)
