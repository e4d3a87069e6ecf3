"""Failure detection without a GPU fault: the device-side waits of the
library's kernels are bounded.  A wait on a flag that nothing sets gives up
after its poll limit, the next ess_sync reports ESS_ERR_TIMEOUT, and the
context stays usable: a render after it still equals the oracle."""
import numpy as np
import pytest

from paper_1912_09596_gb300 import synth
from gpu_util import assert_image_parity, upload

pytestmark = pytest.mark.gpu


def test_wait_that_is_satisfied_reports_nothing(gpu, ctx):
    ess, torch = gpu
    ess.ess_selftest_wait(ctx, True, 1 << 16)
    ess.ess_sync(ctx)


def test_wait_that_runs_out_reports_timeout_and_context_survives(gpu, ctx, ora):
    ess, torch = gpu
    ess.ess_selftest_wait(ctx, False, 1 << 14)
    with pytest.raises(ess.EssError) as e:
        ess.ess_sync(ctx)
    assert e.value.status == ess.ERR_TIMEOUT
    ess.ess_sync(ctx)  # the status word was read and cleared
    v = synth.blobs_u8((24, 20, 28), n_blobs=4, seed=3)
    tf = synth.tf_ramp(256, 40)
    vol, t = upload(ess, torch, ctx, v, 0, 255, tf)
    st = ess.ess_build(ctx, vol, t, ess.LBVH, ess.build_params(brick=4))
    cam = synth.orbit_camera(v.shape[::-1], 32, 32, theta=0.5)
    out = torch.empty((32, 32, 4), dtype=torch.float32, device="cuda")
    ess.ess_render(ctx, st, ess.camera_from(cam), ess.render_params(0.5, 0.99), 32, 32, out)
    ess.ess_sync(ctx)
    ref, _ = ora.render_naive(ora.OVolume(v, 0, 255), ora.OTF(tf), cam, 32, 32, dt=0.5, ert=0.99)
    assert_image_parity(out.cpu().numpy(), ref, "after a timeout")


@pytest.mark.parametrize("bad", [(2, 10), (0, 0), (1, (1 << 24) + 1)])
def test_selftest_arguments_are_checked(gpu, ctx, bad):
    ess, torch = gpu
    with pytest.raises(ess.EssError) as e:
        ess._check(ctx, ess.lib.ess_selftest_wait(ctx, bad[0], bad[1]))
    assert e.value.status == ess.ERR_ARG
