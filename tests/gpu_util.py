"""Helpers shared by the GPU parity tests: run the CUDA path through the C ABI
and the oracle on the same seeded inputs."""
import numpy as np


def bits(a):
    return np.ascontiguousarray(a, dtype=np.float32).view(np.uint32)


TOL = 2e-5   # per-channel absolute bound on images (bitwise equality expected)


def assert_image_parity(got, ref, what=""):
    """Bitwise equality is expected (identical float32 operation sequences);
    the acceptance bar is |got - ref| <= 2e-5 per channel."""
    got = np.asarray(got, dtype=np.float32)
    ref = np.asarray(ref, dtype=np.float32)
    assert got.shape == ref.shape
    if np.array_equal(bits(got), bits(ref)):
        return 0
    diff = np.abs(got.astype(np.float64) - ref.astype(np.float64))
    worst = float(diff.max())
    n = int((bits(got) != bits(ref)).sum())
    assert worst <= TOL, "%s: %d channels differ, max |diff| %g > %g" % (what, n, worst, TOL)
    return n


def upload(ess, torch, ctx, vol_np, lo, hi, tf_np, device=True):
    if device:
        vol = ess.ess_volume_upload(ctx, torch.from_numpy(vol_np).cuda(), lo, hi)
        tf = ess.ess_tf_set(ctx, torch.from_numpy(np.ascontiguousarray(tf_np)).cuda())
    else:
        vol = ess.ess_volume_upload(ctx, np.ascontiguousarray(vol_np), lo, hi)
        tf = ess.ess_tf_set(ctx, np.ascontiguousarray(tf_np))
    return vol, tf


def render(ess, torch, ctx, st, cam, W, H, dt=0.5, ert=2.0, bg=(0, 0, 0, 0)):
    out = torch.empty((H, W, 4), dtype=torch.float32, device="cuda")
    ess.ess_render(ctx, st, cam, ess.render_params(dt, ert, bg), W, H, out)
    ess.ess_sync(ctx)
    return out.cpu().numpy()
