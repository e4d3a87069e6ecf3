"""Batched persistent rendering (one launch for many TFs, views and uneven
image sizes, replayed from a captured CUDA graph) gives exactly the images of
one-at-a-time rendering; the autotuner returns a usable configuration."""
import numpy as np
import pytest

from paper_1912_09596_gb300 import synth
from gpu_util import assert_image_parity, bits, render, upload

pytestmark = pytest.mark.gpu


def _setup(ess, torch, ctx, n_tf=5, dims=(64, 56, 48), dtype="u16"):
    v8 = synth.blobs_u8(dims, n_blobs=7, seed=4)
    v = (v8.astype(np.uint16) * 257) if dtype == "u16" else v8
    hi = 65535 if dtype == "u16" else 255
    vol, _ = upload(ess, torch, ctx, v, 0, hi, synth.tf_ramp(256, 40))
    tfs, sts = [], []
    kinds = [ess.GRID, ess.LBVH, ess.KD]
    for i in range(n_tf):
        tfn = synth.tf_piecewise_random(512, seed=100 + i)
        t = ess.ess_tf_set(ctx, torch.from_numpy(tfn).cuda())
        st = ess.ess_build(ctx, vol, t, kinds[i % 3], ess.build_params(brick=8))
        tfs.append(tfn)
        sts.append(st)
    return v, hi, tfs, sts


@pytest.mark.parametrize("tile_w", [0, 4, 16])
def test_batch_equals_sequential(gpu, ctx, ora, tile_w):
    ess, torch = gpu
    v, hi, tfs, sts = _setup(ess, torch, ctx)
    rng = np.random.default_rng(7)
    sizes = [(64, 64), (96, 40), (37, 53), (128, 72), (1, 1), (200, 3)]
    items, refs = [], []
    for k in range(24):
        st = sts[k % len(sts)]
        W, H = sizes[k % len(sizes)]
        cam = synth.random_camera((64, 56, 48), rng)
        params = ess.render_params(0.5, 0.99 if k % 2 else 2.0, (0.1, 0.0, 0.2, 0.5))
        out = torch.full((H, W, 4), -1.0, dtype=torch.float32, device="cuda")
        items.append((st, cam, params, W, H, out))
        refs.append(render(ess, torch, ctx, st, cam, W, H, dt=0.5, ert=params.ert,
                           bg=(0.1, 0.0, 0.2, 0.5)))
    ess.ess_render_batch(ctx, items, tile_w=tile_w)
    ess.ess_sync(ctx)
    for (st, cam, params, W, H, out), ref in zip(items, refs):
        assert np.array_equal(bits(out.cpu().numpy()), bits(ref))
    # replay of the captured graph with a different item count
    sub = items[3:11]
    for it in sub:
        it[5].fill_(-2.0)
    ess.ess_render_batch(ctx, sub, tile_w=tile_w)
    ess.ess_sync(ctx)
    for it, ref in zip(sub, refs[3:11]):
        assert np.array_equal(bits(it[5].cpu().numpy()), bits(ref))
    # one image against the oracle
    st, cam, params, W, H, out = items[3]
    ov, ot = ora.OVolume(v, 0, hi), ora.OTF(tfs[3 % len(tfs)])
    r, _ = ora.render_naive(ov, ot, cam, W, H, dt=0.5, ert=params.ert, bg=(0.1, 0.0, 0.2, 0.5))
    assert_image_parity(out.cpu().numpy(), r, "batch vs oracle")


def test_batch_mixed_dtypes_and_stale(gpu, ctx, ora):
    ess, torch = gpu
    v16, hi, tfs, sts = _setup(ess, torch, ctx, n_tf=3, dtype="u16")
    v8 = synth.blobs_u8((40, 40, 40), n_blobs=5, seed=9)
    vol8, t8 = upload(ess, torch, ctx, v8, 0, 255, synth.tf_ramp(256, 40))
    st8 = ess.ess_build(ctx, vol8, t8, ess.LBVH, ess.build_params(brick=4))
    cam = synth.orbit_camera((40, 40, 40), 50, 30, 0.4)
    outs = [torch.empty((30, 50, 4), dtype=torch.float32, device="cuda") for _ in range(4)]
    p = ess.render_params()
    items = [(st8, cam, p, 50, 30, outs[0]), (sts[0], cam, p, 50, 30, outs[1]),
             (st8, cam, p, 50, 30, outs[2]), (sts[1], cam, p, 50, 30, outs[3])]
    ess.ess_render_batch(ctx, items)
    ess.ess_sync(ctx)
    for (st, c, pp, W, H, out) in items:
        assert np.array_equal(bits(out.cpu().numpy()), bits(render(ess, torch, ctx, st, c, W, H)))
    ess.ess_tf_update(ctx, t8, synth.tf_ramp(256, 90))
    with pytest.raises(ess.EssError) as e:
        ess.ess_render_batch(ctx, items)
    assert e.value.status == ess.ERR_STALE


def test_autotune_returns_working_config(gpu, ctx, ora):
    ess, torch = gpu
    v = synth.ct_like_u8((96, 96, 96), seed=1, n_vessels=6)
    tf = synth.tf_set_ct()[0]
    vol, t = upload(ess, torch, ctx, v, 0, 255, tf)
    cams = [synth.orbit_camera((96, 96, 96), 96, 96, th) for th in (0.2, 1.9)]
    p = ess.render_params(0.5, 0.99)
    best = ess.ess_autotune(ctx, vol, t, cams, p, 96, 96, frames_per_edit=4.0)
    assert best["kind"] in (ess.GRID, ess.LBVH, ess.KD)
    assert best["brick"] in (4, 8, 16, 32) and best["tile_w"] in (4, 8, 16, 32)
    assert best["render_ms"] > 0 and best["build_ms"] > 0
    st = ess.ess_build(ctx, vol, t, best["kind"], ess.build_params(brick=best["brick"]))
    ov, ot = ora.OVolume(v, 0, 255), ora.OTF(tf)
    ref, _ = ora.render_naive(ov, ot, cams[0], 96, 96, ert=0.99)
    out = torch.empty((96, 96, 4), dtype=torch.float32, device="cuda")
    ess.ess_render(ctx, st, cams[0], ess.render_params(0.5, 0.99, tile_w=best["tile_w"]), 96, 96, out)
    ess.ess_sync(ctx)
    assert_image_parity(out.cpu().numpy(), ref, "autotuned")
