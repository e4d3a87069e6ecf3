"""GPU parity of the second render workload: gradient shading (R13) and
opacity correction (R14), through the C ABI.  Every structure kind, every
voxel type and both samplers give the oracle's naive image (the GPU and the
oracle evaluate the same float32 operation sequence, so bit for bit is
expected; the bar is 2e-5), batched renders equal single renders, and the
samples taken are those of the unshaded renderer."""
import numpy as np
import pytest

from paper_1912_09596_gb300 import synth
from gpu_util import assert_image_parity, bits, upload

pytestmark = pytest.mark.gpu

SHADE = (0.25, 0.6, 0.3, 12)
KINDS = ("NONE", "GRID", "LBVH", "KD", "HYBRID")


def _volumes():
    yield "blobs_u8", synth.blobs_u8((40, 36, 44), n_blobs=6, seed=2), (0, 255), synth.tf_ramp(256, 40)
    u = synth.ct_like_u16((38, 34, 30), seed=3)
    yield "ct_u16", u, (0, 65535), synth.tf_piecewise_random(700, seed=4)
    rng = np.random.default_rng(5)
    f = np.where(rng.random((29, 35, 31)) < 0.85, 0.0, rng.uniform(0, 1, (29, 35, 31)))
    yield "sparse_f32", f.astype(np.float32), (0.0, 1.0), synth.tf_random_sparse(1024, seed=6, p_zero=0.8)


VOLS = list(_volumes())


def _render(ess, torch, ctx, st, cam, W, H, rp):
    out = torch.empty((H, W, 4), dtype=torch.float32, device="cuda")
    ess.ess_render(ctx, st, cam, rp, W, H, out)
    ess.ess_sync(ctx)
    return out.cpu().numpy()


@pytest.mark.parametrize("case", VOLS, ids=lambda c: c[0])
@pytest.mark.parametrize("cells", [1, 0])
@pytest.mark.parametrize("mode", ["shade", "correct", "both"])
def test_shaded_render_equals_oracle(gpu, ctx, ora, case, cells, mode):
    ess, torch = gpu
    name, v, (lo, hi), tf = case
    vol, t = upload(ess, torch, ctx, v, lo, hi, tf)
    ess.ess_volume_set_sampler(ctx, vol, cells)
    ov, ot = ora.OVolume(v, lo, hi), ora.OTF(tf)
    shade = SHADE if mode in ("shade", "both") else None
    dt, dt_ref = (0.5, 0.0) if mode == "shade" else (0.4, 1.3)
    W, H = 40, 36
    rng = np.random.default_rng([[c[0] for c in VOLS].index(name), cells,
                                 ["shade", "correct", "both"].index(mode)])
    cams = [synth.random_camera(v.shape[::-1], rng) for _ in range(2)]
    sts = {k: ess.ess_build(ctx, vol, t, getattr(ess, k),
                            ess.build_params(brick=8, halting=0 if k == "HYBRID" else 1))
           for k in KINDS}
    for ert in (2.0, 0.95):
        rp = ess.render_params(dt, ert, (0.1, 0.2, 0.3, 0.4), shade=shade, dt_ref=dt_ref)
        for cam in cams:
            ref, _ = ora.render_naive(ov, ot, cam, W, H, dt=dt, ert=ert, bg=(0.1, 0.2, 0.3, 0.4),
                                      shade=shade, dt_ref=dt_ref)
            for k, st in sts.items():
                got = _render(ess, torch, ctx, st, ess.camera_from(cam), W, H, rp)
                assert_image_parity(got, ref, "%s %s cells=%d %s ert=%g" % (name, k, cells, mode, ert))


def test_shading_keeps_the_samples(gpu, ctx):
    """Shading changes colours, not the sample lattice or the skipping: every
    kind evaluates the same number of samples shaded as unshaded, and the
    images differ."""
    ess, torch = gpu
    v = synth.ct_like_u8((64, 56, 48), seed=7, n_vessels=6)
    vol, t = upload(ess, torch, ctx, v, 0, 255, synth.tf_set_ct()[3])
    cam = ess.camera_from(synth.orbit_camera(v.shape[::-1], 64, 64, theta=0.4, phi=0.3, dist=1.7))
    for k in KINDS:
        st = ess.ess_build(ctx, vol, t, getattr(ess, k), ess.build_params(brick=8))
        counts, imgs = [], []
        for shade in (None, SHADE):
            ess.ess_sample_count(ctx, reset=True)
            imgs.append(_render(ess, torch, ctx, st, cam, 64, 64,
                                ess.render_params(0.5, 0.99, shade=shade)))
            counts.append(ess.ess_sample_count(ctx))
        assert counts[0] == counts[1] > 0, k
        assert not np.array_equal(bits(imgs[0]), bits(imgs[1])), k


def test_batched_shaded_equals_single(gpu, ctx):
    """A batch mixing shaded, corrected and plain items (different kernels,
    one call) gives every single render's image bit for bit."""
    ess, torch = gpu
    v = synth.blobs_u8((48, 40, 44), n_blobs=7, seed=8)
    vol, t = upload(ess, torch, ctx, v, 0, 255, synth.tf_ramp(256, 40))
    sts = [ess.ess_build(ctx, vol, t, getattr(ess, k), ess.build_params(brick=8))
           for k in ("GRID", "LBVH", "KD")]
    params = [ess.render_params(0.5, 0.99), ess.render_params(0.5, 0.99, shade=SHADE),
              ess.render_params(0.7, 2.0, dt_ref=1.0), ess.render_params(0.3, 0.99, shade=SHADE, dt_ref=0.5)]
    rng = np.random.default_rng(9)
    items, refs = [], []
    for i in range(12):
        st = sts[i % 3]
        rp = params[i % 4]
        W, H = [(32, 24), (48, 40), (64, 64)][i % 3]
        cam = ess.camera_from(synth.random_camera(v.shape[::-1], rng))
        out = torch.empty((H, W, 4), dtype=torch.float32, device="cuda")
        items.append((st, cam, rp, W, H, out))
        refs.append(_render(ess, torch, ctx, st, cam, W, H, rp))
    ess.ess_render_batch(ctx, items)
    ess.ess_sync(ctx)
    for it, ref in zip(items, refs):
        assert np.array_equal(bits(it[5].cpu().numpy()), bits(ref))


@pytest.mark.parametrize("bad", [dict(shading=2), dict(shading=1, shininess=0),
                                 dict(shading=1, shininess=129), dict(shading=1, ka=-0.1),
                                 dict(shading=1, kd=float("nan")), dict(dt_ref=-1.0),
                                 dict(dt_ref=float("inf"))])
def test_shading_parameters_are_checked(gpu, ctx, bad):
    ess, torch = gpu
    v = synth.blobs_u8((16, 16, 16), seed=1)
    vol, t = upload(ess, torch, ctx, v, 0, 255, synth.tf_ramp(256, 40))
    st = ess.ess_build(ctx, vol, t, ess.GRID, ess.build_params(brick=8))
    rp = ess.render_params(0.5, 2.0, shade=(0.2, 0.5, 0.3, 8))
    for key, val in bad.items():
        setattr(rp, key, val)
    out = torch.empty((8, 8, 4), dtype=torch.float32, device="cuda")
    with pytest.raises(ess.EssError) as e:
        ess.ess_render(ctx, st, ess.camera_from(synth.orbit_camera(v.shape[::-1], 8, 8, 0.3)),
                       rp, 8, 8, out)
    assert e.value.status == ess.ERR_ARG
