"""GPU parity of the hybrid grid (Sec. 3.3): a k-d tree (the paper's hybrid
uses the shallow halting rule) whose leaves are crossed with the macrocell
grid of the same brick size.  Its tree is the k-d build (bit-exact node
records), its images equal naive marching bit for bit, and it takes the
samples of the grid's non-empty bricks."""
import numpy as np
import pytest

from paper_1912_09596_gb300 import synth
from gpu_util import assert_image_parity, bits, render, upload

pytestmark = pytest.mark.gpu

CASES = [
    ("ct", lambda: synth.ct_like_u8((96, 96, 96), seed=1, n_vessels=8), (0, 255),
     lambda: synth.tf_set_ct()[2]),
    ("blobs", lambda: synth.blobs_u8((72, 64, 56), n_blobs=9, seed=3), (0, 255),
     lambda: synth.tf_ramp(256, 40)),
    ("menger", lambda: synth.menger_u8(81), (0, 255), lambda: synth.tf_ramp(256, 100)),
]


@pytest.mark.parametrize("case", CASES, ids=lambda c: c[0])
@pytest.mark.parametrize("B,halting", [(8, 0), (16, 0), (8, 1)])
def test_hybrid_tree_is_the_kd_build(gpu, ctx, ora, case, B, halting):
    ess, torch = gpu
    name, vf, (lo, hi), tff = case
    v, tf = vf(), tff()
    vol, t = upload(ess, torch, ctx, v, lo, hi, tf)
    st = ess.ess_build(ctx, vol, t, ess.HYBRID, ess.build_params(brick=B, nbins=4, halting=halting))
    ov, ot = ora.OVolume(v, lo, hi), ora.OTF(tf)
    mask = ora.build_mask(ov, ot, B)
    ref = ora.kd_build(mask, ov.grid(B), B, ov.dims, nbins=4, halting=halting, mls=0)
    got = ess.ess_structure_read(ctx, st, ess.ARR_KD_NODES).reshape(-1, 9)
    assert np.array_equal(got, ref)
    assert np.array_equal(ess.ess_structure_read(ctx, st, ess.ARR_MASK), mask)
    assert ess.ess_structure_info_get(ctx, st)["n_nodes"] == len(ref)


@pytest.mark.parametrize("ert", [2.0, 0.99])
def test_hybrid_render_matches_oracle_and_naive(gpu, ctx, ora, ert):
    ess, torch = gpu
    rng = np.random.default_rng(13)
    for name, vf, (lo, hi), tff in CASES:
        v, tf = vf(), tff()
        vol, t = upload(ess, torch, ctx, v, lo, hi, tf)
        naive = ess.ess_build(ctx, vol, t, ess.NONE)
        ov, ot = ora.OVolume(v, lo, hi), ora.OTF(tf)
        for B in (8, 16):
            st = ess.ess_build(ctx, vol, t, ess.HYBRID, ess.build_params(brick=B, halting=0))
            for cam in (synth.random_camera(ov.dims, rng, ortho=False),
                        synth.random_camera(ov.dims, rng, ortho=True),
                        synth.axis_ortho_camera(ov.dims, axis=2, half=(B * 2.0, B * 2.0))):
                W, H = 41, 31
                ref, _ = ora.render_naive(ov, ot, cam, W, H, ert=ert)
                got = render(ess, torch, ctx, st, cam, W, H, ert=ert)
                assert_image_parity(got, ref, "%s hybrid B=%d" % (name, B))
                assert np.array_equal(bits(got), bits(render(ess, torch, ctx, naive, cam, W, H,
                                                             ert=ert)))
            ess.ess_release(ctx, st)


def test_hybrid_batched_equals_single(gpu, ctx):
    ess, torch = gpu
    name, vf, (lo, hi), tff = CASES[0]
    v = vf()
    vol, _ = upload(ess, torch, ctx, v, lo, hi, tff())
    rng = np.random.default_rng(3)
    items, singles = [], []
    for k in range(6):
        t = ess.ess_tf_set(ctx, synth.tf_piecewise_random(256, seed=k))
        st = ess.ess_build(ctx, vol, t, ess.HYBRID, ess.build_params(brick=8, halting=0))
        cam = synth.random_camera(v.shape[::-1], rng)
        W, H = [(48, 40), (33, 65), (64, 64)][k % 3]
        out = torch.empty((H, W, 4), dtype=torch.float32, device="cuda")
        items.append((st, cam, ess.render_params(0.5, 0.99), W, H, out))
        singles.append(render(ess, torch, ctx, st, cam, W, H, ert=0.99))
    ess.ess_render_batch(ctx, items)
    ess.ess_sync(ctx)
    for (st, cam, p, W, H, out), ref in zip(items, singles):
        assert np.array_equal(bits(out.cpu().numpy()), bits(ref))
