"""Parity at the benchmark's full sizes, on outputs the oracle can compute
one by one: the brick masks of the 512^3 CT-like workload (every brick), the
whole trees that the benchmark step builds for its eight TF edits (k-d node
records and LBVH topology and boxes, bit for bit), and sampled pixels of full frames rendered in the benchmark's launch
configuration (512^3 u8 at 1024^2, 1024^3 f32 at 1920x1080), each checked
against the oracle's naive marching of that pixel."""
import math

import numpy as np
import pytest

from paper_1912_09596_gb300 import synth
from gpu_util import TOL, bits

pytestmark = pytest.mark.gpu


def _pixels(W, H, n, seed):
    rng = np.random.default_rng(seed)
    xy = np.stack([rng.integers(0, W, n), rng.integers(0, H, n)], axis=1)
    fixed = np.array([[0, 0], [W - 1, 0], [0, H - 1], [W - 1, H - 1], [W // 2, H // 2],
                      [W // 2 - 1, H // 2], [W // 3, 2 * H // 3], [2 * W // 3, H // 3]])
    return np.concatenate([fixed, xy]).astype(np.int32)


def _check_pixels(img, xy, ref, what):
    got = img[xy[:, 1], xy[:, 0]]
    if np.array_equal(bits(got), bits(ref)):
        return
    diff = float(np.abs(got.astype(np.float64) - ref.astype(np.float64)).max())
    assert diff <= TOL, "%s: sampled pixels differ by %g" % (what, diff)


@pytest.fixture(scope="module")
def ct512():
    """The 512^3 CT-like workload of the benchmark: volume, 8 TFs, cameras."""
    dims = (512, 512, 512)
    vol = synth.ct_like_u8(dims, seed=1)
    tfs = synth.tf_set_ct(256)
    cams = [synth.orbit_camera(dims, 1024, 1024, theta=2 * math.pi * i / len(tfs), phi=0.35,
                               dist=1.6) for i in range(len(tfs))]
    return vol, tfs, cams


def test_ct512_masks_and_sampled_pixels(gpu, ctx, ora, ct512):
    ess, torch = gpu
    vol_np, tfs, cams = ct512
    W = H = 1024
    ov = ora.OVolume(vol_np, 0, 255)
    mm = {B: ora.brick_minmax(ov, B) for B in (8, 16)}
    vol = ess.ess_volume_upload(ctx, torch.from_numpy(vol_np).cuda(), 0, 255)
    for ti in (0, 3, 7):
        ot = ora.OTF(tfs[ti])
        t = ess.ess_tf_set(ctx, torch.from_numpy(tfs[ti]).cuda())
        xy = _pixels(W, H, 192, seed=ti)
        ref, _ = ora.render_pixels(ov, ot, cams[ti], W, H, xy, dt=0.5, ert=0.99, threads=8)
        for kind, B, params in ((ess.GRID, 8, {}), (ess.LBVH, 8, {}),
                                (ess.KD, 8, dict(nbins=4, halting=1, mls=32)),
                                (ess.HYBRID, 16, dict(nbins=4, halting=0))):
            st = ess.ess_build(ctx, vol, t, kind, ess.build_params(brick=B, rescan=1, **params))
            ref_mask = ora.brick_mask(mm[B][0], mm[B][1], ot, 0, 255)
            assert np.array_equal(ess.ess_structure_read(ctx, st, ess.ARR_MASK), ref_mask)
            out = torch.empty((H, W, 4), dtype=torch.float32, device="cuda")
            ess.ess_render(ctx, st, cams[ti], ess.render_params(0.5, 0.99), W, H, out)
            ess.ess_sync(ctx)
            _check_pixels(out.cpu().numpy(), xy, ref, "ct512 TF %d %s" % (ti, ess.KIND_NAMES[kind]))
            ess.ess_release(ctx, st)
        ess.ess_release(ctx, t)


def test_ct512_cell_vote_masks(gpu, ctx, ora, ct512):
    """The exact per-cell vote over every brick of the 512^3 workload (8^3
    bricks: the staged vote, each warp over several bricks) equals the
    oracle's per-cell mask bit for bit."""
    ess, torch = gpu
    vol_np, tfs, _ = ct512
    ov = ora.OVolume(vol_np, 0, 255)
    vol = ess.ess_volume_upload(ctx, torch.from_numpy(vol_np).cuda(), 0, 255)
    for ti in (0, 7):
        t = ess.ess_tf_set(ctx, torch.from_numpy(tfs[ti]).cuda())
        st = ess.ess_build(ctx, vol, t, ess.GRID, ess.build_params(brick=8, empty_test=1))
        ref = ora.brick_mask_cells(ov, 8, ora.OTF(tfs[ti]))
        assert np.array_equal(ess.ess_structure_read(ctx, st, ess.ARR_MASK), ref), ti
        ess.ess_release(ctx, st)
        ess.ess_release(ctx, t)
    ess.ess_release(ctx, vol)


def _tree_arrays(ess, ctx, st, kind):
    rd = lambda a: ess.ess_structure_read(ctx, st, a)
    if kind == ess.LBVH:
        return dict(ids=rd(ess.ARR_IDS), keys=rd(ess.ARR_KEYS), sorted_keys=rd(ess.ARR_SORTED_KEYS),
                    sorted_ids=rd(ess.ARR_SORTED_IDS), left=rd(ess.ARR_LBVH_LEFT),
                    right=rd(ess.ARR_LBVH_RIGHT), boxes=rd(ess.ARR_LBVH_BOXES).reshape(-1, 6))
    return dict(nodes=rd(ess.ARR_KD_NODES).reshape(-1, 9))


# (brick, kind, k-d parameters): the benchmark step's structures at 8^3 bricks
# (deep binned k-d with maximum leaf 32^3, Sec. 4.3), its hybrid's shallow tree,
# and the other brick sizes of the 512^3 workload.
TREES = [(8, "lbvh", None), (8, "kd", dict(nbins=4, halting=1, mls=32)),
         (8, "kd", dict(nbins=4, halting=0, mls=0)), (16, "lbvh", None),
         (16, "kd", dict(nbins=4, halting=1, mls=32)), (32, "lbvh", None),
         (32, "kd", dict(nbins=4, halting=1, mls=128))]


def test_ct512_trees_bit_exact(gpu, ctx, ora, ct512):
    """Every TF edit of the 512^3 workload: the trees rebuilt with a min/max
    rescan, exactly as the timed step builds them, equal the oracle's builds on
    the oracle's masks (Sec. 3.1 LBVH, Sec. 3.2.2 binned k-d): Morton keys, sort
    order, Karras children and boxes; k-d boxes, axes, planes and children."""
    ess, torch = gpu
    vol_np, tfs, _ = ct512
    ov = ora.OVolume(vol_np, 0, 255)
    mm = {B: ora.brick_minmax(ov, B) for B in (8, 16, 32)}
    vol = ess.ess_volume_upload(ctx, torch.from_numpy(vol_np).cuda(), 0, 255)
    t = ess.ess_tf_set(ctx, torch.from_numpy(tfs[0]).cuda())
    structs = []
    for B, name, kp in TREES:
        kind = ess.LBVH if name == "lbvh" else ess.KD
        structs.append((B, name, kp, kind,
                        ess.ess_build(ctx, vol, t, kind,
                                      ess.build_params(brick=B, rescan=1, **(kp or {})))))
    nodes_seen = 0
    for ti, tf in enumerate(tfs):
        ot = ora.OTF(tf)
        if ti > 0:
            ess.ess_tf_update(ctx, t, torch.from_numpy(tf).cuda())
            for *_, st in structs:
                ess.ess_rebuild(ctx, st)
        for B, name, kp, kind, st in structs:
            mask = ora.brick_mask(mm[B][0], mm[B][1], ot, 0, 255)
            got = _tree_arrays(ess, ctx, st, kind)
            what = "TF %d B %d %s %s" % (ti, B, name, kp)
            if kind == ess.LBVH:
                ref = ora.lbvh_build(mask, ov.grid(B))
                for key in got:
                    assert np.array_equal(got[key], ref[key].reshape(got[key].shape)), \
                        "%s: %s differs" % (what, key)
                n = len(ref["ids"])
                assert ess.ess_structure_info_get(ctx, st)["n_nodes"] == (2 * n - 1 if n else 0)
                nodes_seen += 2 * n - 1
            else:
                ref = ora.kd_build(mask, ov.grid(B), B, ov.dims, **kp)
                assert got["nodes"].shape == ref.shape, (what, got["nodes"].shape, ref.shape)
                assert np.array_equal(got["nodes"], ref), what + ": k-d nodes differ"
                assert ess.ess_structure_info_get(ctx, st)["n_nodes"] == len(ref)
                nodes_seen += len(ref)
    assert nodes_seen > 500000   # whole trees of thousands of nodes, not toy cases
    for *_, st in structs:
        ess.ess_release(ctx, st)


def test_fractal1024_f32_mask_and_sampled_pixels(gpu, ctx, ora):
    """The 1024^3 float32 fractal field (4 GiB) with a 1024-entry TF."""
    ess, torch = gpu
    dims = (1024, 1024, 1024)
    x = synth.fractal_f32_torch(dims, seed=2, device="cuda")
    host = x.cpu().numpy()
    ov = ora.OVolume(host, 0.0, 1.0)
    vol = ess.ess_volume_upload(ctx, x, 0.0, 1.0)
    del x
    tf_np = synth.tf_ramp(1024, 2)
    ot = ora.OTF(tf_np)
    t = ess.ess_tf_set(ctx, torch.from_numpy(tf_np).cuda())
    mn, mx = ora.brick_minmax(ov, 8)
    ref_mask = ora.brick_mask(mn, mx, ot, 0.0, 1.0)
    W, H = 1920, 1080
    cam = synth.orbit_camera(dims, W, H, theta=0.7, phi=0.35, dist=1.6)
    xy = _pixels(W, H, 96, seed=5)
    ref, _ = ora.render_pixels(ov, ot, cam, W, H, xy, dt=0.5, ert=0.99, threads=8)
    for kind, params in ((ess.GRID, {}), (ess.LBVH, {}), (ess.KD, dict(nbins=4, halting=1, mls=32))):
        st = ess.ess_build(ctx, vol, t, kind, ess.build_params(brick=8, **params))
        assert np.array_equal(ess.ess_structure_read(ctx, st, ess.ARR_MASK), ref_mask)
        out = torch.empty((H, W, 4), dtype=torch.float32, device="cuda")
        ess.ess_render(ctx, st, cam, ess.render_params(0.5, 0.99), W, H, out)
        ess.ess_sync(ctx)
        _check_pixels(out.cpu().numpy(), xy, ref, "fractal1024 %s" % ess.KIND_NAMES[kind])
        ess.ess_release(ctx, st)


def test_ct512_shaded_sampled_pixels(gpu, ctx, ora, ct512):
    """The second render workload at the benchmark's size: gradient shading
    and opacity correction (dt 0.5 against dt_ref 1) on full 1024^2 frames of
    the 512^3 workload, sampled pixels against the oracle."""
    ess, torch = gpu
    vol_np, tfs, cams = ct512
    W = H = 1024
    shade = (0.25, 0.6, 0.3, 12)
    ov = ora.OVolume(vol_np, 0, 255)
    vol = ess.ess_volume_upload(ctx, torch.from_numpy(vol_np).cuda(), 0, 255)
    rp = ess.render_params(0.5, 0.99, shade=shade, dt_ref=1.0)
    for ti in (2, 6):
        ot = ora.OTF(tfs[ti])
        t = ess.ess_tf_set(ctx, torch.from_numpy(tfs[ti]).cuda())
        xy = _pixels(W, H, 128, seed=10 + ti)
        ref, _ = ora.render_pixels(ov, ot, cams[ti], W, H, xy, dt=0.5, ert=0.99, threads=8,
                                   shade=shade, dt_ref=1.0)
        for kind, params in ((ess.GRID, {}), (ess.LBVH, {}),
                             (ess.KD, dict(nbins=4, halting=1, mls=32))):
            st = ess.ess_build(ctx, vol, t, kind, ess.build_params(brick=8, **params))
            out = torch.empty((H, W, 4), dtype=torch.float32, device="cuda")
            ess.ess_render(ctx, st, cams[ti], rp, W, H, out)
            ess.ess_sync(ctx)
            _check_pixels(out.cpu().numpy(), xy, ref,
                          "ct512 shaded TF %d %s" % (ti, ess.KIND_NAMES[kind]))
            ess.ess_release(ctx, st)
        ess.ess_release(ctx, t)
