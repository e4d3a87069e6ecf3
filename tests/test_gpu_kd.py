"""GPU parity of the level-synchronous k-d build (bit-exact node records) and
of the k-d renderer, against the oracle."""
import numpy as np
import pytest

from paper_1912_09596_gb300 import synth
from gpu_util import assert_image_parity, bits, render, upload

pytestmark = pytest.mark.gpu


def kd_height(nodes):
    if len(nodes) == 0:
        return 0
    depth = np.zeros(len(nodes), int)
    depth[0] = 1
    for i in range(len(nodes)):
        fc = nodes[i, 8]
        if fc >= 0:
            depth[fc] = depth[fc + 1] = depth[i] + 1
    return int(depth.max())


def check_kd(gpu, ctx, ora, v, lo, hi, tf, B, nbins, halting, mls):
    ess, torch = gpu
    vol, t = upload(ess, torch, ctx, v, lo, hi, tf)
    st = ess.ess_build(ctx, vol, t, ess.KD, ess.build_params(brick=B, nbins=nbins, halting=halting,
                                                             mls=mls))
    ov, ot = ora.OVolume(v, lo, hi), ora.OTF(tf)
    mask = ora.build_mask(ov, ot, B)
    ref = ora.kd_build(mask, ov.grid(B), B, ov.dims, nbins=nbins, halting=halting, mls=mls)
    got = ess.ess_structure_read(ctx, st, ess.ARR_KD_NODES).reshape(-1, 9)
    assert got.shape == ref.shape, (got.shape, ref.shape)
    assert np.array_equal(got, ref)
    info = ess.ess_structure_info_get(ctx, st)
    assert info["n_nodes"] == len(ref) and info["height"] == kd_height(ref)
    ess.ess_sync(ctx)
    return st, ov, ot


CASES = [
    ("blobs", lambda: synth.blobs_u8((72, 64, 56), n_blobs=9, seed=3), (0, 255), lambda: synth.tf_ramp(256, 40)),
    ("ct", lambda: synth.ct_like_u8((96, 96, 96), seed=1, n_vessels=8), (0, 255), lambda: synth.tf_set_ct()[2]),
    ("sparse", lambda: synth.random_u8((60, 50, 70), seed=5, p_zero=0.995), (0, 255),
     lambda: synth.tf_random_sparse(256, seed=5, p_zero=0.5)),
]


@pytest.mark.parametrize("case", CASES, ids=lambda c: c[0])
@pytest.mark.parametrize("nbins", [0, 2, 4])
@pytest.mark.parametrize("halting,mls", [(0, 0), (1, 0), (1, 32), (1, 16)])
@pytest.mark.parametrize("B", [4, 8])
def test_kd_nodes_bit_exact(gpu, ctx, ora, case, nbins, halting, mls, B):
    name, vf, (lo, hi), tff = case
    check_kd(gpu, ctx, ora, vf(), lo, hi, tff(), B, nbins, halting, mls)


@pytest.mark.parametrize("case", CASES[:2], ids=lambda c: c[0])
@pytest.mark.parametrize("env", [{"ESS_KD_GRAPH": "0"}, {"ESS_KD_PERSIST": "0"}, {}],
                         ids=["host_loop", "graph", "persistent"])
def test_kd_build_paths_equal_oracle(gpu, ctx, ora, case, env, monkeypatch):
    """The three drivers of a 4-bin build give the oracle's tree: the
    host-driven level loop (ESS_KD_GRAPH=0, the one per-kernel profilers
    need), the CUDA graph with a conditional while node (ESS_KD_PERSIST=0)
    and the default single cooperative launch."""
    name, vf, (lo, hi), tff = case
    for k in ("ESS_KD_GRAPH", "ESS_KD_PERSIST"):
        monkeypatch.delenv(k, raising=False)
    for k, val in env.items():
        monkeypatch.setenv(k, val)
    check_kd(gpu, ctx, ora, vf(), lo, hi, tff(), 8, 4, 1, 32)
    check_kd(gpu, ctx, ora, vf(), lo, hi, tff(), 4, 4, 0, 0)


def test_kd_menger_shallow_single_node(gpu, ctx, ora):
    """Table 1: the Menger sponge's shallow tree is one node (GPU builder)."""
    st, ov, ot = check_kd(gpu, ctx, ora, synth.menger_u8(81), 0, 255, synth.tf_ramp(256, 100),
                          8, 4, 0, 0)
    ess, _ = gpu
    assert ess.ess_structure_info_get(ctx, st)["n_nodes"] == 1


@pytest.mark.parametrize("nonempty", [0, 1, 2])
def test_kd_tiny(gpu, ctx, ora, nonempty):
    v = np.zeros((24, 24, 24), np.uint8)
    for (x, y, z) in [(2, 3, 4), (20, 18, 21)][:nonempty]:
        v[z, y, x] = 250
    st, ov, ot = check_kd(gpu, ctx, ora, v, 0, 255, synth.tf_ramp(256, 100), 4, 4, 1, 0)
    ess, torch = gpu
    cam = synth.orbit_camera(ov.dims, 33, 27, 2.0)
    ref, _ = ora.render_naive(ov, ot, cam, 33, 27)
    assert_image_parity(render(ess, torch, ctx, st, cam, 33, 27), ref, "kd tiny")


@pytest.mark.parametrize("ert", [2.0, 0.99])
def test_kd_render_matches_oracle_and_naive(gpu, ctx, ora, ert):
    ess, torch = gpu
    rng = np.random.default_rng(11)
    for name, vf, (lo, hi), tff in CASES:
        v, tf = vf(), tff()
        vol, t = upload(ess, torch, ctx, v, lo, hi, tf)
        naive = ess.ess_build(ctx, vol, t, ess.NONE)
        ov, ot = ora.OVolume(v, lo, hi), ora.OTF(tf)
        for (B, nbins, halting, mls) in [(4, 4, 1, 16), (8, 0, 0, 0), (8, 4, 1, 0)]:
            st = ess.ess_build(ctx, vol, t, ess.KD, ess.build_params(brick=B, nbins=nbins,
                                                                     halting=halting, mls=mls))
            for cam in (synth.random_camera(ov.dims, rng, ortho=False),
                        synth.random_camera(ov.dims, rng, ortho=True),
                        synth.axis_ortho_camera(ov.dims, axis=2, half=(B * 2.0, B * 2.0))):
                W, H = 41, 31
                ref, _ = ora.render_naive(ov, ot, cam, W, H, ert=ert)
                got = render(ess, torch, ctx, st, cam, W, H, ert=ert)
                assert_image_parity(got, ref, "%s kd" % name)
                assert np.array_equal(bits(got), bits(render(ess, torch, ctx, naive, cam, W, H,
                                                             ert=ert)))
            ess.ess_release(ctx, st)


@pytest.mark.parametrize("threshold", [8, 9])
def test_kd_and_lbvh_over_258k_bricks(gpu, ctx, ora, threshold):
    """Over 155,648 non-empty bricks (2^3 bricks of a 128^3 volume, nearly all
    non-empty): the cooperative k-d build keeps its bricks' nodes in a device
    array instead of registers, and the LBVH's node boxes use chunks of 32768
    leaves.  Both trees equal the oracle's, and the images the naive march."""
    from test_gpu_lbvh import check_lbvh
    ess, torch = gpu
    v = synth.blobs_u8((128, 128, 128), n_blobs=12, seed=21)
    tf = synth.tf_ramp(256, threshold)
    vol, t = upload(ess, torch, ctx, v, 0, 255, tf)
    ov, ot = ora.OVolume(v, 0, 255), ora.OTF(tf)
    mask = ora.build_mask(ov, ot, 2)
    assert int(mask.sum()) > 4 * 152 * 256
    st, _, _ = check_kd(gpu, ctx, ora, v, 0, 255, tf, 2, 4, 1, 32)
    lb = ess.ess_build(ctx, vol, t, ess.LBVH, ess.build_params(brick=2))
    check_lbvh(ess, ctx, lb, ora.lbvh_build(mask, ov.grid(2)))
    naive = ess.ess_build(ctx, vol, t, ess.NONE)
    cam = synth.orbit_camera(ov.dims, 48, 40, theta=0.7, phi=0.3)
    ref = render(ess, torch, ctx, naive, cam, 48, 40)
    for s in (st, lb):
        assert np.array_equal(bits(render(ess, torch, ctx, s, cam, 48, 40)), bits(ref))
