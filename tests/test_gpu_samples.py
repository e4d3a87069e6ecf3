"""Sample counts of the skipping renders against the oracle.

Image parity cannot see a traversal that marches through empty space: the
extra samples there have zero opacity and leave the image unchanged.  So the
number of samples each structure's render takes (early termination off) is
compared with the oracle's brute-force rule-S enumeration over the
structure's leaf boxes: non-empty bricks for the grid, the LBVH and the
hybrid grid, leaf boxes for the k-d tree.  The GPU slab tests and DDA crossings round differently from
the oracle's, which can move the sample taken at either end of an interval,
hence a small relative tolerance."""
import numpy as np
import pytest

from paper_1912_09596_gb300 import synth
from gpu_util import upload

pytestmark = pytest.mark.gpu

TOL = 0.002  # relative; the margin samples at interval ends


def _cases():
    yield "ct96", synth.ct_like_u8((96, 96, 96), seed=1, n_vessels=8), synth.tf_set_ct()[3]
    yield "blobs64", synth.blobs_u8((64, 64, 64), seed=0), synth.tf_ramp(256, 40)
    yield "ragged", synth.blobs_u8((37, 53, 45), n_blobs=6, seed=4), \
        synth.tf_random_sparse(256, seed=5, p_zero=0.7)


@pytest.mark.parametrize("case", list(_cases()), ids=lambda c: c[0])
@pytest.mark.parametrize("B", [4, 8])
def test_sample_counts_match_oracle_boxes(gpu, ctx, ora, case, B):
    ess, torch = gpu
    name, v, tf = case
    vol, t = upload(ess, torch, ctx, v, 0, 255, tf)
    ov, ot = ora.OVolume(v, 0, 255), ora.OTF(tf)
    mask = ora.build_mask(ov, ot, B)
    grid = ov.grid(B)
    boxes = {ess.GRID: ora.brick_boxes(np.nonzero(mask)[0], grid, B, ov.dims)}
    boxes[ess.LBVH] = boxes[ess.GRID]
    boxes[ess.HYBRID] = boxes[ess.GRID]  # the grid inside the tree's leaves
    rng = np.random.default_rng(B)
    W, H = 80, 64
    cams = [synth.orbit_camera(v.shape[::-1], W, H, 0.7), synth.random_camera(v.shape[::-1], rng)]
    for kind in (ess.GRID, ess.LBVH, ess.KD, ess.HYBRID):
        halting, mls = (0, 0) if kind == ess.HYBRID else (1, 32)
        st = ess.ess_build(ctx, vol, t, kind, ess.build_params(brick=B, nbins=4, halting=halting,
                                                               mls=mls))
        if kind == ess.KD:
            nodes = ess.ess_structure_read(ctx, st, ess.ARR_KD_NODES).reshape(-1, 9)
            boxes[kind] = ora.kd_leaf_boxes(nodes, B, ov.dims)
        for cam in cams:
            out = torch.empty((H, W, 4), dtype=torch.float32, device="cuda")
            ess.ess_sample_count(ctx, reset=True)
            ess.ess_render(ctx, st, ess.camera_from(cam), ess.render_params(0.5, 2.0), W, H, out)
            n_gpu = ess.ess_sample_count(ctx, reset=True)
            _, n_ref = ora.render_boxes(ov, ot, cam, W, H, boxes[kind], dt=0.5, ert=2.0)
            assert abs(n_gpu - n_ref) <= max(8, TOL * n_ref), (name, B, ess.KIND_NAMES[kind], n_gpu, n_ref)
        ess.ess_release(ctx, st)
