"""The benchmark's main workload is what its description says: the 512^3 CT-like
volume is deterministic in its seed, and its 8 TF edits leave 5-30 % of the
8^3 bricks non-empty (the range of the paper's data sets' occupancies is
0.15-50 %, Sec. 4.2).  Oracle min/max and range test, no GPU."""
import hashlib

import numpy as np

from paper_1912_09596_gb300 import synth


def test_ct512_recipe_occupancy_and_determinism(ora):
    small = [synth.ct_like_u8((64, 64, 64), seed=1) for _ in range(2)]
    assert hashlib.sha256(small[0].tobytes()).digest() == hashlib.sha256(small[1].tobytes()).digest()
    v = synth.ct_like_u8((512, 512, 512), seed=1)
    assert v.shape == (512, 512, 512) and v.dtype == np.uint8
    ov = ora.OVolume(v, 0, 255)
    mn, mx = ora.brick_minmax(ov, 8)
    occ = [float(ora.brick_mask(mn, mx, ora.OTF(tf), 0, 255).mean()) for tf in synth.tf_set_ct(256)]
    assert len(occ) == 8
    assert all(0.05 <= o <= 0.30 for o in occ), occ
    assert max(occ) - min(occ) > 0.1          # the edits really change the empty space


def test_blobs64_recipe_occupancy():
    """The small case (64^3 blobs, TF alpha 0 below 40 and a ramp above):
    about 10 % of the voxels are visible."""
    v = synth.blobs_u8((64, 64, 64), seed=0)
    frac = float((v >= 40).mean())
    assert 0.05 <= frac <= 0.2, frac
    tf = synth.tf_ramp(256, 40)
    assert np.all(tf[:40, 3] == 0) and np.all(tf[41:, 3] > 0)
