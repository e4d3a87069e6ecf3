"""The allocation-free compaction entry point (ess_compact_mask_noalloc), for
callers that cannot allocate device memory, called through the C ABI.

Its ids are checked against the oracle's compaction of the same mask
(ascending ids of the non-zero flags) and, where a volume produced the mask,
against the ids that the allocating path (ess_build) keeps, on calls in a row
(each reuses the shared scratch left by the one before).  Random masks of
4,194,305 and 16,777,216 flags cover more than 1024 tiles, where the tile scan
carries across its rounds, and the size limit itself.

This file is collected last on purpose."""
import ctypes

import numpy as np
import pytest

from paper_1912_09596_gb300 import synth

pytestmark = pytest.mark.gpu

LIMIT = 4096 * 4096   # flags one call accepts (4096 tiles of 4096 flags)


def _noalloc(ess, torch, stream, mask):
    n = mask.shape[0]
    mask_d = torch.from_numpy(np.ascontiguousarray(mask)).cuda()
    ids_d = torch.full((max(n, 1),), -1, dtype=torch.int32, device="cuda")
    count_d = torch.full((1,), -7, dtype=torch.int32, device="cuda")
    st = ess.lib.ess_compact_mask_noalloc(
        ctypes.c_void_p(mask_d.data_ptr()), n, ctypes.c_void_p(ids_d.data_ptr()),
        ctypes.c_void_p(count_d.data_ptr()), ctypes.c_void_p(stream.cuda_stream))
    assert st == ess.OK
    torch.cuda.synchronize()
    count = int(count_d.item())
    assert 0 <= count <= n
    return ids_d.cpu().numpy()[:count].view(np.uint32)


def test_compact_noalloc_matches_oracle_and_build(gpu, ora):
    ess, torch = gpu
    stream = torch.cuda.current_stream()
    ctx = ess.ess_create(0, stream)
    try:
        cases = [
            (synth.ct_like_u8((128, 128, 128), seed=1, n_vessels=6), synth.tf_set_ct()[3], 2),
            (synth.blobs_u8((40, 36, 44), n_blobs=5, seed=2), synth.tf_ramp(256, 40), 4),
        ]
        for v, tf, B in cases:       # two calls in a row, the second one smaller
            ov, ot = ora.OVolume(v, 0, 255), ora.OTF(tf)
            mask = ora.build_mask(ov, ot, B)
            got = _noalloc(ess, torch, stream, mask)
            assert len(got) > 0
            assert np.array_equal(got, ora.compact(mask))
            # the allocating path (mask, compaction and ids of ess_build) agrees
            vol = ess.ess_volume_upload(ctx, torch.from_numpy(v).cuda(), 0, 255)
            t = ess.ess_tf_set(ctx, torch.from_numpy(tf).cuda())
            st = ess.ess_build(ctx, vol, t, ess.GRID, ess.build_params(brick=B))
            assert np.array_equal(got, ess.ess_structure_read(ctx, st, ess.ARR_IDS))
            ess.ess_release(ctx, st)
    finally:
        ess.ess_destroy(ctx)


@pytest.mark.parametrize("n,p", [(LIMIT // 4 + 1, 0.3), (LIMIT, 0.05), (5, 1.0), (1, 0.0)])
def test_compact_noalloc_large_and_edge_masks(gpu, ora, n, p):
    """Seeded random byte masks (any non-zero byte is a flag) past 1024 tiles
    and at the limit, then a tiny all-set and a single empty flag."""
    ess, torch = gpu
    rng = np.random.default_rng(n)
    mask = np.where(rng.random(n) < p, rng.integers(1, 256, n), 0).astype(np.uint8)
    for _ in range(2):           # the same mask twice: the scratch keeps old sums
        got = _noalloc(ess, torch, torch.cuda.current_stream(), mask)
        assert np.array_equal(got, ora.compact(mask))


def test_compact_noalloc_rejects_oversize(gpu):
    ess, torch = gpu
    z = ctypes.c_void_p(0)
    count_d = torch.zeros(1, dtype=torch.int32, device="cuda")
    assert ess.lib.ess_compact_mask_noalloc(z, LIMIT + 1, z, ctypes.c_void_p(count_d.data_ptr()),
                                            None) == ess.ERR_ARG
    assert ess.lib.ess_compact_mask_noalloc(z, -1, z, ctypes.c_void_p(count_d.data_ptr()),
                                            None) == ess.ERR_ARG
