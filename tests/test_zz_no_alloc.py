"""The allocation-free compaction entry point (ess_compact_mask_noalloc), for
callers that cannot allocate device memory, called through the C ABI and
checked against the ids that ess_build keeps for the same mask, on two calls
in a row (the second reuses the shared scratch left by the first).

This file is collected last on purpose."""
import ctypes

import numpy as np
import pytest

from paper_1912_09596_gb300 import synth

pytestmark = pytest.mark.gpu


def _reference(ess, torch, ctx, v, tf, B):
    vol = ess.ess_volume_upload(ctx, torch.from_numpy(v).cuda(), 0, 255)
    t = ess.ess_tf_set(ctx, torch.from_numpy(tf).cuda())
    st = ess.ess_build(ctx, vol, t, ess.GRID, ess.build_params(brick=B))
    mask = ess.ess_structure_read(ctx, st, ess.ARR_MASK)
    ids = ess.ess_structure_read(ctx, st, ess.ARR_IDS)
    return mask, ids


def test_compact_noalloc_matches_build_twice(gpu):
    ess, torch = gpu
    stream = torch.cuda.current_stream()
    ctx = ess.ess_create(0, stream)
    try:
        cases = [
            (synth.ct_like_u8((128, 128, 128), seed=1, n_vessels=6), synth.tf_set_ct()[3], 2),
            (synth.blobs_u8((40, 36, 44), n_blobs=5, seed=2), synth.tf_ramp(256, 40), 4),
        ]
        for v, tf, B in cases:       # two calls in a row, the second one smaller
            mask, ids_ref = _reference(ess, torch, ctx, v, tf, B)
            n = mask.shape[0]
            mask_d = torch.from_numpy(mask).cuda()
            ids_d = torch.full((n,), -1, dtype=torch.int32, device="cuda")
            count_d = torch.full((1,), -7, dtype=torch.int32, device="cuda")
            st = ess.lib.ess_compact_mask_noalloc(
                ctypes.c_void_p(mask_d.data_ptr()), n, ctypes.c_void_p(ids_d.data_ptr()),
                ctypes.c_void_p(count_d.data_ptr()), ctypes.c_void_p(stream.cuda_stream))
            assert st == ess.OK
            torch.cuda.synchronize()
            count = int(count_d.item())
            got = ids_d.cpu().numpy()[:count].view(np.uint32)
            assert count == len(ids_ref) and count > 0
            assert np.array_equal(got, ids_ref)
    finally:
        ess.ess_destroy(ctx)


def test_compact_noalloc_rejects_oversize(gpu):
    ess, torch = gpu
    z = ctypes.c_void_p(0)
    count_d = torch.zeros(1, dtype=torch.int32, device="cuda")
    too_big = 4096 * 4096 + 1
    assert ess.lib.ess_compact_mask_noalloc(z, too_big, z, ctypes.c_void_p(count_d.data_ptr()),
                                            None) == ess.ERR_ARG
    assert ess.lib.ess_compact_mask_noalloc(z, -1, z, ctypes.c_void_p(count_d.data_ptr()),
                                            None) == ess.ERR_ARG
