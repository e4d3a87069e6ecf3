"""The serving loop: requests (renders and TF edits) submitted from another
thread while earlier batches run are admitted by memory, batched, and each
result equals the same request rendered alone (bit for bit, hence within
2e-5), in submission order per structure.  Every served image is also checked
against the oracle's naive marching (no skipping) of the same volume, camera
and transfer function -- the one in force after the structure's edits up to
that request -- within 2e-5 per channel: skipping reproduces the naive image
(paper Sec. 1-2, Table 2 "Naive"), in the mix as alone."""
import threading
import time

import numpy as np
import pytest

from paper_1912_09596_gb300 import synth
from gpu_util import assert_image_parity, bits, upload

pytestmark = pytest.mark.gpu


def _volumes():
    """(array, value_lo, value_hi) of the three served volumes (u8, u16, f32)."""
    rng3, rng4 = np.random.default_rng(3), np.random.default_rng(4)
    vols = [(synth.blobs_u8((48, 40, 56), n_blobs=6, seed=1), 0, 255),
            (synth.blobs_u8((32, 32, 32), n_blobs=4, seed=2).astype(np.uint16) * 200, 0, 65535),
            (np.where(rng3.random((24, 40, 32)) < 0.8, 0, rng4.uniform(0, 1, (24, 40, 32)))
             .astype(np.float32), 0.0, 1.0)]
    return vols


def _initial_tf(i, k):
    return synth.tf_piecewise_random(256, seed=10 * i + k)


def _scene(ess, torch, ctx):
    """3 volumes (u8, u16, f32) x 3 structure kinds, each with its own TF.
    Returns [(structure, dims, tf handle)]."""
    out = []
    for i, (v, lo, hi) in enumerate(_volumes()):
        vol, _ = upload(ess, torch, ctx, v, lo, hi, synth.tf_ramp(256, 40))
        for k, kind in enumerate((ess.GRID, ess.LBVH, ess.KD)):
            t = ess.ess_tf_set(ctx, _initial_tf(i, k))
            st = ess.ess_build(ctx, vol, t, kind, ess.build_params(brick=4 + 4 * (k % 2)))
            out.append((st, v.shape[::-1], t))
    return out


def _requests(ess, n_scene, n, seed):
    rng = np.random.default_rng(seed)
    sizes = [(32, 32), (64, 48), (17, 61), (96, 64)]
    reqs = []
    for i in range(n):
        j = int(rng.integers(n_scene))
        W, H = sizes[int(rng.integers(len(sizes)))]
        edit = rng.random() < 0.3
        reqs.append(dict(scene=j, W=W, H=H, edit=edit, cam_seed=int(rng.integers(1 << 30)),
                         rgba=synth.tf_piecewise_random(256, seed=1000 + i) if edit else None,
                         ert=0.98 if rng.random() < 0.5 else 2.0,
                         out=np.full((H, W, 4), -1.0, np.float32)))
    return reqs


def _cam(r, dims):
    return synth.random_camera(dims, np.random.default_rng(r["cam_seed"]))


@pytest.mark.parametrize("budget_kb,max_batch,inflight", [(0, 256, 2), (128, 4, 3), (2048, 1, 1)])
def test_served_equals_alone(gpu, budget_kb, max_batch, inflight):
    ess, torch = gpu
    ctx = ess.ess_create(0, torch.cuda.current_stream())
    scene = _scene(ess, torch, ctx)
    reqs = _requests(ess, len(scene), 60, seed=budget_kb + max_batch)
    srv = ess.ess_server_create(ctx, memory_budget=budget_kb * 1024, max_batch=max_batch,
                                max_inflight=inflight)
    ids = []

    def producer():
        for r in reqs:
            st, dims, _ = scene[r["scene"]]
            ids.append(ess.ess_server_submit(
                srv, ess.REQ_EDIT if r["edit"] else ess.REQ_RENDER, st, _cam(r, dims),
                ess.render_params(0.5, r["ert"]), r["W"], r["H"], r["out"], rgba=r["rgba"]))
            time.sleep(0.0003)

    th = threading.Thread(target=producer)
    th.start()
    th.join()
    ess.ess_server_drain(srv)
    stats = [ess.ess_server_wait(srv, i) for i in ids]
    ess.ess_server_destroy(srv)
    ess.ess_destroy(ctx)
    assert all(s["done"] == 1 and s["status"] == ess.OK for s in stats)
    assert all(s["latency_ms"] >= s["queue_ms"] >= 0 for s in stats)
    _check_served_against_oracle(reqs)

    # alone: a fresh context with the same scene, one request at a time, in order
    ctx2 = ess.ess_create(0, torch.cuda.current_stream())
    scene2 = _scene(ess, torch, ctx2)
    for r in reqs:
        st, dims, t = scene2[r["scene"]]
        if r["edit"]:
            ess.ess_tf_update(ctx2, t, r["rgba"])
            ess.ess_rebuild(ctx2, st)
        out = torch.empty((r["H"], r["W"], 4), dtype=torch.float32, device="cuda")
        ess.ess_render(ctx2, st, _cam(r, dims), ess.render_params(0.5, r["ert"]), r["W"], r["H"],
                       out)
        ess.ess_sync(ctx2)
        assert np.array_equal(bits(out.cpu().numpy()), bits(r["out"])), "served != alone"
    ess.ess_destroy(ctx2)


def _check_served_against_oracle(reqs):
    """Every served image against the oracle's naive image of the same request,
    with the TF in force for its structure at that point of the submission
    order (an edit request renders with its own new table)."""
    import oracle as ora
    vols = [ora.OVolume(v, lo, hi) for v, lo, hi in _volumes()]
    tfs = {3 * i + k: _initial_tf(i, k) for i in range(3) for k in range(3)}
    kinds_after_edit = set()
    for n, r in enumerate(reqs):
        j = r["scene"]
        if r["edit"]:
            tfs[j] = r["rgba"]
            kinds_after_edit.add(j % 3)
        ov = vols[j // 3]
        ref, _ = ora.render_naive(ov, ora.OTF(tfs[j]), _cam(r, ov.dims), r["W"], r["H"],
                                  dt=0.5, ert=r["ert"])
        assert_image_parity(r["out"], ref, "served request %d (structure %d)" % (n, j))
    # the mix covered every structure kind, and each kind after an edit
    assert {r["scene"] % 3 for r in reqs} == {0, 1, 2}
    assert kinds_after_edit == {0, 1, 2}


def test_request_over_budget_is_refused(gpu):
    ess, torch = gpu
    ctx = ess.ess_create(0, torch.cuda.current_stream())
    scene = _scene(ess, torch, ctx)
    srv = ess.ess_server_create(ctx, memory_budget=1024, max_batch=8, max_inflight=2)
    out = np.zeros((64, 64, 4), np.float32)
    st, dims, _ = scene[0]
    rid = ess.ess_server_submit(srv, ess.REQ_RENDER, st, synth.orbit_camera(dims, 64, 64, 0.3),
                                ess.render_params(), 64, 64, out)
    s = ess.ess_server_wait(srv, rid)
    assert s["done"] == 1 and s["status"] == ess.ERR_BUSY
    ess.ess_server_destroy(srv)
    ess.ess_destroy(ctx)
