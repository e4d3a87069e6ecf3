#!/usr/bin/env python3
"""Benchmark of the empty-space-skipping hot path on one GB300 (per rank).

A step is one pass of the whole hot path over the 512^3 CT-like workload:
for each of 8 transfer-function edits, the TF table is replaced, every
skipping structure (macrocell grid, LBVH, k-d tree) is rebuilt from it and a
1024 x 1024 frame is rendered through each structure (dt 0.5, early ray
termination at opacity 0.99; the camera rotates by 45 degrees per edit).

value: ray samples per second, counting for every frame the samples the naive
       (non-skipping) marcher takes for that frame, i.e. the work each image
       stands for; the time covers TF upload, rebuilds and renders, with all
       inputs resident in device memory.  The samples the skipping renderers
       actually evaluate are reported beside it.
e2e:   the same metric through the C ABI with host buffers: TF tables copied
       from pinned host memory and every frame read back to pinned host memory
       inside the timed region.

`--impl reference` times the CPU oracle (the plain definition: naive marcher)
on the same workload instead; under torchrun only rank 0 runs it.

Multi-GPU: the path does not shard; N ranks run N independent replicas (weak
scaling), timed between barriers with the maximum over ranks.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

WORKLOADS = {
    "ct512": dict(
        desc="512^3 uint8 CT-like volume (noisy shells, vessels, 2% smooth noise); "
             "8 TF edits with 5-30% non-empty 8^3 bricks; rebuild per edit; "
             "1024x1024 perspective, dt 0.5 voxel, ERT 0.99",
        dims=(512, 512, 512), W=1024, H=1024, dt=0.5, ert=0.99, brick=8),
    "fractal1024": dict(
        desc="1024^3 float32 fractal field (4 octaves of value noise, thresholded: 1-5% "
             "non-empty 8^3 bricks), 1024-entry TF; one TF upload and rebuild of every "
             "structure, then 16 orbit views at 1920x1080 perspective, dt 0.5 voxel, no ERT",
        dims=(1024, 1024, 1024), W=1920, H=1080, dt=0.5, ert=2.0, brick=8),
    "blobs64": dict(
        desc="64^3 uint8 Gaussian blobs, TF ramp from 40, brick 8^3, 256x256 perspective, "
             "dt 0.5, no ERT", dims=(64, 64, 64), W=256, H=256, dt=0.5, ert=2.0, brick=8),
}
KD_PARAMS = dict(nbins=4, halting=1, mls=32)   # GPU k-d, deep, maximum leaf 32^3 (Sec. 4.3)
FALLBACK_HBM_GBS = 6800.0
L2_FLUSH_BYTES = 512 << 20
FP32_LANES_PER_SM = 128
# FP32 operations of one evaluated sample as the method defines it (FMA = 2):
# position 3 FMA (6); cell weights 3 floor + 3 sub (6); trilinear 7 x (sub +
# FMA) (21); TF coordinate FMA + 2 clamps + floor + sub (6); TF lerp 4 x (sub +
# FMA) (12); compositing sub, mul, 3 FMA, add (9); termination compare (1).
FLOP_PER_SAMPLE = 61

# The bench.py argument lists of the runs that the summaries under profiles/
# were captured from (each summary names its entry); a CPU test parses them all.
PROFILE_COMMANDS = {
    "step_ct512": "--steps 1 --warmup 1 --no-cpu-baseline --no-batched --no-serve --no-minmax "
                  "--no-hybrid --no-structures --no-shaded --no-cell-vote --no-fractal",
    "step_ct512_shaded": "--steps 1 --warmup 1 --no-cpu-baseline --no-batched --no-serve "
                         "--no-minmax --no-hybrid --no-structures --no-cell-vote --no-fractal",
    "step_ct512_hybrid": "--steps 1 --warmup 1 --no-cpu-baseline --no-batched --no-serve "
                         "--no-minmax --no-structures --no-shaded --no-cell-vote --no-fractal",
    "step_ct512_vote_batch": "--steps 1 --warmup 1 --no-cpu-baseline --no-serve --no-minmax "
                             "--no-hybrid --no-structures --no-shaded --no-fractal",
    "step_ct512_vote": "--steps 1 --warmup 1 --no-cpu-baseline --no-batched --no-serve "
                       "--no-minmax --no-hybrid --no-structures --no-shaded --no-fractal",
    "step_ct512_hybrid_only": "--steps 1 --warmup 1 --no-cpu-baseline --no-batched --no-serve "
                              "--no-minmax --no-structures --no-shaded --no-cell-vote --no-fractal",
    "step_fractal1024": "--workload fractal1024 --steps 1 --warmup 1 --no-cpu-baseline "
                        "--no-batched --no-minmax",
    "bench_default": "",
}


def make_inputs(name, dev=None):
    """Volume (numpy, or a torch tensor for the 1024^3 field), value range,
    the TF tables of the edits and, per edit, the cameras rendered after it."""
    from paper_1912_09596_gb300 import synth
    w = WORKLOADS[name]
    if name == "fractal1024":
        vol = synth.fractal_f32_torch(w["dims"], seed=2, device=dev if dev is not None else "cpu")
        tfs = [synth.tf_ramp(1024, 2)]
        views = [[synth.orbit_camera(w["dims"], w["W"], w["H"], theta=2 * math.pi * k / 16,
                                     phi=0.35, dist=1.6) for k in range(16)]]
        return vol, (0.0, 1.0), tfs, views
    if name == "ct512":
        vol = synth.ct_like_u8(w["dims"], seed=1)
        tfs = synth.tf_set_ct(256)
    else:
        vol = synth.blobs_u8(w["dims"], seed=0)
        tfs = [synth.tf_ramp(256, 40) for _ in range(8)]
    views = [[synth.orbit_camera(w["dims"], w["W"], w["H"], theta=2 * math.pi * i / len(tfs),
                                 phi=0.35, dist=1.6)] for i in range(len(tfs))]
    return vol, (0.0, 255.0), tfs, views


def host_array(vol):
    """The volume as a host numpy array (the oracle's input)."""
    return vol if isinstance(vol, np.ndarray) else vol.cpu().numpy()


# ---------------------------------------------------------------- clocks
class ClockSampler:
    """nvidia-smi samples of SM clock and throttle reasons while running."""
    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device):
        self.lines = []
        try:
            self.p = subprocess.Popen(
                ["nvidia-smi", "--id=%d" % device, "--query-gpu=" + self.FIELDS,
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except (OSError, ValueError):
            self.p = None

    def _read(self):
        for line in self.p.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.p is None:
            return None
        self.p.terminate()
        try:
            self.p.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.p.kill()
        self.t.join(timeout=5)
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 8:
                continue
            try:
                sm.append(float(f[0]))
                mx.append(float(f[1]))
            except ValueError:
                continue
            for n, v in zip(names, f[4:8]):
                if v.lower().startswith("active"):
                    reasons.add(n)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_min_mhz": min(sm), "sm_max_mhz": max(mx),
                "reasons": sorted(reasons), "samples": len(sm)}


# ---------------------------------------------------------------- helpers
def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except (OSError, KeyError, ValueError):
        return FALLBACK_HBM_GBS, "fallback"


def fp32_peak_tflops(sms):
    """FP32 roof from unit counts and the maximum SM clock: the device's SMs x
    128 FP32 lanes x 2 FLOP per FMA x clock."""
    mhz = 2070.0
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            mhz = float(json.load(f).get("sm_max_mhz", mhz))
    except (OSError, ValueError):
        pass
    return sms * FP32_LANES_PER_SM * 2 * mhz * 1e6 / 1e12, mhz


# source files that define each kernel (by profiling-name prefix); every
# kernel also depends on the shared internal header
KERNEL_FILES = (("render_shaded", ("render_shaded.cu", "render_kernels.h")),
                ("render", ("render.cu", "render_kernels.h")),
                ("brick_minmax", ("classify.cu", "minmax_tma.cu")), ("brick_", ("classify.cu",)),
                ("compact", ("classify.cu",)), ("tf_prefix", ("classify.cu",)),
                ("vote_bricks", ("classify.cu",)), ("build_cells", ("classify.cu",)),
                ("check_finite", ("classify.cu",)), ("sort", ("lbvh.cu",)),
                ("lbvh", ("lbvh.cu",)), ("kd", ("kd.cu",)))


def kernel_source_sha(kernel):
    """Hash of the source files that define `kernel` (None if unknown)."""
    for prefix, fnames in KERNEL_FILES:
        if kernel.startswith(prefix):
            break
    else:
        return None
    h = hashlib.sha256()
    csrc = os.path.join(ROOT, "paper_1912_09596_gb300", "csrc")
    for f in fnames + ("ess_internal.h",):
        with open(os.path.join(csrc, f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def ncu_traffic(kernel, workload):
    """dram bytes per launch recorded by an ncu capture (profiles/traffic.txt),
    valid only if the kernel's sources are unchanged since the capture."""
    path = os.path.join(ROOT, "profiles", "traffic.txt")
    if not os.path.exists(path):
        return None
    sha = kernel_source_sha(kernel)
    for line in open(path):
        f = line.split()
        if len(f) >= 4 and not line.startswith("#") and f[0] == kernel and f[1] == workload \
                and f[3] == sha:
            return float(f[2])
    return None


def dist_setup():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    if ws <= 1:
        return 0, 0, 1, None
    import torch.distributed as dist
    rank = int(os.environ["RANK"])
    local = int(os.environ.get("LOCAL_RANK", rank))
    return rank, local, ws, dist


def max_over_ranks(dist, x, device):
    """The largest of the ranks' values of x (each rank's timing): the job
    is as slow as its slowest replica.  x itself when there is one rank."""
    if not dist:
        return float(x)
    import torch
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_rate(units_per_rank_step, world_size, steps, ms):
    """Whole-job throughput of `world_size` replicas that each process
    `units_per_rank_step` units per step, over `steps` steps in `ms`
    milliseconds (the max over ranks)."""
    return world_size * units_per_rank_step * steps / (ms / 1000.0)


# ---------------------------------------------------------------- reference
def cpu_cores():
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count() or 1


def oracle_rate(vol_np, vlo, vhi, tf_np, cam, w, budget_s, threads):
    """Naive CPU marcher (the oracle) on a stripe of rows of one frame, sized
    to about `budget_s` seconds.  Returns (samples/s, description)."""
    import oracle
    ov, ot = oracle.OVolume(vol_np, vlo, vhi), oracle.OTF(tf_np)
    W, H = w["W"], w["H"]
    y0 = H // 2 - 2
    t0 = time.perf_counter()
    _, n0 = oracle.render_naive(ov, ot, cam, W, H, dt=w["dt"], ert=w["ert"], rows=(y0, y0 + 4),
                                threads=threads)
    probe = time.perf_counter() - t0
    rows = int(max(4, min(H, 4 * budget_s / max(probe, 1e-3))))
    ya = max(0, H // 2 - rows // 2)
    yb = min(H, ya + rows)
    t0 = time.perf_counter()
    _, n = oracle.render_naive(ov, ot, cam, W, H, dt=w["dt"], ert=w["ert"], rows=(ya, yb),
                               threads=threads)
    dt = time.perf_counter() - t0
    return n / dt, "rows %d..%d of a %dx%d frame (%d samples, %.1f s, %d threads)" % (
        ya, yb, W, H, n, dt, threads)


def run_reference(args, rank):
    if rank != 0:
        return
    w = WORKLOADS[args.workload]
    vol, (vlo, vhi), tfs, views = make_inputs(args.workload)
    vol = host_array(vol)
    cams = [(tfs[i], c) for i, vs in enumerate(views) for c in vs]
    cores = cpu_cores()
    for _ in range(args.warmup):
        oracle_rate(vol, vlo, vhi, cams[0][0], cams[0][1], w, 0.2, cores)
    rates, descs, t_all = [], [], 0.0
    for k in range(args.steps):
        tf_k, cam_k = cams[k % len(cams)]
        t0 = time.perf_counter()
        r, d = oracle_rate(vol, vlo, vhi, tf_k, cam_k, w, args.ref_budget, cores)
        t_all += time.perf_counter() - t0
        rates.append(r)
        descs.append(d)
    value = float(statistics.mean(rates))
    out = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "samples/s",
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": 1000.0 * t_all / max(1, args.steps), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": args.workload + ": " + w["desc"]},
        "cpu_baseline": {"value": value, "unit": "samples/s", "cores": cores, "kind": "oracle",
                         "sample": "per step: " + descs[0]},
        "e2e": {"value": value, "unit": "samples/s", "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0},
    }
    print(json.dumps(out))


METRIC = ("ray samples/s, naive-equivalent (per frame, the samples the non-skipping marcher "
          "takes; the samples the skipping renderers evaluate are in evaluated_samples_per_s), over "
          "TF edit + rebuild + render of grid, LBVH and k-d structures")

BATCH_SIZES = [(256, 256), (512, 512), (1024, 1024), (1920, 1080)]


def run_batched(ess, torch, dev, stream, ctx, reps=3):
    """512^3 uint16 volume x 64 random piecewise-linear TFs x 4 views with
    image sizes drawn from 256^2 .. 1920x1080: autotuned structure kind, brick
    and tile shape; 256 sequential ess_render calls against one
    ess_render_batch launch (captured graph), same outputs."""
    from paper_1912_09596_gb300 import synth
    dims = (512, 512, 512)
    v = synth.ct_like_u16(dims, seed=3)
    vol = ess.ess_volume_upload(ctx, torch.from_numpy(v).to(dev), 0, 65535)
    del v
    tfs = [synth.tf_piecewise_random(1024, seed=500 + i) for i in range(64)]
    tf_handles = [ess.ess_tf_set(ctx, torch.from_numpy(t).to(dev)) for t in tfs]
    rng = np.random.default_rng(42)
    views = [synth.orbit_camera(dims, 1024, 1024, theta=float(rng.uniform(0, 2 * math.pi)),
                                phi=float(rng.uniform(-0.6, 0.6)), dist=1.7) for _ in range(4)]
    rp = ess.render_params(0.5, 0.99)
    best = ess.ess_autotune(ctx, vol, tf_handles[0], views[:2], rp, 1024, 1024, frames_per_edit=4.0)
    kdp = dict(KD_PARAMS)
    sts = [ess.ess_build(ctx, vol, t, best["kind"], ess.build_params(brick=best["brick"], **kdp))
           for t in tf_handles]
    items_plain, items_batch = [], []
    for i in range(256):
        W, H = BATCH_SIZES[int(rng.integers(len(BATCH_SIZES)))]
        cam = synth.orbit_camera(dims, W, H, theta=2 * math.pi * (i % 4) / 4 + 0.3, phi=0.3, dist=1.7)
        st = sts[i // 4]
        items_plain.append((st, cam, W, H, torch.empty((H, W, 4), dtype=torch.float32, device=dev)))
        items_batch.append((st, cam, rp, W, H, torch.empty((H, W, 4), dtype=torch.float32, device=dev)))
    rpt = ess.render_params(0.5, 0.99, tile_w=best["tile_w"])
    ecams = [ess.camera_from(it[1]) for it in items_plain]

    def plain():
        for (st, cam, W, H, out), ec in zip(items_plain, ecams):
            ess.ess_render(ctx, st, ec, rpt, W, H, out)

    def batched():
        ess.ess_render_batch(ctx, items_batch, tile_w=best["tile_w"])

    def timeit(fn):
        fn()
        torch.cuda.synchronize(dev)
        ts = []
        for _ in range(reps):
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            fn()
            b.record(stream)
            torch.cuda.synchronize(dev)
            ts.append(a.elapsed_time(b))
        return float(np.median(ts))

    t_plain = timeit(plain)
    t_batch = timeit(batched)
    same = all(torch.equal(a[4], b[5]) for a, b in zip(items_plain, items_batch))
    pixels = sum(W * H for (_, _, W, H, _) in items_plain)
    out = {"workload": "512^3 uint16 CT-like, 64 random piecewise-linear TFs (1024 entries) x 4 "
                       "views, image sizes drawn from 256^2, 512^2, 1024^2, 1920x1080, dt 0.5, "
                       "ERT 0.99",
           "images": 256, "megapixels": round(pixels / 1e6, 2),
           "autotune": {"kind": ess.KIND_NAMES[best["kind"]], "brick": best["brick"],
                        "tile_w": best["tile_w"], "build_ms": round(best["build_ms"], 3),
                        "render_ms_1024sq": round(best["render_ms"], 3)},
           "plain_ms": round(t_plain, 3), "batched_ms": round(t_batch, 3),
           "plain_frames_per_s": 256 / (t_plain / 1000.0),
           "batched_frames_per_s": 256 / (t_batch / 1000.0),
           "speedup": t_plain / t_batch, "bit_identical": bool(same)}
    out["rebuild"] = run_rebuild_batch(ess, torch, dev, ctx, vol, tf_handles, sts, reps)
    for st in sts:
        ess.ess_release(ctx, st)
    for t in tf_handles:
        ess.ess_release(ctx, t)
    ess.ess_release(ctx, vol)
    return out


def run_rebuild_batch(ess, torch, dev, ctx, vol, tf_handles, sts, reps):
    """The batched build of the TF structures: one ess_rebuild per structure
    against one ess_rebuild_batch of them all, host wall time from the first
    call to the end of the last build (median of `reps`), for the render
    batch's 64 autotuned structures and for 16 TFs x {grid, LBVH, k-d} built
    with a min/max rescan (the benchmark step's parameters).  The batch's
    masks must equal the one-by-one rebuilds' masks."""
    def wall(fn):
        fn()
        ess.ess_sync(ctx)
        ts = []
        for _ in range(reps):
            torch.cuda.synchronize(dev)
            t0 = time.perf_counter()
            fn()
            ess.ess_sync(ctx)
            ts.append(1000.0 * (time.perf_counter() - t0))
        return float(np.median(ts))

    def compare(handles):
        one = lambda: [ess.ess_rebuild(ctx, h) for h in handles]
        batch = lambda: ess.ess_rebuild_batch(ctx, handles)
        t_one, t_batch = wall(one), wall(batch)
        masks = [ess.ess_structure_read(ctx, h, ess.ARR_MASK) for h in handles]
        one()
        same = all(np.array_equal(m, ess.ess_structure_read(ctx, h, ess.ARR_MASK))
                   for m, h in zip(masks, handles))
        return {"structures": len(handles), "one_by_one_ms": round(t_one, 3),
                "batched_ms": round(t_batch, 3), "speedup": round(t_one / t_batch, 2),
                "masks_identical": bool(same)}

    res = {"autotuned_64": compare(sts)}
    mixed = []
    for t in tf_handles[:16]:
        for k in (ess.GRID, ess.LBVH, ess.KD):
            mixed.append(ess.ess_build(ctx, vol, t, k, ess.build_params(brick=8, rescan=1,
                                                                        **KD_PARAMS)))
    res["grid_lbvh_kd_48_rescan"] = compare(mixed)
    for h in mixed:
        ess.ess_release(ctx, h)
    return res


SERVE_SIZES = [(256, 256), (512, 512), (1024, 768), (1920, 1080)]


def serve_scene(ess, torch, dev, ctx, ct512):
    """6 resident volumes from the workload generators, each with one
    structure (kinds in turn) and its own TF."""
    from paper_1912_09596_gb300 import synth
    vols = [("128^3 u8 blobs", synth.blobs_u8((128, 128, 128), seed=0), 0, 255, 256),
            ("256^3 u8 blobs", synth.blobs_u8((256, 256, 256), n_blobs=24, seed=5), 0, 255, 256),
            ("512^3 u8 CT-like", ct512, 0, 255, 256),
            ("256^3 f32 fractal", synth.fractal_f32((256, 256, 256), seed=2), 0.0, 1.0, 1024),
            ("512^3 u16 CT-like", synth.ct_like_u16((512, 512, 512), seed=3), 0, 65535, 1024),
            ("1024^3 f32 fractal", None, 0.0, 1.0, 1024)]
    scene = []
    kinds = [ess.GRID, ess.LBVH, ess.KD]
    for i, (name, v, lo, hi, nt) in enumerate(vols):
        if v is None:
            data = synth.fractal_f32_torch((1024, 1024, 1024), seed=2, device=dev)
            dims = (1024, 1024, 1024)
        else:
            data = torch.from_numpy(v).to(dev)
            dims = v.shape[::-1]
        vol = ess.ess_volume_upload(ctx, data, lo, hi)
        del data
        tf0 = synth.tf_piecewise_random(nt, seed=700 + i)
        t = ess.ess_tf_set(ctx, torch.from_numpy(tf0).to(dev))
        kind = kinds[i % 3]
        st = ess.ess_build(ctx, vol, t, kind, ess.build_params(brick=8, **KD_PARAMS))
        scene.append(dict(name=name, vol=vol, tf=t, st=st, dims=dims, nt=nt, kind=kind, tf0=tf0))
    torch.cuda.synchronize(dev)
    return scene


def serve_requests(ess, scene, n, seed):
    from paper_1912_09596_gb300 import synth
    rng = np.random.default_rng(seed)
    reqs = []
    for i in range(n):
        j = int(rng.integers(len(scene)))
        W, H = SERVE_SIZES[int(rng.integers(len(SERVE_SIZES)))]
        edit = rng.random() < 0.3
        cam = synth.orbit_camera(scene[j]["dims"], W, H, theta=float(rng.uniform(0, 2 * math.pi)),
                                 phi=float(rng.uniform(-0.6, 0.6)), dist=float(rng.uniform(1.4, 2.2)))
        reqs.append(dict(scene=j, W=W, H=H, edit=edit, cam=ess.camera_from(cam),
                         rgba=synth.tf_piecewise_random(scene[j]["nt"], seed=9000 + i) if edit else None))
    return reqs


def run_served(ess, torch, dev, ctx, ct512, n_req=240, load=3.0):
    """Poisson stream of render and TF-edit requests (30 % edits) over 6
    resident volumes, image sizes 256^2 .. 1920x1080.  Serial plain processing
    (one request at a time through ess_render with a host image) against the
    continuous-batching server, both fed at the same arrival times; the rate is
    `load` times the serial service rate measured first, so that both arms are
    busy and their throughputs are their capacities."""
    import threading
    scene = serve_scene(ess, torch, dev, ctx, ct512)
    reqs = serve_requests(ess, scene, n_req, seed=11)
    outs = [torch.empty((r["H"], r["W"], 4), dtype=torch.float32).pin_memory() for r in reqs]
    rp = ess.render_params(0.5, 0.99)

    def serve_one(r, out):
        sc = scene[r["scene"]]
        if r["edit"]:
            ess.ess_tf_update(ctx, sc["tf"], r["rgba"])
            ess.ess_rebuild(ctx, sc["st"])
        ess.ess_render(ctx, sc["st"], r["cam"], rp, r["W"], r["H"], out)

    def reset():
        for sc in scene:
            ess.ess_tf_update(ctx, sc["tf"], sc["tf0"])
            ess.ess_rebuild(ctx, sc["st"])
        ess.ess_sync(ctx)

    # the request loops are host-driven: keep the interpreter's garbage
    # collector from pausing them (it is switched back on at the end)
    import gc
    gc.collect()
    gc.disable()
    # serial service rate: the whole request list back to back (requests differ
    # a lot in cost, so a short prefix would be a noisy estimate); median of
    # three passes after two untimed ones
    rates = []
    for _ in range(5):
        reset()
        t0 = time.perf_counter()
        for r, o in zip(reqs, outs):
            serve_one(r, o)
        ess.ess_sync(ctx)
        rates.append(n_req / (time.perf_counter() - t0))
    mu = float(np.median(rates[2:]))
    lam = load * mu
    gaps = np.random.default_rng(12).exponential(1.0 / lam, size=n_req)
    arrivals = np.cumsum(gaps)

    def run_serial():
        reset()
        lat = []
        start = time.perf_counter()
        for r, o, at in zip(reqs, outs, arrivals):
            now = time.perf_counter() - start
            if now < at:
                time.sleep(at - now)
            serve_one(r, o)
            lat.append((time.perf_counter() - start - at) * 1000.0)
        return lat, time.perf_counter() - start

    # one long-lived server for all repetitions, as a service would run (its
    # memory pool and batch graphs are set up once)
    srv = ess.ess_server_create(ctx, memory_budget=8 << 30, max_batch=64, max_inflight=2)

    def run_server():
        reset()
        ids = [None] * n_req
        t_sub = [0.0] * n_req
        start = time.perf_counter()

        def producer():
            for k, (r, o, at) in enumerate(zip(reqs, outs, arrivals)):
                now = time.perf_counter() - start
                if now < at:
                    time.sleep(at - now)
                sc = scene[r["scene"]]
                t_sub[k] = time.perf_counter() - start
                ids[k] = ess.ess_server_submit(srv, ess.REQ_EDIT if r["edit"] else ess.REQ_RENDER,
                                               sc["st"], r["cam"], rp, r["W"], r["H"], o,
                                               rgba=r["rgba"])

        th = threading.Thread(target=producer)
        th.start()
        th.join()
        ess.ess_server_drain(srv)
        span = time.perf_counter() - start
        st = [ess.ess_server_wait(srv, i) for i in ids]
        return st, t_sub, span

    # plain and served alternate REPS times at the same arrival times; each
    # arm reports its repetition of median throughput and the spread (the host is shared, so
    # a single repetition can catch a stall of either arm, the plain loop's
    # more often: it waits for every request).  Clocks are
    # sampled before and after the repetitions, not during them: an
    # nvidia-smi query can hold up these host-driven request loops.
    REPS = 7

    def clock_snapshot():
        sampler = ClockSampler(torch.cuda.current_device())
        time.sleep(0.5)
        return sampler.stop()

    clk_before = clock_snapshot()
    plain_runs, served_runs = [], []
    same = True
    for rep in range(REPS):
        lat_plain, span_plain = run_serial()
        plain_runs.append((n_req / span_plain, lat_plain))
        plain_imgs = [o.clone() for o in outs]
        for o in outs:
            o.fill_(-1.0)
        st, t_sub, span_served = run_server()
        served_runs.append((n_req / span_served, st, t_sub))
        # the served images must equal the serial ones: both apply the same edits in order
        same = same and all(torch.equal(a, b) for a, b in zip(plain_imgs, outs))
    clk = {"before": clk_before, "after": clock_snapshot()}
    gc.enable()
    ess.ess_server_destroy(srv)
    pct = lambda a, q: float(np.percentile(np.asarray(a), q))
    med = lambda runs: sorted(runs, key=lambda x: x[0])[len(runs) // 2]
    fps_plain, lat_plain = med(plain_runs)
    fps_served, st, t_sub = med(served_runs)
    spread = lambda runs: {"min": round(min(r[0] for r in runs), 1),
                           "median": round(med(runs)[0], 1),
                           "max": round(max(r[0] for r in runs), 1)}
    lat_served = [x["latency_ms"] for x in st]
    queue_ms = [x["queue_ms"] for x in st]
    # requests issued together share one launch time
    launches = {round(ts * 1000.0 + q, 2) for ts, q in zip(t_sub, queue_ms)}
    ok = all(x["status"] == ess.OK for r in served_runs for x in r[1])
    return {
        "workload": "6 resident volumes (" + ", ".join(s["name"] for s in scene) + "), kinds "
                    "grid/lbvh/kd in turn, brick 8; Poisson arrivals at %.1fx the serial service "
                    "rate, 30%% TF edits (rebuild), " % load +
                    "image sizes 256^2..1920x1080, dt 0.5, ERT 0.99; images read back to pinned "
                    "host memory",
        "requests": n_req, "rate_hz": round(lam, 2), "serial_service_rate_hz": round(mu, 2),
        "repetitions": REPS,
        "plain": {"frames_per_s": fps_plain, "p50_ms": pct(lat_plain, 50),
                  "p99_ms": pct(lat_plain, 99), "frames_per_s_spread": spread(plain_runs),
                  "frames_per_s_all": [round(r[0], 1) for r in plain_runs]},
        "served": {"frames_per_s": fps_served, "p50_ms": pct(lat_served, 50),
                   "p99_ms": pct(lat_served, 99), "all_ok": ok,
                   "mean_queue_ms": float(np.mean(queue_ms)),
                   "mean_service_ms": float(np.mean(np.subtract(lat_served, queue_ms))),
                   "batches": len(launches), "frames_per_s_spread": spread(served_runs),
                   "frames_per_s_all": [round(r[0], 1) for r in served_runs]},
        "bit_identical_to_plain": bool(same),
        "clocks": clk,
    }


def run_hybrid(ess, torch, dev, ctx, vol, tf, tf_dev, ecams, rp, W, H, steps=3):
    """The hybrid grid (Sec. 3.3: a shallow k-d tree whose leaves are crossed
    with the macrocell grid) on the main workload's TF edits: rebuild and one
    frame per edit, CUDA-event time per kernel, for 16^3 and 8^3 bricks."""
    out = torch.empty((H, W, 4), dtype=torch.float32, device=dev)
    res = {}
    for B in (16, 8):
        st = ess.ess_build(ctx, vol, tf, ess.HYBRID, ess.build_params(brick=B, nbins=4, halting=0))
        for i in range(len(tf_dev)):      # warm-up pass
            ess.ess_tf_update(ctx, tf, tf_dev[i])
            ess.ess_rebuild(ctx, st)
            ess.ess_render(ctx, st, ecams[i], rp, W, H, out)
        ess.ess_sync(ctx)
        ess.ess_sample_count(ctx, reset=True)
        ess.ess_profile_reset(ctx)
        ess.ess_profile_enable(ctx, True)
        for _ in range(steps):
            for i in range(len(tf_dev)):
                ess.ess_tf_update(ctx, tf, tf_dev[i])
                ess.ess_rebuild(ctx, st)
                ess.ess_render(ctx, st, ecams[i], rp, W, H, out)
        ess.ess_sync(ctx)
        ess.ess_profile_enable(ctx, False)
        prof = ess.ess_profile_read(ctx)
        frames = steps * len(tf_dev)
        n, ms = prof["render_hybrid"]
        build = sum(v[1] for k, v in prof.items() if not k.startswith("render")) / frames
        info = ess.ess_structure_info_get(ctx, st)
        res["brick%d" % B] = {"ms_per_frame": round(ms / n, 4), "build_ms_per_edit": round(build, 4),
                              "kd_nodes_last_edit": info["n_nodes"],
                              "samples_per_frame": ess.ess_sample_count(ctx, reset=True) / frames}
        ess.ess_release(ctx, st)
    return {"structure": "hybrid grid: shallow k-d tree (halting 0, 3 binned planes per axis) "
                         "whose leaves are crossed with the macrocell grid of the same brick size",
            "workload": "the main workload's 8 TF edits, one rebuild and one frame each", **res}


def run_cell_vote(ess, torch, dev, ctx, vol, tf, tf_dev, ecams, rp, W, H, B, vox_bytes, reps=3):
    """The exact per-cell vote (the paper's per-voxel classification, Sec.
    3.1) against the brick min/max range test on the main workload's TF
    edits.  Both read the volume once per edit (the min/max pass); the vote
    then tests the cells of the bricks the range test passes.  Reported: each
    path's empty-test time per edit (its kernels' CUDA-event times) and its
    rate on the volume's bytes against the measured HBM peak, the non-empty
    fraction of each mask (the vote's is a subset of the range test's), and
    the grid frame through each."""
    peak, src = measured_peaks()
    out = torch.empty((H, W, 4), dtype=torch.float32, device=dev)
    paths = {"vote": ess.ess_build(ctx, vol, tf, ess.GRID, ess.build_params(brick=B, empty_test=1,
                                                                            rescan=1)),
             "minmax": ess.ess_build(ctx, vol, tf, ess.GRID, ess.build_params(brick=B, rescan=1))}
    frac = {k: [] for k in paths}
    test_ms = {k: [] for k in paths}
    vote_ms = []
    frame = {k: [] for k in paths}
    cur = torch.cuda.current_stream()
    for rep in range(reps + 1):          # the first pass warms up
        for i in range(len(tf_dev)):
            for name, st in paths.items():
                ess.ess_tf_update(ctx, tf, tf_dev[i])   # an edit: the volume pass runs again
                ess.ess_sync(ctx)
                ess.ess_profile_reset(ctx)
                ess.ess_profile_enable(ctx, True)
                ess.ess_rebuild(ctx, st)
                ess.ess_sync(ctx)
                ess.ess_profile_enable(ctx, False)
                prof = ess.ess_profile_read(ctx)
                a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                a.record(cur)
                ess.ess_render(ctx, st, ecams[i], rp, W, H, out)
                b.record(cur)
                b.synchronize()
                if rep == 0:
                    info = ess.ess_structure_info_get(ctx, st)
                    frac[name].append(info["n_nonempty"] / info["n_bricks"])
                    continue
                test_ms[name].append(sum(prof.get(k, (0, 0.0))[1] for k in
                                         ("brick_minmax", "brick_mask", "vote_bricks")))
                if name == "vote":
                    vote_ms.append(prof["vote_bricks"][1])
                frame[name].append(a.elapsed_time(b))
    for st in paths.values():
        ess.ess_release(ctx, st)
    res = {}
    for name in paths:
        ms = float(np.mean(test_ms[name]))
        gbs = vox_bytes / (ms / 1000.0) / 1e9
        res[name] = {"empty_test_us_per_edit": round(1000.0 * ms, 2),
                     "hbm_on_volume_bytes": {"achieved_gbs": round(gbs, 1), "peak_gbs": peak,
                                             "peak_source": src, "frac": round(gbs / peak, 3)},
                     "nonempty_fraction": [round(x, 4) for x in frac[name]],
                     "grid_frame_ms": round(float(np.mean(frame[name])), 4)}
    return {"workload": "the main workload's 8 TF edits, grid structure at %d^3 bricks, one "
                        "volume pass (min/max) per edit on both paths" % B,
            "vote_bricks_us": round(1000.0 * float(np.mean(vote_ms)), 2),
            "kernels": {"vote": "brick_minmax + brick_mask + vote_bricks",
                        "minmax": "brick_minmax + brick_mask"},
            **res,
            "note": "the vote's mask is never larger than the range test's, and the images are "
                    "the same"}


SHADE = (0.25, 0.6, 0.3, 12)   # ka, kd, ks, shininess of the shaded workload


def run_shaded(ess, torch, dev, ctx, vol, tf, tf_dev, ecams, W, H, B, kd_params, steps=2):
    """The second render workload: gradient shading (central differences of the
    reconstruction, headlight Blinn-Phong) and opacity correction (dt 0.5 for
    a TF defined per voxel) on the main workload's TF edits, one frame per
    structure and edit, against the same frames unshaded (CUDA-event time per
    frame; samples per frame are the same)."""
    out = torch.empty((H, W, 4), dtype=torch.float32, device=dev)
    kinds = (ess.GRID, ess.LBVH, ess.KD)
    sts = {k: ess.ess_build(ctx, vol, tf, k, ess.build_params(
        brick=B, **(kd_params if k == ess.KD else {}))) for k in kinds}
    rps = {"plain": ess.render_params(0.5, 0.99),
           "shaded": ess.render_params(0.5, 0.99, shade=SHADE, dt_ref=1.0)}
    res = {}
    for name, rp in rps.items():
        for rep in range(2):           # warm-up pass, then the timed one
            ess.ess_sync(ctx)
            ess.ess_profile_reset(ctx)
            ess.ess_profile_enable(ctx, rep == 1)
            for _ in range(steps if rep else 1):
                for i in range(len(tf_dev)):
                    ess.ess_tf_update(ctx, tf, tf_dev[i])
                    for k in kinds:
                        ess.ess_rebuild(ctx, sts[k])
                    for k in kinds:
                        ess.ess_render(ctx, sts[k], ecams[i], rp, W, H, out)
            ess.ess_sync(ctx)
        ess.ess_profile_enable(ctx, False)
        prof = ess.ess_profile_read(ctx)
        res[name] = {ess.KIND_NAMES[k]: round(
            prof[("render_shaded_" if name == "shaded" else "render_") + ess.KIND_NAMES[k]][1] /
            prof[("render_shaded_" if name == "shaded" else "render_") + ess.KIND_NAMES[k]][0], 4)
            for k in kinds}
    for st in sts.values():
        ess.ess_release(ctx, st)
    return {"workload": "the main workload's 8 TF edits, one 1024^2 frame per structure and edit; "
                        "shading ka, kd, ks, shininess = %s, dt_ref 1 voxel" % (SHADE,),
            "ms_per_frame": res,
            "slowdown": {k: round(res["shaded"][k] / res["plain"][k], 3) for k in res["plain"]}}


def run_structures(ess, torch, dev, ctx, vol, tf, tf_dev, ecams, rp, W, H, reps=3):
    """Table 1 / Table 2 style comparison on the main workload (Sec. 4.3): node
    count, height, build time and frame time of the LBVH and of the k-d tree
    built shallow, deep, deep with MLS 32 and MLS 128 (binned planes, 4 bins, as
    the GPU builder of the paper, and exhaustive brick-boundary planes), plus
    the grid and the hybrid grid, for the sparsest and the densest TF edit."""
    out = torch.empty((H, W, 4), dtype=torch.float32, device=dev)
    configs = [("grid", ess.GRID, {}), ("lbvh", ess.LBVH, {}), ("hybrid", ess.HYBRID, dict(halting=0))]
    for nb in (4, 0):
        for name, prm in (("shallow", dict(halting=0)), ("deep", dict(halting=1)),
                          ("deep_mls32", dict(halting=1, mls=32)), ("deep_mls128", dict(halting=1, mls=128))):
            configs.append(("kd_%s_%s" % ("binned" if nb else "exhaustive", name), ess.KD, dict(nbins=nb, **prm)))
    nonempty = []
    for i in range(len(tf_dev)):
        ess.ess_tf_update(ctx, tf, tf_dev[i])
        g = ess.ess_build(ctx, vol, tf, ess.GRID, ess.build_params(brick=8))
        nonempty.append(ess.ess_structure_info_get(ctx, g)["n_nonempty"])
        ess.ess_release(ctx, g)
    picks = sorted({int(np.argmin(nonempty)), int(np.argmax(nonempty))})
    rows = []
    runs = [(8,) + c for c in configs]
    for B in (16, 32):
        runs += [(B, "grid", ess.GRID, {}), (B, "lbvh", ess.LBVH, {}),
                 (B, "kd_binned_deep_mls32", ess.KD, dict(KD_PARAMS))]
    for i in picks:
        ess.ess_tf_update(ctx, tf, tf_dev[i])
        for B, name, kind, prm in runs:
            st = ess.ess_build(ctx, vol, tf, kind, ess.build_params(brick=B, **prm))
            ess.ess_render(ctx, st, ecams[i], rp, W, H, out)   # warm
            ess.ess_sync(ctx)
            ess.ess_profile_reset(ctx)
            ess.ess_profile_enable(ctx, True)
            for _ in range(reps):
                ess.ess_rebuild(ctx, st)
                ess.ess_render(ctx, st, ecams[i], rp, W, H, out)
            ess.ess_sync(ctx)
            ess.ess_profile_enable(ctx, False)
            prof = ess.ess_profile_read(ctx)
            info = ess.ess_structure_info_get(ctx, st)
            render = sum(v[1] for k, v in prof.items() if k.startswith("render")) / reps
            build = sum(v[1] for k, v in prof.items() if not k.startswith("render")) / reps
            rows.append({"tf_edit": i, "nonempty_bricks": int(info["n_nonempty"]),
                         "structure": name, "brick": B, "nodes": int(info["n_nodes"]),
                         "height": int(info["height"]), "build_ms": round(build, 4),
                         "frame_ms": round(render, 4)})
            ess.ess_release(ctx, st)
    return {"workload": "the main workload (512^3 CT-like, 1024^2 frame), sparsest and densest of "
                        "its TF edits; every structure at 8^3 bricks, the step's three at 16^3 and "
                        "32^3 too; build = one rebuild (min/max cached), frame = one render, "
                        "CUDA-event means of %d" % reps, "rows": rows}


def run_minmax_sweep(ess, torch, dev, ctx, reps=10):
    """The per-brick min/max pass (rebuild with rescan) over larger volumes and
    every dtype: device time per launch with L2 flushed before each, against
    the measured HBM peak on the algorithmic bytes (the volume once plus the
    min/max pairs)."""
    from paper_1912_09596_gb300 import synth
    peak, src = measured_peaks()
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=dev)
    g = torch.Generator(device=dev)
    g.manual_seed(5)
    rows = []
    for name, dims in (("u8", (512, 512, 512)), ("u16", (512, 512, 512)), ("f32", (512, 512, 512)),
                       ("f32", (1024, 1024, 1024))):
        if name == "u8":
            x = torch.randint(0, 256, dims, device=dev, dtype=torch.uint8, generator=g)
            lo, hi = 0, 255
        elif name == "u16":
            x = torch.randint(0, 256, dims[:2] + (2 * dims[2],), device=dev, dtype=torch.uint8,
                              generator=g).view(torch.uint16)
            lo, hi = 0, 65535
        else:
            x = torch.rand(dims, device=dev, dtype=torch.float32, generator=g)
            lo, hi = 0.0, 1.0
        vol = ess.ess_volume_upload(ctx, x, lo, hi)
        ess.ess_volume_set_sampler(ctx, vol, 0)
        tf_np = synth.tf_ramp(256, 40)
        tf = ess.ess_tf_set(ctx, tf_np)
        for B in (8, 16, 32):
            st = ess.ess_build(ctx, vol, tf, ess.GRID, ess.build_params(brick=B, rescan=1))
            for _ in range(2):
                ess.ess_tf_update(ctx, tf, tf_np)
                ess.ess_rebuild(ctx, st)
            ess.ess_sync(ctx)
            ess.ess_profile_reset(ctx)
            ess.ess_profile_enable(ctx, True)
            for _ in range(reps):
                # a TF edit (the same table again): the rebuild reads the volume
                # once more.  The rebuild runs on the library's build stream,
                # which does not wait for this stream: finish the flush first,
                # and the rebuild before the next flush
                ess.ess_tf_update(ctx, tf, tf_np)
                flush.zero_()
                torch.cuda.synchronize(dev)
                ess.ess_rebuild(ctx, st)
                ess.ess_sync(ctx)
            ess.ess_profile_enable(ctx, False)
            n, ms = ess.ess_profile_read(ctx)["brick_minmax"]
            nb = 1
            for d in dims:
                nb *= (d + B - 1) // B
            byts = x.numel() * x.element_size() + 8 * nb
            gbs = byts / (ms / n / 1000.0) / 1e9
            rows.append({"dtype": name, "dims": "%dx%dx%d" % dims[::-1], "brick": B,
                         "us": round(1000.0 * ms / n, 2), "achieved_gbs": round(gbs, 1),
                         "frac": round(gbs / peak, 3)})
            ess.ess_release(ctx, st)
        ess.ess_release(ctx, tf)
        ess.ess_release(ctx, vol)
        del x
        torch.cuda.empty_cache()
    return {"kernel": "brick_minmax", "peak_gbs": peak, "peak_source": src,
            "l2": "flushed before each launch", "rows": rows}


# ---------------------------------------------------------------- ours
# The paper's own timings for its 512^3-class data sets (Table 2; NVIDIA Titan V; 1024^2
# orthographic views of real data sets, early termination and shading off; build in seconds,
# rendering in frames/s).  Context only: other hardware, other data, other camera.
PAPER_TABLE2_512 = {
    "Magnetic 512^3, 16.6 % occupied": {"naive_fps": 105, "lbvh_build_s": 0.004, "lbvh_fps": 103,
                                        "kd_gpu_mls32_build_s": 1.758, "kd_gpu_mls32_fps": 156},
    "Xmas Tree 512x499x512, 2.90 %": {"naive_fps": 97.1, "lbvh_build_s": 0.004, "lbvh_fps": 69,
                                      "kd_gpu_mls32_build_s": 2.163, "kd_gpu_mls32_fps": 115},
    "N-Body 512^3, 0.15 %": {"naive_fps": 100, "lbvh_build_s": 0.003, "lbvh_fps": 144,
                             "kd_gpu_mls32_build_s": 1.168, "kd_gpu_mls32_fps": 233},
}


def measure_step(ess, torch, dev, stream, ctx, name, steps, warmup, dist=None, ws=1,
                 e2e=True, sample_clocks=True, inputs=None):
    """Times `steps` passes of the hot path over workload `name` (after
    `warmup` untimed ones) inside the library's context `ctx`: per TF edit the
    table upload, the rebuild of the grid, LBVH and k-d structures with a
    min/max rescan (one volume pass per edit, shared by the three), then one
    frame through each structure for every view of that edit.  Returns (the
    bench line's measurement fields, the resident objects for further legs)."""
    w = WORKLOADS[name]
    vol_in, (vlo, vhi), tfs_np, views = inputs if inputs is not None else make_inputs(name, dev)
    W, H, B = w["W"], w["H"], w["brick"]
    kinds = [k for k in ess.KINDS if k != ess.NONE]
    sms = torch.cuda.get_device_properties(dev).multi_processor_count
    data = vol_in.to(dev) if hasattr(vol_in, "to") else torch.from_numpy(vol_in).to(dev)
    itemsize = data.element_size()
    nvox = data.numel()
    vshape = tuple(data.shape)
    vol = ess.ess_volume_upload(ctx, data, vlo, vhi)
    del data
    tf_dev = [torch.from_numpy(t).to(dev) for t in tfs_np]
    tf_host = [torch.from_numpy(t).pin_memory() for t in tfs_np]
    tf = ess.ess_tf_set(ctx, tf_dev[0])
    # rescan: the first rebuild of each edit recomputes the brick min/max from
    # the voxels, and the other structures of the edit reuse it
    params = {k: ess.build_params(brick=B, rescan=1, **KD_PARAMS) for k in kinds}
    st = {k: ess.ess_build(ctx, vol, tf, k, params[k]) for k in kinds}
    naive = ess.ess_build(ctx, vol, tf, ess.NONE)
    outs = {k: torch.empty((H, W, 4), dtype=torch.float32, device=dev) for k in kinds}
    host_out = torch.empty((H, W, 4), dtype=torch.float32).pin_memory()
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=dev)
    rp = ess.render_params(w["dt"], w["ert"])
    ecams = [[ess.camera_from(c) for c in vs] for vs in views]
    frames_step = sum(len(vs) for vs in views) * len(kinds)

    # per-frame reference counts (untimed): naive samples, evaluated samples,
    # non-empty bricks, algorithmic bytes of each render, naive frame time
    n_naive, n_eval = [], {k: [] for k in kinds}
    alg_bytes, nonempty = {k: [] for k in kinds}, []
    naive_ms = []
    cur = torch.cuda.current_stream(dev)
    for i in range(len(tfs_np)):
        ess.ess_tf_update(ctx, tf, tf_dev[i])
        ess.ess_rebuild(ctx, naive)
        for k in kinds:
            ess.ess_rebuild(ctx, st[k])
        infos = {k: ess.ess_structure_info_get(ctx, st[k]) for k in kinds}
        nonempty.append(infos[kinds[0]]["n_nonempty"] / max(1, infos[kinds[0]]["n_bricks"]))
        for cam in ecams[i]:
            ess.ess_sync(ctx)
            ess.ess_sample_count(ctx, reset=True)
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(cur)
            ess.ess_render(ctx, naive, cam, rp, W, H, outs[kinds[0]])
            b.record(cur)
            n_naive.append(ess.ess_sample_count(ctx, reset=True))
            naive_ms.append(a.elapsed_time(b))
            for k in kinds:
                ess.ess_render(ctx, st[k], cam, rp, W, H, outs[k])
                n_eval[k].append(ess.ess_sample_count(ctx, reset=True))
                info = infos[k]
                # compulsory bytes of one frame: the image, the voxels of the
                # non-empty bricks and the structure itself
                struct_b = info["n_bricks"] if k == ess.GRID else 32 * max(1, info["n_nodes"])
                alg_bytes[k].append(W * H * 16 + info["n_nonempty"] * B ** 3 * itemsize + struct_b)
    ess.ess_sync(ctx)

    def step(host_io=False):
        # the library runs the rebuilds on its build stream: the k-d and LBVH
        # rebuilds overlap the grid's frame
        for i in range(len(tfs_np)):
            ess.ess_tf_update(ctx, tf, tf_host[i] if host_io else tf_dev[i])
            for k in kinds:
                ess.ess_rebuild(ctx, st[k])
            for cam in ecams[i]:
                for k in kinds:
                    ess.ess_render(ctx, st[k], cam, rp, W, H, host_out if host_io else outs[k])

    for _ in range(warmup):
        step()
    ess.ess_sync(ctx)
    launches0 = ess.ess_launch_count(ctx)
    ess.ess_profile_reset(ctx)
    ess.ess_profile_enable(ctx, True)
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for _ in range(steps)]
    if dist:
        dist.barrier()
    torch.cuda.synchronize(dev)
    clocks = ClockSampler(dev.index or 0) if sample_clocks else None
    for s_ in range(steps):
        flush.zero_()                        # L2 flush between timed steps (untimed)
        ev[s_][0].record(stream)
        step()
        ev[s_][1].record(stream)
    torch.cuda.synchronize(dev)
    clk = clocks.stop() if clocks else None
    launches = ess.ess_launch_count(ctx) - launches0
    ess.ess_profile_enable(ctx, False)
    prof = ess.ess_profile_read(ctx)
    ess.ess_sync(ctx)
    t_ms = max_over_ranks(dist, sum(a.elapsed_time(b) for a, b in ev), dev)

    e2e_ms = None
    if e2e:
        # end to end through the ABI with host buffers
        for _ in range(max(1, warmup // 2)):
            step(host_io=True)
        ess.ess_sync(ctx)
        if dist:
            dist.barrier()
        torch.cuda.synchronize(dev)
        t0 = time.perf_counter()
        for _ in range(steps):
            step(host_io=True)
        ess.ess_sync(ctx)
        e2e_ms = max_over_ranks(dist, 1000.0 * (time.perf_counter() - t0), dev)

    # the step's rebuilds alone (no frame beside them): per edit, the TF
    # upload and the three rebuilds, waited for before the next edit
    ess.ess_profile_reset(ctx)
    ess.ess_profile_enable(ctx, True)
    for _ in range(steps):
        for i in range(len(tfs_np)):
            ess.ess_tf_update(ctx, tf, tf_dev[i])
            for k in kinds:
                ess.ess_rebuild(ctx, st[k])
            ess.ess_sync(ctx)
    ess.ess_profile_enable(ctx, False)
    prof_alone = ess.ess_profile_read(ctx)

    units_step = sum(n_naive) * len(kinds)
    evaluated_step = sum(sum(v) for v in n_eval.values())
    value = job_rate(units_step, ws, steps, t_ms)

    # dominant kernel and its roofline on algorithmic bytes (among the renders:
    # the build kernels run on the build stream alongside them, so their event
    # intervals include the time they share the GPU with a render)
    kind_of = {"render_grid": ess.GRID, "render_lbvh": ess.LBVH, "render_kd": ess.KD}
    peak, peak_src = measured_peaks()
    fpeak, mhz = fp32_peak_tflops(sms)

    def render_roof(kname, n, ms):
        k = kind_of[kname]
        avg_ms = ms / max(1, n)
        bytes_per_launch = float(np.mean(alg_bytes[k]))
        flop = float(np.mean(n_eval[k])) * FLOP_PER_SAMPLE
        achieved = flop / (avg_ms / 1000.0) / 1e12
        # the render kernels are bound by instruction issue, not DRAM: their
        # roof is FP32 throughput on the sample arithmetic
        return {"bound": "alu", "achieved": achieved, "peak": fpeak, "unit": "TFLOP/s",
                "frac": achieved / fpeak, "traffic": ncu_traffic(kname, name),
                "kernel": kname, "avg_launch_ms": avg_ms,
                "algorithmic_flop_per_launch": flop, "flop_per_sample": FLOP_PER_SAMPLE,
                "peak_source": "derived: %d SMs x %d FP32 lanes x 2 FLOP x %.0f MHz"
                               % (sms, FP32_LANES_PER_SM, mhz),
                "hbm": {"achieved_gbs": bytes_per_launch / (avg_ms / 1000.0) / 1e9,
                        "peak_gbs": peak, "peak_source": peak_src,
                        "algorithmic_bytes_per_launch": bytes_per_launch,
                        "frac": bytes_per_launch / (avg_ms / 1000.0) / 1e9 / peak}}

    renders = [(k, v) for k, v in prof.items() if k in kind_of]
    dom_name, (dom_n, dom_ms) = max(renders, key=lambda kv: kv[1][1])
    roof = render_roof(dom_name, dom_n, dom_ms)

    # HBM roofline of every kernel with a fixed algorithmic byte count
    gxyz = [(n + B - 1) // B for n in vshape]
    n_bricks = int(np.prod(gxyz))
    fixed_bytes = {"brick_minmax": nvox * itemsize + 8 * n_bricks, "brick_mask": 9 * n_bricks}
    kroof = {}
    for kname, (n, ms) in prof.items():
        if kname in kind_of:
            kroof[kname] = render_roof(kname, n, ms)
            continue
        if kname not in fixed_bytes:
            continue
        b = fixed_bytes[kname]
        avg = ms / max(1, n)
        ach = b / (avg / 1000.0) / 1e9
        kroof[kname] = {"bound": "hbm", "achieved": round(ach, 1), "peak": peak, "unit": "GB/s",
                        "frac": round(ach / peak, 4), "avg_launch_ms": round(avg, 5),
                        "launches": n, "algorithmic_bytes_per_launch": b,
                        "traffic": ncu_traffic(kname, name)}

    per_frame = {ess.KIND_NAMES[kind_of[kname]]: ms / max(1, n)
                 for kname, (n, ms) in prof.items() if kname in kind_of}
    build_kernels = {nm: v for nm, v in prof.items() if not nm.startswith("render")}
    edits = steps * len(tfs_np)
    build_ms = {
        "all_structures_per_edit": sum(v[1] for v in build_kernels.values()) / edits,
        "note": "event intervals of the build kernels on the library's build stream, which run "
                "while the frames of the same edit render",
        "alone_per_edit": sum(v[1] for v in prof_alone.values()) / edits,
        "alone_by_kernel": {nm: round(v[1] / edits, 4) for nm, v in prof_alone.items()},
        "brick_minmax_launches_per_edit": prof.get("brick_minmax", (0, 0.0))[0] / edits}

    result = {
        "metric": METRIC, "value": value, "unit": "samples/s", "n_gpus": ws,
        "steps": steps, "warmup": warmup, "ms_per_step": t_ms / steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
        "data": "synthetic",
        "config": {"workload": name + ": " + w["desc"],
                   "structures": [ess.KIND_NAMES[k] for k in kinds],
                   "kd": KD_PARAMS, "brick": B, "image": "%dx%d" % (W, H),
                   "tf_edits_per_step": len(tfs_np), "frames_per_step": frames_step,
                   "nonempty_brick_fraction": [round(x, 4) for x in nonempty],
                   "l2": "flushed between timed steps (%d MiB write, untimed)" % (L2_FLUSH_BYTES >> 20),
                   "parallelism": "replicas" if ws > 1 else "single GPU"},
        "evaluated_samples_per_s": job_rate(evaluated_step, ws, steps, t_ms),
        "evaluated_samples_per_s_note": "ray samples/s as evaluated samples / time: the samples the "
                                        "skipping renderers actually take",
        "samples_per_frame": {"naive_equivalent": float(np.mean(n_naive)),
                              **{ess.KIND_NAMES[k]: float(np.mean(v)) for k, v in n_eval.items()}},
        "ms_per_frame": per_frame,
        "naive_ms_per_frame": float(np.mean(naive_ms)),
        "build_ms_per_edit": build_ms,
        "kernel_ms": {k: {"launches": v[0], "total_ms": round(v[1], 4)} for k, v in prof.items()},
        "gpu_launches": int(launches),
        "roofline": roof,
        "kernel_rooflines": kroof,
        "clocks": clk,
    }
    if e2e_ms is not None:
        result["e2e"] = {"value": job_rate(units_step, ws, steps, e2e_ms), "unit": "samples/s",
                         "h2d_bytes_per_step": int(sum(t.numel() * 4 for t in tf_host)),
                         "d2h_bytes_per_step": int(frames_step * W * H * 16),
                         "ms_per_step": e2e_ms / steps}
    env = dict(vol=vol, tf=tf, tf_dev=tf_dev, ecams=[vs[0] for vs in ecams], rp=rp, W=W, H=H,
               B=B, structures=list(st.values()) + [naive], nvox=nvox, itemsize=itemsize,
               tfs_np=tfs_np, views=views, vlo=vlo, vhi=vhi, vol_in=vol_in)
    return result, env


def release_env(ess, ctx, env):
    for h in env["structures"]:
        ess.ess_release(ctx, h)
    ess.ess_release(ctx, env["tf"])
    ess.ess_release(ctx, env["vol"])


def run_fractal_leg(ess, torch, dev, stream, ctx, cpu, ref_budget, steps=2, warmup=1):
    """The 1024^3 float32 field with a 1024-entry TF at 1920x1080 over 16 orbit
    views (the paper compares the structures' build and render times per data
    set, Table 2): per structure its rebuild (with the min/max pass over the
    4 GiB volume) and its frames, each against its roofline, and the CPU
    oracle on a row stripe of one view."""
    res, env = measure_step(ess, torch, dev, stream, ctx, "fractal1024", steps, warmup,
                            e2e=False, sample_clocks=False)
    kr = res["kernel_rooflines"]
    out = {"workload": res["config"]["workload"], "steps": steps,
           "ms_per_step": res["ms_per_step"], "naive_equivalent_samples_per_s": res["value"],
           "evaluated_samples_per_s": res["evaluated_samples_per_s"],
           "nonempty_brick_fraction": res["config"]["nonempty_brick_fraction"],
           "samples_per_frame": res["samples_per_frame"],
           "naive_ms_per_frame": res["naive_ms_per_frame"],
           "ms_per_frame": res["ms_per_frame"], "build_ms_per_edit": res["build_ms_per_edit"],
           "render_rooflines": {k: v for k, v in kr.items() if k.startswith("render")},
           "brick_minmax_roofline": kr.get("brick_minmax"), "gpu_launches": res["gpu_launches"]}
    if cpu:
        w = WORKLOADS["fractal1024"]
        host = host_array(env["vol_in"])
        cores = cpu_cores()
        rate, desc = oracle_rate(host, 0.0, 1.0, env["tfs_np"][0], env["views"][0][0], w,
                                 ref_budget, cores)
        out["cpu_baseline"] = {"value": rate, "unit": "samples/s", "cores": cores,
                               "kind": "oracle", "sample": desc}
        del host
    release_env(ess, ctx, env)
    del env
    torch.cuda.empty_cache()
    return out


def run_ours(args, rank, local, ws, dist):
    import torch
    import __graft_entry__
    __graft_entry__.build()
    from paper_1912_09596_gb300 import ess

    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    stream = torch.cuda.Stream(device=dev)
    with torch.cuda.stream(stream):
        ctx = ess.ess_create(local, stream)
        result, env = measure_step(ess, torch, dev, stream, ctx, args.workload, args.steps,
                                   args.warmup, dist=dist, ws=ws)
    if args.workload == "ct512":
        result["paper_context"] = {
            "source": "Table 2 of the paper (NVIDIA Titan V, Xeon Gold 5122; Sec. 4.1)",
            "note": "real 512^3-class data sets, 1024^2 orthographic, early termination and "
                    "shading off: context, not a target; this run's frames/s are 1000 / "
                    "ms_per_frame and its builds are in build_ms_per_edit and structures",
            "rows": PAPER_TABLE2_512,
            "this_run_fps": {k: round(1000.0 / v, 1) for k, v in result["ms_per_frame"].items()}}
    vol, tf, tf_dev, ecams = env["vol"], env["tf"], env["tf_dev"], env["ecams"]
    rp, W, H, B = env["rp"], env["W"], env["H"], env["B"]
    ct = args.workload == "ct512"   # the legs below run on the 512^3 workload's TF edits
    if ct and not args.no_hybrid:
        with torch.cuda.stream(stream):
            result["hybrid"] = run_hybrid(ess, torch, dev, ctx, vol, tf, tf_dev, ecams, rp, W, H)
    if ct and not args.no_cell_vote:
        with torch.cuda.stream(stream):
            result["cell_vote"] = run_cell_vote(ess, torch, dev, ctx, vol, tf, tf_dev, ecams, rp,
                                                W, H, B, env["nvox"] * env["itemsize"])
    if ct and not args.no_shaded:
        with torch.cuda.stream(stream):
            result["shaded"] = run_shaded(ess, torch, dev, ctx, vol, tf, tf_dev, ecams, W, H, B,
                                          KD_PARAMS)
    if ct and not args.no_structures:
        with torch.cuda.stream(stream):
            result["structures"] = run_structures(ess, torch, dev, ctx, vol, tf, tf_dev, ecams,
                                                  rp, W, H)
    vol_host = host_array(env["vol_in"])
    vlo, vhi, tfs_np, views = env["vlo"], env["vhi"], env["tfs_np"], env["views"]
    with torch.cuda.stream(stream):
        release_env(ess, ctx, env)
    del env
    torch.cuda.empty_cache()
    if ct and not args.no_fractal:
        with torch.cuda.stream(stream):
            result["fractal1024"] = run_fractal_leg(
                ess, torch, dev, stream, ctx, rank == 0 and ws == 1 and not args.no_cpu_baseline,
                min(args.ref_budget, 4.0))
    if not args.no_batched:
        with torch.cuda.stream(stream):
            result["batched"] = run_batched(ess, torch, dev, stream, ctx)
    if ct and not args.no_serve:
        with torch.cuda.stream(stream):
            result["served"] = run_served(ess, torch, dev, ctx, vol_host)
    if not args.no_minmax:
        with torch.cuda.stream(stream):
            result["minmax_sweep"] = run_minmax_sweep(ess, torch, dev, ctx)
    if rank == 0 and ws == 1 and not args.no_cpu_baseline:
        cores = cpu_cores()
        w = WORKLOADS[args.workload]
        rate, desc = oracle_rate(vol_host, vlo, vhi, tfs_np[0], views[0][0], w, args.ref_budget,
                                 cores)
        result["cpu_baseline"] = {"value": rate, "unit": "samples/s", "cores": cores,
                                  "kind": "oracle", "sample": desc}
        # the same marcher on one core, for the per-core rate
        rate1, desc1 = oracle_rate(vol_host, vlo, vhi, tfs_np[0], views[0][0], w,
                                   min(args.ref_budget, 1.5), 1)
        result["cpu_baseline"]["single_core"] = {"value": rate1, "unit": "samples/s",
                                                 "sample": desc1}
    with torch.cuda.stream(stream):
        ess.ess_destroy(ctx)
    if rank == 0:
        print(json.dumps(result))


def make_parser():
    ap = argparse.ArgumentParser(description=__doc__.split("\n")[0])
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--workload", choices=sorted(WORKLOADS), default="ct512")
    ap.add_argument("--ref-budget", type=float, default=6.0,
                    help="seconds of oracle work per CPU measurement")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-batched", action="store_true",
                    help="skip the batched-render comparison (64 TFs x 4 views)")
    ap.add_argument("--no-serve", action="store_true",
                    help="skip the serving comparison (Poisson request stream)")
    ap.add_argument("--no-minmax", action="store_true",
                    help="skip the brick min/max sweep over dtypes and sizes")
    ap.add_argument("--no-hybrid", action="store_true",
                    help="skip the hybrid-grid leg")
    ap.add_argument("--no-cell-vote", action="store_true",
                    help="skip the per-cell vote (exact empty test) leg")
    ap.add_argument("--no-shaded", action="store_true",
                    help="skip the shaded-render workload (gradient shading, opacity correction)")
    ap.add_argument("--no-structures", action="store_true",
                    help="skip the structure comparison (node counts, heights, build and frame times)")
    ap.add_argument("--no-fractal", action="store_true",
                    help="skip the 1024^3 float32 leg (16 views at 1920x1080, every structure)")
    return ap


def main():
    args = make_parser().parse_args()
    rank, local, ws, dist = dist_setup()
    if args.impl == "reference":
        run_reference(args, rank)
        return
    if dist:
        import torch
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    try:
        run_ours(args, rank, local, ws, dist)
    finally:
        if dist:
            dist.destroy_process_group()


if __name__ == "__main__":
    main()
