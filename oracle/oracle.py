"""ctypes front end of the plain-C oracle in ``ess_oracle.c``.

TEST INFRASTRUCTURE ONLY: imported by the tests, by ``__graft_entry__.smoke()``
and by the benchmark's CPU-baseline leg, never by the library product.  The C
file states the passage of the paper each function follows and the readings
(R1..R14, S) taken where the paper is silent.

The C code is compiled with ``-ffp-contract=off`` and without fast-math so that
its float32 arithmetic is exactly what the source says (every fused
multiply-add is an explicit ``fmaf``).
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "ess_oracle.c")
_LIB = os.path.join(_HERE, "libess_oracle.so")
_lock = threading.Lock()
_lib = None

U8, U16, F32 = 0, 1, 2
_DT = {np.dtype(np.uint8): U8, np.dtype(np.uint16): U16, np.dtype(np.float32): F32}

GCC_FLAGS = ["-O2", "-std=c11", "-fPIC", "-shared", "-ffp-contract=off",
             "-fno-fast-math", "-fno-unsafe-math-optimizations", "-Wall"]


def build(force: bool = False) -> str:
    """Compile the oracle into a shared library next to its source."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + ".tmp.%d" % os.getpid()
        subprocess.check_call(["gcc", *GCC_FLAGS, "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


class Volume(C.Structure):
    _fields_ = [("data", C.c_void_p), ("dtype", C.c_int), ("nx", C.c_int),
                ("ny", C.c_int), ("nz", C.c_int), ("value_lo", C.c_float),
                ("value_hi", C.c_float)]


class TF(C.Structure):
    _fields_ = [("rgba", C.c_void_p), ("nt", C.c_int)]


class Camera(C.Structure):
    _fields_ = [("eye", C.c_float * 3), ("u", C.c_float * 3), ("v", C.c_float * 3),
                ("w", C.c_float * 3), ("ortho", C.c_int)]


class RenderParams(C.Structure):
    _fields_ = [("dt", C.c_float), ("ert", C.c_float), ("bg", C.c_float * 4),
                ("shade", C.c_int), ("ka", C.c_float), ("kd", C.c_float), ("ks", C.c_float),
                ("shininess", C.c_int), ("dt_ref", C.c_float)]


def lib():
    global _lib
    with _lock:
        if _lib is None:
            L = C.CDLL(build())
            vp, i, f = C.c_void_p, C.c_int, C.c_float
            P = C.POINTER
            L.ora_sample_value.argtypes = [P(Volume), f, f, f]
            L.ora_sample_value.restype = f
            L.ora_point_rgba.argtypes = [P(Volume), P(TF), f, f, f, vp]
            L.ora_tf_coord.argtypes = [f, f, f, i]
            L.ora_tf_coord.restype = f
            L.ora_ray.argtypes = [P(Camera), i, i, i, i, vp, vp]
            L.ora_slab.argtypes = [vp, vp, vp, vp, f, f, vp, vp]
            L.ora_render_naive.argtypes = [P(Volume), P(TF), P(Camera), P(RenderParams),
                                           i, i, vp, i, i]
            L.ora_render_naive.restype = C.c_int64
            L.ora_render_pixels.argtypes = [P(Volume), P(TF), P(Camera), P(RenderParams),
                                            i, i, vp, i, vp]
            L.ora_render_pixels.restype = C.c_int64
            L.ora_render_boxes.argtypes = [P(Volume), P(TF), P(Camera), P(RenderParams),
                                           i, i, vp, i, vp, i, i]
            L.ora_render_boxes.restype = C.c_int64
            L.ora_brick_minmax.argtypes = [P(Volume), i, vp, vp]
            L.ora_brick_mask.argtypes = [vp, vp, i, P(TF), f, f, vp]
            L.ora_brick_mask_cells.argtypes = [P(Volume), i, P(TF), vp]
            L.ora_compact.argtypes = [vp, i, vp]
            L.ora_compact.restype = i
            L.ora_morton30.argtypes = [C.c_uint32] * 3
            L.ora_morton30.restype = C.c_uint32
            L.ora_morton_keys.argtypes = [vp, i, i, i, vp]
            L.ora_sort_pairs.argtypes = [vp, vp, i]
            L.ora_lbvh_topdown.argtypes = [vp, i, vp, vp, vp]
            L.ora_lbvh_topdown.restype = i
            L.ora_lbvh_karras.argtypes = [vp, i, vp, vp]
            L.ora_lbvh_karras.restype = i
            L.ora_lbvh_boxes.argtypes = [vp, i, i, i, vp, vp]
            L.ora_kd_build.argtypes = [vp, i, i, i, i, i, i, i, i, i, i, vp, i]
            L.ora_kd_build.restype = i
            L.ora_log2_own.argtypes = [f]
            L.ora_log2_own.restype = f
            L.ora_exp2_own.argtypes = [f]
            L.ora_exp2_own.restype = f
            L.ora_opacity_correct.argtypes = [f, f]
            L.ora_opacity_correct.restype = f
            L.ora_gradient.argtypes = [P(Volume), f, f, f, vp]
            L.ora_shade.argtypes = [vp, vp, f, f, f, i, vp]
            _lib = L
    return _lib


def _p(a: np.ndarray):
    return a.ctypes.data_as(C.c_void_p)


# ---------------------------------------------------------------------------
class OVolume:
    """A volume as the oracle sees it; keeps the numpy array alive."""

    def __init__(self, data: np.ndarray, value_lo: float, value_hi: float):
        data = np.ascontiguousarray(data)
        if data.ndim != 3 or data.dtype not in _DT:
            raise ValueError("volume must be a 3-d uint8/uint16/float32 array")
        self.data = data
        nz, ny, nx = data.shape
        self.dims = (nx, ny, nz)
        self.c = Volume(data.ctypes.data, _DT[data.dtype], nx, ny, nz,
                        float(value_lo), float(value_hi))

    def grid(self, B):
        nx, ny, nz = self.dims
        return (-(-nx // B), -(-ny // B), -(-nz // B))


class OTF:
    def __init__(self, rgba: np.ndarray):
        self.rgba = np.ascontiguousarray(rgba, dtype=np.float32)
        assert self.rgba.ndim == 2 and self.rgba.shape[1] == 4
        self.c = TF(self.rgba.ctypes.data, self.rgba.shape[0])


def camera_struct(cam) -> Camera:
    c = Camera()
    for name in ("eye", "u", "v", "w"):
        arr = getattr(cam, name)
        for i in range(3):
            getattr(c, name)[i] = float(arr[i])
    c.ortho = int(cam.ortho)
    return c


def params_struct(dt=0.5, ert=2.0, bg=(0.0, 0.0, 0.0, 0.0), shade=None,
                  dt_ref=0.0) -> RenderParams:
    """`shade`: None (off) or (ka, kd, ks, shininess) for R13; `dt_ref` > 0
    switches on the opacity correction of R14."""
    p = RenderParams()
    p.dt = dt
    p.ert = ert
    for i in range(4):
        p.bg[i] = float(bg[i])
    if shade is not None:
        p.shade = 1
        p.ka, p.kd, p.ks = float(shade[0]), float(shade[1]), float(shade[2])
        p.shininess = int(shade[3])
    p.dt_ref = float(dt_ref)
    return p


def log2_own(x):
    return lib().ora_log2_own(float(x))


def exp2_own(y):
    return lib().ora_exp2_own(float(y))


def opacity_correct(alpha, r):
    return lib().ora_opacity_correct(float(alpha), float(r))


def gradient(vol: "OVolume", p):
    g = np.zeros(3, dtype=np.float32)
    lib().ora_gradient(C.byref(vol.c), float(p[0]), float(p[1]), float(p[2]), _p(g))
    return g


def shade(g, d, ka, kd, ks, shininess, rgb):
    g, d = (np.ascontiguousarray(a, dtype=np.float32) for a in (g, d))
    out = np.array(rgb, dtype=np.float32)
    lib().ora_shade(_p(g), _p(d), ka, kd, ks, int(shininess), _p(out))
    return out


# ---------------------------------------------------------------------------
def sample_value(vol: OVolume, p):
    return lib().ora_sample_value(C.byref(vol.c), float(p[0]), float(p[1]), float(p[2]))


def point_rgba(vol: OVolume, tf: OTF, p):
    out = np.zeros(4, dtype=np.float32)
    lib().ora_point_rgba(C.byref(vol.c), C.byref(tf.c), float(p[0]), float(p[1]),
                         float(p[2]), _p(out))
    return out


def ray(cam, x, y, W, H):
    o = np.zeros(3, dtype=np.float32)
    d = np.zeros(3, dtype=np.float32)
    cs = camera_struct(cam)
    lib().ora_ray(C.byref(cs), x, y, W, H, _p(o), _p(d))
    return o, d


def slab(o, d, lo, hi, tmin=0.0, tmax=float("inf")):
    o, d, lo, hi = (np.asarray(a, dtype=np.float32) for a in (o, d, lo, hi))
    ta = np.zeros(1, dtype=np.float32)
    tb = np.zeros(1, dtype=np.float32)
    lib().ora_slab(_p(o), _p(d), _p(lo), _p(hi), tmin, tmax, _p(ta), _p(tb))
    return float(ta[0]), float(tb[0])


def _row_split(H, threads):
    threads = max(1, min(threads, H))
    cuts = [H * i // threads for i in range(threads + 1)]
    return [(cuts[i], cuts[i + 1]) for i in range(threads) if cuts[i] < cuts[i + 1]]


def render_naive(vol: OVolume, tf: OTF, cam, W, H, dt=0.5, ert=2.0,
                 bg=(0.0, 0.0, 0.0, 0.0), rows=None, threads=1, shade=None, dt_ref=0.0):
    """Naive ray marching of rows [y0, y1) (default: all rows).  Returns
    (image (H, W, 4) float32 with only the requested rows filled, samples).
    `threads` > 1 renders row bands on parallel threads (ctypes drops the GIL)."""
    out = np.zeros((H, W, 4), dtype=np.float32)
    y0, y1 = (0, H) if rows is None else rows
    cs, ps = camera_struct(cam), params_struct(dt, ert, bg, shade, dt_ref)
    L = lib()
    counts = []

    def work(a, b):
        counts.append(L.ora_render_naive(C.byref(vol.c), C.byref(tf.c), C.byref(cs),
                                         C.byref(ps), W, H, _p(out), y0 + a, y0 + b))

    bands = _row_split(y1 - y0, threads)
    if len(bands) == 1:
        work(*bands[0])
    else:
        ts = [threading.Thread(target=work, args=b) for b in bands]
        for t in ts:
            t.start()
        for t in ts:
            t.join()
    return out, int(sum(counts))


def render_pixels(vol: OVolume, tf: OTF, cam, W, H, xy, dt=0.5, ert=2.0,
                  bg=(0.0, 0.0, 0.0, 0.0), threads=1, shade=None, dt_ref=0.0):
    """Naive marching of the pixels `xy` ((n, 2) int: x, y).  Returns the
    (n, 4) pixels and the number of samples taken."""
    xy = np.ascontiguousarray(np.asarray(xy, dtype=np.int32).reshape(-1, 2))
    out = np.zeros((xy.shape[0], 4), dtype=np.float32)
    cs, ps = camera_struct(cam), params_struct(dt, ert, bg, shade, dt_ref)
    L = lib()
    counts = []

    def work(a, b):
        counts.append(L.ora_render_pixels(C.byref(vol.c), C.byref(tf.c), C.byref(cs),
                                          C.byref(ps), W, H, _p(xy[a:b]), b - a,
                                          _p(out[a:b])))

    bands = _row_split(xy.shape[0], threads)
    ts = [threading.Thread(target=work, args=b) for b in bands]
    for t in ts:
        t.start()
    for t in ts:
        t.join()
    return out, int(sum(counts))


def render_boxes(vol: OVolume, tf: OTF, cam, W, H, boxes, dt=0.5, ert=2.0,
                 bg=(0.0, 0.0, 0.0, 0.0), rows=None, shade=None, dt_ref=0.0):
    """Skipping render by brute-force interval enumeration (rule S) over the
    closed voxel-space boxes `boxes` (m, 6) = lo xyz, hi xyz."""
    out = np.zeros((H, W, 4), dtype=np.float32)
    y0, y1 = (0, H) if rows is None else rows
    b = np.ascontiguousarray(np.asarray(boxes, dtype=np.float32).reshape(-1, 6))
    cs, ps = camera_struct(cam), params_struct(dt, ert, bg, shade, dt_ref)
    n = lib().ora_render_boxes(C.byref(vol.c), C.byref(tf.c), C.byref(cs), C.byref(ps),
                               W, H, _p(b), b.shape[0], _p(out), y0, y1)
    return out, int(n)


def brick_minmax(vol: OVolume, B):
    gx, gy, gz = vol.grid(B)
    mn = np.zeros(gx * gy * gz, dtype=np.float32)
    mx = np.zeros(gx * gy * gz, dtype=np.float32)
    lib().ora_brick_minmax(C.byref(vol.c), B, _p(mn), _p(mx))
    return mn, mx


def brick_mask(bmin, bmax, tf: OTF, value_lo, value_hi):
    bmin = np.ascontiguousarray(bmin, dtype=np.float32)
    bmax = np.ascontiguousarray(bmax, dtype=np.float32)
    m = np.zeros(bmin.shape[0], dtype=np.uint8)
    lib().ora_brick_mask(_p(bmin), _p(bmax), bmin.shape[0], C.byref(tf.c),
                         float(value_lo), float(value_hi), _p(m))
    return m


def brick_mask_cells(vol: OVolume, B, tf: OTF):
    gx, gy, gz = vol.grid(B)
    m = np.zeros(gx * gy * gz, dtype=np.uint8)
    lib().ora_brick_mask_cells(C.byref(vol.c), B, C.byref(tf.c), _p(m))
    return m


def compact(mask):
    mask = np.ascontiguousarray(mask, dtype=np.uint8)
    ids = np.zeros(max(1, mask.shape[0]), dtype=np.uint32)
    n = lib().ora_compact(_p(mask), mask.shape[0], _p(ids))
    return ids[:n].copy()


def morton30(x, y, z):
    return int(lib().ora_morton30(x, y, z))


def morton_keys(ids, gx, gy):
    ids = np.ascontiguousarray(ids, dtype=np.uint32)
    keys = np.zeros(max(1, ids.shape[0]), dtype=np.uint32)
    lib().ora_morton_keys(_p(ids), ids.shape[0], gx, gy, _p(keys))
    return keys[: ids.shape[0]].copy()


def sort_pairs(keys, ids):
    k = np.array(keys, dtype=np.uint32)
    v = np.array(ids, dtype=np.uint32)
    lib().ora_sort_pairs(_p(k), _p(v), k.shape[0])
    return k, v


def lbvh_topdown(sorted_keys):
    k = np.ascontiguousarray(sorted_keys, dtype=np.uint32)
    n = k.shape[0]
    m = max(1, n - 1)
    left = np.zeros(m, dtype=np.int32)
    right = np.zeros(m, dtype=np.int32)
    ranges = np.zeros(2 * m, dtype=np.int32)
    if lib().ora_lbvh_topdown(_p(k), n, _p(left), _p(right), _p(ranges)) != 0:
        raise ValueError("keys not strictly increasing")
    return left[: n - 1], right[: n - 1], ranges[: 2 * (n - 1)].reshape(-1, 2)


def lbvh_karras(sorted_keys):
    k = np.ascontiguousarray(sorted_keys, dtype=np.uint32)
    n = k.shape[0]
    m = max(1, n - 1)
    left = np.zeros(m, dtype=np.int32)
    right = np.zeros(m, dtype=np.int32)
    if lib().ora_lbvh_karras(_p(k), n, _p(left), _p(right)) != 0:
        raise ValueError("keys not strictly increasing")
    return left[: n - 1], right[: n - 1]


def lbvh_boxes(sorted_ids, ranges, gx, gy):
    ids = np.ascontiguousarray(sorted_ids, dtype=np.uint32)
    r = np.ascontiguousarray(ranges, dtype=np.int32).reshape(-1)
    n = ids.shape[0]
    boxes = np.zeros((max(1, n - 1), 6), dtype=np.int32)
    lib().ora_lbvh_boxes(_p(ids), n, gx, gy, _p(r), _p(boxes))
    return boxes[: n - 1]


def kd_build(mask, grid, B, dims, nbins=4, halting=1, mls=0, max_nodes=None):
    """Returns an (m, 9) int32 array: lo xyz, hi xyz, axis, plane, first_child."""
    mask = np.ascontiguousarray(mask, dtype=np.uint8)
    gx, gy, gz = grid
    nx, ny, nz = dims
    if max_nodes is None:
        max_nodes = 2 * int(mask.sum()) + 1
    out = np.zeros((max(1, max_nodes), 9), dtype=np.int32)
    m = lib().ora_kd_build(_p(mask), gx, gy, gz, B, nx, ny, nz, nbins, halting, mls,
                           _p(out), max_nodes)
    if m < 0:
        raise RuntimeError("k-d node buffer too small")
    return out[:m].copy()


# ---------------------------------------------------------------------------
# pipeline helpers (compositions of the above, used by tests and the bench)
# ---------------------------------------------------------------------------
def build_mask(vol: OVolume, tf: OTF, B):
    mn, mx = brick_minmax(vol, B)
    return brick_mask(mn, mx, tf, vol.c.value_lo, vol.c.value_hi)


def brick_boxes(ids, grid, B, dims):
    """Closed voxel-space boxes of the given bricks."""
    gx, gy, gz = grid
    ids = np.asarray(ids, dtype=np.int64)
    c = np.stack([ids % gx, (ids // gx) % gy, ids // (gx * gy)], axis=1)
    lo = c * B
    hi = np.minimum((c + 1) * B, np.array(dims))
    return np.concatenate([lo, hi], axis=1).astype(np.float32)


def kd_leaf_boxes(nodes, B, dims):
    leaves = nodes[nodes[:, 8] < 0]
    lo = leaves[:, 0:3] * B
    hi = np.minimum(leaves[:, 3:6] * B, np.array(dims))
    return np.concatenate([lo, hi], axis=1).astype(np.float32)


def lbvh_build(mask, grid):
    """Oracle LBVH: compaction, Morton keys, sort, top-down radix tree, boxes."""
    gx, gy, gz = grid
    ids = compact(mask)
    keys = morton_keys(ids, gx, gy)
    skeys, sids = sort_pairs(keys, ids)
    if skeys.shape[0] >= 2:
        left, right, ranges = lbvh_topdown(skeys)
        boxes = lbvh_boxes(sids, ranges, gx, gy)
    else:
        left = right = np.zeros(0, np.int32)
        ranges = np.zeros((0, 2), np.int32)
        boxes = np.zeros((0, 6), np.int32)
    return dict(ids=ids, keys=keys, sorted_keys=skeys, sorted_ids=sids, left=left,
                right=right, ranges=ranges, boxes=boxes)
