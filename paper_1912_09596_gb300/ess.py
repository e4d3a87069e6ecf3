"""Thin ctypes binding of libess (the C ABI in ``include/ess.h``).

Only argument marshalling happens here: every step of volume upload, empty
test, structure build and rendering runs in the library's CUDA kernels.  The
functions keep the C names (``ess_create``, ``ess_volume_upload``, ...); a
failing call raises :class:`EssError` carrying the status and the library's
message.  Buffers may be numpy arrays (host) or torch tensors (host or CUDA);
PyTorch only provides device memory and the CUDA stream.

Importing this module loads ``libess.so`` and fails loudly if it is missing:
there is no CPU fallback.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libess.so")

OK, ERR_ARG, ERR_OOM, ERR_CUDA, ERR_HANDLE, ERR_TIMEOUT, ERR_BUSY, ERR_STALE = 0, -1, -2, -3, -4, -5, -6, -7
U8, U16, F32 = 0, 1, 2
GRID, LBVH, KD, NONE, HYBRID = 0, 1, 2, 3, 4
KIND_NAMES = {GRID: "grid", LBVH: "lbvh", KD: "kd", NONE: "none", HYBRID: "hybrid"}
KINDS = (NONE, GRID, LBVH, KD)   # the paper's three structures and the naive marcher
ALL_KINDS = KINDS + (HYBRID,)    # with the hybrid grid (Sec. 3.3)
(ARR_MINMAX, ARR_MASK, ARR_IDS, ARR_KEYS, ARR_SORTED_KEYS, ARR_SORTED_IDS, ARR_LBVH_LEFT,
 ARR_LBVH_RIGHT, ARR_LBVH_BOXES, ARR_KD_NODES) = range(10)

_NP_DTYPE = {np.dtype(np.uint8): U8, np.dtype(np.uint16): U16, np.dtype(np.float32): F32}


class EssError(RuntimeError):
    def __init__(self, status, message):
        super().__init__("ess status %d: %s" % (status, message))
        self.status = status
        self.message = message


class BuildParams(C.Structure):
    _fields_ = [("brick", C.c_int), ("nbins", C.c_int), ("halting", C.c_int),
                ("mls", C.c_int), ("empty_test", C.c_int), ("rescan", C.c_int)]


class Camera(C.Structure):
    _fields_ = [("eye", C.c_float * 3), ("u", C.c_float * 3), ("v", C.c_float * 3),
                ("w", C.c_float * 3), ("ortho", C.c_int)]


class RenderParams(C.Structure):
    _fields_ = [("dt", C.c_float), ("ert", C.c_float), ("bg", C.c_float * 4),
                ("tile_w", C.c_int), ("shading", C.c_int), ("ka", C.c_float), ("kd", C.c_float),
                ("ks", C.c_float), ("shininess", C.c_int), ("dt_ref", C.c_float)]


class RenderItem(C.Structure):
    _fields_ = [("structure", C.c_uint64), ("camera", Camera), ("params", RenderParams),
                ("W", C.c_int), ("H", C.c_int), ("out", C.c_void_p)]


class ServerConfig(C.Structure):
    _fields_ = [("memory_budget", C.c_size_t), ("max_batch", C.c_int),
                ("max_inflight", C.c_int), ("tile_w", C.c_int)]


class Request(C.Structure):
    _fields_ = [("kind", C.c_int), ("structure", C.c_uint64), ("rgba", C.c_void_p),
                ("nt", C.c_int), ("camera", Camera), ("params", RenderParams),
                ("W", C.c_int), ("H", C.c_int), ("out", C.c_void_p)]


class RequestStatus(C.Structure):
    _fields_ = [("done", C.c_int), ("status", C.c_int), ("queue_ms", C.c_double),
                ("latency_ms", C.c_double)]


REQ_RENDER, REQ_EDIT = 0, 1


class TuneResult(C.Structure):
    _fields_ = [("kind", C.c_int), ("brick", C.c_int), ("tile_w", C.c_int),
                ("build_ms", C.c_float), ("render_ms", C.c_float)]


class StructureInfo(C.Structure):
    _fields_ = [("kind", C.c_int), ("brick", C.c_int), ("gx", C.c_int), ("gy", C.c_int),
                ("gz", C.c_int), ("n_bricks", C.c_int64), ("n_nonempty", C.c_int64),
                ("n_nodes", C.c_int64), ("height", C.c_int), ("device_bytes", C.c_size_t)]


def _load():
    if not os.path.exists(LIB_PATH):
        raise RuntimeError("libess.so is not built (run __graft_entry__.build()); "
                           "there is no CPU fallback")
    L = C.CDLL(LIB_PATH)
    vp, i, f, h = C.c_void_p, C.c_int, C.c_float, C.c_uint64
    P = C.POINTER
    sigs = {
        "ess_create": [i, vp, P(vp)],
        "ess_destroy": [vp],
        "ess_sync": [vp],
        "ess_release": [vp, h],
        "ess_volume_upload": [vp, vp, i, i, i, i, i, f, f, P(h)],
        "ess_tf_set": [vp, vp, i, i, P(h)],
        "ess_volume_set_sampler": [vp, h, i],
        "ess_tf_update": [vp, h, vp, i, i],
        "ess_build": [vp, h, h, i, P(BuildParams), P(h)],
        "ess_rebuild": [vp, h],
        "ess_rebuild_batch": [vp, P(h), i],
        "ess_structure_info_get": [vp, h, P(StructureInfo)],
        "ess_structure_read": [vp, h, i, vp, C.c_size_t, P(C.c_size_t)],
        "ess_render": [vp, h, P(Camera), P(RenderParams), i, i, vp, i],
        "ess_sample_count": [vp, P(C.c_uint64), i],
        "ess_profile_enable": [vp, i],
        "ess_profile_read": [vp, i, P(C.c_char_p), P(C.c_uint64), P(C.c_double), P(i)],
        "ess_profile_reset": [vp],
        "ess_selftest_wait": [vp, i, C.c_int64],
        "ess_compact_mask_noalloc": [vp, C.c_int64, vp, vp, vp],
        "ess_render_batch": [vp, P(RenderItem), i, i],
        "ess_server_create": [vp, P(ServerConfig), P(vp)],
        "ess_server_submit": [vp, P(Request), P(C.c_uint64)],
        "ess_server_poll": [vp, C.c_uint64, P(RequestStatus)],
        "ess_server_wait": [vp, C.c_uint64, P(RequestStatus)],
        "ess_server_drain": [vp],
        "ess_server_destroy": [vp],
        "ess_autotune": [vp, h, h, P(Camera), i, P(RenderParams), i, i, f, P(TuneResult)],
    }
    for name, args in sigs.items():
        fn = getattr(L, name)
        fn.argtypes = args
        fn.restype = i
    L.ess_last_error.argtypes = [vp]
    L.ess_last_error.restype = C.c_char_p
    L.ess_launch_count.argtypes = [vp]
    L.ess_launch_count.restype = C.c_uint64
    return L


lib = _load()


def _check(ctx, st):
    if st != OK:
        msg = lib.ess_last_error(ctx) if ctx else b""
        raise EssError(st, (msg or b"").decode())


def _ptr(buf):
    """(address, on_device) of a numpy array or torch tensor (contiguous)."""
    if isinstance(buf, np.ndarray):
        if not buf.flags["C_CONTIGUOUS"]:
            raise ValueError("buffer must be C-contiguous")
        return buf.ctypes.data, 0
    if hasattr(buf, "data_ptr"):
        if not buf.is_contiguous():
            raise ValueError("tensor must be contiguous")
        return buf.data_ptr(), int(buf.is_cuda)
    raise TypeError("expected a numpy array or a torch tensor")


def _dtype_code(buf):
    if isinstance(buf, np.ndarray):
        return _NP_DTYPE[buf.dtype]
    import torch
    return {torch.uint8: U8, torch.uint16: U16, torch.float32: F32}[buf.dtype]


# ------------------------------------------------------------------ the ABI
def ess_create(device=0, stream=None):
    """`stream`: a torch.cuda.Stream, a raw cudaStream_t int, or None."""
    raw = getattr(stream, "cuda_stream", stream)
    ctx = C.c_void_p()
    _check(None, lib.ess_create(device, C.c_void_p(raw) if raw else None, C.byref(ctx)))
    return ctx


def ess_destroy(ctx):
    _check(None, lib.ess_destroy(ctx))


def ess_last_error(ctx):
    return (lib.ess_last_error(ctx) or b"").decode()


def ess_sync(ctx):
    _check(ctx, lib.ess_sync(ctx))


def ess_release(ctx, handle):
    _check(ctx, lib.ess_release(ctx, handle))


def ess_volume_upload(ctx, data, value_lo, value_hi):
    """`data`: (nz, ny, nx) uint8 / uint16 / float32 array or tensor."""
    nz, ny, nx = data.shape
    p, dev = _ptr(data)
    h = C.c_uint64()
    _check(ctx, lib.ess_volume_upload(ctx, p, dev, _dtype_code(data), nx, ny, nz,
                                      float(value_lo), float(value_hi), C.byref(h)))
    return h.value


def ess_volume_set_sampler(ctx, vol, cells):
    _check(ctx, lib.ess_volume_set_sampler(ctx, vol, int(cells)))


def ess_tf_set(ctx, rgba):
    """`rgba`: (nt, 4) float32 array or tensor."""
    p, dev = _ptr(rgba)
    h = C.c_uint64()
    _check(ctx, lib.ess_tf_set(ctx, p, dev, int(rgba.shape[0]), C.byref(h)))
    return h.value


def ess_tf_update(ctx, tf, rgba):
    p, dev = _ptr(rgba)
    _check(ctx, lib.ess_tf_update(ctx, tf, p, dev, int(rgba.shape[0])))


def build_params(brick=8, nbins=4, halting=1, mls=0, empty_test=0, rescan=0):
    return BuildParams(brick, nbins, halting, mls, empty_test, rescan)


def ess_build(ctx, vol, tf, kind, params=None):
    params = params or build_params()
    h = C.c_uint64()
    _check(ctx, lib.ess_build(ctx, vol, tf, kind, C.byref(params), C.byref(h)))
    return h.value


def ess_rebuild(ctx, structure):
    _check(ctx, lib.ess_rebuild(ctx, structure))


def ess_rebuild_batch(ctx, structures):
    arr = (C.c_uint64 * len(structures))(*structures)
    _check(ctx, lib.ess_rebuild_batch(ctx, arr, len(structures)))


def ess_structure_info_get(ctx, structure):
    info = StructureInfo()
    _check(ctx, lib.ess_structure_info_get(ctx, structure, C.byref(info)))
    return {k: getattr(info, k) for k, _ in StructureInfo._fields_}


_ARR_DTYPE = {ARR_MINMAX: np.float32, ARR_MASK: np.uint8, ARR_IDS: np.uint32,
              ARR_KEYS: np.uint32, ARR_SORTED_KEYS: np.uint32, ARR_SORTED_IDS: np.uint32,
              ARR_LBVH_LEFT: np.int32, ARR_LBVH_RIGHT: np.int32, ARR_LBVH_BOXES: np.int32,
              ARR_KD_NODES: np.int32}


def ess_structure_read(ctx, structure, which, capacity=None):
    """Returns the array as numpy (1-d; reshape per include/ess.h)."""
    if capacity is None:
        info = ess_structure_info_get(ctx, structure)
        capacity = 16 * max(info["n_bricks"], 9 * info["n_nodes"], 1) + 64
    buf = np.empty(capacity, dtype=np.uint8)
    written = C.c_size_t()
    _check(ctx, lib.ess_structure_read(ctx, structure, which, buf.ctypes.data, capacity,
                                       C.byref(written)))
    return buf[: written.value].view(_ARR_DTYPE[which]).copy()


def camera(eye, u, v, w, ortho=0):
    c = Camera()
    for name, val in (("eye", eye), ("u", u), ("v", v), ("w", w)):
        for i in range(3):
            getattr(c, name)[i] = float(val[i])
    c.ortho = int(ortho)
    return c


def camera_from(cam):
    """From any object with eye/u/v/w/ortho attributes (e.g. synth.Camera)."""
    return camera(cam.eye, cam.u, cam.v, cam.w, cam.ortho)


def render_params(dt=0.5, ert=2.0, bg=(0.0, 0.0, 0.0, 0.0), tile_w=0, shade=None, dt_ref=0.0):
    """`shade`: None (off) or (ka, kd, ks, shininess) for gradient shading;
    `dt_ref` > 0 switches on the opacity correction."""
    p = RenderParams()
    p.dt = dt
    p.ert = ert
    for i in range(4):
        p.bg[i] = float(bg[i])
    p.tile_w = int(tile_w)
    if shade is not None:
        p.shading = 1
        p.ka, p.kd, p.ks = float(shade[0]), float(shade[1]), float(shade[2])
        p.shininess = int(shade[3])
    p.dt_ref = float(dt_ref)
    return p


def ess_render(ctx, structure, cam, params, W, H, out):
    """`out`: (H, W, 4) float32 numpy array (host) or CUDA tensor (device)."""
    if not isinstance(cam, Camera):
        cam = camera_from(cam)
    p, dev = _ptr(out)
    _check(ctx, lib.ess_render(ctx, structure, C.byref(cam), C.byref(params), W, H, p, dev))
    return out


def ess_compact_mask_noalloc(mask, ids, count, stream=None):
    """`mask`: device uint8 tensor of n bricks; `ids`: device int32/uint32
    tensor of at least n entries; `count`: device int32 tensor of 1 entry.
    Raises EssError on a non-OK status (there is no context message)."""
    raw = getattr(stream, "cuda_stream", stream)
    st = lib.ess_compact_mask_noalloc(_ptr(mask)[0], int(mask.numel()), _ptr(ids)[0],
                                      _ptr(count)[0], C.c_void_p(raw) if raw else None)
    if st != OK:
        raise EssError(st, "ess_compact_mask_noalloc failed")


def ess_render_batch(ctx, items, tile_w=0):
    """`items`: list of (structure, camera, params, W, H, out CUDA tensor)."""
    arr = (RenderItem * len(items))()
    for k, (st, cam, params, W, H, out) in enumerate(items):
        if not isinstance(cam, Camera):
            cam = camera_from(cam)
        p, dev = _ptr(out)
        if not dev:
            raise ValueError("batched outputs must be device memory")
        arr[k] = RenderItem(st, cam, params, W, H, p)
    _check(ctx, lib.ess_render_batch(ctx, arr, len(items), int(tile_w)))


def ess_autotune(ctx, vol, tf, cameras, params, W, H, frames_per_edit=1.0):
    cams = (Camera * len(cameras))(*[c if isinstance(c, Camera) else camera_from(c)
                                      for c in cameras])
    res = TuneResult()
    _check(ctx, lib.ess_autotune(ctx, vol, tf, cams, len(cameras), C.byref(params), W, H,
                                 float(frames_per_edit), C.byref(res)))
    return {k: getattr(res, k) for k, _ in TuneResult._fields_}


def ess_server_create(ctx, memory_budget=0, max_batch=256, max_inflight=2, tile_w=0):
    srv = C.c_void_p()
    cfg = ServerConfig(memory_budget, max_batch, max_inflight, tile_w)
    st = lib.ess_server_create(ctx, C.byref(cfg), C.byref(srv))
    if st != OK:
        raise EssError(st, "ess_server_create failed")
    return srv


def ess_server_submit(srv, kind, structure, cam, params, W, H, out, rgba=None):
    """`out`: host float32 (H, W, 4) numpy array or pinned tensor that stays
    alive until the request is done; `rgba`: (nt, 4) host table for an edit."""
    if not isinstance(cam, Camera):
        cam = camera_from(cam)
    p_out, dev = _ptr(out)
    if dev:
        raise ValueError("server outputs are host memory")
    p_tf, nt = (None, 0)
    if rgba is not None:
        p_tf, _ = _ptr(rgba)
        nt = int(rgba.shape[0])
    req = Request(kind, structure, p_tf, nt, cam, params, W, H, p_out)
    rid = C.c_uint64()
    st = lib.ess_server_submit(srv, C.byref(req), C.byref(rid))
    if st != OK:
        raise EssError(st, "ess_server_submit failed")
    return rid.value


def _status(fn, srv, rid):
    s = RequestStatus()
    st = fn(srv, rid, C.byref(s))
    if st != OK:
        raise EssError(st, "unknown request")
    return {k: getattr(s, k) for k, _ in RequestStatus._fields_}


def ess_server_poll(srv, rid):
    return _status(lib.ess_server_poll, srv, rid)


def ess_server_wait(srv, rid):
    return _status(lib.ess_server_wait, srv, rid)


def ess_server_drain(srv):
    if lib.ess_server_drain(srv) != OK:
        raise EssError(ERR_ARG, "ess_server_drain failed")


def ess_server_destroy(srv):
    if lib.ess_server_destroy(srv) != OK:
        raise EssError(ERR_ARG, "ess_server_destroy failed")


def ess_launch_count(ctx):
    return int(lib.ess_launch_count(ctx))


def ess_sample_count(ctx, reset=False):
    v = C.c_uint64()
    _check(ctx, lib.ess_sample_count(ctx, C.byref(v), int(bool(reset))))
    return v.value


def ess_profile_enable(ctx, enable=True):
    _check(ctx, lib.ess_profile_enable(ctx, int(bool(enable))))


def ess_profile_read(ctx):
    """{kernel name: (launches, total ms)}"""
    n = C.c_int()
    _check(ctx, lib.ess_profile_read(ctx, 0, None, None, None, C.byref(n)))
    m = n.value
    names = (C.c_char_p * max(1, m))()
    launches = (C.c_uint64 * max(1, m))()
    ms = (C.c_double * max(1, m))()
    _check(ctx, lib.ess_profile_read(ctx, m, names, launches, ms, C.byref(n)))
    return {names[i].decode(): (int(launches[i]), float(ms[i])) for i in range(m)}


def ess_profile_reset(ctx):
    _check(ctx, lib.ess_profile_reset(ctx))


def ess_selftest_wait(ctx, set_flag, polls):
    _check(ctx, lib.ess_selftest_wait(ctx, int(bool(set_flag)), int(polls)))
