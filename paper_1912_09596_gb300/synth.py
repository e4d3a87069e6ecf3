"""Seeded synthetic inputs: volumes, RGBA transfer functions and camera bases.

This module only *makes inputs*. It holds none of the method's arithmetic (no
classification, no sampling, no skipping structure), so both the CPU oracle and
the CUDA path can take their inputs from here without sharing any of the
computation they are checked on.

The paper's data sets (Section 4, Fig. "Data sets": Aneurism, Magnetic,
N-Body, ...) are not available, so every workload here is a seeded stand-in
with the size, dtype and occupancy range of the paper's workloads (0.15 % to
50 % occupancy, 256^3 to 2048^3 voxels, 8-bit voxels in the paper).

All generators use numpy's PCG64 (``np.random.default_rng``), which gives the
same stream on every platform.  Floating-point field construction may differ in
the last ulp between machines (libm, BLAS); tests therefore always generate an
input once and hand the *same bytes* to both sides.
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np

DTYPES = {"u8": np.uint8, "u16": np.uint16, "f32": np.float32}


# ---------------------------------------------------------------------------
# smooth value noise (Perlin-style), separable so that 512^3 and 1024^3 fields
# are cheap to make: a coarse random lattice is upsampled one axis at a time
# with quintic "fade" weights.
# ---------------------------------------------------------------------------
def _fade_matrix(n_out: int, n_cells: int) -> np.ndarray:
    """(n_out, n_cells+1) matrix mapping lattice values to n_out samples."""
    x = (np.arange(n_out, dtype=np.float64) + 0.5) * (n_cells / n_out)
    i0 = np.minimum(np.floor(x).astype(np.int64), n_cells - 1)
    f = x - i0
    w = f * f * f * (f * (f * 6.0 - 15.0) + 10.0)
    m = np.zeros((n_out, n_cells + 1), dtype=np.float64)
    m[np.arange(n_out), i0] = 1.0 - w
    m[np.arange(n_out), i0 + 1] += w
    return m


def value_noise(dims, cells, rng, chunk=64) -> np.ndarray:
    """Smooth noise in [-1, 1] of shape (nz, ny, nx), lattice of `cells` per axis."""
    nx, ny, nz = dims
    cx, cy, cz = (cells, cells, cells) if np.isscalar(cells) else cells
    lat = rng.uniform(-1.0, 1.0, size=(cz + 1, cy + 1, cx + 1))
    mx, my, mz = _fade_matrix(nx, cx), _fade_matrix(ny, cy), _fade_matrix(nz, cz)
    a = np.einsum("zyc,xc->zyx", lat, mx)          # (cz+1, cy+1, nx)
    a = np.einsum("zcx,yc->zyx", a, my)            # (cz+1, ny, nx)
    out = np.empty((nz, ny, nx), dtype=np.float32)
    a2 = a.reshape(cz + 1, ny * nx)
    for z0 in range(0, nz, chunk):
        z1 = min(nz, z0 + chunk)
        out[z0:z1] = (mz[z0:z1] @ a2).reshape(z1 - z0, ny, nx)
    return out


# ---------------------------------------------------------------------------
# volumes
# ---------------------------------------------------------------------------
def blobs_u8(dims=(64, 64, 64), n_blobs=12, seed=0, sigma=(3.0, 6.0), iso=40,
             target_frac=0.10, noise_max=8) -> np.ndarray:
    """Gaussian blobs plus uniform noise, uint8, shape (nz, ny, nx).

    The amplitude is set so that about `target_frac` of the voxels reach `iso`
    (the first visible value of the matching transfer function)."""
    nx, ny, nz = dims
    rng = np.random.default_rng(seed)
    centres = rng.uniform(0.0, 1.0, size=(n_blobs, 3)) * np.array([nx, ny, nz])
    sig = rng.uniform(sigma[0], sigma[1], size=n_blobs)
    z, y, x = np.meshgrid(np.arange(nz) + 0.5, np.arange(ny) + 0.5,
                          np.arange(nx) + 0.5, indexing="ij")
    field = np.zeros((nz, ny, nx), dtype=np.float64)
    for c, s in zip(centres, sig):
        r2 = (x - c[0]) ** 2 + (y - c[1]) ** 2 + (z - c[2]) ** 2
        field += np.exp(-r2 / (2.0 * s * s))
    q = np.quantile(field, 1.0 - target_frac)
    amp = iso / max(q, 1e-12)
    noise = rng.uniform(0.0, noise_max, size=field.shape)
    return np.clip(np.rint(amp * field + noise), 0, 255).astype(np.uint8)


def _stamp_tube(vol, pts, radius, value):
    """Rasterise a tube (max-blend) by stamping balls along a polyline."""
    nz, ny, nx = vol.shape
    r = int(math.ceil(radius))
    oz, oy, ox = np.meshgrid(np.arange(-r, r + 1), np.arange(-r, r + 1),
                             np.arange(-r, r + 1), indexing="ij")
    ball = (ox ** 2 + oy ** 2 + oz ** 2) <= radius * radius
    offs = np.stack([ox[ball], oy[ball], oz[ball]], axis=1)
    for p in pts:
        c = np.rint(p).astype(np.int64)
        q = offs + c
        ok = ((q[:, 0] >= 0) & (q[:, 0] < nx) & (q[:, 1] >= 0) & (q[:, 1] < ny)
              & (q[:, 2] >= 0) & (q[:, 2] < nz))
        q = q[ok]
        cur = vol[q[:, 2], q[:, 1], q[:, 0]]
        vol[q[:, 2], q[:, 1], q[:, 0]] = np.maximum(cur, value)


def ct_like_u8(dims=(512, 512, 512), seed=1, n_vessels=24) -> np.ndarray:
    """CT-like uint8 volume: concentric noisy shells, thin tubular vessels and
    2 % smooth noise, shape (nz, ny, nx)."""
    nx, ny, nz = dims
    rng = np.random.default_rng(seed)
    wob = value_noise(dims, 6, rng)                      # shell radius wobble
    fine = value_noise(dims, max(4, nx // 16), rng)      # 2 % texture noise
    zc, yc, xc = (nz / 2.0, ny / 2.0, nx / 2.0)
    half = 0.5 * min(nx, ny, nz)
    out = np.zeros((nz, ny, nx), dtype=np.float32)
    shells = [(0.30, 0.030, 70.0), (0.52, 0.025, 120.0), (0.72, 0.030, 165.0),
              (0.90, 0.020, 215.0)]
    for z0 in range(0, nz, 32):
        z1 = min(nz, z0 + 32)
        z = (np.arange(z0, z1, dtype=np.float32) + 0.5 - zc)[:, None, None]
        y = (np.arange(ny, dtype=np.float32) + 0.5 - yc)[None, :, None]
        x = (np.arange(nx, dtype=np.float32) + 0.5 - xc)[None, None, :]
        r = np.sqrt(x * x + y * y + z * z) / half + 0.04 * wob[z0:z1]
        acc = np.zeros((z1 - z0, ny, nx), dtype=np.float32)
        for rad, th, val in shells:
            d = np.abs(r - rad) / th
            acc = np.maximum(acc, val * np.clip(1.0 - d * d, 0.0, 1.0))
        out[z0:z1] = acc
    out += 0.02 * 255.0 * fine
    vol = np.clip(np.rint(out), 0, 255).astype(np.uint8)
    # vessels: random smooth curves inside the outer shell
    for _ in range(n_vessels):
        p0 = rng.uniform(0.15, 0.85, size=3) * np.array([nx, ny, nz])
        d0 = rng.normal(size=3)
        d0 /= np.linalg.norm(d0)
        bend = rng.normal(size=3) * 0.02
        length = int(rng.uniform(0.3, 0.8) * nx)
        pts = []
        p, d = p0.copy(), d0.copy()
        for _s in range(length):
            pts.append(p.copy())
            d = d + bend + rng.normal(size=3) * 0.01
            d /= np.linalg.norm(d)
            p = p + d
        radius = rng.uniform(1.2, 3.0) * nx / 512.0 + 0.6
        value = int(rng.uniform(200, 255))
        _stamp_tube(vol, pts, radius, value)
    return vol


def fractal_f32(dims=(1024, 1024, 1024), seed=2, octaves=4, threshold=0.42,
                base_cells=8) -> np.ndarray:
    """Sparse simulation-like float32 field in [0, 1], shape (nz, ny, nx):
    `octaves` of smooth noise summed with halving amplitude, then everything
    below `threshold` (about 1-5 % of voxels remain above) is set to 0 and the
    rest is rescaled to (0, 1]."""
    rng = np.random.default_rng(seed)
    acc = None
    amp, total = 1.0, 0.0
    for o in range(octaves):
        n = value_noise(dims, base_cells * (2 ** o), rng)
        acc = n * amp if acc is None else acc + n * amp
        total += amp
        amp *= 0.5
    acc *= 1.0 / total                                   # ~[-1, 1]
    acc = np.clip((acc - threshold) / (1.0 - threshold), 0.0, 1.0)
    return acc.astype(np.float32)


def fractal_f32_torch(dims=(1024, 1024, 1024), seed=2, octaves=4, threshold=0.42,
                      base_cells=8, device="cuda"):
    """The fractal_f32 field computed with torch on `device` (for sizes that
    numpy makes slowly): the same seeded lattices and fade matrices; float32
    matrix products, so values may differ from fractal_f32 in low bits.
    Returns a contiguous (nz, ny, nx) float32 tensor."""
    import torch
    nx, ny, nz = dims
    rng = np.random.default_rng(seed)
    acc = torch.zeros((nz, ny, nx), dtype=torch.float32, device=device)
    amp, total = 1.0, 0.0
    for o in range(octaves):
        c = base_cells * (2 ** o)
        lat = torch.from_numpy(rng.uniform(-1.0, 1.0, size=(c + 1, c + 1, c + 1))).to(device)
        mx = torch.from_numpy(_fade_matrix(nx, c)).to(device)
        my = torch.from_numpy(_fade_matrix(ny, c)).to(device)
        mz = torch.from_numpy(_fade_matrix(nz, c)).to(device)
        a = torch.einsum("zyc,xc->zyx", lat, mx)
        a = torch.einsum("zcx,yc->zyx", a, my).float().reshape(c + 1, ny * nx)
        mzf = mz.float()
        for z0 in range(0, nz, 128):
            z1 = min(nz, z0 + 128)
            acc[z0:z1] += amp * (mzf[z0:z1] @ a).reshape(z1 - z0, ny, nx)
        total += amp
        amp *= 0.5
    acc *= 1.0 / total
    acc = ((acc - threshold) / (1.0 - threshold)).clamp_(0.0, 1.0)
    return acc.contiguous()


def ct_like_u16(dims=(512, 512, 512), seed=3) -> np.ndarray:
    """uint16 variant of the CT-like volume (values scaled by 257 plus a
    low-order smooth noise so that all 16 bits are in use)."""
    v8 = ct_like_u8(dims, seed=seed)
    rng = np.random.default_rng(seed + 1000)
    n = value_noise(dims, 8, rng)
    v = v8.astype(np.float32) * 257.0 + 96.0 * n
    return np.clip(np.rint(v), 0, 65535).astype(np.uint16)


def menger_u8(n=81, level=None, value=200) -> np.ndarray:
    """Menger sponge sampled on an n^3 grid (n a power of 3 gives the exact
    sponge): voxel (i,j,k) is solid unless, at some level, two or more of its
    base-3 digits are 1.  Solid voxels get `value`, holes 0."""
    if level is None:
        level = max(1, int(round(math.log(n, 3))))
    m = 3 ** level
    cell = (np.arange(n) * m) // n            # sponge cell of each voxel row
    solid = np.ones((n, n, n), dtype=bool)
    for l in range(level):
        one = ((cell // (3 ** l)) % 3 == 1).astype(np.int8)
        cnt = one[:, None, None] + one[None, :, None] + one[None, None, :]
        solid &= cnt < 2
    return np.where(solid, value, 0).astype(np.uint8)


def random_u8(dims, seed, p_zero=0.7, hi=255) -> np.ndarray:
    """Sparse random uint8 volume for small property tests."""
    nx, ny, nz = dims
    rng = np.random.default_rng(seed)
    v = rng.integers(1, hi + 1, size=(nz, ny, nx))
    v[rng.random(size=v.shape) < p_zero] = 0
    return v.astype(np.uint8)


# ---------------------------------------------------------------------------
# transfer functions: float32 RGBA tables, shape (NT, 4), alpha in [0, 1]
# ---------------------------------------------------------------------------
def _rgb_ramp(nt):
    t = np.linspace(0.0, 1.0, nt)
    return np.stack([t, 0.25 + 0.5 * t * (1.0 - t), 1.0 - t], axis=1)


def tf_ramp(nt=256, start=40, end=None, alpha_max=1.0) -> np.ndarray:
    """Alpha 0 below entry `start`, linear ramp to `alpha_max` at `end`."""
    end = nt - 1 if end is None else end
    tf = np.zeros((nt, 4), dtype=np.float64)
    tf[:, :3] = _rgb_ramp(nt)
    i = np.arange(nt)
    a = np.clip((i - start + 1) / max(1, end - start + 1), 0.0, 1.0) * alpha_max
    a[i < start] = 0.0
    tf[:, 3] = a
    return tf.astype(np.float32)


def tf_window(nt, lo, hi, alpha_max=0.6) -> np.ndarray:
    """Alpha > 0 only for entries in [lo, hi] (a tent over the window)."""
    tf = np.zeros((nt, 4), dtype=np.float64)
    tf[:, :3] = _rgb_ramp(nt)
    i = np.arange(nt, dtype=np.float64)
    c = 0.5 * (lo + hi)
    hw = max(0.5 * (hi - lo), 0.5)
    a = alpha_max * np.clip(1.0 - np.abs(i - c) / (hw + 1.0), 0.0, 1.0)
    a[(i < lo) | (i > hi)] = 0.0
    tf[:, 3] = a
    return tf.astype(np.float32)


# alpha windows (entry ranges of a 256-entry table) used with ct_like_u8; they
# select different shells / vessels and give 5-30 % non-empty 8^3 bricks.
CT_WINDOWS = [(200, 255), (150, 185), (100, 135), (60, 90), (190, 230),
              (110, 180), (216, 255), (55, 125)]


def tf_set_ct(nt=256):
    """The 8 transfer functions of the 512^3 CT-like workload."""
    return [tf_window(nt, lo * (nt - 1) // 255, hi * (nt - 1) // 255,
                      alpha_max=0.35 + 0.05 * k)
            for k, (lo, hi) in enumerate(CT_WINDOWS)]


def tf_piecewise_random(nt, seed, knots_range=(4, 8)) -> np.ndarray:
    """Random piecewise-linear RGBA table with 4-8 knots; alpha is 0 on at
    least the lowest quarter so that empty space exists."""
    rng = np.random.default_rng(seed)
    k = int(rng.integers(knots_range[0], knots_range[1] + 1))
    xs = np.sort(rng.uniform(0.25, 1.0, size=k))
    xs[0] = max(xs[0], 0.25)
    ys = rng.uniform(0.0, 1.0, size=(k, 4))
    ys[:, 3] = np.where(rng.random(k) < 0.35, 0.0, ys[:, 3] * 0.8)
    ys[0, 3] = 0.0
    xi = np.linspace(0.0, 1.0, nt)
    tf = np.empty((nt, 4))
    for c in range(4):
        tf[:, c] = np.interp(xi, xs, ys[:, c], left=ys[0, c], right=ys[-1, c])
    tf[xi < xs[0], 3] = 0.0
    return np.clip(tf, 0.0, 1.0).astype(np.float32)


def tf_random_sparse(nt, seed, p_zero=0.6) -> np.ndarray:
    """Random table with many exact-zero alpha entries (property tests)."""
    rng = np.random.default_rng(seed)
    tf = rng.uniform(0.0, 1.0, size=(nt, 4))
    tf[rng.random(nt) < p_zero, 3] = 0.0
    return tf.astype(np.float32)


# ---------------------------------------------------------------------------
# cameras: a host-side basis (eye, u, v, w) in float32, world units = voxels,
# volume box [0,nx]x[0,ny]x[0,nz]
# ---------------------------------------------------------------------------
@dataclass
class Camera:
    eye: np.ndarray
    u: np.ndarray
    v: np.ndarray
    w: np.ndarray
    ortho: int

    def as_floats(self):
        return [float(x) for x in np.concatenate([self.eye, self.u, self.v, self.w])]


def orbit_camera(dims, W, H, theta, phi=0.35, dist=1.8, fov_deg=40.0,
                 ortho=False) -> Camera:
    """Camera on a sphere around the volume centre looking at it.

    Perspective: w is the unit forward vector, u/v are right/up scaled by
    tan(fov/2) (u also by the aspect ratio).  Orthographic: u/v are the
    half-extents of the view plane, sized so that the volume fills it."""
    nx, ny, nz = dims
    c = np.array([nx, ny, nz], dtype=np.float64) * 0.5
    radius = 0.5 * math.sqrt(nx * nx + ny * ny + nz * nz)
    fwd = -np.array([math.cos(phi) * math.sin(theta), math.sin(phi),
                     math.cos(phi) * math.cos(theta)])
    eye = c - fwd * radius * dist
    upw = np.array([0.0, 1.0, 0.0])
    right = np.cross(fwd, upw)
    right /= np.linalg.norm(right)
    up = np.cross(right, fwd)
    aspect = W / H
    if ortho:
        hh = radius
        u = right * hh * aspect
        v = up * hh
    else:
        t = math.tan(math.radians(fov_deg) * 0.5)
        u = right * t * aspect
        v = up * t
    f32 = lambda a: np.asarray(a, dtype=np.float32)
    return Camera(f32(eye), f32(u), f32(v), f32(fwd), int(bool(ortho)))


def axis_ortho_camera(dims, axis=2, half=None, offset=(0.0, 0.0), eye_back=8.0):
    """Orthographic camera looking along +axis, centred on the volume."""
    n = np.array(dims, dtype=np.float64)
    c = n * 0.5
    w = np.zeros(3)
    w[axis] = 1.0
    a1, a2 = [a for a in range(3) if a != axis]
    u = np.zeros(3)
    v = np.zeros(3)
    h = (0.5 * n[a1], 0.5 * n[a2]) if half is None else half
    u[a1] = h[0]
    v[a2] = h[1]
    eye = c.copy()
    eye[axis] = -eye_back
    eye[a1] += offset[0]
    eye[a2] += offset[1]
    f32 = lambda a: np.asarray(a, dtype=np.float32)
    return Camera(f32(eye), f32(u), f32(v), f32(w), 1)


def random_camera(dims, rng, ortho=None) -> Camera:
    """Random perspective or orthographic view of the volume (tests)."""
    W = H = 1
    if ortho is None:
        ortho = bool(rng.random() < 0.3)
    cam = orbit_camera(dims, W, H, theta=float(rng.uniform(0, 2 * math.pi)),
                       phi=float(rng.uniform(-1.2, 1.2)),
                       dist=float(rng.uniform(1.1, 2.5)),
                       fov_deg=float(rng.uniform(25, 70)), ortho=ortho)
    return cam
