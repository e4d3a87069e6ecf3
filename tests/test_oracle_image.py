"""Pins of the oracle's image arithmetic (R1, R2, R5, R6, R7, S) against facts
fixed outside the oracle: closed forms, library routines and special cases."""
import math

import numpy as np
import pytest
from scipy import ndimage

from paper_1912_09596_gb300 import synth


def bits(a):
    return np.ascontiguousarray(a, dtype=np.float32).view(np.uint32)


# --------------------------------------------------------------- R6 closed form
@pytest.mark.parametrize("a", [0.01, 0.05, 0.2, 0.6, 1.0])
@pytest.mark.parametrize("nz", [8, 37])
def test_constant_slab_transmittance(ora, a, nz):
    """Constant volume, axis-aligned orthographic rays: n samples of alpha a
    give 1 - A = (1-a)^n and C = c (1 - (1-a)^n) (absorption + emission,
    Sec. 4.1), within n * 4 * 2^-24 in double."""
    v = np.full((nz, 6, 6), 100, dtype=np.uint8)
    tf = np.zeros((256, 4), dtype=np.float32)
    c = np.array([0.3, 0.6, 0.9], dtype=np.float32)
    tf[:, :3] = c
    tf[:, 3] = a
    vol, otf = ora.OVolume(v, 0, 255), ora.OTF(tf)
    cam = synth.axis_ortho_camera(vol.dims, axis=2, half=(2.0, 2.0), eye_back=8.0)
    img, nsamp = ora.render_naive(vol, otf, cam, 4, 4, dt=0.5)
    n = 2 * nz                                   # t_near = 8, t_far = 8 + nz, dt = 0.5
    assert nsamp == 16 * n
    T = (1.0 - np.float64(np.float32(a))) ** n
    tol = n * 4 * 2.0 ** -24
    assert np.all(np.abs(img[..., 3] - (1.0 - T)) <= tol)
    for ch in range(3):
        assert np.all(np.abs(img[..., ch] - c[ch] * (1.0 - T)) <= tol)


def test_constant_volume_any_direction(ora):
    """For any ray through a constant volume, A = 1 - (1-a)^n with n the
    ray's own sample count."""
    v = np.full((20, 24, 28), 7, dtype=np.uint8)
    tf = np.zeros((256, 4), dtype=np.float32)
    tf[:, 3] = 0.03
    tf[:, 0] = 1.0
    vol, otf = ora.OVolume(v, 0, 255), ora.OTF(tf)
    rng = np.random.default_rng(5)
    for _ in range(6):
        cam = synth.random_camera(vol.dims, rng)
        for (x, y) in [(0, 0), (3, 5), (7, 7)]:
            img, n = ora.render_naive(vol, otf, cam, 8, 8, rows=(y, y + 1))
            px = img[y, x]
            # n counts the whole row: re-render the single pixel's count
            o, d = ora.ray(cam, x, y, 8, 8)
            tn, tf_ = ora.slab(o, d, [0, 0, 0], list(vol.dims))
            k = 0
            while tn < tf_ and np.float32(np.float32(k) * np.float32(0.5) + np.float32(tn)) < tf_:
                k += 1
            T = (1.0 - np.float64(np.float32(0.03))) ** k
            assert abs(px[3] - (1 - T)) <= (k + 1) * 4 * 2.0 ** -24
            assert abs(px[0] - (1 - T)) <= (k + 1) * 4 * 2.0 ** -24


def test_all_empty_is_background(ora):
    """A transfer function with alpha 0 everywhere returns the background
    exactly, whatever the volume and camera."""
    v = synth.random_u8((17, 13, 11), seed=3, p_zero=0.2)
    tf = synth.tf_random_sparse(256, seed=1)
    tf[:, 3] = 0.0
    bg = (0.1, 0.2, 0.3, 0.4)
    vol, otf = ora.OVolume(v, 0, 255), ora.OTF(tf)
    rng = np.random.default_rng(0)
    for _ in range(4):
        cam = synth.random_camera(vol.dims, rng)
        img, _ = ora.render_naive(vol, otf, cam, 9, 7, bg=bg)
        assert np.array_equal(bits(img), bits(np.broadcast_to(np.float32(bg), img.shape)))


def test_miss_is_background(ora):
    v = np.full((8, 8, 8), 255, dtype=np.uint8)
    vol, otf = ora.OVolume(v, 0, 255), ora.OTF(synth.tf_ramp(256, 0))
    cam = synth.axis_ortho_camera(vol.dims, axis=2, half=(4.0, 4.0), offset=(100.0, 0.0))
    img, n = ora.render_naive(vol, otf, cam, 4, 4, bg=(1, 0, 0, 1))
    assert n == 0 and np.all(img == np.float32([1, 0, 0, 1]))


# ---------------------------------------------------------------- R2 sampling
def test_sample_at_voxel_centres_is_exact(ora):
    v = synth.random_u8((9, 7, 5), seed=2, p_zero=0.0)
    vol = ora.OVolume(v, 0, 255)
    for k in range(5):
        for j in range(7):
            for i in range(9):
                assert ora.sample_value(vol, (i + 0.5, j + 0.5, k + 0.5)) == float(v[k, j, i])


def test_sample_constant_volume(ora):
    v = np.full((6, 6, 6), 0.3, dtype=np.float32)
    vol = ora.OVolume(v, 0, 1)
    rng = np.random.default_rng(1)
    for p in rng.uniform(-1, 7, size=(200, 3)):
        assert ora.sample_value(vol, p) == np.float32(0.3)


@pytest.mark.parametrize("dtype", ["u8", "u16", "f32"])
def test_sample_matches_scipy_trilinear(ora, dtype):
    """R2 against scipy's order-1 spline (trilinear) with clamp-to-edge:
    voxel centre at i+0.5 means map_coordinates index p - 0.5."""
    rng = np.random.default_rng(7)
    shape = (7, 9, 11)  # (nz, ny, nx)
    if dtype == "f32":
        v = rng.standard_normal(shape).astype(np.float32)
    elif dtype == "u16":
        v = rng.integers(0, 65536, size=shape).astype(np.uint16)
    else:
        v = rng.integers(0, 256, size=shape).astype(np.uint8)
    vol = ora.OVolume(v, 0, 1)
    pts = rng.uniform(-0.8, 1.0, size=(500, 3)) * np.array([11.6, 9.6, 7.6])
    ref = ndimage.map_coordinates(v.astype(np.float64),
                                  [pts[:, 2] - 0.5, pts[:, 1] - 0.5, pts[:, 0] - 0.5],
                                  order=1, mode="nearest")
    got = np.array([ora.sample_value(vol, p.astype(np.float32)) for p in pts])
    scale = float(np.abs(v.astype(np.float64)).max())
    ref32 = ndimage.map_coordinates(v.astype(np.float64),
                                    [np.float32(pts[:, 2]) - 0.5, np.float32(pts[:, 1]) - 0.5,
                                     np.float32(pts[:, 0]) - 0.5], order=1, mode="nearest")
    assert np.allclose(got, ref32, rtol=0, atol=scale * 1e-6)
    assert ref.shape == got.shape


# ------------------------------------------------------------- R5 classification
def test_u8_full_table_is_exact_entry(ora):
    """u8 volume, NT = 256, value range [0, 255]: the TF coordinate equals the
    voxel value, so a sample at a voxel centre returns that table entry."""
    v = synth.random_u8((6, 5, 4), seed=4, p_zero=0.0)
    tf = synth.tf_random_sparse(256, seed=9, p_zero=0.0)
    vol, otf = ora.OVolume(v, 0, 255), ora.OTF(tf)
    for (i, j, k) in [(0, 0, 0), (5, 4, 3), (2, 3, 1)]:
        got = ora.point_rgba(vol, otf, (i + 0.5, j + 0.5, k + 0.5))
        assert np.array_equal(got, tf[v[k, j, i]])


@pytest.mark.parametrize("nt,lo,hi", [(256, 0, 255), (1024, 0.0, 1.0), (100, -3.0, 7.5)])
def test_classify_matches_numpy_interp(ora, nt, lo, hi):
    """R5 against numpy.interp of each channel at x = clamp((v-lo)s, 0, NT-1)."""
    rng = np.random.default_rng(nt)
    tf = rng.uniform(0, 1, size=(nt, 4)).astype(np.float32)
    v = np.full((2, 2, 2), 0, dtype=np.float32)
    vol, otf = ora.OVolume(v, lo, hi), ora.OTF(tf)
    s = np.float32(nt - 1) / np.float32(np.float32(hi) - np.float32(lo))
    for val in rng.uniform(lo - 1, hi + 1, size=50).astype(np.float32):
        v[...] = val
        x = min(max(float(np.float32(val - np.float32(lo)) * s), 0.0), nt - 1.0)
        ref = [np.interp(x, np.arange(nt), tf[:, c].astype(np.float64)) for c in range(4)]
        got = ora.point_rgba(vol, otf, (1.0, 1.0, 1.0))
        assert np.allclose(got, ref, atol=2e-6)


# ------------------------------------------------------------------- R1 rays
def test_ortho_rays_parallel_and_centred(ora):
    dims = (32, 32, 32)
    cam = synth.axis_ortho_camera(dims, axis=2)
    for (x, y) in [(0, 0), (7, 3), (15, 15)]:
        o, d = ora.ray(cam, x, y, 16, 16)
        assert np.array_equal(d, np.float32([0, 0, 1]))
        # pixel centres map to the centres of a 16 x 16 raster over [0,32]^2;
        # y = 0 is the top row
        assert o[0] == np.float32(2 * x + 1) and o[1] == np.float32(32 - (2 * y + 1))


def test_perspective_field_of_view(ora):
    W, H, fov = 64, 48, 50.0
    cam = synth.orbit_camera((16, 16, 16), W, H, theta=0.7, phi=0.2, fov_deg=fov)
    w = cam.w / np.linalg.norm(cam.w)
    _, d0 = ora.ray(cam, W // 2, H // 2, W, H)
    _, d1 = ora.ray(cam, W // 2 - 1, H // 2 - 1, W, H)
    assert abs(np.linalg.norm(d0) - 1) < 1e-6
    mid = (d0 + d1) / np.linalg.norm(d0 + d1)
    assert np.dot(mid, w) > 1 - 1e-6
    _, dtop = ora.ray(cam, W // 2, 0, W, H)
    _, dbot = ora.ray(cam, W // 2, H - 1, W, H)
    ang = math.degrees(math.acos(np.clip(np.dot(dtop.astype(np.float64), dbot), -1, 1)))
    # pinhole geometry: pixel centre (x, y) lies on the image plane at
    # (tan(fov/2) * aspect * sx, tan(fov/2) * sy, 1), sx, sy in (-1, 1)
    t = math.tan(math.radians(fov / 2))
    sx = (2 * (W // 2) + 1) / W - 1
    a = np.array([t * W / H * sx, t * (1 - 1 / H), 1.0])
    b = np.array([t * W / H * sx, -t * (1 - 1 / H), 1.0])
    expect = math.degrees(math.acos(a @ b / np.linalg.norm(a) / np.linalg.norm(b)))
    assert abs(ang - expect) < 2e-4


def test_slab_against_point_stepping(ora):
    rng = np.random.default_rng(3)
    for _ in range(200):
        lo = rng.uniform(-5, 5, 3)
        hi = lo + rng.uniform(0.5, 6, 3)
        o = rng.uniform(-10, 10, 3).astype(np.float32)
        d = rng.standard_normal(3)
        d = (d / np.linalg.norm(d)).astype(np.float32)
        ta, tb = ora.slab(o, d, lo, hi, -1e30, 1e30)
        ts = np.linspace(-40, 40, 4001)
        pts = o[None, :].astype(np.float64) + ts[:, None] * d[None, :]
        inside = np.all((pts >= lo - 1e-4) & (pts <= hi + 1e-4), axis=1)
        strict = np.all((pts > lo + 1e-3) & (pts < hi - 1e-3), axis=1)
        if ta <= tb:
            assert not np.any(strict & ((ts < ta - 1e-3) | (ts > tb + 1e-3)))
            mid = 0.5 * (ta + tb)
            p = o + mid * d
            assert np.all(p >= lo - 1e-3) and np.all(p <= hi + 1e-3)
        else:
            assert not np.any(strict)
        assert inside is not None


def test_axis_parallel_slab_on_face(ora):
    """A direction component of 0 with the origin on the box face is inside."""
    ta, tb = ora.slab([8.0, 3.0, -5.0], [0.0, 0.0, 1.0], [0, 0, 0], [8, 8, 8], 0.0, 1e30)
    assert ta == 5.0 and tb == 13.0
    ta, tb = ora.slab([8.5, 3.0, -5.0], [0.0, 0.0, 1.0], [0, 0, 0], [8, 8, 8], 0.0, 1e30)
    assert not ta <= tb


# ---------------------------------------------------- S: skipping invariance
def _cases():
    yield "blobs", synth.blobs_u8((24, 20, 28), n_blobs=5, seed=11), (0, 255), synth.tf_ramp(256, 40)
    yield "sparse_u8", synth.random_u8((19, 23, 17), seed=12, p_zero=0.97), (0, 255), \
        synth.tf_random_sparse(256, seed=3, p_zero=0.7)
    rng = np.random.default_rng(13)
    f = np.where(rng.random((18, 15, 21)) < 0.9, 0.0, rng.uniform(0, 1, (18, 15, 21)))
    yield "sparse_f32", f.astype(np.float32), (0.0, 1.0), synth.tf_random_sparse(1024, seed=4, p_zero=0.8)
    yield "menger", synth.menger_u8(27), (0, 255), synth.tf_ramp(256, 100)


@pytest.mark.parametrize("case", list(_cases()), ids=lambda c: c[0])
@pytest.mark.parametrize("B", [4, 8])
@pytest.mark.parametrize("ert", [2.0, 0.9])
def test_skipping_never_changes_image(ora, case, B, ert):
    """S + R3 + R4: marching only the intervals of non-empty bricks (and of the
    k-d leaves built over them) gives the naive image bit for bit."""
    name, v, (lo, hi), tf = case
    vol, otf = ora.OVolume(v, lo, hi), ora.OTF(tf)
    grid = vol.grid(B)
    mask = ora.build_mask(vol, otf, B)
    brick_boxes = ora.brick_boxes(ora.compact(mask), grid, B, vol.dims)
    kd = ora.kd_build(mask, grid, B, vol.dims, nbins=4, halting=0)
    kd_boxes = ora.kd_leaf_boxes(kd, B, vol.dims) if len(kd) else np.zeros((0, 6), np.float32)
    rng = np.random.default_rng(B * 7 + int(ert * 10))
    cams = [synth.random_camera(vol.dims, rng) for _ in range(3)]
    # adversarial: orthographic rays exactly on brick boundary planes
    cams.append(synth.axis_ortho_camera(vol.dims, axis=2, half=(B * 1.0, B * 1.0),
                                        offset=(1.0 - vol.dims[0] / 2 % 1, 1.0 - vol.dims[1] / 2 % 1)))
    cams.append(synth.axis_ortho_camera(vol.dims, axis=0, half=(B * 1.0, B * 1.0)))
    W, H = 12, 10
    for cam in cams:
        ref, nref = ora.render_naive(vol, otf, cam, W, H, dt=0.5, ert=ert)
        for boxes in (brick_boxes, kd_boxes):
            got, n = ora.render_boxes(vol, otf, cam, W, H, boxes, dt=0.5, ert=ert)
            assert np.array_equal(bits(ref), bits(got)), name
            assert n <= nref


@pytest.mark.parametrize("axis", [0, 1, 2])
@pytest.mark.parametrize("B", [4, 8])
def test_skipping_rays_on_brick_planes(ora, axis, B):
    """Orthographic rays whose origins sit on integer lattice points, so that
    many run exactly inside brick boundary planes (zero direction components):
    the skipping render still equals the naive one bit for bit."""
    v = synth.random_u8((16, 16, 16), seed=40 + axis, p_zero=0.9)
    tf = synth.tf_random_sparse(256, seed=axis, p_zero=0.5)
    vol, otf = ora.OVolume(v, 0, 255), ora.OTF(tf)
    a1, a2 = [a for a in range(3) if a != axis]
    W, H = 16, 16
    c = np.array(vol.dims) * 0.5
    # origin[a1] = x + 1 and origin[a2] = H - y: integers 1..16
    cam = synth.axis_ortho_camera(vol.dims, axis=axis, half=(W / 2, H / 2),
                                  offset=(0.5 + W / 2 - c[a1], 0.5 + H / 2 - c[a2]))
    o, d = ora.ray(cam, 7, 8, W, H)
    assert o[a1] == 8.0 and float(o[a2]).is_integer()
    mask = ora.build_mask(vol, otf, B)
    boxes = ora.brick_boxes(ora.compact(mask), vol.grid(B), B, vol.dims)
    ref, _ = ora.render_naive(vol, otf, cam, W, H)
    got, _ = ora.render_boxes(vol, otf, cam, W, H, boxes)
    assert np.array_equal(bits(ref), bits(got))
    assert np.any(ref[..., 3] > 0)


# ------------------------------------------------------- R6 order, R7 stop
def test_two_layers_composite_front_to_back(ora):
    """Two layers along the ray: values 50 (front, z < 8) and 200 (back); the
    TF gives (c1, a1) at 50, (c2, a2) at 200 and alpha 0 in between, so the one
    sample on the interface (value 125) adds nothing.  Front-to-back
    absorption + emission (Sec. 4.1): A = 1 - (1-a1)^16 (1-a2)^15 and
    C = c1 (1 - (1-a1)^16) + (1-a1)^16 c2 (1 - (1-a2)^15); the back-to-front
    order would weight the layers the other way."""
    v = np.full((16, 4, 4), 50, dtype=np.uint8)
    v[8:] = 200
    tf = np.zeros((256, 4), dtype=np.float32)
    c1, a1 = np.float32([0.9, 0.2, 0.1]), np.float32(0.05)
    c2, a2 = np.float32([0.1, 0.3, 0.8]), np.float32(0.2)
    tf[50, :3], tf[50, 3] = c1, a1
    tf[200, :3], tf[200, 3] = c2, a2
    vol, otf = ora.OVolume(v, 0, 255), ora.OTF(tf)
    cam = synth.axis_ortho_camera(vol.dims, axis=2, half=(1.0, 1.0), eye_back=8.0)
    img, nsamp = ora.render_naive(vol, otf, cam, 2, 2, dt=0.5)
    assert nsamp == 4 * 32
    T1 = (1.0 - np.float64(a1)) ** 16
    T2 = (1.0 - np.float64(a2)) ** 15
    tol = 32 * 8 * 2.0 ** -24
    assert np.all(np.abs(img[..., 3] - (1.0 - T1 * T2)) <= tol)
    for ch in range(3):
        want = c1[ch] * (1.0 - T1) + T1 * c2[ch] * (1.0 - T2)
        assert np.all(np.abs(img[..., ch] - want) <= tol)
        back_first = c2[ch] * (1.0 - T2) + T2 * c1[ch] * (1.0 - T1)
        assert np.all(np.abs(img[..., ch] - back_first) > 100 * tol)


def test_early_termination_stops_at_the_first_sample_over_the_threshold(ora):
    """R7: alpha 0.5 per sample gives A = 1 - 2^-k exactly after k samples;
    with ert 0.9 every ray stops after its 4th sample (A = 0.9375)."""
    v = np.full((16, 4, 4), 100, dtype=np.uint8)
    tf = np.zeros((256, 4), dtype=np.float32)
    tf[:, 0], tf[:, 3] = 1.0, 0.5
    vol, otf = ora.OVolume(v, 0, 255), ora.OTF(tf)
    cam = synth.axis_ortho_camera(vol.dims, axis=2, half=(1.0, 1.0), eye_back=8.0)
    img, nsamp = ora.render_naive(vol, otf, cam, 2, 2, dt=0.5, ert=0.9)
    assert nsamp == 4 * 4
    assert np.all(img[..., 3] == np.float32(0.9375))
    assert np.all(img[..., 0] == np.float32(0.9375))
    img, nsamp = ora.render_naive(vol, otf, cam, 2, 2, dt=0.5, ert=0.9375)
    assert nsamp == 4 * 4                         # A >= ert at the 4th sample
