"""Pins of the oracle's second render workload: gradient shading (R13) and
opacity correction (R14).  The paper only mentions gradient shading (it
switches it off for its measurements, Sec. 4.1); the readings are pinned here
to facts fixed outside the oracle: float64 log2/exp2, closed forms of
constant and ramp slabs, exact gradients of linear fields, and the skipping
invariance that must survive both switches."""
import numpy as np
import pytest

from paper_1912_09596_gb300 import synth


def bits(a):
    return np.ascontiguousarray(a, dtype=np.float32).view(np.uint32)


SHADE = (0.25, 0.6, 0.3, 12)   # ka, kd, ks, shininess


# ------------------------------------------------------------ own log2 / exp2
def test_log2_own_against_float64(ora):
    """R14's log2: relative error below 1e-6 over (0, 1], exact 0 at 1 and
    exact integers at powers of two."""
    xs = np.concatenate([np.float32(2.0) ** -np.linspace(0, 24, 4001),
                         np.float32(1.0) - np.arange(1, 2000, dtype=np.float32) * np.float32(2 ** -24),
                         np.random.default_rng(1).random(3000).astype(np.float32) + np.float32(1e-6)])
    xs = np.unique(np.clip(xs.astype(np.float32), np.float32(2 ** -24), np.float32(1.0)))
    got = np.array([ora.log2_own(x) for x in xs], dtype=np.float64)
    ref = np.log2(xs.astype(np.float64))
    nz = ref != 0
    assert np.all(np.abs(got[nz] - ref[nz]) <= 1e-6 * np.abs(ref[nz]))
    assert ora.log2_own(1.0) == 0.0
    for e in range(0, 25):
        assert ora.log2_own(2.0 ** -e) == -float(e)


def test_exp2_own_against_float64(ora):
    """R14's exp2 on [-126, 0]: relative error below 1e-6, exact at integers."""
    ys = np.concatenate([-np.linspace(0, 126, 20001), -np.random.default_rng(2).random(5000) * 30])
    ys = ys.astype(np.float32)
    got = np.array([ora.exp2_own(y) for y in ys], dtype=np.float64)
    ref = np.exp2(ys.astype(np.float64))
    assert np.all(np.abs(got - ref) <= 1e-6 * ref)
    for n in range(0, 127):
        assert ora.exp2_own(-float(n)) == 2.0 ** -n
    assert ora.exp2_own(-127.5) == 0.0


# --------------------------------------------------------- opacity correction
def test_opacity_correction_special_cases(ora):
    """alpha 0 and 1 are fixed points; ratio 0 (off) and 1 leave alpha as is."""
    for a in np.float32([0.0, 1e-7, 0.01, 0.3, 0.999, 1.0]):
        assert ora.opacity_correct(a, 0.0) == a
        assert ora.opacity_correct(a, 1.0) == a
    for r in [0.1, 0.5, 2.0, 7.3, 1000.0]:
        assert ora.opacity_correct(0.0, r) == 0.0
        assert ora.opacity_correct(1.0, r) == 1.0


@pytest.mark.parametrize("r", [0.125, 0.5, 2.0, 3.7])
def test_opacity_correction_closed_form(ora, r):
    """1 - (1 - alpha)^r in float64, within 4e-7 absolute, and monotone."""
    a = np.linspace(0, 1, 1001).astype(np.float32)
    got = np.array([ora.opacity_correct(x, r) for x in a], dtype=np.float64)
    ref = 1.0 - (1.0 - a.astype(np.float64)) ** np.float64(np.float32(r))
    assert np.all(np.abs(got - ref) <= 4e-7)
    assert np.all(np.diff(got) >= 0)


@pytest.mark.parametrize("dt", [0.5, 0.25])
@pytest.mark.parametrize("a", [0.02, 0.2])
def test_corrected_slab_does_not_depend_on_the_step(ora, dt, a):
    """A constant slab 16 voxels deep with alpha a per voxel (dt_ref = 1):
    with the correction, 1 - A = (1 - a)^16 whatever the step; without it the
    slab gets more opaque as the step shrinks."""
    v = np.full((16, 6, 6), 100, dtype=np.uint8)
    tf = np.zeros((256, 4), dtype=np.float32)
    tf[:, :3] = (0.3, 0.6, 0.9)
    tf[:, 3] = a
    vol, otf = ora.OVolume(v, 0, 255), ora.OTF(tf)
    cam = synth.axis_ortho_camera(vol.dims, axis=2, half=(2.0, 2.0), eye_back=8.0)
    img, nsamp = ora.render_naive(vol, otf, cam, 4, 4, dt=dt, dt_ref=1.0)
    n = int(round(16 / dt))
    assert nsamp == 16 * n
    T = (1.0 - np.float64(np.float32(a))) ** 16
    tol = n * 8 * 2.0 ** -24 + 1e-6
    assert np.all(np.abs(img[..., 3] - (1.0 - T)) <= tol)
    plain, _ = ora.render_naive(vol, otf, cam, 4, 4, dt=dt)
    assert np.all(plain[..., 3] >= img[..., 3] - tol)
    if dt < 1.0:
        assert np.all(plain[..., 3] > img[..., 3])


# ------------------------------------------------------------------ gradient
def test_gradient_of_linear_ramp_is_exact(ora):
    """f = 2x - 3y + 5z on the voxel centres: central differences of the
    trilinear reconstruction at interior points with dyadic fractions give
    (2, -3, 5) exactly."""
    n = 12
    k, j, i = np.meshgrid(np.arange(n), np.arange(n), np.arange(n), indexing="ij")
    v = (2 * i - 3 * j + 5 * k + 100).astype(np.float32)
    vol = ora.OVolume(v, 0.0, 200.0)
    rng = np.random.default_rng(3)
    for _ in range(200):
        p = rng.integers(2, n - 3, 3) + 0.5 + rng.integers(0, 8, 3) / 8.0
        assert np.array_equal(ora.gradient(vol, p), np.float32([2.0, -3.0, 5.0]))


def test_gradient_of_constant_volume_is_zero(ora):
    v = np.full((9, 10, 11), 42, dtype=np.uint8)
    vol = ora.OVolume(v, 0, 255)
    for p in [(0.1, 0.2, 0.3), (5.5, 5.0, 4.25), (10.9, 9.9, 8.9)]:
        assert np.array_equal(ora.gradient(vol, p), np.zeros(3, np.float32))


# ------------------------------------------------------------------- shading
def test_shade_closed_forms(ora):
    """Headlight Blinn-Phong: normal along the ray gives rgb (ka + kd) + ks,
    normal across it rgb ka, a zero gradient leaves the colour, and
    |n . d| = 3/5 gives ks 0.6^s against float64."""
    ka, kd, ks, s = SHADE
    rgb = np.float32([0.2, 0.5, 0.8])
    got = ora.shade([4.0, 0, 0], [-1.0, 0, 0], ka, kd, ks, s, rgb)
    assert np.allclose(got, rgb.astype(np.float64) * (ka + kd) + ks, rtol=0, atol=2e-7)
    got = ora.shade([0, 2.5, 0], [1.0, 0, 0], ka, kd, ks, s, rgb)
    assert np.allclose(got, rgb.astype(np.float64) * ka, rtol=0, atol=1e-7)
    assert np.array_equal(ora.shade([0, 0, 0], [1.0, 0, 0], ka, kd, ks, s, rgb), rgb)
    got = ora.shade([3.0, 4.0, 0], [1.0, 0, 0], ka, kd, ks, s, rgb)
    ref = rgb.astype(np.float64) * (ka + kd * 0.6) + ks * 0.6 ** s
    assert np.allclose(got, ref, rtol=0, atol=5e-7)


@pytest.mark.parametrize("axis,c", [(0, 1.0), (1, 0.0)])
def test_shaded_ramp_slab_closed_form(ora, axis, c):
    """A volume ramping along x with a TF of constant colour and alpha a:
    every sample's normal is +-x, so rays along x see rgb (ka + kd) + ks and
    rays along y see rgb ka; C = c' (1 - (1-a)^n)."""
    ka, kd, ks, s = SHADE
    nx, ny, nz = 16, 10, 6
    k, j, i = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    v = (10 * i + 20).astype(np.uint8)
    a = 0.05
    tf = np.zeros((256, 4), dtype=np.float32)
    rgb = np.float32([0.3, 0.6, 0.9])
    tf[:, :3] = rgb
    tf[:, 3] = a
    vol, otf = ora.OVolume(v, 0, 255), ora.OTF(tf)
    cam = synth.axis_ortho_camera(vol.dims, axis=axis, half=(2.0, 2.0), eye_back=8.0)
    img, nsamp = ora.render_naive(vol, otf, cam, 4, 4, dt=0.5, shade=SHADE)
    n = 2 * vol.dims[axis]
    assert nsamp == 16 * n
    shaded = rgb.astype(np.float64) * (ka + kd * c) + ks * c ** s
    T = (1.0 - np.float64(np.float32(a))) ** n
    tol = n * 8 * 2.0 ** -24
    assert np.all(np.abs(img[..., 3] - (1.0 - T)) <= tol)
    for ch in range(3):
        assert np.all(np.abs(img[..., ch] - shaded[ch] * (1.0 - T)) <= tol)


# ------------------------------------------------------ skipping invariance
@pytest.mark.parametrize("ert", [2.0, 0.9])
def test_skipping_never_changes_shaded_image(ora, ert):
    """Shading changes colours only where alpha > 0 and the correction keeps
    alpha 0 at 0, so marching only the non-empty bricks (and k-d leaves) still
    gives the naive image bit for bit."""
    v = synth.blobs_u8((24, 20, 28), n_blobs=5, seed=11)
    tf = synth.tf_ramp(256, 40)
    vol, otf = ora.OVolume(v, 0, 255), ora.OTF(tf)
    for B in (4, 8):
        grid = vol.grid(B)
        mask = ora.build_mask(vol, otf, B)
        brick_boxes = ora.brick_boxes(ora.compact(mask), grid, B, vol.dims)
        kd = ora.kd_build(mask, grid, B, vol.dims, nbins=4, halting=1)
        kd_boxes = ora.kd_leaf_boxes(kd, B, vol.dims)
        rng = np.random.default_rng(B)
        for cam in [synth.random_camera(vol.dims, rng) for _ in range(3)]:
            for dt, dt_ref in [(0.5, 0.0), (0.5, 1.0), (0.3, 0.7)]:
                ref, nref = ora.render_naive(vol, otf, cam, 12, 10, dt=dt, ert=ert,
                                             shade=SHADE, dt_ref=dt_ref)
                plain, _ = ora.render_naive(vol, otf, cam, 12, 10, dt=dt, ert=ert)
                assert not np.array_equal(bits(ref), bits(plain))
                for boxes in (brick_boxes, kd_boxes):
                    got, n = ora.render_boxes(vol, otf, cam, 12, 10, boxes, dt=dt, ert=ert,
                                              shade=SHADE, dt_ref=dt_ref)
                    assert np.array_equal(bits(ref), bits(got))
                    assert n <= nref


def test_gradient_at_the_volume_faces_uses_clamped_neighbours(ora):
    """At the first and last voxel centres along x the outer neighbour is
    clamped to the edge voxel (R2), so the central difference of a ramp of
    slope a is a/2 there and a one voxel further in."""
    n = 10
    k, j, i = np.meshgrid(np.arange(6), np.arange(6), np.arange(n), indexing="ij")
    v = (4 * i + 20).astype(np.float32)
    vol = ora.OVolume(v, 0.0, 100.0)
    for x, want in ((0.5, 2.0), (1.5, 4.0), (n - 1.5, 4.0), (n - 0.5, 2.0)):
        assert np.array_equal(ora.gradient(vol, (x, 3.0, 3.0)), np.float32([want, 0.0, 0.0])), x
