"""Pins of the FP64 oracle against what the mathematics fixes (CPU only).

The paper prints no worked example, so every pin is a closed form, an
invariant, a special case that reduces to a library routine, or brute force on
tiny inputs. Each is chosen so that a plausible mistake in the oracle (a
dropped term, a wrong sign or index, transposed axes, a wrong composite order,
double-counted or dropped samples at brick faces) fails at least one of them.
"""
import math

import numpy as np
import pytest
import scipy.ndimage

import oracle
from paper_2501_01628_gb300 import synth

pytestmark = pytest.mark.usefixtures("oracle_lib")


def _ramp_tf(n=257):
    # entries i/(n-1) with n-1 = 256 are exact in float32, so rgba(u) = u exactly
    t = (np.arange(n, dtype=np.float64) / (n - 1)).astype(np.float32)
    return np.stack([t, t, t, t], axis=1)


# --------------------------------------------------------------------------
# P1 constant slab: closed forms of the discrete EA sum
# --------------------------------------------------------------------------


@pytest.mark.parametrize("alpha", [0.0, 0.013, 0.05, 0.5, 1.0])
@pytest.mark.parametrize("grid", [(1, 1, 1), (2, 2, 2), (1, 1, 4)])
def test_p1_constant_slab(alpha, grid):
    n = 16
    vol = np.full((n, n, n), 0.25, np.float32)
    tf = synth.constant_tf([0.9, 0.4, 0.1, alpha])
    rgb = tf[0, :3].astype(np.float64)  # the table is float32: use its exact values
    alpha = float(tf[0, 3])
    cam = synth.ortho_camera_z(8, 8)
    boxes = oracle.grid_partition((n, n, n), grid)
    out = oracle.render(vol, boxes, tf, 0.0, 1.0, cam, 0.5, with_partials=True)
    nsamp = 2 * n  # chord 1, dt = 0.5/n
    A = 1.0 - (1.0 - alpha) ** nsamp
    img = out["img"]
    np.testing.assert_allclose(img[..., 3], A, rtol=0, atol=1e-13)
    for c in range(3):
        np.testing.assert_allclose(img[..., c], rgb[c] * A, rtol=0, atol=1e-13)
    assert out["nsamples"] == 64 * nsamp
    # per-brick partials: bricks stacked along z each hold 2n/gz samples
    if grid[0] == grid[1] == 1:
        per = nsamp // grid[2]
        for b in range(grid[2]):
            np.testing.assert_allclose(out["partials"][b][..., 3], 1 - (1 - alpha) ** per,
                                       atol=1e-13)


@pytest.mark.parametrize("alpha", [0.02, 0.05, 0.2])
@pytest.mark.parametrize("gz", [1, 2, 4])
def test_p1_slab_with_early_termination(alpha, gz):
    """ERT at 0.99 stops each brick after the first sample with T <= 0.01; with
    bricks stacked along z each brick restarts from T = 1 (local test)."""
    n = 64
    vol = np.full((n, n, n), 0.5, np.float32)
    tf = synth.constant_tf([1.0, 0.5, 0.25, alpha])
    alpha = float(tf[0, 3])
    cam = synth.ortho_camera_z(4, 4)
    boxes = oracle.grid_partition((n, n, n), (1, 1, gz))
    out = oracle.render(vol, boxes, tf, 0.0, 1.0, cam, 0.5, ert_alpha=0.99)
    per = 2 * n // gz
    kstop = math.ceil(math.log(0.01) / math.log(1 - alpha))
    taken = min(per, kstop)
    A_b = 1 - (1 - alpha) ** taken
    A = 1 - (1 - A_b) ** gz
    np.testing.assert_allclose(out["img"][..., 3], A, atol=1e-12)
    np.testing.assert_allclose(out["img"][..., 0], A, atol=1e-12)
    assert out["nsamples"] == 16 * gz * taken


# --------------------------------------------------------------------------
# P5 exact trilinear and classification
# --------------------------------------------------------------------------


def test_p5_trilinear_reproduces_linear_and_multilinear_functions():
    rng = np.random.default_rng(7)
    nz, ny, nx = 9, 7, 11
    k, j, i = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    a, b, c, e = 0.3, -1.7, 2.1, 0.4
    lin = (a * i + b * j + c * k + e).astype(np.float64)
    prod = (i * j * k).astype(np.float64)
    nm = max(nx, ny, nz)
    # interior points (all 8 neighbours in range): v in [0, N-1] per axis
    v = np.stack([rng.uniform(0, nx - 1, 200), rng.uniform(0, ny - 1, 200),
                  rng.uniform(0, nz - 1, 200)], axis=1)
    p = (v + 0.5) / nm
    np.testing.assert_allclose(oracle.sample(lin, p), a * v[:, 0] + b * v[:, 1] + c * v[:, 2] + e,
                               atol=1e-12)
    np.testing.assert_allclose(oracle.sample(prod, p), v[:, 0] * v[:, 1] * v[:, 2], atol=1e-10)
    # clamp-to-edge outside the centre lattice: value held at the end voxel
    edge = np.array([[0.1 / nm, 0.5 / nm, 0.5 / nm], [(nx - 0.1) / nm, 0.5 / nm, 0.5 / nm]])
    np.testing.assert_allclose(oracle.sample(lin, edge), [a * 0 + e, a * (nx - 1) + e], atol=1e-12)


def test_p5_trilinear_matches_library_interpolation():
    rng = np.random.default_rng(3)
    vol = rng.uniform(size=(6, 5, 8))
    p = rng.uniform(-0.05, 1.05, size=(300, 3)) * np.array([8, 5, 6]) / 8
    coords = (p[:, ::-1] * 8 - 0.5).T
    ref = scipy.ndimage.map_coordinates(vol, coords, order=1, mode="nearest")
    np.testing.assert_allclose(oracle.sample(vol, p), ref, atol=1e-12)


def test_p5_classification_ramp_and_clamp():
    tf = _ramp_tf()
    vals = np.array([-1.0, 0.0, 0.1234, 0.5, 0.987654321, 1.0, 3.0])
    out = oracle.classify(tf, 0.0, 1.0, vals)
    np.testing.assert_allclose(out, np.clip(vals, 0, 1)[:, None] * np.ones(4), atol=1e-12)
    # affine range: u = (s - vmin)/(vmax - vmin)
    out = oracle.classify(tf, -2.0, 6.0, [2.0])
    np.testing.assert_allclose(out[0], 0.5, atol=1e-12)
    # random table: equals np.interp on the entry positions
    rng = np.random.default_rng(1)
    t = synth.random_tf(rng)
    s = rng.uniform(-0.2, 1.2, 100)
    ref = np.stack([np.interp(np.clip(s, 0, 1) * 255, np.arange(256), t[:, c].astype(np.float64))
                    for c in range(4)], axis=1)
    np.testing.assert_allclose(oracle.classify(t, 0.0, 1.0, s), ref, atol=1e-12)


def test_p5_small_config_lattice_exact_weights():
    """64^3, 256x256 ortho along +z, step 0.5: x-ramp volume; each ray sees a
    constant value whose trilinear weights are in {1/8, 3/8, 5/8, 7/8}."""
    n = 64
    k, j, i = np.meshgrid(np.arange(n), np.arange(n), np.arange(n), indexing="ij")
    vol = i.astype(np.float32)
    tf = _ramp_tf()
    tf[:, 3] = 0.01
    a32 = float(tf[0, 3])
    cam = synth.ortho_camera_z(256, 256)
    out = oracle.render(vol, oracle.grid_partition((n,) * 3, (2, 2, 2)), tf, 0.0, 63.0, cam,
                        0.5, crop=(0, 100, 256, 2))
    px = np.arange(256)
    s = np.clip((px + 0.5) / 4 - 0.5, 0, 63)
    frac = ((px + 0.5) / 4 - 0.5) % 1
    assert set(np.round(frac, 6)) == {0.125, 0.375, 0.625, 0.875}
    A = 1 - (1 - a32) ** 128
    np.testing.assert_allclose(out["img"][0, :, 0], s / 63 * A, atol=1e-12)
    np.testing.assert_allclose(out["img"][1, :, 3], A, atol=1e-12)


def test_rays_orthographic_and_perspective_geometry():
    cam = synth.ortho_camera_z(256, 128)
    o, d = oracle.primary_ray(cam, 3, 5)
    np.testing.assert_allclose(o, [3.5 / 256, 5.5 / 128, 0.0], atol=1e-15)
    np.testing.assert_allclose(d, [0, 0, 1], atol=1e-15)
    # odd image: the centre pixel looks exactly along the view direction, and
    # edge-pixel rays make the angle fixed by the field of view
    cam = synth.orbit_camera(9, 9, 30.0, fovy_deg=60.0)
    o, d = oracle.primary_ray(cam, 4, 4)
    f = np.asarray(cam["dir"]) / np.linalg.norm(cam["dir"])
    np.testing.assert_allclose(d, f, atol=1e-14)
    np.testing.assert_allclose(o, cam["eye"], atol=1e-15)
    o, d = oracle.primary_ray(cam, 4, 8)
    ang = math.degrees(math.acos(np.clip(np.dot(d, f), -1, 1)))
    np.testing.assert_allclose(math.tan(math.radians(ang)), 8 / 9 * math.tan(math.radians(30)),
                               rtol=1e-12)
    assert np.dot(d, [0, 1, 0]) > np.dot(f, [0, 1, 0])  # row index grows upwards


# --------------------------------------------------------------------------
# P3 brute force: explicit O(n^2) products, no bricks, bisection for the chord
# --------------------------------------------------------------------------


def _chord_by_bisection(o, d, E):
    inside = lambda t: np.all((o + t * d >= 0) & (o + t * d <= E))
    ts = np.linspace(0, 6, 60001)
    ins = [t for t in ts[::10] if inside(t)]
    if not ins:
        ins = [t for t in ts if inside(t)]
        if not ins:
            return None
    tm = ins[0]
    if inside(0.0):
        t0 = 0.0
    else:
        lo, hi = 0.0, tm
        for _ in range(200):
            mid = 0.5 * (lo + hi)
            lo, hi = (lo, mid) if inside(mid) else (mid, hi)
        t0 = hi
    lo, hi = tm, 10.0
    for _ in range(200):
        mid = 0.5 * (lo + hi)
        lo, hi = (mid, hi) if inside(mid) else (lo, mid)
    return t0, lo


def _brute_force_pixel(vol, tf, vmin, vmax, o, d, step):
    nz, ny, nx = vol.shape
    nm = max(nx, ny, nz)
    E = np.array([nx, ny, nz]) / nm
    ch = _chord_by_bisection(o, d, E)
    if ch is None:
        return np.zeros(4)
    t0, t1 = ch
    dt = step / nm
    k = np.arange(int((t1 - t0) / dt) + 2)
    t = t0 + (k + 0.5) * dt
    t = t[t < t1]
    p = o[None, :] + t[:, None] * d[None, :]
    s = scipy.ndimage.map_coordinates(vol.astype(np.float64), (p[:, ::-1] * nm - 0.5).T,
                                      order=1, mode="nearest")
    x = np.clip((s - vmin) / (vmax - vmin), 0, 1) * (tf.shape[0] - 1)
    rgba = np.stack([np.interp(x, np.arange(tf.shape[0]), tf[:, c].astype(np.float64))
                     for c in range(4)], axis=1)
    a = rgba[:, 3]
    out = np.zeros(4)
    for kk in range(a.size):
        trans = np.prod(1.0 - a[:kk])  # explicit product, no recurrence
        out[:3] += a[kk] * rgba[kk, :3] * trans
    out[3] = 1.0 - np.prod(1.0 - a)
    return out


@pytest.mark.parametrize("camkind", ["ortho", "persp0", "persp1"])
def test_p3_brute_force_8x8(camkind):
    rng = np.random.default_rng(11)
    n = 12
    vol = synth.blob_volume(n, synth.draw_blobs(rng, 5))
    vol = vol + rng.uniform(0, 0.05, vol.shape).astype(np.float32)
    tf = synth.random_tf(rng, alpha_max=0.3)
    vmin, vmax = float(vol.min()), float(vol.max())
    if camkind == "ortho":
        cam = synth.ortho_camera_z(8, 8)
    elif camkind == "persp0":
        cam = synth.orbit_camera(8, 8, 30.0, radius=1.6, fovy_deg=50.0)
    else:
        cam = synth.orbit_camera(8, 8, 200.0, radius=1.5, elevation_deg=-35, fovy_deg=40.0)
    boxes = oracle.kd_partition((n,) * 3, 5, rng.uniform(0.3, 0.7, 4))
    got = oracle.render(vol, boxes, tf, vmin, vmax, cam, 0.5)["img"]
    for py in range(8):
        for px in range(8):
            o, d = oracle.primary_ray(cam, px, py)
            ref = _brute_force_pixel(vol, tf, vmin, vmax, o, d, 0.5)
            np.testing.assert_allclose(got[py, px], ref, atol=1e-11, err_msg=str((px, py)))


# --------------------------------------------------------------------------
# P2 / P4 single brick and associativity of "over" across splits
# --------------------------------------------------------------------------


def _scene(n=24, seed=5):
    rng = np.random.default_rng(seed)
    vol = synth.blob_volume(n, synth.draw_blobs(rng, 6))
    tf = synth.random_tf(rng, alpha_max=0.2)
    return vol, tf, float(vol.min()), float(vol.max())


def test_p2_single_brick_equals_unsplit_bitwise():
    vol, tf, lo, hi = _scene()
    cam = synth.orbit_camera(24, 16, 75.0)
    whole = [[0, 0, 0, 24, 24, 24]]
    a = oracle.render(vol, whole, tf, lo, hi, cam, 0.5, with_partials=True)
    # the single partial is the image itself
    np.testing.assert_array_equal(a["partials"][0], a["img"])


@pytest.mark.parametrize("split", ["grid222", "grid413", "kd7", "kd16", "boxes"])
@pytest.mark.parametrize("az", [0.0, 135.0, 290.0])
def test_p4_associativity_of_splits(split, az):
    vol, tf, lo, hi = _scene()
    n = 24
    cam = synth.orbit_camera(20, 14, az, elevation_deg=25.0 if az != 135 else -40.0)
    whole = oracle.render(vol, [[0, 0, 0, n, n, n]], tf, lo, hi, cam, 0.5)
    rng = np.random.default_rng(hash(split) % 1000)
    if split == "grid222":
        boxes = oracle.grid_partition((n,) * 3, (2, 2, 2))
    elif split == "grid413":
        boxes = oracle.grid_partition((n,) * 3, (4, 1, 3))
    elif split.startswith("kd"):
        k = int(split[2:])
        boxes = oracle.kd_partition((n,) * 3, k, rng.uniform(0.3, 0.7, k - 1))
    else:
        # an uneven hand-made tiling (not a grid)
        boxes = [[0, 0, 0, 10, 24, 24], [10, 0, 0, 24, 7, 24], [10, 7, 0, 24, 24, 13],
                 [10, 7, 13, 17, 24, 24], [17, 7, 13, 24, 24, 24]]
    split_img = oracle.render(vol, boxes, tf, lo, hi, cam, 0.5)
    np.testing.assert_allclose(split_img["img"], whole["img"], atol=1e-12)
    assert split_img["nsamples"] == whole["nsamples"]


def test_p4_wrong_order_would_be_detected():
    """Control: compositing the same partials back to front differs from the
    unsplit image (so P4 has power against an order mistake)."""
    vol, tf, lo, hi = _scene()
    n = 24
    cam = synth.ortho_camera_z(12, 12)
    boxes = oracle.grid_partition((n,) * 3, (1, 1, 2))
    out = oracle.render(vol, boxes, tf, lo, hi, cam, 0.5, with_partials=True)
    front, back = out["partials"][0], out["partials"][1]
    wrong = back + (1 - back[..., 3:4]) * front
    right = front + (1 - front[..., 3:4]) * back
    np.testing.assert_allclose(right, out["img"], atol=1e-14)
    assert np.max(np.abs(wrong - out["img"])) > 1e-3


# --------------------------------------------------------------------------
# P6 invariants
# --------------------------------------------------------------------------


def test_p6_invariants():
    vol, tf, lo, hi = _scene()
    n = 24
    cam = synth.orbit_camera(16, 16, 60.0)
    boxes = oracle.grid_partition((n,) * 3, (2, 2, 2))
    img = oracle.render(vol, boxes, tf, lo, hi, cam, 0.5)["img"]
    assert img[..., 3].min() >= 0 and img[..., 3].max() <= 1
    maxrgb = tf[:, :3].max()
    assert np.all(img[..., :3] <= img[..., 3:4] * maxrgb + 1e-12)
    # alpha == 0 everywhere: empty image
    tf0 = tf.copy()
    tf0[:, 3] = 0
    assert np.all(oracle.render(vol, boxes, tf0, lo, hi, cam, 0.5)["img"] == 0)
    # alpha == 1 everywhere: the colour of the first sample on the ray
    tf1 = tf.copy()
    tf1[:, 3] = 1
    got = oracle.render(vol, boxes, tf1, lo, hi, cam, 0.5)["img"]
    whole = oracle.render(vol, [[0, 0, 0, n, n, n]], tf1, lo, hi, cam, 0.5)["img"]
    np.testing.assert_array_equal(got, whole)
    hit = got[..., 3] == 1
    assert hit.any()
    for py, px in zip(*np.nonzero(hit)):
        o, d = oracle.primary_ray(cam, px, py)
        # first sample colour via the point probes
        ch = _chord_by_bisection(o, d, np.ones(3))
        p = o + (ch[0] + 0.25 / n) * d
        rgba = oracle.classify(tf1, lo, hi, oracle.sample(vol, p[None]))[0]
        np.testing.assert_allclose(got[py, px, :3], rgba[:3], atol=1e-9)


# --------------------------------------------------------------------------
# Partitions
# --------------------------------------------------------------------------


def _check_tiling(boxes, dims):
    boxes = np.asarray(boxes)
    vol = np.zeros(dims[::-1], np.int32)
    for b in boxes:
        assert np.all(b[:3] < b[3:])
        vol[b[2]:b[5], b[1]:b[4], b[0]:b[3]] += 1
    assert np.all(vol == 1)


def test_grid_partition_boundaries():
    b = oracle.grid_partition((512, 512, 512), (4, 3, 3))
    _check_tiling(b, (512, 512, 512))
    assert sorted(set(b[:, 1])) == [0, 170, 341]
    assert sorted(set(b[:, 0])) == [0, 128, 256, 384]
    assert list(b[1]) == [128, 0, 0, 256, 170, 170]  # x fastest brick ids


def test_kd_partition_rules():
    dims = (64, 64, 64)
    b = oracle.kd_partition(dims, 8, [0.5] * 7)
    _check_tiling(b, dims)
    g = oracle.grid_partition(dims, (2, 2, 2))
    assert sorted(map(tuple, b)) == sorted(map(tuple, g))
    # first cut on x (longest-axis tie -> x) at round(u*N)
    b = oracle.kd_partition(dims, 2, [0.3])
    assert list(b[0]) == [0, 0, 0, 19, 64, 64] and list(b[1]) == [19, 0, 0, 64, 64, 64]
    # second cut splits the larger (high) leaf along its longest axis (y/z tie -> y)
    b = oracle.kd_partition(dims, 3, [0.3, 0.7])
    assert list(b[2]) == [19, 45, 0, 64, 64, 64]
    rng = np.random.default_rng(2)
    for n in (5, 36, 64):
        dd = (96, 80, 72)
        _check_tiling(oracle.kd_partition(dd, n, rng.uniform(0.3, 0.7, n - 1)), dd)


# --------------------------------------------------------------------------
# Ray-state cycling (one (C, T) carried through the bricks, global termination)
# --------------------------------------------------------------------------


@pytest.mark.parametrize("split", ["grid", "kd"])
def test_cycling_without_termination_equals_sort_last(split):
    vol, tf, lo, hi = _scene()
    n = 24
    cam = synth.orbit_camera(18, 13, 250.0, elevation_deg=-15.0)
    rng = np.random.default_rng(4)
    boxes = (oracle.grid_partition((n,) * 3, (3, 2, 2)) if split == "grid"
             else oracle.kd_partition((n,) * 3, 9, rng.uniform(0.3, 0.7, 8)))
    a = oracle.render(vol, boxes, tf, lo, hi, cam, 0.5)
    b = oracle.render(vol, boxes, tf, lo, hi, cam, 0.5, ert_global=True)
    np.testing.assert_allclose(b["img"], a["img"], atol=1e-12)
    assert a["nsamples"] == b["nsamples"]


@pytest.mark.parametrize("alpha", [0.02, 0.05, 0.2])
def test_cycling_global_termination_closed_form(alpha):
    """Bricks stacked along z: the ray stops after the first sample anywhere
    with T <= 0.01, k* = ceil(log 0.01 / log(1-alpha)) samples in all."""
    n, gz = 64, 4
    vol = np.full((n, n, n), 0.5, np.float32)
    tf = synth.constant_tf([1.0, 0.5, 0.25, alpha])
    alpha = float(tf[0, 3])
    cam = synth.ortho_camera_z(4, 4)
    boxes = oracle.grid_partition((n, n, n), (1, 1, gz))
    out = oracle.render(vol, boxes, tf, 0.0, 1.0, cam, 0.5, ert_alpha=0.99, ert_global=True)
    taken = min(2 * n, math.ceil(math.log(0.01) / math.log(1 - alpha)))
    np.testing.assert_allclose(out["img"][..., 3], 1 - (1 - alpha) ** taken, atol=1e-12)
    assert out["nsamples"] == 16 * taken
    local = oracle.render(vol, boxes, tf, 0.0, 1.0, cam, 0.5, ert_alpha=0.99)
    assert local["nsamples"] >= out["nsamples"]


# --------------------------------------------------------------------------
# Opacity correction: alpha' = 1 - (1 - alpha)^(step / reference step)
# --------------------------------------------------------------------------


@pytest.mark.parametrize("alpha", [0.01, 0.05, 0.3])
@pytest.mark.parametrize("step", [0.25, 0.5, 1.0])
def test_opacity_correction_makes_the_slab_step_invariant(alpha, step):
    n = 32
    vol = np.full((n, n, n), 0.5, np.float32)
    tf = synth.constant_tf([0.8, 0.6, 0.4, alpha])
    alpha = float(tf[0, 3])
    cam = synth.ortho_camera_z(4, 4)
    boxes = oracle.grid_partition((n, n, n), (1, 1, 2))
    out = oracle.render(vol, boxes, tf, 0.0, 1.0, cam, step, opacity_ref_step=0.5)
    # the chord is n voxels; the reference step 0.5 gives 2n samples of alpha
    np.testing.assert_allclose(out["img"][..., 3], 1 - (1 - alpha) ** (2 * n), atol=1e-12)
    np.testing.assert_allclose(out["img"][..., 0], 0.8 * (1 - (1 - alpha) ** (2 * n)), atol=1e-12)


def test_opacity_correction_at_the_reference_step_is_the_identity():
    vol, tf, lo, hi = _scene()
    cam = synth.orbit_camera(10, 9, 30.0)
    boxes = oracle.grid_partition((24,) * 3, (2, 2, 2))
    a = oracle.render(vol, boxes, tf, lo, hi, cam, 0.5)
    b = oracle.render(vol, boxes, tf, lo, hi, cam, 0.5, opacity_ref_step=0.5)
    np.testing.assert_array_equal(a["img"], b["img"])


# --------------------------------------------------------------------------
# 16-bit storage decoders: every code against its IEEE-754 definition
# --------------------------------------------------------------------------


def _decode_all_codes(codes, dtype):
    """Oracle value of each 16-bit code: the codes form a 256 x 256 x 1 volume
    and each is sampled at its own voxel centre, where the trilinear weights
    are exactly (1, 0, ..., 0) (every neighbour must then be finite)."""
    vol = np.ascontiguousarray(codes.reshape(1, 256, 256))
    j, i = np.divmod(np.arange(codes.size), 256)
    pts = np.stack([(i + 0.5) / 256, (j + 0.5) / 256, np.full(i.size, 0.5 / 256)], axis=1)
    return oracle.sample(vol, pts, dtype=dtype)


def _uniform_code_value(code, dtype):
    """Oracle value inside a 2x2x2 volume whose voxels all hold one code,
    sampled at the volume centre (all eight weights 1/8)."""
    vol = np.full((2, 2, 2), code, dtype=np.uint16)
    return oracle.sample(vol, [[0.5, 0.5, 0.5]], dtype=dtype)[0]


def test_f16_decoder_every_code():
    # IEEE binary16: numpy's float16 is the independent definition; this covers
    # the subnormals (exponent field 0: m * 2^-24), the normals, and +-0
    codes = np.arange(65536, dtype=np.uint32).astype(np.uint16)
    want = codes.view(np.float16).astype(np.float64)
    finite = np.isfinite(want)
    got = _decode_all_codes(np.where(finite, codes, 0).astype(np.uint16), oracle.F16)
    np.testing.assert_array_equal(got[finite], want[finite])
    # a few values written out by hand from the format's definition
    assert got[0x0001] == 2.0 ** -24 and got[0x03FF] == 1023 * 2.0 ** -24
    assert got[0x0400] == 2.0 ** -14 and got[0x3C00] == 1.0 and got[0x7BFF] == 65504.0
    assert got[0xC000] == -2.0 and got[0x8001] == -(2.0 ** -24)
    # exponent field 31: infinities and NaNs
    assert _uniform_code_value(0x7C00, oracle.F16) == math.inf
    assert _uniform_code_value(0xFC00, oracle.F16) == -math.inf
    for c in (0x7C01, 0x7E00, 0xFFFF):
        assert math.isnan(_uniform_code_value(c, oracle.F16))


def test_bf16_decoder_every_code():
    # bfloat16 is the top half of an IEEE binary32: the value of code c is the
    # float32 whose bit pattern is c << 16
    codes = np.arange(65536, dtype=np.uint32)
    with np.errstate(invalid="ignore"):
        want = (codes << 16).view(np.float32).astype(np.float64)
    finite = np.isfinite(want)
    got = _decode_all_codes(np.where(finite, codes, 0).astype(np.uint16), oracle.BF16)
    np.testing.assert_array_equal(got[finite], want[finite])
    assert got[0x3F80] == 1.0 and got[0xC000] == -2.0 and got[0x0001] == 2.0 ** -133
    assert got[0x0080] == 2.0 ** -126 and got[0x7F7F] == (2 - 2.0 ** -7) * 2.0 ** 127
    assert _uniform_code_value(0x7F80, oracle.BF16) == math.inf
    assert _uniform_code_value(0xFF80, oracle.BF16) == -math.inf
    for c in (0x7F81, 0x7FC0, 0xFFFF):
        assert math.isnan(_uniform_code_value(c, oracle.BF16))


# --------------------------------------------------------------------------
# Perspective geometry on non-square images: square pixels on the image plane
# --------------------------------------------------------------------------


@pytest.mark.parametrize("W,H", [(16, 9), (9, 16), (37, 5)])
def test_perspective_pixels_are_square_on_non_square_images(W, H):
    """A pinhole camera with vertical field of view fovy puts pixel centres on
    a regular grid of SQUARE cells on the image plane at unit distance: the
    rows span 2 tan(fovy/2) in H steps, and the columns use the same spacing,
    so the horizontal extent is the aspect ratio W/H times the vertical one.
    Checked on the rays' intersections with that plane, in the camera basis
    built here from the camera's definition (f = dir, r = up x f, u = f x r)."""
    fovy = 50.0
    cam = synth.orbit_camera(W, H, 115.0, radius=1.7, elevation_deg=15.0, fovy_deg=fovy)
    f = np.asarray(cam["dir"], float)
    f /= np.linalg.norm(f)
    r = np.cross(np.asarray(cam["up"], float), f)
    r /= np.linalg.norm(r)
    u = np.cross(f, r)
    x = np.zeros((H, W))
    y = np.zeros((H, W))
    for py in range(H):
        for px in range(W):
            o, d = oracle.primary_ray(cam, px, py)
            np.testing.assert_allclose(o, cam["eye"], atol=1e-15)
            hit = d / np.dot(d, f)  # intersection with the plane at unit distance
            x[py, px], y[py, px] = np.dot(hit, r), np.dot(hit, u)
    step = 2 * math.tan(math.radians(fovy / 2)) / H
    np.testing.assert_allclose(np.diff(y, axis=0), step, rtol=1e-12)  # rows: fovy over H
    np.testing.assert_allclose(np.diff(x, axis=1), step, rtol=1e-12)  # columns: same pitch
    np.testing.assert_allclose(np.diff(y, axis=1), 0, atol=1e-13)
    np.testing.assert_allclose(np.diff(x, axis=0), 0, atol=1e-13)
    # centred on the view direction; half-pixel inset at the edges
    np.testing.assert_allclose(x[:, 0] + x[:, -1], 0, atol=1e-13)
    np.testing.assert_allclose(y[0] + y[-1], 0, atol=1e-13)
    np.testing.assert_allclose(x[0, -1], (W / 2 - 0.5) * step, rtol=1e-12)
    np.testing.assert_allclose(y[-1, 0], (H / 2 - 0.5) * step, rtol=1e-12)
