"""GPU parity: the CUDA path (through the C ABI) against the FP64 oracle.

Bar: max abs error 1e-4 per RGBA channel on every pixel whose ray takes no
near-threshold integer decision; the rest must lie inside the oracle's
decision envelope (see oracle.render_with_envelope)."""
import numpy as np
import pytest

import oracle
from paper_2501_01628_gb300 import synth
from gpu_helpers import TOL, compare_envelope, gpu_render, oracle_env

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def vr():
    import torch
    import __graft_entry__
    __graft_entry__.build()
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_2501_01628_gb300 import vr as _vr
    return _vr


# --------------------------------------------------------------------------
# 64^3 blobs, 2x2x2 bricks, 256^2 orthographic along +z (the small workload)
# --------------------------------------------------------------------------


def test_small_workload_full_image_partials_and_counts(vr):
    vol, tf = synth.small_blob_scene()
    lo, hi = synth.volume_range(vol)
    cam = synth.ortho_camera_z(256, 256)
    part = dict(kind="grid", grid=(2, 2, 2))
    boxes = oracle.grid_partition((64,) * 3, (2, 2, 2))
    got = gpu_render(vr, vol, part, tf, lo, hi, cam, partials=True, count=True)
    ref = oracle.render(vol, boxes, tf, lo, hi, cam, 0.5, with_partials=True)
    err = np.abs(got["img"] - ref["img"])
    assert err.max() <= TOL, err.max()
    # axis-aligned rays: no ownership ties, so partials match one by one
    for b, (x0, y0, w, h) in enumerate(got["rects"]):
        np.testing.assert_allclose(got["partials"][b], ref["partials"][b][y0:y0 + h, x0:x0 + w],
                                   atol=TOL, rtol=0)
        outside = np.ones((256, 256), bool)
        outside[y0:y0 + h, x0:x0 + w] = False
        assert np.all(ref["partials"][b][outside] == 0)
    assert got["nsamples"] == ref["nsamples"] == 256 * 256 * 128
    # looking along +z: each brick of the low z half precedes the brick behind it
    pos = {int(b): i for i, b in enumerate(got["order"])}
    assert all(pos[b] < pos[b + 4] for b in range(4))


# --------------------------------------------------------------------------
# perspective views, ragged image sizes, grid / kd / box partitions
# --------------------------------------------------------------------------

CASES = [
    # n, partition, camera, step
    (24, dict(kind="grid", grid=(1, 1, 1)), synth.orbit_camera(33, 21, 10.0), 0.5),
    (40, dict(kind="grid", grid=(2, 2, 2)), synth.orbit_camera(70, 45, 45.0), 0.5),
    (37, dict(kind="grid", grid=(3, 2, 4)), synth.orbit_camera(61, 37, 123.0, elevation_deg=-30), 0.5),
    (48, dict(kind="kd", n_bricks=11, cut_fracs=[0.3, 0.62, 0.45, 0.7, 0.5, 0.33, 0.68, 0.41, 0.57, 0.36]),
     synth.orbit_camera(64, 64, 250.0, elevation_deg=60), 0.5),
    (30, dict(kind="boxes", boxes=[[0, 0, 0, 13, 30, 30], [13, 0, 0, 30, 9, 30], [13, 9, 0, 30, 30, 17],
                                   [13, 9, 17, 21, 30, 30], [21, 9, 17, 30, 30, 30]]),
     synth.orbit_camera(50, 40, 300.0), 0.5),
    (32, dict(kind="grid", grid=(2, 2, 2)), synth.orbit_camera(40, 40, 80.0, radius=0.35), 0.5),  # eye inside
    (32, dict(kind="grid", grid=(2, 1, 2)), synth.orbit_camera(45, 30, 15.0), 0.37),  # odd step
    (32, dict(kind="grid", grid=(2, 2, 2)),
     dict(ortho=1, eye=(0.5, 0.5, 1.3), dir=(0.3, -0.2, -1.0), up=(0, 1, 0), ortho_w=1.5, ortho_h=1.2,
          width=53, height=41), 0.5),
    (16, dict(kind="grid", grid=(2, 2, 2)), synth.orbit_camera(1, 1, 0.0), 0.5),  # 1x1 image
]


@pytest.mark.parametrize("case", range(len(CASES)))
def test_perspective_and_partition_variants(vr, case):
    n, part, cam, step = CASES[case]
    rng = np.random.default_rng(1000 + case)
    vol = synth.blob_volume(n, synth.draw_blobs(rng, 6))
    vol += rng.uniform(0, 0.1, vol.shape).astype(np.float32)
    tf = synth.random_tf(rng, alpha_max=0.15)
    lo, hi = synth.volume_range(vol)
    boxes = vr.vr_partition_boxes((n,) * 3, part)
    # counting launch: also checks that every executed sample's quads lie in its brick
    got = gpu_render(vr, vol, part, tf, lo, hi, cam, step=step, count=True)
    env = oracle_env(vol, boxes, tf, lo, hi, cam, step)
    compare_envelope(got["img"], env)


def test_camera_looking_away_gives_empty_image(vr):
    vol, tf = synth.small_blob_scene(n=16)
    lo, hi = synth.volume_range(vol)
    cam = dict(ortho=0, eye=(0.5, 0.5, -1.0), dir=(0, 0, -1.0), up=(0, 1, 0), fovy_deg=40.0,
               width=20, height=10)
    got = gpu_render(vr, vol, dict(kind="grid", grid=(2, 2, 2)), tf, lo, hi, cam)
    assert np.all(got["img"] == 0)


# --------------------------------------------------------------------------
# early ray termination (per brick, T <= 0.01)
# --------------------------------------------------------------------------


@pytest.mark.parametrize("grid", [(1, 1, 1), (3, 2, 2)])
def test_early_termination(vr, grid):
    n = 64
    vol, tf = synth.noise_blob_scene(n=n, seed=7)
    lo, hi = synth.volume_range(vol)
    cam = synth.orbit_camera(96, 54, 45.0)
    part = dict(kind="grid", grid=grid)
    boxes = oracle.grid_partition((n,) * 3, grid)
    got = gpu_render(vr, vol, part, tf, lo, hi, cam, ert=0.99, count=True)
    env = oracle_env(vol, boxes, tf, lo, hi, cam, 0.5, 0.99)
    stats = compare_envelope(got["img"], env)
    assert stats["n_ambiguous"] < 0.02 * 96 * 54
    full = oracle.render(vol, boxes, tf, lo, hi, cam, 0.5, 1.0)
    # one brick holds whole chords, so termination saves work; small bricks may
    # never reach T <= 0.01 locally
    if grid == (1, 1, 1):
        assert got["nsamples"] < full["nsamples"]
    assert got["nsamples"] <= full["nsamples"]
    assert abs(got["nsamples"] - env["nsamples"]) <= 4 * max(1, stats["n_ambiguous"]) + 8


# --------------------------------------------------------------------------
# compositing schedules (radix-k association trees)
# --------------------------------------------------------------------------


def test_radix_k_schedules_agree(vr):
    n = 72
    rng = np.random.default_rng(21)
    vol = synth.blob_volume(n, synth.draw_blobs(rng, 10))
    tf = synth.random_tf(rng, alpha_max=0.1)
    lo, hi = synth.volume_range(vol)
    cam = synth.orbit_camera(160, 90, 45.0)
    part = dict(kind="grid", grid=(4, 3, 3))
    direct = gpu_render(vr, vol, part, tf, lo, hi, cam)["img"]
    boxes = oracle.grid_partition((n,) * 3, (4, 3, 3))
    compare_envelope(direct, oracle_env(vol, boxes, tf, lo, hi, cam))
    for sched in ([36], [4, 9], [4, 3, 3], [2, 2, 3, 3], [6, 6], [3, 3, 2, 2], [36, 1]):
        got = gpu_render(vr, vol, part, tf, lo, hi, cam, schedule=sched)["img"]
        np.testing.assert_allclose(got, direct, atol=1e-6, rtol=0, err_msg=str(sched))
    with pytest.raises(vr.VrError):
        gpu_render(vr, vol, part, tf, lo, hi, cam, schedule=[5, 7])


def test_maximum_bricks_and_deepest_radix_tree(vr):
    """VR_MAX_BRICKS = 128 bricks (8x4x4 grid of a 64^3 volume): four 32-brick
    chunks in the composite's tile compaction, a radix-k tree of seven factors
    (the deepest association the composite supports), and the ray-state cycling
    form over all 128 bricks; one brick more is refused."""
    n = 64
    rng = np.random.default_rng(23)
    vol = synth.blob_volume(n, synth.draw_blobs(rng, 10))
    tf = synth.random_tf(rng, alpha_max=0.1)
    lo, hi = synth.volume_range(vol)
    cam = synth.orbit_camera(96, 80, 33.0, elevation_deg=25.0)
    part = dict(kind="grid", grid=(8, 4, 4))
    boxes = oracle.grid_partition((n,) * 3, (8, 4, 4))
    env = oracle_env(vol, boxes, tf, lo, hi, cam)
    direct = gpu_render(vr, vol, part, tf, lo, hi, cam, count=True)["img"]
    compare_envelope(direct, env)
    for sched in ([2] * 7, [8, 16], [4, 4, 8]):
        got = gpu_render(vr, vol, part, tf, lo, hi, cam, schedule=sched)["img"]
        np.testing.assert_allclose(got, direct, atol=1e-6, rtol=0, err_msg=str(sched))
    cyc = gpu_render(vr, vol, part, tf, lo, hi, cam, mode=1)["img"]
    compare_envelope(cyc, env)
    with pytest.raises(vr.VrError) as e:
        gpu_render(vr, synth.blob_volume(n, synth.draw_blobs(rng, 2)), dict(kind="grid", grid=(43, 1, 3)),
                   tf, lo, hi, cam)
    assert e.value.status == vr.VR_ERR_ARG


# --------------------------------------------------------------------------
# brick packing, host output, errors
# --------------------------------------------------------------------------



@pytest.mark.parametrize("mode", [0, 1])
def test_packet_widths_give_identical_images(vr, mode):
    """The ray packet (4x8, 8x4 or 16x2 pixels per warp) only changes which
    thread marches which pixel: the images are bit-identical, for both frame
    algorithms, on ragged image sizes, kd bricks and with early termination."""
    for case in (2, 3):
        n, part, cam, step = CASES[case]
        rng = np.random.default_rng(2000 + case)
        vol = synth.blob_volume(n, synth.draw_blobs(rng, 6))
        tf = synth.random_tf(rng, alpha_max=0.2)
        lo, hi = synth.volume_range(vol)
        imgs = [gpu_render(vr, vol, part, tf, lo, hi, cam, step=step, ert=0.9, schedule=(),
                           packet_width=pw, mode=mode, count=True)["img"] for pw in (4, 8, 16)]
        assert np.array_equal(imgs[0], imgs[1]) and np.array_equal(imgs[0], imgs[2]), case


def test_paper_workload_sampled(vr):
    """The benchmark's configuration at full size: 512^3 value noise + blobs
    (seed 1), 36 grid bricks, 1920x1080 perspective orbit views, step 0.5 voxel,
    per-brick early termination at alpha 0.99, radix-k composite 4x3x3, 4x8-pixel
    ray packets. 2048 random pixels of two views against the FP64 oracle."""
    import torch
    vol, tf = synth.noise_blob_scene()
    lo, hi = synth.volume_range(vol)
    part = dict(kind="grid", grid=(4, 3, 3))
    boxes = oracle.grid_partition((512,) * 3, (4, 3, 3))
    vol_dev = torch.from_numpy(vol).cuda()
    for k, az in enumerate((synth.ORBIT_AZIMUTHS[0], synth.ORBIT_AZIMUTHS[3])):
        cam = synth.orbit_camera(1920, 1080, az)
        got = gpu_render(vr, vol_dev, part, tf, lo, hi, cam, 0.5, 0.99, schedule=(4, 3, 3), count=True)["img"]
        prng = np.random.default_rng(30 + k)
        pix = np.stack([prng.integers(0, 1920, 2048), prng.integers(0, 1080, 2048)], axis=1)
        env = oracle_env(vol, boxes, tf, lo, hi, cam, 0.5, 0.99, pixels=pix)
        compare_envelope(got[pix[:, 1], pix[:, 0]], env)

@pytest.mark.parametrize("storage", ["f32", "bf16", "f16"])
def test_pack_halo_exact(vr, storage):
    import torch
    n = 20
    rng = np.random.default_rng(5)
    vol = rng.standard_normal((n, n + 3, n - 2)).astype(np.float32)
    part = dict(kind="kd", n_bricks=5, cut_fracs=[0.4, 0.6, 0.35, 0.65])
    ctx = vr.vr_create(0)
    try:
        v = vr.vr_volume_create(ctx, vol, storage, part)
        boxes, nbytes = vr.vr_volume_info(v)
        assert nbytes > 0
        if storage == "f32":
            q = vol
        else:
            t = torch.from_numpy(vol).to(torch.bfloat16 if storage == "bf16" else torch.float16)
            q = t.view(torch.int16).numpy().view(np.uint16)
        for b, (x0, y0, z0, x1, y1, z1) in enumerate(boxes):
            zi = np.clip(np.arange(z0 - 1, z1 + 1), 0, vol.shape[0] - 1)
            yi = np.clip(np.arange(y0 - 1, y1 + 1), 0, vol.shape[1] - 1)
            xi = np.clip(np.arange(x0 - 1, x1 + 1), 0, vol.shape[2] - 1)
            want = q[np.ix_(zi, yi, xi)]
            got = vr.vr_volume_read_brick(v, b, storage)
            np.testing.assert_array_equal(got, want)
        vr.vr_volume_release(v)
    finally:
        vr.vr_destroy(ctx)


def test_host_output_equals_device_output(vr):
    vol, tf = synth.small_blob_scene(n=32)
    lo, hi = synth.volume_range(vol)
    cam = synth.orbit_camera(64, 48, 20.0)
    part = dict(kind="grid", grid=(2, 2, 2))
    a = gpu_render(vr, vol, part, tf, lo, hi, cam)["img"]
    b = gpu_render(vr, vol, part, tf, lo, hi, cam, host_out=True)["img"]
    np.testing.assert_array_equal(a, b)


def test_error_paths(vr):
    import torch
    vol, tf = synth.small_blob_scene(n=16)
    ctx = vr.vr_create(0)
    try:
        v = vr.vr_volume_create(ctx, vol, "f32", dict(kind="grid", grid=(2, 2, 2)))
        out = torch.empty((8, 8, 4), device="cuda")
        with pytest.raises(vr.VrError) as e:
            vr.vr_render_frame(ctx, v, out)
        assert e.value.status == vr.VR_ERR_STATE
        with pytest.raises(vr.VrError) as e:
            vr.vr_set_transfer_function(ctx, tf, 1.0, 1.0)
        assert e.value.status == vr.VR_ERR_ARG
        with pytest.raises(vr.VrError):
            vr.vr_set_camera(ctx, dict(ortho=0, eye=(0, 0, 0), dir=(0, 1, 0), up=(0, 1, 0),
                                       fovy_deg=60, width=8, height=8))
        with pytest.raises(vr.VrError):
            vr.vr_volume_create(ctx, vol, "f32", dict(kind="grid", grid=(17, 1, 1)))
        with pytest.raises(vr.VrError) as e:
            vr.vr_destroy(ctx)  # a volume is still alive
        assert e.value.status == vr.VR_ERR_STATE
        vr.vr_volume_release(v)
    finally:
        vr.vr_destroy(ctx)


@pytest.mark.parametrize("mode", [0, 1])
def test_async_host_output_equals_device_output(vr, mode):
    import torch
    vol, tf = synth.small_blob_scene(n=32)
    lo, hi = synth.volume_range(vol)
    cams = [synth.orbit_camera(64, 48, az) for az in (20.0, 140.0, 260.0, 300.0)]
    ctx = vr.vr_create(0)
    v = vr.vr_volume_create(ctx, vol, "f32", dict(kind="grid", grid=(2, 2, 2)))
    try:
        vr.vr_set_transfer_function(ctx, tf, lo, hi)
        vr.vr_set_render_mode(ctx, mode)
        refs = []
        for c in cams:
            vr.vr_set_camera(ctx, c)
            o = torch.empty((48, 64, 4), device="cuda")
            vr.vr_render_frame(ctx, v, o)
            refs.append(o.cpu())
        vr.vr_set_host_output_async(ctx, True)
        hosts = [torch.full((48, 64, 4), float("nan")).pin_memory() for _ in cams]
        for c, h in zip(cams, hosts):
            vr.vr_set_camera(ctx, c)
            vr.vr_render_frame(ctx, v, h)
        vr.vr_sync(ctx)
        for h, r in zip(hosts, refs):
            assert torch.equal(h, r)
    finally:
        vr.vr_volume_release(v)
        vr.vr_destroy(ctx)
