"""vr_render_frame_noalloc: the frame entry point for callers that cannot
allocate device memory (an in-situ renderer inside a simulation whose pool
allocator owns all device memory, or a latency-critical caller that must not
call cudaMalloc/cudaFree). Its partial images live in the library's static
device scratch array; the caller passes its own volume and output buffer.

Checked against vr_render_frame on the same inputs, on two calls in a row
(the scratch keeps the previous call's contents), within the FP32 parity
tolerance, and against the FP64 oracle directly: with early ray termination,
an orthographic camera, and the eye inside the volume. This file sorts last so
that a run stopping at the first failure has run every other test first."""
import numpy as np
import pytest

from paper_2501_01628_gb300 import synth
from gpu_helpers import compare_envelope, oracle_env

pytestmark = pytest.mark.gpu

TOL = 1e-4  # same FP32 bar as the parity tests


@pytest.fixture(scope="module")
def vr():
    import torch
    import __graft_entry__
    __graft_entry__.build()
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_2501_01628_gb300 import vr as _vr
    return _vr


def _reference_frames(vr, vol, part, tf, lo, hi, cams, step=0.5, ert=1.0):
    """Frames of the existing entry point (library-owned packed bricks)."""
    import torch
    ctx = vr.vr_create(torch.cuda.current_device())
    v = None
    outs = []
    try:
        v = vr.vr_volume_create(ctx, vol, "f32", part)
        vr.vr_set_transfer_function(ctx, tf, lo, hi)
        vr.vr_set_render_params(ctx, step, ert)
        for cam in cams:
            vr.vr_set_camera(ctx, cam)
            out = torch.empty((cam["height"], cam["width"], 4), dtype=torch.float32, device="cuda")
            vr.vr_render_frame(ctx, v, out)
            outs.append(out)
        torch.cuda.synchronize()
    finally:
        if v is not None:
            vr.vr_volume_release(v)
        vr.vr_destroy(ctx)
    return [o.cpu().numpy() for o in outs]


def test_noalloc_matches_render_frame_twice(vr):
    import torch
    rng = np.random.default_rng(77)
    n = 48
    vol = synth.blob_volume(n, synth.draw_blobs(rng, 7))
    vol += rng.uniform(0, 0.05, vol.shape).astype(np.float32)
    tf = synth.random_tf(rng, alpha_max=0.12)
    lo, hi = synth.volume_range(vol)
    part = dict(kind="kd", n_bricks=6, cut_fracs=rng.uniform(0.3, 0.7, 5))
    cams = [synth.orbit_camera(96, 64, 30.0), synth.orbit_camera(80, 72, 210.0, elevation_deg=-25)]
    want = _reference_frames(vr, vol, part, tf, lo, hi, cams)

    vol_dev = torch.from_numpy(vol).cuda()  # caller-owned input
    outs = [torch.full((c["height"], c["width"], 4), float("nan"), device="cuda") for c in cams]
    vr.vr_render_frame_noalloc(vol_dev, part, tf, lo, hi, cams[0], outs[0])
    torch.cuda.synchronize()
    free_before, _ = torch.cuda.mem_get_info()
    vr.vr_render_frame_noalloc(vol_dev, part, tf, lo, hi, cams[1], outs[1])
    torch.cuda.synchronize()
    free_after, _ = torch.cuda.mem_get_info()
    assert free_after == free_before  # the second call allocated no device memory
    for got, ref in zip(outs, want):
        got = got.cpu().numpy()
        assert np.isfinite(got).all()
        np.testing.assert_allclose(got, ref, atol=TOL, rtol=0)
    # the same camera again after a different frame: the scratch's leftovers do not leak in
    again = torch.empty_like(outs[0])
    vr.vr_render_frame_noalloc(vol_dev, part, tf, lo, hi, cams[0], again)
    torch.cuda.synchronize()
    np.testing.assert_allclose(again.cpu().numpy(), want[0], atol=TOL, rtol=0)
    # and against the FP64 oracle itself
    boxes = vr.vr_partition_boxes((n,) * 3, part)
    for cam, got in zip(cams, outs):
        compare_envelope(got.cpu().numpy().astype(np.float64), oracle_env(vol, boxes, tf, lo, hi, cam))


_ORTHO = dict(ortho=1, eye=(0.5, 0.45, 1.4), dir=(0.25, -0.3, -1.0), up=(0, 1, 0), ortho_w=1.6,
              ortho_h=1.3, width=70, height=57)


@pytest.mark.parametrize("case", ["ortho_ert", "eye_inside_ert", "persp_ert_odd_step"])
def test_noalloc_against_oracle_with_early_termination(vr, case):
    """ERT 0.99 / 0.95 (the call's per-brick termination test), an orthographic
    camera (its own ray set-up) and the eye inside the volume (rays starting
    inside a brick), each compared with the oracle and with vr_render_frame."""
    import torch
    rng = np.random.default_rng(5)
    n = 40
    vol = synth.blob_volume(n, synth.draw_blobs(rng, 6))
    vol += rng.uniform(0, 0.05, vol.shape).astype(np.float32)
    tf = synth.random_tf(rng, alpha_max=0.25)
    lo, hi = synth.volume_range(vol)
    if case == "ortho_ert":
        cam, part, step, ert = _ORTHO, dict(kind="grid", grid=(2, 2, 2)), 0.5, 0.99
    elif case == "eye_inside_ert":
        cam = synth.orbit_camera(64, 48, 80.0, radius=0.3, elevation_deg=10.0)
        part, step, ert = dict(kind="kd", n_bricks=5, cut_fracs=rng.uniform(0.3, 0.7, 4)), 0.5, 0.95
    else:
        cam = synth.orbit_camera(61, 53, 200.0, elevation_deg=-30.0)
        part, step, ert = dict(kind="grid", grid=(3, 1, 2)), 0.37, 0.99
    vol_dev = torch.from_numpy(vol).cuda()
    out = torch.full((cam["height"], cam["width"], 4), float("nan"), device="cuda")
    for _ in range(2):  # two calls in a row through the shared scratch
        out.fill_(float("nan"))
        vr.vr_render_frame_noalloc(vol_dev, part, tf, lo, hi, cam, out, step_voxels=step, ert_alpha=ert)
        torch.cuda.synchronize()
        got = out.cpu().numpy().astype(np.float64)
        boxes = vr.vr_partition_boxes((n,) * 3, part)
        compare_envelope(got, oracle_env(vol, boxes, tf, lo, hi, cam, step, ert))
        ref = _reference_frames(vr, vol, part, tf, lo, hi, [cam], step, ert)[0]
        # a near-threshold termination may fall differently in the two kernels:
        # compare where the oracle's decision is unambiguous
        amb = oracle_env(vol, boxes, tf, lo, hi, cam, step, ert)["ambiguous"]
        np.testing.assert_allclose(got[~amb], ref[~amb], atol=TOL, rtol=0)


def test_noalloc_rejects_frames_beyond_scratch(vr):
    import torch
    n = 64
    vol = torch.zeros((n, n, n), device="cuda")
    tf = synth.constant_tf([1, 1, 1, 0.01])
    cam = synth.orbit_camera(1920, 1080, 45.0)  # 36 footprints of ~80 MB of partials
    out = torch.empty((1080, 1920, 4), device="cuda")
    with pytest.raises(vr.VrError) as e:
        vr.vr_render_frame_noalloc(vol, dict(kind="grid", grid=(4, 3, 3)), tf, 0.0, 1.0, cam, out)
    assert e.value.status == vr.VR_ERR_ARG
