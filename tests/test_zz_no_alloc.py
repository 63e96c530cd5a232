"""vr_render_frame_noalloc: the frame entry point for callers that cannot
allocate device memory (an in-situ renderer inside a simulation whose pool
allocator owns all device memory, or a latency-critical caller that must not
call cudaMalloc/cudaFree). Its partial images live in the library's static
device scratch array; the caller passes its own volume and output buffer.

Checked against vr_render_frame on the same inputs, on two calls in a row
(the scratch keeps the previous call's contents), within the FP32 parity
tolerance. This file sorts last so that a run stopping at the first failure
has run every other test first."""
import numpy as np
import pytest

from paper_2501_01628_gb300 import synth

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


def _reference_frames(vr, vol, part, tf, lo, hi, cams):
    """Frames of the existing entry point (library-owned packed bricks)."""
    import torch
    ctx = vr.vr_create(torch.cuda.current_device())
    v = None
    outs = []
    try:
        v = vr.vr_volume_create(ctx, vol, "f32", part)
        vr.vr_set_transfer_function(ctx, tf, lo, hi)
        vr.vr_set_render_params(ctx, 0.5, 1.0)
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
