"""The staged march (brick slabs copied into shared memory with bulk
asynchronous copies) against the xy-quad march and the FP64 oracle.

Both marches evaluate every sample with the same arithmetic in the same order,
so their images must be equal bit for bit; against the oracle the FP32 bar of
the parity tests applies. The counting launch variant checks that every sample
read from a staged box lies inside it (else vr_sync reports VR_ERR_BOUNDS)."""
import numpy as np
import pytest

from paper_2501_01628_gb300 import synth
from gpu_helpers import compare_envelope, oracle_env

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def vr():
    import torch
    import __graft_entry__
    __graft_entry__.build()
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_2501_01628_gb300 import vr as _vr
    return _vr


def _render_both(vr, vol, part, tf, lo, hi, cams, step=0.5, ert=1.0, schedule=(), count=True):
    """Images (and executed-sample counts) of the quad march and the staged march."""
    import torch
    out = {}
    for staged in (False, True):
        ctx = vr.vr_create(0)
        v = None
        try:
            vr.vr_set_march_staging(ctx, staged)
            v = vr.vr_volume_create(ctx, vol, "f32", part)
            vr.vr_set_transfer_function(ctx, tf, lo, hi)
            vr.vr_set_render_params(ctx, step, ert)
            vr.vr_set_composite_schedule(ctx, schedule)
            vr.vr_set_count_samples(ctx, count)
            imgs, counts = [], []
            for cam in cams:
                vr.vr_set_camera(ctx, cam)
                o = torch.full((cam["height"], cam["width"], 4), float("nan"), device="cuda")
                vr.vr_render_frame(ctx, v, o)
                vr.vr_sync(ctx)  # VR_ERR_BOUNDS / VR_ERR_TIMEOUT would raise here
                if count:
                    counts.append(vr.vr_get_sample_count(ctx))
                imgs.append(o)
            out[staged] = (imgs, counts)
        finally:
            if v is not None:
                vr.vr_volume_release(v)
            vr.vr_destroy(ctx)
    return out[False], out[True]


_ORTHO = dict(ortho=1, eye=(0.5, 0.45, 1.4), dir=(0.25, -0.3, -1.0), up=(0, 1, 0), ortho_w=1.6, ortho_h=1.3,
              width=70, height=57)


@pytest.mark.parametrize("case", ["ortho_z", "ortho_oblique", "persp_kd", "eye_inside", "close_wide", "odd_step"])
def test_staged_equals_quads_and_oracle(vr, case):
    rng = np.random.default_rng(17)
    n = 48
    vol = synth.blob_volume(n, synth.draw_blobs(rng, 7))
    vol += rng.uniform(0, 0.05, vol.shape).astype(np.float32)
    tf = synth.random_tf(rng, alpha_max=0.2)
    lo, hi = synth.volume_range(vol)
    step, ert = 0.5, 0.99
    part = dict(kind="grid", grid=(2, 2, 2))
    if case == "ortho_z":
        cams = [synth.ortho_camera_z(96, 80)]
        ert = 1.0
    elif case == "ortho_oblique":
        cams = [_ORTHO]
    elif case == "persp_kd":
        part = dict(kind="kd", n_bricks=7, cut_fracs=rng.uniform(0.3, 0.7, 6))
        cams = [synth.orbit_camera(101, 67, az, elevation_deg=el) for az, el in ((20, 25), (200, -40))]
    elif case == "eye_inside":
        cams = [synth.orbit_camera(64, 48, 80.0, radius=0.3, elevation_deg=10.0)]
    elif case == "close_wide":  # wide field of view near the volume: large slab boxes
        cams = [synth.orbit_camera(90, 70, 130.0, radius=0.95, fovy_deg=120.0)]
    else:
        cams = [synth.orbit_camera(77, 61, 310.0, elevation_deg=15.0)]
        step = 0.37
    (qi, qc), (si, sc) = _render_both(vr, vol, part, tf, lo, hi, cams, step, ert)
    assert qc == sc  # the same executed samples
    boxes = vr.vr_partition_boxes((n,) * 3, part)
    for cam, a, b in zip(cams, qi, si):
        import torch
        assert torch.equal(a, b), float((a - b).abs().max())
        compare_envelope(b.cpu().numpy().astype(np.float64), oracle_env(vol, boxes, tf, lo, hi, cam, step, ert))


def test_staged_paper_workload_equals_quads(vr):
    """512^3 noise + blobs, 36 bricks, 1920x1080 orbit views, ERT 0.99, radix-k
    4x3x3: staged and quad marches give the same image and sample count."""
    import torch
    vol, tf = synth.noise_blob_scene()
    lo, hi = float(vol.min()), float(vol.max())
    cams = [synth.orbit_camera(1920, 1080, az) for az in (0.0, 135.0)]
    vol_dev = torch.from_numpy(vol).cuda()
    (qi, qc), (si, sc) = _render_both(vr, vol_dev, dict(kind="grid", grid=(4, 3, 3)), tf, lo, hi, cams, 0.5,
                                      0.99, (4, 3, 3))
    assert qc == sc
    for a, b in zip(qi, si):
        assert torch.equal(a, b), float((a - b).abs().max())
