"""Ray-state cycling on the GPU (vr_set_render_mode(ctx, 1)): each ray carries
one (C, T) through the bricks in visibility order, with global early
termination. Checked against the oracle's cycling mode and, with termination
off, against the sort-last frame."""
import numpy as np
import pytest

import oracle
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


def _render(vr, vol, part, tf, lo, hi, cam, mode, ert=1.0, count=False):
    import torch
    ctx = vr.vr_create(0)
    v = None
    try:
        v = vr.vr_volume_create(ctx, vol, "f32", part)
        vr.vr_set_transfer_function(ctx, tf, lo, hi)
        vr.vr_set_camera(ctx, cam)
        vr.vr_set_render_params(ctx, 0.5, ert)
        vr.vr_set_render_mode(ctx, mode)
        vr.vr_set_count_samples(ctx, count)
        out = torch.empty((cam["height"], cam["width"], 4), device="cuda")
        vr.vr_render_frame(ctx, v, out)
        vr.vr_sync(ctx)
        n = vr.vr_get_sample_count(ctx) if count else None
        return out.cpu().numpy().astype(np.float64), n
    finally:
        if v is not None:
            vr.vr_volume_release(v)
        vr.vr_destroy(ctx)


CASES = [
    (40, dict(kind="grid", grid=(2, 2, 2)), synth.orbit_camera(70, 45, 45.0)),
    (48, dict(kind="kd", n_bricks=11, cut_fracs=[0.3, 0.62, 0.45, 0.7, 0.5, 0.33, 0.68, 0.41, 0.57, 0.36]),
     synth.orbit_camera(64, 64, 250.0, elevation_deg=60)),
    (32, dict(kind="grid", grid=(2, 2, 2)), synth.orbit_camera(40, 40, 80.0, radius=0.35)),  # eye inside
    (64, dict(kind="grid", grid=(1, 1, 4)), synth.ortho_camera_z(32, 32)),
]


@pytest.mark.parametrize("case", range(len(CASES)))
def test_cycling_equals_sort_last_without_termination(vr, case):
    n, part, cam = CASES[case]
    rng = np.random.default_rng(700 + case)
    vol = synth.blob_volume(n, synth.draw_blobs(rng, 6))
    vol += rng.uniform(0, 0.1, vol.shape).astype(np.float32)
    tf = synth.random_tf(rng, alpha_max=0.15)
    lo, hi = synth.volume_range(vol)
    a, na = _render(vr, vol, part, tf, lo, hi, cam, 0, count=True)
    b, nb = _render(vr, vol, part, tf, lo, hi, cam, 1, count=True)
    np.testing.assert_allclose(b, a, atol=2e-6, rtol=0)
    assert na == nb
    boxes = vr.vr_partition_boxes((n,) * 3, part)
    compare_envelope(b, oracle_env(vol, boxes, tf, lo, hi, cam, ert_global=True))


@pytest.mark.parametrize("grid", [(1, 1, 1), (3, 2, 2)])
def test_cycling_global_termination(vr, grid):
    n = 64
    vol, tf = synth.noise_blob_scene(n=n, seed=7)
    lo, hi = synth.volume_range(vol)
    cam = synth.orbit_camera(96, 54, 45.0)
    part = dict(kind="grid", grid=grid)
    boxes = oracle.grid_partition((n,) * 3, grid)
    got, ncyc = _render(vr, vol, part, tf, lo, hi, cam, 1, ert=0.99, count=True)
    env = oracle_env(vol, boxes, tf, lo, hi, cam, 0.5, 0.99, ert_global=True)
    stats = compare_envelope(got, env)
    assert stats["n_ambiguous"] < 0.02 * 96 * 54
    _, nloc = _render(vr, vol, part, tf, lo, hi, cam, 0, ert=0.99, count=True)
    assert ncyc <= nloc  # global termination never does more work than per-brick termination
    assert abs(ncyc - env["nsamples"]) <= 4 * max(1, stats["n_ambiguous"]) + 8


def test_cycling_paper_workload_sampled(vr):
    """512^3 noise + blobs, 36 bricks, 1920x1080, ERT 0.99: 2048 random pixels
    against the oracle's cycling mode."""
    import torch
    vol, tf = synth.noise_blob_scene()
    lo, hi = synth.volume_range(vol)
    part = dict(kind="grid", grid=(4, 3, 3))
    boxes = oracle.grid_partition((512,) * 3, (4, 3, 3))
    cam = synth.orbit_camera(1920, 1080, 45.0)
    got, _ = _render(vr, torch.from_numpy(vol).cuda(), part, tf, lo, hi, cam, 1, ert=0.99)
    prng = np.random.default_rng(12)
    pix = np.stack([prng.integers(0, 1920, 2048), prng.integers(0, 1080, 2048)], axis=1)
    env = oracle_env(vol, boxes, tf, lo, hi, cam, 0.5, 0.99, ert_global=True, pixels=pix)
    compare_envelope(got[pix[:, 1], pix[:, 0]], env)


@pytest.mark.parametrize("mode", [0, 1])
@pytest.mark.parametrize("step", [0.25, 0.8])
def test_opacity_correction(vr, mode, step):
    import torch
    n = 40
    rng = np.random.default_rng(900)
    vol = synth.blob_volume(n, synth.draw_blobs(rng, 6))
    tf = synth.random_tf(rng, alpha_max=0.2)
    lo, hi = synth.volume_range(vol)
    part = dict(kind="kd", n_bricks=5, cut_fracs=[0.4, 0.6, 0.45, 0.55])
    cam = synth.orbit_camera(56, 48, 120.0)
    ctx = vr.vr_create(0)
    v = vr.vr_volume_create(ctx, vol, "f32", part)
    try:
        vr.vr_set_transfer_function(ctx, tf, lo, hi)
        vr.vr_set_camera(ctx, cam)
        vr.vr_set_render_params(ctx, step, 1.0)
        vr.vr_set_opacity_correction(ctx, 0.5)
        vr.vr_set_render_mode(ctx, mode)
        out = torch.empty((48, 56, 4), device="cuda")
        vr.vr_render_frame(ctx, v, out)
        vr.vr_sync(ctx)
        got = out.cpu().numpy().astype(np.float64)
    finally:
        vr.vr_volume_release(v)
        vr.vr_destroy(ctx)
    boxes = vr.vr_partition_boxes((n,) * 3, part)
    compare_envelope(got, oracle_env(vol, boxes, tf, lo, hi, cam, step, opacity_ref_step=0.5,
                                     ert_global=(mode == 1)))
