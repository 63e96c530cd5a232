"""Batched form: every (volume, view) render and its compositing in one
persistent, CUDA-graph-captured launch. Each render must equal the plain
vr_render_frame of the same volume and view, and match the FP64 oracle."""
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


def _plain(vr, ctx, vol, cam, lo, hi, tf):
    import torch
    vr.vr_set_transfer_function(ctx, tf, lo, hi)
    vr.vr_set_camera(ctx, cam)
    out = torch.empty((cam["height"], cam["width"], 4), device="cuda")
    vr.vr_render_frame(ctx, vol, out)
    return out


@pytest.mark.parametrize("storage", ["f32", "f16"])
def test_small_batch_equals_plain_renders(vr, storage):
    import torch
    n, steps, nfields = 40, 2, 2
    draws = synth.draw_fields(seed=31, n_fields=nfields)
    rng = np.random.default_rng(31)
    tf = synth.random_tf(rng, alpha_max=0.12)
    part = dict(kind="kd", n_bricks=7, cut_fracs=rng.uniform(0.3, 0.7, 6))
    cams = [synth.orbit_camera(72, 56, az, elevation_deg=el) for az, el in
            ((10, 20), (100, -30), (190, 45), (280, 0), (333, 15))]
    ctx = vr.vr_create(0)
    vols, srcs, ranges = [], [], []
    try:
        for s in range(steps):
            for f in range(nfields):
                src = synth.field_volume_torch(draws[f], s, n)
                srcs.append(src)
                ranges.append((float(src.min()), float(src.max())))
                vols.append(vr.vr_volume_create(ctx, src, storage, part))
        vr.vr_set_transfer_function(ctx, tf, 0.0, 1.0)
        vr.vr_set_render_params(ctx, 0.5, 1.0)
        nr = len(vols) * len(cams)
        out = torch.full((nr, 56, 72, 4), float("nan"), device="cuda")
        b = vr.vr_batch_create(ctx, vols, cams, out, vmins=[r[0] for r in ranges], vmaxs=[r[1] for r in ranges])
        vr.vr_batch_launch(b)
        vr.vr_sync(ctx)
        first = out.clone()
        # neither the work order nor the packet shape changes any pixel
        for pw, bps, order in ((4, 0, 1), (16, 6, 0), (8, 0, 1)):
            vr.vr_batch_configure(b, pw, bps, order)
            out.fill_(float("nan"))
            vr.vr_batch_launch(b)
            vr.vr_sync(ctx)
            assert torch.equal(out, first), (pw, bps, order)
        chosen = vr.vr_batch_autotune(b)
        assert chosen[0] in (4, 8, 16) and chosen[1] >= 1 and chosen[3] in (0, 1)
        out.fill_(float("nan"))
        vr.vr_batch_launch(b)
        vr.vr_sync(ctx)
        assert torch.equal(out, first)
        for v, (vol, (lo, hi)) in enumerate(zip(vols, ranges)):
            for w, cam in enumerate(cams):
                ref = _plain(vr, ctx, vol, cam, lo, hi, tf)
                got = out[v * len(cams) + w]
                assert torch.equal(got, ref), (v, w, float((got - ref).abs().max()))
        vr.vr_sync(ctx)
        # one render against the oracle (same quantised values for f16)
        src = srcs[3].cpu().numpy()
        q = src if storage == "f32" else synth.quantize(src, "f16")
        boxes = vr.vr_partition_boxes((n,) * 3, part)
        env = oracle_env(q, boxes, tf, ranges[3][0], ranges[3][1], cams[2],
                         dtype=None if storage == "f32" else oracle.F16)
        compare_envelope(out[3 * len(cams) + 2].cpu().numpy().astype(np.float64), env)
        vr.vr_batch_release(b)
    finally:
        for v in vols:
            vr.vr_volume_release(v)
        vr.vr_destroy(ctx)


def test_batching_workload_sampled(vr):
    """6 time steps x 3 fields of 768^3 f16 (seed 3), 48 kd bricks, 32 views at
    1024^2: 576 renders in one launch; 4 renders checked on 256 pixels each
    against the oracle on the same f16 values."""
    import torch
    n, steps, nfields, nviews = 768, 6, 3, 32
    draws = synth.draw_fields(seed=3, n_fields=nfields)
    rng = np.random.default_rng(3)
    tf = synth.random_tf(rng)
    cuts = synth.kd_cut_fractions(rng, 48)
    part = dict(kind="kd", n_bricks=48, cut_fracs=cuts)
    cams = [synth.orbit_camera(1024, 1024, 360.0 * w / nviews, elevation_deg=20.0 * np.cos(w))
            for w in range(nviews)]
    ctx = vr.vr_create(0)
    vols, ranges = [], []
    try:
        for s in range(steps):
            for f in range(nfields):
                src = synth.field_volume_torch(draws[f], s, n)
                ranges.append((float(src.min()), float(src.max())))
                vols.append(vr.vr_volume_create(ctx, src, "f16", part))
                del src
        vr.vr_set_transfer_function(ctx, tf, 0.0, 1.0)
        vr.vr_set_render_params(ctx, 0.5, 1.0)
        out = torch.empty((len(vols) * nviews, 1024, 1024, 4), device="cuda")
        b = vr.vr_batch_create(ctx, vols, cams, out, vmins=[r[0] for r in ranges], vmaxs=[r[1] for r in ranges])
        vr.vr_batch_launch(b)
        vr.vr_sync(ctx)
        boxes = vr.vr_partition_boxes((n,) * 3, part)
        prng = np.random.default_rng(8)
        for r in (0, 77, 301, 575):
            v, w = divmod(r, nviews)
            s, f = divmod(v, nfields)
            q = synth.quantize(synth.field_volume_torch(draws[f], s, n).cpu().numpy(), "f16")
            pix = np.stack([prng.integers(0, 1024, 256), prng.integers(0, 1024, 256)], axis=1)
            env = oracle_env(q, boxes, tf, ranges[v][0], ranges[v][1], cams[w], dtype=oracle.F16, pixels=pix)
            got = out[r].cpu().numpy().astype(np.float64)[pix[:, 1], pix[:, 0]]
            compare_envelope(got, env)
        vr.vr_batch_release(b)
    finally:
        for v in vols:
            vr.vr_volume_release(v)
        vr.vr_destroy(ctx)


def test_bounded_wait_gives_up_and_reports_timeout(vr):
    """The batched kernel's waits are bounded. A test hook raises unit 0's
    composite target past its march item count, so those waits can never
    succeed, and shortens every wait to 64 sleeps: the launch must end within
    milliseconds, vr_sync must return VR_ERR_TIMEOUT, and the next launch with
    the hook cleared must be bit-identical to plain renders. Nothing faults:
    the wait gives up, sets the error word, and every other claim stops."""
    import time
    import torch
    n = 32
    draws = synth.draw_fields(seed=41, n_fields=1)
    rng = np.random.default_rng(41)
    tf = synth.random_tf(rng, alpha_max=0.12)
    part = dict(kind="grid", grid=(2, 2, 1))
    cams = [synth.orbit_camera(48, 40, az) for az in (20.0, 150.0, 260.0)]
    ctx = vr.vr_create(0)
    vols, ranges = [], []
    try:
        for s in range(2):
            src = synth.field_volume_torch(draws[0], s, n)
            ranges.append((float(src.min()), float(src.max())))
            vols.append(vr.vr_volume_create(ctx, src, "f32", part))
        vr.vr_set_transfer_function(ctx, tf, 0.0, 1.0)
        vr.vr_set_render_params(ctx, 0.5, 1.0)
        nr = len(vols) * len(cams)
        out = torch.full((nr, 40, 48, 4), float("nan"), device="cuda")
        b = vr.vr_batch_create(ctx, vols, cams, out, vmins=[r[0] for r in ranges],
                               vmaxs=[r[1] for r in ranges])
        refs = [_plain(vr, ctx, vol, cam, lo, hi, tf).clone()
                for vol, (lo, hi) in zip(vols, ranges) for cam in cams]
        vr.vr_sync(ctx)
        for order in (0, 1):  # render-major and brick-major units
            vr.vr_batch_configure(b, 8, 0, order)
            vr.vr_batch_debug_wait(b, 64, 1)
            out.fill_(float("nan"))
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            vr.vr_batch_launch(b)
            with pytest.raises(vr.VrError) as e:
                vr.vr_sync(ctx)
            elapsed = time.perf_counter() - t0
            assert e.value.status == vr.VR_ERR_TIMEOUT
            assert elapsed < 0.5, elapsed  # the 2^25-sleep default would take seconds
            vr.vr_sync(ctx)  # the error word was cleared by the report
            vr.vr_batch_debug_wait(b, 0, 0)
            out.fill_(float("nan"))
            vr.vr_batch_launch(b)
            vr.vr_sync(ctx)
            for r, ref in enumerate(refs):
                assert torch.equal(out[r], ref), (order, r)
        with pytest.raises(vr.VrError):
            vr.vr_batch_debug_wait(b, -1, 0)
        vr.vr_batch_release(b)
    finally:
        for v in vols:
            vr.vr_volume_release(v)
        vr.vr_destroy(ctx)
