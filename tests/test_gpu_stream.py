"""Time-step streaming through a fixed device budget: the renders of each time
step equal those of a volume created directly from that step, whether or not
the next step's upload overlaps them, and match the FP64 oracle on that step's
values (Sec. 4: time steps are loaded and later evicted)."""
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


@pytest.mark.parametrize("slots,prefetch", [(2, True), (3, True), (2, False)])
def test_streamed_steps_equal_direct_renders(vr, slots, prefetch):
    import torch
    from paper_2501_01628_gb300.streaming import TimeSeriesRenderer
    n, steps = 40, 5
    draws = synth.draw_fields(seed=41, n_fields=1)[0]
    host = [synth.field_volume_torch(draws, t, n, device="cpu").pin_memory() for t in range(steps)]
    rng = np.random.default_rng(41)
    tf = synth.random_tf(rng, alpha_max=0.15)
    part = dict(kind="kd", n_bricks=6, cut_fracs=rng.uniform(0.3, 0.7, 5))
    cams = [synth.orbit_camera(48, 40, az) for az in (0.0, 130.0, 250.0)]
    ctx = vr.vr_create(0)
    try:
        vr.vr_set_transfer_function(ctx, tf, 0.0, 1.1)
        vr.vr_set_render_params(ctx, 0.5, 1.0)
        r = TimeSeriesRenderer(ctx, host, part, slots=slots)
        got = [[torch.empty((40, 48, 4), device="cuda") for _ in cams] for _ in range(steps)]
        for t in range(steps):
            r.render_step(t, cams, got[t], prefetch=prefetch)
        torch.cuda.synchronize()
        r.close()
        for t in range(steps):
            v = vr.vr_volume_create(ctx, host[t], "f32", part)
            for c, g in zip(cams, got[t]):
                vr.vr_set_camera(ctx, c)
                ref = torch.empty_like(g)
                vr.vr_render_frame(ctx, v, ref)
                assert torch.equal(g, ref), t
            vr.vr_volume_release(v)
        vr.vr_sync(ctx)
        # against the oracle: every step at one view, and every view at the last step
        boxes = vr.vr_partition_boxes((n,) * 3, part)
        checks = [(t, 1) for t in range(steps)] + [(steps - 1, 0), (steps - 1, 2)]
        for t, c in checks:
            env = oracle_env(host[t].numpy(), boxes, tf, 0.0, 1.1, cams[c])
            compare_envelope(got[t][c].cpu().numpy().astype(np.float64), env)
    finally:
        vr.vr_destroy(ctx)
