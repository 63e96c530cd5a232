"""Helpers shared by the GPU parity tests: run the CUDA path through the C ABI
and compare with the FP64 oracle."""
import numpy as np

import oracle

# max abs error per RGBA channel against the FP64 oracle for the FP32 path
TOL = 1e-4


def gpu_render(vr, vol, part, tf, lo, hi, cam, step=0.5, ert=1.0, storage="f32", schedule=(),
               count=False, partials=False, host_out=False, packet_width=None, mode=None):
    import torch
    ctx = vr.vr_create(0)
    v = None
    try:
        v = vr.vr_volume_create(ctx, vol, storage, part)
        vr.vr_set_transfer_function(ctx, tf, lo, hi)
        vr.vr_set_camera(ctx, cam)
        vr.vr_set_render_params(ctx, step, ert)
        vr.vr_set_composite_schedule(ctx, schedule)
        vr.vr_set_count_samples(ctx, count)
        if packet_width is not None:
            vr.vr_set_packet_width(ctx, packet_width)
        if mode is not None:
            vr.vr_set_render_mode(ctx, mode)
        H, W = cam["height"], cam["width"]
        res = {}
        if partials:
            fr = vr.vr_render_partials(ctx, v)
            rects, order = vr.vr_frame_info(fr)
            res["rects"], res["order"] = rects, order
            res["partials"] = [p.cpu().numpy() for p in vr.frame_partials_torch(fr)]
            out = torch.empty((H, W, 4), dtype=torch.float32, device="cuda")
            vr.vr_composite(ctx, fr, out)
            torch.cuda.synchronize()
            vr.vr_frame_release(fr)
        elif host_out:
            out = torch.empty((H, W, 4), dtype=torch.float32).pin_memory()
            vr.vr_render_frame(ctx, v, out)
        else:
            out = torch.empty((H, W, 4), dtype=torch.float32, device="cuda")
            vr.vr_render_frame(ctx, v, out)
        vr.vr_sync(ctx)
        if count:
            res["nsamples"] = vr.vr_get_sample_count(ctx)
        res["img"] = out.cpu().numpy().astype(np.float64)
    finally:
        if v is not None:
            vr.vr_volume_release(v)
        vr.vr_destroy(ctx)
    return res


def compare_envelope(got, env, tol=TOL):
    """Unambiguous pixels within tol of the oracle; pixels whose ray carries a
    near-threshold decision (sample count or early termination) within tol of
    the range spanned by the oracle's decision alternatives."""
    amb = env["ambiguous"]
    err = np.abs(got - env["img"])
    clean = err[~amb]
    max_clean = float(clean.max()) if clean.size else 0.0
    inside = np.all((got >= env["lo"] - tol) & (got <= env["hi"] + tol), axis=-1)
    assert max_clean <= tol, "max abs err %.3g > %.1g on unambiguous pixels" % (max_clean, tol)
    assert inside.all(), "%d ambiguous pixels outside the oracle envelope" % int((~inside).sum())
    return dict(max_err=max_clean, mean_err=float(clean.mean()) if clean.size else 0.0,
                n_ambiguous=int(amb.sum()))


def oracle_env(vol, boxes, tf, lo, hi, cam, step=0.5, ert=1.0, **kw):
    return oracle.render_with_envelope(vol, boxes, tf, lo, hi, cam, step, ert, **kw)
