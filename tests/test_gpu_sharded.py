"""The brick-sharded path on one GPU: every rank of the exchange emulated in
this process, each with its share volume (vr_volume_create_share) and its
image from vr_render_frame, the radix-k rounds combined by vr_composite_images.
The frame must match vr_render_frame of the whole volume (up to the rounding of
the association) and the FP64 oracle."""
import numpy as np
import pytest

from paper_2501_01628_gb300 import sharded, synth
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


def test_composite_images_against_numpy(vr):
    import torch
    rng = np.random.default_rng(3)
    ctx = vr.vr_create(0)
    try:
        for n in (1, 3, 7):
            a = rng.uniform(0, 1, (n, 37, 29, 1))
            rgb = rng.uniform(0, 1, (n, 37, 29, 3)) * a  # premultiplied
            ims = np.concatenate([rgb, a], axis=-1).astype(np.float32)
            dev = [torch.from_numpy(im).cuda() for im in ims]
            out = torch.empty_like(dev[0])
            vr.vr_composite_images(ctx, dev, out)
            want = np.zeros(ims[0].shape)
            for im in ims.astype(np.float64):
                want = want + (1 - want[..., 3:4]) * im
            np.testing.assert_allclose(out.cpu().numpy(), want, atol=1e-6, rtol=0)
            vr.vr_composite_images(ctx, dev, dev[0])  # in place over the first input
            np.testing.assert_array_equal(dev[0].cpu().numpy(), out.cpu().numpy())
        with pytest.raises(ValueError):
            vr.vr_composite_images(ctx, [torch.zeros((4, 4, 4), device="cuda")], torch.zeros((4, 5, 4), device="cuda"))
    finally:
        vr.vr_destroy(ctx)


@pytest.mark.parametrize("world,factors", [(2, (2,)), (4, (2, 2)), (4, (4,)), (8, (2, 2, 2))])
def test_emulated_ranks_equal_whole_volume_and_oracle(vr, world, factors):
    import torch
    rng = np.random.default_rng(29)
    n = 48
    vol = synth.blob_volume(n, synth.draw_blobs(rng, 7))
    vol += rng.uniform(0, 0.05, vol.shape).astype(np.float32)
    tf = synth.random_tf(rng, alpha_max=0.2)
    lo, hi = synth.volume_range(vol)
    part = dict(kind="kd", n_bricks=12, cut_fracs=rng.uniform(0.3, 0.7, 11))
    cams = [synth.orbit_camera(83, 61, az, elevation_deg=el) for az, el in ((35, 20), (220, -30))]
    dims = (n, n, n)
    boxes = vr.vr_partition_boxes(dims, part)
    shares, tree = sharded.brick_shares(boxes, world)
    ctx = vr.vr_create(0)
    vols = []
    try:
        full = vr.vr_volume_create(ctx, vol, "f32", part)
        vols.append(full)
        share_vols = [vr.vr_volume_create_share(ctx, vol, s, "f32", part) for s in shares]
        vols += share_vols
        vr.vr_set_transfer_function(ctx, tf, lo, hi)
        vr.vr_set_render_params(ctx, 0.5, 1.0)
        for cam in cams:
            vr.vr_set_camera(ctx, cam)
            shape = (cam["height"], cam["width"], 4)
            imgs = []
            for v in share_vols:
                im = torch.empty(shape, device="cuda")
                vr.vr_render_frame(ctx, v, im)
                imgs.append(im)
            order = sharded.share_order(tree, cam, dims)
            got = sharded.composite_bands(imgs, order, factors,
                                          lambda pieces, out: vr.vr_composite_images(ctx, pieces, out),
                                          lambda s: torch.empty(s, device="cuda"))
            ref = torch.empty(shape, device="cuda")
            vr.vr_render_frame(ctx, full, ref)
            vr.vr_sync(ctx)
            np.testing.assert_allclose(got.cpu().numpy(), ref.cpu().numpy(), atol=2e-6, rtol=0)
            compare_envelope(got.cpu().numpy().astype(np.float64), oracle_env(vol, boxes, tf, lo, hi, cam))
        # shares hold only their bricks: no batching, no read-back of others
        with pytest.raises(vr.VrError):
            vr.vr_batch_create(ctx, [share_vols[0]], cams[:1], torch.empty((1,) + shape, device="cuda"))
        missing = next(b for b in range(len(boxes)) if b not in shares[0])
        with pytest.raises(vr.VrError):
            vr.vr_volume_read_brick(share_vols[0], missing)
    finally:
        for v in vols:
            vr.vr_volume_release(v)
        vr.vr_destroy(ctx)


def test_sharded_renderer_single_rank(vr):
    """ShardedRenderer through a one-rank gloo group: the frame is the rank's
    whole-volume render."""
    import os
    import socket
    import torch
    import torch.distributed as dist
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        port = s.getsockname()[1]
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=0, world_size=1)
    ctx = vr.vr_create(0)
    r = None
    try:
        vol, tf = synth.small_blob_scene(n=32)
        lo, hi = synth.volume_range(vol)
        vr.vr_set_transfer_function(ctx, tf, lo, hi)
        part = dict(kind="grid", grid=(2, 2, 2))
        r = sharded.ShardedRenderer(ctx, vol, part)
        cam = synth.orbit_camera(40, 30, 60.0)
        got = r.render(cam)
        full = vr.vr_volume_create(ctx, vol, "f32", part)
        ref = torch.empty_like(got)
        vr.vr_render_frame(ctx, full, ref)
        vr.vr_sync(ctx)
        vr.vr_volume_release(full)
        assert torch.equal(got, ref)
    finally:
        if r is not None:
            r.close()
        vr.vr_destroy(ctx)
        dist.destroy_process_group()
