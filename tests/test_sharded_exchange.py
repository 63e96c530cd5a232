"""Brick-sharded compositing across ranks, on CPU: shares of the bricks
separated by axis-aligned planes, and the radix-k exchange of the ranks'
images, run in one process and as world-size 2 and 4 gloo process groups.

The ranks' images are built from the FP64 oracle's per-brick partials (each
share composited front to back in the library's visibility order); the
exchanged and gathered frame must equal the oracle's unsplit render up to the
rounding of the association ("over" is associative, Sec. 3 composites the
ranks' images into one framebuffer)."""
import os
import socket

import numpy as np
import pytest
import torch.multiprocessing as mp

import oracle
from paper_2501_01628_gb300 import sharded, synth

pytestmark = pytest.mark.usefixtures("oracle_lib")


@pytest.fixture(scope="module")
def vr():
    import __graft_entry__
    __graft_entry__.build_library()
    from paper_2501_01628_gb300 import vr as _vr
    return _vr


def _over_np(pieces, out):
    """Front-to-back "over" of numpy/torch CPU arrays (the CPU stand-in for the
    library's vr_composite_images in these CPU-only tests)."""
    acc = np.zeros(np.asarray(pieces[0]).shape)
    for p in pieces:
        p = np.asarray(p, dtype=np.float64)
        acc = acc + (1.0 - acc[..., 3:4]) * p
    out[...] = acc if isinstance(out, np.ndarray) else type(out)(acc)


def _scene(n=16):
    rng = np.random.default_rng(23)
    vol = synth.blob_volume(n, synth.draw_blobs(rng, 6))
    vol += rng.uniform(0, 0.05, vol.shape).astype(np.float32)
    tf = synth.random_tf(rng, alpha_max=0.3)
    return vol, tf, float(vol.min()), float(vol.max())


def _rank_images(vr, vol, tf, lo, hi, cam, part, world):
    """Per rank: its share's partials composited front to back (library order)."""
    dims = vol.shape[::-1]
    boxes = vr.vr_partition_boxes(dims, part)
    shares, tree = sharded.brick_shares(boxes, world)
    res = oracle.render(vol, boxes, tf, lo, hi, cam, 0.5, with_partials=True)
    order, _ = vr.vr_plan_view(dims, part, cam)
    imgs = []
    for share in shares:
        acc = np.zeros(res["img"].shape)
        for b in order:
            if b in share:
                acc = acc + (1.0 - acc[..., 3:4]) * res["partials"][b]
        imgs.append(acc)
    return imgs, sharded.share_order(tree, cam, dims), res["img"], shares, tree, boxes


@pytest.mark.parametrize("part", [dict(kind="grid", grid=(4, 3, 3)), dict(kind="kd", n_bricks=16,
                                                                         cut_fracs=np.linspace(0.3, 0.7, 15))])
@pytest.mark.parametrize("world", [1, 2, 3, 4, 6, 8])
def test_shares_are_separable_and_cover_every_brick(vr, part, world):
    dims = (24, 18, 18)
    boxes = vr.vr_partition_boxes(dims, part)
    shares, tree = sharded.brick_shares(boxes, world)
    assert len(shares) == world and all(shares)
    assert sorted(b for s in shares for b in s) == list(range(len(boxes)))

    def check(node):
        if node[0] == "leaf":
            return set(shares[node[1]])
        _, axis, cut, low, high = node
        lo_ids, hi_ids = check(low), check(high)
        assert all(boxes[b][3 + axis] <= cut for b in lo_ids)
        assert all(boxes[b][axis] >= cut for b in hi_ids)
        return lo_ids | hi_ids

    assert check(tree) == set(range(len(boxes)))


def test_radix_schedule_bands_tile_the_image():
    for world, factors in ((4, (2, 2)), (6, (2, 3)), (6, (3, 2)), (8, (2, 2, 2)), (8, (8,)), (5, (5,))):
        for H in (7, 40, 1080):
            _, region = sharded.radix_rounds(world, factors, H)
            rows = sorted(region.values())
            assert rows[0][0] == 0 and rows[-1][1] == H
            assert all(a[1] == b[0] for a, b in zip(rows, rows[1:]))
    with pytest.raises(ValueError):
        sharded.radix_rounds(4, (3,), 10)


@pytest.mark.parametrize("world,factors", [(2, (2,)), (4, (2, 2)), (4, (4,)), (6, (3, 2)), (8, (2, 2, 2))])
@pytest.mark.parametrize("camkind", ["persp", "ortho"])
def test_exchange_in_one_process_equals_unsplit_render(vr, world, factors, camkind):
    vol, tf, lo, hi = _scene()
    cam = (synth.orbit_camera(20, 14, 130.0, elevation_deg=-25.0) if camkind == "persp"
           else dict(ortho=1, eye=(0.5, 0.5, 1.5), dir=(0.3, -0.2, -1.0), up=(0, 1, 0), ortho_w=1.5, ortho_h=1.2,
                     width=20, height=14))
    part = dict(kind="grid", grid=(4, 2, 2))
    imgs, rank_of_pos, want, *_ = _rank_images(vr, vol, tf, lo, hi, cam, part, world)
    got = sharded.composite_bands(imgs, rank_of_pos, factors, _over_np, lambda shape: np.zeros(shape))
    np.testing.assert_allclose(got, want, atol=1e-12, rtol=0)


def test_wrong_share_order_is_detected(vr):
    """Control: the exchange in reverse share order no longer equals the render."""
    vol, tf, lo, hi = _scene()
    cam = synth.orbit_camera(20, 14, 130.0, elevation_deg=-25.0)
    imgs, rank_of_pos, want, *_ = _rank_images(vr, vol, tf, lo, hi, cam, dict(kind="grid", grid=(4, 2, 2)), 4)
    got = sharded.composite_bands(imgs, rank_of_pos[::-1], (4,), _over_np, lambda shape: np.zeros(shape))
    assert np.abs(got - want).max() > 1e-3


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, factors, port, q):
    import torch
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        import __graft_entry__
        __graft_entry__.build_library()
        oracle.build()
        from paper_2501_01628_gb300 import vr
        vol, tf, lo, hi = _scene()
        cam = synth.orbit_camera(20, 14, 250.0, elevation_deg=30.0)
        imgs, rank_of_pos, want, *_ = _rank_images(vr, vol, tf, lo, hi, cam, dict(kind="grid", grid=(4, 2, 2)),
                                                   world)
        t = sharded.TorchDistributedTransport()
        mine = torch.from_numpy(imgs[rank])

        def combine(pieces, out):
            acc = torch.zeros_like(out)
            for p in pieces:
                acc = acc + (1.0 - acc[..., 3:4]) * p
            out.copy_(acc)

        _, band = sharded.run_exchange(rank_of_pos, rank, mine, factors, t, combine,
                                       lambda shape: torch.zeros(shape, dtype=torch.float64))
        frame = torch.zeros(mine.shape, dtype=torch.float64) if rank == 0 else None
        frame = sharded.gather_bands(band, rank_of_pos, rank, factors, t, frame)
        err = float(np.abs(frame.numpy() - want).max()) if rank == 0 else None
        q.put((rank, err))
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("world,factors", [(2, (2,)), (4, (2, 2)), (4, (4,))])
def test_exchange_over_gloo_ranks_equals_unsplit_render(world, factors):
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, world, factors, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = {}
    for _ in procs:
        r, err = q.get(timeout=240)
        res[r] = err
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert res[0] is not None and res[0] < 1e-12
