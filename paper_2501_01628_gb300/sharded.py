"""Brick-sharded rendering across GPUs: bricks are ranks.

The paper distributes the data spatially over ranks, each holding a share
(Sec. 2.2; shares may be uneven, Sec. 4), and one collective render call
leaves the frame in one framebuffer on the main rank (Sec. 3). Here each rank
(one process per GPU) holds a contiguous share of the partition's bricks
(vr_volume_create_share), marches and composites it into a full-frame rank
image with the library (vr_render_frame), and the rank images are composited
front to back with a radix-k exchange; the final bands are gathered on rank 0.

Radix-k, for factors k_0 k_1 ... k_{m-1} = world: rank position p in the
view's front-to-back order of shares has digits d_i = (p / (k_0...k_{i-1})) % k_i.
In round i the k_i positions that differ only in digit i form a group; all hold
the same row band R_i of the image, split it into k_i bands, send band j to the
member with digit j, and composite the k_i pieces of their own band in digit
order (front to back) with vr_composite_images. After the last round every rank
holds 1/world of the rows, composited over all shares.

Orchestration only: marching, compositing and the per-round "over" run in the
library's kernels; this module decides who sends which row band to whom and
moves the bands with torch.distributed point-to-point calls. composite_bands
runs the same schedule for ranks emulated in one process (tests on one GPU).
"""
from __future__ import annotations

import numpy as np

from . import vr

# --------------------------------------------------------------------------
# shares: a kd split of the bricks into `world` contiguous groups
# --------------------------------------------------------------------------


def brick_shares(boxes, world: int):
    """Split the bricks (boxes: (n, 6) voxel boxes lo xyz, hi xyz) into `world`
    shares by axis-aligned planes, balancing voxel counts. Returns (shares,
    tree): shares[r] = sorted brick ids of rank r; tree = nested tuples
    ("leaf", r) or ("split", axis, cut, low, high), whose traversal towards the
    eye gives the shares' front-to-back order (share_order)."""
    boxes = np.asarray(boxes, dtype=np.int64).reshape(-1, 6)
    if world < 1 or world > boxes.shape[0]:
        raise ValueError("need 1 <= world <= number of bricks")
    vox = np.prod(boxes[:, 3:] - boxes[:, :3], axis=1).astype(np.float64)
    shares = []

    def build(ids, m):
        if m == 1:
            shares.append(sorted(int(i) for i in ids))
            return ("leaf", len(shares) - 1)
        m1 = m // 2
        total = vox[ids].sum()
        best = None
        for axis in range(3):
            for cut in np.unique(np.concatenate([boxes[ids, axis], boxes[ids, 3 + axis]])):
                low = [i for i in ids if boxes[i, 3 + axis] <= cut]
                high = [i for i in ids if boxes[i, axis] >= cut]
                if len(low) + len(high) != len(ids) or len(low) < m1 or len(high) < m - m1:
                    continue  # not a separating plane, or too few bricks for the ranks
                err = abs(vox[low].sum() / total - m1 / m)
                if best is None or err < best[0]:
                    best = (err, axis, int(cut), low, high)
        if best is None:
            raise ValueError("the bricks cannot be separated into %d shares by axis-aligned planes" % m)
        _, axis, cut, low, high = best
        return ("split", axis, cut, build(low, m1), build(high, m - m1))

    tree = build(list(range(boxes.shape[0])), world)
    return shares, tree


def share_order(tree, cam: dict, dims):
    """Front-to-back order of the shares for a camera: the library's rule for
    its brick tree (near side = the eye's side of the plane, perspective; the
    low side when the view direction is >= 0 on the axis, orthographic)."""
    nmax = float(max(dims))
    out = []

    def walk(node):
        if node[0] == "leaf":
            out.append(node[1])
            return
        _, axis, cut, low, high = node
        low_first = cam["dir"][axis] >= 0.0 if cam["ortho"] else cam["eye"][axis] * nmax <= cut
        walk(low if low_first else high)
        walk(high if low_first else low)

    walk(tree)
    return out


# --------------------------------------------------------------------------
# radix-k schedule
# --------------------------------------------------------------------------


def _band(lo: int, hi: int, k: int, j: int):
    n = hi - lo
    return lo + (n * j) // k, lo + (n * (j + 1)) // k


def radix_rounds(world: int, factors, height: int):
    """Per round i and position p: (group positions in digit order, the band
    split of the group's rows, p's own band). The product of factors must be
    world."""
    factors = [int(k) for k in factors] or [world]
    if int(np.prod(factors)) != world:
        raise ValueError("radix-k factors must multiply to the number of ranks")
    region = {p: (0, height) for p in range(world)}
    rounds = []
    stride = 1
    for k in factors:
        rnd = {}
        new_region = {}
        for p in range(world):
            d = (p // stride) % k
            base = p - d * stride
            group = [base + j * stride for j in range(k)]
            lo, hi = region[p]
            bands = [_band(lo, hi, k, j) for j in range(k)]
            rnd[p] = dict(group=group, digit=d, bands=bands)
            new_region[p] = bands[d]
        rounds.append(rnd)
        region = new_region
        stride *= k
    return rounds, region


# --------------------------------------------------------------------------
# transports
# --------------------------------------------------------------------------


class TorchDistributedTransport:
    """Row bands between ranks with torch.distributed point-to-point calls
    (NCCL for CUDA tensors, gloo for CPU tensors)."""

    def __init__(self, group=None):
        import torch.distributed as dist
        self.dist = dist
        self.group = group
        self.rank = dist.get_rank(group)
        self.world = dist.get_world_size(group)

    def exchange(self, sends, recvs):
        """sends: [(peer rank, tensor)]; recvs: [(peer rank, tensor to fill)]."""
        reqs = []
        for peer, t in recvs:
            reqs.append(self.dist.irecv(t, src=peer, group=self.group))
        for peer, t in sends:
            reqs.append(self.dist.isend(t.contiguous(), dst=peer, group=self.group))
        for r in reqs:
            r.wait()


def run_exchange(rank_of_pos, my_rank: int, image, factors, transport, combine, new_buffer):
    """Radix-k over the ranks' full-frame images (image: [H, W, 4], this rank's
    image). rank_of_pos[p] = rank at front-to-back position p. combine(pieces,
    out) writes pieces[0] over pieces[1] over ... into out. Returns (band rows
    (lo, hi), the composited band) held by this rank after the last round."""
    world = len(rank_of_pos)
    H = image.shape[0]
    pos = rank_of_pos.index(my_rank)
    rounds, region = radix_rounds(world, factors, H)
    cur, cur_lo = image, 0  # cur holds rows [cur_lo, cur_lo + cur.shape[0])
    for rnd in rounds:
        me = rnd[pos]
        lo, hi = me["bands"][me["digit"]]
        pieces = []
        sends, recvs = [], []
        for j, q in enumerate(me["group"]):
            blo, bhi = me["bands"][j]
            if q == pos:
                pieces.append(cur[lo - cur_lo:hi - cur_lo])
            else:
                if bhi > blo:  # both sides skip empty bands alike
                    sends.append((rank_of_pos[q], cur[blo - cur_lo:bhi - cur_lo]))
                buf = new_buffer((hi - lo,) + tuple(image.shape[1:]))
                if hi > lo:
                    recvs.append((rank_of_pos[q], buf))
                pieces.append(buf)
        transport.exchange(sends, recvs)
        out = new_buffer((hi - lo,) + tuple(image.shape[1:]))
        if hi > lo:
            combine(pieces, out)
        cur, cur_lo = out, lo
    return region[pos], cur


def gather_bands(band, rank_of_pos, my_rank: int, factors, transport, frame=None, root: int = 0):
    """Collect every rank's final band on `root` into `frame` ([H, W, 4]; root
    only). The bands follow from the same schedule (factors) on every rank."""
    world = len(rank_of_pos)
    if my_rank != root:
        if band.shape[0] > 0:
            transport.exchange([(root, band)], [])
        return None
    _, region = radix_rounds(world, factors, frame.shape[0])
    recvs = []
    for pos in range(world):
        r = rank_of_pos[pos]
        lo, hi = region[pos]
        if r == root:
            frame[lo:hi] = band
        elif hi > lo:
            recvs.append((r, frame[lo:hi]))
    transport.exchange([], recvs)
    return frame


def composite_bands(images, rank_of_pos, factors, combine, new_buffer):
    """The whole exchange for ranks emulated in one process (images[r] is rank
    r's full-frame image), round by round as run_exchange runs it on every
    rank. Returns the composited frame."""
    world = len(images)
    H = images[0].shape[0]
    rounds, region = radix_rounds(world, factors, H)
    cur = {r: (images[r], 0) for r in range(world)}  # rank -> (rows held, first row)
    for rnd in rounds:
        nxt = {}
        for pos in range(world):
            me = rnd[pos]
            lo, hi = me["bands"][me["digit"]]
            pieces = []
            for q in me["group"]:
                src, src_lo = cur[rank_of_pos[q]]
                pieces.append(src[lo - src_lo:hi - src_lo])
            out = new_buffer((hi - lo,) + tuple(images[0].shape[1:]))
            if hi > lo:
                combine(pieces, out)
            nxt[rank_of_pos[pos]] = (out, lo)
        cur = nxt
    frame = new_buffer(tuple(images[0].shape))
    for pos in range(world):
        band, lo = cur[rank_of_pos[pos]]
        frame[lo:lo + band.shape[0]] = band
    return frame


# --------------------------------------------------------------------------
# the renderer of one rank
# --------------------------------------------------------------------------


class ShardedRenderer:
    """One rank of a brick-sharded renderer: holds its share of the bricks on
    its GPU, renders its image with the library and takes part in the radix-k
    exchange; render() returns the frame on `root` (None elsewhere).

    ctx: this rank's library context (on its GPU; the context's transfer
    function, step and early termination apply); volume: [Nz, Ny, Nx] float32
    (the whole volume: only this rank's bricks and halos are read); partition:
    as for vr_volume_create; factors: radix-k factors multiplying to the number
    of ranks (default: one round of all ranks); transport: a
    TorchDistributedTransport (default: the default process group)."""

    def __init__(self, ctx, volume, partition, factors=None, transport=None, storage: str = "f32", root: int = 0):
        import torch
        self.transport = transport or TorchDistributedTransport()
        self.world, self.rank = self.transport.world, self.transport.rank
        self.factors = [int(k) for k in factors] if factors else [self.world]
        self.ctx = ctx
        self.root = root
        self.dims = tuple(int(d) for d in tuple(volume.shape)[::-1])
        boxes = vr.vr_partition_boxes(self.dims, partition)
        self.shares, self.tree = brick_shares(boxes, self.world)
        self.vol = vr.vr_volume_create_share(ctx, volume, self.shares[self.rank], storage, partition)
        self.torch = torch

    def _combine(self, pieces, out):
        vr.vr_composite_images(self.ctx, pieces, out)

    def _buffer(self, shape):
        return self.torch.empty(shape, dtype=self.torch.float32, device="cuda")

    def render(self, cam: dict, frame=None):
        vr.vr_set_camera(self.ctx, cam)
        img = self._buffer((int(cam["height"]), int(cam["width"]), 4))
        vr.vr_render_frame(self.ctx, self.vol, img)
        rank_of_pos = share_order(self.tree, cam, self.dims)  # share r is held by rank r
        if self.world == 1:
            if frame is not None:
                frame.copy_(img)
                return frame
            return img
        _, band = run_exchange(rank_of_pos, self.rank, img, self.factors, self.transport, self._combine,
                               self._buffer)
        if self.rank == self.root and frame is None:
            frame = self._buffer(tuple(img.shape))
        return gather_bands(band, rank_of_pos, self.rank, self.factors, self.transport, frame, self.root)

    def close(self):
        if self.vol is not None:
            vr.vr_volume_release(self.vol)
            self.vol = None
