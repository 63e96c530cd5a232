"""Pipelined frames (vr_set_frame_pipelining) against the plain sequence.

A pipelined vr_render_frame marches into one of two partial pools and may start
while the previous frame's composite runs; the per-pixel arithmetic is the
plain path's (Sec. 3: render, then composite front to back), so every image
must equal the plain sequence's bit for bit. The sequences are launched without
host synchronisation between frames, into distinct outputs and into one output
read by stream-ordered torch copies, and are interleaved with everything that
changes what a march reads (volume updates, transfer-function uploads, camera
and image-size changes, another stream, host outputs, other frame calls)."""
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


def _scene(n=48, seed=11):
    rng = np.random.default_rng(seed)
    vol = synth.blob_volume(n, synth.draw_blobs(rng, 7))
    vol += rng.uniform(0, 0.05, vol.shape).astype(np.float32)
    tf = synth.random_tf(rng, alpha_max=0.2)
    return vol, tf, rng


def _ctx(vr, vol, part, tf, pipelined, storage="f32", schedule=(), ert=1.0, pw=4, count=False, lo_hi=None):
    lo, hi = lo_hi or synth.volume_range(vol)
    ctx = vr.vr_create(0)
    vr.vr_set_frame_pipelining(ctx, pipelined)
    v = vr.vr_volume_create(ctx, vol, storage, part)
    vr.vr_set_transfer_function(ctx, tf, lo, hi)
    vr.vr_set_render_params(ctx, 0.5, ert)
    vr.vr_set_composite_schedule(ctx, schedule)
    vr.vr_set_packet_width(ctx, pw)
    vr.vr_set_count_samples(ctx, count)
    return ctx, v


def _close(vr, ctx, v):
    vr.vr_volume_release(v)
    vr.vr_destroy(ctx)


def _sequence(vr, ctx, v, cams, reuse_out=False):
    """All frames launched back to back on the current stream, one sync at the end."""
    import torch
    outs = []
    if reuse_out:
        shared = {}
        for cam in cams:
            vr.vr_set_camera(ctx, cam)
            key = (cam["height"], cam["width"])
            if key not in shared:
                shared[key] = torch.full((cam["height"], cam["width"], 4), float("nan"), device="cuda")
            vr.vr_render_frame(ctx, v, shared[key])
            outs.append(shared[key].clone())  # stream-ordered after this frame's composite
    else:
        for cam in cams:
            vr.vr_set_camera(ctx, cam)
            o = torch.full((cam["height"], cam["width"], 4), float("nan"), device="cuda")
            vr.vr_render_frame(ctx, v, o)
            outs.append(o)
    vr.vr_sync(ctx)
    return [o.cpu() for o in outs]


def _assert_equal(a, b):
    import torch
    assert len(a) == len(b)
    for i, (x, y) in enumerate(zip(a, b)):
        assert not torch.isnan(y).any(), i
        assert torch.equal(x, y), (i, float((x - y).abs().max()))


_CASES = ["grid_direct", "kd_radix", "ert_pw8", "bf16_octets", "count", "reuse_out"]


@pytest.mark.parametrize("case", _CASES)
def test_pipelined_sequence_equals_plain(vr, case):
    vol, tf, rng = _scene()
    part = dict(kind="grid", grid=(2, 2, 2))
    cams = [synth.orbit_camera(101, 67, az, elevation_deg=el)
            for az, el in ((20, 25), (200, -40), (290, 5), (20, 25), (110, 60), (330, -10))]
    kw, reuse = {}, False
    if case == "kd_radix":
        part = dict(kind="kd", n_bricks=12, cut_fracs=rng.uniform(0.3, 0.7, 11))
        kw["schedule"] = (3, 2, 2)
    elif case == "ert_pw8":
        kw.update(ert=0.95, pw=8)
    elif case == "bf16_octets":
        kw["storage"] = "bf16"
    elif case == "count":
        kw["count"] = True
    elif case == "reuse_out":
        reuse = True
    res = {}
    for pipelined in (False, True):
        ctx, v = _ctx(vr, vol, part, tf, pipelined, **kw)
        try:
            if case == "bf16_octets":
                vr.vr_volume_release(v)
                vr.vr_set_cell_layout(ctx, 1)
                v = vr.vr_volume_create(ctx, vol, "bf16", part)
            if case == "count":
                counts = []
                for cam in cams:
                    vr.vr_set_camera(ctx, cam)
                    import torch
                    o = torch.empty((cam["height"], cam["width"], 4), device="cuda")
                    vr.vr_render_frame(ctx, v, o)
                    counts.append(vr.vr_get_sample_count(ctx))
                res[pipelined, "count"] = counts
            res[pipelined] = _sequence(vr, ctx, v, cams, reuse_out=reuse)
        finally:
            _close(vr, ctx, v)
    _assert_equal(res[False], res[True])
    if case == "count":
        assert res[False, "count"] == res[True, "count"]


def _ops(vr, ctx, v, vols, tfs, lo_hi, cams, stream2, sync_each):
    """One fixed sequence of frames and state changes; returns every image."""
    import torch
    lo, hi = lo_hi
    imgs = []

    def frame(cam, stream=None, host=False):
        vr.vr_set_camera(ctx, cam)
        shape = (cam["height"], cam["width"], 4)
        if host:
            o = np.full(shape, np.nan, np.float32)
            vr.vr_render_frame(ctx, v, o)
            imgs.append(torch.from_numpy(o))
            return
        o = torch.full(shape, float("nan"), device="cuda")
        if stream is None:
            vr.vr_render_frame(ctx, v, o)
        else:
            stream.wait_stream(torch.cuda.current_stream())
            o.record_stream(stream)
            vr.vr_render_frame(ctx, v, o, stream=stream)
            torch.cuda.current_stream().wait_stream(stream)
        imgs.append(o)
        if sync_each:
            vr.vr_sync(ctx)

    a, b, c = cams
    frame(a)
    frame(b)
    vr.vr_volume_update(v, vols[1])          # synchronous re-pack between frames
    frame(a)
    frame(c)                                 # another image size: the pools grow
    vr.vr_set_transfer_function(ctx, tfs[1], lo, hi)
    frame(b)
    frame(b, stream=stream2)                 # another stream
    frame(b)
    frame(a, host=True)                      # host output: the plain sequence
    frame(a)
    vr.vr_set_camera(ctx, c)                 # partials + composite of a caller-owned frame
    fr = vr.vr_render_partials(ctx, v)
    o = torch.full((c["height"], c["width"], 4), float("nan"), device="cuda")
    vr.vr_composite(ctx, fr, o)
    imgs.append(o)
    frame(c)
    vr.vr_volume_update_async(v, vols[2])    # asynchronous re-pack from device memory
    frame(a)
    frame(b)
    vr.vr_sync(ctx)
    vr.vr_frame_release(fr)
    return [i.cpu() for i in imgs]


def test_pipelined_frames_interleaved_with_state_changes(vr):
    import torch
    vol, tf, rng = _scene(n=40, seed=13)
    vol2 = (vol[::-1].copy() * 0.8 + 0.1).astype(np.float32)
    vol3 = torch.from_numpy(np.ascontiguousarray(vol.transpose(1, 0, 2))).cuda()
    tf2 = synth.random_tf(rng, alpha_max=0.3)
    lo_hi = (float(min(vol.min(), vol2.min())), float(max(vol.max(), vol2.max())))
    part = dict(kind="kd", n_bricks=9, cut_fracs=rng.uniform(0.3, 0.7, 8))
    cams = [synth.orbit_camera(96, 64, 35.0), synth.orbit_camera(80, 72, 160.0, elevation_deg=-30.0),
            synth.orbit_camera(150, 90, 260.0, radius=1.2)]
    s2 = torch.cuda.Stream()
    res = {}
    for pipelined in (False, True):
        ctx, v = _ctx(vr, vol, part, tf, pipelined, schedule=(3, 3), ert=0.99, lo_hi=lo_hi)
        try:
            res[pipelined] = _ops(vr, ctx, v, [vol, vol2, vol3], [tf, tf2], lo_hi, cams, s2,
                                  sync_each=not pipelined)
        finally:
            _close(vr, ctx, v)
    _assert_equal(res[False], res[True])


def test_pipelined_sequence_against_oracle(vr):
    vol, tf, rng = _scene(seed=17)
    part = dict(kind="kd", n_bricks=7, cut_fracs=rng.uniform(0.3, 0.7, 6))
    cams = [synth.orbit_camera(83, 61, az, elevation_deg=20.0) for az in (0.0, 120.0, 240.0)]
    cams.append(dict(ortho=1, eye=(0.5, 0.45, 1.4), dir=(0.25, -0.3, -1.0), up=(0, 1, 0), ortho_w=1.6,
                     ortho_h=1.3, width=70, height=57))
    ctx, v = _ctx(vr, vol, part, tf, True, schedule=(7,), ert=0.99)
    try:
        got = _sequence(vr, ctx, v, cams)
    finally:
        _close(vr, ctx, v)
    boxes = vr.vr_partition_boxes(vol.shape[::-1], part)
    lo, hi = synth.volume_range(vol)
    for cam, img in zip(cams, got):
        compare_envelope(img.numpy().astype(np.float64), oracle_env(vol, boxes, tf, lo, hi, cam, 0.5, 0.99))


def test_pipelined_paper_workload(vr):
    """512^3 noise + blobs, 36 bricks, the 8 orbit views at 1920x1080 twice,
    ERT 0.99, radix-k 4x3x3: pipelined frames equal the plain sequence."""
    import torch
    vol, tf = synth.noise_blob_scene()
    lo_hi = (float(vol.min()), float(vol.max()))
    vol_dev = torch.from_numpy(vol).cuda()
    cams = [synth.orbit_camera(1920, 1080, az) for az in synth.ORBIT_AZIMUTHS] * 2
    part = dict(kind="grid", grid=(4, 3, 3))
    res = {}
    for pipelined in (False, True):
        ctx, v = _ctx(vr, vol_dev, part, tf, pipelined, schedule=(4, 3, 3), ert=0.99, lo_hi=lo_hi)
        try:
            res[pipelined] = _sequence(vr, ctx, v, cams, reuse_out=True)
        finally:
            _close(vr, ctx, v)
    _assert_equal(res[False], res[True])


def test_pipelined_asynchronous_host_outputs(vr):
    """Asynchronous host outputs (two staging images, copies on the copy stream)
    in a pipelined sequence equal the plain sequence's device images."""
    import torch
    vol, tf, rng = _scene(seed=19)
    part = dict(kind="grid", grid=(3, 2, 2))
    cams = [synth.orbit_camera(88, 70, az, elevation_deg=15.0) for az in (10.0, 100.0, 190.0, 280.0, 10.0)]
    ctx, v = _ctx(vr, vol, part, tf, False, schedule=(3, 4), ert=0.99)
    try:
        want = _sequence(vr, ctx, v, cams)
    finally:
        _close(vr, ctx, v)
    ctx, v = _ctx(vr, vol, part, tf, True, schedule=(3, 4), ert=0.99)
    try:
        vr.vr_set_host_output_async(ctx, True)
        hosts = [torch.full((c["height"], c["width"], 4), float("nan")).pin_memory() for c in cams]
        for cam, h in zip(cams, hosts):
            vr.vr_set_camera(ctx, cam)
            vr.vr_render_frame(ctx, v, h)
        vr.vr_sync(ctx)
    finally:
        _close(vr, ctx, v)
    _assert_equal(want, hosts)


def test_pipelined_cycling_and_mixed_modes(vr):
    """Ray-state cycling frames (mode 1) pipelined, alone and alternating with
    sort-last frames, equal the plain sequence bit for bit."""
    vol, tf, rng = _scene(seed=23)
    part = dict(kind="kd", n_bricks=8, cut_fracs=rng.uniform(0.3, 0.7, 7))
    cams = [synth.orbit_camera(97, 63, az, elevation_deg=el) for az, el in ((5, 20), (95, -15), (185, 40), (275, 0))]
    modes = [1, 1, 1, 0, 1, 0, 0, 1]
    res = {}
    for pipelined in (False, True):
        ctx, v = _ctx(vr, vol, part, tf, pipelined, schedule=(2, 4), ert=0.97)
        try:
            import torch
            outs = []
            for i, m in enumerate(modes):
                vr.vr_set_render_mode(ctx, m)
                cam = cams[i % len(cams)]
                vr.vr_set_camera(ctx, cam)
                o = torch.full((cam["height"], cam["width"], 4), float("nan"), device="cuda")
                vr.vr_render_frame(ctx, v, o)
                outs.append(o)
            vr.vr_sync(ctx)
            res[pipelined] = [o.cpu() for o in outs]
        finally:
            _close(vr, ctx, v)
    _assert_equal(res[False], res[True])


def test_pipelined_frames_with_kernel_timing_and_toggles(vr):
    """Kernel timing switched on and off, pipelining switched off and on, and
    the maximum of 128 bricks, all inside one sequence: every frame equals the
    plain sequence's."""
    import torch
    vol, tf, rng = _scene(n=64, seed=29)
    part = dict(kind="grid", grid=(8, 4, 4))  # 128 bricks
    cams = [synth.orbit_camera(120, 80, az, elevation_deg=el) for az, el in ((15, 20), (135, -25), (255, 45))]
    plan = [("frame", 0), ("frame", 1), ("timing", True), ("frame", 2), ("frame", 0), ("timing", False),
            ("frame", 1), ("pipe", False), ("frame", 2), ("pipe", True), ("frame", 0), ("frame", 1)]
    res = {}
    for pipelined in (False, True):
        ctx, v = _ctx(vr, vol, part, tf, pipelined, schedule=(2, 4, 4, 4), ert=0.99)
        try:
            outs = []
            for op, arg in plan:
                if op == "timing":
                    vr.vr_set_kernel_timing(ctx, arg)
                    if not arg:
                        t = vr.vr_get_kernel_timing(ctx)
                        assert t["march_launches"] == 2 and t["composite_launches"] == 2
                elif op == "pipe":
                    vr.vr_set_frame_pipelining(ctx, arg and pipelined)
                else:
                    cam = cams[arg]
                    vr.vr_set_camera(ctx, cam)
                    o = torch.full((cam["height"], cam["width"], 4), float("nan"), device="cuda")
                    vr.vr_render_frame(ctx, v, o)
                    outs.append(o)
            vr.vr_sync(ctx)
            res[pipelined] = [o.cpu() for o in outs]
        finally:
            _close(vr, ctx, v)
    _assert_equal(res[False], res[True])


def test_pipelined_mesh_frames(vr):
    """Tetrahedral-mesh frames pipelined (the mesh march writes the tile masks,
    starts in the previous frame's tail and writes after it), alternating with
    voxel frames of the same context: every image equals the plain sequence's,
    and the mesh images equal a fresh plain render."""
    import torch
    n = 32
    part = dict(kind="kd", n_bricks=6, cut_fracs=np.linspace(0.35, 0.65, 5))
    boxes = vr.vr_partition_boxes((n, n, n), part)
    rng = np.random.default_rng(31)
    verts, tets = synth.tet_mesh((n, n, n), boxes, rng, cell_voxels=3.0, jitter=0.2, refine=1.5,
                                 focus=(0.35, 0.6, 0.45))
    vals = synth.mesh_field(rng, verts)
    tf = synth.random_tf(rng, alpha_max=0.04)
    lo, hi = float(vals.min()), float(vals.max())
    vol = synth.blob_volume(n, synth.draw_blobs(rng, 5))
    cams = [synth.orbit_camera(90, 66, az, elevation_deg=el) for az, el in ((10, 20), (130, -30), (250, 50))]
    plan = ["mesh", "mesh", "vol", "mesh", "mesh", "vol", "vol", "mesh"]
    res = {}
    for pipelined in (False, True):
        ctx = vr.vr_create(0)
        m = v = None
        try:
            vr.vr_set_frame_pipelining(ctx, pipelined)
            m = vr.vr_mesh_create(ctx, verts, vals, tets, (n, n, n), part)
            v = vr.vr_volume_create(ctx, vol, "f32", part)
            vr.vr_set_transfer_function(ctx, tf, lo, hi)
            vr.vr_set_render_params(ctx, 0.5, 0.99)
            vr.vr_set_composite_schedule(ctx, (2, 3))
            outs = []
            for i, kind in enumerate(plan):
                cam = cams[i % len(cams)]
                vr.vr_set_camera(ctx, cam)
                o = torch.full((cam["height"], cam["width"], 4), float("nan"), device="cuda")
                if kind == "mesh":
                    vr.vr_render_mesh_frame(ctx, m, o)
                else:
                    vr.vr_render_frame(ctx, v, o)
                outs.append(o)
            vr.vr_sync(ctx)
            res[pipelined] = [o.cpu() for o in outs]
        finally:
            if m is not None:
                vr.vr_mesh_release(m)
            if v is not None:
                vr.vr_volume_release(v)
            vr.vr_destroy(ctx)
    _assert_equal(res[False], res[True])


def test_pipelined_pool_wait_runs_out_and_recovers(vr):
    """The bounded pool wait of a pipelined march: a frame whose pool release
    never comes (vr_debug_pipeline_gap) gives up within seconds, vr_sync returns
    VR_ERR_TIMEOUT, and the frames after it equal the plain sequence's. Nothing
    faults or hangs."""
    import time
    import torch
    vol, tf, rng = _scene(n=32, seed=37)
    part = dict(kind="grid", grid=(2, 2, 1))
    cams = [synth.orbit_camera(48, 40, az) for az in (30.0, 150.0, 270.0)]
    ctx, v = _ctx(vr, vol, part, tf, False, ert=0.99)
    try:
        want = _sequence(vr, ctx, v, cams)
    finally:
        _close(vr, ctx, v)
    ctx, v = _ctx(vr, vol, part, tf, True, ert=0.99)
    try:
        first = _sequence(vr, ctx, v, cams)
        _assert_equal(want, first)
        vr.vr_debug_pipeline_gap(ctx)
        vr.vr_set_camera(ctx, cams[0])
        o = torch.empty((cams[0]["height"], cams[0]["width"], 4), device="cuda")
        t0 = time.perf_counter()
        vr.vr_render_frame(ctx, v, o)
        with pytest.raises(vr.VrError) as e:
            vr.vr_sync(ctx)
        assert e.value.status == vr.VR_ERR_TIMEOUT
        assert time.perf_counter() - t0 < 30.0
        after = _sequence(vr, ctx, v, cams)
        _assert_equal(want, after)
    finally:
        _close(vr, ctx, v)
