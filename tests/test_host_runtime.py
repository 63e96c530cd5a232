"""CPU tests of the C-ABI library: it loads, exports every declared symbol, and
its host-side planning (partitions, kd visibility order, footprint rectangles)
agrees with the oracle. No GPU calls."""
import re
import os

import numpy as np
import pytest

import oracle
from paper_2501_01628_gb300 import synth

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def vr():
    import __graft_entry__
    __graft_entry__.build_library()
    from paper_2501_01628_gb300 import vr as _vr
    _vr.lib()
    return _vr


def _declared_functions():
    text = open(os.path.join(ROOT, "include", "vr.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"^\s*(?:vr_status|const char \*)\s*(vr_\w+)\s*\(", text, flags=re.M)))


def test_library_exports_every_declared_symbol(vr):
    declared = _declared_functions()
    assert len(declared) >= 20
    L = vr.lib()
    missing = [n for n in declared if not hasattr(L, n)]
    assert not missing
    assert sorted(vr.EXPORTS) == declared


def test_status_strings(vr):
    L = vr.lib()
    for s in range(7):
        assert L.vr_status_string(s)
    assert L.vr_last_error(None) == b"null context"


def test_create_without_gpu_fails_cleanly(vr):
    import torch
    if torch.cuda.is_available():
        pytest.skip("GPU present")
    with pytest.raises(vr.VrError):
        vr.vr_create(0)


@pytest.mark.parametrize("dims,g", [((64, 64, 64), (2, 2, 2)), ((512, 512, 512), (4, 3, 3)),
                                    ((37, 20, 9), (3, 2, 1))])
def test_grid_partition_matches_oracle(vr, dims, g):
    got = vr.vr_partition_boxes(dims, dict(kind="grid", grid=g))
    np.testing.assert_array_equal(got, oracle.grid_partition(dims, g))


@pytest.mark.parametrize("dims,n,seed", [((1024,) * 3, 64, 2), ((768,) * 3, 48, 3), ((50, 40, 30), 17, 9)])
def test_kd_partition_matches_oracle(vr, dims, n, seed):
    u = synth.kd_cut_fractions(np.random.default_rng(seed), n)
    got = vr.vr_partition_boxes(dims, dict(kind="kd", n_bricks=n, cut_fracs=u))
    np.testing.assert_array_equal(got, oracle.kd_partition(dims, n, u))


def test_box_partitions_validated(vr):
    ok = [[0, 0, 0, 10, 24, 24], [10, 0, 0, 24, 7, 24], [10, 7, 0, 24, 24, 13],
          [10, 7, 13, 17, 24, 24], [17, 7, 13, 24, 24, 24]]
    np.testing.assert_array_equal(vr.vr_partition_boxes((24, 24, 24), dict(kind="boxes", boxes=ok)), ok)
    gap = [b[:] for b in ok]
    gap[4][3] = 23
    overlap = [b[:] for b in ok]
    overlap[3][3] = 18
    # a pinwheel tiling of a 3x3 square: no axis-aligned cut separates it
    pin = [[0, 0, 0, 2, 1, 1], [2, 0, 0, 3, 2, 1], [1, 2, 0, 3, 3, 1], [0, 1, 0, 1, 3, 1],
           [1, 1, 0, 2, 2, 1]]
    for bad, dims in ((gap, (24, 24, 24)), (overlap, (24, 24, 24)), (pin, (3, 3, 1))):
        with pytest.raises(vr.VrError):
            vr.vr_partition_boxes(dims, dict(kind="boxes", boxes=bad))
    with pytest.raises(vr.VrError):
        vr.vr_partition_boxes((8, 8, 8), dict(kind="grid", grid=(9, 1, 1)))
    with pytest.raises(vr.VrError):
        vr.vr_partition_boxes((8, 8, 8), dict(kind="kd", n_bricks=200, cut_fracs=[0.5] * 199))


def _over(parts_in_order):
    acc = np.zeros(parts_in_order[0].shape)
    for p in parts_in_order:
        acc = acc + (1 - acc[..., 3:4]) * p
    return acc


@pytest.mark.parametrize("case", range(6))
def test_visibility_order_and_footprints_against_oracle(vr, case):
    """Compositing the oracle's per-brick partials in the library's kd order
    reproduces the oracle's image (which orders bricks along each ray), and
    every partial is zero outside the library's footprint rectangle."""
    rng = np.random.default_rng(100 + case)
    n = 20
    vol = synth.blob_volume(n, synth.draw_blobs(rng, 5))
    tf = synth.random_tf(rng, alpha_max=0.2)
    cams = [synth.orbit_camera(30, 22, 37.0), synth.orbit_camera(25, 25, 200.0, elevation_deg=-50),
            synth.orbit_camera(31, 17, 90.0, radius=0.9, elevation_deg=5),  # eye close to the volume
            synth.ortho_camera_z(24, 24),
            dict(ortho=1, eye=(0.5, 0.5, 1.2), dir=(0.2, -0.3, -1.0), up=(0, 1, 0), ortho_w=1.6,
                 ortho_h=1.4, width=27, height=23),
            synth.orbit_camera(28, 20, 300.0, radius=0.3, elevation_deg=10)]  # eye inside
    cam = cams[case]
    parts = [dict(kind="grid", grid=(2, 3, 2)),
             dict(kind="kd", n_bricks=9, cut_fracs=rng.uniform(0.3, 0.7, 8))]
    for part in parts:
        boxes = vr.vr_partition_boxes((n,) * 3, part)
        order, rects = vr.vr_plan_view((n,) * 3, part, cam)
        assert sorted(order) == list(range(len(boxes)))
        ref = oracle.render(vol, boxes, tf, float(vol.min()), float(vol.max()), cam, 0.5,
                            with_partials=True)
        got = _over([ref["partials"][b] for b in order])
        np.testing.assert_allclose(got, ref["img"], atol=1e-12)
        H, W = cam["height"], cam["width"]
        for b, (x0, y0, w, h) in enumerate(rects):
            mask = np.ones((H, W), bool)
            mask[y0:y0 + h, x0:x0 + w] = False
            assert np.all(ref["partials"][b][mask] == 0), (b, (x0, y0, w, h))


def test_binding_rejects_mistyped_or_misshaped_buffers_before_any_launch():
    """The C side gets bare pointers and cannot check sizes, so the binding
    refuses a wrong dtype, rank, shape, layout or memory space up front (a
    16-bit volume read as float32, or an image smaller than H x W x 4, would be
    an out-of-bounds access on the device). Nothing here reaches the library."""
    import ctypes
    import torch
    from paper_2501_01628_gb300 import vr
    cam = synth.orbit_camera(8, 6, 30.0)
    part = dict(kind="grid", grid=(1, 1, 1))
    tf = synth.constant_tf([1, 1, 1, 0.1])
    good_vol = torch.zeros((4, 4, 4))
    good_out = torch.zeros((6, 8, 4))
    bad = [
        (torch.zeros((4, 4, 4), dtype=torch.bfloat16), good_out, "float32"),
        (torch.zeros((4, 16)), good_out, "3 dimensions"),
        (torch.zeros((4, 4, 8))[:, :, ::2], good_out, "contiguous"),
        (good_vol, torch.zeros((8, 6, 4)), "shape"),
        (good_vol, torch.zeros((6, 8, 4), dtype=torch.float64), "float32"),
        (good_vol, good_out, "CUDA"),  # host memory where device memory is required
    ]
    for vol, out, msg in bad:
        with pytest.raises(ValueError, match=msg):
            vr.vr_render_frame_noalloc(vol, part, tf, 0.0, 1.0, cam, out)
    # context calls: the image must match the camera last set on the context
    fake = ctypes.c_void_p(0x1234)
    with pytest.raises(vr.VrError, match="no camera") as e:
        vr.vr_render_frame(fake, None, good_out)
    assert e.value.status == vr.VR_ERR_STATE
    vr._cam_size[vr._key(fake)] = (6, 8)
    try:
        for out, msg in ((torch.zeros((6, 8, 3)), "shape"), (torch.zeros(6 * 8 * 4), "shape"),
                         (torch.zeros((6, 8, 4), dtype=torch.float16), "float32"),
                         (np.zeros((6, 8, 4), np.float64), "float32"),
                         (np.zeros((8, 6, 4), np.float32).transpose(1, 0, 2), "contiguous")):
            with pytest.raises(ValueError, match=msg):
                vr.vr_render_frame(fake, None, out)
        with pytest.raises(ValueError, match="float32"):
            vr.vr_volume_create(fake, np.zeros((4, 4, 4), np.float64))
        with pytest.raises(ValueError, match="CUDA"):
            vr.vr_render_backward(fake, None, good_out, torch.zeros((2, 4)))
    finally:
        vr._cam_size.pop(vr._key(fake), None)
