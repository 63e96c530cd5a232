"""Error paths under injected faults (vr_debug_inject_fault): a device
allocation or kernel launch made by the library fails on the host, without
calling CUDA and without any GPU fault. The call reports the failure, and the
context and its objects stay usable: the next call succeeds and gives the same
image as a run without the fault."""
import numpy as np
import pytest

from paper_2501_01628_gb300 import synth


@pytest.fixture(scope="module")
def vrlib():
    import __graft_entry__
    __graft_entry__.build_library()
    from paper_2501_01628_gb300 import vr as _vr
    return _vr


def test_fault_plan_arguments(vrlib):
    vr = vrlib
    for kind, after in ((3, 0), (-1, 0), (vr.VR_FAULT_ALLOC, -1)):
        with pytest.raises(vr.VrError) as e:
            vr.vr_debug_inject_fault(kind, after)
        assert e.value.status == vr.VR_ERR_ARG
    vr.vr_debug_inject_fault(vr.VR_FAULT_LAUNCH, 5)
    vr.vr_debug_inject_fault(vr.VR_FAULT_NONE, 0)


def _scene():
    vol, tf = synth.small_blob_scene(n=32)
    cam = synth.orbit_camera(40, 36, 30.0)
    return vol, tf, cam


def _setup(vr, ctx, vol, tf, cam):
    vr.vr_set_transfer_function(ctx, tf, float(vol.min()), float(vol.max()))
    vr.vr_set_camera(ctx, cam)
    vr.vr_set_render_params(ctx, 0.5, 0.99)
    vr.vr_set_composite_schedule(ctx, (2, 4))


def _render(vr, ctx, v, cam):
    import torch
    out = torch.empty((cam["height"], cam["width"], 4), dtype=torch.float32, device="cuda")
    vr.vr_render_frame(ctx, v, out)
    vr.vr_sync(ctx)
    return out.cpu().numpy()


@pytest.fixture(scope="module")
def reference(vrlib):
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    vr = vrlib
    vol, tf, cam = _scene()
    ctx = vr.vr_create(0)
    try:
        _setup(vr, ctx, vol, tf, cam)
        v = vr.vr_volume_create(ctx, vol, "f32", dict(kind="grid", grid=(2, 2, 2)))
        img = _render(vr, ctx, v, cam)
        vr.vr_volume_release(v)
    finally:
        vr.vr_destroy(ctx)
    return img


@pytest.mark.gpu
def test_allocation_fault_in_volume_creation(vrlib, reference):
    vr = vrlib
    vol, tf, cam = _scene()
    ctx = vr.vr_create(0)
    try:
        _setup(vr, ctx, vol, tf, cam)
        vr.vr_debug_inject_fault(vr.VR_FAULT_ALLOC, 0)
        with pytest.raises(vr.VrError) as e:
            vr.vr_volume_create(ctx, vol, "f32", dict(kind="grid", grid=(2, 2, 2)))
        assert e.value.status == vr.VR_ERR_OOM
        v = vr.vr_volume_create(ctx, vol, "f32", dict(kind="grid", grid=(2, 2, 2)))
        assert np.array_equal(_render(vr, ctx, v, cam), reference)
        vr.vr_volume_release(v)
    finally:
        vr.vr_debug_inject_fault(vr.VR_FAULT_NONE, 0)
        vr.vr_destroy(ctx)


@pytest.mark.gpu
def test_allocation_fault_in_frame_pool(vrlib, reference):
    vr = vrlib
    vol, tf, cam = _scene()
    ctx = vr.vr_create(0)
    try:
        _setup(vr, ctx, vol, tf, cam)
        v = vr.vr_volume_create(ctx, vol, "f32", dict(kind="grid", grid=(2, 2, 2)))
        vr.vr_debug_inject_fault(vr.VR_FAULT_ALLOC, 0)  # the first frame grows the partial pool
        with pytest.raises(vr.VrError) as e:
            _render(vr, ctx, v, cam)
        assert e.value.status == vr.VR_ERR_OOM
        assert np.array_equal(_render(vr, ctx, v, cam), reference)
        vr.vr_volume_release(v)
    finally:
        vr.vr_debug_inject_fault(vr.VR_FAULT_NONE, 0)
        vr.vr_destroy(ctx)


@pytest.mark.gpu
def test_launch_fault_in_composite(vrlib, reference):
    vr = vrlib
    vol, tf, cam = _scene()
    ctx = vr.vr_create(0)
    try:
        _setup(vr, ctx, vol, tf, cam)
        v = vr.vr_volume_create(ctx, vol, "f32", dict(kind="grid", grid=(2, 2, 2)))
        _render(vr, ctx, v, cam)
        vr.vr_debug_inject_fault(vr.VR_FAULT_LAUNCH, 1)  # the march launches, the composite fails
        with pytest.raises(vr.VrError) as e:
            _render(vr, ctx, v, cam)
        assert e.value.status == vr.VR_ERR_CUDA
        assert "injected" in str(e.value)
        assert np.array_equal(_render(vr, ctx, v, cam), reference)
        vr.vr_volume_release(v)
    finally:
        vr.vr_debug_inject_fault(vr.VR_FAULT_NONE, 0)
        vr.vr_destroy(ctx)


@pytest.mark.gpu
def test_launch_fault_in_pack(vrlib, reference):
    vr = vrlib
    vol, tf, cam = _scene()
    ctx = vr.vr_create(0)
    try:
        _setup(vr, ctx, vol, tf, cam)
        v = vr.vr_volume_create(ctx, vol, "f32", dict(kind="grid", grid=(2, 2, 2)))
        other = np.ascontiguousarray(vol[::-1])
        vr.vr_volume_update(v, other)
        vr.vr_debug_inject_fault(vr.VR_FAULT_LAUNCH, 0)
        with pytest.raises(vr.VrError) as e:
            vr.vr_volume_update(v, vol)
        assert e.value.status == vr.VR_ERR_CUDA
        vr.vr_volume_update(v, vol)
        assert np.array_equal(_render(vr, ctx, v, cam), reference)
        vr.vr_volume_release(v)
    finally:
        vr.vr_debug_inject_fault(vr.VR_FAULT_NONE, 0)
        vr.vr_destroy(ctx)
