"""Thin ctypes binding of libvr (include/vr.h): same call names, argument
marshalling only. Every step of the rendering path runs in the library's CUDA
kernels; this module never computes pixels itself and raises if the library is
missing.

Arrays: volumes are [Nz, Ny, Nx] float32 (numpy or torch, host or CUDA);
images are [H, W, 4] float32 torch tensors (CUDA for device output, pinned or
pageable CPU for host output). Streams default to torch's current CUDA stream.
"""
from __future__ import annotations

import ctypes
import os
import threading

import numpy as np

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "libvr.so")
_lock = threading.Lock()
_lib = None

VR_OK, VR_ERR_ARG, VR_ERR_OOM, VR_ERR_CUDA, VR_ERR_STATE, VR_ERR_TIMEOUT, VR_ERR_BOUNDS = range(7)
VR_F32, VR_BF16, VR_F16 = 0, 1, 2
VR_PART_GRID, VR_PART_KD, VR_PART_BOXES = 0, 1, 2
VR_MAX_BRICKS = 128
DTYPES = {"f32": VR_F32, "bf16": VR_BF16, "f16": VR_F16}

# Every function the header declares (checked by the CPU test-suite).
EXPORTS = (
    "vr_create", "vr_destroy", "vr_status_string", "vr_last_error", "vr_sync",
    "vr_volume_create", "vr_volume_release", "vr_volume_info", "vr_volume_read_brick",
    "vr_set_transfer_function", "vr_set_camera", "vr_set_render_params",
    "vr_set_composite_schedule", "vr_set_count_samples", "vr_get_sample_count",
    "vr_render_partials", "vr_frame_info", "vr_frame_partial", "vr_composite",
    "vr_frame_release", "vr_render_frame", "vr_partition_boxes", "vr_plan_view",
    "vr_set_kernel_timing", "vr_get_kernel_timing", "vr_render_frame_noalloc",
    "vr_volume_update", "vr_render_backward", "vr_batch_create", "vr_batch_launch",
    "vr_batch_autotune", "vr_batch_release", "vr_batch_configure", "vr_set_render_mode",
    "vr_set_opacity_correction", "vr_volume_update_async", "vr_set_packet_width",
    "vr_set_host_output_async", "vr_mesh_create", "vr_mesh_release", "vr_mesh_info",
    "vr_render_mesh_frame", "vr_debug_inject_fault", "vr_batch_debug_wait", "vr_set_march_staging",
    "vr_volume_create_share", "vr_composite_images", "vr_set_cell_layout", "vr_set_frame_pipelining",
    "vr_debug_pipeline_gap",
)


class VrError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(msg)
        self.status = status


class vr_camera(ctypes.Structure):
    _fields_ = [("ortho", ctypes.c_int), ("eye", ctypes.c_double * 3),
                ("dir", ctypes.c_double * 3), ("up", ctypes.c_double * 3),
                ("fovy_deg", ctypes.c_double), ("ortho_w", ctypes.c_double),
                ("ortho_h", ctypes.c_double), ("width", ctypes.c_int), ("height", ctypes.c_int)]


class vr_partition(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int), ("grid", ctypes.c_int * 3), ("n_bricks", ctypes.c_int),
                ("cut_fracs", ctypes.c_void_p), ("boxes", ctypes.c_void_p)]


_P = ctypes.c_void_p
_I = ctypes.c_int
_SIG = {
    "vr_create": (_I, [_I, ctypes.POINTER(_P)]),
    "vr_destroy": (_I, [_P]),
    "vr_status_string": (ctypes.c_char_p, [_I]),
    "vr_last_error": (ctypes.c_char_p, [_P]),
    "vr_sync": (_I, [_P, _P]),
    "vr_volume_create": (_I, [_P, _P, _I, ctypes.POINTER(vr_partition), _P, _I, _P, ctypes.POINTER(_P)]),
    "vr_volume_release": (_I, [_P]),
    "vr_volume_create_share": (_I, [_P, _P, _I, ctypes.POINTER(vr_partition), _I, _P, _P, _I, _P,
                                    ctypes.POINTER(_P)]),
    "vr_composite_images": (_I, [_P, _I, _P, _P, ctypes.c_longlong, _P]),
    "vr_volume_info": (_I, [_P, _P, _P, _P]),
    "vr_volume_read_brick": (_I, [_P, _I, _P, ctypes.c_size_t]),
    "vr_set_transfer_function": (_I, [_P, _P, _I, ctypes.c_float, ctypes.c_float, _I]),
    "vr_set_camera": (_I, [_P, ctypes.POINTER(vr_camera)]),
    "vr_set_render_params": (_I, [_P, ctypes.c_float, ctypes.c_float]),
    "vr_set_composite_schedule": (_I, [_P, _I, _P]),
    "vr_set_count_samples": (_I, [_P, _I]),
    "vr_get_sample_count": (_I, [_P, ctypes.POINTER(ctypes.c_longlong)]),
    "vr_render_partials": (_I, [_P, _P, ctypes.POINTER(_P), _P]),
    "vr_frame_info": (_I, [_P, _P, _P, _P]),
    "vr_frame_partial": (_I, [_P, _I, ctypes.POINTER(_P)]),
    "vr_composite": (_I, [_P, _P, _P, _I, _P]),
    "vr_frame_release": (_I, [_P]),
    "vr_render_frame": (_I, [_P, _P, _P, _I, _P]),
    "vr_set_kernel_timing": (_I, [_P, _I]),
    "vr_debug_inject_fault": (_I, [_I, _I]),
    "vr_get_kernel_timing": (_I, [_P, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_longlong),
                                  ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_longlong)]),
    "vr_render_frame_noalloc": (_I, [_P, _P, ctypes.POINTER(vr_partition), _P, _I, ctypes.c_float,
                                     ctypes.c_float, ctypes.POINTER(vr_camera), ctypes.c_float,
                                     ctypes.c_float, _P, _P]),
    "vr_volume_update": (_I, [_P, _P, _I, _P]),
    "vr_volume_update_async": (_I, [_P, _P, _I, _P]),
    "vr_batch_create": (_I, [_P, _I, _P, _P, _P, _I, _P, _P, ctypes.POINTER(_P)]),
    "vr_batch_launch": (_I, [_P, _P]),
    "vr_batch_autotune": (_I, [_P, _P, ctypes.c_char_p, _P]),
    "vr_batch_release": (_I, [_P]),
    "vr_batch_configure": (_I, [_P, _I, _I, _I]),
    "vr_batch_debug_wait": (_I, [_P, _I, _I]),
    "vr_set_render_mode": (_I, [_P, _I]),
    "vr_set_opacity_correction": (_I, [_P, ctypes.c_float]),
    "vr_set_packet_width": (_I, [_P, _I]),
    "vr_set_march_staging": (_I, [_P, _I]),
    "vr_set_frame_pipelining": (_I, [_P, _I]),
    "vr_debug_pipeline_gap": (_I, [_P]),
    "vr_set_cell_layout": (_I, [_P, _I]),
    "vr_set_host_output_async": (_I, [_P, _I]),
    "vr_render_backward": (_I, [_P, _P, _P, _P, _P, _P]),
    "vr_partition_boxes": (_I, [_P, ctypes.POINTER(vr_partition), _P, _P]),
    "vr_plan_view": (_I, [_P, ctypes.POINTER(vr_partition), ctypes.POINTER(vr_camera), _P, _P]),
    "vr_mesh_create": (_I, [_P, _P, ctypes.POINTER(vr_partition), _P, ctypes.c_longlong, _P, _P,
                            ctypes.c_longlong, ctypes.POINTER(_P)]),
    "vr_mesh_release": (_I, [_P]),
    "vr_mesh_info": (_I, [_P, _P, _P, _P]),
    "vr_render_mesh_frame": (_I, [_P, _P, _P, _I, _P]),
}


def lib():
    """Load libvr.so (built by ``__graft_entry__.build()``); raise if absent."""
    global _lib
    with _lock:
        if _lib is None:
            if not os.path.exists(LIB_PATH):
                raise RuntimeError("libvr.so is not built (%s); run __graft_entry__.build()" % LIB_PATH)
            L = ctypes.CDLL(LIB_PATH)
            for name, (res, args) in _SIG.items():
                fn = getattr(L, name)
                fn.restype = res
                fn.argtypes = args
            _lib = L
    return _lib


def _check(status: int, ctx=None, what: str = ""):
    if status != VR_OK:
        L = lib()
        msg = L.vr_status_string(status).decode()
        if ctx is not None:
            detail = L.vr_last_error(ctx).decode()
            if detail:
                msg += ": " + detail
        raise VrError(status, "%s failed: %s" % (what, msg))


def _stream(stream):
    if stream is None:
        import torch
        if torch.cuda.is_available():
            return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
        return ctypes.c_void_p(0)
    if isinstance(stream, int):
        return ctypes.c_void_p(stream)
    return ctypes.c_void_p(stream.cuda_stream)


# The C side receives bare pointers and cannot check a buffer's size or type,
# so every array argument is checked here, before anything is launched: an
# undersized or mistyped buffer would otherwise be read or written out of
# bounds on the device. Image sizes come from the camera last set on a
# context (recorded per handle), volume shapes from vr_volume_create.
_cam_size = {}    # context handle -> (H, W)
_tf_len = {}      # context handle -> entries of the transfer function
_vol_shape = {}   # volume handle -> (Nz, Ny, Nx)
_frame_size = {}  # frame handle -> (H, W)


def _key(h):
    return h.value if isinstance(h, ctypes.c_void_p) else int(h)


def _array(x, what, shape=None, ndim=None, device=None, writable=False):
    """(pointer, on_device, keepalive) of a float32 C-contiguous tensor/array
    with the given shape (or number of dimensions); ValueError otherwise.
    device: True = must be CUDA, False = must be host, None = either."""
    try:
        import torch
        is_t = isinstance(x, torch.Tensor)
    except ImportError:
        is_t = False
    if is_t:
        dt_ok, contig, on_dev, shp = x.dtype == torch.float32, x.is_contiguous(), bool(x.is_cuda), tuple(x.shape)
    elif isinstance(x, np.ndarray):
        dt_ok, contig, on_dev, shp = x.dtype == np.float32, x.flags.c_contiguous, False, x.shape
        if writable and not x.flags.writeable:
            raise ValueError("%s must be writable" % what)
    else:
        raise ValueError("%s must be a torch tensor or numpy array" % what)
    if not dt_ok:
        raise ValueError("%s must be float32, got %s" % (what, x.dtype))
    if ndim is not None and len(shp) != ndim:
        raise ValueError("%s must have %d dimensions, got shape %s" % (what, ndim, shp))
    if shape is not None and shp != tuple(shape):
        raise ValueError("%s must have shape %s, got %s" % (what, tuple(shape), shp))
    if not contig:
        raise ValueError("%s must be contiguous" % what)
    if device is True and not on_dev:
        raise ValueError("%s must be a CUDA tensor" % what)
    if device is False and on_dev:
        raise ValueError("%s must be in host memory" % what)
    if on_dev:
        import torch
        if x.device.index != torch.cuda.current_device():
            raise ValueError("%s is on cuda:%d, not on the current device" % (what, x.device.index))
    return (x.data_ptr() if is_t else x.ctypes.data), int(on_dev), x


def _camera_size(ctx):
    size = _cam_size.get(_key(ctx))
    if size is None:  # the library's own answer to a render without a camera
        raise VrError(VR_ERR_STATE, "no camera set on this context")
    return size


def _image_of(ctx, out, what="out"):
    return _array(out, what, shape=_camera_size(ctx) + (4,), writable=True)


# --------------------------------------------------------------------------
# Calls (same names as the C ABI)
# --------------------------------------------------------------------------


def vr_create(cuda_device: int = 0):
    h = ctypes.c_void_p()
    _check(lib().vr_create(int(cuda_device), ctypes.byref(h)), None, "vr_create")
    return h


def vr_destroy(ctx):
    _check(lib().vr_destroy(ctx), ctx, "vr_destroy")
    _cam_size.pop(_key(ctx), None)
    _tf_len.pop(_key(ctx), None)


def vr_sync(ctx, stream=None):
    _check(lib().vr_sync(ctx, _stream(stream)), ctx, "vr_sync")


def make_partition(kind: str = "grid", grid=(1, 1, 1), n_bricks: int = 1, cut_fracs=None,
                   boxes=None):
    """Returns (vr_partition, keepalive)."""
    p = vr_partition()
    keep = []
    if kind == "grid":
        p.kind = VR_PART_GRID
        p.grid[:] = [int(g) for g in grid]
    elif kind == "kd":
        p.kind = VR_PART_KD
        p.n_bricks = int(n_bricks)
        u = np.ascontiguousarray(cut_fracs if cut_fracs is not None else [], dtype=np.float64)
        keep.append(u)
        p.cut_fracs = u.ctypes.data if u.size else None
    elif kind == "boxes":
        p.kind = VR_PART_BOXES
        b = np.ascontiguousarray(boxes, dtype=np.int32).reshape(-1, 6)
        keep.append(b)
        p.n_bricks = b.shape[0]
        p.boxes = b.ctypes.data
    else:
        raise ValueError(kind)
    return p, keep


def vr_partition_boxes(dims, partition=None):
    """Host-only: (n, 6) voxel boxes of a partition description for dims (x, y, z)."""
    d = (ctypes.c_int * 3)(*[int(v) for v in dims])
    part, keep = make_partition(**(partition or {}))
    n = ctypes.c_int()
    _check(lib().vr_partition_boxes(d, ctypes.byref(part), ctypes.byref(n), None), None,
           "vr_partition_boxes")
    boxes = np.zeros((n.value, 6), np.int32)
    _check(lib().vr_partition_boxes(d, ctypes.byref(part), None, boxes.ctypes.data), None,
           "vr_partition_boxes")
    return boxes


def vr_plan_view(dims, partition, cam: dict):
    """Host-only: (order (n,), rects (n, 4)) of a partitioned volume for a camera."""
    boxes = vr_partition_boxes(dims, partition)
    d = (ctypes.c_int * 3)(*[int(v) for v in dims])
    part, keep = make_partition(**(partition or {}))
    c = camera_struct(cam)
    order = np.zeros(boxes.shape[0], np.int32)
    rects = np.zeros((boxes.shape[0], 4), np.int32)
    _check(lib().vr_plan_view(d, ctypes.byref(part), ctypes.byref(c), order.ctypes.data,
                              rects.ctypes.data), None, "vr_plan_view")
    return order, rects


def vr_volume_create(ctx, volume, storage: str = "f32", partition=None, stream=None):
    """volume: [Nz, Ny, Nx] float32 (numpy / torch, host or CUDA).
    partition: dict for make_partition (default: one brick)."""
    ptr, on_dev, keep = _array(volume, "volume", ndim=3)
    nz, ny, nx = tuple(keep.shape)
    dims = (ctypes.c_int * 3)(nx, ny, nz)
    part, pk = make_partition(**(partition or {}))
    h = ctypes.c_void_p()
    _check(lib().vr_volume_create(ctx, dims, DTYPES[storage], ctypes.byref(part), ptr, on_dev,
                                  _stream(stream), ctypes.byref(h)), ctx, "vr_volume_create")
    _vol_shape[_key(h)] = (nz, ny, nx)
    return h


def vr_volume_create_share(ctx, volume, held, storage: str = "f32", partition=None, stream=None):
    """A rank's share: only the bricks in `held` (brick ids of the partition)
    are stored and marched; the others render as empty partials."""
    ptr, on_dev, keep = _array(volume, "volume", ndim=3)
    nz, ny, nx = tuple(keep.shape)
    dims = (ctypes.c_int * 3)(nx, ny, nz)
    part, pk = make_partition(**(partition or {}))
    ids = np.ascontiguousarray(list(held), dtype=np.int32)
    h = ctypes.c_void_p()
    _check(lib().vr_volume_create_share(ctx, dims, DTYPES[storage], ctypes.byref(part), int(ids.size),
                                        ids.ctypes.data, ptr, on_dev, _stream(stream), ctypes.byref(h)), ctx,
           "vr_volume_create_share")
    _vol_shape[_key(h)] = (nz, ny, nx)
    return h


def vr_composite_images(ctx, images, out, stream=None):
    """out = images[0] over images[1] over ... (front to back), pixel by pixel;
    CUDA float32 tensors of one shape [..., 4]. out may be images[0]."""
    if not images:
        raise ValueError("at least one image")
    shape = tuple(images[0].shape)
    if len(shape) < 1 or shape[-1] != 4:
        raise ValueError("images are [..., 4] RGBA")
    ptrs = [_array(im, "image", shape=shape, device=True)[0] for im in images]
    optr, _, _ = _array(out, "out", shape=shape, device=True, writable=True)
    arr = (ctypes.c_void_p * len(ptrs))(*ptrs)
    pixels = int(np.prod(shape[:-1]))
    _check(lib().vr_composite_images(ctx, len(ptrs), arr, optr, pixels, _stream(stream)), ctx,
           "vr_composite_images")


def vr_batch_create(ctx, vols, cams, out, vmins=None, vmaxs=None):
    """Batch of len(vols) x len(cams) renders into `out` ([n_vols * n_views, H, W, 4]
    CUDA float32; render r = v * n_views + w)."""
    nv = len(vols)
    vh = (ctypes.c_void_p * nv)(*[v.value for v in vols])
    cs = (vr_camera * len(cams))(*[camera_struct(c) for c in cams])
    lo = np.ascontiguousarray(vmins, dtype=np.float32) if vmins is not None else None
    hi = np.ascontiguousarray(vmaxs, dtype=np.float32) if vmaxs is not None else None
    if (lo is not None and lo.size != nv) or (hi is not None and hi.size != nv):
        raise ValueError("one vmin and one vmax per volume")
    H, W = int(cams[0]["height"]), int(cams[0]["width"])
    optr, oon, _ = _array(out, "out", shape=(nv * len(cams), H, W, 4), device=True)
    h = ctypes.c_void_p()
    _check(lib().vr_batch_create(ctx, nv, vh, lo.ctypes.data if lo is not None else None,
                                 hi.ctypes.data if hi is not None else None, len(cams), cs, optr,
                                 ctypes.byref(h)), ctx, "vr_batch_create")
    return h


def vr_batch_launch(batch, stream=None):
    _check(lib().vr_batch_launch(batch, _stream(stream)), None, "vr_batch_launch")


def vr_batch_autotune(batch, cache_path=None, stream=None):
    """Returns (packet width, blocks per SM, ring slots, work order) of the fastest candidate."""
    chosen = (ctypes.c_int * 4)()
    _check(lib().vr_batch_autotune(batch, _stream(stream), cache_path.encode() if cache_path else None,
                                   chosen), None, "vr_batch_autotune")
    return tuple(chosen)


def vr_batch_configure(batch, packet_width: int = 8, blocks_per_sm: int = 0, order: int = 0):
    _check(lib().vr_batch_configure(batch, int(packet_width), int(blocks_per_sm), int(order)), None,
           "vr_batch_configure")


def vr_batch_debug_wait(batch, wait_limit: int = 0, extra_march: int = 0):
    """Test hook: bounded waits give up after wait_limit sleeps (0: default), and
    unit 0's composite waits for extra_march more march items than exist."""
    _check(lib().vr_batch_debug_wait(batch, int(wait_limit), int(extra_march)), None, "vr_batch_debug_wait")


def vr_batch_release(batch):
    _check(lib().vr_batch_release(batch), None, "vr_batch_release")


def vr_volume_update(vol, volume, stream=None):
    """Re-pack `vol` from a float32 [Nz, Ny, Nx] array (same dims)."""
    ptr, on_dev, keep = _array(volume, "volume", shape=_vol_shape.get(_key(vol)), ndim=3)
    _check(lib().vr_volume_update(vol, ptr, on_dev, _stream(stream)), None, "vr_volume_update")


def vr_volume_update_async(vol, volume, stream=None):
    """Asynchronous re-pack on `stream` (host sources should be pinned)."""
    ptr, on_dev, keep = _array(volume, "volume", shape=_vol_shape.get(_key(vol)), ndim=3)
    _check(lib().vr_volume_update_async(vol, ptr, on_dev, _stream(stream)), None, "vr_volume_update_async")


def vr_render_backward(ctx, vol, grad_rgba, grad_tf, grad_density=None, stream=None):
    """Adds dL/d(table) to grad_tf and dL/d(voxels) to grad_density (CUDA float32
    tensors) for dL/dI = grad_rgba ([H, W, 4] CUDA float32)."""
    size = _camera_size(ctx)
    g, _, _ = _array(grad_rgba, "grad_rgba", shape=size + (4,), device=True)
    t, _, _ = _array(grad_tf, "grad_tf", shape=(_tf_len.get(_key(ctx), -1), 4), device=True)
    d = None
    if grad_density is not None:
        d, _, _ = _array(grad_density, "grad_density", shape=_vol_shape.get(_key(vol)), ndim=3, device=True)
    _check(lib().vr_render_backward(ctx, vol, g, t, d, _stream(stream)), ctx, "vr_render_backward")


def vr_volume_release(vol):
    _check(lib().vr_volume_release(vol), None, "vr_volume_release")
    _vol_shape.pop(_key(vol), None)


def vr_volume_info(vol):
    n = ctypes.c_int()
    _check(lib().vr_volume_info(vol, ctypes.byref(n), None, None), None, "vr_volume_info")
    boxes = np.zeros((n.value, 6), np.int32)
    nbytes = ctypes.c_longlong()
    _check(lib().vr_volume_info(vol, None, boxes.ctypes.data, ctypes.byref(nbytes)), None,
           "vr_volume_info")
    return boxes, int(nbytes.value)


def vr_volume_read_brick(vol, brick: int, storage: str = "f32"):
    boxes, _ = vr_volume_info(vol)
    b = boxes[brick]
    shape = (b[5] - b[2] + 2, b[4] - b[1] + 2, b[3] - b[0] + 2)
    out = np.zeros(shape, np.float32 if storage == "f32" else np.uint16)
    _check(lib().vr_volume_read_brick(vol, int(brick), out.ctypes.data, out.nbytes), None,
           "vr_volume_read_brick")
    return out


def vr_set_transfer_function(ctx, rgba, vmin: float, vmax: float):
    if isinstance(rgba, np.ndarray) or not hasattr(rgba, "data_ptr"):
        rgba = np.ascontiguousarray(rgba, dtype=np.float32)
    ptr, on_dev, keep = _array(rgba, "transfer function", ndim=2)
    if keep.shape[1] != 4:
        raise ValueError("transfer function must be (n, 4) RGBA")
    n = int(keep.shape[0])
    _check(lib().vr_set_transfer_function(ctx, ptr, n, float(vmin), float(vmax), on_dev), ctx,
           "vr_set_transfer_function")
    _tf_len[_key(ctx)] = n


def camera_struct(cam: dict) -> vr_camera:
    c = vr_camera()
    c.ortho = int(cam["ortho"])
    for k in ("eye", "dir", "up"):
        getattr(c, k)[:] = [float(v) for v in cam[k]]
    c.fovy_deg = float(cam.get("fovy_deg", 0.0))
    c.ortho_w = float(cam.get("ortho_w", 0.0))
    c.ortho_h = float(cam.get("ortho_h", 0.0))
    c.width = int(cam["width"])
    c.height = int(cam["height"])
    return c


def vr_set_camera(ctx, cam: dict):
    c = camera_struct(cam)
    _check(lib().vr_set_camera(ctx, ctypes.byref(c)), ctx, "vr_set_camera")
    _cam_size[_key(ctx)] = (c.height, c.width)


def vr_set_render_params(ctx, step_voxels: float = 0.5, ert_alpha: float = 1.0):
    _check(lib().vr_set_render_params(ctx, float(step_voxels), float(ert_alpha)), ctx,
           "vr_set_render_params")


def vr_set_composite_schedule(ctx, factors=()):
    f = np.ascontiguousarray(list(factors), dtype=np.int32)
    _check(lib().vr_set_composite_schedule(ctx, int(f.size), f.ctypes.data if f.size else None),
           ctx, "vr_set_composite_schedule")


def vr_set_opacity_correction(ctx, ref_step_voxels: float):
    """alpha' = 1 - (1 - alpha)^(step / ref_step) per sample; 0 turns it off."""
    _check(lib().vr_set_opacity_correction(ctx, float(ref_step_voxels)), ctx, "vr_set_opacity_correction")


def vr_set_host_output_async(ctx, on: bool):
    """Host outputs return at once; images land in host memory by vr_sync."""
    _check(lib().vr_set_host_output_async(ctx, int(bool(on))), ctx, "vr_set_host_output_async")


def vr_set_packet_width(ctx, packet_width: int):
    """Warp ray packet packet_width x (32/packet_width) pixels (4, 8 or 16)."""
    _check(lib().vr_set_packet_width(ctx, int(packet_width)), ctx, "vr_set_packet_width")


def vr_set_march_staging(ctx, on: bool):
    """Float32 volumes created afterwards keep a scalar brick copy and march with
    brick slabs staged in shared memory (same image, different speed)."""
    _check(lib().vr_set_march_staging(ctx, int(bool(on))), ctx, "vr_set_march_staging")


def vr_set_frame_pipelining(ctx, on: bool):
    """Consecutive vr_render_frame calls into device memory overlap (the next
    march starts in the previous frame's tail); same images. On by default."""
    _check(lib().vr_set_frame_pipelining(ctx, int(bool(on))), ctx, "vr_set_frame_pipelining")


def vr_debug_pipeline_gap(ctx):
    """Test hook: the next pipelined frame's bounded pool wait runs out."""
    _check(lib().vr_debug_pipeline_gap(ctx), ctx, "vr_debug_pipeline_gap")


def vr_set_cell_layout(ctx, layout: int):
    """16-bit volumes created afterwards: 0 xy-quads (default), 1 octets (both
    planes of a cell per element: one load per sample, twice the memory)."""
    _check(lib().vr_set_cell_layout(ctx, int(layout)), ctx, "vr_set_cell_layout")


def vr_set_render_mode(ctx, mode: int):
    """0: sort-last partials + composite (default); 1: ray-state cycling."""
    _check(lib().vr_set_render_mode(ctx, int(mode)), ctx, "vr_set_render_mode")


def vr_set_count_samples(ctx, on: bool):
    _check(lib().vr_set_count_samples(ctx, int(bool(on))), ctx, "vr_set_count_samples")


def vr_get_sample_count(ctx) -> int:
    v = ctypes.c_longlong()
    _check(lib().vr_get_sample_count(ctx, ctypes.byref(v)), ctx, "vr_get_sample_count")
    return int(v.value)


VR_FAULT_NONE, VR_FAULT_ALLOC, VR_FAULT_LAUNCH = 0, 1, 2


def vr_debug_inject_fault(kind: int, after: int = 0):
    """One-shot, process-wide: the device allocation (VR_FAULT_ALLOC) or kernel
    launch (VR_FAULT_LAUNCH) after `after` successful ones fails on the host."""
    _check(lib().vr_debug_inject_fault(int(kind), int(after)), None, "vr_debug_inject_fault")


def vr_set_kernel_timing(ctx, on: bool):
    _check(lib().vr_set_kernel_timing(ctx, int(bool(on))), ctx, "vr_set_kernel_timing")


def vr_get_kernel_timing(ctx):
    """dict(march_ms, march_launches, composite_ms, composite_launches) since the last call."""
    a, c = ctypes.c_double(), ctypes.c_double()
    na, nc = ctypes.c_longlong(), ctypes.c_longlong()
    _check(lib().vr_get_kernel_timing(ctx, ctypes.byref(a), ctypes.byref(na), ctypes.byref(c),
                                      ctypes.byref(nc)), ctx, "vr_get_kernel_timing")
    return dict(march_ms=a.value, march_launches=na.value, composite_ms=c.value,
                composite_launches=nc.value)


def vr_render_partials(ctx, vol, stream=None):
    h = ctypes.c_void_p()
    _check(lib().vr_render_partials(ctx, vol, ctypes.byref(h), _stream(stream)), ctx,
           "vr_render_partials")
    _frame_size[_key(h)] = _cam_size[_key(ctx)]
    return h


def vr_frame_info(frame):
    n = ctypes.c_int()
    _check(lib().vr_frame_info(frame, ctypes.byref(n), None, None), None, "vr_frame_info")
    rects = np.zeros((n.value, 4), np.int32)
    order = np.zeros(n.value, np.int32)
    _check(lib().vr_frame_info(frame, None, rects.ctypes.data, order.ctypes.data), None,
           "vr_frame_info")
    return rects, order


def vr_frame_partial(frame, brick: int):
    """Device pointer (int) of brick's partial: rect h rows x w float4."""
    p = ctypes.c_void_p()
    _check(lib().vr_frame_partial(frame, int(brick), ctypes.byref(p)), None, "vr_frame_partial")
    return int(p.value or 0)


def vr_composite(ctx, frame, out, stream=None):
    size = _frame_size.get(_key(frame))
    if size is None:
        raise VrError(VR_ERR_ARG, "unknown frame")
    ptr, on_dev, _ = _array(out, "out", shape=size + (4,), writable=True)
    _check(lib().vr_composite(ctx, frame, ptr, on_dev, _stream(stream)), ctx, "vr_composite")


def vr_frame_release(frame):
    _check(lib().vr_frame_release(frame), None, "vr_frame_release")
    _frame_size.pop(_key(frame), None)


def vr_render_frame(ctx, vol, out, stream=None):
    ptr, on_dev, _ = _image_of(ctx, out)
    _check(lib().vr_render_frame(ctx, vol, ptr, on_dev, _stream(stream)), ctx, "vr_render_frame")


def vr_mesh_create(ctx, verts, values, tets, dims, partition=None):
    """Tetrahedral-mesh volume from host arrays: verts (nv, 3) float32 world
    positions, values (nv,) float32, tets (nt, 4) int32; dims the nominal
    lattice (Nx, Ny, Nz); partition as for vr_volume_create."""
    v = np.ascontiguousarray(verts, dtype=np.float32).reshape(-1, 3)
    s = np.ascontiguousarray(values, dtype=np.float32).ravel()
    t = np.ascontiguousarray(tets, dtype=np.int32).reshape(-1, 4)
    if s.size != v.shape[0]:
        raise ValueError("one value per vertex")
    d = (ctypes.c_int * 3)(*[int(x) for x in dims])
    part, keep = make_partition(**(partition or {}))
    h = ctypes.c_void_p()
    _check(lib().vr_mesh_create(ctx, d, ctypes.byref(part), v.ctypes.data, v.shape[0], s.ctypes.data,
                                t.ctypes.data, t.shape[0], ctypes.byref(h)), ctx, "vr_mesh_create")
    return h


def vr_mesh_release(mesh):
    _check(lib().vr_mesh_release(mesh), None, "vr_mesh_release")


def vr_mesh_info(mesh):
    """(elements per brick (n,) int64, device bytes)."""
    n = ctypes.c_int()
    _check(lib().vr_mesh_info(mesh, ctypes.byref(n), None, None), None, "vr_mesh_info")
    cnt = np.zeros(n.value, np.int64)
    nbytes = ctypes.c_longlong()
    _check(lib().vr_mesh_info(mesh, None, cnt.ctypes.data, ctypes.byref(nbytes)), None, "vr_mesh_info")
    return cnt, int(nbytes.value)


def vr_render_mesh_frame(ctx, mesh, out, stream=None):
    ptr, on_dev, _ = _image_of(ctx, out)
    _check(lib().vr_render_mesh_frame(ctx, mesh, ptr, on_dev, _stream(stream)), ctx, "vr_render_mesh_frame")


def vr_render_frame_noalloc(volume, partition, tf, vmin: float, vmax: float, cam: dict, out,
                            step_voxels: float = 0.5, ert_alpha: float = 1.0, stream=None):
    """Frame without device allocation: `volume` and `out` are caller-owned CUDA
    tensors ([Nz, Ny, Nx] and [H, W, 4] float32); scratch is the library's static
    device array (see include/vr.h)."""
    vptr, von, vk = _array(volume, "volume", ndim=3)
    optr, oon, _ = _array(out, "out", shape=(int(cam["height"]), int(cam["width"]), 4), writable=True)
    if not (von and oon):
        raise ValueError("volume and out must be CUDA tensors")
    nz, ny, nx = tuple(vk.shape)
    dims = (ctypes.c_int * 3)(nx, ny, nz)
    part, keep = make_partition(**(partition or {}))
    t = np.ascontiguousarray(tf, dtype=np.float32).reshape(-1, 4)
    c = camera_struct(cam)
    _check(lib().vr_render_frame_noalloc(vptr, dims, ctypes.byref(part), t.ctypes.data, int(t.shape[0]),
                                         float(vmin), float(vmax), ctypes.byref(c), float(step_voxels),
                                         float(ert_alpha), optr, _stream(stream)), None,
           "vr_render_frame_noalloc")


# --------------------------------------------------------------------------
# Convenience: torch views of a frame's partials (tests, debugging)
# --------------------------------------------------------------------------


def frame_partials_torch(frame):
    """List of [h, w, 4] CUDA tensors (copies) of each brick's partial."""
    import torch
    rects, _ = vr_frame_info(frame)
    out = []
    for b, (x0, y0, w, h) in enumerate(rects):
        if w * h == 0:
            out.append(torch.zeros((int(h), int(w), 4), dtype=torch.float32, device="cuda"))
            continue
        view = _tensor_from_ptr(vr_frame_partial(frame, b), int(w * h * 4))
        out.append(view.clone().reshape(int(h), int(w), 4))
    return out


class _CudaArray:
    def __init__(self, ptr: int, n: int):
        self.__cuda_array_interface__ = dict(shape=(n,), typestr="<f4", data=(ptr, False),
                                             version=3, strides=None, stream=None)


def _tensor_from_ptr(ptr: int, n: int):
    """float32 CUDA tensor view of n elements at a device address owned by libvr."""
    import torch
    return torch.as_tensor(_CudaArray(ptr, n), device="cuda")
