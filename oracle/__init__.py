"""FP64 CPU oracle for the volume rendering path -- TEST INFRASTRUCTURE ONLY.

Only the test-suite, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package. The product library never links, loads
or calls it, and it imports nothing from the product package.

``vr_oracle.c`` holds the arithmetic (each function cites the passage or the
reading it follows); this module compiles it with gcc and marshals arguments.

Parity pins (checked in ``tests/test_oracle_pins.py``):
  P1 constant slab: A = 1-(1-a)^n, C = rgb (1-(1-a)^n) (closed form)
  P2 one brick equals the unsplit volume (special case)
  P3 brute-force O(n^2) product per pixel on 8x8 images (brute force)
  P4 any kd/grid/box split composited in ray order equals the unsplit render
  P5 exact trilinear weights on the axis-aligned 64^3 / 256^2 lattice with a
     linear ramp volume (closed form)
  P6 range / alpha-0 / alpha-1 / identity invariants
  16-bit storage: every f16 / bf16 code decodes to its IEEE-754 value
  (numpy float16; float32 with the code in the top half)
  cameras: pixel rays meet the image plane on square cells on non-square
  images (fixes the W/H aspect factor of the perspective rays)
Mesh pins (``tests/test_oracle_mesh.py``): linear fields reproduced exactly,
barycentric partition of unity and containment, bins equal brute force, mesh
renders equal the pinned voxel renders on rays along shared grid lines, the
constant-slab closed form, and brick-split associativity.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "vr_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None

F32, BF16, F16, F64 = 0, 1, 2, 3


def build(force: bool = False) -> str:
    """Compile vr_oracle.c with gcc (-O2, no FP contraction, OpenMP)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + ".tmp%d" % os.getpid()
        cmd = ["gcc", "-O2", "-fPIC", "-shared", "-fopenmp", "-ffp-contract=off",
               "-fno-fast-math", "-std=gnu11", "-o", tmp, _SRC, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _LIB)
    return _LIB


class _Camera(ctypes.Structure):
    _fields_ = [("ortho", ctypes.c_int), ("eye", ctypes.c_double * 3),
                ("dir", ctypes.c_double * 3), ("up", ctypes.c_double * 3),
                ("fovy_deg", ctypes.c_double), ("ortho_w", ctypes.c_double),
                ("ortho_h", ctypes.c_double), ("width", ctypes.c_int),
                ("height", ctypes.c_int)]


class _Scene(ctypes.Structure):
    _fields_ = [("vol", ctypes.c_void_p), ("dtype", ctypes.c_int),
                ("dims", ctypes.c_int * 3), ("nb", ctypes.c_int),
                ("boxes", ctypes.c_void_p), ("tf", ctypes.c_void_p),
                ("ntf", ctypes.c_int), ("vmin", ctypes.c_double),
                ("vmax", ctypes.c_double), ("cam", _Camera),
                ("step_voxels", ctypes.c_double), ("ert_alpha", ctypes.c_double),
                ("ert_bias", ctypes.c_double), ("end_bias", ctypes.c_double),
                ("tf64", ctypes.c_void_p), ("ert_global", ctypes.c_int),
                ("opc_ratio", ctypes.c_double), ("mesh_verts", ctypes.c_void_p),
                ("mesh_vals", ctypes.c_void_p), ("mesh_tets", ctypes.c_void_p),
                ("mesh_nt", ctypes.c_longlong), ("mesh_nv", ctypes.c_int),
                ("mesh_bruteforce", ctypes.c_int)]


class Mesh:
    """Tetrahedral-mesh input in place of a voxel volume.

    verts (nv, 3) world positions, vals (nv,) vertex values, tets (nt, 4)
    vertex indices, dims the nominal lattice (Nx, Ny, Nz) that fixes the domain
    box [0, dims/Nmax], the lattice spacing and the ownership cells. float32
    inputs are converted to double exactly."""

    def __init__(self, verts, vals, tets, dims, bruteforce: bool = False):
        self.verts = np.ascontiguousarray(np.asarray(verts, dtype=np.float64).reshape(-1, 3))
        self.vals = np.ascontiguousarray(np.asarray(vals, dtype=np.float64).ravel())
        self.tets = np.ascontiguousarray(np.asarray(tets, dtype=np.int32).reshape(-1, 4))
        self.dims = tuple(int(d) for d in dims)
        self.bruteforce = bool(bruteforce)
        if self.vals.size != self.verts.shape[0]:
            raise ValueError("one value per vertex")


def lib():
    global _lib
    with _lock:
        if _lib is None:
            _lib = ctypes.CDLL(build())
            _lib.orc_render_pixels.argtypes = [ctypes.POINTER(_Scene), ctypes.c_int,
                                               ctypes.c_void_p, ctypes.c_void_p,
                                               ctypes.c_void_p, ctypes.POINTER(ctypes.c_longlong),
                                               ctypes.c_int]
            _lib.orc_render_pixels.restype = ctypes.c_int
            _lib.orc_grid_partition.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]
            _lib.orc_kd_partition.argtypes = [ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p,
                                              ctypes.c_void_p]
            _lib.orc_render_grad.argtypes = [ctypes.POINTER(_Scene), ctypes.c_int, ctypes.c_void_p,
                                             ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                             ctypes.c_int]
            _lib.orc_render_grad.restype = ctypes.c_int
            _lib.orc_sample.argtypes = [ctypes.POINTER(_Scene), ctypes.c_void_p]
            _lib.orc_sample.restype = ctypes.c_double
            _lib.orc_classify.argtypes = [ctypes.POINTER(_Scene), ctypes.c_double, ctypes.c_void_p]
            _lib.orc_primary_ray.argtypes = [ctypes.POINTER(_Camera), ctypes.c_int, ctypes.c_int,
                                             ctypes.c_void_p, ctypes.c_void_p]
            _lib.orc_mesh_sample.argtypes = [ctypes.POINTER(_Scene), ctypes.c_int, ctypes.c_void_p,
                                             ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                             ctypes.c_void_p]
            _lib.orc_mesh_sample.restype = ctypes.c_int
    return _lib


def _camera(cam: dict) -> _Camera:
    c = _Camera()
    c.ortho = int(cam["ortho"])
    for k in ("eye", "dir", "up"):
        getattr(c, k)[:] = [float(v) for v in cam[k]]
    c.fovy_deg = float(cam.get("fovy_deg", 0.0))
    c.ortho_w = float(cam.get("ortho_w", 0.0))
    c.ortho_h = float(cam.get("ortho_h", 0.0))
    c.width = int(cam["width"])
    c.height = int(cam["height"])
    return c


def grid_partition(dims, g) -> np.ndarray:
    """Regular g[0] x g[1] x g[2] split, boundaries floor(N j / g)."""
    d = np.ascontiguousarray(dims, dtype=np.int32)
    gg = np.ascontiguousarray(g, dtype=np.int32)
    out = np.zeros((int(np.prod(gg)), 6), dtype=np.int32)
    rc = lib().orc_grid_partition(d.ctypes.data, gg.ctypes.data, out.ctypes.data)
    if rc != 0:
        raise ValueError("grid partition rejected (%d)" % rc)
    return out


def kd_partition(dims, n: int, fracs) -> np.ndarray:
    """kd split into n leaves from n-1 cut fractions (largest leaf first,
    longest axis, cut at lo + round(u * extent))."""
    d = np.ascontiguousarray(dims, dtype=np.int32)
    u = np.ascontiguousarray(fracs, dtype=np.float64)
    if u.size < n - 1:
        raise ValueError("need n-1 cut fractions")
    out = np.zeros((n, 6), dtype=np.int32)
    rc = lib().orc_kd_partition(d.ctypes.data, int(n), u.ctypes.data, out.ctypes.data)
    if rc != 0:
        raise ValueError("kd partition rejected (%d)" % rc)
    return out


def _dtype_code(vol: np.ndarray, dtype):
    if dtype is not None:
        return dtype
    if vol.dtype == np.float32:
        return F32
    if vol.dtype == np.float64:
        return F64
    raise ValueError("16-bit volumes need an explicit dtype code (BF16 or F16)")


def _scene(vol, boxes, tf, vmin, vmax, cam, step_voxels, ert_alpha, dtype, keep):
    mesh = vol if isinstance(vol, Mesh) else None
    if mesh is not None:
        keep.append(mesh)
        vol = np.zeros((1, 1, 1), np.float32)
    vol = np.ascontiguousarray(vol)
    code = _dtype_code(vol, dtype)
    boxes = np.ascontiguousarray(boxes, dtype=np.int32).reshape(-1, 6)
    tf_in = np.asarray(tf)
    tf64 = None
    if tf_in.dtype == np.float64:  # exact table (finite-difference probes)
        tf64 = np.ascontiguousarray(tf_in).reshape(-1, 4)
    tf = np.ascontiguousarray(tf_in, dtype=np.float32).reshape(-1, 4)
    keep.extend([vol, boxes, tf, tf64])
    sc = _Scene()
    sc.vol = vol.ctypes.data
    sc.dtype = code
    sc.dims[:] = [vol.shape[2], vol.shape[1], vol.shape[0]]
    sc.nb = boxes.shape[0]
    sc.boxes = boxes.ctypes.data
    sc.tf = tf.ctypes.data
    sc.ntf = tf.shape[0]
    sc.vmin, sc.vmax = float(vmin), float(vmax)
    sc.cam = _camera(cam)
    sc.step_voxels = float(step_voxels)
    sc.ert_alpha = float(ert_alpha)
    sc.tf64 = tf64.ctypes.data if tf64 is not None else None
    if mesh is not None:
        sc.dims[:] = list(mesh.dims)
        sc.mesh_verts = mesh.verts.ctypes.data
        sc.mesh_vals = mesh.vals.ctypes.data
        sc.mesh_tets = mesh.tets.ctypes.data
        sc.mesh_nt = mesh.tets.shape[0]
        sc.mesh_nv = mesh.verts.shape[0]
        sc.mesh_bruteforce = int(mesh.bruteforce)
    return sc


_DUMMY_CAM = dict(ortho=1, eye=(0, 0, 0), dir=(0, 0, 1), up=(0, 1, 0), width=1, height=1)


def sample(vol, points, dtype=None) -> np.ndarray:
    """Trilinear value at world points (m, 3)."""
    keep = []
    nz, ny, nx = np.asarray(vol).shape
    sc = _scene(vol, [[0, 0, 0, nx, ny, nz]], np.zeros((2, 4), np.float32), 0.0, 1.0,
                _DUMMY_CAM, 0.5, 1.0, dtype, keep)
    pts = np.ascontiguousarray(points, dtype=np.float64).reshape(-1, 3)
    return np.array([lib().orc_sample(ctypes.byref(sc), pts[i].ctypes.data)
                     for i in range(pts.shape[0])])


def mesh_sample(mesh: Mesh, boxes, points) -> dict:
    """Mesh value at world points (m, 3): per point the owner brick (cell rule),
    the value from that brick's elements, the chosen element and its smallest
    barycentric coordinate."""
    keep = []
    sc = _scene(mesh, boxes, np.zeros((2, 4), np.float32), 0.0, 1.0, _DUMMY_CAM, 0.5, 1.0, None, keep)
    pts = np.ascontiguousarray(points, dtype=np.float64).reshape(-1, 3)
    m = pts.shape[0]
    vals = np.zeros(m)
    elem = np.zeros(m, np.int64)
    minb = np.zeros(m)
    brick = np.zeros(m, np.int32)
    rc = lib().orc_mesh_sample(ctypes.byref(sc), m, pts.ctypes.data, vals.ctypes.data, elem.ctypes.data,
                               minb.ctypes.data, brick.ctypes.data)
    if rc != 0:
        raise RuntimeError("oracle mesh sample failed (%d)" % rc)
    return dict(vals=vals, elem=elem, minb=minb, brick=brick)


def classify(tf, vmin, vmax, values) -> np.ndarray:
    """RGBA of scalar values (m,) through the table."""
    keep = []
    sc = _scene(np.zeros((1, 1, 1), np.float32), [[0, 0, 0, 1, 1, 1]], tf, vmin, vmax,
                _DUMMY_CAM, 0.5, 1.0, None, keep)
    vals = np.asarray(values, dtype=np.float64).ravel()
    out = np.zeros((vals.size, 4))
    for i, v in enumerate(vals):
        lib().orc_classify(ctypes.byref(sc), float(v), out[i].ctypes.data)
    return out


def primary_ray(cam, px, py):
    c = _camera(cam)
    o = np.zeros(3)
    d = np.zeros(3)
    lib().orc_primary_ray(ctypes.byref(c), int(px), int(py), o.ctypes.data, d.ctypes.data)
    return o, d


def render(vol: np.ndarray, boxes, tf: np.ndarray, vmin: float, vmax: float, cam: dict,
           step_voxels: float = 0.5, ert_alpha: float = 1.0, pixels=None, crop=None,
           dtype=None, with_partials: bool = False, ert_bias: float = 0.0,
           end_bias: float = 0.0, threads: int | None = None, ert_global: bool = False,
           opacity_ref_step: float = 0.0):
    """Render pixels with the FP64 oracle.

    vol     [Nz, Ny, Nx] array (float32/float64, or uint16 bits with dtype BF16/F16),
            or a Mesh (tetrahedral elements)
    boxes   (nb, 6) int half-open voxel boxes (lo xyz, hi xyz)
    pixels  (m, 2) int (px, py) list, or crop = (x0, y0, w, h); default = full image
    Returns dict(img=(m,4) or (h,w,4), partials=(nb, ...,4) or None, nsamples=int).
    """
    keep = []
    sc = _scene(vol, boxes, tf, vmin, vmax, cam, step_voxels, ert_alpha, dtype, keep)
    sc.ert_bias = float(ert_bias)
    sc.end_bias = float(end_bias)
    sc.ert_global = int(bool(ert_global))
    sc.opc_ratio = float(step_voxels) / opacity_ref_step if opacity_ref_step > 0 else 0.0
    W, H = int(cam["width"]), int(cam["height"])
    shape = None
    if pixels is None:
        x0, y0, w, h = crop if crop is not None else (0, 0, W, H)
        ys, xs = np.mgrid[y0:y0 + h, x0:x0 + w]
        pixels = np.stack([xs.ravel(), ys.ravel()], axis=1)
        shape = (h, w)
    pix = np.ascontiguousarray(pixels, dtype=np.int32).reshape(-1, 2)
    m = pix.shape[0]
    img = np.zeros((m, 4), dtype=np.float64)
    parts = np.zeros((sc.nb, m, 4), dtype=np.float64) if with_partials else None
    ns = ctypes.c_longlong(0)
    nthreads = threads if threads is not None else (os.cpu_count() or 1)
    rc = lib().orc_render_pixels(ctypes.byref(sc), m, pix.ctypes.data, img.ctypes.data,
                                 parts.ctypes.data if parts is not None else None,
                                 ctypes.byref(ns), int(nthreads))
    if rc != 0:
        raise RuntimeError("oracle render failed (%d)" % rc)
    if shape is not None:
        img = img.reshape(shape + (4,))
        if parts is not None:
            parts = parts.reshape((sc.nb,) + shape + (4,))
    return dict(img=img, partials=parts, nsamples=int(ns.value))


def render_grad(vol, boxes, tf, vmin, vmax, cam, grad_img, step_voxels: float = 0.5, pixels=None,
                crop=None, dtype=None, want_volume: bool = True, threads: int | None = None):
    """Vector-Jacobian product of the rendered pixels: returns (dL/dT (ntf, 4),
    dL/dv (vol.shape) or None) for the upstream gradient grad_img (same shape as
    the rendered pixels, RGBA). Early termination is off."""
    keep = []
    sc = _scene(vol, boxes, tf, vmin, vmax, cam, step_voxels, 1.0, dtype, keep)
    W, H = int(cam["width"]), int(cam["height"])
    if pixels is None:
        x0, y0, w, h = crop if crop is not None else (0, 0, W, H)
        ys, xs = np.mgrid[y0:y0 + h, x0:x0 + w]
        pixels = np.stack([xs.ravel(), ys.ravel()], axis=1)
    pix = np.ascontiguousarray(pixels, dtype=np.int32).reshape(-1, 2)
    g = np.ascontiguousarray(grad_img, dtype=np.float64).reshape(-1, 4)
    if g.shape[0] != pix.shape[0]:
        raise ValueError("grad_img must hold one RGBA row per pixel")
    gtf = np.zeros((sc.ntf, 4), np.float64)
    gvol = np.zeros(np.asarray(vol).shape, np.float64) if want_volume else None
    nthreads = threads if threads is not None else (os.cpu_count() or 1)
    rc = lib().orc_render_grad(ctypes.byref(sc), pix.shape[0], pix.ctypes.data, g.ctypes.data,
                               gtf.ctypes.data, gvol.ctypes.data if gvol is not None else None,
                               int(nthreads))
    if rc != 0:
        raise RuntimeError("oracle gradient failed (%d)" % rc)
    return gtf, gvol


# Decision-ambiguity probes. A float decides two integers per ray: how many
# lattice samples lie before t_out, and after which sample a brick terminates
# early. FP32 and FP64 may take those decisions differently only when the
# deciding value is within rounding of its threshold; these widths cover FP32
# rounding of t (|t| < 4, ~1e-6) and of an accumulated transmittance (<1e-6).
TAU_T = 4e-6
TAU_TRANSMITTANCE = 4e-6


def render_with_envelope(vol, boxes, tf, vmin, vmax, cam, step_voxels=0.5, ert_alpha=1.0,
                         **kw):
    """Main render plus the two renders with every near-threshold decision taken
    the other way (early: stop sooner / drop the last sample; late: the reverse).
    Pixels where early != late carry an ambiguous decision."""
    main = render(vol, boxes, tf, vmin, vmax, cam, step_voxels, ert_alpha, **kw)
    kw.pop("with_partials", None)
    early = render(vol, boxes, tf, vmin, vmax, cam, step_voxels, ert_alpha,
                   ert_bias=TAU_TRANSMITTANCE, end_bias=-TAU_T, **kw)["img"]
    late = render(vol, boxes, tf, vmin, vmax, cam, step_voxels, ert_alpha,
                  ert_bias=-TAU_TRANSMITTANCE, end_bias=TAU_T, **kw)["img"]
    amb = np.any(early != late, axis=-1)
    lo = np.minimum(np.minimum(main["img"], early), late)
    hi = np.maximum(np.maximum(main["img"], early), late)
    main.update(ambiguous=amb, lo=lo, hi=hi)
    return main
