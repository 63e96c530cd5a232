"""Seeded synthetic inputs shared by the CUDA path's tests/bench and the oracle.

This module only *generates inputs*: scalar volumes, transfer-function tables,
camera descriptions and the random cut fractions of a kd partition. It holds
none of the rendering method's arithmetic (no ray generation, sampling,
classification, accumulation or compositing), so both sides consume identical
bytes without sharing any of the computation under test.

The paper (Sec. 4) renders the NASA Mars Lander mixed-element data set, which
is not available; these volumes stand in for it with the shapes, sizes and
partition structure of the workloads (Sec. 2.2: data spatially distributed
across ranks, possibly unevenly; Sec. 4: 36 GPUs, several parts per GPU).

Draw order is part of the contract: every generator takes a
``numpy.random.Generator`` (PCG64 via ``default_rng(seed)``) and documents
which draws it makes, in which order.
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np

# --------------------------------------------------------------------------
# Volumes (x fastest: array index [z, y, x])
# --------------------------------------------------------------------------


@dataclass(frozen=True)
class Blobs:
    centers: np.ndarray  # (n, 3) xyz in [0,1]^3 (world units of the unit cube)
    sigmas: np.ndarray   # (n,)
    amps: np.ndarray     # (n,)


def draw_blobs(rng: np.random.Generator, n: int) -> Blobs:
    """Draws, in order: n*3 centers U[0,1] (row-major, xyz per blob),
    n sigmas U[0.05, 0.15], n amplitudes U[0.2, 1.0]."""
    centers = rng.uniform(0.0, 1.0, size=(n, 3))
    sigmas = rng.uniform(0.05, 0.15, size=n)
    amps = rng.uniform(0.2, 1.0, size=n)
    return Blobs(centers, sigmas, amps)


def _voxel_centers(n: int) -> np.ndarray:
    return (np.arange(n, dtype=np.float64) + 0.5) / n


def blob_volume(n: int, blobs: Blobs, offset: np.ndarray | None = None,
                out: np.ndarray | None = None) -> np.ndarray:
    """Sum of isotropic Gaussians a*exp(-|x-mu|^2/(2 sigma^2)) evaluated at the
    voxel centres of an n^3 grid over [0,1]^3 (separable per axis, float64
    factors, accumulated into float32 in z slabs to bound host memory)."""
    x = _voxel_centers(n)
    if out is None:
        out = np.zeros((n, n, n), dtype=np.float32)
    centers = blobs.centers if offset is None else blobs.centers + offset
    for (cx, cy, cz), s, a in zip(centers, blobs.sigmas, blobs.amps):
        gx = np.exp(-((x - cx) ** 2) / (2 * s * s))
        gy = np.exp(-((x - cy) ** 2) / (2 * s * s))
        gz = a * np.exp(-((x - cz) ** 2) / (2 * s * s))
        plane = (gy[:, None] * gx[None, :]).astype(np.float32)
        gz32 = gz.astype(np.float32)
        step = max(1, (1 << 24) // (n * n))
        for z0 in range(0, n, step):
            z1 = min(n, z0 + step)
            out[z0:z1] += gz32[z0:z1, None, None] * plane[None, :, :]
    return out


def _lerp_axis(a: np.ndarray, n: int, cells: int, axis: int) -> np.ndarray:
    """Linear interpolation of lattice values along one axis onto the voxel
    centres of an n-voxel axis (lattice spacing 1/cells over [0,1])."""
    pos = _voxel_centers(n) * cells
    i0 = np.minimum(np.floor(pos).astype(np.int64), cells - 1)
    w = (pos - i0).astype(np.float32)
    a0 = np.take(a, i0, axis=axis)
    a1 = np.take(a, i0 + 1, axis=axis)
    shape = [1] * a.ndim
    shape[axis] = n
    w = w.reshape(shape)
    return a0 + w * (a1 - a0)


def value_noise(n: int, rng: np.random.Generator, octaves: int = 6) -> np.ndarray:
    """Fractal value noise normalised to [0,1].

    Octave o (o = 0..octaves-1) has 4*2^o lattice cells per unit; its
    (cells+1)^3 lattice values are drawn U[0,1] in octave order (array order
    [z,y,x]) and trilinearly upsampled to the voxel centres; octaves are summed
    with amplitude 0.5^o and the sum is min-max normalised."""
    acc = np.zeros((n, n, n), dtype=np.float32)
    for o in range(octaves):
        cells = 4 * (2 ** o)
        lat = rng.uniform(0.0, 1.0, size=(cells + 1,) * 3).astype(np.float32)
        a = _lerp_axis(lat, n, cells, 2)
        a = _lerp_axis(a, n, cells, 1)
        a = _lerp_axis(a, n, cells, 0)
        acc += np.float32(0.5 ** o) * a
        del a
    lo, hi = float(acc.min()), float(acc.max())
    acc -= np.float32(lo)
    acc *= np.float32(1.0 / (hi - lo))
    return acc


# --------------------------------------------------------------------------
# Transfer function tables
# --------------------------------------------------------------------------


def random_tf(rng: np.random.Generator, n_entries: int = 256, n_points: int = 4,
              alpha_max: float = 0.05) -> np.ndarray:
    """Piecewise-linear RGBA table of n_entries (entry i sits at u = i/(n-1)).

    Draws, in order: n_points positions U[0,1] (then sorted), n_points*3 rgb
    U[0,1] (row-major), n_points alphas U[0, alpha_max]. Control points are
    joined linearly; outside [x_0, x_last] the end values are held."""
    xs = np.sort(rng.uniform(0.0, 1.0, size=n_points))
    rgb = rng.uniform(0.0, 1.0, size=(n_points, 3))
    alpha = rng.uniform(0.0, alpha_max, size=n_points)
    ctrl = np.concatenate([rgb, alpha[:, None]], axis=1)
    u = np.arange(n_entries, dtype=np.float64) / (n_entries - 1)
    table = np.stack([np.interp(u, xs, ctrl[:, c]) for c in range(4)], axis=1)
    return table.astype(np.float32)


def ramp_tf(n_entries: int = 256, alpha_max: float = 0.05) -> np.ndarray:
    """Deterministic table whose opacity and colour change across the whole
    range (alpha = alpha_max*u, rgb = (u, 1-u, 1/2)): every change of the scalar
    shows in the image, which makes storage-precision effects visible."""
    u = np.arange(n_entries, dtype=np.float64) / (n_entries - 1)
    return np.stack([u, 1.0 - u, np.full_like(u, 0.5), alpha_max * u], axis=1).astype(np.float32)


def constant_tf(rgba, n_entries: int = 256) -> np.ndarray:
    return np.tile(np.asarray(rgba, dtype=np.float32)[None, :], (n_entries, 1))


# --------------------------------------------------------------------------
# Cameras (plain dicts; each side marshals them into its own struct)
# --------------------------------------------------------------------------


def ortho_camera_z(width: int, height: int, extent=(1.0, 1.0)) -> dict:
    """Orthographic camera looking along +z whose image plane covers the
    volume's xy extent exactly, placed on the z = 0 face."""
    return dict(ortho=1, eye=(extent[0] / 2, extent[1] / 2, 0.0), dir=(0.0, 0.0, 1.0),
                up=(0.0, 1.0, 0.0), fovy_deg=0.0, ortho_w=float(extent[0]),
                ortho_h=float(extent[1]), width=int(width), height=int(height))


def orbit_camera(width: int, height: int, azimuth_deg: float, radius: float = 1.8,
                 elevation_deg: float = 20.0, fovy_deg: float = 60.0,
                 center=(0.5, 0.5, 0.5)) -> dict:
    """Perspective camera on a circle around the volume centre, looking at it,
    +y up. azimuth 0 sits on the -z side looking towards +z."""
    el = math.radians(elevation_deg)
    az = math.radians(azimuth_deg)
    c = np.asarray(center, dtype=np.float64)
    eye = c + radius * np.array([math.cos(el) * math.sin(az), math.sin(el),
                                 -math.cos(el) * math.cos(az)])
    d = c - eye
    return dict(ortho=0, eye=tuple(eye), dir=tuple(d), up=(0.0, 1.0, 0.0),
                fovy_deg=float(fovy_deg), ortho_w=0.0, ortho_h=0.0,
                width=int(width), height=int(height))


ORBIT_AZIMUTHS = tuple(45.0 * i for i in range(8))


# --------------------------------------------------------------------------
# Partition randomness
# --------------------------------------------------------------------------


def kd_cut_fractions(rng: np.random.Generator, n_bricks: int, lo: float = 0.3,
                     hi: float = 0.7) -> np.ndarray:
    """n_bricks-1 cut fractions U[lo, hi], one per kd split in split order."""
    return rng.uniform(lo, hi, size=max(0, n_bricks - 1))


# --------------------------------------------------------------------------
# Workload recipes (sizes and seeds of the five benchmark workloads)
# --------------------------------------------------------------------------


def small_blob_scene(n: int = 64, seed: int = 0, n_blobs: int = 8):
    """64^3 blobs, 256-entry random TF (seed order: blobs then TF)."""
    rng = np.random.default_rng(seed)
    blobs = draw_blobs(rng, n_blobs)
    vol = blob_volume(n, blobs)
    tf = random_tf(rng)
    return vol, tf


def noise_blob_scene(n: int = 512, seed: int = 1, n_blobs: int = 16):
    """Value noise (6 octaves) + 16 blobs, then a random TF (seed order:
    noise lattices, blobs, TF)."""
    rng = np.random.default_rng(seed)
    vol = value_noise(n, rng)
    blobs = draw_blobs(rng, n_blobs)
    blob_volume(n, blobs, out=vol)
    tf = random_tf(rng)
    return vol, tf


def precision_scene(n: int = 1024, seed: int = 2, n_bricks: int = 64, n_blobs: int = 8):
    """Blob volume of the small workload's generator at n^3 plus its TF, then
    n_bricks-1 kd cut fractions U[0.3, 0.7] (seed order: blobs, TF, cuts)."""
    rng = np.random.default_rng(seed)
    blobs = draw_blobs(rng, n_blobs)
    vol = blob_volume(n, blobs)
    tf = random_tf(rng)
    cuts = kd_cut_fractions(rng, n_bricks)
    return vol, tf, cuts


def quantize(vol: np.ndarray, storage: str) -> np.ndarray:
    """Round-to-nearest-even bf16/f16 bits (uint16) of a float32 volume, as
    torch's CPU conversion produces them."""
    import torch
    t = torch.from_numpy(np.ascontiguousarray(vol, dtype=np.float32))
    t = t.to(torch.bfloat16 if storage == "bf16" else torch.float16)
    return t.view(torch.int16).numpy().view(np.uint16)


# --------------------------------------------------------------------------
# Time-varying multi-field data (batching workload), generated with torch on a
# chosen device because 18 x 768^3 volumes take minutes in numpy
# --------------------------------------------------------------------------


@dataclass(frozen=True)
class FieldDraws:
    blobs: Blobs
    velocity: np.ndarray   # (n_blobs, 3) per-step displacement
    lattice: np.ndarray    # (L+1)^3 noise lattice values U[0,1]


def draw_fields(seed: int = 3, n_fields: int = 3, n_blobs: int = 8, cells: int = 16):
    """Per field, draws in order: blobs (draw_blobs), n_blobs*3 velocities
    U[-0.05, 0.05], a (cells+1)^3 noise lattice U[0,1]."""
    rng = np.random.default_rng(seed)
    out = []
    for _ in range(n_fields):
        blobs = draw_blobs(rng, n_blobs)
        vel = rng.uniform(-0.05, 0.05, size=(n_blobs, 3))
        lat = rng.uniform(0.0, 1.0, size=(cells + 1,) * 3)
        out.append(FieldDraws(blobs, vel, lat))
    return out


def field_volume_torch(draws: FieldDraws, step: int, n: int, device="cuda", noise_amp: float = 0.05):
    """Field at time step `step`: the blobs moved by step * velocity, plus the
    field's lattice noise (trilinear at voxel centres, lattice spacing
    1/cells) times noise_amp. float32 [n, n, n] on `device`."""
    import torch
    x = (torch.arange(n, dtype=torch.float64, device=device) + 0.5) / n
    out = torch.zeros((n, n, n), dtype=torch.float32, device=device)
    for (cx, cy, cz), v, s_, a in zip(draws.blobs.centers, draws.velocity, draws.blobs.sigmas, draws.blobs.amps):
        cx, cy, cz = cx + step * v[0], cy + step * v[1], cz + step * v[2]
        gx = torch.exp(-((x - cx) ** 2) / (2 * s_ * s_))
        gy = torch.exp(-((x - cy) ** 2) / (2 * s_ * s_))
        gz = a * torch.exp(-((x - cz) ** 2) / (2 * s_ * s_))
        out += (gz[:, None, None] * gy[None, :, None] * gx[None, None, :]).float()
    cells = draws.lattice.shape[0] - 1
    lat = torch.from_numpy(draws.lattice).to(device=device, dtype=torch.float32)
    pos = x * cells
    i0 = torch.clamp(torch.floor(pos).long(), max=cells - 1)
    w = (pos - i0).float()
    for axis in (2, 1, 0):
        shape = [1, 1, 1]
        shape[axis] = n
        a0 = torch.index_select(lat, axis, i0)
        a1 = torch.index_select(lat, axis, i0 + 1)
        lat = a0 + w.reshape(shape) * (a1 - a0)
    out += noise_amp * lat
    return out


def volume_range(vol: np.ndarray):
    return float(vol.min()), float(vol.max())


# --------------------------------------------------------------------------
# Tetrahedral meshes (unstructured-element workloads). The paper's data set is
# a mixed finite-element mesh whose parts sit unevenly in space (Sec. 5); these
# meshes stand in for it: graded, jittered, conforming, each element inside
# one brick, so that every rank holds whole elements.
# --------------------------------------------------------------------------

# Kuhn split of a hexahedral cell into six tetrahedra: each follows a monotone
# corner path 000 -> e_a -> e_a + e_b -> 111 for one axis order (a, b, c). Both
# sides of a shared face split it along the same diagonal, so neighbouring
# cells conform.
_KUHN_ORDERS = ((0, 1, 2), (0, 2, 1), (1, 0, 2), (1, 2, 0), (2, 0, 1), (2, 1, 0))


def grid_tets(nx: int, ny: int, nz: int) -> np.ndarray:
    """Six Kuhn tetrahedra per cell of an nx x ny x nz node grid (node index
    (iz*ny + iy)*nx + ix), int32 (6 (nx-1)(ny-1)(nz-1), 4)."""
    cx, cy, cz = np.meshgrid(np.arange(nx - 1), np.arange(ny - 1), np.arange(nz - 1), indexing="ij")
    cx, cy, cz = cx.ravel(), cy.ravel(), cz.ravel()
    tets = []
    for order in _KUHN_ORDERS:
        corner = [cx.copy(), cy.copy(), cz.copy()]
        path = [(corner[2] * ny + corner[1]) * nx + corner[0]]
        for a in order:
            corner[a] = corner[a] + 1
            path.append((corner[2] * ny + corner[1]) * nx + corner[0])
        tets.append(np.stack(path, axis=1))
    return np.concatenate(tets, axis=0).astype(np.int32)


def _axis_nodes(cuts, cell_voxels: float, focus: float, refine: float, width: float, nmax: int):
    """Node coordinates (voxel units) along one axis and a flag per node that
    is a cut. Between consecutive cuts the nodes are uniform, about
    cell_voxels / (1 + refine * exp(-(x - focus)^2 / (2 width^2))) apart, x the
    interval's midpoint in world units."""
    xs, fixed = [float(cuts[0])], [True]
    for a, b in zip(cuts[:-1], cuts[1:]):
        mid = 0.5 * (a + b) / nmax
        h = cell_voxels / (1.0 + refine * math.exp(-((mid - focus) ** 2) / (2.0 * width * width)))
        m = max(1, int(round((b - a) / h)))
        xs.extend(a + (b - a) * np.arange(1, m) / m)
        xs.append(float(b))
        fixed.extend([False] * (m - 1) + [True])
    return np.asarray(xs, dtype=np.float64), np.asarray(fixed, dtype=bool)


def tet_mesh(dims, boxes, rng: np.random.Generator, cell_voxels: float = 4.0, jitter: float = 0.15,
             focus=(0.5, 0.5, 0.5), refine: float = 0.0, width: float = 0.15):
    """Conforming tetrahedral mesh of the domain [0, dims/Nmax] in which every
    element lies inside one half-open brick box of `boxes` (voxel units).

    Per axis, every brick boundary is a node plane and the nodes between two
    consecutive boundaries are uniform (see _axis_nodes: graded towards
    `focus` when refine > 0, so bricks hold very different element counts).
    Each cell of the node grid is split into six tetrahedra (Kuhn). Nodes off a
    boundary plane are moved along that axis by U[-1, 1] * jitter * (the
    smaller adjacent spacing). Draws, in order: nv*3 U[-1, 1] (nodes x fastest,
    then y, then z; xyz per node).

    Returns (verts float32 (nv, 3) world units, tets int32 (nt, 4)), every
    element positively oriented."""
    dims = [int(d) for d in dims]
    nmax = max(dims)
    boxes = np.asarray(boxes, dtype=np.int64).reshape(-1, 6)
    nodes, fixed, gaps = [], [], []
    for a in range(3):
        cuts = np.unique(np.concatenate([boxes[:, a], boxes[:, 3 + a], [0, dims[a]]]))
        x, f = _axis_nodes(cuts, cell_voxels, focus[a], refine, width, nmax)
        d = np.diff(x)
        g = np.minimum(np.concatenate([[np.inf], d]), np.concatenate([d, [np.inf]]))
        nodes.append(x)
        fixed.append(f)
        gaps.append(g)
    nx, ny, nz = (len(x) for x in nodes)
    zz, yy, xx = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    idx = [xx.ravel(), yy.ravel(), zz.ravel()]
    u = rng.uniform(-1.0, 1.0, size=(idx[0].size, 3))
    verts = np.empty((idx[0].size, 3), dtype=np.float64)
    for a in range(3):
        i = idx[a]
        move = np.where(fixed[a][i], 0.0, jitter * np.where(np.isfinite(gaps[a][i]), gaps[a][i], 0.0))
        verts[:, a] = (nodes[a][i] + u[:, a] * move) / nmax
    tets = grid_tets(nx, ny, nz)
    v32 = verts.astype(np.float32)
    p = v32.astype(np.float64)[tets]
    vol = np.einsum("ij,ij->i", p[:, 1] - p[:, 0], np.cross(p[:, 2] - p[:, 0], p[:, 3] - p[:, 0]))
    flip = vol < 0
    tets[flip] = tets[flip][:, [0, 2, 1, 3]]
    if not np.all(np.abs(vol) > 0):
        raise ValueError("degenerate element; lower the jitter")
    return v32, tets


def mesh_field(rng: np.random.Generator, verts: np.ndarray, n_blobs: int = 12, n_waves: int = 8):
    """Vertex values: blobs (draw_blobs) plus 0.1 * mean of n_waves sinusoids
    sin(k . p + phi), min-max normalised to [0, 1]. Draws, in order: the blobs,
    n_waves*3 wave numbers N(0, 12), n_waves phases U[0, 2 pi]."""
    blobs = draw_blobs(rng, n_blobs)
    k = rng.normal(0.0, 12.0, size=(n_waves, 3))
    phi = rng.uniform(0.0, 2.0 * math.pi, size=n_waves)
    p = verts.astype(np.float64)
    val = np.zeros(p.shape[0])
    for c, s, a in zip(blobs.centers, blobs.sigmas, blobs.amps):
        val += a * np.exp(-np.sum((p - c) ** 2, axis=1) / (2.0 * s * s))
    val += 0.1 * np.mean(np.sin(p @ k.T + phi), axis=1)
    val = (val - val.min()) / (val.max() - val.min())
    return val.astype(np.float32)


def mesh_scene(n: int = 512, seed: int = 5, grid=(4, 3, 3), cell_voxels: float = 5.0, refine: float = 1.5,
               focus=(0.35, 0.55, 0.45)):
    """Unstructured-element workload: a graded, jittered tetrahedral mesh of the
    n^3 nominal domain conforming to a grid of bricks (element density up to
    (1 + refine)^3 times higher near `focus`, so bricks hold very different
    element counts), vertex values from mesh_field, then a random TF. Draws, in
    order (default_rng(seed)): tet_mesh's jitter, mesh_field, random_tf.
    Returns (verts, vals, tets, tf, boxes)."""
    rng = np.random.default_rng(seed)
    gx, gy, gz = grid
    boxes = []
    for bz in range(gz):
        for by in range(gy):
            for bx in range(gx):
                b = (bx, by, bz)
                g = (gx, gy, gz)
                boxes.append([n * b[a] // g[a] for a in range(3)] + [n * (b[a] + 1) // g[a] for a in range(3)])
    boxes = np.asarray(boxes, dtype=np.int32)
    verts, tets = tet_mesh((n, n, n), boxes, rng, cell_voxels=cell_voxels, jitter=0.2, focus=focus,
                           refine=refine)
    vals = mesh_field(rng, verts)
    tf = random_tf(rng)
    return verts, vals, tets, tf, boxes
