"""Pins of the oracle's tetrahedral-mesh sampling (unstructured elements; the
paper's data set is a mixed-element mesh distributed over ranks, Sec. 5).

Each pin fixes the mesh path against something other than itself:
  M1 a linear vertex field is reproduced exactly (linear precision of
     barycentric interpolation), at random points of a jittered mesh;
  M2 the chosen element contains the point: barycentrics recomputed here from
     signed sub-volumes (np.linalg.det, not Cramer's rule) are >= 0, sum to 1
     and give the returned value; the bin index equals brute force;
  M3 on rays along shared grid lines the mesh render equals the pinned voxel
     render of the same data (trilinear and the Kuhn interpolant agree there);
  M4 constant field: A = 1 - (1 - a)^n, C = rgb A (closed form);
  M5 any brick split of a conforming mesh composites to the unsplit render;
  M6 a hole in the mesh fails loudly; generator validity (volumes tile the
     domain, every element inside its brick).
"""
import numpy as np
import pytest

import oracle
from paper_2501_01628_gb300 import synth


def _mesh(n=32, g=(2, 2, 2), seed=0, **kw):
    boxes = oracle.grid_partition((n, n, n), g)
    rng = np.random.default_rng(seed)
    verts, tets = synth.tet_mesh((n, n, n), boxes, rng, **kw)
    return boxes, verts, tets


def _points_inside(rng, m, lo=0.0, hi=1.0):
    return rng.uniform(lo, hi, size=(m, 3))


def test_m1_linear_field_reproduced_exactly():
    boxes, verts, tets = _mesh(seed=1, jitter=0.2)
    rng = np.random.default_rng(11)
    a = rng.normal(size=3)
    b = 0.3
    vals = verts.astype(np.float64) @ a + b
    mesh = oracle.Mesh(verts, vals, tets, (32, 32, 32))
    pts = _points_inside(rng, 2000)
    out = oracle.mesh_sample(mesh, boxes, pts)
    np.testing.assert_allclose(out["vals"], pts @ a + b, rtol=0, atol=1e-12)
    assert np.all(out["minb"] >= -1e-12)


def test_m2_containment_by_signed_volumes_and_bins_equal_brute_force():
    boxes, verts, tets = _mesh(seed=2, jitter=0.2, refine=1.0, focus=(0.3, 0.6, 0.5))
    rng = np.random.default_rng(12)
    vals = rng.uniform(size=verts.shape[0])
    mesh = oracle.Mesh(verts, vals, tets, (32, 32, 32))
    pts = _points_inside(rng, 1500)
    out = oracle.mesh_sample(mesh, boxes, pts)
    V = verts.astype(np.float64)
    for i in range(pts.shape[0]):
        t = tets[out["elem"][i]]
        P = V[t]

        def vol(q):
            return np.linalg.det(np.stack([q[1] - q[0], q[2] - q[0], q[3] - q[0]]))

        full = vol(P)
        lam = []
        for j in range(4):
            Q = P.copy()
            Q[j] = pts[i]
            lam.append(vol(Q) / full)
        lam = np.array(lam)
        assert lam.min() >= -1e-10, (i, lam)
        assert abs(lam.sum() - 1.0) < 1e-12
        assert abs(lam @ vals[t] - out["vals"][i]) < 1e-12
        # the element belongs to the point's owner brick (centroid rule)
        cell = np.clip(np.floor(P.mean(axis=0) * 32), 0, 31).astype(int)
        b = out["brick"][i]
        assert np.all(cell >= boxes[b, :3]) and np.all(cell < boxes[b, 3:])
    brute = oracle.mesh_sample(oracle.Mesh(verts, vals, tets, (32, 32, 32), bruteforce=True), boxes, pts)
    assert np.array_equal(brute["vals"], out["vals"])
    assert np.array_equal(brute["elem"], out["elem"])


def _axis_node_values(vol_axis_len, nodes):
    """Clamped 1D linear weights of voxel-centred samples at node positions
    (voxel units): the matrix W with W @ column = interpolated values."""
    n = vol_axis_len
    W = np.zeros((nodes.size, n))
    v = nodes - 0.5
    i0 = np.floor(v).astype(int)
    f = v - i0
    for r, (i, w) in enumerate(zip(i0, f)):
        W[r, min(max(i, 0), n - 1)] += 1.0 - w
        W[r, min(max(i + 1, 0), n - 1)] += w
    return W


@pytest.mark.parametrize("ert", [1.0, 0.9])
def test_m3_mesh_equals_voxel_render_on_grid_lines(ert):
    n = 16
    rng = np.random.default_rng(13)
    vol = rng.uniform(0.0, 1.0, size=(n, n, n))
    boxes = oracle.grid_partition((n, n, n), (2, 2, 2))
    cuts = np.array([0, n // 2, n], dtype=np.float64)
    nodes = np.unique(np.concatenate([cuts, np.arange(n) + 0.5]))
    W = _axis_node_values(n, nodes)
    # node values = trilinear (clamp-to-edge) of the voxel data at the nodes
    node_vals = np.einsum("zk,yj,xi,kji->zyx", W, W, W, vol)
    m = nodes.size
    zz, yy, xx = np.meshgrid(nodes, nodes, nodes, indexing="ij")
    verts = np.stack([xx.ravel(), yy.ravel(), zz.ravel()], axis=1) / n
    tets = synth.grid_tets(m, m, m)
    mesh = oracle.Mesh(verts, node_vals.ravel(), tets, (n, n, n))
    tf = synth.random_tf(np.random.default_rng(14), alpha_max=0.3)
    cam = synth.ortho_camera_z(n, n)
    ref = oracle.render(vol, boxes, tf, 0.0, 1.0, cam, ert_alpha=ert)
    got = oracle.render(mesh, boxes, tf, 0.0, 1.0, cam, ert_alpha=ert)
    assert got["nsamples"] == ref["nsamples"]
    np.testing.assert_allclose(got["img"], ref["img"], rtol=0, atol=1e-12)
    assert ref["img"][..., 3].max() > 0.2


def test_m4_constant_slab_closed_form():
    boxes, verts, tets = _mesh(seed=3, jitter=0.2)
    vals = np.full(verts.shape[0], 0.4)
    mesh = oracle.Mesh(verts, vals, tets, (32, 32, 32))
    rgba = np.array([0.2, 0.7, 0.5, 0.05], np.float32)
    tf = synth.constant_tf(rgba)
    cam = synth.ortho_camera_z(24, 20)
    out = oracle.render(mesh, boxes, tf, 0.0, 1.0, cam)
    a = np.float64(rgba[3])
    A = 1.0 - (1.0 - a) ** 64  # 32 voxels at half-voxel steps
    np.testing.assert_allclose(out["img"][..., 3], A, rtol=0, atol=1e-13)
    for c in range(3):
        np.testing.assert_allclose(out["img"][..., c], np.float64(rgba[c]) * A, rtol=0, atol=1e-13)
    assert out["nsamples"] == 24 * 20 * 64


@pytest.mark.parametrize("kind", ["grid", "kd"])
def test_m5_brick_split_equals_unsplit(kind):
    n = 32
    if kind == "grid":
        boxes = oracle.grid_partition((n, n, n), (2, 3, 2))
    else:
        boxes = oracle.kd_partition((n, n, n), 7, np.random.default_rng(5).uniform(0.3, 0.7, 6))
    rng = np.random.default_rng(15)
    verts, tets = synth.tet_mesh((n, n, n), boxes, rng, cell_voxels=3.0, jitter=0.2, refine=1.0)
    vals = synth.mesh_field(rng, verts)
    mesh = oracle.Mesh(verts, vals, tets, (n, n, n))
    tf = synth.random_tf(np.random.default_rng(16), alpha_max=0.1)
    cam = synth.orbit_camera(40, 32, 37.0, elevation_deg=25.0)
    split = oracle.render(mesh, boxes, tf, 0.0, 1.0, cam)
    whole = oracle.render(mesh, [[0, 0, 0, n, n, n]], tf, 0.0, 1.0, cam)
    assert split["nsamples"] == whole["nsamples"] > 0
    np.testing.assert_allclose(split["img"], whole["img"], rtol=0, atol=1e-12)
    assert whole["img"][..., 3].max() > 0.05


def test_m6_hole_fails_and_generator_validity():
    boxes, verts, tets = _mesh(seed=4, jitter=0.2, refine=2.0, focus=(0.7, 0.3, 0.5))
    V = verts.astype(np.float64)
    P = V[tets]
    vol = np.einsum("ij,ij->i", P[:, 1] - P[:, 0], np.cross(P[:, 2] - P[:, 0], P[:, 3] - P[:, 0])) / 6.0
    assert np.all(vol > 0)
    assert abs(vol.sum() - 1.0) < 1e-6  # float32 vertices
    cells = np.clip(np.floor(P.mean(axis=1) * 32), 0, 31).astype(int)
    for b, box in enumerate(boxes):
        inb = np.all((cells >= box[:3]) & (cells < box[3:]), axis=1)
        pv = P[inb].reshape(-1, 3) * 32
        assert np.all(pv >= box[:3] - 1e-5) and np.all(pv <= box[3:] + 1e-5)
    # drop the elements around the domain centre: rays through it must fail
    c = P.mean(axis=1)
    keep = np.linalg.norm(c - 0.5, axis=1) > 0.15
    mesh = oracle.Mesh(verts, np.full(verts.shape[0], 0.5), tets[keep], (32, 32, 32))
    tf = synth.constant_tf([1, 1, 1, 0.01])
    cam = synth.ortho_camera_z(9, 9)  # the centre pixel's ray crosses the hole
    with pytest.raises(RuntimeError, match="-5"):
        oracle.render(mesh, boxes, tf, 0.0, 1.0, cam)
