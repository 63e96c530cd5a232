"""Tetrahedral-mesh volumes (unstructured elements): the CUDA path (per-brick
BVH point location + face-neighbour walk) against the FP64 oracle (barycentric
sampling of the owner brick's elements), element by element on whole images,
plus the library's validation of the mesh it is given."""
import numpy as np
import pytest

import oracle
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


def mesh_render(vr, verts, vals, tets, dims, part, tf, lo, hi, cam, step=0.5, ert=1.0, count=False,
                opc_ref=0.0, host_out=False):
    import torch
    ctx = vr.vr_create(0)
    m = None
    try:
        m = vr.vr_mesh_create(ctx, verts, vals, tets, dims, part)
        vr.vr_set_transfer_function(ctx, tf, lo, hi)
        vr.vr_set_camera(ctx, cam)
        vr.vr_set_render_params(ctx, step, ert)
        vr.vr_set_count_samples(ctx, count)
        if opc_ref:
            vr.vr_set_opacity_correction(ctx, opc_ref)
        H, W = cam["height"], cam["width"]
        if host_out:
            out = torch.empty((H, W, 4), dtype=torch.float32).pin_memory()
        else:
            out = torch.full((H, W, 4), float("nan"), dtype=torch.float32, device="cuda")
        vr.vr_render_mesh_frame(ctx, m, out)
        vr.vr_sync(ctx)
        res = dict(img=out.cpu().numpy().astype(np.float64))
        if count:
            res["nsamples"] = vr.vr_get_sample_count(ctx)
        res["counts"] = vr.vr_mesh_info(m)[0]
        return res
    finally:
        if m is not None:
            vr.vr_mesh_release(m)
        vr.vr_destroy(ctx)


def _scene(n, part, seed, cell=3.0, refine=1.5, jitter=0.2):
    boxes = vr_boxes(n, part)
    rng = np.random.default_rng(seed)
    verts, tets = synth.tet_mesh((n, n, n), boxes, rng, cell_voxels=cell, jitter=jitter, refine=refine,
                                 focus=(0.35, 0.6, 0.45))
    vals = synth.mesh_field(rng, verts)
    tf = synth.random_tf(rng, alpha_max=0.04)
    return boxes, verts, vals, tets, tf


def vr_boxes(n, part):
    from paper_2501_01628_gb300 import vr as _vr
    return _vr.vr_partition_boxes((n, n, n), part)


@pytest.mark.parametrize("az,ert", [(20.0, 1.0), (135.0, 1.0), (250.0, 0.95), (315.0, 0.99)])
def test_mesh_kd_bricks_perspective(vr, az, ert):
    """40^3 nominal lattice (not a power of two), 7 kd bricks, a graded jittered
    mesh (~26k elements), 72x56 perspective views."""
    n = 40
    rng = np.random.default_rng(40)
    part = dict(kind="kd", n_bricks=7, cut_fracs=rng.uniform(0.3, 0.7, 6))
    boxes, verts, vals, tets, tf = _scene(n, part, seed=41)
    cam = synth.orbit_camera(72, 56, az, elevation_deg=25.0)
    got = mesh_render(vr, verts, vals, tets, (n, n, n), part, tf, 0.0, 1.0, cam, ert=ert, count=True)
    mesh = oracle.Mesh(verts, vals, tets, (n, n, n))
    env = oracle_env(mesh, boxes, tf, 0.0, 1.0, cam, ert=ert)
    stats = compare_envelope(got["img"], env)
    assert env["img"][..., 3].max() > 0.2
    assert abs(got["nsamples"] - env["nsamples"]) <= 4 * max(1, stats["n_ambiguous"]) + 8
    assert got["counts"].sum() == tets.shape[0]


def test_mesh_rays_along_element_edges(vr):
    """Orthographic rays exactly along shared grid lines of an unjittered Kuhn
    mesh (every ray runs along element edges and faces: the walk's degenerate
    case), 2x2x2 bricks."""
    n = 16
    part = dict(kind="grid", grid=(2, 2, 2))
    boxes = vr_boxes(n, part)
    nodes = np.unique(np.concatenate([[0.0, n / 2, n], np.arange(n) + 0.5]))
    m = nodes.size
    zz, yy, xx = np.meshgrid(nodes, nodes, nodes, indexing="ij")
    verts = (np.stack([xx.ravel(), yy.ravel(), zz.ravel()], axis=1) / n).astype(np.float32)
    tets = synth.grid_tets(m, m, m)
    rng = np.random.default_rng(42)
    vals = rng.uniform(0.0, 1.0, size=verts.shape[0]).astype(np.float32)
    tf = synth.random_tf(rng, alpha_max=0.2)
    cam = synth.ortho_camera_z(n, n)
    got = mesh_render(vr, verts, vals, tets, (n, n, n), part, tf, 0.0, 1.0, cam)
    env = oracle_env(oracle.Mesh(verts, vals, tets, (n, n, n)), boxes, tf, 0.0, 1.0, cam)
    compare_envelope(got["img"], env)


def test_mesh_one_brick_equals_split_and_opacity_correction(vr):
    """The same mesh as one brick and as a 3x2x2 grid gives the same image
    (associativity of over); with opacity correction at step 0.75 against
    reference 0.5 both match the oracle."""
    n = 32
    part = dict(kind="grid", grid=(3, 2, 2))
    boxes, verts, vals, tets, tf = _scene(n, part, seed=43, cell=4.0, refine=1.0)
    cam = synth.orbit_camera(64, 48, 60.0, elevation_deg=-15.0)
    split = mesh_render(vr, verts, vals, tets, (n, n, n), part, tf, 0.0, 1.0, cam, step=0.75, opc_ref=0.5)
    whole = mesh_render(vr, verts, vals, tets, (n, n, n), dict(kind="grid", grid=(1, 1, 1)), tf, 0.0, 1.0, cam,
                        step=0.75, opc_ref=0.5)
    assert np.abs(split["img"] - whole["img"]).max() <= 2e-6
    env = oracle_env(oracle.Mesh(verts, vals, tets, (n, n, n)), boxes, tf, 0.0, 1.0, cam, step=0.75,
                     opacity_ref_step=0.5)
    compare_envelope(split["img"], env)


def test_mesh_host_output(vr):
    n = 24
    part = dict(kind="grid", grid=(2, 1, 2))
    boxes, verts, vals, tets, tf = _scene(n, part, seed=44, cell=3.0, refine=0.0)
    cam = synth.orbit_camera(40, 40, 200.0)
    dev = mesh_render(vr, verts, vals, tets, (n, n, n), part, tf, 0.0, 1.0, cam)
    host = mesh_render(vr, verts, vals, tets, (n, n, n), part, tf, 0.0, 1.0, cam, host_out=True)
    assert np.array_equal(dev["img"], host["img"])


def test_mesh_validation(vr):
    """Elements across a brick boundary, a hole, a degenerate element and an
    out-of-range index are rejected with VR_ERR_ARG before any device work."""
    n = 16
    part = dict(kind="grid", grid=(2, 1, 1))
    boxes = vr_boxes(n, part)
    rng = np.random.default_rng(45)
    verts, tets = synth.tet_mesh((n, n, n), boxes, rng, cell_voxels=4.0)
    vals = np.zeros(verts.shape[0], np.float32)
    ctx = vr.vr_create(0)
    try:
        # a mesh built for one brick does not respect the x = 5, 10 cuts of a 3-brick grid
        v1, t1 = synth.tet_mesh((n, n, n), [[0, 0, 0, n, n, n]], np.random.default_rng(1), cell_voxels=6.0)
        with pytest.raises(vr.VrError) as e:
            vr.vr_mesh_create(ctx, v1, np.zeros(v1.shape[0], np.float32), t1, (n, n, n),
                              dict(kind="grid", grid=(3, 1, 1)))
        assert e.value.status == vr.VR_ERR_ARG
        with pytest.raises(vr.VrError) as e:  # hole: drop one element
            vr.vr_mesh_create(ctx, verts, vals, tets[1:], (n, n, n), part)
        assert e.value.status == vr.VR_ERR_ARG
        bad = tets.copy()
        bad[5] = [bad[5, 0], bad[5, 0], bad[5, 2], bad[5, 3]]
        with pytest.raises(vr.VrError) as e:  # degenerate element
            vr.vr_mesh_create(ctx, verts, vals, bad, (n, n, n), part)
        assert e.value.status == vr.VR_ERR_ARG
        bad = tets.copy()
        bad[0, 0] = verts.shape[0]
        with pytest.raises(vr.VrError) as e:
            vr.vr_mesh_create(ctx, verts, vals, bad, (n, n, n), part)
        assert e.value.status == vr.VR_ERR_ARG
        m = vr.vr_mesh_create(ctx, verts, vals, tets, (n, n, n), part)
        cnt, nbytes = vr.vr_mesh_info(m)
        assert cnt.sum() == tets.shape[0] and nbytes >= 80 * tets.shape[0]
        vr.vr_mesh_release(m)
    finally:
        vr.vr_destroy(ctx)


def test_mesh_workload_sampled(vr):
    """The benchmark's 25.0M-element mesh (36 bricks, 1920x1080, ERT 0.99) in
    the launch configuration the bench times: 2 views, 300 pixels each against
    the oracle on the same float32 mesh."""
    import torch
    verts, vals, tets, tf, boxes = synth.mesh_scene()
    part = dict(kind="grid", grid=(4, 3, 3))
    ctx = vr.vr_create(0)
    m = vr.vr_mesh_create(ctx, verts, vals, tets, (512, 512, 512), part)
    try:
        vr.vr_set_transfer_function(ctx, tf, 0.0, 1.0)
        vr.vr_set_render_params(ctx, 0.5, 0.99)
        vr.vr_set_composite_schedule(ctx, (4, 3, 3))
        out = torch.empty((1080, 1920, 4), device="cuda")
        mesh = oracle.Mesh(verts, vals, tets, (512, 512, 512))
        rng = np.random.default_rng(77)
        for az in (45.0, 270.0):
            cam = synth.orbit_camera(1920, 1080, az)
            vr.vr_set_camera(ctx, cam)
            vr.vr_render_mesh_frame(ctx, m, out)
            vr.vr_sync(ctx)
            img = out.cpu().numpy().astype(np.float64)
            pix = np.stack([rng.integers(0, 1920, 300), rng.integers(0, 1080, 300)], axis=1)
            env = oracle_env(mesh, boxes, tf, 0.0, 1.0, cam, ert=0.99, pixels=pix)
            assert env["img"][:, 3].max() > 0.5
            compare_envelope(img[pix[:, 1], pix[:, 0]], env)
    finally:
        vr.vr_mesh_release(m)
        vr.vr_destroy(ctx)
