"""Pins of the oracle's adjoint (vector-Jacobian product of rendered pixels):
central finite differences of the oracle's own FP64 forward render, the
constant-slab closed form dA/dalpha = n (1-alpha)^(n-1), and split invariance
(the gradient does not depend on how the volume is bricked)."""
import math

import numpy as np
import pytest

import oracle
from paper_2501_01628_gb300 import synth

pytestmark = pytest.mark.usefixtures("oracle_lib")


def _scene(seed=3, n=10):
    rng = np.random.default_rng(seed)
    vol = synth.blob_volume(n, synth.draw_blobs(rng, 4)).astype(np.float64)
    vol += rng.uniform(0, 0.05, vol.shape)
    tf = synth.random_tf(rng, alpha_max=0.3).astype(np.float64)
    return vol, tf, rng


def _loss(vol, boxes, tf, lo, hi, cam, G, crop):
    img = oracle.render(vol, boxes, tf, lo, hi, cam, 0.5, crop=crop, dtype=oracle.F64)["img"]
    return float(np.sum(G * img))


@pytest.mark.parametrize("camkind", ["persp", "ortho"])
def test_vjp_matches_central_differences(camkind):
    vol, tf, rng = _scene()
    n = vol.shape[0]
    lo, hi = float(vol.min()) - 0.01, float(vol.max()) + 0.01
    cam = (synth.orbit_camera(7, 6, 40.0, radius=1.6) if camkind == "persp"
           else dict(ortho=1, eye=(0.5, 0.5, 1.5), dir=(0.2, -0.1, -1.0), up=(0, 1, 0), ortho_w=1.3,
                     ortho_h=1.2, width=7, height=6))
    boxes = oracle.kd_partition((n,) * 3, 5, [0.4, 0.6, 0.5, 0.35])
    crop = (0, 0, 7, 6)
    G = rng.standard_normal((6, 7, 4))
    gtf, gvol = oracle.render_grad(vol, boxes, tf, lo, hi, cam, G, crop=crop, dtype=oracle.F64)
    h = 1e-6
    # table entries with the largest gradients, plus a few random ones
    flat = np.argsort(-np.abs(gtf).ravel())[:12].tolist() + rng.integers(0, gtf.size, 4).tolist()
    for idx in flat:
        i, c = divmod(int(idx), 4)
        tp, tm = tf.copy(), tf.copy()
        tp[i, c] += h
        tm[i, c] -= h
        fd = (_loss(vol, boxes, tp, lo, hi, cam, G, crop) - _loss(vol, boxes, tm, lo, hi, cam, G, crop)) / (2 * h)
        assert abs(fd - gtf[i, c]) <= 1e-6 * max(1.0, abs(fd)), (i, c, fd, gtf[i, c])
    vflat = np.argsort(-np.abs(gvol).ravel())[:12]
    assert np.abs(gvol).max() > 0
    for idx in vflat:
        k = np.unravel_index(idx, vol.shape)
        vp, vm = vol.copy(), vol.copy()
        vp[k] += h
        vm[k] -= h
        fd = (_loss(vp, boxes, tf, lo, hi, cam, G, crop) - _loss(vm, boxes, tf, lo, hi, cam, G, crop)) / (2 * h)
        assert abs(fd - gvol[k]) <= 1e-5 * max(1e-3, abs(fd)), (k, fd, gvol[k])


@pytest.mark.parametrize("alpha", [0.01, 0.2, 0.7])
def test_constant_slab_closed_form_derivatives(alpha):
    n = 8
    vol = np.full((n, n, n), 0.3)
    tf = np.tile(np.array([[0.9, 0.5, 0.2, alpha]]), (16, 1))
    cam = synth.ortho_camera_z(3, 3)
    boxes = oracle.grid_partition((n,) * 3, (1, 1, 2))
    nsamp = 2 * n
    # dI_A / d(alpha shift of every entry) = n (1-alpha)^(n-1)
    G = np.zeros((3, 3, 4))
    G[1, 1, 3] = 1.0
    gtf, gvol = oracle.render_grad(vol, boxes, tf, 0.0, 1.0, cam, G, dtype=oracle.F64)
    np.testing.assert_allclose(gtf[:, 3].sum(), nsamp * (1 - alpha) ** (nsamp - 1), rtol=1e-12, atol=1e-14)
    assert np.allclose(gvol, 0)  # constant table: the scalar has no influence
    # dI_r / dr = 1 - (1-alpha)^n, dI_r / dalpha = r n (1-alpha)^(n-1)
    G = np.zeros((3, 3, 4))
    G[0, 2, 0] = 1.0
    gtf, _ = oracle.render_grad(vol, boxes, tf, 0.0, 1.0, cam, G, dtype=oracle.F64)
    np.testing.assert_allclose(gtf[:, 0].sum(), 1 - (1 - alpha) ** nsamp, rtol=1e-12)
    np.testing.assert_allclose(gtf[:, 3].sum(), 0.9 * nsamp * (1 - alpha) ** (nsamp - 1), rtol=1e-12, atol=1e-14)


@pytest.mark.parametrize("split", ["grid", "kd"])
def test_gradient_independent_of_bricking(split):
    vol, tf, rng = _scene(seed=8, n=12)
    n = vol.shape[0]
    lo, hi = float(vol.min()), float(vol.max())
    cam = synth.orbit_camera(9, 8, 130.0, radius=1.7, elevation_deg=-30)
    G = rng.standard_normal((8, 9, 4))
    whole = oracle.render_grad(vol, [[0, 0, 0, n, n, n]], tf, lo, hi, cam, G, dtype=oracle.F64)
    boxes = (oracle.grid_partition((n,) * 3, (2, 3, 2)) if split == "grid"
             else oracle.kd_partition((n,) * 3, 7, rng.uniform(0.3, 0.7, 6)))
    parts = oracle.render_grad(vol, boxes, tf, lo, hi, cam, G, dtype=oracle.F64)
    np.testing.assert_allclose(parts[0], whole[0], atol=1e-11)
    np.testing.assert_allclose(parts[1], whole[1], atol=1e-11)
