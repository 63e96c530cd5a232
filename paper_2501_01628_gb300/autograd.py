"""Differentiable rendering through libvr: a torch.autograd.Function whose
forward is vr_render_frame and whose backward is vr_render_backward (the
checkpointed adjoint kernels). Argument marshalling only; no pixel or gradient
arithmetic happens in Python.

    r = Renderer(partition=dict(kind="grid", grid=(2, 2, 2)), vmin=0.0, vmax=1.5)
    img = r.render(tf, density, cam)       # tf [n, 4], density [Nz, Ny, Nx]: CUDA float32
    loss = ((img - target) ** 2).mean()
    loss.backward()                         # tf.grad, density.grad

Early termination is off (the adjoint differentiates every lattice sample).
"""
from __future__ import annotations

import torch

from . import vr


class Renderer:
    """One context plus one packed volume, re-packed when the density tensor
    changes (data pointer or version)."""

    def __init__(self, partition: dict, vmin: float, vmax: float, step_voxels: float = 0.5,
                 device: int | None = None, storage: str = "f32"):
        self.device = torch.cuda.current_device() if device is None else int(device)
        self.ctx = vr.vr_create(self.device)
        self.partition = partition
        self.vmin, self.vmax = float(vmin), float(vmax)
        self.step = float(step_voxels)
        self.storage = storage
        self.vol = None
        self._key = None
        self._shape = None
        vr.vr_set_render_params(self.ctx, self.step, 1.0)

    def _bind(self, tf: torch.Tensor, density: torch.Tensor, cam: dict):
        d = density.detach()
        if not (d.is_cuda and d.dtype == torch.float32 and d.is_contiguous()):
            raise ValueError("density must be a contiguous CUDA float32 tensor")
        key = (d.data_ptr(), d._version, tuple(d.shape))
        if self.vol is None or tuple(d.shape) != self._shape:
            if self.vol is not None:
                vr.vr_volume_release(self.vol)
            self.vol = vr.vr_volume_create(self.ctx, d, self.storage, self.partition)
            self._shape = tuple(d.shape)
        elif key != self._key:
            vr.vr_volume_update(self.vol, d)
        self._key = key
        vr.vr_set_transfer_function(self.ctx, tf.detach().contiguous(), self.vmin, self.vmax)
        vr.vr_set_camera(self.ctx, cam)

    def render(self, tf: torch.Tensor, density: torch.Tensor, cam: dict) -> torch.Tensor:
        return _Render.apply(tf, density, self, cam)

    def close(self):
        if self.vol is not None:
            vr.vr_volume_release(self.vol)
            self.vol = None
        if self.ctx is not None:
            vr.vr_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class _Render(torch.autograd.Function):
    @staticmethod
    def forward(ctx, tf, density, renderer: Renderer, cam: dict):
        renderer._bind(tf, density, cam)
        out = torch.empty((cam["height"], cam["width"], 4), dtype=torch.float32, device=density.device)
        vr.vr_render_frame(renderer.ctx, renderer.vol, out)
        ctx.save_for_backward(tf, density)
        ctx.renderer = renderer
        ctx.cam = cam
        return out

    @staticmethod
    def backward(ctx, grad_out):
        tf, density = ctx.saved_tensors
        r = ctx.renderer
        r._bind(tf, density, ctx.cam)
        gtf = torch.zeros_like(tf, dtype=torch.float32)
        gden = torch.zeros_like(density) if ctx.needs_input_grad[1] else None
        vr.vr_render_backward(r.ctx, r.vol, grad_out.contiguous().float(), gtf, gden)
        vr.vr_sync(r.ctx)
        return (gtf if ctx.needs_input_grad[0] else None), gden, None, None
