"""Time-varying data through a fixed device budget.

The paper's deployment keeps only some of a time-varying data set's time steps
in GPU memory, loading and later evicting them (Sec. 4). Here the time steps
stay in pinned host memory and `slots` packed volumes live on the device; while
step t renders on the render stream, step t+1 is uploaded and re-packed into the
slot that step t+1-slots used, on a copy stream (vr_volume_update_async). CUDA
events order the two. Orchestration only: the copies, packing and rendering are
library calls.
"""
from __future__ import annotations

import torch

from . import vr


class TimeSeriesRenderer:
    def __init__(self, ctx, steps_host, partition: dict, storage: str = "f32", slots: int = 2):
        if slots < 2:
            raise ValueError("streaming needs at least two slots")
        self.ctx = ctx
        self.steps = steps_host
        self.slots = slots
        self.render_stream = torch.cuda.current_stream()
        self.copy_stream = torch.cuda.Stream()
        self.vols = [vr.vr_volume_create(ctx, steps_host[min(i, len(steps_host) - 1)], storage, partition)
                     for i in range(slots)]
        self.resident = list(range(slots))  # time step held by each slot
        self.ready = [torch.cuda.Event() for _ in range(slots)]
        self.released = [torch.cuda.Event() for _ in range(slots)]
        for e in self.ready:
            e.record(self.render_stream)

    def _load(self, t: int):
        """Upload step t into its slot once the slot's previous step is rendered."""
        s = t % self.slots
        if self.resident[s] == t:
            return
        self.copy_stream.wait_event(self.released[s])
        vr.vr_volume_update_async(self.vols[s], self.steps[t], stream=self.copy_stream)
        self.ready[s].record(self.copy_stream)
        self.resident[s] = t

    def render_step(self, t: int, cams, outs, prefetch: bool = True):
        """Render step t for each camera into outs[i] (device [H, W, 4]); with
        prefetch the next step's upload overlaps these renders."""
        self._load(t)
        s = t % self.slots
        self.render_stream.wait_event(self.ready[s])
        if prefetch and t + 1 < len(self.steps):
            # the next step's slot was released by the render of step t+1-slots
            self._load(t + 1)
        for cam, out in zip(cams, outs):
            vr.vr_set_camera(self.ctx, cam)
            vr.vr_render_frame(self.ctx, self.vols[s], out, stream=self.render_stream)
        self.released[s].record(self.render_stream)

    def close(self):
        torch.cuda.synchronize()
        for v in self.vols:
            vr.vr_volume_release(v)
        self.vols = []
