"""BOS reconstruction of a voxel temperature field by minibatch gradient descent on
L_BOS (Sec. 2.4 with lambda_2 = lambda_3 = 0: no boundary or PINN terms; Sec. 3.2's
random pixel minibatches and AdaBelief).  Argument marshalling only: every iteration is
bos_sample_pixels, bos_set_grid, bos_render_pixels, bos_loss_l2_pixels, bos_backward,
bos_adabelief_step and bos_counter_add, all on the device.  The iteration number lives in
device memory, so one iteration can be captured in a CUDA graph and replayed: run()
launches the whole iteration with a single graph launch instead of ~10 API calls."""
from __future__ import annotations

import torch

from . import bos


class Reconstructor:
    """Minibatch reconstruction of the voxel temperatures from one BOS image.

    loss_scale multiplies L_BOS.  AdaBelief's step does not depend on the gradient's scale
    only while eps is small against the squared gradient; image-loss gradients are often
    near 1e-10 per voxel (I carries the 1/path-length weight), so pick loss_scale to bring
    them to order one."""

    def __init__(self, scene, target, T_init, batch: int = 5000, lr: float = 0.05, beta1: float = 0.9,
                 beta2: float = 0.999, eps: float = 1e-16, loss_scale: float = 1.0,
                 prec: int = bos.BOS_PREC_FP32_COMP, seed: int = 0, device: int = 0, sort: bool = True):
        self.scene, self.prec, self.seed = scene, prec, seed
        self.sort = sort and batch <= 16384
        self.dev = torch.device("cuda", device)
        self.ctx = bos.Context(device)
        self.ctx.set_geometry(scene.camera, scene.wall, scene.light, scene.integ)
        self.T = T_init.to(self.dev, torch.float32).contiguous().clone()
        self.target = target.to(self.dev, torch.float32).contiguous()
        self.m = torch.zeros_like(self.T)
        self.s = torch.zeros_like(self.T)
        self.g = torch.empty_like(self.T)
        self.batch = batch
        self.pix = torch.empty(batch, dtype=torch.int32, device=self.dev)
        self.I = torch.empty(batch, dtype=torch.float32, device=self.dev)
        self.dLdI = torch.empty(batch, dtype=torch.float32, device=self.dev)
        self.loss = torch.empty(1, dtype=torch.float64, device=self.dev)
        self.lr, self.b1, self.b2, self.eps, self.loss_scale = lr, beta1, beta2, eps, loss_scale
        self.it = 0                                   # iterations issued (host copy)
        self.it_dev = torch.zeros(1, dtype=torch.int64, device=self.dev)   # iterations done (device)
        self.gd = bos.grid_desc(scene.grid, prec)
        self.graph = None

    def _iteration(self, sp: int) -> None:
        L = bos.lib()
        h = self.ctx.h
        npx = self.scene.camera.width * self.scene.camera.height
        it = self.it_dev.data_ptr()
        bos.bos_sample_pixels(self.pix.data_ptr(), self.batch, npx, self.seed, 0, sp, draw_dev=it)
        if self.sort:   # neighbouring pixels per warp: coherent rays, larger scatter groups
            bos.bos_sort_pixels(self.pix.data_ptr(), self.batch, self.scene.camera.width, self.scene.camera.height, sp)
        bos.check(L.bos_set_grid(h, bos.C.byref(self.gd), self.T.data_ptr(), sp), "bos_set_grid")
        bos.bos_render_pixels(h, self.pix.data_ptr(), self.batch, self.I.data_ptr(), None, 1, sp)
        bos.bos_loss_l2_pixels(self.I.data_ptr(), self.target.data_ptr(), self.pix.data_ptr(), self.batch,
                               self.loss.data_ptr(), self.dLdI.data_ptr(), sp, self.loss_scale)
        bos.bos_backward(h, self.dLdI.data_ptr(), self.g.data_ptr(), sp)
        bos.bos_adabelief_step(self.T.data_ptr(), self.g.data_ptr(), self.m.data_ptr(), self.s.data_ptr(),
                               self.T.numel(), self.lr, self.b1, self.b2, self.eps, 1, sp, step_dev=it)
        bos.bos_counter_add(it, 1, sp)

    def step(self) -> torch.Tensor:
        """One iteration, launched call by call; returns the minibatch loss (a device scalar)."""
        self._iteration(torch.cuda.current_stream().cuda_stream)
        self.it += 1
        return self.loss

    def run(self, iterations: int) -> torch.Tensor:
        """`iterations` iterations by replaying a CUDA graph of one iteration (captured on the
        first call, after one eager iteration has sized every buffer); returns the last
        minibatch loss."""
        if iterations <= 0:
            return self.loss
        if self.graph is None:
            self.step()                               # allocations happen outside the capture
            iterations -= 1
            side = torch.cuda.Stream(device=self.dev)
            side.wait_stream(torch.cuda.current_stream())
            torch.cuda.current_stream().wait_stream(side)
            g = torch.cuda.CUDAGraph()
            with torch.cuda.graph(g, stream=side):
                self._iteration(side.cuda_stream)
            self.graph = g
            # the capture only recorded the iteration; replays below do the work
        for _ in range(iterations):
            self.graph.replay()
        self.it += iterations
        return self.loss

    def close(self):
        self.ctx.close()
