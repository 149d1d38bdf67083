"""torch.autograd bridge for the finite-temperature occupation (Sec. IV.B).

``SoftOccupation.apply(Cdd, Cgd, handle, raster, kT, t, closed, n_charges)``
returns <n> [P, N] from the CUDA kernels; its backward calls the hand-written
backward kernel (dL/dCdd, dL/dCgd with every pixel's candidate set frozen).
Cdd is the Maxwell dot-dot block (symmetrised on the device), Cgd the
gate-dot block; both FP64 CUDA tensors.  PyTorch supplies device memory,
streams, the loss and the optimiser; every step of the model runs in the
library's kernels.
"""
from __future__ import annotations

import time

import torch

from . import api


class SoftOccupation(torch.autograd.Function):
    @staticmethod
    def forward(ctx, Cdd, Cgd, handle, raster, kT, t, closed, n_charges):
        n, ng = api.qa_model_shape(handle)
        P = int(raster["W"]) * int(raster["H"])
        Cdd_c = Cdd.detach().contiguous()
        Cgd_c = Cgd.detach().contiguous()
        api.qa_model_update_dev(handle, Cdd_c, Cgd_c)
        mean = torch.empty((P, n), dtype=torch.float32, device=Cdd.device)
        pctx = torch.empty(P, dtype=torch.int64, device=Cdd.device)
        api.qa_soft_occupation_ctx(handle, raster, kT, t, closed, n_charges, mean, None, pctx)
        ctx.save_for_backward(mean, pctx)
        ctx.handle = handle
        ctx.raster = raster
        ctx.args = (kT, t, closed, n_charges)
        ctx.shape = (n, ng)
        return mean

    @staticmethod
    def backward(ctx, grad_mean):
        n, ng = ctx.shape
        g = grad_mean.detach().to(torch.float32).contiguous()
        dCdd = torch.empty((n, n), dtype=torch.float64, device=g.device)
        dCgd = torch.empty((n, ng), dtype=torch.float64, device=g.device)
        kT, t, closed, n_charges = ctx.args
        mean, pctx = ctx.saved_tensors
        api.qa_soft_occupation_backward_ctx(ctx.handle, ctx.raster, kT, t, closed, n_charges,
                                            g, mean, pctx, dCdd, dCgd)
        return dCdd, dCgd, None, None, None, None, None, None


def soft_occupation(Cdd, Cgd, handle, raster, kT, t=1.0, closed=False, n_charges=0):
    return SoftOccupation.apply(Cdd, Cgd, handle, raster, float(kT), float(t),
                                bool(closed), int(n_charges))


class CapacitanceFit:
    """Fits (Cdd, Cgd) so that the soft occupation over a raster matches a
    target (MSE), with Adam.  The target is either a charge-sensing style
    diagram, sum_i <n_i> per pixel (shape [P] or [H, W]), or the occupation
    of every dot (shape [P, N]).

    fused=True (default): one qa_fit_step call per step -- model update
    (device FP64 inverse), soft occupation, the loss and its gradient per pixel,
    the backward reduction and the Adam update, all in the library's kernels.
    fused=False: the same step through torch autograd (SoftOccupation), a
    torch loss and torch.optim.Adam.  Either way, after a warm-up the step is
    captured once into a CUDA graph and replayed (graph=True)."""

    def __init__(self, Cdd0, Cgd0, raster, target, kT, t=1.0, lr=2e-3, graph=True,
                 fused=True, betas=(0.9, 0.999), eps=1e-8):
        dev = torch.device("cuda")
        self.Cdd = torch.tensor(Cdd0, dtype=torch.float64, device=dev, requires_grad=not fused)
        self.Cgd = torch.tensor(Cgd0, dtype=torch.float64, device=dev, requires_grad=not fused)
        self.model = api.Model(Cdd0, Cgd0)
        self.raster = raster
        self.kT = float(kT)
        self.t = float(t)
        tg = torch.as_tensor(target, dtype=torch.float32, device=dev)
        n, ng = self.Cdd.shape[0], self.Cgd.shape[1]
        P = int(raster["W"]) * int(raster["H"])
        self.per_dot = tg.numel() == P * n and tg.dim() == 2
        self.target = tg.contiguous() if self.per_dot else tg.reshape(-1).contiguous()
        self.fused = fused
        self.lr, self.betas, self.eps = float(lr), betas, float(eps)
        if fused:
            self.state = torch.zeros(api.fit_state_len(n, ng), dtype=torch.float64, device=dev)
            self._raster_c = api.make_raster(raster, ng)
        else:
            # fused: one optimiser kernel for both tensors
            self.opt = torch.optim.Adam([self.Cdd, self.Cgd], lr=lr, betas=betas, eps=eps,
                                        capturable=graph, fused=True)
        self.use_graph = graph
        self.graph = None
        self.loss = torch.zeros((), dtype=torch.float32, device=dev)

    def _step(self):
        if self.fused:
            api.qa_fit_step(self.model.handle, self._raster_c, self.kT, self.t, False, 0,
                            self.target, self.per_dot, self.Cdd, self.Cgd, self.state, self.lr,
                            self.betas[0], self.betas[1], self.eps, loss=self.loss)
            return
        # gradients are assigned by the backward (no zeroing, no accumulate);
        # under capture they live in the graph's pool at fixed addresses
        self.opt.zero_grad(set_to_none=True)
        mean = soft_occupation(self.Cdd, self.Cgd, self.model.handle, self.raster,
                               self.kT, self.t)
        pred = mean if self.per_dot else mean.sum(1)
        loss = torch.mean((pred - self.target) ** 2)
        loss.backward()
        self.opt.step()
        self.loss.copy_(loss.detach())

    def step(self):
        if not self.use_graph:
            self._step()
            return
        if self.graph is None:
            # warm-up on a side stream (sizes the library workspace and the
            # optimiser state), then capture one step
            s = torch.cuda.Stream()
            s.wait_stream(torch.cuda.current_stream())
            with torch.cuda.stream(s):
                for _ in range(3):
                    self._step()
            torch.cuda.current_stream().wait_stream(s)
            self.graph = torch.cuda.CUDAGraph()
            with torch.cuda.graph(self.graph):
                self._step()
        self.graph.replay()

    def close(self):
        self.model.close()


def target_diagram(Cdd, Cgd, raster, kT, t=1.0, per_dot=False):
    """sum_i <n_i> of a model on the GPU (the synthetic fitting target), or
    with per_dot the occupations <n> [P, N] themselves."""
    m = api.Model(Cdd, Cgd)
    mean, _ = m.soft_occupation(raster, kT, threshold=t)
    out = mean.clone() if per_dot else mean.sum(1).clone()
    m.close()
    return out


def time_grad_step(cfg, kT, steps=100, flush=None, graph=True, fused=True):
    """Milliseconds per capacitance-fitting step (100 Adam steps timed end to
    end on the device; CUDA graph replay, or plain launches with graph=False;
    the fused library step, or the autograd + torch.optim path)."""
    target = target_diagram(cfg["Cdd_target"], cfg["Cgd_target"], cfg["raster"], kT)
    fit = CapacitanceFit(cfg["Cdd"], cfg["Cgd"], cfg["raster"], target, kT, graph=graph,
                         fused=fused)
    for _ in range(3):
        fit.step()
    torch.cuda.synchronize()
    a = torch.cuda.Event(enable_timing=True)
    b = torch.cuda.Event(enable_timing=True)
    if flush is not None:
        flush.zero_()
    a.record()
    for _ in range(steps):
        fit.step()
    b.record()
    torch.cuda.synchronize()
    fit.close()
    return a.elapsed_time(b) / steps
