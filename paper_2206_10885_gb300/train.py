"""NeuS-style fine-tuning step of a Kilo-grid (Sec. 3.2.2 loss, Sec. 3.3 finite differences).

The loss and its gradient run in libkns.so (kns_train_forward / kns_train_backward); this module
marshals tensors and wraps the pair in a torch.autograd.Function, so the canonical weight tensor can
be an ordinary leaf parameter driven by any torch optimiser:

    params = torch.nn.Parameter(torch.from_numpy(w).cuda())
    loss = kns.train.neus_loss(ctx, desc, params, batch)
    loss.backward()          # params.grad from the hand-written backward kernels

A batch holds the rays (origins, unit directions, target colours), the random draws of the step
(stratified jitter, ascending importance uniforms, eikonal points) and the scalars s, s_up, lambda, h.
"""
from __future__ import annotations

import dataclasses

from . import _capi as capi


@dataclasses.dataclass
class TrainBatch:
    origins: "torch.Tensor"      # (B, 3) float32, device
    dirs: "torch.Tensor"         # (B, 3) unit
    target: "torch.Tensor"       # (B, 3)
    u_strat: "torch.Tensor"      # (B, Ns) in [0, 1)
    u_imp: "torch.Tensor"        # (B, Ni), rows ascending
    eik_points: "torch.Tensor"   # (M, 3)
    s: float = 20.0
    s_up: float = 64.0
    lam: float = 0.1
    h: float = 1e-2
    t_fixed: "torch.Tensor" = None  # (B, Ns + Ni) sample positions to use instead of placing them
    timing: bool = False            # time the phases with CUDA events (stats())

    def __post_init__(self):
        for k in ("origins", "dirs", "target", "u_strat", "u_imp", "eik_points", "t_fixed"):
            t = getattr(self, k)
            if t is not None and not t.is_contiguous():
                setattr(self, k, t.contiguous())

    @property
    def n_rays(self) -> int:
        return int(self.origins.shape[0])

    @property
    def samples(self) -> int:
        return int(self.u_strat.shape[1]) + int(self.u_imp.shape[1])

    def c_struct(self) -> capi.kns_train_batch:
        b = capi.kns_train_batch()
        b.n_rays = self.n_rays
        b.origins = self.origins.data_ptr()
        b.dirs = self.dirs.data_ptr()
        b.target = self.target.data_ptr()
        b.n_strat = int(self.u_strat.shape[1])
        b.n_imp = int(self.u_imp.shape[1])
        b.u_strat = self.u_strat.data_ptr()
        b.u_imp = self.u_imp.data_ptr() if self.u_imp.numel() else None
        b.n_eik = int(self.eik_points.shape[0])
        b.eik_points = self.eik_points.data_ptr() if self.eik_points.numel() else None
        b.s, b.s_up, b.lambda_, b.h = float(self.s), float(self.s_up), float(self.lam), float(self.h)
        b.t_fixed = self.t_fixed.data_ptr() if self.t_fixed is not None else None
        b.timing = 1 if self.timing else 0
        return b


def _stream(stream):
    import torch
    s = stream if stream is not None else torch.cuda.current_stream()
    return int(s.cuda_stream)


def forward(ctx, desc, params, batch: TrainBatch, want_rgb: bool = False, want_t: bool = False, stream=None):
    """Loss parts (L, L_color, L_eik) as a 3-float device tensor, the forward token, rgb, t."""
    import torch
    dev = params.device
    loss = torch.empty(3, dtype=torch.float32, device=dev)
    rgb = torch.empty((batch.n_rays, 3), dtype=torch.float32, device=dev) if want_rgb else None
    t = torch.empty((batch.n_rays, batch.samples), dtype=torch.float32, device=dev) if want_t else None
    tok = capi.kns_train_forward(ctx.handle, desc, params.data_ptr(), batch.c_struct(), loss.data_ptr(),
                                 rgb.data_ptr() if rgb is not None else None,
                                 t.data_ptr() if t is not None else None, _stream(stream))
    return loss, tok, rgb, t


def backward(ctx, token: int, params, dloss=None, stream=None):
    """Gradient of dloss * L (dloss: device scalar tensor or None = 1) for the forward `token`."""
    import torch
    grad = torch.empty_like(params)
    dl = None
    if dloss is not None:
        dl = dloss.detach().to(device=params.device, dtype=torch.float32).reshape(1).contiguous()
    capi.kns_train_backward(ctx.handle, token, dl.data_ptr() if dl is not None else None, grad.data_ptr(),
                            _stream(stream))
    return grad


def step(ctx, desc, params, batch: TrainBatch, stream=None, loss_out=None, grad_out=None):
    """One fused training step (kns_train_step): (loss parts tensor, gradient tensor).

    loss_out (3 floats) and grad_out (params' shape) may be given to reuse buffers."""
    import torch
    loss = loss_out if loss_out is not None else torch.empty(3, dtype=torch.float32, device=params.device)
    grad = grad_out if grad_out is not None else torch.empty_like(params)
    capi.kns_train_step(ctx.handle, desc, params.data_ptr(), batch.c_struct(), loss.data_ptr(), grad.data_ptr(),
                        _stream(stream))
    return loss, grad


def stats(ctx) -> dict:
    """Record counts and per-phase device ms (batches built with timing=True) of the latest step."""
    return capi.kns_train_get_stats(ctx.handle)


def _function():
    import torch

    class KiloNeuSLoss(torch.autograd.Function):
        """L(params) with the library's hand-written backward (one pending forward per context)."""

        @staticmethod
        def forward(fctx, params, ctx, desc, batch):
            loss, tok, _, _ = forward(ctx, desc, params.detach(), batch)
            fctx.kns = (ctx, tok)
            fctx.save_for_backward(params)
            fctx.mark_non_differentiable(loss)
            return loss[0].clone(), loss

        @staticmethod
        def backward(fctx, g_loss, g_parts):
            (params,) = fctx.saved_tensors
            ctx, tok = fctx.kns
            return backward(ctx, tok, params.detach(), dloss=g_loss), None, None, None

    return KiloNeuSLoss


_FN = None


def neus_loss(ctx, desc, params, batch: TrainBatch, return_parts: bool = False):
    """Differentiable loss L = L_color + lambda L_eik (scalar tensor); parts (L, L_color, L_eik) optional."""
    global _FN
    if _FN is None:
        _FN = _function()
    loss, parts = _FN.apply(params, ctx, desc, batch)
    return (loss, parts) if return_parts else loss
