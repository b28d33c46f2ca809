"""torch.autograd.Function wrappers of the hand-written kernels, so the
Stage-1 loss can be written as a composition and differentiated with
`loss.backward()`:

    mean_t, quat_t = NTCTransform.apply(table, weights, mean, quat, ctx)   # Section 4.1, Eq. 5
    img = Rasterize.apply(mean_t, quat_t, raster_ctx)                       # Section 3.2, Eq. 2-4
    loss = L1DSSIM.apply(img, target, loss_module)                          # Eq. 6

Each forward calls the library's forward kernels and each backward the
library's reverse kernels (nothing is differentiated by PyTorch); the
per-pixel compositing state is recomputed in the reverse pass from T_final
and the last-contributor index, not stored per pair.  The training engine
(`engine.Stage1`) issues the same calls directly for CUDA-graph capture;
these wrappers are for composing the path with other PyTorch code.

A Rasterizer or Loss object holds the state of one forward until its
backward: run one forward/backward at a time per object.
"""
from __future__ import annotations

import dataclasses
from typing import Optional, Sequence

import torch

from . import gs3
from .engine import Loss, Rasterizer


@dataclasses.dataclass
class NTCContext:
    """Constant inputs of the transformation cache: the grid, its box, the
    quaternion product order and the MLP precision (GS_MLP_FP32 or
    GS_MLP_BF16; the BF16 path reads FP16/BF16 copies of the FP32 inputs)."""

    grid: gs3.GsHashgrid
    precision: int = gs3.GS_MLP_FP32
    order: int = 0

    @property
    def aabb(self) -> Sequence[float]:
        return list(self.grid.aabb)


class NTCTransform(torch.autograd.Function):
    """(hash table [entries][2], MLP weights [6592]) -> transformed means
    [n][3] and rotations [n][4] of the frozen Gaussians (mean, quat)."""

    @staticmethod
    def forward(ctx, table: torch.Tensor, weights: torch.Tensor, mean: torch.Tensor,
                quat: torch.Tensor, c: NTCContext):
        n = mean.shape[0]
        dev = mean.device
        bf16 = c.precision == gs3.GS_MLP_BF16
        table_in = table.detach().to(torch.float16) if bf16 else table.detach().contiguous()
        w32 = weights.detach().contiguous()
        w16 = w32.to(torch.bfloat16) if bf16 else None
        mlp = gs3.mlp_struct(c.precision, w32, w16)
        enc = torch.empty(n, 32, dtype=torch.bfloat16 if bf16 else torch.float32, device=dev)
        raw7 = torch.empty(n, 7, device=dev)
        mean_t = torch.empty(n, 3, device=dev)
        quat_t = torch.empty(n, 4, device=dev)
        gs3.ntc_encode_fwd(mean, n, c.grid, table_in, enc)
        gs3.ntc_mlp_fwd(enc, n, mlp, raw7)
        gs3.ntc_apply(mean, quat, raw7, n, c.aabb, c.order, mean_t, quat_t)
        ctx.c, ctx.mlp, ctx.table_shape = c, mlp, table.shape
        ctx.save_for_backward(mean, quat, enc, raw7)
        return mean_t, quat_t

    @staticmethod
    def backward(ctx, d_mean_t: Optional[torch.Tensor], d_quat_t: Optional[torch.Tensor]):
        mean, quat, enc, raw7 = ctx.saved_tensors
        c, n, dev = ctx.c, mean.shape[0], mean.device
        d_mean_t = torch.zeros(n, 3, device=dev) if d_mean_t is None else d_mean_t.contiguous()
        d_quat_t = torch.zeros(n, 4, device=dev) if d_quat_t is None else d_quat_t.contiguous()
        d_raw7 = torch.empty(n, 7, device=dev)
        gs3.ntc_apply_bwd(mean, quat, raw7, n, c.aabb, c.order, d_mean_t, d_quat_t, d_raw7)
        d_w = torch.zeros(gs3.MLP_PARAMS, device=dev)
        d_enc = torch.empty(n, 32, device=dev)
        gs3.ntc_mlp_bwd(enc, n, ctx.mlp, d_raw7, None, d_w, d_enc)
        d_table = torch.zeros(ctx.table_shape, device=dev)
        gs3.ntc_encode_bwd(mean, n, c.grid, d_enc, d_table)
        return d_table, d_w, None, None, None


@dataclasses.dataclass
class RasterContext:
    """A rasterizer for V views of W x H, the frozen Gaussian attributes
    (scales, opacities, SH) and the device cameras of the batch."""

    raster: Rasterizer
    gaussians: gs3.Gaussians
    cams_dev: torch.Tensor


class Rasterize(torch.autograd.Function):
    """(means [n][3], rotations [n][4]) -> images [V][3][H][W]: projection,
    binning and compositing forward; compositing and projection reverse."""

    @staticmethod
    def forward(ctx, mean: torch.Tensor, quat: torch.Tensor, rc: RasterContext):
        mean, quat = mean.detach().contiguous(), quat.detach().contiguous()
        img = rc.raster.forward(rc.gaussians, rc.cams_dev, mean, quat)
        ctx.rc = rc
        ctx.save_for_backward(mean, quat)
        return img.clone()

    @staticmethod
    def backward(ctx, d_img: torch.Tensor):
        mean, quat = ctx.saved_tensors
        rc = ctx.rc
        d_mean, d_quat = rc.raster.backward(rc.gaussians, rc.cams_dev, d_img.contiguous(), mean,
                                            quat)
        return d_mean.clone(), d_quat.clone(), None


class L1DSSIM(torch.autograd.Function):
    """(images, targets) -> (1 - lambda) L1 + lambda (1 - SSIM) (Eq. 6)."""

    @staticmethod
    def forward(ctx, img: torch.Tensor, target: torch.Tensor, loss: Loss):
        loss(img.detach().contiguous(), target.contiguous())
        ctx.save_for_backward(loss.d_img.clone())
        return loss.d_loss.clone().reshape(())

    @staticmethod
    def backward(ctx, g: torch.Tensor):
        (d_img,) = ctx.saved_tensors
        return d_img * g, None, None
