"""Stage-1 training engine: device buffers and the kernel sequence of one
training iteration of the Neural Transformation Cache (Section 4.1), the
plain direct-optimisation comparator (Section 5.3, "Direct Opt."), the
warm-up (Eq. 7) and a render helper.  All computation happens in libgs3;
this module owns buffers, streams and the order of calls.
"""
from __future__ import annotations

import math
import time
from typing import List, Optional

import numpy as np
import torch

from . import gs3
from .gs3 import Gaussians, Projected

LAMBDA_DSSIM = 0.2          # Eq. 6
NTC_LR = 0.002              # Suppl. A
ITERS_PER_FRAME = 150       # Stage-1 iterations per frame (Section 5.2)
ADAM_BETAS = (0.9, 0.99)    # I-NGP's Adam constants (the paper's NTC follows I-NGP)
# Stage 1: the rate decays exponentially to 1 % over a frame's iterations
# (an exponential decay as in 3DG-S's schedule for Gaussian means, whose
# other hyper-parameters the paper keeps), and epsilon is set against the
# unscaled gradients of a loss averaged over V x 3 x H x W pixel channels
# (table gradients of order 1e-9 .. 1e-6): entries touched only by Gaussians
# that no view sees get no full-rate steps.  The warm-up keeps I-NGP's
# epsilon and a constant rate.
STAGE1_LR_FINAL = 0.01
STAGE1_EPS = 1e-6
WARMUP_EPS = 1e-15
DEFAULT_BIN = 4             # tiles per bin side of the binned pair lists (autotuned best at 1352x1014)
TILE_LIST_CAP = 1024        # staged records a tile keeps for the reverse (more: the reverse re-tests its bin list)


def _i32(*shape, device="cuda"):
    return torch.zeros(*shape, dtype=torch.int32, device=device)


def _f32(*shape, device="cuda"):
    return torch.zeros(*shape, dtype=torch.float32, device=device)


class Rasterizer:
    """Projection + binning + compositing (+ reverse) for V views of W x H."""

    def __init__(self, n: int, V: int, W: int, H: int, capacity: int, device="cuda",
                 bg=(0.0, 0.0, 0.0), bin: int = DEFAULT_BIN, n_max: Optional[int] = None):
        self.V, self.W, self.H = V, W, H
        self.device = device
        self.bg = tuple(float(x) for x in bg)
        self.bin = int(bin)
        self.bins = gs3.bins_of(W, H, self.bin)
        self.n_max = max(n, n_max or n)
        nm = self.n_max
        # flat storage for up to n_max Gaussians; the [V][n] views follow n
        self._proj = Projected.empty(V, nm, device)
        self._grads = _f32(V * nm * 8, device=device)
        self._d_mean = _f32(nm * 3, device=device)
        self._d_quat = _f32(nm * 4, device=device)
        self.ranges = _i32(V * self.bins, 2, device=device)
        self.d_count = torch.zeros(1, dtype=torch.int64, device=device)
        self.d_err = _i32(1, device=device)
        self.img = _f32(V, 3, H, W, device=device)
        self.T_final = _f32(V, H, W, device=device)
        self.last = _i32(V, H, W, device=device)
        # the records each tile's forward staged, for the reverse
        self.lists = gs3.TileLists(V, W, H, TILE_LIST_CAP, device)
        self._listed = False
        self.set_n(n)
        self.set_capacity(capacity)

    def set_n(self, n: int):
        """Number of Gaussians of the next calls (<= n_max); the per-record
        arrays are [V][n] views of the same storage."""
        if not 0 <= n <= self.n_max:
            raise ValueError("Rasterizer.set_n: %d Gaussians outside [0, %d]" % (n, self.n_max))
        self.n = n
        V = self.V
        sub = lambda t, *tail: t.view(-1)[:V * n * int(np.prod(tail or (1,)))].view(V, n, *tail)
        P = self._proj
        self.proj = Projected(sub(P.mean2d, 2), sub(P.conic_opacity, 4), sub(P.rgb, 3),
                              sub(P.depth), sub(P.radius), sub(P.tiles_touched))
        self.grads = self._grads[:V * n * 8].view(V, n, 8)
        self.d_mean = self._d_mean[:n * 3].view(n, 3)
        self.d_quat = self._d_quat[:n * 4].view(n, 4)

    def set_capacity(self, capacity: int):
        self.capacity = int(capacity)
        self.vals = _i32(max(self.capacity, 1), device=self.device)
        ws = gs3.gs_bin_sort_workspace_size(self.n_max, self.V, self.W, self.H, self.capacity)
        self.ws = torch.empty(ws, dtype=torch.uint8, device=self.device)

    def forward(self, g: Gaussians, cams_dev, mean=None, quat=None, stream=None, keys=None,
                lists: bool = True):
        """lists: keep each tile's staged records for backward() (a render
        with no reverse to follow can leave them out)."""
        V, W, H, n = self.V, self.W, self.H, self.n
        gs3.gs_project(g, cams_dev, V, W, H, self.proj, mean, quat, stream, self.d_err)
        gs3.gs_bin_sort(self.proj, n, V, W, H, self.bin, self.capacity, self.vals, self.ranges, keys,
                        self.d_count, self.d_err, self.ws, stream)
        gs3.gs_raster_fwd(self.proj, n, V, W, H, self.bin, self.bg, self.vals, self.ranges, self.img,
                          self.T_final, self.last, None, stream, lists=self.lists if lists else None)
        self._listed = lists
        return self.img

    def backward(self, g: Gaussians, cams_dev, d_img, mean=None, quat=None, stream=None):
        V, W, H, n = self.V, self.W, self.H, self.n
        gs3.gs_raster_bwd(self.proj, n, V, W, H, self.bin, self.bg, self.vals, self.ranges,
                          self.T_final, self.last, d_img, self.grads, None, None, stream,
                          lists=self.lists if self._listed else None)
        gs3.gs_project_bwd(g, cams_dev, V, W, H, self.grads, self.d_mean, self.d_quat, mean, quat,
                           stream)
        return self.d_mean, self.d_quat

    def count(self) -> int:
        return int(self.d_count.item())

    def check(self):
        """Raise if the device reported an error (reads device memory: syncs):
        a non-finite Gaussian met by the projection, or more pairs than the
        binning capacity."""
        err = int(self.d_err.item())
        if err == gs3.GS_ERR_NONFINITE:
            raise gs3.GsError("gs_project", err, "a non-finite Gaussian was culled")
        if err != 0:
            raise gs3.GsError("gs_bin_sort", err, "device reported error (count %d, capacity %d)"
                              % (self.count(), self.capacity))

    def fit_capacity(self, g: Gaussians, cams_dev, mean=None, quat=None, margin=1.5):
        """Run the forward once and grow the pair buffers to margin x the count."""
        self.d_err.zero_()
        self.forward(g, cams_dev, mean, quat)
        c = self.count()
        want = max(1024, int(c * margin))
        if want > self.capacity or self.d_err.item() != 0:
            self.set_capacity(want)
            self.d_err.zero_()
            self.forward(g, cams_dev, mean, quat)
        self.check()
        return c


class Loss:
    def __init__(self, V, W, H, device="cuda", lam=LAMBDA_DSSIM):
        self.V, self.W, self.H, self.lam = V, W, H, lam
        self.ws = torch.empty(gs3.gs_loss_workspace_size(3 * V, H, W), dtype=torch.uint8,
                              device=device)
        self.d_img = _f32(V, 3, H, W, device=device)
        self.d_loss = _f32(1, device=device)
        self.d_ssim = _f32(1, device=device)

    def __call__(self, img, target, stream=None):
        gs3.gs_loss_l1_dssim(img, target, 3 * self.V, self.H, self.W, self.lam, self.d_img,
                             self.d_loss, self.d_ssim, self.ws, stream)
        return self.d_loss


def adam_hp(lr, eps=STAGE1_EPS, lr_final_ratio=STAGE1_LR_FINAL, decay_steps=ITERS_PER_FRAME,
            betas=ADAM_BETAS) -> gs3.GsAdam:
    """Adam hyper-parameters: rate lr decaying to lr * lr_final_ratio over
    decay_steps applied updates (decay_steps <= 1: constant)."""
    return gs3.GsAdam(lr, betas[0], betas[1], eps, lr_final_ratio, decay_steps)


class AdamBuffers:
    def __init__(self, p: torch.Tensor, lr: float, shadow_dtype=None, hp: Optional[gs3.GsAdam] = None):
        self.p = p
        self.g = torch.zeros_like(p)
        self.m = torch.zeros_like(p)
        self.v = torch.zeros_like(p)
        self.hp = hp if hp is not None else adam_hp(lr)
        self.shadow = None if shadow_dtype is None else p.to(shadow_dtype)

    def reset(self, values: Optional[torch.Tensor] = None):
        if values is not None:
            self.p.copy_(values)
            if self.shadow is not None:
                self.shadow.copy_(values.to(self.shadow.dtype))
        self.g.zero_()
        self.m.zero_()
        self.v.zero_()

    def step(self, d_state, stream=None, hp: Optional[gs3.GsAdam] = None):
        gs3.adam_step(self.p, self.g, self.m, self.v, self.hp if hp is None else hp, d_state,
                      self.shadow, stream)


class NTC:
    """Hash table (FP32 master + FP16 shadow) and MLP (FP32 master + BF16 shadow)."""

    def __init__(self, table: np.ndarray, weights: List[np.ndarray], grid: gs3.GsHashgrid,
                 precision: int = gs3.GS_MLP_BF16, device="cuda", lr=NTC_LR,
                 hp: Optional[gs3.GsAdam] = None, iters: int = ITERS_PER_FRAME):
        self.grid = grid
        self.precision = precision
        self.entries = gs3.ntc_hashgrid_entries(grid)
        if table.shape != (self.entries, 2):
            raise ValueError("NTC: table of shape %s, the grid has %d entries x 2 features"
                             % (table.shape, self.entries))
        w = np.concatenate([x.reshape(-1) for x in weights]).astype(np.float32)
        if w.size != gs3.MLP_PARAMS:
            raise ValueError("NTC: %d MLP weights, expected %d" % (w.size, gs3.MLP_PARAMS))
        tab = torch.from_numpy(np.ascontiguousarray(table, np.float32)).to(device)
        # Stage 1's Adam (hp, default: the decayed schedule) and the warm-up's
        # (I-NGP's epsilon, constant rate)
        hp = hp if hp is not None else adam_hp(lr, decay_steps=iters)
        self.warm_hp = adam_hp(lr, eps=WARMUP_EPS, lr_final_ratio=1.0, decay_steps=0)
        self.table = AdamBuffers(tab, lr, torch.float16, hp)
        self.mlp = AdamBuffers(torch.from_numpy(w).to(device), lr, torch.bfloat16, hp)
        self.init_table = tab.clone()
        self.init_mlp = self.mlp.p.clone()

    def mlp_struct(self):
        return gs3.mlp_struct(self.precision, self.mlp.p, self.mlp.shadow)

    def table_for_encode(self):
        # the mixed-precision path reads the FP16 shadow; the FP32 path the master
        return self.table.shadow if self.precision == gs3.GS_MLP_BF16 else self.table.p

    def enc_dtype(self):
        return torch.bfloat16 if self.precision == gs3.GS_MLP_BF16 else torch.float32

    def reset_to(self, table: torch.Tensor, mlp: torch.Tensor):
        self.table.reset(table)
        self.mlp.reset(mlp)

    def weights_numpy(self):
        w = self.mlp.p.detach().cpu().numpy().astype(np.float64)
        return [w[:2048].reshape(64, 32), w[2048:6144].reshape(64, 64), w[6144:].reshape(7, 64)]


class Stage1:
    """One Stage-1 training iteration (Section 4.1): NTC query of the frozen
    previous-frame means, transformation, render of a batch of views, L1 +
    D-SSIM loss, hand-written backward into the hash table and MLP, Adam."""

    def __init__(self, g: Gaussians, ntc: NTC, V: int, W: int, H: int, capacity: int,
                 order: int = 0, loss_scale: Optional[float] = None, growth_interval=2000,
                 device="cuda", bin: int = DEFAULT_BIN, fused: bool = False):
        n = g.n
        # the fused cache kernels exist for the BF16 tensor-core MLP
        self.fused = fused and ntc.precision == gs3.GS_MLP_BF16
        self.g, self.ntc, self.V, self.W, self.H, self.order = g, ntc, V, W, H, order
        self.raster = Rasterizer(n, V, W, H, capacity, device, bin=bin)
        self.loss = Loss(V, W, H, device)
        self.enc = torch.zeros(n, 32, dtype=ntc.enc_dtype(), device=device)
        self.raw7 = _f32(n, 7, device=device)
        self.mean_t = _f32(n, 3, device=device)
        self.quat_t = _f32(n, 4, device=device)
        self.d_raw7 = _f32(n, 7, device=device)
        self.d_enc = _f32(n, 32, device=device)
        # the rows with a nonzero cache-output gradient (most Gaussians are
        # seen by no view of a batch): the cache's reverse works on those only
        self.active = torch.zeros(max(n, 1), dtype=torch.int32, device=device)
        self.n_active = torch.zeros(1, dtype=torch.int64, device=device)
        if loss_scale is None:
            loss_scale = 2.0 ** 15 if ntc.precision == gs3.GS_MLP_BF16 else 1.0
        self.growth = growth_interval if ntc.precision == gs3.GS_MLP_BF16 else 0
        self.state = gs3.new_train_state(loss_scale, device)
        self.aabb = list(ntc.grid.aabb)
        self.track = None  # (accum [n], denom [n]) while tracking view-space gradients
        # the encoding kernels' order over the Gaussians (refresh_order); kept
        # in place so that captured graphs read the refreshed order
        self.visit = torch.empty(max(n, 1), dtype=torch.int32, device=device)[:n]
        self._visit_ws = torch.empty(max(gs3.ntc_spatial_order_workspace_size(n), 1), dtype=torch.uint8,
                                     device=device)
        self.refresh_order()

    def refresh_order(self, stream=None):
        """Spatial order of the encoding kernels' work over the Gaussians (for
        table locality; any permutation gives the same results).  Called when
        the Gaussians' means change (each frame of a stream)."""
        gs3.ntc_spatial_order(self.g.mean, self.g.n, self.ntc.grid, self.visit, self._visit_ws, stream)

    def track_viewspace(self, on: bool = True):
        """Start (zeroed) or stop accumulating the view-space positional
        gradient statistics of the Gaussians (Section 4.2: during the final
        epoch of Stage 1).  Graphs captured while tracking include it."""
        if on:
            n = self.g.n
            dev = self.g.mean.device
            self.track = (torch.zeros(n, device=dev), torch.zeros(n, dtype=torch.int32, device=dev))
        else:
            self.track = None
        return self.track

    def reset_state(self, loss_scale=None):
        """Start a frame: the step count (and with it the bias correction and
        the rate schedule) restarts at 0; the loss scale is kept unless given.
        Device operations only (no host read), so it can sit in a timed loop."""
        if loss_scale is None:
            self.state[4:].zero_()
        else:
            self.state.copy_(gs3.new_train_state(loss_scale, self.state.device))

    def transform(self, stream=None):
        """NTC query + transformation: writes mean_t, quat_t."""
        g, ntc, n = self.g, self.ntc, self.g.n
        if self.fused:
            gs3.ntc_fused_fwd(g.mean, g.quat, n, ntc.grid, ntc.table.shadow, ntc.mlp_struct(), self.order,
                              self.mean_t, self.quat_t, self.raw7, self.enc, stream)
            return self.mean_t, self.quat_t
        gs3.ntc_encode_fwd(g.mean, n, ntc.grid, ntc.table_for_encode(), self.enc, stream, order=self.visit)
        gs3.ntc_mlp_fwd(self.enc, n, ntc.mlp_struct(), self.raw7, stream)
        gs3.ntc_apply(g.mean, g.quat, self.raw7, n, self.aabb, self.order, self.mean_t, self.quat_t,
                      stream)
        return self.mean_t, self.quat_t

    def compute_grads(self, cams_dev, target, stream=None):
        """Forward and backward of one iteration; leaves the scaled gradients
        in ntc.table.g and ntc.mlp.g (no update)."""
        g, ntc, n = self.g, self.ntc, self.g.n
        self.transform(stream)
        img = self.raster.forward(g, cams_dev, self.mean_t, self.quat_t, stream)
        self.loss(img, target, stream)
        d_mean, d_quat = self.raster.backward(g, cams_dev, self.loss.d_img, self.mean_t, self.quat_t,
                                              stream)
        if self.track is not None:
            # view-space positional gradients of the final epoch feed Stage 2's spawn
            accum, denom = self.track
            gs3.gs_viewspace_grad_accum(self.raster.grads, self.raster.proj.radius, self.V, n, 0, n,
                                        self.W, self.H, float(self.V), accum, denom, stream)
        if self.fused:
            gs3.ntc_fused_bwd(g.mean, g.quat, self.raw7, self.enc, n, ntc.grid, ntc.mlp_struct(), self.order,
                              d_mean, d_quat, self.loss_scale_view(), ntc.mlp.g, ntc.table.g, stream)
            return self.loss.d_loss
        gs3.ntc_apply_bwd(g.mean, g.quat, self.raw7, n, self.aabb, self.order, d_mean, d_quat,
                          self.d_raw7, stream)
        gs3.ntc_active_rows(self.d_raw7, n, self.active, self.n_active, stream)
        gs3.ntc_mlp_bwd(self.enc, n, ntc.mlp_struct(), self.d_raw7, self.loss_scale_view(),
                        ntc.mlp.g, self.d_enc, stream, rows=self.active, d_rows=self.n_active)
        # the reverse encoding over the same rows (not in spatial order: there
        # neighbouring Gaussians' atomics would meet on the same table rows)
        gs3.ntc_encode_bwd(g.mean, n, ntc.grid, self.d_enc, ntc.table.g, stream, order=self.active,
                           d_count=self.n_active)
        return self.loss.d_loss

    def loss_scale_view(self):
        return self.state[0:4].view(torch.float32)

    def update(self, stream=None):
        ntc = self.ntc
        gs3.gs_check_finite(ntc.table.g, self.state, stream)
        gs3.gs_check_finite(ntc.mlp.g, self.state, stream)
        ntc.table.step(self.state, stream)
        ntc.mlp.step(self.state, stream)
        gs3.gs_train_state_advance(self.state, self.growth, stream)

    def step(self, cams_dev, target, stream=None):
        d_loss = self.compute_grads(cams_dev, target, stream)
        self.update(stream)
        return d_loss

    def capture(self, batches):
        """One CUDA graph of step() per (cams_dev, target) batch; a replay runs
        the whole iteration with no host work.  Captured after one eager step
        per batch (side stream), which also advances the training state: reset
        the cache and the state before timing or training."""
        return capture_graphs(self.step, batches)


STAGE2_LR = (0.0024, 0.015, 0.075, 0.75, 0.0375, 0.0375 / 20)  # Suppl. A; SH bands >= 1 at 1/20
STAGE2_BETAS = (0.9, 0.999)   # 3DG-S's Adam for Gaussian attributes
STAGE2_EPS = 1e-15
TAU_GRAD = 0.00015            # Section 4.2
TAU_ALPHA = 0.01
SPAWN_OPACITY = 0.1
SPLIT_SCALE = 0.8


class Stage2:
    """Stage 2, adaptive 3DG addition (Section 4.2): Gaussians added around
    the transformed Gaussians with large view-space positional gradients are
    trained (every attribute, Adam) while the transformed ones stay fixed;
    at the end of each epoch (one pass over the view batches) the added ones
    above the gradient threshold spawn one more nearby and those below the
    opacity threshold are discarded.

    The rasterizer draws one set: the n fixed Gaussians first, then the
    added ones, from buffers of n + capacity rows."""

    def __init__(self, g: Gaussians, V: int, W: int, H: int, capacity: int,
                 pair_capacity: int = 1 << 22, device="cuda", bin: int = DEFAULT_BIN,
                 lr=STAGE2_LR, tau_grad=TAU_GRAD, tau_alpha=TAU_ALPHA, seed: int = 0):
        self.g, self.V, self.W, self.H = g, V, W, H
        self.n_fixed, self.cap = g.n, int(capacity)
        self.deg = g.sh_deg
        K = (self.deg + 1) ** 2
        P = gs3.added_cols(self.deg)
        nm = self.n_fixed + self.cap
        f = lambda *sh: _f32(*sh, device=device)
        self.all = Gaussians(f(nm, 3), f(nm, 4), f(nm, 3), f(nm), f(nm, K, 3), self.deg)
        self.rows = [f(self.cap, P) for _ in range(2)]
        self.m = [f(self.cap, P) for _ in range(2)]
        self.v = [f(self.cap, P) for _ in range(2)]
        self.cur = 0
        self.n_add = 0
        self.d_n = torch.zeros(1, dtype=torch.int64, device=device)
        self.d_nsel = torch.zeros(1, dtype=torch.int64, device=device)
        self.d_err = _i32(1, device=device)
        self.idx = _i32(max(self.n_fixed, self.cap), device=device)
        self.d_mean, self.d_quat, self.d_scale = f(self.cap, 3), f(self.cap, 4), f(self.cap, 3)
        self.d_ologit, self.d_sh = f(self.cap), f(self.cap, K, 3)
        self.accum = f(self.cap)
        self.denom = _i32(self.cap, device=device)
        self.raster = Rasterizer(self.n_fixed, V, W, H, pair_capacity, device, bin=bin, n_max=nm)
        self._d_op = f(V * nm)
        self.loss = Loss(V, W, H, device)
        self.lr = tuple(lr)
        self.tau_grad, self.tau_alpha = tau_grad, tau_alpha
        self.state = gs3.new_train_state(1.0, device)
        self.gen = torch.Generator(device=device)
        self.gen.manual_seed(seed)

    def added(self, k=None) -> gs3.GsAdded:
        k = self.cur if k is None else k
        return gs3.added_struct(self.rows[k], self.m[k], self.v[k], self.deg)

    def view(self) -> Gaussians:
        """The drawn set: fixed Gaussians followed by the current added ones."""
        n = self.n_fixed + self.n_add
        a = self.all
        return Gaussians(a.mean[:n], a.quat[:n], a.scale[:n], a.opacity_logit[:n], a.sh[:n], self.deg)

    def begin(self, mean_t, quat_t, accum, denom, random_count: Optional[int] = None):
        """Fixed set = the previous frame's Gaussians at the transformed means
        and rotations; one added Gaussian around each with an average
        view-space gradient above tau_grad (accum / denom from the final epoch
        of Stage 1).  random_count = k instead spawns around k fixed
        Gaussians drawn uniformly (the random-spawn ablation of Section 5.3).
        Reads the number added back to the host."""
        n, g, a = self.n_fixed, self.g, self.all
        a.mean[:n].copy_(mean_t)
        a.quat[:n].copy_(quat_t)
        a.scale[:n].copy_(g.scale)
        a.opacity_logit[:n].copy_(g.opacity_logit)
        a.sh[:n].copy_(g.sh)
        fixed = Gaussians(a.mean[:n], a.quat[:n], a.scale[:n], a.opacity_logit[:n], a.sh[:n], self.deg)
        if random_count is None:
            gs3.gs_select_above(accum, denom, n, self.tau_grad, self.idx, self.d_nsel)
        else:
            pick = torch.randperm(n, generator=self.gen, device=mean_t.device)[:random_count]
            self.idx[:pick.numel()].copy_(pick.sort().values.to(torch.int32))
            self.d_nsel.fill_(pick.numel())
        z = torch.randn(n, 3, generator=self.gen, device=mean_t.device)
        self.cur = 0
        self.d_n.zero_()
        self.d_err.zero_()
        gs3.gs_added_spawn(fixed, self.idx, self.d_nsel, z, SPAWN_OPACITY, self.added(), self.d_n,
                           self.d_err)
        self.n_add = int(self.d_n.item())
        self._after_resize()
        self.state.copy_(gs3.new_train_state(1.0, self.state.device))
        return self.n_add

    def _after_resize(self):
        self.accum.zero_()
        self.denom.zero_()
        self.raster.set_n(self.n_fixed + self.n_add)
        gs3.gs_added_to_render(self.added(), self.n_add, self.view(), self.n_fixed)

    def compute_grads(self, cams_dev, target, stream=None):
        """Forward and backward of one iteration: gradients of the added rows
        in d_mean .. d_sh, view-space statistics accumulated."""
        g = self.view()
        r, n, V, W, H = self.raster, g.n, self.V, self.W, self.H
        r.forward(g, cams_dev, stream=stream)
        self.loss(r.img, target, stream)
        d_op = self._d_op[:V * n]
        gs3.gs_raster_bwd(r.proj, n, V, W, H, r.bin, r.bg, r.vals, r.ranges, r.T_final, r.last,
                          self.loss.d_img, r.grads, d_op, None, stream, lists=r.lists)
        gs3.gs_project_bwd_full(g, cams_dev, V, W, H, r.grads, d_op, self.n_fixed, self.n_add,
                                self.d_mean, self.d_quat, self.d_scale, self.d_ologit, self.d_sh,
                                stream)
        gs3.gs_viewspace_grad_accum(r.grads, r.proj.radius, V, n, self.n_fixed, self.n_add, W, H,
                                    float(V), self.accum, self.denom, stream)
        return self.loss.d_loss

    def step(self, cams_dev, target, stream=None):
        d_loss = self.compute_grads(cams_dev, target, stream)
        gs3.gs_added_adam(self.added(), self.n_add, self.d_mean, self.d_quat, self.d_scale,
                          self.d_ologit, self.d_sh, self.lr, STAGE2_BETAS[0], STAGE2_BETAS[1],
                          STAGE2_EPS, self.state, self.view(), self.n_fixed, stream)
        gs3.gs_train_state_advance(self.state, 0, stream)
        return d_loss

    def epoch_end(self):
        """Split the added Gaussians above tau_grad (one more each: 80 % scale,
        rotation and SH inherited, opacity as a spawned Gaussian's) and
        discard those below tau_alpha; reads the new count back."""
        z = torch.randn(max(self.n_add, 1), 3, generator=self.gen, device=self.accum.device)
        gs3.gs_added_densify_prune(self.added(), self.n_add, self.accum, self.denom, self.tau_grad,
                                   self.tau_alpha, SPLIT_SCALE, SPAWN_OPACITY, z,
                                   self.added(1 - self.cur), self.d_n, self.d_err)
        self.cur = 1 - self.cur
        self.n_add = int(self.d_n.item())
        self._after_resize()
        return self.n_add

    def fit_capacity(self, cams_dev, margin=1.5):
        self.raster.fit_capacity(self.view(), cams_dev, margin=margin)

    def run(self, batches, iters: int = 100):
        """iters iterations over the view batches in turn, quantity control at
        the end of every epoch (len(batches) iterations)."""
        nb = len(batches)
        for it in range(iters):
            cd, tg = batches[it % nb]
            if it % nb == 0:
                self.fit_capacity(cd, margin=1.5)
            self.step(cd, tg)
            if (it + 1) % nb == 0 and it + 1 < iters:
                self.epoch_end()
        self.raster.check()
        if int(self.d_err.item()) != 0:
            raise gs3.GsError("Stage2", int(self.d_err.item()), "added-Gaussian capacity exceeded")
        return self.n_add


class Streamer:
    """Per-frame reconstruction of a multi-view video (Section 3): every frame
    restarts the transformation cache from its warm-up parameters, trains it
    for iters1 Stage-1 iterations (view-space statistics over the final
    epoch), carries the transformed Gaussians to the next frame, and runs
    Stage 2 (frame-specific added Gaussians, not carried) on a second CUDA
    stream, overlapped with the next frame's Stage 1.

    Per frame it records the held-out-view PSNR of the carried Gaussians
    before the frame's training and after each stage, the number of added
    Gaussians and the frame's storage: the cache parameters (FP16 table, BF16
    MLP) and the added Gaussians' rows (FP32)."""

    def __init__(self, g0: Gaussians, ntc: NTC, warm_table, warm_mlp, cams_dev, n_cams: int,
                 Vb: int, W: int, H: int, heldout_dev=None, stage2: bool = True,
                 iters1: int = 150, iters2: int = 100, added_capacity: int = 300_000,
                 device="cuda", bin: int = DEFAULT_BIN, graphs: bool = True,
                 sh_rotation: bool = True, save_dir: Optional[str] = None):
        self.frames_done = 0
        self.save_dir = save_dir
        clone = lambda t: t.clone()
        self.g = Gaussians(clone(g0.mean), clone(g0.quat), g0.scale, g0.opacity_logit, clone(g0.sh),
                           g0.sh_deg)
        self.sh_rotation = sh_rotation
        self.ntc, self.warm = ntc, (warm_table, warm_mlp)
        self.Vb, self.W, self.H = Vb, W, H
        self.nb = n_cams // Vb
        self.cams = [gs3.camera_slice(cams_dev, b * Vb, Vb) for b in range(self.nb)]
        self.heldout = heldout_dev
        self.iters1, self.iters2 = iters1, iters2
        self.st1 = Stage1(self.g, ntc, Vb, W, H, capacity=1 << 20, device=device, bin=bin)
        self.st2 = Stage2(self.g, Vb, W, H, added_capacity, pair_capacity=1 << 22, device=device,
                          bin=bin) if stage2 else None
        # frame t's views for Stage 1 (graphs read this buffer) and a copy for
        # Stage 2, which still trains frame t while Stage 1 runs frame t + 1
        self.targets = _f32(n_cams, 3, H, W, device=device)
        self.targets2 = _f32(n_cams, 3, H, W, device=device) if stage2 else None
        self.batches = [(self.cams[b], self.targets[b * Vb:(b + 1) * Vb]) for b in range(self.nb)]
        self.batches2 = ([(self.cams[b], self.targets2[b * Vb:(b + 1) * Vb]) for b in range(self.nb)]
                         if stage2 else None)
        self.side = torch.cuda.Stream() if stage2 else None
        self.use_graphs = graphs
        self.graphs = None
        self.graphs_track = None
        self.track = None

    def _stage1(self, targets):
        """Issue one frame of Stage 1 on the current stream (no host wait)."""
        st = self.st1
        self.targets.copy_(targets)
        self.ntc.reset_to(*self.warm)
        st.reset_state()
        st.refresh_order()  # the carried means moved
        if self.track is None:
            self.track = st.track_viewspace(True)
            st.track_viewspace(False)
        accum, denom = self.track
        if self.use_graphs and self.graphs is None:
            st.raster.fit_capacity(self.g, self.cams[0], *st.transform(), margin=2.0)
            self.graphs = st.capture(self.batches)
            st.track = self.track
            self.graphs_track = st.capture(self.batches)
            st.track = None
            self.ntc.reset_to(*self.warm)
            st.reset_state()
        elif not self.use_graphs and st.raster.count() == 0:
            st.raster.fit_capacity(self.g, self.cams[0], *st.transform(), margin=2.0)
        for it in range(self.iters1):
            b = it % self.nb
            final = it >= self.iters1 - self.nb
            if final and it == self.iters1 - self.nb:
                accum.zero_()
                denom.zero_()
            if self.use_graphs:
                (self.graphs_track if final else self.graphs)[b].replay()
            else:
                st.track = self.track if final else None
                st.step(*self.batches[b])
                st.track = None
        return st.transform()

    def _psnr(self, gs: Gaussians, gt_img, mean=None, quat=None):
        img = render_dev(gs, self.heldout, 1, self.W, self.H, mean, quat)
        return -10 * math.log10(float(((img - gt_img) ** 2).mean().item()))

    def run(self, frame_targets, heldout_gt=None, motion_ref=None):
        """frame_targets(t) (or a list): the [n_cams, 3, H, W] device tensor of
        frame t + 1's training views, t = 0 .. n_frames - 1; heldout_gt: per
        frame the held-out view [1, 3, H, W] (or None); motion_ref: (mean_gt,
        weight) with mean_gt(t) the ground-truth means of frame t + 1 and
        weight [n] per-Gaussian weights, to record the weighted error of the
        carried means (or None).  Returns one record per frame."""
        get = frame_targets if callable(frame_targets) else (lambda t: frame_targets[t])
        n_frames = len(heldout_gt) if heldout_gt is not None else len(frame_targets)
        records = []
        main = torch.cuda.current_stream()
        K = (self.g.sh_deg + 1) ** 2
        cache_bytes = self.ntc.entries * 2 * 2 + gs3.MLP_PARAMS * 2
        t_all = time.perf_counter()
        mt, qt = self._stage1(get(0))
        for t in range(n_frames):
            rec = {"frame": self.frames_done + 1}
            main.synchronize()  # frame t's Stage 1 is done
            # a binning overflow or a non-finite Gaussian met by the projection
            # (e.g. after a tensor-core wait gave up) ends the run loudly
            self.st1.raster.check()
            rec["tc_timeouts"] = gs3.gs_tc_timeouts()
            # the frame's cache as stored (FP16 table, BF16 MLP), before the
            # next frame's Stage 1 restarts it from the warm-up parameters
            cache = (self.ntc.table.shadow.clone(), self.ntc.mlp.shadow.clone())
            if heldout_gt is not None and self.heldout is not None:
                # the previous frame's Gaussians unchanged
                rec["psnr_carried"] = self._psnr(self.g, heldout_gt[t])
            mt_c, qt_c = mt.clone(), qt.clone()
            if self.sh_rotation:
                # the frame's rotations turn the colours too (Suppl. B)
                gs3.gs_sh_rotate(self.g.quat, qt_c, self.g.sh, self.g.n, self.g.sh_deg, self.g.sh)
            if heldout_gt is not None and self.heldout is not None:
                rec["psnr_stage1"] = self._psnr(self.g, heldout_gt[t], mt_c, qt_c)
            acc, den = self.track
            if self.st2 is not None:
                self.targets2.copy_(self.targets)
                self.side.wait_stream(main)
                with torch.cuda.stream(self.side):
                    self.st2.begin(mt_c, qt_c, acc, den)  # reads back the spawn count
            if motion_ref is not None:
                mgt, wgt = motion_ref
                err = (mt_c - mgt(t)).norm(dim=1)
                rec["motion_err_weighted"] = float((err * wgt).sum() / wgt.sum())
                rec["motion_err_carried_weighted"] = float(((self.g.mean - mgt(t)).norm(dim=1) * wgt).sum()
                                                           / wgt.sum())
            # carry the transformed Gaussians; issue the next frame's Stage 1
            self.g.mean.copy_(mt_c)
            self.g.quat.copy_(qt_c)
            if t + 1 < n_frames:
                mt, qt = self._stage1(get(t + 1))
            if self.st2 is not None:
                # frame t's Stage 2 on the side stream, overlapped with the above
                with torch.cuda.stream(self.side):
                    self.st2.run(self.batches2, iters=self.iters2)
                    if heldout_gt is not None and self.heldout is not None:
                        rec["psnr_stage2"] = self._psnr(self.st2.view(), heldout_gt[t])
                    rec["added"] = self.st2.n_add
                self.side.synchronize()
            rec["storage_bytes"] = cache_bytes + rec.get("added", 0) * 4 * (11 + 3 * K)
            if self.save_dir is not None:
                rec["file"] = self._save_frame(rec["frame"], cache)
            records.append(rec)
            self.frames_done += 1
        torch.cuda.synchronize()
        self.wall_s = time.perf_counter() - t_all
        return records


    def _save_frame(self, frame: int, cache) -> str:
        """The frame's record (what the next frame does not carry): the cache
        that transforms the previous frame's Gaussians and the frame's added
        Gaussians, as npz in save_dir."""
        import os
        os.makedirs(self.save_dir, exist_ok=True)
        path = os.path.join(self.save_dir, "frame_%05d.npz" % frame)
        added = (self.st2.rows[self.st2.cur][:self.st2.n_add].cpu().numpy()
                 if self.st2 is not None else np.zeros((0, 11 + 3 * (self.g.sh_deg + 1) ** 2), np.float32))
        np.savez(path, table_f16=cache[0].cpu().numpy(),
                 mlp_bf16=cache[1].view(torch.int16).cpu().numpy(), added_rows=added,
                 sh_deg=self.g.sh_deg)
        return path

    def checkpoint(self, path: str):
        """Everything a later run needs to continue the video from the next
        frame: the carried Gaussians (transformed means and rotations, SH as
        rotated, scales and opacities) and the cache's warm-up parameters."""
        g = self.g
        np.savez(path, frames_done=self.frames_done, mean=g.mean.cpu().numpy(),
                 quat=g.quat.cpu().numpy(), sh=g.sh.cpu().numpy(),
                 scale=g.scale.cpu().numpy(), opacity_logit=g.opacity_logit.cpu().numpy(),
                 sh_deg=g.sh_deg, warm_table=self.warm[0].cpu().numpy(),
                 warm_mlp=self.warm[1].cpu().numpy())

    def resume(self, path: str):
        """Continue from a checkpoint written by checkpoint(): every field it
        holds is restored; one of another scene (Gaussian count or SH degree)
        is refused before anything changes."""
        d = np.load(path)
        dev = self.g.mean.device
        t = lambda a: torch.from_numpy(np.ascontiguousarray(a)).to(dev)
        if int(d["sh_deg"]) != self.g.sh_deg or d["mean"].shape[0] != self.g.n:
            raise ValueError("Streamer.resume: checkpoint of %d Gaussians (SH %d), this run has %d (SH %d)"
                             % (d["mean"].shape[0], int(d["sh_deg"]), self.g.n, self.g.sh_deg))
        self.g.mean.copy_(t(d["mean"]))
        self.g.quat.copy_(t(d["quat"]))
        self.g.sh.copy_(t(d["sh"]))
        self.g.scale.copy_(t(d["scale"]))
        self.g.opacity_logit.copy_(t(d["opacity_logit"]))
        self.warm = (t(d["warm_table"]), t(d["warm_mlp"]))
        self.frames_done = int(d["frames_done"])


def render_dev(g: Gaussians, cams_dev, V: int, W: int, H: int, mean=None, quat=None,
               capacity=None, device="cuda", bin: int = DEFAULT_BIN) -> torch.Tensor:
    """Render V device cameras (one launch); returns [V, 3, H, W]."""
    r = Rasterizer(g.n, V, W, H, capacity or 1 << 20, device, bin=bin)
    r.fit_capacity(g, cams_dev, mean, quat)
    return r.img.clone()


class DirectOpt:
    """Plain FP32 direct optimisation of the previous frame's means and
    rotations (the "Direct Opt." comparator of Section 5.3), same rasterizer."""

    def __init__(self, g: Gaussians, V: int, W: int, H: int, capacity: int, lr_mean=0.0024,
                 lr_quat=0.015, device="cuda", bin: int = DEFAULT_BIN, iters: int = ITERS_PER_FRAME):
        """Rates: the paper's Stage-2 rates for means and rotations (Suppl. A)
        by default, with Stage 1's schedule and epsilon over `iters`
        iterations (the same treatment as the cache)."""
        self.g = g
        self.V, self.W, self.H = V, W, H
        self.raster = Rasterizer(g.n, V, W, H, capacity, device, bin=bin)
        self.loss = Loss(V, W, H, device)
        self.mean = AdamBuffers(g.mean.clone(), lr_mean, hp=adam_hp(lr_mean, decay_steps=iters))
        self.quat = AdamBuffers(g.quat.clone(), lr_quat, hp=adam_hp(lr_quat, decay_steps=iters))
        self.state = gs3.new_train_state(1.0, device)

    def step(self, cams_dev, target, stream=None):
        img = self.raster.forward(self.g, cams_dev, self.mean.p, self.quat.p, stream)
        self.loss(img, target, stream)
        d_mean, d_quat = self.raster.backward(self.g, cams_dev, self.loss.d_img, self.mean.p,
                                              self.quat.p, stream)
        self.mean.g.copy_(d_mean)
        self.quat.g.copy_(d_quat)
        self.mean.step(self.state, stream)
        self.quat.step(self.state, stream)
        gs3.gs_train_state_advance(self.state, 0, stream)
        return self.loss.d_loss

    def capture(self, batches):
        return capture_graphs(self.step, batches)


class TargetFeeder:
    """Training targets resident in pinned host memory, fed to the device one
    step ahead.  Batch b's targets go host -> device into dev[b] (the buffer
    its step, eager or a captured graph, reads) on a copy stream while the
    previous step runs: `before(b)` makes the compute stream wait for that
    copy, `after(b)` marks dev[b] free again and starts the copy of the next
    batch, which waits until the step that last read its buffer is done."""

    def __init__(self, host: List[torch.Tensor], dev: List[torch.Tensor]):
        if len(host) != len(dev) or not host:
            raise ValueError("TargetFeeder: one pinned host batch per device buffer")
        for h, d in zip(host, dev):
            if not h.is_pinned() or h.shape != d.shape or d.device.type != "cuda":
                raise ValueError("TargetFeeder: pinned host batches shaped like the device buffers")
        self.host, self.dev = host, dev
        self.copy_stream = torch.cuda.Stream(device=dev[0].device)
        self.ready = [torch.cuda.Event() for _ in dev]
        self.free = [torch.cuda.Event() for _ in dev]
        self.bytes_per_step = host[0].numel() * host[0].element_size()

    def _copy(self, b: int):
        with torch.cuda.stream(self.copy_stream):
            self.copy_stream.wait_event(self.free[b])
            self.dev[b].copy_(self.host[b], non_blocking=True)
            self.ready[b].record(self.copy_stream)

    def start(self, b: int, stream=None):
        """Record every buffer free on `stream` and copy batch b."""
        stream = stream or torch.cuda.current_stream()
        for e in self.free:
            e.record(stream)
        self._copy(b)

    def before(self, b: int, stream=None):
        (stream or torch.cuda.current_stream()).wait_event(self.ready[b])

    def after(self, b: int, next_b: int, stream=None):
        self.free[b].record(stream or torch.cuda.current_stream())
        self._copy(next_b)


def capture_graphs(step_fn, batches):
    side = torch.cuda.Stream()
    side.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(side):
        for cd, tg in batches:
            step_fn(cd, tg)
    torch.cuda.current_stream().wait_stream(side)
    graphs = []
    for cd, tg in batches:
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g):
            step_fn(cd, tg)
        graphs.append(g)
    torch.cuda.synchronize()
    return graphs


def warmup(ntc: NTC, g: Gaussians, iters=3000, noise=0.01, extent=2.0, seed=0, stream=None,
           loss_scale=None):
    """NTC warm-up (Eq. 7): train towards the identity transformation on
    noise-augmented means; returns the final loss."""
    n = g.n
    gen = torch.Generator(device=g.mean.device)
    gen.manual_seed(seed)
    enc = torch.zeros(n, 32, dtype=ntc.enc_dtype(), device=g.mean.device)
    raw7 = _f32(n, 7, device=g.mean.device)
    d_raw7 = _f32(n, 7, device=g.mean.device)
    d_enc = _f32(n, 32, device=g.mean.device)
    d_loss = _f32(1, device=g.mean.device)
    if loss_scale is None:
        loss_scale = 2.0 ** 15 if ntc.precision == gs3.GS_MLP_BF16 else 1.0
    state = gs3.new_train_state(loss_scale, g.mean.device)
    scale_view = state[0:4].view(torch.float32)
    mu = torch.empty_like(g.mean)
    # the noisy means stay near the Gaussians: their spatial order serves
    visit = gs3.spatial_order(g.mean, n, ntc.grid, stream)
    for _ in range(iters):
        # the noise the method draws is an input of the kernels
        torch.randn(mu.shape, generator=gen, device=mu.device, out=mu)
        mu.mul_(noise * extent).add_(g.mean)
        gs3.ntc_encode_fwd(mu, n, ntc.grid, ntc.table_for_encode(), enc, stream, order=visit)
        gs3.ntc_mlp_fwd(enc, n, ntc.mlp_struct(), raw7, stream)
        gs3.ntc_warmup_loss(raw7, n, d_raw7, d_loss, stream)
        gs3.ntc_mlp_bwd(enc, n, ntc.mlp_struct(), d_raw7, scale_view, ntc.mlp.g, d_enc, stream)
        gs3.ntc_encode_bwd(mu, n, ntc.grid, d_enc, ntc.table.g, stream)
        gs3.gs_check_finite(ntc.table.g, state, stream)
        gs3.gs_check_finite(ntc.mlp.g, state, stream)
        ntc.table.step(state, stream, ntc.warm_hp)
        ntc.mlp.step(state, stream, ntc.warm_hp)
        gs3.gs_train_state_advance(state, 2000, stream)
    return float(d_loss.item())


class Renderer:
    """Render-only path (Section 5.4's rendering of a streamed frame): NTC
    query of the frozen means, transformation, projection, binning and
    compositing of V views into a device buffer, with no backward.  capture()
    records one frame as a CUDA graph, the headless analogue of the viewer's
    per-frame work."""

    def __init__(self, g: Gaussians, ntc: NTC, V: int, W: int, H: int, capacity: int,
                 order: int = 0, device="cuda", bin: int = DEFAULT_BIN, sh_rotation: bool = True):
        n = g.n
        self.g, self.ntc, self.V, self.W, self.H, self.order = g, ntc, V, W, H, order
        self.raster = Rasterizer(n, V, W, H, capacity, device, bin=bin)
        # SH rotation (Suppl. B): the colours turn with the Gaussians
        self.sh_rot = torch.empty_like(g.sh) if sh_rotation else None
        self.g_rot = (Gaussians(g.mean, g.quat, g.scale, g.opacity_logit, self.sh_rot, g.sh_deg)
                      if sh_rotation else g)
        self.enc = torch.zeros(n, 32, dtype=ntc.enc_dtype(), device=device)
        self.visit = gs3.spatial_order(g.mean, n, ntc.grid)  # the Gaussians are fixed
        self.raw7 = _f32(n, 7, device=device)
        self.mean_t = _f32(n, 3, device=device)
        self.quat_t = _f32(n, 4, device=device)
        self.aabb = list(ntc.grid.aabb)

    def frame(self, cams_dev, stream=None):
        g, ntc, n = self.g, self.ntc, self.g.n
        gs3.ntc_encode_fwd(g.mean, n, ntc.grid, ntc.table_for_encode(), self.enc, stream, order=self.visit)
        gs3.ntc_mlp_fwd(self.enc, n, ntc.mlp_struct(), self.raw7, stream)
        gs3.ntc_apply(g.mean, g.quat, self.raw7, n, self.aabb, self.order, self.mean_t, self.quat_t,
                      stream)
        if self.sh_rot is not None:
            gs3.gs_sh_rotate(g.quat, self.quat_t, g.sh, n, g.sh_deg, self.sh_rot, stream)
        return self.raster.forward(self.g_rot, cams_dev, self.mean_t, self.quat_t, stream, lists=False)

    def capture(self, cams_dev):
        side = torch.cuda.Stream()
        side.wait_stream(torch.cuda.current_stream())
        with torch.cuda.stream(side):
            self.frame(cams_dev)
        torch.cuda.current_stream().wait_stream(side)
        graph = torch.cuda.CUDAGraph()
        with torch.cuda.graph(graph):
            self.frame(cams_dev)
        torch.cuda.synchronize()
        return graph


def autotune_bin(g: Gaussians, cams_dev, V: int, W: int, H: int, mean=None, quat=None,
                 candidates=(1, 2, 4, 8, 16), backward=True, iters=5, device="cuda"):
    """Time projection + binning + compositing (and, with backward=True, the
    reverse of compositing and projection under a constant image gradient) at
    each bin size (bins of S x S 16-pixel tiles); returns ({S: ms}, best S).
    Every bin size composites the same records in the same order, so the
    choice changes the time only."""
    times = {}
    stream = torch.cuda.current_stream()
    for S in candidates:
        r = Rasterizer(g.n, V, W, H, 1 << 20, device, bin=S)
        r.fit_capacity(g, cams_dev, mean, quat, margin=1.2)
        d_img = torch.full_like(r.img, 1e-3)

        def once():
            r.forward(g, cams_dev, mean, quat)
            if backward:
                r.backward(g, cams_dev, d_img, mean, quat)

        once()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(iters):
            once()
        e1.record(stream)
        torch.cuda.synchronize()
        r.check()
        times[S] = e0.elapsed_time(e1) / iters
        del r, d_img
    return times, min(times, key=times.get)


def render(g: Gaussians, cams, W: int, H: int, mean=None, quat=None, capacity=None,
           device="cuda", bin: int = DEFAULT_BIN) -> torch.Tensor:
    """Render all cams (one launch) with the CUDA rasterizer; returns [V,3,H,W]."""
    cams_dev = gs3.cameras_to_device(cams, device)
    r = Rasterizer(g.n, len(cams), W, H, capacity or 1 << 20, device, bin=bin)
    r.fit_capacity(g, cams_dev, mean, quat)
    return r.img.clone()
