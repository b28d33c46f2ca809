"""Thin ctypes binding of libgs3 (include/gs3.h): argument marshalling only.

Each function here has the name of the C entry point it calls and takes
torch CUDA tensors (or plain ints/floats) in place of raw pointers; every
step of the computation runs in the CUDA library.  The library is loaded
from this package directory; if it is missing the import of a compute call
raises -- there is no fallback path.
"""
from __future__ import annotations

import ctypes
import dataclasses
import os
from typing import Optional, Sequence

import numpy as np
import torch

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libgs3.so")

GS_OK, GS_ERR_INVALID_ARG, GS_ERR_CAPACITY, GS_ERR_CUDA, GS_ERR_TIMEOUT, GS_ERR_NONFINITE = 0, -1, -2, -3, -4, -5
GS_F32, GS_F16, GS_BF16, GS_NONE = 0, 1, 2, 3
GS_MLP_FP32, GS_MLP_BF16 = 0, 1
MLP_PARAMS = 64 * 32 + 64 * 64 + 7 * 64
TILE = 16


def bins_of(W, H, bin):
    """Number of bins (of bin x bin tiles) of a W x H view."""
    tx, ty = (W + TILE - 1) // TILE, (H + TILE - 1) // TILE
    return ((tx + bin - 1) // bin) * ((ty + bin - 1) // bin)

c_void_p, c_int, c_int32, c_int64, c_float, c_size_t = (
    ctypes.c_void_p, ctypes.c_int, ctypes.c_int32, ctypes.c_int64, ctypes.c_float, ctypes.c_size_t)


class GsError(RuntimeError):
    def __init__(self, name, status, msg):
        super().__init__("%s failed with status %d: %s" % (name, status, msg))
        self.status = status


class GsGaussians(ctypes.Structure):
    _fields_ = [("mean", c_void_p), ("quat", c_void_p), ("scale", c_void_p),
                ("opacity_logit", c_void_p), ("sh", c_void_p), ("n", c_int64), ("sh_deg", c_int32)]


class GsCamera(ctypes.Structure):
    _fields_ = [("viewmat", c_float * 12), ("fx", c_float), ("fy", c_float), ("cx", c_float),
                ("cy", c_float), ("width", c_int32), ("height", c_int32), ("campos", c_float * 3)]


class GsProjected(ctypes.Structure):
    _fields_ = [("mean2d", c_void_p), ("conic_opacity", c_void_p), ("rgb", c_void_p),
                ("depth", c_void_p), ("radius", c_void_p), ("tiles_touched", c_void_p)]


class GsTileLists(ctypes.Structure):
    _fields_ = [("rec", c_void_p), ("count", c_void_p), ("cap", ctypes.c_int32)]


class GsHashgrid(ctypes.Structure):
    _fields_ = [("levels", c_int32), ("features", c_int32), ("log2_table", c_int32),
                ("n_min", c_int32), ("n_max", c_int32), ("aabb", c_float * 6)]


class GsMlp(ctypes.Structure):
    _fields_ = [("precision", c_int32), ("w_f32", c_void_p), ("w_bf16", c_void_p)]


class GsAdam(ctypes.Structure):
    _fields_ = [("lr", c_float), ("beta1", c_float), ("beta2", c_float), ("eps", c_float),
                ("lr_final_ratio", c_float), ("decay_steps", ctypes.c_int32)]


class GsAdded(ctypes.Structure):
    _fields_ = [("rows", c_void_p), ("m", c_void_p), ("v", c_void_p), ("capacity", c_int64),
                ("sh_deg", c_int32)]


def added_cols(sh_deg: int) -> int:
    """Floats per row of an added Gaussian: mean 3, quat 4, log scale 3, opacity logit 1, SH."""
    return 11 + 3 * (sh_deg + 1) ** 2


class GsTrainState(ctypes.Structure):
    _fields_ = [("loss_scale", c_float), ("found_inf", c_int32), ("step", c_int32),
                ("clean_steps", c_int32)]


_lib = None


def lib():
    """Load libgs3.so (built by paper_2403_01444_gb300.build); raise if absent."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError("libgs3.so is not built (%s); run __graft_entry__.build()" % LIB_PATH)
        L = ctypes.CDLL(LIB_PATH)
        for name in ("gs_bin_sort_workspace_size", "gs_loss_workspace_size"):
            getattr(L, name).restype = c_size_t
        L.gs_bin_sort_workspace_size.argtypes = [c_int64, c_int, c_int, c_int, c_int64]
        L.gs_loss_workspace_size.argtypes = [c_int, c_int, c_int]
        L.ntc_hashgrid_entries.restype = c_int64
        L.gs_last_error.restype = ctypes.c_char_p
        _lib = L
    return _lib


def _check(name, st):
    if st != GS_OK:
        raise GsError(name, st, lib().gs_last_error().decode(errors="replace"))


def _ptr(t: Optional[torch.Tensor]):
    if t is None:
        return None
    if not (t.is_cuda and t.is_contiguous()):
        raise ValueError("expected a contiguous CUDA tensor, got %s on %s%s"
                         % (t.dtype, t.device, "" if t.is_contiguous() else " (not contiguous)"))
    return c_void_p(t.data_ptr())


def _stream(stream=None):
    s = stream if stream is not None else torch.cuda.current_stream()
    return c_void_p(s.cuda_stream)


# ------------------------------------------------------------------ structs
@dataclasses.dataclass
class Gaussians:
    """Device Gaussian set (float32, contiguous)."""

    mean: torch.Tensor
    quat: torch.Tensor
    scale: torch.Tensor
    opacity_logit: torch.Tensor
    sh: torch.Tensor
    sh_deg: int

    @property
    def n(self) -> int:
        return int(self.mean.shape[0])

    @staticmethod
    def from_numpy(g, device="cuda") -> "Gaussians":
        t = lambda a: torch.from_numpy(np.ascontiguousarray(a, np.float32)).to(device)
        return Gaussians(t(g.mean), t(g.quat), t(g.scale), t(g.opacity_logit), t(g.sh), int(g.sh_deg))

    def struct(self, mean=None, quat=None) -> GsGaussians:
        m = self.mean if mean is None else mean
        q = self.quat if quat is None else quat
        return GsGaussians(_ptr(m), _ptr(q), _ptr(self.scale), _ptr(self.opacity_logit),
                           _ptr(self.sh), self.n, self.sh_deg)


def cameras_to_device(cams, device="cuda") -> torch.Tensor:
    """Pack cameras (objects with viewmat, fx, fy, cx, cy, W, H, campos) into a
    device byte tensor laid out as gs_camera[V]."""
    arr = (GsCamera * len(cams))()
    for i, c in enumerate(cams):
        vm = np.asarray(c.viewmat, np.float32).reshape(12)
        arr[i].viewmat[:] = [float(x) for x in vm]
        arr[i].fx, arr[i].fy, arr[i].cx, arr[i].cy = float(c.fx), float(c.fy), float(c.cx), float(c.cy)
        arr[i].width, arr[i].height = int(c.W), int(c.H)
        arr[i].campos[:] = [float(x) for x in np.asarray(c.campos, np.float32)]
    buf = torch.frombuffer(bytearray(bytes(arr)), dtype=torch.uint8)
    return buf.to(device)


def camera_slice(cams_dev: torch.Tensor, start: int, count: int) -> torch.Tensor:
    sz = ctypes.sizeof(GsCamera)
    return cams_dev[start * sz:(start + count) * sz]


@dataclasses.dataclass
class Projected:
    mean2d: torch.Tensor         # [V, N, 2]
    conic_opacity: torch.Tensor  # [V, N, 4]
    rgb: torch.Tensor            # [V, N, 3]
    depth: torch.Tensor          # [V, N]
    radius: torch.Tensor         # [V, N] int32
    tiles_touched: torch.Tensor  # [V, N] int32

    @staticmethod
    def empty(V, N, device="cuda") -> "Projected":
        f = dict(device=device, dtype=torch.float32)
        i = dict(device=device, dtype=torch.int32)
        return Projected(torch.empty(V, N, 2, **f), torch.empty(V, N, 4, **f), torch.empty(V, N, 3, **f),
                         torch.empty(V, N, **f), torch.empty(V, N, **i), torch.empty(V, N, **i))

    def struct(self) -> GsProjected:
        return GsProjected(_ptr(self.mean2d), _ptr(self.conic_opacity), _ptr(self.rgb),
                           _ptr(self.depth), _ptr(self.radius), _ptr(self.tiles_touched))


def hashgrid(levels=16, features=2, log2_table=17, n_min=16, n_max=1024,
             aabb=(-1.5, -1.5, -1.5, 1.5, 1.5, 1.5)) -> GsHashgrid:
    g = GsHashgrid(levels, features, log2_table, n_min, n_max)
    g.aabb[:] = [float(x) for x in aabb]
    return g


def mlp_struct(precision: int, w_f32: torch.Tensor, w_bf16: Optional[torch.Tensor] = None) -> GsMlp:
    s = GsMlp(precision, _ptr(w_f32), _ptr(w_bf16))
    s._keep = (w_f32, w_bf16)  # the struct holds raw pointers: keep the tensors alive with it
    return s


# ------------------------------------------------------------------ calls
def gs_project(g: Gaussians, cams_dev, V, W, H, out: Projected, mean=None, quat=None, stream=None,
               d_err=None):
    gg = g.struct(mean, quat)
    po = out.struct()
    _check("gs_project", lib().gs_project(ctypes.byref(gg), _ptr(cams_dev), c_int(V), c_int(W),
                                          c_int(H), ctypes.byref(po), _ptr(d_err), _stream(stream)))


def gs_project_bwd(g: Gaussians, cams_dev, V, W, H, grads, d_mean, d_quat, mean=None, quat=None,
                   stream=None):
    gg = g.struct(mean, quat)
    _check("gs_project_bwd", lib().gs_project_bwd(ctypes.byref(gg), _ptr(cams_dev), c_int(V), c_int(W),
                                                  c_int(H), _ptr(grads), _ptr(d_mean), _ptr(d_quat),
                                                  _stream(stream)))


def gs_project_bwd_full(g: Gaussians, cams_dev, V, W, H, grads, d_opacity, first, count, d_mean,
                        d_quat, d_scale, d_opacity_logit, d_sh, stream=None):
    gg = g.struct()
    _check("gs_project_bwd_full", lib().gs_project_bwd_full(
        ctypes.byref(gg), _ptr(cams_dev), c_int(V), c_int(W), c_int(H), _ptr(grads), _ptr(d_opacity),
        c_int64(first), c_int64(count), _ptr(d_mean), _ptr(d_quat), _ptr(d_scale),
        _ptr(d_opacity_logit), _ptr(d_sh), _stream(stream)))


def gs_bin_sort_workspace_size(n, V, W, H, capacity) -> int:
    return int(lib().gs_bin_sort_workspace_size(n, V, W, H, capacity))


def gs_bin_sort(proj: Projected, n, V, W, H, bin, capacity, vals, ranges, keys, d_count, d_err, ws,
                stream=None):
    po = proj.struct()
    _check("gs_bin_sort", lib().gs_bin_sort(
        ctypes.byref(po), c_int64(n), c_int(V), c_int(W), c_int(H), c_int(bin), c_int64(capacity), _ptr(vals),
        _ptr(ranges), _ptr(keys), _ptr(d_count), _ptr(d_err), _ptr(ws), c_size_t(ws.numel()),
        _stream(stream)))


def gs_bin_sort_noalloc(proj: Projected, n, V, W, H, bin, capacity, vals, ranges, keys, d_count,
                        d_err, stream=None):
    """gs_bin_sort with the library's built-in scratch (no workspace argument):
    for callers that cannot allocate device memory.  Limits and sharing rules
    are those of the C entry point."""
    po = proj.struct()
    _check("gs_bin_sort_noalloc", lib().gs_bin_sort_noalloc(
        ctypes.byref(po), c_int64(n), c_int(V), c_int(W), c_int(H), c_int(bin), c_int64(capacity), _ptr(vals),
        _ptr(ranges), _ptr(keys), _ptr(d_count), _ptr(d_err), _stream(stream)))


def _bg(bg):
    a = (c_float * 3)(*[float(x) for x in (bg if bg is not None else (0.0, 0.0, 0.0))])
    return a


class TileLists:
    """gs_tile_lists: each tile's staged records (Gaussian, list position),
    written by gs_raster_fwd and read by gs_raster_bwd; cap records a tile."""

    def __init__(self, V: int, W: int, H: int, cap: int = 1024, device="cuda"):
        tiles = ((W + 15) // 16) * ((H + 15) // 16)
        self.cap = int(cap)
        self.rec = torch.zeros(V * tiles * self.cap * 2, dtype=torch.int32, device=device)
        self.count = torch.full((V * tiles,), -1, dtype=torch.int32, device=device)

    def struct(self) -> GsTileLists:
        return GsTileLists(_ptr(self.rec), _ptr(self.count), self.cap)


def _lists(lists: Optional[TileLists]):
    return None if lists is None else ctypes.byref(lists.struct())


def gs_raster_fwd(proj: Projected, n, V, W, H, bin, bg, vals, ranges, img, T_final, last,
                  stats=None, stream=None, lists: Optional[TileLists] = None):
    po = proj.struct()
    tl = _lists(lists)
    _check("gs_raster_fwd", lib().gs_raster_fwd(
        ctypes.byref(po), c_int64(n), c_int(V), c_int(W), c_int(H), c_int(bin), _bg(bg), _ptr(vals), _ptr(ranges),
        _ptr(img), _ptr(T_final), _ptr(last), _ptr(stats), tl, _stream(stream)))


def gs_raster_bwd(proj: Projected, n, V, W, H, bin, bg, vals, ranges, T_final, last, d_img, grads,
                  d_opacity=None, stats=None, stream=None, lists: Optional[TileLists] = None):
    po = proj.struct()
    tl = _lists(lists)
    _check("gs_raster_bwd", lib().gs_raster_bwd(
        ctypes.byref(po), c_int64(n), c_int(V), c_int(W), c_int(H), c_int(bin), _bg(bg), _ptr(vals), _ptr(ranges),
        _ptr(T_final), _ptr(last), _ptr(d_img), _ptr(grads), _ptr(d_opacity), _ptr(stats), tl,
        _stream(stream)))


def gs_loss_workspace_size(planes, H, W) -> int:
    return int(lib().gs_loss_workspace_size(planes, H, W))


def gs_loss_l1_dssim(img, target, planes, H, W, lam, d_img, d_loss, d_ssim, ws, stream=None):
    _check("gs_loss_l1_dssim", lib().gs_loss_l1_dssim(
        _ptr(img), _ptr(target), c_int(planes), c_int(H), c_int(W), c_float(lam), _ptr(d_img),
        _ptr(d_loss), _ptr(d_ssim), _ptr(ws), c_size_t(ws.numel()), _stream(stream)))


def ntc_hashgrid_entries(grid: GsHashgrid) -> int:
    return int(lib().ntc_hashgrid_entries(ctypes.byref(grid)))


_DT = {torch.float32: GS_F32, torch.float16: GS_F16, torch.bfloat16: GS_BF16}


def ntc_encode_fwd(mean, n, grid: GsHashgrid, table, enc, stream=None, order=None):
    _check("ntc_encode_fwd", lib().ntc_encode_fwd(
        _ptr(mean), c_int64(n), ctypes.byref(grid), _ptr(table), c_int(_DT[table.dtype]), _ptr(enc),
        c_int(_DT[enc.dtype]), _ptr(order), _stream(stream)))


def ntc_encode_bwd(mean, n, grid: GsHashgrid, d_enc, d_table, stream=None, order=None, d_count=None):
    _check("ntc_encode_bwd", lib().ntc_encode_bwd(
        _ptr(mean), c_int64(n), ctypes.byref(grid), _ptr(d_enc), _ptr(d_table), _ptr(order), _ptr(d_count),
        _stream(stream)))


def ntc_active_rows(d_raw7, n, rows, d_count, stream=None):
    _check("ntc_active_rows", lib().ntc_active_rows(_ptr(d_raw7), c_int64(n), _ptr(rows), _ptr(d_count),
                                                    _stream(stream)))


def ntc_spatial_order_workspace_size(n) -> int:
    L = lib()
    L.ntc_spatial_order_workspace_size.restype = ctypes.c_size_t
    return int(L.ntc_spatial_order_workspace_size(c_int64(n)))


def ntc_spatial_order(mean, n, grid: GsHashgrid, order, ws, stream=None):
    _check("ntc_spatial_order", lib().ntc_spatial_order(
        _ptr(mean), c_int64(n), ctypes.byref(grid), _ptr(order), _ptr(ws), ctypes.c_size_t(ws.numel()),
        _stream(stream)))


def spatial_order(mean, n, grid: GsHashgrid, stream=None):
    """ntc_spatial_order of the first n means into a new int32[n] tensor
    (the order's device words)."""
    order = torch.empty(max(n, 1), dtype=torch.int32, device=mean.device)
    ws = torch.empty(max(ntc_spatial_order_workspace_size(n), 1), dtype=torch.uint8, device=mean.device)
    ntc_spatial_order(mean, n, grid, order, ws, stream)
    return order[:n]


def ntc_mlp_fwd(enc, n, mlp: GsMlp, raw7, stream=None):
    _check("ntc_mlp_fwd", lib().ntc_mlp_fwd(_ptr(enc), c_int(_DT[enc.dtype]), c_int64(n),
                                            ctypes.byref(mlp), _ptr(raw7), _stream(stream)))


def ntc_mlp_bwd(enc, n, mlp: GsMlp, d_raw7, d_scale, dW, d_enc, stream=None, rows=None, d_rows=None):
    _check("ntc_mlp_bwd", lib().ntc_mlp_bwd(
        _ptr(enc), c_int(_DT[enc.dtype]), c_int64(n), ctypes.byref(mlp), _ptr(d_raw7), _ptr(d_scale),
        _ptr(dW), _ptr(d_enc), _ptr(rows), _ptr(d_rows), _stream(stream)))


def _aabb(aabb):
    return (c_float * 6)(*[float(x) for x in aabb])


def ntc_apply(mean, quat, raw7, n, aabb, order, mean_out, quat_out, stream=None):
    _check("ntc_apply", lib().ntc_apply(_ptr(mean), _ptr(quat), _ptr(raw7), c_int64(n), _aabb(aabb),
                                        c_int(order), _ptr(mean_out), _ptr(quat_out), _stream(stream)))


def ntc_apply_bwd(mean, quat, raw7, n, aabb, order, d_mean_out, d_quat_out, d_raw7, stream=None):
    _check("ntc_apply_bwd", lib().ntc_apply_bwd(
        _ptr(mean), _ptr(quat), _ptr(raw7), c_int64(n), _aabb(aabb), c_int(order), _ptr(d_mean_out),
        _ptr(d_quat_out), _ptr(d_raw7), _stream(stream)))


def ntc_fused_fwd(mean, quat, n, grid: GsHashgrid, table_f16, mlp: GsMlp, order, mean_out, quat_out,
                  raw7, enc_save, stream=None):
    _check("ntc_fused_fwd", lib().ntc_fused_fwd(
        _ptr(mean), _ptr(quat), c_int64(n), ctypes.byref(grid), _ptr(table_f16), ctypes.byref(mlp),
        c_int(order), _ptr(mean_out), _ptr(quat_out), _ptr(raw7), _ptr(enc_save), _stream(stream)))


def ntc_fused_bwd(mean, quat, raw7, enc_save, n, grid: GsHashgrid, mlp: GsMlp, order, d_mean_out,
                  d_quat_out, d_scale, dW, d_table, stream=None):
    _check("ntc_fused_bwd", lib().ntc_fused_bwd(
        _ptr(mean), _ptr(quat), _ptr(raw7), _ptr(enc_save), c_int64(n), ctypes.byref(grid),
        ctypes.byref(mlp), c_int(order), _ptr(d_mean_out), _ptr(d_quat_out), _ptr(d_scale), _ptr(dW),
        _ptr(d_table), _stream(stream)))


def ntc_warmup_loss(raw7, n, d_raw7, d_loss, stream=None):
    _check("ntc_warmup_loss", lib().ntc_warmup_loss(_ptr(raw7), c_int64(n), _ptr(d_raw7), _ptr(d_loss),
                                                    _stream(stream)))


def gs_check_finite(g, d_state, stream=None):
    _check("gs_check_finite", lib().gs_check_finite(_ptr(g), c_int64(g.numel()), _ptr(d_state),
                                                    _stream(stream)))


def adam_step(p, g, m, v, hp: GsAdam, d_state, shadow=None, stream=None):
    sd = GS_NONE if shadow is None else _DT[shadow.dtype]
    _check("adam_step", lib().adam_step(_ptr(p), _ptr(g), _ptr(m), _ptr(v), c_int64(p.numel()),
                                        ctypes.byref(hp), _ptr(d_state), _ptr(shadow), c_int(sd),
                                        _stream(stream)))


def gs_train_state_advance(d_state, growth_interval, stream=None):
    _check("gs_train_state_advance", lib().gs_train_state_advance(_ptr(d_state), c_int(growth_interval),
                                                                  _stream(stream)))


def new_train_state(loss_scale=2.0 ** 15, device="cuda") -> torch.Tensor:
    """A gs_train_state in device memory (16 bytes)."""
    st = GsTrainState(loss_scale, 0, 0, 0)
    return torch.frombuffer(bytearray(bytes(st)), dtype=torch.uint8).to(device)


def read_train_state(d_state: torch.Tensor) -> GsTrainState:
    b = bytes(d_state.cpu().numpy().tobytes())
    return GsTrainState.from_buffer_copy(b)


# ------------------------------------------------------------------ Stage 2
def added_struct(rows, m, v, sh_deg) -> GsAdded:
    s = GsAdded(_ptr(rows), _ptr(m), _ptr(v), int(rows.shape[0]), int(sh_deg))
    s._keep = (rows, m, v)
    return s


def gs_viewspace_grad_accum(grads, radius, V, n, first, count, W, H, grad_scale, accum, denom,
                            stream=None):
    _check("gs_viewspace_grad_accum", lib().gs_viewspace_grad_accum(
        _ptr(grads), _ptr(radius), c_int(V), c_int64(n), c_int64(first), c_int64(count), c_int(W),
        c_int(H), c_float(grad_scale), _ptr(accum), _ptr(denom), _stream(stream)))


def gs_select_above(accum, denom, count, tau, idx, d_nsel, stream=None):
    _check("gs_select_above", lib().gs_select_above(
        _ptr(accum), _ptr(denom), c_int64(count), c_float(tau), _ptr(idx), _ptr(d_nsel),
        _stream(stream)))


def gs_added_spawn(src: Gaussians, idx, d_nsel, z, opacity_init, dst: GsAdded, d_nadd, d_err,
                   stream=None):
    gg = src.struct()
    _check("gs_added_spawn", lib().gs_added_spawn(
        ctypes.byref(gg), _ptr(idx), _ptr(d_nsel), _ptr(z), c_float(opacity_init), ctypes.byref(dst),
        _ptr(d_nadd), _ptr(d_err), _stream(stream)))


def gs_added_densify_prune(src: GsAdded, n_src, accum, denom, tau_grad, tau_opacity, split_scale,
                           opacity_init, z, dst: GsAdded, d_ndst, d_err, stream=None):
    _check("gs_added_densify_prune", lib().gs_added_densify_prune(
        ctypes.byref(src), c_int64(n_src), _ptr(accum), _ptr(denom), c_float(tau_grad),
        c_float(tau_opacity), c_float(split_scale), c_float(opacity_init), _ptr(z), ctypes.byref(dst),
        _ptr(d_ndst), _ptr(d_err), _stream(stream)))


def gs_added_adam(a: GsAdded, n, d_mean, d_quat, d_scale, d_opacity_logit, d_sh, lr, beta1, beta2,
                  eps, d_state, out: Gaussians, out_first, stream=None):
    lr6 = (c_float * 6)(*[float(x) for x in lr])
    gg = out.struct()
    _check("gs_added_adam", lib().gs_added_adam(
        ctypes.byref(a), c_int64(n), _ptr(d_mean), _ptr(d_quat), _ptr(d_scale), _ptr(d_opacity_logit),
        _ptr(d_sh), lr6, c_float(beta1), c_float(beta2), c_float(eps), _ptr(d_state), ctypes.byref(gg),
        c_int64(out_first), _stream(stream)))


def gs_added_to_render(a: GsAdded, n, out: Gaussians, out_first, stream=None):
    gg = out.struct()
    _check("gs_added_to_render", lib().gs_added_to_render(
        ctypes.byref(a), c_int64(n), ctypes.byref(gg), c_int64(out_first), _stream(stream)))


def gs_sh_rotate(quat_from, quat_to, sh_in, n, sh_deg, sh_out, stream=None):
    _check("gs_sh_rotate", lib().gs_sh_rotate(_ptr(quat_from), _ptr(quat_to), _ptr(sh_in), c_int64(n),
                                              c_int(sh_deg), _ptr(sh_out), _stream(stream)))


def gs_tc_set_wait_limit(tries: int):
    _check("gs_tc_set_wait_limit", lib().gs_tc_set_wait_limit(ctypes.c_uint32(tries)))


GS_TC_WAIT_TRIES_DEFAULT = 4194304


def gs_tc_timeouts() -> int:
    return int(lib().gs_tc_timeouts())


def gs_tc_wait_selftest(tries, d_status, stream=None):
    _check("gs_tc_wait_selftest", lib().gs_tc_wait_selftest(ctypes.c_uint32(tries), _ptr(d_status),
                                                            _stream(stream)))

