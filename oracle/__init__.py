"""FP64 CPU oracle for the Stage-1 training step (TEST INFRASTRUCTURE ONLY).

Only the tests, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  It wraps ``liborc.so`` (plain C,
double precision, built from ``gs3_oracle.c`` by :func:`build`) with ctypes
and composes its functions into the whole step.  It shares no code with the
CUDA library and imports nothing from the product package.

Citations (paper sections / equations) are given in the C source beside each
function; this file only marshals arrays.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from typing import Dict, List, Optional, Sequence

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "gs3_oracle.c")
_LIB = os.path.join(_HERE, "liborc.so")
_lib = None

TILE = 16


def build(force: bool = False) -> str:
    """Compile liborc.so with gcc (OpenMP, no FMA contraction)."""
    if (not force and os.path.exists(_LIB)
            and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC)):
        return _LIB
    tmp = _LIB + ".tmp%d" % os.getpid()
    cmd = ["gcc", "-O2", "-fopenmp", "-fPIC", "-shared", "-ffp-contract=off",
           "-std=c11", "-o", tmp, _SRC, "-lm"]
    subprocess.check_call(cmd)
    os.replace(tmp, _LIB)
    return _LIB


def lib():
    global _lib
    if _lib is None:
        build()
        _lib = ctypes.CDLL(_LIB)
        _lib.orc_grid_levels.restype = ctypes.c_int64
        _lib.orc_corner_index.restype = ctypes.c_int64
        _lib.orc_bin_sort.restype = ctypes.c_int64
        _lib.orc_loss_l1_dssim.restype = ctypes.c_double
        _lib.orc_warmup_loss.restype = ctypes.c_double
        _lib.orc_num_threads.restype = ctypes.c_int
    return _lib


def num_threads() -> int:
    return int(lib().orc_num_threads())


# ---------------------------------------------------------------- helpers
def _d(a) -> np.ndarray:
    return np.ascontiguousarray(a, dtype=np.float64)


def _p(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


I64 = ctypes.c_int64
I32 = ctypes.c_int
F64 = ctypes.c_double


# ---------------------------------------------------------------- hash grid
class Grid:
    """Hash-grid layout: L levels, F features, T = 2^log2T, Nmin..Nmax, AABB."""

    def __init__(self, L=16, F=2, log2T=17, Nmin=16, Nmax=1024,
                 aabb=(-1.5, -1.5, -1.5, 1.5, 1.5, 1.5)):
        self.L, self.F, self.log2T, self.Nmin, self.Nmax = L, F, log2T, Nmin, Nmax
        self.aabb = _d(aabb)
        self.res = np.zeros(L, np.int32)
        self.offset = np.zeros(L, np.int64)
        self.dense = np.zeros(L, np.int32)
        self.n_entries = int(lib().orc_grid_levels(I32(L), I32(Nmin), I32(Nmax), I32(log2T),
                                                   _p(self.res), _p(self.offset), _p(self.dense)))


def corner_index(n: int, dense: int, log2T: int, x: int, y: int, z: int) -> int:
    return int(lib().orc_corner_index(I32(n), I32(dense), I32(log2T), I64(x), I64(y), I64(z)))


def encode(grid: Grid, mean, table) -> np.ndarray:
    mean, table = _d(mean), _d(table)
    N = mean.shape[0]
    enc = np.zeros((N, grid.L * grid.F))
    lib().orc_encode(_p(mean), I64(N), I32(grid.L), I32(grid.F), I32(grid.log2T), _p(grid.res),
                     _p(grid.offset), _p(grid.dense), _p(grid.aabb), _p(table), _p(enc))
    return enc


def encode_bwd(grid: Grid, mean, d_enc) -> np.ndarray:
    mean, d_enc = _d(mean), _d(d_enc)
    N = mean.shape[0]
    d_table = np.zeros((grid.n_entries, grid.F))
    lib().orc_encode_bwd(_p(mean), I64(N), I32(grid.L), I32(grid.F), I32(grid.log2T),
                         _p(grid.res), _p(grid.offset), _p(grid.dense), _p(grid.aabb),
                         _p(d_enc), _p(d_table))
    return d_table


# ---------------------------------------------------------------- MLP
def mlp_fwd(enc, Ws: Sequence[np.ndarray]):
    enc = _d(enc)
    W1, W2, W3 = (_d(w) for w in Ws)
    N, din = enc.shape
    dh, dout = W1.shape[0], W3.shape[0]
    h1, h2, out = np.zeros((N, dh)), np.zeros((N, dh)), np.zeros((N, dout))
    lib().orc_mlp_fwd(_p(enc), I64(N), I32(din), I32(dh), I32(dout), _p(W1), _p(W2), _p(W3),
                      _p(h1), _p(h2), _p(out))
    return h1, h2, out


def mlp_bwd(enc, Ws, h1, h2, d_out):
    enc, h1, h2, d_out = _d(enc), _d(h1), _d(h2), _d(d_out)
    W1, W2, W3 = (_d(w) for w in Ws)
    N, din = enc.shape
    dh, dout = W1.shape[0], W3.shape[0]
    dW1, dW2, dW3 = np.zeros_like(W1), np.zeros_like(W2), np.zeros_like(W3)
    d_enc = np.zeros_like(enc)
    lib().orc_mlp_bwd(_p(enc), I64(N), I32(din), I32(dh), I32(dout), _p(W1), _p(W2), _p(W3),
                      _p(h1), _p(h2), _p(d_out), _p(dW1), _p(dW2), _p(dW3), _p(d_enc))
    return [dW1, dW2, dW3], d_enc


# ---------------------------------------------------------------- transform
def qmul(a, b) -> np.ndarray:
    a, b = _d(a), _d(b)
    o = np.zeros(4)
    lib().orc_qmul(_p(a), _p(b), _p(o))
    return o


def apply(mean, quat, raw7, aabb, order=0):
    mean, quat, raw7, aabb = _d(mean), _d(quat), _d(raw7), _d(aabb)
    N = mean.shape[0]
    mo, qo = np.zeros_like(mean), np.zeros_like(quat)
    lib().orc_apply(_p(mean), _p(quat), _p(raw7), I64(N), _p(aabb), I32(order), _p(mo), _p(qo))
    return mo, qo


def apply_bwd(mean, quat, raw7, aabb, d_mean_out, d_quat_out, order=0):
    mean, quat, raw7, aabb = _d(mean), _d(quat), _d(raw7), _d(aabb)
    d_mean_out, d_quat_out = _d(d_mean_out), _d(d_quat_out)
    N = mean.shape[0]
    d_raw7 = np.zeros((N, 7))
    lib().orc_apply_bwd(_p(mean), _p(quat), _p(raw7), I64(N), _p(aabb), I32(order),
                        _p(d_mean_out), _p(d_quat_out), _p(d_raw7))
    return d_raw7


# ---------------------------------------------------------------- SH / projection
def sh_basis(deg: int, dirs) -> (np.ndarray, np.ndarray):
    dirs = _d(dirs)
    K = (deg + 1) ** 2
    Y = np.zeros((len(dirs), K))
    G = np.zeros((len(dirs), K, 3))
    yb, gb = np.zeros(16), np.zeros(48)
    for i, (x, y, z) in enumerate(dirs):
        lib().orc_sh_basis(I32(deg), F64(x), F64(y), F64(z), _p(yb), _p(gb))
        Y[i] = yb[:K]
        G[i] = gb[:3 * K].reshape(K, 3)
    return Y, G


def cam_array(cams) -> np.ndarray:
    """Cameras as the oracle's 21-double records."""
    out = np.zeros((len(cams), 21))
    for i, c in enumerate(cams):
        out[i, :12] = np.asarray(c.viewmat, np.float64).reshape(12)
        out[i, 12:18] = [c.fx, c.fy, c.cx, c.cy, c.W, c.H]
        out[i, 18:21] = np.asarray(c.campos, np.float64)
    return out


def _fibonacci_sphere(n, off=0.5):
    t = np.arange(n) + off
    z = 1.0 - 2.0 * t / n
    r = np.sqrt(1.0 - z * z)
    phi = t * np.pi * (3.0 - np.sqrt(5.0))
    return np.stack([r * np.cos(phi), r * np.sin(phi), z], 1)


def _rotation(q):
    q = _d(q)
    q = q / np.linalg.norm(q, axis=-1, keepdims=True)
    w, x, y, z = np.moveaxis(q, -1, 0)
    return np.stack([np.stack([1 - 2 * (y * y + z * z), 2 * (x * y - w * z), 2 * (x * z + w * y)], -1),
                     np.stack([2 * (x * y + w * z), 1 - 2 * (x * x + z * z), 2 * (y * z - w * x)], -1),
                     np.stack([2 * (x * z - w * y), 2 * (y * z + w * x), 1 - 2 * (x * x + y * y)], -1)],
                    -2)


def sh_rotate(sh, quat_from, quat_to, deg, n_dirs=64):
    """SH rotation (Suppl. B) by its definition: after a Gaussian turns by
    Rw = R(quat_to) R(quat_from)^T its colour seen from d is the colour seen
    from Rw^T d before; the new coefficients are those of that function, found
    by least squares over n_dirs sample directions (exact, the function being
    band-limited to deg).  sh [n, K, 3] -> [n, K, 3]."""
    sh = _d(sh)
    n, K = sh.shape[0], (deg + 1) ** 2
    D = _fibonacci_sphere(n_dirs)
    Yd, _ = sh_basis(deg, D)
    Rw = _rotation(quat_to) @ np.swapaxes(_rotation(quat_from), -1, -2)
    out = np.empty_like(sh)
    for i in range(n):
        Yr, _ = sh_basis(deg, D @ Rw[i])        # rows: Rw^T d
        f = Yr @ sh[i]                           # [n_dirs, 3]: colours at Rw^T d
        out[i] = np.linalg.lstsq(Yd, f, rcond=None)[0]
    return out


def project(g, cams, tile=TILE, mean=None, quat=None) -> Dict[str, np.ndarray]:
    """Project GaussianSet g (optionally with replaced mean/quat) into cams."""
    mean = _d(g.mean if mean is None else mean)
    quat = _d(g.quat if quat is None else quat)
    scale, op, sh = _d(g.scale), _d(g.opacity_logit), _d(g.sh)
    N, V = mean.shape[0], len(cams)
    ca = cam_array(cams)
    out = dict(mean2d=np.zeros((V, N, 2)), conic=np.zeros((V, N, 3)), opacity=np.zeros((V, N)),
               rgb=np.zeros((V, N, 3)), depth=np.zeros((V, N)),
               radius=np.zeros((V, N), np.int32), rect=np.zeros((V, N, 4), np.int32),
               margin=np.zeros((V, N)))
    lib().orc_project(I64(N), I32(V), _p(mean), _p(quat), _p(scale), _p(op), _p(sh),
                      I32(g.sh_deg), _p(ca), I32(tile), _p(out["mean2d"]), _p(out["conic"]),
                      _p(out["opacity"]), _p(out["rgb"]), _p(out["depth"]), _p(out["radius"]),
                      _p(out["rect"]), _p(out["margin"]))
    return out


def project_bwd(g, cams, grads, tile=TILE, mean=None, quat=None):
    mean = _d(g.mean if mean is None else mean)
    quat = _d(g.quat if quat is None else quat)
    scale, op, sh = _d(g.scale), _d(g.opacity_logit), _d(g.sh)
    grads = _d(grads)
    N, V = mean.shape[0], len(cams)
    ca = cam_array(cams)
    dm, dq = np.zeros((N, 3)), np.zeros((N, 4))
    lib().orc_project_bwd(I64(N), I32(V), _p(mean), _p(quat), _p(scale), _p(op), _p(sh),
                          I32(g.sh_deg), _p(ca), I32(tile), _p(grads), _p(dm), _p(dq))
    return dm, dq


def project_bwd_full(g, cams, grads, d_opacity=None, tile=TILE):
    """Reverse of the projection wrt every parameter of g: returns a dict of
    d_mean [N,3], d_quat [N,4], d_scale [N,3] (wrt s), d_ologit [N] and
    d_sh [N,K,3], from grads [V,N,8] and d_opacity [V,N]."""
    mean, quat, scale = _d(g.mean), _d(g.quat), _d(g.scale)
    op, sh = _d(g.opacity_logit), _d(g.sh)
    grads = _d(grads)
    N, V = mean.shape[0], len(cams)
    K = (g.sh_deg + 1) ** 2
    ca = cam_array(cams)
    out = dict(d_mean=np.zeros((N, 3)), d_quat=np.zeros((N, 4)), d_scale=np.zeros((N, 3)),
               d_ologit=np.zeros(N), d_sh=np.zeros((N, K, 3)))
    dop = None if d_opacity is None else _d(d_opacity)
    lib().orc_project_bwd_full(I64(N), I32(V), _p(mean), _p(quat), _p(scale), _p(op), _p(sh),
                               I32(g.sh_deg), _p(ca), I32(tile), _p(grads),
                               _p(dop) if dop is not None else None, _p(out["d_mean"]),
                               _p(out["d_quat"]), _p(out["d_scale"]), _p(out["d_ologit"]),
                               _p(out["d_sh"]))
    return out


# ---------------------------------------------------------------- binning
def bin_sort(mean2d, radius, depth, W, H, tile=TILE, capacity=None):
    """Integer binning of FP32 projected records -> (count, keys, vals, ranges)."""
    mean2d = np.ascontiguousarray(mean2d, np.float32)
    depth = np.ascontiguousarray(depth, np.float32)
    radius = np.ascontiguousarray(radius, np.int32)
    V, N = depth.shape
    tiles = ((W + tile - 1) // tile) * ((H + tile - 1) // tile)
    count = int(lib().orc_bin_sort(I32(V), I64(N), I32(W), I32(H), I32(tile), _p(mean2d),
                                   _p(radius), _p(depth), I64(0), None, None,
                                   _p(np.zeros(2 * V * tiles, np.uint32))))
    cap = count if capacity is None else capacity
    keys = np.zeros(max(cap, 1), np.uint64)
    vals = np.zeros(max(cap, 1), np.uint32)
    ranges = np.zeros((V * tiles, 2), np.uint32)
    lib().orc_bin_sort(I32(V), I64(N), I32(W), I32(H), I32(tile), _p(mean2d), _p(radius),
                       _p(depth), I64(cap), _p(keys), _p(vals), _p(ranges))
    return count, keys[:min(count, cap)], vals[:min(count, cap)], ranges


# ---------------------------------------------------------------- compositing
def _win(window):
    return None if window is None else _p(np.ascontiguousarray(window, np.int32))


def _reach(eps, V, N):
    if np.isscalar(eps) and eps == 0:
        return None
    return _p(np.ascontiguousarray(np.broadcast_to(_d(eps), (V, N))))


def raster_fwd(proj, W, H, bg=(0.0, 0.0, 0.0), tile=TILE, window=None, tie=0.0,
               tie_budget=0.0, pos_eps=0.0, rel_eps=0.0, depth_eps=0.0):
    """window = (tx0, ty0, tx1, ty1) tiles: composite only that crop (other
    pixels are left 0, T_final 1).  Ambiguity flags: tie is the relative
    depth gap under which two consecutive added Gaussians may be ordered
    either way; the swaps' exact effects T a_i a_j |c_i - c_j| add up to a
    per-pixel bound that flags the pixel above tie_budget; depth_eps widens
    that gap by each Gaussian's absolute depth reach.  pos_eps (pixels)
    and rel_eps (relative) widen the threshold margins by the reach of a
    displacement of the 2D means and a relative change of the conics
    (scalars or per-record [V, N] arrays)."""
    m2, cn, op, rgb, dp = (_d(proj[k]) for k in ("mean2d", "conic", "opacity", "rgb", "depth"))
    rad = np.ascontiguousarray(proj["radius"], np.int32)
    V, N = dp.shape
    img = np.zeros((V, 3, H, W))
    Tf = np.ones((V, H, W))
    last = np.zeros((V, H, W), np.int32)
    amb = np.zeros((V, H, W), np.int32)
    lib().orc_raster_fwd(I32(V), I64(N), I32(W), I32(H), I32(tile), _p(m2), _p(cn), _p(op),
                         _p(rgb), _p(dp), _p(rad), _p(_d(bg)), _win(window), F64(tie),
                         F64(tie_budget), _reach(depth_eps, V, N), _reach(pos_eps, V, N),
                         _reach(rel_eps, V, N), _p(img),
                         _p(Tf), _p(last), _p(amb))
    return img, Tf, last, amb


def raster_bwd(proj, W, H, T_final, last, d_img, bg=(0.0, 0.0, 0.0), tile=TILE,
               want_opacity=False, window=None):
    m2, cn, op, rgb, dp = (_d(proj[k]) for k in ("mean2d", "conic", "opacity", "rgb", "depth"))
    rad = np.ascontiguousarray(proj["radius"], np.int32)
    V, N = dp.shape
    grads = np.zeros((V, N, 8))
    dop = np.zeros((V, N)) if want_opacity else None
    lib().orc_raster_bwd(I32(V), I64(N), I32(W), I32(H), I32(tile), _p(m2), _p(cn), _p(op),
                         _p(rgb), _p(dp), _p(rad), _p(_d(bg)), _win(window), _p(_d(T_final)),
                         _p(np.ascontiguousarray(last, np.int32)), _p(_d(d_img)), _p(grads),
                         _p(dop) if dop is not None else None)
    return (grads, dop) if want_opacity else grads


# ---------------------------------------------------------------- loss / adam
def ssim_window() -> np.ndarray:
    g = np.zeros(11)
    lib().orc_ssim_window(_p(g))
    return g


def loss_l1_dssim(img, tgt, lam=0.2, want_grad=True):
    img, tgt = _d(img), _d(tgt)
    H, W = img.shape[-2:]
    P = int(np.prod(img.shape[:-2]))
    d = np.zeros_like(img) if want_grad else None
    ss = np.zeros(1)
    L = lib().orc_loss_l1_dssim(_p(img), _p(tgt), I32(P), I32(H), I32(W), F64(lam),
                                _p(d) if d is not None else None, _p(ss))
    return float(L), d, float(ss[0])


def warmup_loss(raw7):
    raw7 = _d(raw7)
    d = np.zeros_like(raw7)
    L = lib().orc_warmup_loss(_p(raw7), I64(raw7.shape[0]), _p(d))
    return float(L), d


def adam_rate(lr, lr_final_ratio, decay_steps, t):
    """Rate of the Adam update with 0-based step number t under an exponential
    decay from lr to lr * lr_final_ratio over decay_steps updates (constant
    after them; no decay when decay_steps <= 1)."""
    if decay_steps <= 1:
        return lr
    return lr * lr_final_ratio ** (min(t, decay_steps - 1) / (decay_steps - 1))


def adam(p, g, m, v, step, lr=0.002, b1=0.9, b2=0.99, eps=1e-15, inv_scale=1.0):
    """In-place Adam on float64 arrays p, m, v."""
    for a in (p, m, v):
        assert a.dtype == np.float64 and a.flags.c_contiguous
    g = _d(g)
    lib().orc_adam(_p(p), _p(g), _p(m), _p(v), I64(p.size), F64(lr), F64(b1), F64(b2),
                   F64(eps), I32(step), F64(inv_scale))


# ---------------------------------------------------------------- whole step
class NTCParams:
    """FP64 copy of the cache parameters: hash table [entries, F] and MLP."""

    def __init__(self, grid: Grid, table, Ws: List[np.ndarray]):
        self.grid = grid
        self.table = _d(table).copy()
        self.Ws = [_d(w).copy() for w in Ws]


def ntc_forward(p: NTCParams, mean, quat, order=0):
    enc = encode(p.grid, mean, p.table)
    h1, h2, raw7 = mlp_fwd(enc, p.Ws)
    mo, qo = apply(mean, quat, raw7, p.grid.aabb, order)
    return dict(enc=enc, h1=h1, h2=h2, raw7=raw7, mean=mo, quat=qo)


def render(g, cams, mean=None, quat=None, bg=(0.0, 0.0, 0.0), tile=TILE, window=None,
           tie=4e-7, tie_budget=2.5e-5, pos_eps=0.0, rel_eps=0.0, depth_eps=0.0):
    """Projection + compositing of g in FP64.  The ambiguity flags default to
    an FP32 computation of the same inputs: depth ties within 4e-7 (the reach
    of FP32 depth rounding) whose swaps could move the pixel by more than
    2.5e-5, a quarter of the FP32 image tolerance."""
    pr = project(g, cams, tile, mean=mean, quat=quat)
    W, H = cams[0].W, cams[0].H
    img, Tf, last, amb = raster_fwd(pr, W, H, bg, tile, window, tie, tie_budget, pos_eps, rel_eps,
                                    depth_eps)
    return dict(proj=pr, img=img, T_final=Tf, last=last, ambig=amb)


def stage1_loss_grads(p: NTCParams, g, cams, targets, lam=0.2, order=0,
                      bg=(0.0, 0.0, 0.0), tile=TILE):
    """One Stage-1 forward + backward (Section 4.1): returns the loss, the
    gradients of the hash table and of the MLP weights, and intermediates."""
    f = ntc_forward(p, g.mean, g.quat, order)
    r = render(g, cams, f["mean"], f["quat"], bg, tile)
    W, H = cams[0].W, cams[0].H
    L, d_img, ssim = loss_l1_dssim(r["img"], targets, lam)
    grads = raster_bwd(r["proj"], W, H, r["T_final"], r["last"], d_img, bg, tile)
    dm, dq = project_bwd(g, cams, grads, tile, mean=f["mean"], quat=f["quat"])
    d_raw7 = apply_bwd(g.mean, g.quat, f["raw7"], p.grid.aabb, dm, dq, order)
    dWs, d_enc = mlp_bwd(f["enc"], p.Ws, f["h1"], f["h2"], d_raw7)
    d_table = encode_bwd(p.grid, g.mean, d_enc)
    return dict(loss=L, ssim=ssim, d_table=d_table, dWs=dWs, d_raw7=d_raw7, d_mean=dm,
                d_quat=dq, d_img=d_img, grads=grads, fwd=f, render=r)


def stage1_loss(p: NTCParams, g, cams, targets, lam=0.2, order=0, bg=(0.0, 0.0, 0.0),
                tile=TILE) -> float:
    f = ntc_forward(p, g.mean, g.quat, order)
    r = render(g, cams, f["mean"], f["quat"], bg, tile)
    return loss_l1_dssim(r["img"], targets, lam, want_grad=False)[0]
