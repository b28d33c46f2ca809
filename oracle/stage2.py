"""FP64 oracle of Stage 2, the adaptive 3DG addition (Section 4.2).

Test infrastructure: only the tests, the smoke check and the benchmark's
CPU-baseline leg use it.  Plain numpy in float64, in the order the section
gives the steps:

  view-space positional gradient statistics (the gradient of the loss wrt the
  2D mean in normalised device coordinates, averaged over the views where the
  Gaussian is visible) -> the Gaussians above tau_grad -> one added Gaussian
  each, at a draw from N(mu, 2 Sigma), SH and scale copied, rotation identity,
  opacity 0.1 -> optimisation of the added Gaussians only (same loss as
  Stage 1) -> at the end of each epoch: added Gaussians above tau_grad spawn
  one more nearby (draw from N(mu, Sigma), scale x 0.8, rotation and SH
  inherited, opacity 0.1 as at a spawn), then those with opacity below
  tau_alpha are discarded.

An added Gaussian is a row [mean 3 | quat 4 | log scale 3 | opacity logit 1 |
SH K x 3].  Random draws are inputs (z), so the CUDA path can be given the
same ones.
"""
from __future__ import annotations

import numpy as np

from . import (loss_l1_dssim, project_bwd_full, raster_bwd, render)

COL_MEAN, COL_QUAT, COL_LOGS, COL_OPL, COL_SH = 0, 3, 7, 10, 11


def cols(sh_deg: int) -> int:
    return COL_SH + 3 * (sh_deg + 1) ** 2


def rotation(q) -> np.ndarray:
    """Rotation matrices of quaternions q [n, 4] (w, x, y, z), normalised first."""
    q = np.asarray(q, np.float64)
    q = q / np.linalg.norm(q, axis=1, keepdims=True)
    w, x, y, z = q.T
    R = np.empty((q.shape[0], 3, 3))
    R[:, 0, 0] = 1 - 2 * (y * y + z * z)
    R[:, 0, 1] = 2 * (x * y - w * z)
    R[:, 0, 2] = 2 * (x * z + w * y)
    R[:, 1, 0] = 2 * (x * y + w * z)
    R[:, 1, 1] = 1 - 2 * (x * x + z * z)
    R[:, 1, 2] = 2 * (y * z - w * x)
    R[:, 2, 0] = 2 * (x * z - w * y)
    R[:, 2, 1] = 2 * (y * z + w * x)
    R[:, 2, 2] = 1 - 2 * (x * x + y * y)
    return R


def viewspace_grad(grads, radius, W, H, grad_scale=1.0):
    """accum[i] = sum over views with radius > 0 of grad_scale |(dL/du W/2,
    dL/dv H/2)|, denom[i] = the number of such views."""
    g = np.asarray(grads, np.float64)
    vis = np.asarray(radius) > 0
    norm = grad_scale * np.hypot(g[..., 0] * (W / 2), g[..., 1] * (H / 2))
    return np.sum(norm * vis, axis=0), np.sum(vis, axis=0).astype(np.int64)


def above(accum, denom, tau) -> np.ndarray:
    with np.errstate(invalid="ignore", divide="ignore"):
        return (denom > 0) & (np.asarray(accum, np.float64) / np.maximum(denom, 1) > tau)


def select_above(accum, denom, tau) -> np.ndarray:
    return np.nonzero(above(accum, denom, tau))[0]


def spawn(g, idx, z, opacity_init=0.1) -> np.ndarray:
    """Rows of the Gaussians added around g's Gaussians idx, z [len(idx), 3]."""
    idx = np.asarray(idx)
    K = (g.sh_deg + 1) ** 2
    rows = np.zeros((len(idx), cols(g.sh_deg)))
    mu = np.asarray(g.mean, np.float64)[idx]
    s = np.asarray(g.scale, np.float64)[idx]
    R = rotation(np.asarray(g.quat, np.float64)[idx])
    # N(mu, 2 Sigma) with Sigma = R diag(s)^2 R^T: mu + sqrt(2) R diag(s) z
    rows[:, COL_MEAN:COL_QUAT] = mu + np.sqrt(2.0) * np.einsum("nij,nj->ni", R, s * np.asarray(z))
    rows[:, COL_QUAT] = 1.0
    rows[:, COL_LOGS:COL_OPL] = np.log(s)
    rows[:, COL_OPL] = np.log(opacity_init / (1.0 - opacity_init))
    rows[:, COL_SH:] = np.asarray(g.sh, np.float64)[idx].reshape(len(idx), 3 * K)
    return rows


def densify_prune(rows, accum, denom, tau_grad, tau_opacity, split_scale, z, opacity_init=0.1):
    """Quantity control at the end of an epoch: returns (new rows, kept mask,
    split mask).  Kept rows first, in order, then one new row per kept row
    above tau_grad, in order (rotation and SH inherited, scale x split_scale,
    opacity opacity_init as at a spawn)."""
    rows = np.asarray(rows, np.float64)
    opacity = 1.0 / (1.0 + np.exp(-rows[:, COL_OPL]))
    keep = opacity >= tau_opacity
    split = keep & above(accum, denom, tau_grad)
    parents = rows[split]
    new = parents.copy()
    R = rotation(parents[:, COL_QUAT:COL_LOGS])
    s = np.exp(parents[:, COL_LOGS:COL_OPL])
    new[:, COL_MEAN:COL_QUAT] = parents[:, COL_MEAN:COL_QUAT] + np.einsum(
        "nij,nj->ni", R, s * np.asarray(z, np.float64)[split])
    new[:, COL_LOGS:COL_OPL] += np.log(split_scale)
    new[:, COL_OPL] = np.log(opacity_init / (1.0 - opacity_init))
    return np.concatenate([rows[keep], new]), keep, split


def rows_to_gaussians(rows, sh_deg):
    """The rendered attributes of rows, as a float64 GaussianSet."""
    from paper_2403_01444_gb300.scenes import GaussianSet
    rows = np.asarray(rows, np.float64)
    K = (sh_deg + 1) ** 2
    return GaussianSet(rows[:, COL_MEAN:COL_QUAT].copy(), rows[:, COL_QUAT:COL_LOGS].copy(),
                       np.exp(rows[:, COL_LOGS:COL_OPL]), rows[:, COL_OPL].copy(),
                       rows[:, COL_SH:].reshape(-1, K, 3).copy(), sh_deg)


def concat(a, b):
    from paper_2403_01444_gb300.scenes import GaussianSet
    f = lambda x, y: np.concatenate([np.asarray(x, np.float64), np.asarray(y, np.float64)])
    return GaussianSet(f(a.mean, b.mean), f(a.quat, b.quat), f(a.scale, b.scale),
                       f(a.opacity_logit, b.opacity_logit), f(a.sh, b.sh), a.sh_deg)


def grads_to_rows(d, rows):
    """Row gradients from project_bwd_full's dict (d/d log s = d/ds * s)."""
    rows = np.asarray(rows, np.float64)
    n = rows.shape[0]
    g = np.zeros_like(rows)
    g[:, COL_MEAN:COL_QUAT] = d["d_mean"]
    g[:, COL_QUAT:COL_LOGS] = d["d_quat"]
    g[:, COL_LOGS:COL_OPL] = d["d_scale"] * np.exp(rows[:, COL_LOGS:COL_OPL])
    g[:, COL_OPL] = d["d_ologit"]
    g[:, COL_SH:] = d["d_sh"].reshape(n, -1)
    return g


def loss_grads(fixed, rows, cams, targets, lam=0.2):
    """One Stage-2 forward + backward: the fixed (transformed) Gaussians and
    the added rows rendered together, Stage 1's loss, gradients of the rows.
    Returns (loss, row gradients [n, cols], render dict)."""
    added = rows_to_gaussians(rows, fixed.sh_deg)
    g = concat(fixed, added)
    r = render(g, cams)
    W, H = cams[0].W, cams[0].H
    L, d_img, _ = loss_l1_dssim(r["img"], targets, lam)
    grads, d_op = raster_bwd(r["proj"], W, H, r["T_final"], r["last"], d_img, want_opacity=True)
    d = project_bwd_full(g, cams, grads, d_op)
    nf = np.asarray(fixed.mean).shape[0]
    part = {k: v[nf:] for k, v in d.items()}
    return L, grads_to_rows(part, rows), r, grads


def lr_columns(sh_deg, lr6) -> np.ndarray:
    """Per-column learning rates from {mean, rotation, log scale, opacity
    logit, SH band 0, SH bands >= 1}."""
    c = np.empty(cols(sh_deg))
    c[COL_MEAN:COL_QUAT] = lr6[0]
    c[COL_QUAT:COL_LOGS] = lr6[1]
    c[COL_LOGS:COL_OPL] = lr6[2]
    c[COL_OPL] = lr6[3]
    c[COL_SH:COL_SH + 3] = lr6[4]
    c[COL_SH + 3:] = lr6[5]
    return c


def adam_rows(rows, m, v, g, lr6, step, b1, b2, eps, sh_deg):
    """Bias-corrected Adam (step = 1 for the first update) with per-column
    learning rates; returns new (rows, m, v)."""
    lr = lr_columns(sh_deg, lr6)[None, :]
    m = b1 * m + (1 - b1) * g
    v = b2 * v + (1 - b2) * g * g
    mh = m / (1 - b1 ** step)
    vh = v / (1 - b2 ** step)
    return rows - lr * mh / (np.sqrt(vh) + eps), m, v
