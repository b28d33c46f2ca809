"""Seeded synthetic inputs for the Stage-1 training step.

This module only draws inputs: Gaussian sets, pinhole cameras, ground-truth
motion fields and raw projected records.  It holds none of the method's
arithmetic (no projection, no compositing, no hash encoding, no MLP), so that
both the FP64 CPU oracle and the CUDA path can take the same inputs from it
without sharing any of the computation being checked.

The distributions stand in for the multi-view video workloads of the paper's
experiments (N3DV: ~1e5 Gaussians, 1352x1014 views; Meet Room: 1280x720,
Section 5.1).  Those datasets are not available, so the scenes are synthetic:

* centres uniform in [-1, 1]^3, log-scales N(-3, 0.3), random unit
  quaternions, opacity logits N(0, 1), SH DC terms giving colours of about
  0.5 +- 0.4, higher SH bands N(0, 0.05^2);
* pinhole cameras with a 60 degree horizontal field of view on a ring or arc
  of radius 4 looking at the origin (OpenCV frame: +z forward, +y down);
* ground-truth motion: a rigid rotation about the origin plus a translation,
  and/or a smooth field made of a sum of Gaussian radial basis displacements.

Every array is generated in float64 and handed out as float32, the precision
both paths read.
"""
from __future__ import annotations

import dataclasses
import math
from typing import List, Optional

import numpy as np
from scipy.spatial.transform import Rotation

__all__ = [
    "GaussianSet", "Camera", "SceneConfig", "CONFIGS", "make_gaussians",
    "look_at_camera", "ring_cameras", "arc_cameras", "rigid_motion",
    "rbf_motion", "random_projected", "random_hashgrid_table", "random_mlp",
    "make_scene", "make_sequence", "emerging_content", "union",
]


@dataclasses.dataclass
class GaussianSet:
    """Gaussian parameters, one row per Gaussian (float32)."""

    mean: np.ndarray           # [N, 3]
    quat: np.ndarray           # [N, 4] (w, x, y, z), unit
    scale: np.ndarray          # [N, 3] positive scales (already exponentiated)
    opacity_logit: np.ndarray  # [N]
    sh: np.ndarray             # [N, K, 3], K = (deg + 1)^2
    sh_deg: int

    @property
    def n(self) -> int:
        return int(self.mean.shape[0])

    def copy(self) -> "GaussianSet":
        return GaussianSet(self.mean.copy(), self.quat.copy(), self.scale.copy(),
                           self.opacity_logit.copy(), self.sh.copy(), self.sh_deg)

    def subset(self, idx) -> "GaussianSet":
        return GaussianSet(self.mean[idx].copy(), self.quat[idx].copy(),
                           self.scale[idx].copy(), self.opacity_logit[idx].copy(),
                           self.sh[idx].copy(), self.sh_deg)


@dataclasses.dataclass
class Camera:
    """Pinhole camera; viewmat is world->camera [R | t], row-major 3x4."""

    viewmat: np.ndarray  # [3, 4] float32
    fx: float
    fy: float
    cx: float
    cy: float
    W: int
    H: int
    campos: np.ndarray   # [3] float32


def make_gaussians(n: int, sh_deg: int, rng: np.random.Generator,
                   extent: float = 1.0) -> GaussianSet:
    """Draw n Gaussians with the distributions listed in the module docstring."""
    mean = rng.uniform(-extent, extent, size=(n, 3))
    log_s = rng.normal(-3.0, 0.3, size=(n, 3))
    q = rng.normal(size=(n, 4))
    q /= np.linalg.norm(q, axis=1, keepdims=True)
    op = rng.normal(0.0, 1.0, size=n)
    k = (sh_deg + 1) ** 2
    sh = np.zeros((n, k, 3))
    # DC band: colour offsets of about +-0.4 around mid-grey once the DC
    # basis constant (about 0.282) is applied.
    sh[:, 0, :] = rng.uniform(-1.4, 1.4, size=(n, 3))
    if k > 1:
        sh[:, 1:, :] = rng.normal(0.0, 0.05, size=(n, k - 1, 3))
    f = np.float32
    return GaussianSet(mean.astype(f), q.astype(f), np.exp(log_s).astype(f),
                       op.astype(f), sh.astype(f), sh_deg)


def emerging_content(rng: np.random.Generator, n_new: int, sh_deg: int, radius: float = 0.2,
                     centre_extent: float = 0.5) -> GaussianSet:
    """Gaussians of an object absent from the previous frame (the emerging
    content of Section 4.2): centres uniform in a ball of `radius` around a
    centre at x, y uniform in [-centre_extent, centre_extent] and z = 1 +
    radius, just in front of the scene's +z face (the side the arc and ring
    cameras at azimuth 0 look at, so the object is not hidden inside the
    cloud), smaller and more
    opaque than the scene's (log-scales N(-3.5, 0.3), opacity logits
    N(2, 0.5)) and of one saturated hue (SH DC terms 3 (hue - 1/3) +
    N(0, 0.1^2), hue a Dirichlet(0.3) draw; higher bands zero)."""
    centre = np.array([rng.uniform(-centre_extent, centre_extent),
                       rng.uniform(-centre_extent, centre_extent), 1.0 + radius])
    d = rng.normal(size=(n_new, 3))
    d /= np.linalg.norm(d, axis=1, keepdims=True)
    r = radius * rng.uniform(size=(n_new, 1)) ** (1.0 / 3.0)
    mean = centre + d * r
    log_s = rng.normal(-3.5, 0.3, size=(n_new, 3))
    q = rng.normal(size=(n_new, 4))
    q /= np.linalg.norm(q, axis=1, keepdims=True)
    op = rng.normal(2.0, 0.5, size=n_new)
    hue = rng.dirichlet(np.ones(3) * 0.3)
    k = (sh_deg + 1) ** 2
    sh = np.zeros((n_new, k, 3))
    sh[:, 0, :] = 3.0 * (hue - 1.0 / 3.0) + rng.normal(0.0, 0.1, size=(n_new, 3))
    f = np.float32
    return GaussianSet(mean.astype(f), q.astype(f), np.exp(log_s).astype(f), op.astype(f),
                       sh.astype(f), sh_deg)


def union(a: GaussianSet, b: GaussianSet) -> GaussianSet:
    c = lambda x, y: np.concatenate([x, y]).astype(np.float32)
    return GaussianSet(c(a.mean, b.mean), c(a.quat, b.quat), c(a.scale, b.scale),
                       c(a.opacity_logit, b.opacity_logit), c(a.sh, b.sh), a.sh_deg)


def look_at_camera(pos, W: int, H: int, fov_x_deg: float = 60.0,
                   target=(0.0, 0.0, 0.0), up=(0.0, 1.0, 0.0)) -> Camera:
    """OpenCV-frame pinhole camera at pos looking at target, square pixels."""
    pos = np.asarray(pos, np.float64)
    fwd = np.asarray(target, np.float64) - pos
    fwd /= np.linalg.norm(fwd)
    right = np.cross(fwd, np.asarray(up, np.float64))
    right /= np.linalg.norm(right)
    down = np.cross(fwd, right)
    R = np.stack([right, down, fwd])
    t = -R @ pos
    fx = W / (2.0 * math.tan(math.radians(fov_x_deg) / 2.0))
    vm = np.concatenate([R, t[:, None]], axis=1).astype(np.float32)
    return Camera(vm, float(np.float32(fx)), float(np.float32(fx)), W / 2.0, H / 2.0,
                  int(W), int(H), pos.astype(np.float32))


def _orbit_pos(radius, az_deg, el_deg):
    az, el = math.radians(az_deg), math.radians(el_deg)
    return (radius * math.sin(az) * math.cos(el), radius * math.sin(el),
            radius * math.cos(az) * math.cos(el))


def ring_cameras(azimuths, elevations, W, H, radius=4.0, fov_x_deg=60.0) -> List[Camera]:
    return [look_at_camera(_orbit_pos(radius, a, e), W, H, fov_x_deg)
            for a, e in zip(azimuths, elevations)]


def arc_cameras(n, W, H, az_range=(-60.0, 60.0), elevations=(0.0, 10.0, -10.0),
                radius=4.0, fov_x_deg=60.0) -> List[Camera]:
    az = np.linspace(az_range[0], az_range[1], n)
    el = [elevations[i % len(elevations)] for i in range(n)]
    return ring_cameras(az, el, W, H, radius, fov_x_deg)


def _random_unit(rng, n=None):
    v = rng.normal(size=(3,) if n is None else (n, 3))
    return v / np.linalg.norm(v, axis=-1, keepdims=True)


def rigid_motion(g: GaussianSet, rng: np.random.Generator, angle_deg=5.0,
                 translation=0.05) -> GaussianSet:
    """Ground truth: rotate about the origin by angle_deg around a random axis,
    then translate by `translation` along a random direction."""
    axis = _random_unit(rng)
    rot = Rotation.from_rotvec(axis * math.radians(angle_deg))
    tdir = _random_unit(rng)
    out = g.copy()
    out.mean = (rot.apply(g.mean.astype(np.float64)) + translation * tdir).astype(np.float32)
    # scipy stores quaternions as (x, y, z, w); the set stores (w, x, y, z).
    q_xyzw = g.quat[:, [1, 2, 3, 0]].astype(np.float64)
    q_new = (rot * Rotation.from_quat(q_xyzw)).as_quat()
    out.quat = q_new[:, [3, 0, 1, 2]].astype(np.float32)
    return out


def rbf_motion(g: GaussianSet, rng: np.random.Generator, n_centres=8,
               max_disp=0.1) -> GaussianSet:
    """Ground truth: mu + sum_k dir_k exp(-|mu - c_k|^2 / (2 s_k^2)), rescaled
    so that the largest displacement over the set equals max_disp; rotations
    are left unchanged."""
    c = rng.uniform(-1.0, 1.0, size=(n_centres, 3))
    s = rng.uniform(0.2, 0.5, size=n_centres)
    d = _random_unit(rng, n_centres)
    mu = g.mean.astype(np.float64)
    disp = np.zeros_like(mu)
    for k in range(n_centres):
        w = np.exp(-np.sum((mu - c[k]) ** 2, axis=1) / (2.0 * s[k] ** 2))
        disp += w[:, None] * d[k]
    scale = max_disp / max(np.max(np.linalg.norm(disp, axis=1)), 1e-12)
    out = g.copy()
    out.mean = (mu + scale * disp).astype(np.float32)
    return out


def random_projected(V: int, N: int, W: int, H: int, rng: np.random.Generator,
                     cull_frac=0.1, radius_range=(1, 40), margin=48):
    """Raw per-(view, Gaussian) projected records for checking binning and
    compositing on their own: 2D means (some off-image), integer radii,
    conics of random SPD 2D covariances, depths, opacities and colours.
    Culled entries have radius 0."""
    u = rng.uniform(-margin, W + margin, size=(V, N))
    v = rng.uniform(-margin, H + margin, size=(V, N))
    # covariance = R diag(l1, l2) R^T with eigenvalues from the radius range
    sig = rng.uniform(radius_range[0] / 3.0, radius_range[1] / 3.0, size=(V, N, 2))
    th = rng.uniform(0.0, math.pi, size=(V, N))
    c, s = np.cos(th), np.sin(th)
    l1, l2 = sig[..., 0] ** 2 + 0.3, sig[..., 1] ** 2 + 0.3
    a = c * c * l1 + s * s * l2
    b = c * s * (l1 - l2)
    cc = s * s * l1 + c * c * l2
    det = a * cc - b * b
    conic = np.stack([cc / det, -b / det, a / det], axis=-1)
    radius = np.ceil(3.0 * np.sqrt(np.maximum(l1, l2))).astype(np.int32)
    cull = rng.uniform(size=(V, N)) < cull_frac
    radius[cull] = 0
    depth = rng.uniform(0.5, 8.0, size=(V, N))
    opacity = 1.0 / (1.0 + np.exp(-rng.normal(0.0, 1.5, size=(V, N))))
    rgb = rng.uniform(0.0, 1.0, size=(V, N, 3))
    f = np.float32
    return dict(mean2d=np.stack([u, v], axis=-1).astype(f), conic=conic.astype(f),
                opacity=opacity.astype(f), rgb=rgb.astype(f), depth=depth.astype(f),
                radius=radius)


def random_hashgrid_table(n_entries: int, F: int, rng: np.random.Generator,
                          scale=1e-4) -> np.ndarray:
    """Hash-table features ~ U[-scale, scale] (the I-NGP initialisation range)."""
    return rng.uniform(-scale, scale, size=(n_entries, F)).astype(np.float32)


def random_mlp(dims, rng: np.random.Generator) -> List[np.ndarray]:
    """Bias-free layer weights [out, in], Kaiming-uniform bound sqrt(6 / in)."""
    ws = []
    for din, dout in zip(dims[:-1], dims[1:]):
        bound = math.sqrt(6.0 / din)
        ws.append(rng.uniform(-bound, bound, size=(dout, din)).astype(np.float32))
    return ws


@dataclasses.dataclass
class SceneConfig:
    name: str
    n_gauss: int
    sh_deg: int
    n_cams: int
    W: int
    H: int
    views_per_batch: int
    iters: int
    motion: str            # "rigid", "rbf", "rigid+rbf"
    cam_layout: str        # "ring4", "ring8", "arc20", "arc12", "ring16"
    emerging: bool = False  # the target holds an object absent from the previous frame


CONFIGS = {
    1: SceneConfig("plain-fp32-4k", 4096, 1, 4, 128, 96, 4, 50, "rigid", "ring4"),
    2: SceneConfig("ntc-50k-8v-480x360", 50_000, 2, 8, 480, 360, 8, 150, "rbf", "ring8"),
    3: SceneConfig("ntc-250k-20v-1352x1014", 250_000, 3, 20, 1352, 1014, 4, 150,
                   "rigid+rbf", "arc20"),
    4: SceneConfig("stage2-500k-12v-1280x720", 500_000, 3, 12, 1280, 720, 4, 100,
                   "rigid+rbf", "arc12", emerging=True),
    5: SceneConfig("large-1m-16v-1920x1080", 1_000_000, 3, 16, 1920, 1080, 16, 150,
                   "rbf", "ring16"),
}


def cameras_for(cfg: SceneConfig) -> List[Camera]:
    W, H = cfg.W, cfg.H
    if cfg.cam_layout == "ring4":
        return ring_cameras([0, 90, 180, 270], [0, 0, 0, 0], W, H)
    if cfg.cam_layout == "ring8":
        return ring_cameras([45 * k for k in range(8)],
                            [15 if k % 2 == 0 else -15 for k in range(8)], W, H)
    if cfg.cam_layout == "arc20":
        return arc_cameras(20, W, H, (-60.0, 60.0))
    if cfg.cam_layout == "arc12":
        return arc_cameras(12, W, H, (-45.0, 45.0), (0.0,))
    if cfg.cam_layout == "ring16":
        return ring_cameras([22.5 * k for k in range(16)], [0] * 16, W, H)
    raise ValueError(cfg.cam_layout)


def heldout_camera(cfg: SceneConfig) -> Camera:
    if cfg.cam_layout == "ring4":
        return ring_cameras([45], [0], cfg.W, cfg.H)[0]
    return ring_cameras([7.5], [5.0], cfg.W, cfg.H)[0]


@dataclasses.dataclass
class Scene:
    cfg: SceneConfig
    prev: GaussianSet          # previous-frame (frozen) Gaussians
    target: GaussianSet        # ground-truth moved Gaussians
    cams: List[Camera]
    heldout: Camera


def _motion_step(g: GaussianSet, motion: str, rng: np.random.Generator) -> GaussianSet:
    if motion == "rigid":
        return rigid_motion(g, rng, 5.0, 0.05)
    if motion == "rbf":
        return rbf_motion(g, rng, 8, 0.1)
    return rbf_motion(rigid_motion(g, rng, 1.0, 0.01), rng, 8, 0.02)


def make_sequence(cfg_index: int, n_frames: int, n_gauss: Optional[int] = None,
                  W: Optional[int] = None, H: Optional[int] = None):
    """A multi-view video of n_frames + 1 frames: frame 0 is the config's
    previous-frame Gaussians and frame t applies one more step of the config's
    motion to frame t - 1 (cumulative), drawn from the same seeded stream as
    make_scene, so frame 1 is make_scene's target.  Returns (config, frames,
    cameras, held-out camera)."""
    cfg = dataclasses.replace(CONFIGS[cfg_index])
    if n_gauss is not None:
        cfg.n_gauss = n_gauss
    if W is not None:
        cfg.W = W
    if H is not None:
        cfg.H = H
    rng = np.random.default_rng(cfg_index)
    frames = [make_gaussians(cfg.n_gauss, cfg.sh_deg, rng)]
    for _ in range(n_frames):
        frames.append(_motion_step(frames[-1], cfg.motion, rng))
    return cfg, frames, cameras_for(cfg), heldout_camera(cfg)


def make_scene(cfg_index: int, n_gauss: Optional[int] = None, W: Optional[int] = None,
               H: Optional[int] = None, n_cams: Optional[int] = None) -> Scene:
    """Scene of config cfg_index (seed = config index), optionally shrunk."""
    cfg = dataclasses.replace(CONFIGS[cfg_index])
    if n_gauss is not None:
        cfg.n_gauss = n_gauss
    if W is not None:
        cfg.W = W
    if H is not None:
        cfg.H = H
    rng = np.random.default_rng(cfg_index)
    prev = make_gaussians(cfg.n_gauss, cfg.sh_deg, rng)
    tgt = _motion_step(prev, cfg.motion, rng)
    if cfg.emerging:
        # an object absent from the previous frame appears (Section 4.2):
        # 5 000 to 10 000 new Gaussians in a ball of radius 0.2, scaled with n
        n_new = int(rng.integers(5000, 10001) * cfg.n_gauss / CONFIGS[cfg_index].n_gauss)
        tgt = union(tgt, emerging_content(rng, max(n_new, 1), cfg.sh_deg))
    cams = cameras_for(cfg)
    if n_cams is not None:
        cams = cams[:n_cams]
        cfg.n_cams = n_cams
    return Scene(cfg, prev, tgt, cams, heldout_camera(cfg))
