"""Edge cases of the GPU path against the FP64 oracle: an empty scene, a
scene entirely behind the cameras, ragged and tiny image sizes, the largest
number of views in one launch, needle footprints whose FP32 a c - b^2
cancels, a fully transparent Gaussian, and a whole Stage-1 step on an empty
set."""
import numpy as np
import pytest
import torch

import oracle
from paper_2403_01444_gb300 import gs3, scenes
from paper_2403_01444_gb300.engine import NTC, Rasterizer, Stage1, render

pytestmark = pytest.mark.gpu
DEV = "cuda"


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2403_01444_gb300 import build
    build.build()
    gs3.lib()
    oracle.build()


def _compare(g, cams, W, H, tol=1e-4, min_ok=0.98):
    r = oracle.render(g, cams)
    img = render(gs3.Gaussians.from_numpy(g), cams, W, H).cpu().numpy()
    ok = np.broadcast_to((r["ambig"] == 0)[:, None], img.shape)
    assert ok.mean() >= min_ok
    assert np.abs(img - r["img"])[ok].max() <= tol
    return img


def _empty_set(deg=1):
    z = lambda *s: np.zeros(s, np.float32)
    return scenes.GaussianSet(z(0, 3), z(0, 4), z(0, 3), z(0), z(0, (deg + 1) ** 2, 3), deg)


def test_empty_scene_renders_background_and_zero_gradients():
    W, H = 50, 37
    cams = scenes.ring_cameras([0, 90], [0, 0], W, H)
    G = gs3.Gaussians.from_numpy(_empty_set())
    cd = gs3.cameras_to_device(cams)
    r = Rasterizer(0, 2, W, H, 1024, DEV, bg=(0.25, 0.5, 0.75))
    r.fit_capacity(G, cd)
    assert r.count() == 0
    img = r.img.cpu().numpy()
    for c, v in enumerate((0.25, 0.5, 0.75)):
        assert np.all(img[:, c] == np.float32(v))
    assert torch.all(r.T_final == 1.0) and torch.all(r.last == 0)
    d_mean, d_quat = r.backward(G, cd, torch.ones(2, 3, H, W, device=DEV))
    torch.cuda.synchronize()
    assert d_mean.numel() == 0 and d_quat.numel() == 0


def test_scene_behind_the_cameras_is_culled():
    W, H = 64, 48
    cam = scenes.look_at_camera((0.0, 0.0, 4.0), W, H)
    g = scenes.make_gaussians(500, 1, np.random.default_rng(1))
    g.mean[:, 2] = np.float32(4.1) + np.abs(g.mean[:, 2])      # all behind the camera
    img = _compare(g, [cam], W, H)
    assert np.all(img == 0.0)


@pytest.mark.parametrize("W,H", [(1, 1), (17, 33), (129, 7), (16, 16)])
def test_ragged_and_tiny_images(W, H):
    cams = scenes.ring_cameras([0, 150], [5, -5], W, H)
    g = scenes.make_gaussians(800, 2, np.random.default_rng(W * 1000 + H))
    g.scale = (g.scale * 2.0).astype(np.float32)
    _compare(g, cams, W, H, min_ok=0.9 if W * H < 100 else 0.98)


def test_largest_view_count_in_one_launch():
    V = 64   # GS_MAX_VIEWS
    W, H = 40, 30
    cams = scenes.ring_cameras([360.0 * k / V for k in range(V)], [10 * ((k % 3) - 1) for k in range(V)],
                               W, H)
    g = scenes.make_gaussians(600, 1, np.random.default_rng(3))
    g.scale = (g.scale * 2.0).astype(np.float32)
    _compare(g, cams, W, H)
    with pytest.raises(gs3.GsError):
        render(gs3.Gaussians.from_numpy(g), cams + cams[:1], W, H)   # 65 views


U32 = 2.0 ** -24          # FP32 unit roundoff
ETA = 64 * U32            # relative error of a GPU conic entry, see below


def _needles():
    """Needles hundreds of pixels long at 45 degrees in the image plane: their
    2D covariance a, c ~ 3e5 while a c - b^2 ~ 1.6e5, so FP32 a c - b^2
    cancels to nothing (checked below)."""
    W, H = 96, 72
    cam = scenes.look_at_camera((0.0, 0.0, 4.0), W, H)
    rng = np.random.default_rng(4)
    n = 8
    g = scenes.make_gaussians(n, 0, rng)
    g.scale = np.stack([np.full(n, 40.0), np.full(n, 1e-5), np.full(n, 1e-5)], 1).astype(np.float32)
    c, s_ = np.cos(np.pi / 8), np.sin(np.pi / 8)
    g.quat[:] = np.array([c, 0.0, 0.0, s_], np.float32)
    g.mean[:, 2] = rng.uniform(-0.5, 0.5, n).astype(np.float32)
    g.opacity_logit[:] = -1.0
    return g, cam, W, H


def test_thin_footprints_keep_fp32_accuracy():
    """The GPU sums the determinant of the 2D covariance from non-negative
    terms (Cauchy-Binet), so a needle's conic keeps FP32 accuracy: every
    entry within ETA = 64 u of the FP64 oracle's.  (Operation count of one
    entry: rotation from the quaternion <= 6 roundings, R diag(s) 1, T <= 4,
    P = T R diag(s) <= 6, a, b, c <= 6, determinant <= 8, division 1: <= 32
    in first order; doubled.)  The image then differs from the oracle's by at
    most max colour * sum_i alpha_i |d power_i| per pixel (|dC/d alpha_i| <=
    T_i max colour, Eq. 4), |d power_i| <= 0.5 ETA (|A| dx^2 + 2|B||dx dy| +
    |C| dy^2) (conic entries and the FP32 evaluation of the quadratic form)
    + |grad power_i| * 16 u (|u| + |v| + 1) (the 2D mean), on the pixels none
    of whose thresholds (power > 0, alpha >= 1/255) lies within that reach."""
    g, cam, W, H = _needles()
    pr = oracle.project(g, [cam])
    A, B, C = (pr["conic"][0, :, k] for k in range(3))
    dconic = A * C - B * B
    a, b, c2 = C / dconic, -B / dconic, A / dconic             # covariance + 0.3 I
    vis = pr["radius"][0] > 0
    assert vis.sum() >= 4
    # the regime: FP32 a c - b^2 from the correctly rounded a, b, c is off by > 1 %
    a32, b32, c32 = (x.astype(np.float32) for x in (a, b, c2))
    naive = (a32 * c32 - b32 * b32).astype(np.float64)
    assert np.max(np.abs(naive - 1 / dconic)[vis] * dconic[vis]) > 1e-2

    G = gs3.Gaussians.from_numpy(g)
    cd = gs3.cameras_to_device([cam])
    p = gs3.Projected.empty(1, g.n)
    gs3.gs_project(G, cd, 1, W, H, p)
    torch.cuda.synchronize()
    co = p.conic_opacity.cpu().numpy()[0]
    assert np.array_equal(p.radius.cpu().numpy()[0] > 0, vis)
    rel = np.abs(co[:, :3] - pr["conic"][0]) / np.abs(pr["conic"][0])
    assert rel[vis].max() <= ETA, rel[vis].max()

    # image against the derived per-pixel bound
    img = render(G, [cam], W, H).cpu().numpy()[0]
    r = oracle.render(g, [cam])
    ys, xs = np.mgrid[0:H, 0:W] + 0.5
    tol = np.zeros((H, W))
    flag = np.zeros((H, W), bool)
    cm = max(float(pr["rgb"][0][vis].max()), 0.0)
    for i in np.nonzero(vis)[0]:
        u, v = pr["mean2d"][0, i]
        dx, dy = xs - u, ys - v
        q = np.abs(A[i]) * dx * dx + 2 * np.abs(B[i] * dx * dy) + np.abs(C[i]) * dy * dy
        grad = np.abs(A[i] * dx + B[i] * dy) + np.abs(B[i] * dx + C[i] * dy)
        reach = 0.5 * ETA * q + grad * 16 * U32 * (abs(u) + abs(v) + 1)
        power = -0.5 * (A[i] * dx * dx + C[i] * dy * dy) - B[i] * dx * dy
        o = pr["opacity"][0, i]
        alpha = np.minimum(0.99, o * np.exp(power))
        flag |= (np.abs(power) <= reach) | (np.abs(power - np.log(1 / (255 * o))) <= reach)
        tol += np.where(power <= 0, alpha * np.expm1(reach), 0.0)
    tol = cm * tol + 1e-5
    ok = ~flag & (r["ambig"][0] == 0)
    assert ok.mean() >= 0.95
    err = np.abs(img - r["img"][0]).max(0)
    assert np.all(err[ok] <= tol[ok]), (err[ok].max(), tol[ok].min())


def test_transparent_gaussian_contributes_nothing():
    W, H = 48, 48
    cam = scenes.look_at_camera((0.0, 0.0, 4.0), W, H)
    g = scenes.make_gaussians(1, 0, np.random.default_rng(5))
    g.mean[:] = 0.0
    g.scale[:] = 0.3
    g.opacity_logit[:] = -20.0          # opacity 2e-9 < 1/255 everywhere
    img = _compare(g, [cam], W, H)
    assert np.all(img == 0.0)


def test_stage1_step_on_an_empty_set():
    """The cache and Adam on zero Gaussians: the loss is that of the
    background against the targets and no parameter moves."""
    W, H = 32, 24
    cams = scenes.ring_cameras([0, 90], [0, 0], W, H)
    G = gs3.Gaussians.from_numpy(_empty_set())
    rng = np.random.default_rng(6)
    og = oracle.Grid()
    table = rng.uniform(-1e-4, 1e-4, size=(og.n_entries, 2)).astype(np.float32)
    Ws = [w.astype(np.float32) for w in scenes.random_mlp([32, 64, 64, 7], rng)]
    for prec in (gs3.GS_MLP_FP32, gs3.GS_MLP_BF16):
        ntc = NTC(table, Ws, gs3.hashgrid(), prec)
        st = Stage1(G, ntc, 2, W, H, capacity=1024)
        tg = torch.rand(2, 3, H, W, device=DEV)
        t0, m0 = ntc.table.p.clone(), ntc.mlp.p.clone()
        loss = st.step(gs3.cameras_to_device(cams), tg).item()
        torch.cuda.synchronize()
        want, _, _ = oracle.loss_l1_dssim(np.zeros((2, 3, H, W)), tg.cpu().numpy())
        assert abs(loss - want) <= 1e-5 * max(want, 1.0)
        assert torch.equal(ntc.table.p, t0) and torch.equal(ntc.mlp.p, m0)
