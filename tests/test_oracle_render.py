"""Pins of the oracle's projection, SH colour, binning and compositing
(Section 3.2, Eq. 2-4) against closed forms, invariants, library routines,
brute force and finite differences."""
import math

import numpy as np
import pytest
from scipy.spatial.transform import Rotation

import oracle
from paper_2403_01444_gb300 import scenes

C0 = 0.5 / math.sqrt(math.pi)  # the l = 0 real SH constant, 1 / (2 sqrt(pi))


def _one_gaussian(mu, q, s, ologit, rgb, deg=0):
    K = (deg + 1) ** 2
    sh = np.zeros((1, K, 3), np.float32)
    sh[0, 0] = (np.asarray(rgb) - 0.5) / C0
    return scenes.GaussianSet(np.array([mu], np.float32), np.array([q], np.float32),
                              np.array([s], np.float32), np.array([ologit], np.float32), sh, deg)


@pytest.mark.parametrize("sigma,ologit", [(0.3, 0.4), (0.12, 3.0), (0.5, -1.0)])
def test_single_isotropic_gaussian_closed_form(sigma, ologit):
    """On the optical axis at depth z: Sigma2d = ((f sigma / z)^2 + 0.3) I, the
    2D mean is the principal point, pixel = c * min(0.99, o G) where alpha >= 1/255."""
    W, H = 96, 72
    cam = scenes.look_at_camera((0.0, 0.0, 4.0), W, H)
    c = np.array([0.7, 0.2, 0.45])
    g = _one_gaussian((0, 0, 0), (1, 0, 0, 0), (sigma,) * 3, ologit, c)
    r = oracle.render(g, [cam])
    z = 4.0
    sigma = float(np.float32(sigma))  # the set stores float32 scales
    var = (cam.fx * sigma / z) ** 2 + 0.3
    o = 1.0 / (1.0 + math.exp(-float(np.float32(ologit))))
    lam = var + math.sqrt(0.1)          # isotropic: the discriminant floor applies
    rad = math.ceil(3.0 * math.sqrt(lam))
    assert r["proj"]["radius"][0, 0] == rad
    np.testing.assert_allclose(r["proj"]["mean2d"][0, 0], [W / 2, H / 2], atol=1e-12)
    np.testing.assert_allclose(r["proj"]["conic"][0, 0], [1 / var, 0, 1 / var], rtol=1e-12, atol=1e-15)
    tx0, tx1 = max(0, math.floor((W / 2 - rad) / 16)), min(6, math.floor((W / 2 + rad + 15) / 16))
    ty0, ty1 = max(0, math.floor((H / 2 - rad) / 16)), min(5, math.floor((H / 2 + rad + 15) / 16))
    want = np.zeros((3, H, W))
    for j in range(H):
        for i in range(W):
            if not (tx0 <= i // 16 < tx1 and ty0 <= j // 16 < ty1):
                continue
            d2 = (i + 0.5 - W / 2) ** 2 + (j + 0.5 - H / 2) ** 2
            a = min(0.99, o * math.exp(-0.5 * d2 / var))
            if a >= 1 / 255:
                want[:, j, i] = c * a
    np.testing.assert_allclose(r["img"][0], want, atol=1e-12)


def _perspective_jacobian(cam, mu):
    Rw = cam.viewmat[:, :3].astype(np.float64)
    tw = cam.viewmat[:, 3].astype(np.float64)

    def pi(x):
        t = Rw @ x + tw
        return np.array([cam.fx * t[0] / t[2] + cam.cx, cam.fy * t[1] / t[2] + cam.cy])

    h = 1e-6
    Jn = np.zeros((2, 3))
    for k in range(3):
        e = np.zeros(3)
        e[k] = h
        Jn[:, k] = (pi(mu + e) - pi(mu - e)) / (2 * h)
    return pi(mu), Jn, (Rw @ mu + tw)[2]


def test_projection_matches_numerical_jacobian():
    """EWA (Eq. 3): Sigma2d = J W Sigma W^T J^T + 0.3 I with J W the Jacobian of
    the perspective map, Sigma = R S S^T R^T (Eq. 2, rotation via scipy)."""
    rng = np.random.default_rng(11)
    cams = scenes.ring_cameras([0, 70, 200], [0, 15, -10], 320, 240)
    g = scenes.make_gaussians(60, 1, rng)
    g.mean *= 0.5  # keep inside the field of view, where J is not clamped
    g.scale = (g.scale * 4).astype(np.float32)
    pr = oracle.project(g, cams)
    for v, cam in enumerate(cams):
        for i in range(g.n):
            mu = g.mean[i].astype(np.float64)
            uv, Jn, tz = _perspective_jacobian(cam, mu)
            R = Rotation.from_quat(g.quat[i, [1, 2, 3, 0]].astype(np.float64)).as_matrix()
            S = np.diag(g.scale[i].astype(np.float64))
            Sig2 = Jn @ (R @ S @ S @ R.T) @ Jn.T + 0.3 * np.eye(2)
            if pr["radius"][v, i] == 0:
                continue
            A, B, C = pr["conic"][v, i]
            np.testing.assert_allclose(np.linalg.inv([[A, B], [B, C]]), Sig2, rtol=1e-6, atol=1e-7)
            np.testing.assert_allclose(pr["mean2d"][v, i], uv, rtol=1e-12)
            assert abs(pr["depth"][v, i] - tz) < 1e-12
            lmax = np.linalg.eigvalsh(Sig2)[-1]
            assert math.ceil(3 * math.sqrt(lmax)) <= pr["radius"][v, i] <= math.ceil(3 * math.sqrt(lmax + 0.32))


def test_negated_quaternion_same_projection():
    rng = np.random.default_rng(12)
    cams = scenes.ring_cameras([0, 120], [0, 10], 160, 120)
    g = scenes.make_gaussians(40, 2, rng)
    a = oracle.project(g, cams)
    b = oracle.project(g, cams, quat=-g.quat.astype(np.float64) * 3.0)  # any scale, either sign
    for k in ("mean2d", "conic", "rgb", "depth", "radius"):
        np.testing.assert_allclose(a[k], b[k], rtol=1e-12, atol=1e-14)


def test_near_plane_culls():
    cam = scenes.look_at_camera((0.0, 0.0, 4.0), 64, 64)
    g = _one_gaussian((0, 0, 3.85), (1, 0, 0, 0), (0.05,) * 3, 0.0, (0.5, 0.5, 0.5))
    assert oracle.project(g, [cam])["radius"][0, 0] == 0  # depth 0.15 <= 0.2
    g = _one_gaussian((0, 0, 3.75), (1, 0, 0, 0), (0.05,) * 3, 0.0, (0.5, 0.5, 0.5))
    assert oracle.project(g, [cam])["radius"][0, 0] > 0   # depth 0.25


def test_sh_basis_orthonormal_harmonic():
    deg = 3
    # Gauss-Legendre in cos(theta) x uniform phi integrates degree <= 6 exactly
    xg, wg = np.polynomial.legendre.leggauss(12)
    phi = np.arange(24) * (2 * np.pi / 24)
    ct, ph = np.meshgrid(xg, phi, indexing="ij")
    st = np.sqrt(1 - ct ** 2)
    dirs = np.stack([st * np.cos(ph), st * np.sin(ph), ct], -1).reshape(-1, 3)
    w = (wg[:, None] * np.full_like(ph, 2 * np.pi / 24)).reshape(-1)
    Y, G = oracle.sh_basis(deg, dirs)
    gram = (Y * w[:, None]).T @ Y
    np.testing.assert_allclose(gram, np.eye(16), atol=1e-12)
    # each band l is a homogeneous harmonic polynomial of degree l
    rng = np.random.default_rng(13)
    pts = rng.normal(size=(10, 3))
    band = [0] + [1] * 3 + [2] * 5 + [3] * 7
    Y1, G1 = oracle.sh_basis(deg, pts)
    Y2, _ = oracle.sh_basis(deg, 1.7 * pts)
    np.testing.assert_allclose(Y2, Y1 * 1.7 ** np.array(band), rtol=1e-12, atol=1e-12)
    h = 1e-3
    lap = -6 * Y1
    for k in range(3):
        e = np.zeros(3)
        e[k] = h
        lap = lap + oracle.sh_basis(deg, pts + e)[0] + oracle.sh_basis(deg, pts - e)[0]
        gfd = (oracle.sh_basis(deg, pts + e)[0] - oracle.sh_basis(deg, pts - e)[0]) / (2 * h)
        np.testing.assert_allclose(G1[:, :, k], gfd, rtol=1e-5, atol=1e-5)
    np.testing.assert_allclose(lap / h ** 2, 0, atol=1e-5)


def _records(V, N, W, H, seed, **kw):
    rng = np.random.default_rng(seed)
    return scenes.random_projected(V, N, W, H, rng, **kw)


def test_two_gaussians_blend_and_swap():
    W = H = 32
    rec = dict(mean2d=np.array([[[16.5, 16.5], [16.5, 16.5]]], np.float32),
               conic=np.array([[[0.02, 0.0, 0.02], [0.05, 0.01, 0.03]]], np.float32),
               opacity=np.array([[0.6, 0.7]], np.float32),
               rgb=np.array([[[1.0, 0.2, 0.1], [0.0, 0.5, 0.9]]], np.float32),
               depth=np.array([[2.0, 3.0]], np.float32), radius=np.array([[10, 10]], np.int32))
    img, Tf, last, _ = oracle.raster_fwd(rec, W, H)
    a1, a2 = 0.6, 0.7  # at the shared centre power = 0
    c1, c2 = rec["rgb"][0, 0].astype(np.float64), rec["rgb"][0, 1].astype(np.float64)
    np.testing.assert_allclose(img[0, :, 16, 16], c1 * a1 + c2 * a2 * (1 - a1), rtol=1e-6)
    assert abs(Tf[0, 16, 16] - (1 - a1) * (1 - a2)) < 1e-7
    assert last[0, 16, 16] == 2
    rec["depth"] = np.array([[3.0, 2.0]], np.float32)
    img2, _, _, _ = oracle.raster_fwd(rec, W, H)
    np.testing.assert_allclose(img2[0, :, 16, 16], c2 * a2 + c1 * a1 * (1 - a2), rtol=1e-6)


@pytest.mark.parametrize("ologit", [5.0, 10.0])
def test_alpha_cap_closed_form(ologit):
    """Eq. 4 with the 0.99 cap: an isotropic Gaussian of opacity above 0.99
    (logit 5: o = 0.99331; logit 10: o = 0.99995) on the optical axis.  On the
    disc where o G >= 0.99 the pixel is exactly 0.99 c and 0.01 of the light
    is left: T (1 - 0.99) = 0.01 is far above the 1e-4 cutoff, so the Gaussian
    is added.  Outside the disc the pixel is c o G.  (Were the cutoff tested
    on the uncapped alpha, the logit-10 centre would give T (1 - alpha) =
    5e-5 < 1e-4 and stay empty; a cap of 0.999 would give 0.999 c.)"""
    W, H = 96, 72
    cam = scenes.look_at_camera((0.0, 0.0, 4.0), W, H)
    c = np.array([0.7, 0.2, 0.45])
    g = _one_gaussian((0, 0, 0), (1, 0, 0, 0), (1.0,) * 3, ologit, c)
    r = oracle.render(g, [cam])
    var = (cam.fx * 1.0 / 4.0) ** 2 + 0.3
    o = 1.0 / (1.0 + math.exp(-float(np.float32(ologit))))
    assert o > 0.99
    want = np.zeros((3, H, W))
    want_T = np.ones((H, W))
    capped = 0
    for j in range(H):
        for i in range(W):
            x = o * math.exp(-0.5 * ((i + 0.5 - W / 2) ** 2 + (j + 0.5 - H / 2) ** 2) / var)
            assert abs(x - 0.99) > 1e-9 and abs(x - 1 / 255) > 1e-9  # no pixel on a threshold
            if x >= 0.99:
                want[:, j, i], want_T[j, i] = 0.99 * c, 0.01
                capped += 1
            elif x >= 1 / 255:
                want[:, j, i], want_T[j, i] = c * x, 1.0 - x
    assert capped >= 8
    np.testing.assert_allclose(r["img"][0], want, atol=1e-12)
    np.testing.assert_allclose(r["T_final"][0], want_T, atol=1e-12)


def _stack_records(opacities, W=32, H=32, conic=(0.002, 0.0, 0.002)):
    """Gaussians centred on the pixel centre (16.5, 16.5), in depth order,
    with broad footprints (float64 records)."""
    n = len(opacities)
    f = lambda a: np.array([a], np.float64)
    return dict(mean2d=f([[16.5, 16.5]] * n), conic=f([list(conic)] * n),
                opacity=f(list(opacities)), depth=f([1.0 + k for k in range(n)]),
                rgb=f([[0.9, 0.1, 0.3], [0.2, 0.8, 0.4], [0.5, 0.5, 1.0]][:n]),
                radius=np.array([[40] * n], np.int32))


def test_alpha_cap_then_cutoff_sequence():
    """At the shared centre (power 0): a Gaussian of opacity 0.999 is capped
    to alpha 0.99 (T 1 -> 0.01), one of opacity 0.5 is added (T -> 0.005), and
    a third capped one would leave T (1 - 0.99) = 5e-5 < 1e-4, so the loop
    stops without adding it: C = 0.99 c1 + 0.01 * 0.5 c2, T_final = 0.005,
    last = 2 (Eq. 4 with the cap, the 1e-4 cutoff tested on the capped alpha)."""
    rec = _stack_records([0.999, 0.5, 0.999])
    img, Tf, last, _ = oracle.raster_fwd(rec, 32, 32)
    c1, c2 = rec["rgb"][0, 0], rec["rgb"][0, 1]
    np.testing.assert_allclose(img[0, :, 16, 16], 0.99 * c1 + 0.005 * c2, rtol=0, atol=1e-15)
    assert abs(Tf[0, 16, 16] - 0.005) < 1e-15
    assert last[0, 16, 16] == 2


def test_alpha_cap_zero_gradient_finite_differences():
    """Through a capped pixel alpha = 0.99 is constant, so the pixel has no
    gradient with respect to the capped Gaussian's opacity, conic or 2D mean,
    and its colour gradient is 0.99 T; the Gaussian behind still receives its
    gradients through T = 0.01.  The image gradient is non-zero only on
    pixels well inside the capped disc (o G >= 0.99 (1 + 1e-4)), where central
    differences with h = 1e-6 cross no decision: analytic reverse and finite
    differences must agree, and the capped Gaussian's opacity, conic and mean
    gradients must vanish."""
    W = H = 32
    rec = _stack_records([0.9995, 0.6], W, H, conic=(0.004, 0.0005, 0.003))
    rec["mean2d"][0, 1] = [18.2, 15.1]
    rec["conic"][0, 1] = [0.02, -0.004, 0.015]
    yy, xx = np.mgrid[0:H, 0:W] + 0.5
    dx, dy = xx - 16.5, yy - 16.5
    A, B, C = rec["conic"][0, 0]
    x1 = rec["opacity"][0, 0] * np.exp(-0.5 * (A * dx * dx + C * dy * dy) - B * dx * dy)
    inside = x1 >= 0.99 * (1 + 1e-4)
    assert inside.sum() >= 12 and not inside.all()
    rng = np.random.default_rng(17)
    dimg = rng.normal(size=(1, 3, H, W)) * inside[None, None]
    img, Tf, last, _ = oracle.raster_fwd(rec, W, H)
    grads, dop = oracle.raster_bwd(rec, W, H, Tf, last, dimg, want_opacity=True)
    # the capped Gaussian: no opacity / conic / mean gradient, colour gradient 0.99 * sum dimg
    assert np.all(grads[0, 0, :5] == 0) and dop[0, 0] == 0
    np.testing.assert_allclose(grads[0, 0, 5:], 0.99 * dimg[0].sum((1, 2)), rtol=1e-12)
    # the Gaussian behind receives gradients (through T = 0.01)
    assert np.abs(grads[0, 1, :5]).max() > 1e-6 and abs(dop[0, 1]) > 1e-6

    def f(r):
        return np.sum(oracle.raster_fwd(r, W, H)[0] * dimg)

    h = 1e-6
    for i in range(2):
        for key, comp, gi in [("mean2d", 0, 0), ("mean2d", 1, 1), ("conic", 0, 2), ("conic", 1, 3),
                              ("conic", 2, 4), ("rgb", 0, 5), ("rgb", 1, 6), ("rgb", 2, 7),
                              ("opacity", None, None)]:
            rp = {k: v.copy() for k, v in rec.items()}
            rm = {k: v.copy() for k, v in rec.items()}
            if comp is None:
                rp[key][0, i] += h
                rm[key][0, i] -= h
                want = dop[0, i]
            else:
                rp[key][0, i, comp] += h
                rm[key][0, i, comp] -= h
                want = grads[0, i, gi]
            fd = (f(rp) - f(rm)) / (2 * h)
            assert abs(fd - want) <= 1e-7 * max(1.0, abs(fd)), (i, key, comp, fd, want)


def test_transmittance_invariants():
    W, H = 80, 64
    rec = _records(2, 400, W, H, 14)
    img, Tf, last, _ = oracle.raster_fwd(rec, W, H)
    assert np.all(Tf > 0) and np.all(Tf <= 1)
    assert np.all(Tf >= 1e-4)  # the loop stops before T drops below the cutoff
    cmax = rec["rgb"].max()
    assert np.all(img <= cmax + 1e-12) and np.all(img >= 0)
    assert np.all(img.sum(1) <= 3 * cmax * (1 - Tf) + 1e-9)
    # a background shows through by exactly T_final
    img_bg, _, _, _ = oracle.raster_fwd(rec, W, H, bg=(0.25, 0.5, 1.0))
    np.testing.assert_allclose(img_bg - img, Tf[:, None] * np.array([0.25, 0.5, 1.0])[None, :, None, None],
                               atol=1e-12)
    # fewer Gaussians can only raise transmittance (monotone along each list)
    rec2 = {k: v.copy() for k, v in rec.items()}
    rec2["radius"][:, 200:] = 0
    _, Tf2, _, _ = oracle.raster_fwd(rec2, W, H)
    hit = (last > 0)
    assert np.mean(Tf2[hit] >= Tf[hit] - 1e-12) > 0.999


def test_bin_sort_brute_force():
    W, H = 70, 50
    rec = _records(3, 120, W, H, 15)
    count, keys, vals, ranges = oracle.bin_sort(rec["mean2d"], rec["radius"], rec["depth"], W, H)
    tx, ty = math.ceil(W / 16), math.ceil(H / 16)
    pairs = []
    for v in range(3):
        for i in range(120):
            r = int(rec["radius"][v, i])
            if r <= 0:
                continue
            u, w = (float(x) for x in rec["mean2d"][v, i])
            x0 = min(tx, max(0, math.floor((u - r) / 16)))
            x1 = min(tx, max(0, math.floor((u + r + 15) / 16)))
            y0 = min(ty, max(0, math.floor((w - r) / 16)))
            y1 = min(ty, max(0, math.floor((w + r + 15) / 16)))
            dbits = int(np.float32(rec["depth"][v, i]).view(np.uint32))
            for y in range(y0, y1):
                for x in range(x0, x1):
                    pairs.append((((v * tx * ty + y * tx + x) << 32) | dbits, i))
    pairs.sort()
    assert count == len(pairs) > 0
    assert [int(k) for k in keys] == [p[0] for p in pairs]
    assert [int(x) for x in vals] == [p[1] for p in pairs]
    for t in range(3 * tx * ty):
        idx = [j for j, p in enumerate(pairs) if p[0] >> 32 == t]
        want = (idx[0], idx[-1] + 1) if idx else (0, 0)
        assert tuple(int(x) for x in ranges[t]) == want


def _clean_scene_records(W, H, seed, N=150):
    """Records with no pixel near a threshold of the compositing (so that
    finite differences with a tiny step do not cross a decision)."""
    for s in range(seed, seed + 50):
        rec = _records(1, N, W, H, s, radius_range=(4, 18), margin=8)
        rec = {k: (v.astype(np.float64) if v.dtype == np.float32 else v) for k, v in rec.items()}
        _, _, _, amb = oracle.raster_fwd(rec, W, H)
        if not amb.any():
            return rec
    raise RuntimeError("no clean scene")


def test_raster_bwd_finite_differences():
    W, H = 40, 36
    rec = _clean_scene_records(W, H, 100, N=60)
    rng = np.random.default_rng(16)
    dimg = rng.normal(size=(1, 3, H, W))
    img, Tf, last, _ = oracle.raster_fwd(rec, W, H)
    grads, dop = oracle.raster_bwd(rec, W, H, Tf, last, dimg, want_opacity=True)

    def f(r):
        return np.sum(oracle.raster_fwd(r, W, H)[0] * dimg)

    h = 1e-6
    idx = np.argsort(-np.abs(grads[0]).sum(1))[:8]
    for i in idx:
        for key, comp, gi in [("mean2d", 0, 0), ("mean2d", 1, 1), ("conic", 0, 2), ("conic", 1, 3),
                              ("conic", 2, 4), ("rgb", 0, 5), ("rgb", 1, 6), ("rgb", 2, 7)]:
            rp = {k: v.copy() for k, v in rec.items()}
            rm = {k: v.copy() for k, v in rec.items()}
            rp[key][0, i, comp] += h
            rm[key][0, i, comp] -= h
            fd = (f(rp) - f(rm)) / (2 * h)
            assert abs(fd - grads[0, i, gi]) <= 1e-6 * max(1.0, abs(fd)), (i, key, comp)
        rp = {k: v.copy() for k, v in rec.items()}
        rm = {k: v.copy() for k, v in rec.items()}
        rp["opacity"][0, i] += h
        rm["opacity"][0, i] -= h
        fd = (f(rp) - f(rm)) / (2 * h)
        assert abs(fd - dop[0, i]) <= 1e-6 * max(1.0, abs(fd))


def test_project_bwd_finite_differences():
    rng = np.random.default_rng(17)
    cams = scenes.ring_cameras([0, 100], [5, -10], 200, 150)
    g = scenes.make_gaussians(30, 3, rng)
    g.sh[:, 1:, :] *= 10  # make view dependence visible
    mean = g.mean.astype(np.float64)
    quat = g.quat.astype(np.float64) * 1.3
    pr = oracle.project(g, cams, mean=mean, quat=quat)
    G = rng.normal(size=(2, 30, 8))
    G *= (pr["radius"] > 0)[..., None]

    def f(m, q):
        p = oracle.project(g, cams, mean=m, quat=q)
        out = np.concatenate([p["mean2d"], p["conic"], p["rgb"]], -1)
        return np.sum(out * G)

    dm, dq = oracle.project_bwd(g, cams, G, mean=mean, quat=quat)
    h = 1e-6
    for i in range(30):
        for k in range(3):
            mp, mm = mean.copy(), mean.copy()
            mp[i, k] += h
            mm[i, k] -= h
            fd = (f(mp, quat) - f(mm, quat)) / (2 * h)
            assert abs(fd - dm[i, k]) <= 1e-5 * max(1.0, abs(fd)), (i, k)
        for k in range(4):
            qp, qm = quat.copy(), quat.copy()
            qp[i, k] += h
            qm[i, k] -= h
            fd = (f(mean, qp) - f(mean, qm)) / (2 * h)
            assert abs(fd - dq[i, k]) <= 1e-5 * max(1.0, abs(fd)), (i, k)


def test_project_bwd_full_finite_differences():
    """Every parameter (mean, rotation, scale, opacity logit, SH) against
    central finite differences of the FP64 projection, with a gradient on the
    opacity of every record as well."""
    rng = np.random.default_rng(19)
    cams = scenes.ring_cameras([0, 100], [5, -10], 200, 150)
    g0 = scenes.make_gaussians(20, 2, rng)
    g0.sh[:, 1:, :] *= 10
    g = scenes.GaussianSet(g0.mean.astype(np.float64), g0.quat.astype(np.float64) * 1.3,
                           g0.scale.astype(np.float64), g0.opacity_logit.astype(np.float64),
                           g0.sh.astype(np.float64), g0.sh_deg)
    pr = oracle.project(g, cams)
    vis = (pr["radius"] > 0)
    G = rng.normal(size=(2, 20, 8)) * vis[..., None]
    D = rng.normal(size=(2, 20)) * vis

    def f(gg):
        p = oracle.project(gg, cams)
        out = np.concatenate([p["mean2d"], p["conic"], p["rgb"]], -1)
        return np.sum(out * G) + np.sum(p["opacity"] * D)

    d = oracle.project_bwd_full(g, cams, G, D)
    dm, dq = oracle.project_bwd(g, cams, G)
    np.testing.assert_allclose(d["d_mean"], dm, rtol=1e-12, atol=1e-12)
    np.testing.assert_allclose(d["d_quat"], dq, rtol=1e-12, atol=1e-12)
    h = 1e-6
    for name, key in (("scale", "d_scale"), ("opacity_logit", "d_ologit"), ("sh", "d_sh")):
        base = getattr(g, name)
        for idx in np.ndindex(*base.shape):
            if rng.uniform() > (0.35 if name == "sh" else 1.0):
                continue   # a sample of the SH coefficients keeps the test short
            gp, gm = g.copy(), g.copy()
            getattr(gp, name)[idx] += h
            getattr(gm, name)[idx] -= h
            fd = (f(gp) - f(gm)) / (2 * h)
            assert abs(fd - d[key][idx]) <= 1e-5 * max(1.0, abs(fd)), (name, idx, fd, d[key][idx])


def test_project_bwd_clamped_jacobian_finite_differences():
    """Gaussians outside 1.3x the half field of view (J evaluated at the clamp)."""
    cam = scenes.look_at_camera((0.0, 0.0, 4.0), 64, 48)
    rng = np.random.default_rng(18)
    n = 12
    mean = np.stack([rng.uniform(3.2, 3.6, n) * rng.choice([-1, 1], n),
                     rng.uniform(-0.3, 0.3, n), rng.uniform(-0.5, 0.5, n)], 1)
    g = scenes.make_gaussians(n, 0, rng)
    g.scale = np.full((n, 3), 1.2, np.float32)  # large enough to reach the image
    pr = oracle.project(g, [cam], mean=mean)
    assert (pr["radius"] > 0).sum() >= 4
    G = rng.normal(size=(1, n, 8)) * (pr["radius"] > 0)[..., None]

    def f(m):
        p = oracle.project(g, [cam], mean=m)
        return np.sum(np.concatenate([p["mean2d"], p["conic"], p["rgb"]], -1) * G)

    dm, _ = oracle.project_bwd(g, [cam], G, mean=mean)
    h = 1e-6
    for i in range(n):
        for k in range(3):
            mp, mm = mean.copy(), mean.copy()
            mp[i, k] += h
            mm[i, k] -= h
            fd = (f(mp) - f(mm)) / (2 * h)
            assert abs(fd - dm[i, k]) <= 1e-5 * max(1.0, abs(fd)), (i, k)


def _pair_records(depth_a, depth_b, W=32, H=32):
    return dict(mean2d=np.array([[[15.2, 16.1], [17.3, 15.4]]]),
                conic=np.array([[[0.03, 0.004, 0.025], [0.02, -0.003, 0.04]]]),
                opacity=np.array([[0.8, 0.65]]),
                rgb=np.array([[[0.9, 0.2, 0.1], [0.1, 0.6, 0.8]]]),
                depth=np.array([[depth_a, depth_b]]), radius=np.array([[14, 14]], np.int32))


def test_tie_swap_bound_is_the_exact_swap_effect():
    """Two Gaussians at (almost) the same depth: the oracle's per-pixel swap
    bound must equal the change that swapping them actually makes (brute force,
    by re-rendering in the other order), so that the pixel is flagged exactly
    where that change exceeds the budget."""
    W = H = 32
    d = 3.0
    img_ab, Tf_ab, _, _ = oracle.raster_fwd(_pair_records(d, d * (1 + 1e-9)), W, H)
    img_ba, Tf_ba, _, _ = oracle.raster_fwd(_pair_records(d * (1 + 1e-9), d), W, H)
    np.testing.assert_allclose(Tf_ab, Tf_ba, atol=1e-15)   # the product of (1 - alpha) is order-free
    effect = np.abs(img_ab - img_ba).max(axis=1)[0]
    assert effect.max() > 0.05
    for budget in (1e-3, 1e-2, 5e-2):
        _, _, _, amb = oracle.raster_fwd(_pair_records(d, d * (1 + 1e-9)), W, H, tie=1e-8,
                                         tie_budget=budget)
        clear = np.abs(effect - budget) > 1e-9
        assert np.array_equal(amb[0][clear] == 1, effect[clear] > budget)
    # without a tie margin nothing is flagged here
    _, _, _, amb = oracle.raster_fwd(_pair_records(d, d * (1 + 1e-9)), W, H)
    assert not amb.any()


def test_tie_run_of_three_always_flags():
    W = H = 32
    rec = _pair_records(3.0, 3.0 * (1 + 1e-9), W, H)
    rec = {k: np.concatenate([v, v[:, :1]], axis=1) for k, v in rec.items()}
    rec["depth"][0, 2] = 3.0 * (1 + 2e-9)
    rec["rgb"][0, 2] = rec["rgb"][0, 0]
    _, _, _, amb = oracle.raster_fwd(rec, W, H, tie=1e-8, tie_budget=1.0)
    yy, xx = np.mgrid[0:H, 0:W] + 0.5
    added = np.ones((H, W), bool)
    for i in range(3):
        dx, dy = xx[None] - rec["mean2d"][0, i, 0], yy[None] - rec["mean2d"][0, i, 1]
        A, B, C = rec["conic"][0, i]
        a = rec["opacity"][0, i] * np.exp(-0.5 * (A * dx * dx + C * dy * dy) - B * dx * dy)[0]
        added &= a >= 1 / 255 + 1e-9
    assert added.sum() > 100
    assert np.all(amb[0][added] == 1)


def _added_sets(rec, W, H):
    """Brute force over all pixels at once: which Gaussians the compositing
    adds (Eq. 4 with the 1/255, 0.99 and 1e-4 rules), as a [N, H, W] mask.
    Every rectangle covers the image, so tile lists hold every Gaussian."""
    yy, xx = np.mgrid[0:H, 0:W] + 0.5
    T = np.ones((H, W))
    alive = np.ones((H, W), bool)
    N = rec["depth"].shape[1]
    added = np.zeros((N, H, W), bool)
    for i in np.argsort(rec["depth"][0], kind="stable"):
        dx, dy = xx - rec["mean2d"][0, i, 0], yy - rec["mean2d"][0, i, 1]
        A, B, C = rec["conic"][0, i]
        power = -0.5 * (A * dx * dx + C * dy * dy) - B * dx * dy
        a = np.minimum(0.99, rec["opacity"][0, i] * np.exp(power))
        take = alive & (power <= 0) & (a >= 1 / 255)
        tt = T * (1 - a)
        stop = take & (tt < 1e-4)
        alive &= ~stop
        take &= ~stop
        added[i] = take
        T = np.where(take, tt, T)
    return added


@pytest.mark.parametrize("pos_eps,rel_eps", [(0.02, 0.0), (0.0, 5e-3), (0.05, 1e-2)])
def test_perturbation_reach_covers_flipped_decisions(pos_eps, rel_eps):
    """Every pixel whose set of added Gaussians changes when the 2D means move
    by up to pos_eps pixels or the conics by up to rel_eps (relative) must be
    flagged when the oracle is given those reaches (brute force over random
    shifts and scalings of the inputs)."""
    W, H = 48, 40
    rec = _records(1, 40, W, H, 31, radius_range=(4, 14))
    rec = {k: (v.astype(np.float64) if v.dtype == np.float32 else v) for k, v in rec.items()}
    rec["depth"][0] = np.arange(1, 41) * 0.1   # distinct depths: no ties
    rec["radius"][0] = 200                      # rectangles cover the image
    _, _, _, amb = oracle.raster_fwd(rec, W, H, pos_eps=pos_eps, rel_eps=rel_eps)
    base = _added_sets(rec, W, H)
    changed = np.zeros((H, W), bool)
    rng = np.random.default_rng(32)
    for trial in range(24):
        r = {k: v.copy() for k, v in rec.items()}
        ang = rng.uniform(0, 2 * np.pi, size=40)
        r["mean2d"][0] += pos_eps * np.stack([np.cos(ang), np.sin(ang)], 1)
        r["conic"][0] *= 1 + rel_eps * rng.choice([-1.0, 1.0], size=(40, 1))
        changed |= np.any(_added_sets(r, W, H) != base, axis=0)
    assert changed.sum() >= 5
    assert np.all(amb[0][changed] == 1)
    # the reach is not vacuous: most pixels stay unflagged
    assert amb.mean() < 0.5


def _quat_of(rot):
    x, y, z, w = rot.as_quat().T if rot.as_quat().ndim == 2 else rot.as_quat()
    return np.stack([w, x, y, z], -1)


def test_sh_rotate_pins():
    """SH rotation: identity, composition of two rotations, the defining
    identity at directions outside the fit, energy per band (orthonormal
    basis) and the degree-1 closed form (the band is a dot product with a
    vector, which turns with the Gaussian)."""
    rng = np.random.default_rng(60)
    n, deg = 6, 3
    sh = rng.normal(size=(n, 16, 3))
    R1 = Rotation.random(n, random_state=61)
    R2 = Rotation.random(n, random_state=62)
    q0 = _quat_of(Rotation.identity(n))
    q1, q21 = _quat_of(R1), _quat_of(R2 * R1)
    np.testing.assert_allclose(oracle.sh_rotate(sh, q0, q0, deg), sh, atol=1e-12)
    a = oracle.sh_rotate(sh, q0, q1, deg)
    b = oracle.sh_rotate(a, q1, q21, deg)
    np.testing.assert_allclose(b, oracle.sh_rotate(sh, q0, q21, deg), atol=1e-10)
    # colour from d after == colour from R^T d before, d random
    d = rng.normal(size=(50, 3))
    d /= np.linalg.norm(d, axis=1, keepdims=True)
    Yd, _ = oracle.sh_basis(deg, d)
    for i in range(n):
        Rm = R1[i].as_matrix()
        Yr, _ = oracle.sh_basis(deg, d @ Rm)
        np.testing.assert_allclose(Yd @ a[i], Yr @ sh[i], atol=1e-10)
    for lo, hi in ((0, 1), (1, 4), (4, 9), (9, 16)):
        np.testing.assert_allclose(np.linalg.norm(a[:, lo:hi], axis=1),
                                   np.linalg.norm(sh[:, lo:hi], axis=1), rtol=1e-10)
    np.testing.assert_allclose(a[:, 0], sh[:, 0], atol=1e-12)   # band 0 is invariant
    # degree 1: Y = C1 (-y, z, -x), so the band is C1 v.d with v = (-c3, -c1, c2);
    # turning the Gaussian turns v: v' = R v
    for i in range(n):
        c = sh[i, 1:4]                                  # [3 coefficients, 3 channels]
        v = np.stack([-c[2], -c[0], c[1]])              # [xyz, channel]
        v2 = R1[i].as_matrix() @ v
        np.testing.assert_allclose(a[i, 1:4], np.stack([-v2[1], v2[2], -v2[0]]), atol=1e-10)
