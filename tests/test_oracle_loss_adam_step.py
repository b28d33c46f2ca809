"""Pins of the oracle's loss (Eq. 6), Adam (Suppl. A) and of the whole
Stage-1 backward (Section 4.1) by central finite differences in FP64."""
import math

import numpy as np
import pytest
from scipy import ndimage

import oracle
from paper_2403_01444_gb300 import scenes


def _ssim_scipy(x, y):
    """SSIM map mean with scipy's zero-padded correlation (library routine)."""
    g1 = np.exp(-((np.arange(11) - 5) ** 2) / (2 * 1.5 ** 2))
    g1 /= g1.sum()
    k = np.outer(g1, g1)
    f = lambda a: ndimage.correlate(a, k, mode="constant", cval=0.0)
    vals = []
    for a, b in zip(x.reshape(-1, *x.shape[-2:]), y.reshape(-1, *y.shape[-2:])):
        mx, my = f(a), f(b)
        sxx, syy, sxy = f(a * a) - mx ** 2, f(b * b) - my ** 2, f(a * b) - mx * my
        C1, C2 = 0.01 ** 2, 0.03 ** 2
        vals.append(((2 * mx * my + C1) * (2 * sxy + C2)) / ((mx ** 2 + my ** 2 + C1) * (sxx + syy + C2)))
    return float(np.mean(vals))


def test_window_is_normalised_gaussian():
    g = oracle.ssim_window()
    assert abs(g.sum() - 1) < 1e-15
    np.testing.assert_allclose(g / g[5], np.exp(-((np.arange(11) - 5) ** 2) / 4.5), rtol=1e-14)


def test_loss_matches_scipy_ssim():
    rng = np.random.default_rng(20)
    x = rng.uniform(size=(2, 3, 23, 31))
    y = np.clip(x + rng.normal(0, 0.1, size=x.shape), 0, 1)
    L, _, ss = oracle.loss_l1_dssim(x, y, 0.2)
    s_ref = _ssim_scipy(x, y)
    assert abs(ss - s_ref) < 1e-12
    assert abs(L - (0.8 * np.mean(np.abs(x - y)) + 0.2 * (1 - s_ref))) < 1e-12


def test_identical_images_zero_loss_zero_grad():
    rng = np.random.default_rng(21)
    x = rng.uniform(size=(1, 3, 20, 20))
    L, d, ss = oracle.loss_l1_dssim(x, x.copy(), 0.2)
    assert abs(ss - 1) < 1e-12 and abs(L) < 1e-12
    np.testing.assert_allclose(d, 0, atol=1e-14)


def test_l1_gradient_is_sign_over_n():
    rng = np.random.default_rng(22)
    x = rng.uniform(size=(2, 3, 9, 7))
    y = rng.uniform(size=x.shape)
    _, d, _ = oracle.loss_l1_dssim(x, y, 0.0)
    np.testing.assert_allclose(d, np.sign(x - y) / x.size, atol=1e-18)


def test_loss_gradient_finite_differences():
    rng = np.random.default_rng(23)
    x = rng.uniform(size=(1, 3, 14, 17))
    y = rng.uniform(size=x.shape)
    _, d, _ = oracle.loss_l1_dssim(x, y, 0.2)
    h = 1e-7
    for _ in range(40):
        idx = tuple(rng.integers(0, s) for s in x.shape)
        xp, xm = x.copy(), x.copy()
        xp[idx] += h
        xm[idx] -= h
        fd = (oracle.loss_l1_dssim(xp, y, 0.2, False)[0] - oracle.loss_l1_dssim(xm, y, 0.2, False)[0]) / (2 * h)
        assert abs(fd - d[idx]) < 1e-8, idx


def test_adam_first_step_and_constant_gradient():
    rng = np.random.default_rng(24)
    p0 = rng.normal(size=50)
    g = rng.normal(size=50)
    p, m, v = p0.copy(), np.zeros(50), np.zeros(50)
    for t in range(1, 6):
        oracle.adam(p, g, m, v, t, lr=0.002)
        # bias-corrected moments of a constant gradient are g and g^2 exactly
        np.testing.assert_allclose(p, p0 - t * 0.002 * g / (np.abs(g) + 1e-15), rtol=0, atol=1e-14)
    # loss-scale unscaling
    p2, m2, v2 = p0.copy(), np.zeros(50), np.zeros(50)
    oracle.adam(p2, g * 1024.0, m2, v2, 1, inv_scale=1 / 1024.0)
    np.testing.assert_allclose(p2, p0 - 0.002 * np.sign(g), atol=1e-14)


def test_adam_matches_torch():
    torch = pytest.importorskip("torch")
    rng = np.random.default_rng(25)
    p0 = rng.normal(size=40)
    p, m, v = p0.copy(), np.zeros(40), np.zeros(40)
    tp = torch.tensor(p0.copy(), requires_grad=True)
    opt = torch.optim.Adam([tp], lr=0.002, betas=(0.9, 0.99), eps=1e-15)
    for t in range(1, 8):
        g = rng.normal(size=40)
        oracle.adam(p, g, m, v, t)
        tp.grad = torch.tensor(g)
        opt.step()
    np.testing.assert_allclose(p, tp.detach().numpy(), rtol=1e-13, atol=1e-13)


def _fd_scene(seed):
    """64 Gaussians, two 32x32 views, hash grid 16x2 / 2^17 / 16..1024: the
    finite-difference sub-scene.  Resampled until no pixel lies near a
    compositing threshold."""
    for s in range(seed, seed + 40):
        rng = np.random.default_rng(s)
        g = scenes.make_gaussians(64, 1, rng, extent=0.6)
        g.scale = np.full((64, 3), 0.12, np.float32) * rng.uniform(0.7, 1.4, (64, 3)).astype(np.float32)
        cams = scenes.ring_cameras([0, 60], [0, 20], 32, 32)
        grid = oracle.Grid()
        table = rng.normal(0, 0.3, size=(grid.n_entries, 2))
        Ws = [w.astype(np.float64) for w in scenes.random_mlp([32, 64, 64, 7], rng)]
        p = oracle.NTCParams(grid, table, Ws)
        f = oracle.ntc_forward(p, g.mean, g.quat)
        r = oracle.render(g, cams, f["mean"], f["quat"])
        if r["ambig"].any():
            continue
        pr = r["proj"]
        if np.min(pr["margin"][pr["radius"] > 0]) < 1e-3:
            continue
        h_pre = np.concatenate([f["h1"], f["h2"]], 1)
        targets = rng.uniform(size=r["img"].shape)
        return p, g, cams, targets
    raise RuntimeError("no clean FD scene")


def test_stage1_backward_finite_differences():
    """Whole backward (loss -> compositing -> projection -> transformation ->
    MLP -> hash table) against central differences of the whole forward."""
    p, g, cams, targets = _fd_scene(30)
    out = oracle.stage1_loss_grads(p, g, cams, targets)
    rng = np.random.default_rng(31)
    h = 1e-6

    def loss_with(table=None, Ws=None):
        q = oracle.NTCParams(p.grid, p.table if table is None else table, p.Ws if Ws is None else Ws)
        return oracle.stage1_loss(q, g, cams, targets)

    # table entries touched by the points: pick the largest-gradient ones
    flat = np.abs(out["d_table"]).ravel()
    pick = np.argsort(-flat)[:12]
    for e in pick:
        tp, tm = p.table.copy(), p.table.copy()
        tp.ravel()[e] += h
        tm.ravel()[e] -= h
        fd = (loss_with(table=tp) - loss_with(table=tm)) / (2 * h)
        an = out["d_table"].ravel()[e]
        assert abs(fd - an) <= 1e-5 * abs(an) + 1e-10, (e, fd, an)
    for li in range(3):
        W = p.Ws[li]
        dW = out["dWs"][li]
        for e in np.argsort(-np.abs(dW).ravel())[:6]:
            Wp = [w.copy() for w in p.Ws]
            Wm = [w.copy() for w in p.Ws]
            Wp[li].ravel()[e] += h
            Wm[li].ravel()[e] -= h
            fd = (loss_with(Ws=Wp) - loss_with(Ws=Wm)) / (2 * h)
            an = dW.ravel()[e]
            assert abs(fd - an) <= 1e-5 * abs(an) + 1e-10, (li, e, fd, an)
    assert out["loss"] > 0


def test_identity_transform_reproduces_input_render():
    rng = np.random.default_rng(32)
    g = scenes.make_gaussians(300, 2, rng)
    cams = scenes.ring_cameras([0, 90], [0, 0], 64, 48)
    raw = np.zeros((300, 7))
    raw[:, 3] = 1.0
    mo, qo = oracle.apply(g.mean, g.quat, raw, [-1.5] * 3 + [1.5] * 3)
    a = oracle.render(g, cams)["img"]
    b = oracle.render(g, cams, mo, qo)["img"]
    np.testing.assert_allclose(a, b, atol=1e-12)


def test_adam_rate_schedule_closed_form():
    """The oracle's decayed rate: lr at the first update, lr * ratio at update
    decay_steps - 1 and after, a constant factor ratio^(1/(decay_steps - 1))
    between consecutive updates, and no decay for decay_steps <= 1."""
    lr, ratio, S = 0.002, 0.01, 150
    r = [oracle.adam_rate(lr, ratio, S, t) for t in range(S + 5)]
    assert r[0] == lr
    assert abs(r[S - 1] - lr * ratio) <= 1e-15 and all(x == r[S - 1] for x in r[S:])
    q = np.array(r[1:S]) / np.array(r[:S - 1])
    np.testing.assert_allclose(q, math.exp(math.log(ratio) / (S - 1)), rtol=1e-12)
    assert oracle.adam_rate(lr, ratio, 1, 7) == lr and oracle.adam_rate(lr, ratio, 0, 7) == lr
