"""Pins of the Stage-2 oracle (Section 4.2, adaptive 3DG addition) against
hand-worked values, closed forms, sample statistics, library routines and
finite differences."""
import math

import numpy as np
import pytest
from scipy.spatial.transform import Rotation
from scipy.special import expit, logit

import oracle
from oracle import stage2 as s2
from paper_2403_01444_gb300 import scenes


def test_viewspace_grad_hand_example():
    """|(dL/du W/2, dL/dv H/2)| summed over the views where the Gaussian is
    visible: (0.01*100, 0.02*50) -> sqrt(2); view 2 invisible; (-0.03*100, 0) -> 3."""
    grads = np.zeros((3, 1, 8))
    grads[0, 0, :2] = (0.01, 0.02)
    grads[1, 0, :2] = (9.0, 9.0)
    grads[2, 0, :2] = (-0.03, 0.0)
    radius = np.array([[5], [0], [3]])
    acc, den = s2.viewspace_grad(grads, radius, 200, 100)
    assert den[0] == 2
    assert abs(acc[0] - (math.sqrt(2) + 3.0)) < 1e-12
    acc4, _ = s2.viewspace_grad(grads, radius, 200, 100, grad_scale=4.0)
    assert abs(acc4[0] - 4 * acc[0]) < 1e-12


def test_select_above_is_strict_and_ordered():
    acc = np.array([0.3, 0.0, 0.5, 0.2, 0.9])
    den = np.array([2, 0, 1, 1, 3])
    # averages 0.15, -, 0.5, 0.2, 0.3
    assert list(s2.select_above(acc, den, 0.2)) == [2, 4]
    assert list(s2.select_above(acc, den, 0.1)) == [0, 2, 3, 4]


def _set(n, deg, rng):
    g = scenes.make_gaussians(n, deg, rng)
    return g


def test_spawn_identity_rotation_closed_form():
    rng = np.random.default_rng(40)
    g = _set(5, 2, rng)
    g.quat[:] = (1, 0, 0, 0)
    z = rng.normal(size=(3, 3))
    idx = np.array([4, 0, 2])
    rows = s2.spawn(g, idx, z, opacity_init=0.1)
    s = g.scale[idx].astype(np.float64)
    np.testing.assert_allclose(rows[:, 0:3], g.mean[idx] + math.sqrt(2) * s * z, rtol=1e-12, atol=1e-12)
    np.testing.assert_array_equal(rows[:, 3:7], np.tile([1.0, 0, 0, 0], (3, 1)))
    np.testing.assert_allclose(rows[:, 7:10], np.log(s), rtol=1e-12)
    np.testing.assert_allclose(rows[:, 10], logit(0.1), rtol=1e-12)
    np.testing.assert_array_equal(rows[:, 11:], g.sh[idx].reshape(3, -1).astype(np.float64))


def test_spawn_samples_have_twice_the_covariance():
    """Sample covariance of 400 000 spawns around one rotated anisotropic
    Gaussian against 2 Sigma, Sigma = R diag(s)^2 R^T with R from scipy."""
    rng = np.random.default_rng(41)
    g = _set(1, 0, rng)
    g.scale[:] = (0.1, 0.05, 0.02)
    rot = Rotation.random(random_state=42)
    x, y, z_, w = rot.as_quat()          # scipy: (x, y, z, w)
    g.quat[:] = (w, x, y, z_)
    n = 400_000
    rows = s2.spawn(g, np.zeros(n, int), rng.normal(size=(n, 3)))
    Rm = rot.as_matrix()
    Sig = Rm @ np.diag(np.asarray(g.scale[0], np.float64) ** 2) @ Rm.T
    C = np.cov(rows[:, 0:3].T)
    assert np.abs(C - 2 * Sig).max() <= 0.02 * np.abs(2 * Sig).max()
    np.testing.assert_allclose(rows[:, 0:3].mean(0), g.mean[0], atol=3e-4)


def test_densify_prune_invariants():
    rng = np.random.default_rng(43)
    deg, n = 1, 200
    P = s2.cols(deg)
    rows = rng.normal(size=(n, P))
    rows[:, 3:7] /= np.linalg.norm(rows[:, 3:7], axis=1, keepdims=True)
    rows[:, 7:10] = rng.normal(-3.0, 0.3, size=(n, 3))
    rows[:, 10] = logit(0.01) + rng.normal(0, 2.0, size=n)
    acc = rng.uniform(0, 1e-3, size=n)
    den = rng.integers(0, 4, size=n)
    z = rng.normal(size=(n, 3))
    out, keep, split = s2.densify_prune(rows, acc, den, 2e-4, 0.01, 0.8, z)
    want_keep = expit(rows[:, 10]) >= 0.01
    np.testing.assert_array_equal(keep, want_keep)
    avg = np.where(den > 0, acc / np.maximum(den, 1), -1.0)
    np.testing.assert_array_equal(split, want_keep & (den > 0) & (avg > 2e-4))
    k1 = int(keep.sum())
    assert out.shape == (k1 + int(split.sum()), P)
    np.testing.assert_array_equal(out[:k1], rows[keep])
    par = rows[split]
    new = out[k1:]
    np.testing.assert_array_equal(new[:, 3:7], par[:, 3:7])
    np.testing.assert_array_equal(new[:, 11:], par[:, 11:])
    np.testing.assert_allclose(new[:, 10], logit(0.1), rtol=1e-12)
    np.testing.assert_allclose(new[:, 7:10], par[:, 7:10] + math.log(0.8), rtol=0, atol=1e-12)
    # mean = parent + R diag(s) z, R from scipy (scipy quaternions are (x, y, z, w))
    Rm = Rotation.from_quat(par[:, [4, 5, 6, 3]]).as_matrix()
    want = par[:, 0:3] + np.einsum("nij,nj->ni", Rm, np.exp(par[:, 7:10]) * z[split])
    np.testing.assert_allclose(new[:, 0:3], want, rtol=1e-12, atol=1e-12)


def test_adam_rows_equals_adam_per_column_group():
    rng = np.random.default_rng(44)
    deg, n = 2, 30
    P = s2.cols(deg)
    rows, g = rng.normal(size=(n, P)), rng.normal(size=(n, P))
    m, v = rng.normal(size=(n, P)) * 0.1, rng.uniform(size=(n, P)) * 0.1
    lr6 = [0.0024, 0.015, 0.075, 0.75, 0.0375, 0.0375 / 20]
    r1, m1, v1 = s2.adam_rows(rows, m.copy(), v.copy(), g, lr6, 3, 0.9, 0.999, 1e-15, deg)
    lr = s2.lr_columns(deg, lr6)
    for c in range(P):
        p_, mm, vv = rows[:, c].copy(), m[:, c].copy(), v[:, c].copy()
        oracle.adam(p_, g[:, c], mm, vv, 3, lr=lr[c], b1=0.9, b2=0.999, eps=1e-15)
        np.testing.assert_allclose(r1[:, c], p_, rtol=1e-13, atol=1e-15)
        np.testing.assert_allclose(m1[:, c], mm, rtol=1e-13, atol=1e-15)
        np.testing.assert_allclose(v1[:, c], vv, rtol=1e-13, atol=1e-15)


def _stage2_scene(seed):
    W, H = 48, 40
    cams = scenes.ring_cameras([0, 120], [5, -5], W, H)
    rng = np.random.default_rng(seed)
    fixed = scenes.make_gaussians(40, 1, rng)
    fixed.scale = (fixed.scale * 3).astype(np.float32)
    idx = np.arange(6)
    rows = s2.spawn(fixed, idx, rng.normal(size=(6, 3)))
    rows[:, 3:7] = rng.normal(size=(6, 4))
    rows[:, 7:10] += 0.5
    rows[:, 10] = rng.normal(0.5, 0.5, size=6)
    rows[:, 11:] += rng.normal(0, 0.3, size=rows[:, 11:].shape)
    target = oracle.render(scenes.make_gaussians(60, 1, rng), cams)["img"]
    return fixed, rows, cams, target


def test_stage2_loss_gradients_finite_differences():
    """Gradients of the Stage-2 loss wrt every trainable entry of the added
    rows (mean, rotation, log scale, opacity logit, SH) against central
    finite differences of the whole FP64 forward, on a scene with no pixel
    near a compositing threshold."""
    for seed in range(50, 80):
        fixed, rows, cams, target = _stage2_scene(seed)
        L, g, r, _ = s2.loss_grads(fixed, rows, cams, target)
        if not r["ambig"].any():
            break
    else:
        pytest.skip("no threshold-free scene")

    def f(rw):
        return s2.loss_grads(fixed, rw, cams, target)[0]

    h = 1e-6
    rng = np.random.default_rng(0)
    checked = 0
    for i in range(rows.shape[0]):
        for c in range(rows.shape[1]):
            if c >= 14 and rng.uniform() > 0.3:
                continue  # a sample of the higher SH coefficients
            rp, rm = rows.copy(), rows.copy()
            rp[i, c] += h
            rm[i, c] -= h
            fd = (f(rp) - f(rm)) / (2 * h)
            assert abs(fd - g[i, c]) <= 1e-5 * max(1e-3, abs(fd)) + 1e-9, (i, c, fd, g[i, c])
            checked += 1
    assert checked > 60
