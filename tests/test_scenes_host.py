"""The synthetic input recipe (no GPU): the five workloads' sizes, the
distributions Gaussians are drawn from, the camera rigs, and the seeded,
bounded ground-truth motion.  These inputs stand in for the paper's N3DV and
Meet Room videos, so their shapes are what the benchmark and the parity
tests rely on."""
import math

import numpy as np
import pytest

from paper_2403_01444_gb300 import scenes


def test_configs_are_the_stated_workloads():
    # (Gaussians, SH degree, cameras, W, H, views per launch, iterations per frame)
    want = {1: (4096, 1, 4, 128, 96, 4, 50),
            2: (50_000, 2, 8, 480, 360, 8, 150),
            3: (250_000, 3, 20, 1352, 1014, 4, 150),
            4: (500_000, 3, 12, 1280, 720, 4, 100),
            5: (1_000_000, 3, 16, 1920, 1080, 16, 150)}
    for k, w in want.items():
        c = scenes.CONFIGS[k]
        assert (c.n_gauss, c.sh_deg, c.n_cams, c.W, c.H, c.views_per_batch, c.iters) == w, k
    assert scenes.CONFIGS[4].emerging and not any(scenes.CONFIGS[k].emerging for k in (1, 2, 3, 5))


def test_gaussian_draws_follow_the_recipe():
    n = 40_000
    g = scenes.make_gaussians(n, 3, np.random.default_rng(5))
    assert g.mean.shape == (n, 3) and g.sh.shape == (n, 16, 3) and g.mean.dtype == np.float32
    assert np.abs(g.mean).max() <= 1.0
    log_s = np.log(g.scale.astype(np.float64))
    assert abs(log_s.mean() + 3.0) < 0.01 and abs(log_s.std() - 0.3) < 0.01
    np.testing.assert_allclose(np.linalg.norm(g.quat, axis=1), 1.0, atol=1e-6)
    assert abs(g.opacity_logit.mean()) < 0.03 and abs(g.opacity_logit.std() - 1.0) < 0.02
    colour = 0.5 + 0.28209479177387814 * g.sh[:, 0, :]   # the DC band's colour
    assert colour.min() >= 0.5 - 0.4 and colour.max() <= 0.5 + 0.4
    assert abs(g.sh[:, 1:, :].std() - 0.05) < 0.002


@pytest.mark.parametrize("k", [1, 2, 3, 4, 5])
def test_cameras_look_at_the_origin(k):
    cfg = scenes.CONFIGS[k]
    cams = scenes.cameras_for(cfg)
    assert len(cams) == cfg.n_cams
    fx = cfg.W / (2.0 * math.tan(math.radians(30.0)))   # 60 degree horizontal field of view
    for c in cams + [scenes.heldout_camera(cfg)]:
        R, t = c.viewmat[:, :3].astype(np.float64), c.viewmat[:, 3].astype(np.float64)
        np.testing.assert_allclose(R @ R.T, np.eye(3), atol=1e-6)
        pos = c.campos.astype(np.float64)
        assert abs(np.linalg.norm(pos) - 4.0) < 1e-5
        np.testing.assert_allclose(-R @ pos, t, atol=1e-5)
        assert R[2] @ (-pos / np.linalg.norm(pos)) > 1 - 1e-6        # looks at the origin
        assert (c.W, c.H) == (cfg.W, cfg.H) and abs(c.fx - fx) < 1e-3 and c.cx == cfg.W / 2
    if cfg.cam_layout == "arc20":
        az = [math.degrees(math.atan2(c.campos[0], c.campos[2])) for c in cams]
        el = [math.degrees(math.asin(c.campos[1] / 4.0)) for c in cams]
        assert min(az) == pytest.approx(-60.0, abs=1e-4) and max(az) == pytest.approx(60.0, abs=1e-4)
        assert sorted({round(e, 3) for e in el}) == [-10.0, 0.0, 10.0]


def test_motion_is_seeded_bounded_and_frame_one_of_the_video():
    a = scenes.make_scene(3, n_gauss=3000)
    b = scenes.make_scene(3, n_gauss=3000)
    for f in ("mean", "quat", "scale", "opacity_logit", "sh"):
        np.testing.assert_array_equal(getattr(a.prev, f), getattr(b.prev, f))
        np.testing.assert_array_equal(getattr(a.target, f), getattr(b.target, f))
    # rigid 1 degree about the origin (|x| <= sqrt 3) + 0.01, then a field of at most 0.02
    disp = np.linalg.norm(a.target.mean - a.prev.mean, axis=1)
    assert 0 < disp.max() <= 2 * math.sqrt(3) * math.sin(math.radians(0.5)) + 0.01 + 0.02 + 1e-6
    np.testing.assert_allclose(np.linalg.norm(a.target.quat, axis=1), 1.0, atol=1e-5)
    np.testing.assert_array_equal(a.target.scale, a.prev.scale)
    _, frames, _, _ = scenes.make_sequence(3, 2, n_gauss=3000)
    np.testing.assert_array_equal(frames[1].mean, a.target.mean)
    assert not np.array_equal(frames[2].mean, frames[1].mean)   # the motion goes on


def test_emerging_object_in_the_stage2_workload():
    s = scenes.make_scene(4, n_gauss=5000)
    added = s.target.mean.shape[0] - s.prev.mean.shape[0]
    assert 50 <= added <= 100          # 5 000 to 10 000 scaled by 5 000 / 500 000
    new = s.target.mean[-added:].astype(np.float64)
    # inside a ball of radius 0.2: no two of them further apart than its diameter
    assert np.linalg.norm(new[:, None, :] - new[None, :, :], axis=-1).max() <= 0.4 + 1e-6
