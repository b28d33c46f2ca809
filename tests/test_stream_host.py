"""Checkpoint and resume of the streaming driver, host side (no GPU).  A
checkpoint carries what the next frame needs: the carried Gaussians (means
and rotations as transformed, SH as rotated, with their scales and
opacities) and the cache's warm-up parameters.  A run resumed from it
continues at the next frame; a checkpoint of another scene is refused and
leaves the run as it was."""
import types

import numpy as np
import pytest
import torch

from paper_2403_01444_gb300 import engine, gs3, scenes

FIELDS = ("mean", "quat", "sh", "scale", "opacity_logit")


def _driver(n, deg, seed, frames_done=0):
    g = gs3.Gaussians.from_numpy(scenes.make_gaussians(n, deg, np.random.default_rng(seed)), device="cpu")
    gen = torch.Generator().manual_seed(seed)
    warm = (torch.randn(1000, generator=gen), torch.randn(gs3.MLP_PARAMS, generator=gen))
    return types.SimpleNamespace(g=g, warm=warm, frames_done=frames_done)


def test_checkpoint_round_trip(tmp_path):
    a = _driver(300, 2, 0, frames_done=7)
    path = str(tmp_path / "ck.npz")
    engine.Streamer.checkpoint(a, path)
    b = _driver(300, 2, 1)
    assert not torch.equal(b.g.mean, a.g.mean)
    engine.Streamer.resume(b, path)
    assert b.frames_done == 7
    for f in FIELDS:
        assert torch.equal(getattr(b.g, f), getattr(a.g, f)), f
    assert torch.equal(b.warm[0], a.warm[0]) and torch.equal(b.warm[1], a.warm[1])


@pytest.mark.parametrize("n,deg", [(299, 2), (300, 1)])
def test_resume_refuses_another_scene(tmp_path, n, deg):
    path = str(tmp_path / "ck.npz")
    engine.Streamer.checkpoint(_driver(300, 2, 0, frames_done=3), path)
    c = _driver(n, deg, 2)
    before = {f: getattr(c.g, f).clone() for f in FIELDS}
    with pytest.raises(ValueError, match="checkpoint of 300 Gaussians"):
        engine.Streamer.resume(c, path)
    assert c.frames_done == 0
    for f in FIELDS:
        assert torch.equal(getattr(c.g, f), before[f]), f
