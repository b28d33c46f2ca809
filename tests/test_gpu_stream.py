"""The streaming driver (Section 3): frame after frame, the transformed
Gaussians are carried forward, the cache restarts from its warm-up
parameters, and Stage 2 of a frame runs on a second stream while the next
frame's Stage 1 runs."""
import math

import numpy as np
import pytest
import torch

import oracle
from paper_2403_01444_gb300 import gs3, scenes
from paper_2403_01444_gb300.engine import NTC, Streamer, render, warmup

pytestmark = pytest.mark.gpu
DEV = "cuda"


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2403_01444_gb300 import build
    build.build()
    gs3.lib()


@pytest.mark.parametrize("graphs", [True, False])
def test_stream_carries_motion_over_frames(graphs):
    """Three frames of the 4 096-Gaussian rigid-motion video (5 degrees +
    0.05 per frame), with and without CUDA graphs: per frame the records are
    complete and Stage 1 raises the held-out PSNR above that of the
    Gaussians carried from the previous frame."""
    n_frames = 3
    cfg, frames, cams, ho = scenes.make_sequence(1, n_frames)
    W, H, Vb = cfg.W, cfg.H, cfg.views_per_batch
    G0 = gs3.Gaussians.from_numpy(frames[0])
    cd = gs3.cameras_to_device(cams)
    rng = np.random.default_rng(91)
    og = oracle.Grid()
    table = rng.uniform(-1e-4, 1e-4, size=(og.n_entries, 2)).astype(np.float32)
    Ws = [w.astype(np.float32) for w in scenes.random_mlp([32, 64, 64, 7], rng)]
    ntc = NTC(table, Ws, gs3.hashgrid(), gs3.GS_MLP_FP32)
    warmup(ntc, G0, iters=300)
    warm = (ntc.table.p.clone(), ntc.mlp.p.clone())

    def views(t):
        Gt = gs3.Gaussians.from_numpy(frames[t + 1])
        return torch.cat([render(Gt, cams[b * Vb:(b + 1) * Vb], W, H) for b in range(len(cams) // Vb)])

    hod = gs3.cameras_to_device([ho])
    ho_gt = [render(gs3.Gaussians.from_numpy(frames[t + 1]), [ho], W, H) for t in range(n_frames)]
    s = Streamer(G0, ntc, *warm, cd, len(cams), Vb, W, H, heldout_dev=hod, iters1=150, iters2=30,
                 added_capacity=20_000, graphs=graphs)
    rec = s.run(views, ho_gt)
    assert [r["frame"] for r in rec] == list(range(1, n_frames + 1))
    for r in rec:
        assert math.isfinite(r["psnr_stage1"]) and math.isfinite(r["psnr_stage2"])
        assert r["storage_bytes"] >= ntc.entries * 4
    print(rec)
    for r in rec:
        # every frame's Stage 1 improves on the Gaussians carried from the previous frame
        assert r["psnr_stage1"] > r["psnr_carried"] + 0.5, r
    # the carried Gaussians moved from frame 0
    assert float((s.g.mean - G0.mean).abs().max()) > 1e-3
