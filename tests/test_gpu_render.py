"""The render-only path (Section 5.4's rendering of a streamed frame: NTC
query, transformation, SH rotation of Suppl. B, projection, binning and
compositing, no backward) against the FP64 oracle, eager and replayed as a
CUDA graph, and the bin-size autotuner: every bin size composites the same
records in the same order, so the chosen size renders bit-identical images."""
import numpy as np
import pytest
import torch

import oracle
from paper_2403_01444_gb300 import gs3, scenes
from paper_2403_01444_gb300.engine import NTC, Rasterizer, Renderer, autotune_bin

pytestmark = pytest.mark.gpu
DEV = "cuda"


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2403_01444_gb300 import build
    build.build()
    gs3.lib()
    oracle.build()


def _cache(rng, entries):
    """A cache that moves the Gaussians visibly: translations of a few 1e-3
    and rotations of a few degrees (table features of 0.05 spread)."""
    table = rng.normal(0.0, 0.05, size=(entries, 2)).astype(np.float32)
    table[:, 0] += 0.5
    Ws = scenes.random_mlp([32, 64, 64, 7], rng)
    Ws[2][0:3] *= 0.02
    Ws[2][3] = np.abs(Ws[2][3]) + 1.0
    Ws[2][4:7] *= 0.1
    return table, [w.astype(np.float32) for w in Ws]


@pytest.mark.parametrize("graphs", [False, True])
def test_renderer_matches_oracle(graphs):
    W, H = 112, 80
    cams = scenes.ring_cameras([15, 200], [10, -5], W, H)
    rng = np.random.default_rng(91)
    g = scenes.make_gaussians(1500, 2, rng)
    g.scale = (g.scale * 2.5).astype(np.float32)
    og = oracle.Grid()
    table, Ws = _cache(rng, og.n_entries)
    f = oracle.ntc_forward(oracle.NTCParams(og, table, Ws), g.mean, g.quat)
    # keep the Gaussians whose discrete decisions are not within FP32 reach
    # of a boundary at the transformed means and rotations
    o = oracle.project(g, cams, mean=f["mean"], quat=f["quat"])
    keep = np.all((o["radius"] == 0) | (o["margin"] > 1e-3), axis=0)
    for v in range(len(cams)):
        d = o["depth"][v]
        order = np.argsort(d)
        close = np.abs(np.diff(d[order])) < 1e-5 * d[order][1:]
        keep[order[1:][close]] = False
    idx = np.nonzero(keep)[0]
    assert idx.size > 0.9 * g.n
    g = g.subset(idx)
    mean_t, quat_t = f["mean"][idx], f["quat"][idx]
    # the oracle: transformation, SH rotated by the frame's rotation, render
    rot = g.copy()
    rot.sh = oracle.sh_rotate(g.sh.astype(np.float64), g.quat, quat_t, g.sh_deg).astype(np.float32)
    want = oracle.render(rot, cams, mean_t, quat_t)
    # the GPU render-only path (FP32 cache, so that the transformation agrees
    # to FP32 rounding), eager or as one CUDA graph
    G = gs3.Gaussians.from_numpy(g)
    ntc = NTC(table, Ws, gs3.hashgrid(), gs3.GS_MLP_FP32)
    cd = gs3.cameras_to_device(cams)
    r = Renderer(G, ntc, len(cams), W, H, 1 << 18, bin=2)
    r.raster.fit_capacity(G, cd, *_transform(r, cd))
    if graphs:
        graph = r.capture(cd)
        r.raster.img.zero_()
        graph.replay()
        img = r.raster.img
    else:
        img = r.frame(cd)
    torch.cuda.synchronize()
    r.raster.check()
    got = img.cpu().numpy()
    np.testing.assert_allclose(r.mean_t.cpu().numpy(), mean_t, atol=1e-5)
    ok = np.broadcast_to((want["ambig"] == 0)[:, None], got.shape)
    assert ok.mean() > 0.97
    assert np.abs(got - want["img"])[ok].max() <= 1e-4
    # the SH rotation matters here: without it the image differs
    plain = oracle.render(g, cams, mean_t, quat_t)["img"]
    assert np.abs(plain - want["img"]).max() > 2e-4


def _transform(r, cd):
    """The render-only path's transformed means and rotations (one frame)."""
    r.frame(cd)
    return r.mean_t.clone(), r.quat_t.clone()


def test_autotuned_bin_renders_bit_identical_images():
    sc = scenes.make_scene(2, n_gauss=20_000)
    cfg = sc.cfg
    W, H = cfg.W, cfg.H
    G = gs3.Gaussians.from_numpy(sc.prev)
    cd = gs3.cameras_to_device(sc.cams[:4])
    times, best = autotune_bin(G, cd, 4, W, H, candidates=(1, 2, 4, 8), iters=2)
    assert set(times) == {1, 2, 4, 8} and best in times
    assert all(t > 0 for t in times.values())
    out = {}
    for b in sorted({1, best, 8}):
        r = Rasterizer(G.n, 4, W, H, 1 << 20, DEV, bin=b)
        r.fit_capacity(G, cd)
        # `last` is a position in the bin's list, so only whether a pixel
        # has a contributor is common to every bin size
        out[b] = (r.img.clone(), r.T_final.clone(), r.last > 0)
    for b in out:
        for x, y in zip(out[b], out[1]):
            assert torch.equal(x, y), b
