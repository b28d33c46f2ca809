"""The torch.autograd.Function wrappers: the Stage-1 loss written as a
composition (cache -> rasterizer -> L1 + D-SSIM) and differentiated with
loss.backward() gives the FP64 oracle's gradients, and a rasterizer
backward under an arbitrary upstream gradient matches the oracle's reverse
pass."""
import numpy as np
import pytest
import torch

import oracle
from paper_2403_01444_gb300 import gs3, scenes
from paper_2403_01444_gb300.autograd import (L1DSSIM, NTCContext, NTCTransform, RasterContext,
                                             Rasterize)
from paper_2403_01444_gb300.engine import Loss, Rasterizer
from test_gpu_step import _clean_scene, _near_identity_ntc, rel_err

pytestmark = pytest.mark.gpu
DEV = "cuda"


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2403_01444_gb300 import build
    build.build()
    gs3.lib()
    oracle.build()


def test_autograd_stage1_loss_matches_oracle():
    W, H = 96, 72
    cams = scenes.ring_cameras([20, 160], [5, -10], W, H)
    rng = np.random.default_rng(72)
    g = _clean_scene(73, 600, 2, cams)
    og = oracle.Grid()
    table, Ws = _near_identity_ntc(rng, og, gs3.GS_MLP_FP32)
    tgt = scenes.rbf_motion(g, rng, 8, 0.05)
    targets = oracle.render(tgt, cams)["img"]
    out = oracle.stage1_loss_grads(oracle.NTCParams(og, table, Ws), g, cams, targets)

    G = gs3.Gaussians.from_numpy(g)
    cd = gs3.cameras_to_device(cams)
    table_t = torch.from_numpy(table).to(DEV).requires_grad_()
    w_t = torch.from_numpy(np.concatenate([w.ravel() for w in Ws])).to(DEV).requires_grad_()
    c = NTCContext(gs3.hashgrid(), gs3.GS_MLP_FP32)
    rc = RasterContext(Rasterizer(G.n, len(cams), W, H, 1 << 20, DEV), G, cd)
    m, q = NTCTransform.apply(table_t, w_t, G.mean, G.quat, c)
    rc.raster.fit_capacity(G, cd, m.detach(), q.detach())
    img = Rasterize.apply(m, q, rc)
    loss = L1DSSIM.apply(img, torch.from_numpy(targets.astype(np.float32)).to(DEV),
                         Loss(len(cams), W, H, DEV))
    loss.backward()
    rc.raster.check()
    assert abs(loss.item() - out["loss"]) <= 1e-4 * out["loss"]
    assert rel_err(w_t.grad.cpu().numpy(), np.concatenate([w.ravel() for w in out["dWs"]])) <= 1e-3
    assert rel_err(table_t.grad.cpu().numpy(), out["d_table"]) <= 1e-3


def test_rasterize_backward_under_arbitrary_upstream_gradient():
    """sum(img * R) for a random R: d/d mean and d/d quat must be the oracle's
    compositing reverse with d_img = R followed by its projection reverse."""
    W, H = 80, 64
    cams = scenes.ring_cameras([0, 100, 200], [0, 10, -10], W, H)
    g = _clean_scene(77, 500, 1, cams)
    G = gs3.Gaussians.from_numpy(g)
    cd = gs3.cameras_to_device(cams)
    rc = RasterContext(Rasterizer(G.n, len(cams), W, H, 1 << 20, DEV), G, cd)
    mean = G.mean.clone().requires_grad_()
    quat = G.quat.clone().requires_grad_()
    rc.raster.fit_capacity(G, cd, mean.detach(), quat.detach())
    img = Rasterize.apply(mean, quat, rc)
    R = np.random.default_rng(78).normal(size=tuple(img.shape))
    (img * torch.from_numpy(R.astype(np.float32)).to(DEV)).sum().backward()
    r = oracle.render(g, cams)
    ok = r["ambig"] == 0
    assert ok.mean() > 0.98
    d_img = R * ok[:, None]   # the comparison needs the unambiguous pixels only
    mean2 = G.mean.clone().requires_grad_()
    quat2 = G.quat.clone().requires_grad_()
    img2 = Rasterize.apply(mean2, quat2, rc)
    (img2 * torch.from_numpy(d_img.astype(np.float32)).to(DEV)).sum().backward()
    grads = oracle.raster_bwd(r["proj"], W, H, r["T_final"], r["last"], d_img)
    dm, dq = oracle.project_bwd(g, cams, grads)
    assert rel_err(mean2.grad.cpu().numpy(), dm) <= 1e-3
    assert rel_err(quat2.grad.cpu().numpy(), dq) <= 1e-3
    # the unmasked upstream gradient flows through the same reverse pass
    assert torch.isfinite(mean.grad).all() and mean.grad.abs().sum() > 0
