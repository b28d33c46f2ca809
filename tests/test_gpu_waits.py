"""Failure detection on the GPU without a fault: the tensor-core kernels'
bounded mbarrier wait, made to run out on a barrier nothing arrives on,
returns a timeout status the host reads, and the context stays usable."""
import math
import time

import numpy as np
import pytest
import torch

from paper_2403_01444_gb300 import gs3, scenes

pytestmark = pytest.mark.gpu
DEV = "cuda"


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2403_01444_gb300 import build
    build.build()
    gs3.lib()


def test_bounded_wait_times_out_and_context_stays_usable():
    status = torch.full((1,), 12345, dtype=torch.int32, device=DEV)
    t0 = time.perf_counter()
    gs3.gs_tc_wait_selftest(4096, status)
    torch.cuda.synchronize()
    assert int(status.item()) == gs3.GS_ERR_TIMEOUT
    assert time.perf_counter() - t0 < 10.0
    # the context still runs the tensor-core MLP, with the result of the FP32 path
    rng = np.random.default_rng(5)
    n = 1000
    enc = torch.from_numpy(rng.integers(-2, 3, size=(n, 32)).astype(np.float32)).to(DEV)
    Ws = [w.astype(np.float32) for w in scenes.random_mlp([32, 64, 64, 7], rng)]
    w = np.concatenate([(np.round(x * 8) / 8).ravel() for x in Ws]).astype(np.float32)  # exact in BF16
    w32 = torch.from_numpy(w).to(DEV)
    wbf = w32.to(torch.bfloat16)
    out_tc = torch.zeros(n, 7, device=DEV)
    out_32 = torch.zeros(n, 7, device=DEV)
    gs3.ntc_mlp_fwd(enc.to(torch.bfloat16), n, gs3.mlp_struct(gs3.GS_MLP_BF16, w32, wbf), out_tc)
    gs3.ntc_mlp_fwd(enc, n, gs3.mlp_struct(gs3.GS_MLP_FP32, w32), out_32)
    torch.cuda.synchronize()
    scale = float(out_32.abs().max())
    assert float((out_tc - out_32).abs().max()) <= 1e-2 * max(scale, 1.0)


def _small_stage1(fused):
    from paper_2403_01444_gb300.engine import NTC, Rasterizer, Stage1, warmup
    scene = scenes.make_scene(2, n_gauss=3000, W=96, H=72, n_cams=4)
    cfg = scene.cfg
    G = gs3.Gaussians.from_numpy(scene.prev)
    Gt = gs3.Gaussians.from_numpy(scene.target)
    cd = gs3.cameras_to_device(scene.cams)
    rt = Rasterizer(Gt.n, 4, cfg.W, cfg.H, 1 << 18, DEV)
    rt.fit_capacity(Gt, cd)
    target = rt.img.clone()
    rng = np.random.default_rng(9)
    grid = gs3.hashgrid()
    table = scenes.random_hashgrid_table(gs3.ntc_hashgrid_entries(grid), 2, rng)
    Ws = [w.astype(np.float32) for w in scenes.random_mlp([32, 64, 64, 7], rng)]
    ntc = NTC(table, Ws, grid, gs3.GS_MLP_BF16, DEV)
    warmup(ntc, G, iters=20)
    st = Stage1(G, ntc, 4, cfg.W, cfg.H, capacity=1 << 18, fused=fused)
    st.raster.fit_capacity(G, cd, *st.transform())
    return st, ntc, cd, target


@pytest.mark.parametrize("fused", [False, True])
def test_mlp_timeout_skips_the_step(fused):
    """With the tensor-core wait limit at 0 every MMA wait of the cache's
    kernels gives up: each block waits for its batch in flight, releases its
    tensor memory and marks its unfinished rows (forward) and the weight
    gradient (reverse) non-finite.  The projection culls and reports the NaN
    Gaussians, the non-finite check skips the Adam update and halves the loss
    scale, and the parameters do not move.  With the default limit restored
    the next step trains as usual."""
    st, ntc, cd, target = _small_stage1(fused)
    st.step(cd, target)
    torch.cuda.synchronize()
    st.raster.check()
    s0 = gs3.read_train_state(st.state)
    p_table, p_mlp = ntc.table.p.clone(), ntc.mlp.p.clone()
    t0 = gs3.gs_tc_timeouts()
    gs3.gs_tc_set_wait_limit(0)
    try:
        st.step(cd, target)
        torch.cuda.synchronize()
    finally:
        gs3.gs_tc_set_wait_limit(gs3.GS_TC_WAIT_TRIES_DEFAULT)
    assert gs3.gs_tc_timeouts() > t0
    assert int(st.raster.d_err.item()) == gs3.GS_ERR_NONFINITE
    assert torch.isnan(st.mean_t).any()
    s1 = gs3.read_train_state(st.state)
    assert s1.step == s0.step and s1.found_inf == 0
    assert s1.loss_scale == s0.loss_scale * 0.5
    assert torch.equal(ntc.table.p, p_table) and torch.equal(ntc.mlp.p, p_mlp)
    # the context is usable and the next step trains
    st.raster.d_err.zero_()
    t1 = gs3.gs_tc_timeouts()
    d_loss = st.step(cd, target)
    torch.cuda.synchronize()
    st.raster.check()
    assert gs3.gs_tc_timeouts() == t1
    assert math.isfinite(float(d_loss.item()))
    assert gs3.read_train_state(st.state).step == s0.step + 1
    assert not torch.equal(ntc.mlp.p, p_mlp)
    assert not torch.isnan(st.mean_t).any()
