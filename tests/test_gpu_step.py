"""End-to-end parity of the CUDA Stage-1 step with the FP64 oracle, the
closed-form checks on the GPU path, and training behaviour (the trained cache
against the method without it)."""
import math

import numpy as np
import pytest
import torch

import oracle
from paper_2403_01444_gb300 import gs3, scenes
from paper_2403_01444_gb300.engine import NTC, DirectOpt, Rasterizer, Stage1, render, warmup

pytestmark = pytest.mark.gpu
DEV = "cuda"


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2403_01444_gb300 import build
    build.build()
    gs3.lib()


def rel_err(a, b):
    a, b = np.asarray(a, np.float64), np.asarray(b, np.float64)
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-30))


def _clean_scene(seed, N, deg, cams):
    """Gaussians whose discrete decisions (radius, tile rectangle, depth
    order) are not within FP32 reach of a boundary in any view."""
    rng = np.random.default_rng(seed)
    g = scenes.make_gaussians(N, deg, rng)
    g.scale = (g.scale * 2.5).astype(np.float32)
    o = oracle.project(g, cams)
    keep = np.all((o["radius"] == 0) | (o["margin"] > 1e-3), axis=0)
    for v in range(len(cams)):
        d = o["depth"][v]
        order = np.argsort(d)
        close = np.abs(np.diff(d[order])) < 1e-5 * d[order][1:]
        keep[order[1:][close]] = False
    return g.subset(np.nonzero(keep)[0])


def test_render_parity_end_to_end():
    W, H = 150, 110
    cams = scenes.ring_cameras([0, 130], [10, -5], W, H)
    g = _clean_scene(70, 3000, 3, cams)
    r = oracle.render(g, cams)
    G = gs3.Gaussians.from_numpy(g)
    img = render(G, cams, W, H).cpu().numpy()
    ok = np.broadcast_to((r["ambig"] == 0)[:, None], img.shape)
    assert ok.mean() > 0.98
    assert np.abs(img - r["img"])[ok].max() <= 1e-4


def test_single_gaussian_closed_form_on_gpu():
    W, H = 96, 72
    cam = scenes.look_at_camera((0.0, 0.0, 4.0), W, H)
    c = np.array([0.7, 0.2, 0.45])
    C0 = 0.5 / math.sqrt(math.pi)
    sig = float(np.float32(0.3))
    g = scenes.GaussianSet(np.zeros((1, 3), np.float32), np.array([[1, 0, 0, 0]], np.float32),
                           np.full((1, 3), sig, np.float32), np.array([0.4], np.float32),
                           ((c - 0.5) / C0).reshape(1, 1, 3).astype(np.float32), 0)
    img = render(gs3.Gaussians.from_numpy(g), [cam], W, H).cpu().numpy()[0]
    var = (cam.fx * sig / 4.0) ** 2 + 0.3
    o = 1 / (1 + math.exp(-float(np.float32(0.4))))
    yy, xx = np.mgrid[0:H, 0:W]
    a = np.minimum(0.99, o * np.exp(-0.5 * ((xx + 0.5 - W / 2) ** 2 + (yy + 0.5 - H / 2) ** 2) / var))
    rad = math.ceil(3 * math.sqrt(var + math.sqrt(0.1)))
    inrect = ((xx // 16 >= math.floor((W / 2 - rad) / 16)) & (xx // 16 < math.floor((W / 2 + rad + 15) / 16)) &
              (yy // 16 >= math.floor((H / 2 - rad) / 16)) & (yy // 16 < math.floor((H / 2 + rad + 15) / 16)))
    want = np.where((a >= 1 / 255) & inrect, a, 0.0)[None] * c[:, None, None]
    near = np.abs(a - 1 / 255) < 1e-5
    assert np.abs(img - want)[:, ~near].max() <= 1e-5


def test_identity_transform_reproduces_render():
    W, H = 128, 96
    cams = scenes.ring_cameras([0, 90, 180, 270], [0] * 4, W, H)
    g = scenes.make_gaussians(4096, 1, np.random.default_rng(71))
    G = gs3.Gaussians.from_numpy(g)
    n = g.n
    raw = torch.zeros(n, 7, device=DEV)
    raw[:, 3] = 1.0
    mo, qo = torch.zeros(n, 3, device=DEV), torch.zeros(n, 4, device=DEV)
    gs3.ntc_apply(G.mean, G.quat, raw, n, [-1.5] * 3 + [1.5] * 3, 0, mo, qo)
    a = render(G, cams, W, H)
    b = render(G, cams, W, H, mo, qo)
    assert (a - b).abs().max().item() <= 1e-6
    norms = qo.norm(dim=1)
    assert (norms - 1).abs().max().item() <= 1e-6


def _near_identity_ntc(rng, grid_np, precision):
    table = rng.normal(0.0, 0.05, size=(grid_np.n_entries, 2)).astype(np.float32)
    table[:, 0] += 0.5
    Ws = scenes.random_mlp([32, 64, 64, 7], rng)
    Ws[2][0:3] *= 0.01
    Ws[2][3] = np.abs(Ws[2][3]) + 1.0
    Ws[2][4:7] *= 0.1
    return table, [w.astype(np.float32) for w in Ws]


def test_stage1_gradients_match_oracle_fp32():
    W, H = 96, 72
    cams = scenes.ring_cameras([20, 160], [5, -10], W, H)
    rng = np.random.default_rng(72)
    g = _clean_scene(73, 600, 2, cams)
    og = oracle.Grid()
    table, Ws = _near_identity_ntc(rng, og, gs3.GS_MLP_FP32)
    tgt = rbf = scenes.rbf_motion(g, rng, 8, 0.05)
    targets = oracle.render(tgt, cams)["img"]
    p = oracle.NTCParams(og, table, Ws)
    out = oracle.stage1_loss_grads(p, g, cams, targets)
    # the FP32 GPU step on the same FP32 parameters and targets
    G = gs3.Gaussians.from_numpy(g)
    ntc = NTC(table, Ws, gs3.hashgrid(), gs3.GS_MLP_FP32)
    st = Stage1(G, ntc, 2, W, H, capacity=1 << 20)
    cd = gs3.cameras_to_device(cams)
    tg = torch.from_numpy(targets.astype(np.float32)).to(DEV)
    st.raster.fit_capacity(G, cd, *st.transform())
    d_loss = st.compute_grads(cd, tg)
    torch.cuda.synchronize()
    assert abs(d_loss.item() - out["loss"]) <= 1e-4 * out["loss"]
    ambig = out["render"]["ambig"].sum()
    assert ambig <= 0.002 * out["render"]["ambig"].size
    assert rel_err(st.raw7.cpu().numpy(), out["fwd"]["raw7"]) <= 1e-5
    assert rel_err(ntc.mlp.g.cpu().numpy(), np.concatenate([w.ravel() for w in out["dWs"]])) <= 1e-3
    assert rel_err(ntc.table.g.cpu().numpy(), out["d_table"]) <= 1e-3


@pytest.mark.parametrize("precision", [gs3.GS_MLP_FP32])
def test_ntc_training_beats_no_ntc(precision):
    """What the trained cache gains: after 150 Stage-1 iterations on a
    rigid-motion scene, the transformed Gaussians render a held-out view closer
    to the ground truth than the untransformed previous frame, and the means
    the training views see moved towards the true motion (error weighted by
    visibility)."""
    cfg = scenes.CONFIGS[1]
    sc = scenes.make_scene(1)
    W, H = cfg.W, cfg.H
    G = gs3.Gaussians.from_numpy(sc.prev)
    cams = sc.cams
    cd = gs3.cameras_to_device(cams)
    Gt = gs3.Gaussians.from_numpy(sc.target)
    targets = render(Gt, cams, W, H)
    rng = np.random.default_rng(74)
    og = oracle.Grid()
    table = rng.uniform(-1e-4, 1e-4, size=(og.n_entries, 2)).astype(np.float32)
    Ws = [w.astype(np.float32) for w in scenes.random_mlp([32, 64, 64, 7], rng)]
    ntc = NTC(table, Ws, gs3.hashgrid(), precision)
    wl = warmup(ntc, G, iters=300)
    assert wl < -0.9  # near the identity transformation (loss minimum is -1)
    st = Stage1(G, ntc, len(cams), W, H, capacity=1 << 20)
    st.raster.fit_capacity(G, cd, *st.transform(), margin=2.0)
    # each Gaussian's visibility in the training views (sum of alpha T): the
    # motion of a Gaussian no view sees is not observable
    r = Rasterizer(G.n, len(cams), W, H, 1 << 20, DEV)
    r.fit_capacity(G, cd)
    r.backward(G, cd, torch.ones_like(r.img))
    w = r.grads[..., 5].sum(0)
    losses = []
    for it in range(150):
        losses.append(st.step(cd, targets).item())
    st.raster.check()
    mt, qt = st.transform()
    err = lambda m: float(((m - Gt.mean).norm(dim=1) * w).sum() / w.sum())
    err_after, err_before = err(mt), err(G.mean)
    print("weighted motion error %.5f -> %.5f" % (err_before, err_after))
    # the loss falls to about 0.70 of its start here; the exact ratio varies
    # from run to run with the order of the FP32 gradient atomics
    assert losses[-1] < 0.8 * losses[0]
    # this scene moves 5 degrees + 0.05 per frame, five times the video
    # workload's motion that the Stage-1 rate schedule is set for; the error
    # falls by about 16 % within the frame (35 % with a 10 % final rate)
    assert err_after < 0.9 * err_before
    ho = [sc.heldout]
    gt = render(Gt, ho, W, H)
    psnr = lambda a: -10 * math.log10(((a - gt) ** 2).mean().item())
    p_ntc = psnr(render(G, ho, W, H, mt, qt))
    p_none = psnr(render(G, ho, W, H))
    assert p_ntc > p_none + 1.0, (p_ntc, p_none)


def test_stage1_recovers_motion_at_reduced_multiview_size():
    """The headline workload at reduced size (60 000 Gaussians, the 20-camera
    frontal arc at 676x507, 4 views per launch, rigid + RBF motion): over one
    frame of 150 mixed-precision Stage-1 iterations with the engine's Adam
    schedule, the motion error of the Gaussians the training views see
    (|mu' - mu_gt| weighted by their visibility, sum of alpha T) falls at every
    checkpoint, the rotation error stays bounded, and the held-out view ends
    above the untransformed previous frame."""
    sc = scenes.make_scene(3, n_gauss=60_000, W=676, H=507)
    cfg = sc.cfg
    W, H, Vb = cfg.W, cfg.H, cfg.views_per_batch
    nb = cfg.n_cams // Vb
    G = gs3.Gaussians.from_numpy(sc.prev)
    Gt = gs3.Gaussians.from_numpy(sc.target)
    cd = gs3.cameras_to_device(sc.cams)
    bc = [gs3.camera_slice(cd, b * Vb, Vb) for b in range(nb)]
    r = Rasterizer(G.n, Vb, W, H, 1 << 22, DEV)
    targets, w = [], torch.zeros(G.n, device=DEV)
    for b in range(nb):
        r.fit_capacity(Gt, bc[b], margin=1.2)
        targets.append(r.img.clone())
        r.fit_capacity(G, bc[b], margin=1.2)
        r.backward(G, bc[b], torch.ones_like(r.img))
        w += r.grads[..., 5].sum(0)
    rng = np.random.default_rng(75)
    grid = gs3.hashgrid()
    table = scenes.random_hashgrid_table(gs3.ntc_hashgrid_entries(grid), 2, rng)
    Ws = [x.astype(np.float32) for x in scenes.random_mlp([32, 64, 64, 7], rng)]
    ntc = NTC(table, Ws, grid, gs3.GS_MLP_BF16)
    warmup(ntc, G, iters=500)
    st = Stage1(G, ntc, Vb, W, H, capacity=1 << 20)
    st.raster.fit_capacity(G, bc[0], *st.transform(), margin=2.0)
    st.reset_state()

    def errs():
        m, q = st.transform()
        dm = (m - Gt.mean).norm(dim=1)
        qn = q / q.norm(dim=1, keepdim=True)
        ang = 2 * torch.acos((qn * Gt.quat).sum(1).abs().clamp(max=1.0)) * (180 / math.pi)
        return float((dm * w).sum() / w.sum()), float((ang * w).sum() / w.sum())

    curve = [errs()]
    for it in range(150):
        st.step(bc[it % nb], targets[it % nb])
        if (it + 1) % 25 == 0:
            curve.append(errs())
    st.raster.check()
    print("motion error (weighted mean, angle) every 25 iterations:", curve)
    e = [c[0] for c in curve]
    assert all(b < a for a, b in zip(e, e[1:])), e
    assert e[-1] < 0.7 * e[0], e
    assert max(c[1] for c in curve) < 15.0
    mt, qt = st.transform()
    ho = [sc.heldout]
    gt = render(Gt, ho, W, H)
    psnr = lambda a: -10 * math.log10(((a - gt) ** 2).mean().item())
    assert psnr(render(G, ho, W, H, mt, qt)) > psnr(render(G, ho, W, H)) + 0.5


def test_graph_replay_matches_eager_steps():
    """The iteration captured in CUDA graphs (one per view batch) computes what
    the eager calls compute."""
    sc = scenes.make_scene(2, n_gauss=20_000, W=240, H=180)
    W, H, Vb = 240, 180, 4
    G = gs3.Gaussians.from_numpy(sc.prev)
    Gt = gs3.Gaussians.from_numpy(sc.target)
    cd = gs3.cameras_to_device(sc.cams)
    bc = [gs3.camera_slice(cd, 0, Vb), gs3.camera_slice(cd, Vb, Vb)]
    tg = torch.cat([render(Gt, sc.cams[:Vb], W, H), render(Gt, sc.cams[Vb:2 * Vb], W, H)])
    rng = np.random.default_rng(75)
    og = oracle.Grid()
    table, Ws = _near_identity_ntc(rng, og, gs3.GS_MLP_BF16)
    results = []
    for use_graph in (False, True):
        ntc = NTC(table, Ws, gs3.hashgrid(), gs3.GS_MLP_BF16)
        st = Stage1(G, ntc, Vb, W, H, capacity=1 << 20)
        batches = [(bc[0], tg[:Vb]), (bc[1], tg[Vb:])]
        graphs = st.capture(batches) if use_graph else None
        ntc.reset_to(ntc.init_table, ntc.init_mlp)
        st.reset_state()
        losses = []
        for i in range(6):
            if use_graph:
                graphs[i % 2].replay()
            else:
                st.step(*batches[i % 2])
            losses.append(st.loss.d_loss.item())
        st.raster.check()
        results.append((losses, ntc.mlp.p.clone(), ntc.table.p.clone()))
    (l0, w0, t0), (l1, w1, t1) = results
    np.testing.assert_allclose(l1, l0, rtol=1e-4)
    assert rel_err(w1.cpu().numpy(), w0.cpu().numpy()) < 1e-4
    assert rel_err(t1.cpu().numpy(), t0.cpu().numpy()) < 1e-4


def test_direct_optimisation_plain_fp32():
    """The plain method of the 4 096-Gaussian rigid-motion frame: 50 Adam
    iterations of direct optimisation of the means and rotations through the
    same rasterizer lower the training loss by 30 % and raise the held-out
    view above the untransformed previous frame."""
    sc = scenes.make_scene(1)
    W, H = sc.cfg.W, sc.cfg.H
    G = gs3.Gaussians.from_numpy(sc.prev)
    Gt = gs3.Gaussians.from_numpy(sc.target)
    cd = gs3.cameras_to_device(sc.cams)
    targets = render(Gt, sc.cams, W, H)
    gt_ho = render(Gt, [sc.heldout], W, H)
    psnr = lambda img: -10 * math.log10(((img - gt_ho) ** 2).mean().item())
    do = DirectOpt(G, len(sc.cams), W, H, capacity=1 << 20)
    do.raster.fit_capacity(G, cd, margin=2.0)
    losses = [do.step(cd, targets).item() for _ in range(50)]
    do.raster.check()
    assert losses[-1] < 0.7 * losses[0]
    p_direct = psnr(render(G, [sc.heldout], W, H, do.mean.p, do.quat.p))
    p_prev = psnr(render(G, [sc.heldout], W, H))
    print("held-out PSNR: previous frame %.2f dB, direct optimisation %.2f dB" % (p_prev, p_direct))
    assert p_direct > p_prev


def test_mixed_precision_training_tracks_fp32_training():
    """The 50K-Gaussian, 8-view RBF-motion frame trained for 150 iterations
    from the same cache initialisation with the FP32 cache (SIMT MLP, FP32
    table) and with the mixed-precision one (FP16 table, BF16 tensor-core
    MLP, loss scaling): both train, their final losses agree within 10 % and
    the PSNRs of the training views within 1 dB (the loss bound carried over:
    10 % on the L1-dominated loss is about 20 % on the mean squared error,
    10 log10 1.2 = 0.8 dB).  The held-out view is not
    constrained by the eight training views, so where two trajectories settle
    there is not bounded by the arithmetic (1.5 dB apart in one run whose
    training losses agreed to 0.5 %): both only have to exceed 35 dB there."""
    sc = scenes.make_scene(2)
    W, H = sc.cfg.W, sc.cfg.H
    G = gs3.Gaussians.from_numpy(sc.prev)
    Gt = gs3.Gaussians.from_numpy(sc.target)
    cd = gs3.cameras_to_device(sc.cams)
    targets = render(Gt, sc.cams, W, H)
    rng = np.random.default_rng(76)
    og = oracle.Grid()
    table = rng.uniform(-1e-4, 1e-4, size=(og.n_entries, 2)).astype(np.float32)
    Ws = [w.astype(np.float32) for w in scenes.random_mlp([32, 64, 64, 7], rng)]
    gt_ho = render(Gt, [sc.heldout], W, H)
    out = {}
    for prec in (gs3.GS_MLP_FP32, gs3.GS_MLP_BF16):
        ntc = NTC(table, Ws, gs3.hashgrid(), prec)
        warmup(ntc, G, iters=300)
        st = Stage1(G, ntc, len(sc.cams), W, H, capacity=1 << 20)
        st.raster.fit_capacity(G, cd, *st.transform(), margin=2.0)
        losses = [st.step(cd, targets).item() for _ in range(150)]
        st.raster.check()
        mt, qt = st.transform()
        img = render(G, [sc.heldout], W, H, mt, qt)
        tr = render(G, sc.cams, W, H, mt, qt)
        out[prec] = (losses, -10 * math.log10(((img - gt_ho) ** 2).mean().item()),
                     -10 * math.log10(((tr - targets) ** 2).mean().item()))
    (l32, p32, t32), (l16, p16, t16) = out[gs3.GS_MLP_FP32], out[gs3.GS_MLP_BF16]
    print("final loss fp32 %.5f bf16 %.5f; training-view PSNR fp32 %.2f bf16 %.2f; "
          "held-out PSNR fp32 %.2f bf16 %.2f" % (l32[-1], l16[-1], t32, t16, p32, p16))
    assert l16[-1] < 0.8 * l16[0] and l32[-1] < 0.8 * l32[0]
    assert abs(l16[-1] - l32[-1]) <= 0.10 * l32[-1]
    assert abs(t16 - t32) <= 1.0
    assert p16 > 35.0 and p32 > 35.0


def test_target_feeder_orders_copies_and_steps():
    """Batches fed one step ahead from pinned host memory arrive whole before
    the step that reads them: every step, from the first (device buffers
    start as NaN), sees exactly its batch (sums taken on the compute stream,
    with matrix products in between keeping it busy)."""
    from paper_2403_01444_gb300.engine import TargetFeeder
    rng = np.random.default_rng(90)
    nb, shape = 3, (2, 3, 64, 80)
    host = [torch.from_numpy(rng.uniform(size=shape).astype(np.float32)).pin_memory() for _ in range(nb)]
    dev = [torch.full(shape, float("nan"), device=DEV) for _ in range(nb)]   # unread until copied
    feeder = TargetFeeder(host, dev)
    want = [float(h.double().sum()) for h in host]
    got = []
    feeder.start(0)
    big = torch.rand(2048, 2048, device=DEV)
    for i in range(12):
        b = i % nb
        feeder.before(b)
        for _ in range(3):
            big = big @ big / 2048.0          # keeps the compute stream busy
        got.append(dev[b].double().sum())
        feeder.after(b, (i + 1) % nb)
    torch.cuda.synchronize()
    for i, g in enumerate(got):
        assert abs(float(g) - want[i % nb]) <= 1e-9 * abs(want[i % nb])
    assert feeder.bytes_per_step == 2 * 3 * 64 * 80 * 4
