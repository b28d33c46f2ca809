"""Stage 2 (Section 4.2, adaptive 3DG addition) on the GPU against the FP64
oracle: the full projection reverse, the view-space gradient statistics,
selection, spawning, split-and-prune, the Adam update of the added rows, the
whole Stage-2 gradient, and what Stage 2 gains on a scene with an emerging
object over Stage 1 alone and over spawning at random places."""
import math

import numpy as np
import pytest
import torch
from scipy.special import expit

import oracle
from oracle import stage2 as s2
from paper_2403_01444_gb300 import gs3, scenes
from paper_2403_01444_gb300.engine import NTC, Stage1, Stage2, render, warmup
from test_gpu_step import _clean_scene, rel_err

pytestmark = pytest.mark.gpu
DEV = "cuda"


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2403_01444_gb300 import build
    build.build()
    gs3.lib()
    oracle.build()


def _t(a, dt=torch.float32):
    return torch.from_numpy(np.ascontiguousarray(a)).to(DEV, dt)


def test_project_bwd_full_matches_oracle():
    W, H = 80, 64
    cams = scenes.ring_cameras([0, 110, 230], [5, -5, 10], W, H)
    g = _clean_scene(81, 400, 2, cams)
    r = oracle.render(g, cams)
    ok = r["ambig"] == 0
    d_img = np.random.default_rng(82).normal(size=r["img"].shape) * ok[:, None]
    grads, dop = oracle.raster_bwd(r["proj"], W, H, r["T_final"], r["last"], d_img, want_opacity=True)
    want = oracle.project_bwd_full(g, cams, grads, dop)
    G = gs3.Gaussians.from_numpy(g)
    cd = gs3.cameras_to_device(cams)
    first, count = 17, g.n - 40
    K = (g.sh_deg + 1) ** 2
    out = dict(d_mean=torch.zeros(count, 3, device=DEV), d_quat=torch.zeros(count, 4, device=DEV),
               d_scale=torch.zeros(count, 3, device=DEV), d_ologit=torch.zeros(count, device=DEV),
               d_sh=torch.zeros(count, K, 3, device=DEV))
    gs3.gs_project_bwd_full(G, cd, len(cams), W, H, _t(grads), _t(dop), first, count, out["d_mean"],
                            out["d_quat"], out["d_scale"], out["d_ologit"], out["d_sh"])
    torch.cuda.synchronize()
    for k, v in out.items():
        assert rel_err(v.cpu().numpy(), want[k][first:first + count]) <= 1e-4, k


def test_viewspace_statistics_and_selection():
    rng = np.random.default_rng(83)
    V, n, W, H = 3, 5000, 640, 360
    grads = rng.normal(0, 1e-6, size=(V, n, 8)).astype(np.float32)
    radius = (rng.uniform(size=(V, n)) < 0.7) * rng.integers(1, 30, size=(V, n))
    first, count = 100, 4000
    acc = torch.zeros(count, device=DEV)
    den = torch.zeros(count, dtype=torch.int32, device=DEV)
    for _ in range(2):   # accumulates
        gs3.gs_viewspace_grad_accum(_t(grads), _t(radius, torch.int32), V, n, first, count, W, H,
                                    4.0, acc, den)
    a_ref, d_ref = s2.viewspace_grad(grads, radius, W, H, 4.0)
    a_ref, d_ref = 2 * a_ref[first:first + count], 2 * d_ref[first:first + count]
    assert np.array_equal(den.cpu().numpy(), d_ref)
    np.testing.assert_allclose(acc.cpu().numpy(), a_ref, rtol=1e-5, atol=1e-12)
    # selection: bit-exact index list away from the threshold
    tau = float(np.median(a_ref[d_ref > 0] / d_ref[d_ref > 0]))
    avg = np.where(d_ref > 0, a_ref / np.maximum(d_ref, 1), -1)
    acc_np = acc.cpu().numpy().astype(np.float64)
    clear = np.abs(avg - tau) > 1e-4 * tau
    idx = torch.zeros(count, dtype=torch.int32, device=DEV)
    nsel = torch.zeros(1, dtype=torch.int64, device=DEV)
    # rows near the threshold get a zero count so both sides exclude them
    den_c = _t(np.where(clear, d_ref, 0), torch.int32)
    gs3.gs_select_above(acc, den_c, count, tau, idx, nsel)
    want = s2.select_above(acc_np, np.where(clear, d_ref, 0), tau)
    k = int(nsel.item())
    assert k == len(want) > 100
    assert np.array_equal(idx[:k].cpu().numpy(), want)


def _added_buffers(cap, deg):
    P = gs3.added_cols(deg)
    z = lambda: torch.zeros(cap, P, device=DEV)
    rows, m, v = z(), z(), z()
    return rows, m, v, gs3.added_struct(rows, m, v, deg)


def test_spawn_matches_oracle():
    rng = np.random.default_rng(84)
    g = scenes.make_gaussians(3000, 2, rng)
    G = gs3.Gaussians.from_numpy(g)
    idx = np.sort(rng.choice(g.n, 700, replace=False)).astype(np.int32)
    z = rng.normal(size=(700, 3)).astype(np.float32)
    rows, m, v, a = _added_buffers(1000, 2)
    m.fill_(7.0)
    nadd = torch.tensor([200], dtype=torch.int64, device=DEV)   # appended after 200 rows
    err = torch.zeros(1, dtype=torch.int32, device=DEV)
    gs3.gs_added_spawn(G, _t(idx, torch.int32), torch.tensor([700], dtype=torch.int64, device=DEV),
                       _t(z), 0.1, a, nadd, err)
    torch.cuda.synchronize()
    assert int(nadd.item()) == 900 and int(err.item()) == 0
    want = s2.spawn(g, idx, z.astype(np.float64))
    got = rows[200:900].cpu().numpy()
    np.testing.assert_allclose(got, want, rtol=2e-6, atol=2e-6)
    assert float(m[200:900].abs().max()) == 0.0 and float(m[:200].min()) == 7.0
    # capacity: 400 more into 100 free rows -> 100 written, error flagged
    gs3.gs_added_spawn(G, _t(idx, torch.int32), torch.tensor([400], dtype=torch.int64, device=DEV),
                       _t(z), 0.1, a, nadd, err)
    torch.cuda.synchronize()
    assert int(nadd.item()) == 1000 and int(err.item()) == gs3.GS_ERR_CAPACITY


def test_densify_prune_matches_oracle():
    rng = np.random.default_rng(85)
    deg, n = 1, 3000
    P = gs3.added_cols(deg)
    rows = rng.normal(size=(n, P)).astype(np.float32)
    rows[:, 3:7] /= np.linalg.norm(rows[:, 3:7], axis=1, keepdims=True)
    rows[:, 7:10] = rng.normal(-3.0, 0.3, size=(n, 3))
    rows[:, 10] = np.log(0.01 / 0.99) + rng.normal(0, 2.0, size=n)
    op = expit(rows[:, 10].astype(np.float64))
    rows[np.abs(op - 0.01) < 1e-5, 10] += 0.5          # away from the opacity threshold
    acc = rng.uniform(0, 1e-3, size=n).astype(np.float32)
    den = rng.integers(0, 4, size=n).astype(np.int32)
    avg = np.where(den > 0, acc / np.maximum(den, 1), -1)
    den[np.abs(avg - 2e-4) < 1e-8] = 0                  # away from the gradient threshold
    z = rng.normal(size=(n, 3)).astype(np.float32)
    src_rows, sm, sv, src = _added_buffers(n, deg)
    src_rows.copy_(_t(rows))
    sm.copy_(_t(rows * 0.5))
    sv.copy_(_t(rows * 0.25))
    dst_rows, dm, dv, dst = _added_buffers(2 * n, deg)
    nd = torch.zeros(1, dtype=torch.int64, device=DEV)
    err = torch.zeros(1, dtype=torch.int32, device=DEV)
    gs3.gs_added_densify_prune(src, n, _t(acc), _t(den, torch.int32), 2e-4, 0.01, 0.8, 0.1, _t(z),
                               dst, nd, err)
    torch.cuda.synchronize()
    want, keep, split = s2.densify_prune(rows.astype(np.float64), acc.astype(np.float64), den,
                                         2e-4, 0.01, 0.8, z.astype(np.float64))
    k = int(nd.item())
    assert k == want.shape[0] and int(err.item()) == 0
    got = dst_rows[:k].cpu().numpy()
    k1 = int(keep.sum())
    assert np.array_equal(got[:k1], rows[keep])                        # copies: bit-exact
    np.testing.assert_allclose(got[k1:], want[k1:], rtol=2e-6, atol=2e-6)
    assert np.array_equal(dm[:k1].cpu().numpy(), (rows * 0.5)[keep])   # moments travel
    assert float(dm[k1:k].abs().max()) == 0.0


def test_added_adam_and_render_match_oracle():
    rng = np.random.default_rng(86)
    deg, n = 2, 500
    P = gs3.added_cols(deg)
    K = (deg + 1) ** 2
    rows = rng.normal(size=(n, P)).astype(np.float32)
    rows[:, 7:10] = rng.normal(-3, 0.3, size=(n, 3))
    rows_t, m_t, v_t, a = _added_buffers(n, deg)
    rows_t.copy_(_t(rows))
    grads = {"d_mean": rng.normal(size=(n, 3)), "d_quat": rng.normal(size=(n, 4)),
             "d_scale": rng.normal(size=(n, 3)), "d_ologit": rng.normal(size=n),
             "d_sh": rng.normal(size=(n, K, 3))}
    grads = {k: v.astype(np.float32) for k, v in grads.items()}
    nfix = 37
    out = gs3.Gaussians(torch.zeros(nfix + n, 3, device=DEV), torch.zeros(nfix + n, 4, device=DEV),
                        torch.zeros(nfix + n, 3, device=DEV), torch.zeros(nfix + n, device=DEV),
                        torch.zeros(nfix + n, K, 3, device=DEV), deg)
    state = gs3.new_train_state(1.0, DEV)
    lr = [0.0024, 0.015, 0.075, 0.75, 0.0375, 0.0375 / 20]
    # both sides take the hyper-parameters as the FP32 values the kernel gets
    f32 = lambda x: float(np.float32(x))
    lr64 = [f32(x) for x in lr]
    b1, b2, eps = f32(0.9), f32(0.999), f32(1e-15)
    m = np.zeros((n, P))
    v = np.zeros((n, P))
    want = rows.astype(np.float64)
    for step in (1, 2):
        gs3.gs_added_adam(a, n, _t(grads["d_mean"]), _t(grads["d_quat"]), _t(grads["d_scale"]),
                          _t(grads["d_ologit"]), _t(grads["d_sh"]), lr, 0.9, 0.999, 1e-15, state,
                          out, nfix)
        gs3.gs_train_state_advance(state, 0)
        g64 = {k: v.astype(np.float64) for k, v in grads.items()}
        gr = s2.grads_to_rows(g64, want)
        want, m, v = s2.adam_rows(want, m, v, gr, lr64, step, b1, b2, eps, deg)
    torch.cuda.synchronize()
    np.testing.assert_allclose(rows_t.cpu().numpy(), want, rtol=1e-5, atol=1e-6)
    ga = s2.rows_to_gaussians(rows_t.cpu().numpy().astype(np.float64), deg)
    np.testing.assert_allclose(out.mean[nfix:].cpu().numpy(), ga.mean, rtol=1e-7, atol=0)
    np.testing.assert_allclose(out.scale[nfix:].cpu().numpy(), ga.scale, rtol=1e-6)
    np.testing.assert_allclose(out.sh[nfix:].cpu().numpy(), ga.sh, rtol=0, atol=0)
    assert float(out.mean[:nfix].abs().max()) == 0.0


def test_stage2_gradients_match_oracle():
    """One Stage-2 forward + backward through the engine (fixed Gaussians +
    added rows rendered together) against the oracle's loss and row
    gradients."""
    W, H = 96, 72
    cams = scenes.ring_cameras([15, 150], [5, -8], W, H)
    fixed = _clean_scene(87, 500, 1, cams)
    rng = np.random.default_rng(88)
    idx = rng.choice(fixed.n, 60, replace=False)
    rows = s2.spawn(fixed, np.sort(idx), rng.normal(size=(60, 3)))
    rows[:, 10] = rng.normal(0.0, 0.5, size=60)
    rows = rows.astype(np.float32)
    targets = oracle.render(scenes.rbf_motion(fixed, rng, 8, 0.05), cams)["img"]
    L, g_want, r, _ = s2.loss_grads(fixed, rows.astype(np.float64), cams, targets)
    assert r["ambig"].mean() < 0.01
    G = gs3.Gaussians.from_numpy(fixed)
    st = Stage2(G, len(cams), W, H, capacity=128, pair_capacity=1 << 20)
    a = st.all
    n = fixed.n
    a.mean[:n].copy_(G.mean)
    a.quat[:n].copy_(G.quat)
    a.scale[:n].copy_(G.scale)
    a.opacity_logit[:n].copy_(G.opacity_logit)
    a.sh[:n].copy_(G.sh)
    st.rows[0][:60].copy_(_t(rows))
    st.n_add = 60
    st._after_resize()
    cd = gs3.cameras_to_device(cams)
    st.fit_capacity(cd)
    d_loss = st.compute_grads(cd, _t(targets))
    torch.cuda.synchronize()
    assert abs(d_loss.item() - L) <= 1e-4 * L
    got = {"d_mean": st.d_mean[:60], "d_quat": st.d_quat[:60], "d_scale": st.d_scale[:60],
           "d_ologit": st.d_ologit[:60], "d_sh": st.d_sh[:60]}
    got = s2.grads_to_rows({k: v.cpu().numpy().astype(np.float64) for k, v in got.items()},
                           rows.astype(np.float64))
    for c0, c1, name in ((0, 3, "mean"), (3, 7, "quat"), (7, 10, "log scale"), (10, 11, "opacity"),
                         (11, 14, "SH band 0"), (14, s2.cols(1), "SH band 1")):
        assert rel_err(got[:, c0:c1], g_want[:, c0:c1]) <= 2e-3, name


def _psnr(a, b):
    return -10 * math.log10(float(((a - b) ** 2).mean()))


def test_stage2_recovers_an_emerging_object():
    """Stage 1 (transformation cache) cannot create the object that appears in
    the target frame; Stage 2 adds Gaussians around the high-gradient region
    and raises the PSNR of the training views, on the object's pixels and on
    the whole views.  The same number spawned around randomly chosen
    Gaussians (the paper's random-spawn ablation) is run and printed."""
    sc = scenes.make_scene(4, n_gauss=20_000, W=320, H=180)
    W, H, Vb = 320, 180, 4
    cams = sc.cams
    nb = len(cams) // Vb
    G = gs3.Gaussians.from_numpy(sc.prev)
    Gt = gs3.Gaussians.from_numpy(sc.target)
    cd = gs3.cameras_to_device(cams)
    bc = [gs3.camera_slice(cd, b * Vb, Vb) for b in range(nb)]
    tg = torch.cat([render(Gt, cams[b * Vb:(b + 1) * Vb], W, H) for b in range(nb)])
    batches = [(bc[b], tg[b * Vb:(b + 1) * Vb]) for b in range(nb)]
    rng = np.random.default_rng(89)
    og = oracle.Grid()
    table = rng.uniform(-1e-4, 1e-4, size=(og.n_entries, 2)).astype(np.float32)
    Ws = [w.astype(np.float32) for w in scenes.random_mlp([32, 64, 64, 7], rng)]
    ntc = NTC(table, Ws, gs3.hashgrid(), gs3.GS_MLP_FP32)
    warmup(ntc, G, iters=300)
    st1 = Stage1(G, ntc, Vb, W, H, capacity=1 << 20)
    st1.raster.fit_capacity(G, bc[0], *st1.transform(), margin=2.0)
    for it in range(150):
        if it == 150 - nb:
            track = st1.track_viewspace(True)
        st1.step(*batches[it % nb])
    st1.track_viewspace(False)
    mt, qt = [x.clone() for x in st1.transform()]

    def all_views(gs, mean=None, quat=None):
        return torch.cat([render(gs, cams[b * Vb:(b + 1) * Vb], W, H, mean, quat) for b in range(nb)])

    # the object's pixels: where the target differs from the target without it
    n_prev = sc.prev.n
    no_obj = torch.cat([render(gs3.Gaussians.from_numpy(sc.target.subset(np.arange(n_prev))),
                               cams[b * Vb:(b + 1) * Vb], W, H) for b in range(nb)])
    mask = ((tg - no_obj).abs().amax(dim=1, keepdim=True) > 0.02).expand_as(tg)
    assert mask.float().mean() > 0.002

    def psnr_obj(img):
        return -10 * math.log10(float(((img - tg)[mask] ** 2).mean()))

    img1 = all_views(G, mt, qt)
    p1, p1o = _psnr(img1, tg), psnr_obj(img1)
    results = {}
    for mode in ("adaptive", "random"):
        st2 = Stage2(G, Vb, W, H, capacity=20_000, pair_capacity=1 << 22, seed=3)
        if mode == "adaptive":
            k = st2.begin(mt, qt, *track)
            n_spawn = k
        else:
            k = st2.begin(mt, qt, *track, random_count=n_spawn)
        assert k > 0
        st2.run(batches, iters=100)
        img = all_views(st2.view())
        results[mode] = (_psnr(img, tg), psnr_obj(img), st2.n_add)
    print("object pixels %.4f; stage1 %.2f dB (object %.2f); adaptive %.2f dB (object %.2f, %d added, "
          "%d spawned); random %.2f dB (object %.2f, %d added)"
          % (float(mask.float().mean()), p1, p1o, results["adaptive"][0], results["adaptive"][1],
             results["adaptive"][2], n_spawn, results["random"][0], results["random"][1],
             results["random"][2]))
    assert results["adaptive"][1] > p1o + 5.0        # the object's pixels
    assert results["adaptive"][0] > p1 + 2.0          # the whole views
    # the random-spawn ablation is reported, not asserted: with the per-epoch
    # split and prune both sets of added Gaussians end near the object here
    assert results["random"][2] > 0


def test_stage2_degenerate_counts():
    """Nothing above the gradient threshold: no index selected and a spawn of
    zero rows leaves the added set unchanged; every added Gaussian below the
    opacity threshold: quantity control keeps none; an empty source: an empty
    result.  No error flag in any case."""
    rng = np.random.default_rng(87)
    deg, n = 1, 300
    g = scenes.make_gaussians(n, deg, rng)
    G = gs3.Gaussians.from_numpy(g)
    acc = torch.full((n,), 1e-9, device=DEV)
    den = torch.ones(n, dtype=torch.int32, device=DEV)
    idx = torch.full((n,), -7, dtype=torch.int32, device=DEV)
    nsel = torch.full((1,), 99, dtype=torch.int64, device=DEV)
    gs3.gs_select_above(acc, den, n, 1e-3, idx, nsel)
    torch.cuda.synchronize()
    assert int(nsel.item()) == 0
    rows, m, v, a = _added_buffers(64, deg)
    rows.fill_(3.0)
    nadd = torch.tensor([5], dtype=torch.int64, device=DEV)
    err = torch.zeros(1, dtype=torch.int32, device=DEV)
    gs3.gs_added_spawn(G, idx, nsel, torch.zeros(n, 3, device=DEV), 0.1, a, nadd, err)
    torch.cuda.synchronize()
    assert int(nadd.item()) == 5 and int(err.item()) == 0 and float(rows.min()) == 3.0
    # all below tau_alpha
    P = gs3.added_cols(deg)
    src_rows, sm, sv, src = _added_buffers(n, deg)
    r = rng.normal(size=(n, P)).astype(np.float32)
    r[:, 10] = np.log(0.001 / 0.999)                       # opacity 0.001 < 0.01
    src_rows.copy_(_t(r))
    dst_rows, dm, dv, dst = _added_buffers(2 * n, deg)
    nd = torch.full((1,), 42, dtype=torch.int64, device=DEV)
    big = torch.ones(n, device=DEV)                        # all above tau_grad, but pruned first
    gs3.gs_added_densify_prune(src, n, big, den, 2e-4, 0.01, 0.8, 0.1, torch.zeros(n, 3, device=DEV),
                               dst, nd, err)
    torch.cuda.synchronize()
    assert int(nd.item()) == 0 and int(err.item()) == 0
    want, keep, split = s2.densify_prune(r.astype(np.float64), np.ones(n), np.ones(n, np.int64),
                                         2e-4, 0.01, 0.8, np.zeros((n, 3)))
    assert want.shape[0] == 0 and not keep.any() and not split.any()
    # empty source
    nd.fill_(42)
    gs3.gs_added_densify_prune(src, 0, big, den, 2e-4, 0.01, 0.8, 0.1, torch.zeros(n, 3, device=DEV),
                               dst, nd, err)
    torch.cuda.synchronize()
    assert int(nd.item()) == 0 and int(err.item()) == 0
