"""Parity at the benchmark's full sizes, in the launch configuration the
benchmark times (bins of 4x4 tiles, 4-view launches where a view is
compared), on outputs the FP64 oracle can compute in seconds: one full view
of the 250K-Gaussian 1352x1014 and the 1M-Gaussian 1920x1080 workloads, the
full-resolution binning of one view, and the mixed-precision image error of
the transformation cache on every workload."""
import math

import numpy as np
import pytest
import torch

import oracle
from paper_2403_01444_gb300 import gs3, scenes
from paper_2403_01444_gb300.engine import NTC, Rasterizer, Stage1, render

pytestmark = pytest.mark.gpu
DEV = "cuda"


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2403_01444_gb300 import build
    build.build()
    gs3.lib()
    oracle.build()


def rel_err(a, b):
    a, b = np.asarray(a, np.float64), np.asarray(b, np.float64)
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-30))


def _window(W, H, tiles=32):
    """A centred crop of tiles x tiles 16-pixel tiles: (tx0, ty0, tx1, ty1) and a pixel mask."""
    tx, ty = math.ceil(W / 16), math.ceil(H / 16)
    x0, y0 = max(0, tx // 2 - tiles // 2), max(0, ty // 2 - tiles // 2)
    win = (x0, y0, min(tx, x0 + tiles), min(ty, y0 + tiles))
    mask = np.zeros((H, W), bool)
    mask[win[1] * 16:win[3] * 16, win[0] * 16:win[2] * 16] = True
    return win, mask


def _unambiguous(g, cams, margin=1e-3, mean=None, quat=None):
    """Keep the Gaussians whose radius and tile rectangle lie farther than
    `margin` from a rounding boundary in every view (decided by the FP64
    oracle, at the given means and rotations)."""
    o = oracle.project(g, cams, mean=mean, quat=quat)
    keep = np.all((o["radius"] == 0) | (o["margin"] > margin), axis=0)
    return keep


@pytest.mark.parametrize("cfg_index,view", [(3, 7), (5, 3)])
def test_full_size_view_render_and_gradients(cfg_index, view, record_property):
    sc = scenes.make_scene(cfg_index)
    cams = [sc.cams[view]]
    W, H = sc.cfg.W, sc.cfg.H
    keep = _unambiguous(sc.prev, cams)
    assert keep.mean() > 0.99
    g = sc.prev.subset(np.nonzero(keep)[0])
    win, crop = _window(W, H)
    r = oracle.render(g, cams, window=win)
    G = gs3.Gaussians.from_numpy(g)
    cd = gs3.cameras_to_device(cams)
    rast = Rasterizer(g.n, 1, W, H, 1 << 22, DEV, bin=4)  # bins of 4x4 tiles, as timed
    rast.fit_capacity(G, cd)
    img = rast.img.cpu().numpy()
    ok = (r["ambig"] == 0) & crop[None]
    # dense views flag many pixels (depth ties within FP32 reach whose swap
    # could move the pixel by more than 2.5e-5); half the crop must remain
    frac = float(ok.sum() / crop.sum())
    record_property("certified_fraction", frac)
    print("config %d view %d: %.3f of the central crop certified (FP32 image)" % (cfg_index, view, frac))
    assert frac > 0.8, frac
    okc = np.broadcast_to(ok[:, None], img.shape)
    assert np.abs(img - r["img"])[okc].max() <= 1e-4
    # backward of the same view against the oracle's, on the crop's unambiguous pixels
    d_img = np.random.default_rng(cfg_index).normal(size=img.shape) * ok[:, None]
    grads = oracle.raster_bwd(r["proj"], W, H, r["T_final"], r["last"], d_img, window=win)
    gs3.gs_raster_bwd(rast.proj, g.n, 1, W, H, rast.bin, rast.bg, rast.vals, rast.ranges,
                      rast.T_final, rast.last, torch.from_numpy(d_img.astype(np.float32)).to(DEV),
                      rast.grads)
    torch.cuda.synchronize()
    got = rast.grads.cpu().numpy()
    for sl in (slice(0, 2), slice(2, 5), slice(5, 8)):
        assert rel_err(got[..., sl], grads[..., sl]) <= 1e-3
    # the reverse staged from the forward's per-tile lists (as the training
    # step runs it) gives the same gradients, to the order of the FP32 atomics;
    # the densest tiles of the 1M-Gaussian view overflow the list (about 2 %)
    # and take the re-testing path
    listed = int((rast.lists.count >= 0).sum()) / rast.lists.count.numel()
    record_property("listed_tiles", listed)
    assert listed > 0.9, listed
    gs3.gs_raster_bwd(rast.proj, g.n, 1, W, H, rast.bin, rast.bg, rast.vals, rast.ranges,
                      rast.T_final, rast.last, torch.from_numpy(d_img.astype(np.float32)).to(DEV),
                      rast.grads, lists=rast.lists)
    torch.cuda.synchronize()
    assert rel_err(rast.grads.cpu().numpy(), got) <= 1e-5


def test_full_resolution_binning_bit_exact():
    """One 1352x1014 view, 250K records with the footprint sizes of the
    workload: keys, values and ranges identical to the oracle's sort."""
    W, H, N = 1352, 1014, 250_000
    rec = scenes.random_projected(1, N, W, H, np.random.default_rng(33), radius_range=(2, 60))
    p = gs3.Projected.empty(1, N, DEV)
    t = lambda a, dt=torch.float32: torch.from_numpy(np.ascontiguousarray(a)).to(DEV, dt)
    p.mean2d.copy_(t(rec["mean2d"]))
    p.conic_opacity.copy_(t(np.concatenate([rec["conic"], rec["opacity"][..., None]], -1)))
    p.rgb.copy_(t(rec["rgb"]))
    p.depth.copy_(t(rec["depth"]))
    p.radius.copy_(t(rec["radius"], torch.int32))
    count, keys, vals, ranges = oracle.bin_sort(rec["mean2d"], rec["radius"], rec["depth"], W, H)
    r = Rasterizer(N, 1, W, H, count + 16, DEV, bin=1)
    k = torch.zeros(count + 16, dtype=torch.int64, device=DEV)
    gs3.gs_bin_sort(p, N, 1, W, H, 1, r.capacity, r.vals, r.ranges, k, r.d_count, r.d_err, r.ws)
    torch.cuda.synchronize()
    assert r.count() == count and int(r.d_err.item()) == 0
    assert np.array_equal(k[:count].cpu().numpy().view(np.uint64), keys)
    assert np.array_equal(r.vals[:count].cpu().numpy().view(np.uint32), vals)
    assert np.array_equal(r.ranges.cpu().numpy().view(np.uint32), ranges)


U_BF16 = 2.0 ** -9   # unit roundoff of BF16 (8 significant bits, round to nearest)
U_FP16 = 2.0 ** -11  # unit roundoff of FP16 (11 significant bits)
LAMBDA_ROUND = 12.0  # standard deviations of the probabilistic rounding error bound


def _cache_params(rng, entries):
    """Cache parameters giving a visible, smooth transformation: translations
    of a few 1e-3 and rotations of a few degrees, from table features of zero
    mean and 0.05 spread (a trained table starts at zero and stays near it)."""
    table = rng.normal(0.0, 0.05, size=(entries, 2)).astype(np.float32)
    Ws = [w.astype(np.float32) for w in scenes.random_mlp([32, 64, 64, 7], rng)]
    Ws[2][0:3] *= 0.02
    Ws[2][3] = np.abs(Ws[2][3]) + 1.0
    Ws[2][4:7] *= 0.05
    return table, Ws


def _r3(conic):
    """3 sqrt(lambda_max) of the 2D covariance whose inverse is `conic`, with
    the 0.1 floor on the discriminant (Section 3.2's footprint radius before
    rounding up)."""
    A, B, C = (conic[..., k] for k in range(3))
    det = A * C - B * B
    with np.errstate(divide="ignore", invalid="ignore"):
        a, b, c = C / det, -B / det, A / det
    mid = 0.5 * (a + c)
    return 3 * np.sqrt(mid + np.sqrt(np.maximum(mid * mid - (a * c - b * b), 0.1)))


def _reach(g, cams, mean, quat, d_mu, d_q):
    """Per-record reach of a perturbation of the means by up to d_mu[i] and of
    the rotations by up to d_q[i] per component (Gaussian i), from FP64
    projections at every corner of each box (8 for the mean, 16 for the
    rotation; the two reaches add, to first order), plus 10% for the second
    order: displacement of the 2D mean (pixels), change of the conic relative
    to its smallest eigenvalue, change of the unrounded footprint radius
    (pixels), and change of the depth."""
    base = oracle.project(g, cams, mean=mean, quat=quat)
    A, B, C = (base["conic"][..., k] for k in range(3))
    lam_min = 0.5 * (A + C) - np.sqrt(0.25 * (A - C) ** 2 + B * B)
    vis = base["radius"] > 0
    r3 = np.where(vis, _r3(base["conic"]), 0.0)
    total = [np.zeros(A.shape) for _ in range(4)]
    for kind, n in (("mean", 3), ("quat", 4)):
        part = [np.zeros(A.shape) for _ in range(4)]
        for corner in range(1 << n):
            sign = np.array([1.0 if corner >> k & 1 else -1.0 for k in range(n)])
            if kind == "mean":
                p = oracle.project(g, cams, mean=mean + d_mu[:, None] * sign, quat=quat)
            else:
                p = oracle.project(g, cams, mean=mean, quat=quat + d_q[:, None] * sign)
            dc = p["conic"] - base["conic"]
            fro = np.sqrt(dc[..., 0] ** 2 + 2 * dc[..., 1] ** 2 + dc[..., 2] ** 2)
            part[0] = np.maximum(part[0], np.linalg.norm(p["mean2d"] - base["mean2d"], axis=-1))
            part[1] = np.maximum(part[1], np.where(vis, fro / np.where(vis, lam_min, 1.0), 0.0))
            part[2] = np.maximum(part[2], np.where(vis, np.abs(_r3(p["conic"]) - r3), 0.0))
            part[3] = np.maximum(part[3], np.abs(p["depth"] - base["depth"]))
        total = [t + q for t, q in zip(total, part)]
    pos, rel, dr3, dz = (1.1 * t for t in total)
    return pos, rel, dr3, dz, base


@pytest.mark.parametrize("cfg_index", [1, 2, 3, 4, 5])
def test_mixed_precision_cache_and_image(cfg_index, record_property):
    """The mixed-precision cache (FP16 table, BF16 tensor-core MLP with an FP32
    output layer) against the FP64 oracle holding the same FP32 master
    parameters, on one view of every workload:
    - each raw output of the cache lies within a probabilistic rounding error
      bound of the mixed path (FP16 table, BF16 operands of the hidden layers);
    - the rendered image lies within 2e-3 (max abs) of the oracle's on every
      pixel whose decisions that cache error cannot flip: the oracle flags
      threshold decisions within the reach of the error (means moved by the
      bound on the translation, rotations by the bound on the rotation) and
      depth ties within its depth reach whose swap could move the pixel by
      more than 5e-4; Gaussians whose footprint radius or tile rectangle lies
      within that reach of a boundary are left out of both renders;
    - the PSNR of the whole crop against the target lies within 0.05 dB of the
      oracle's."""
    sc = scenes.make_scene(cfg_index)
    cams = [sc.cams[0]]
    W, H = sc.cfg.W, sc.cfg.H
    rng = np.random.default_rng(80 + cfg_index)
    og = oracle.Grid()
    table, Ws = _cache_params(rng, og.n_entries)
    g = sc.prev
    f = oracle.ntc_forward(oracle.NTCParams(og, table, Ws), g.mean, g.quat)
    G = gs3.Gaussians.from_numpy(g)
    ntc = NTC(table, Ws, gs3.hashgrid(), gs3.GS_MLP_BF16)
    st = Stage1(G, ntc, 1, W, H, capacity=1 << 20)
    m, q = st.transform()
    torch.cuda.synchronize()
    raw = st.raw7.cpu().numpy().astype(np.float64)
    # the cache: probabilistic rounding error bound of the mixed path
    # (independent roundings add in quadrature; Higham and Mary, 2019): FP16
    # table entries (unit 2^-11), BF16 operands of both hidden layers (unit
    # 2^-9 on each of the two factors), each a uniform error of variance
    # u^2 x^2 / 3, carried through the layers (ReLU passes errors on unchanged
    # at most); FP32 accumulation and output layer.  LAMBDA_ROUND standard
    # deviations leave a wide margin over the largest ratio seen in 7M outputs
    # (about 7.6)
    W1, W2, W3 = (w.astype(np.float64) for w in Ws)
    v1 = (f["enc"] ** 2 * (2 * U_BF16 ** 2 + U_FP16 ** 2) / 3) @ (W1 ** 2).T
    v2 = (f["h1"] ** 2 * 2 * U_BF16 ** 2 / 3 + v1) @ (W2 ** 2).T
    bnd = LAMBDA_ROUND * np.sqrt(v2 @ (W3 ** 2).T)
    assert np.all(np.abs(raw - f["raw7"]) <= bnd + 1e-7)
    # per-Gaussian bounds on the transformation: the translation (+ FP32
    # rounding of the sum), and the normalised rotation r / |r|, whose change
    # is the part of dr orthogonal to r over |r|: with r = (w, v), at most
    # (|dv| + |dw| |v| / |r|) / |r| to first order; multiplying by the unit
    # previous rotation keeps that length
    d_mu = bnd[:, 0:3].max(axis=1) + 1e-6
    r = f["raw7"][:, 3:7]
    nr, nv = np.linalg.norm(r, axis=1), np.linalg.norm(r[:, 1:], axis=1)
    d_q = 1.01 * (np.sqrt(3) * bnd[:, 4:7].max(axis=1) + bnd[:, 3] * nv / nr) / nr + 1e-6
    # the image
    win, crop = _window(W, H)
    pos, rel, dr3, dz, base = _reach(g, cams, f["mean"], f["quat"], d_mu, d_q)
    keep = _unambiguous(g, cams, pos + dr3 + 1e-3, f["mean"], f["quat"])
    assert keep.mean() > 0.85
    # the three densest workloads are thinned (every 2nd, 4th, 16th Gaussian)
    # for this part: at full density nearly every pixel holds a run of
    # Gaussians whose order the cache error can permute, and certifies nothing
    thin = {3: 2, 4: 4, 5: 16}.get(cfg_index, 1)
    idx = np.nonzero(keep & (np.arange(g.n) % thin == 0))[0]
    sub = g.subset(idx)
    want = oracle.render(sub, cams, f["mean"][idx], f["quat"][idx], window=win, tie=4e-7,
                         tie_budget=5e-4, depth_eps=dz[:, idx], pos_eps=pos[:, idx],
                         rel_eps=rel[:, idx])
    kd = torch.from_numpy(idx).to(DEV)
    img = render(gs3.Gaussians.from_numpy(sub), cams, W, H, m[kd].contiguous(),
                 q[kd].contiguous()).cpu().numpy()
    ok = (want["ambig"] == 0) & crop[None]
    frac = float(ok.sum() / crop.sum())
    record_property("certified_fraction", frac)
    record_property("thinned_every", thin)
    print("config %d: %.3f of the central crop certified (mixed precision, every %d-th Gaussian)"
          % (cfg_index, frac, thin))
    # measured 0.88, 0.67, 0.19, 0.22, 0.25 for configs 1..5
    assert frac > {1: 0.8, 2: 0.55, 3: 0.15, 4: 0.15, 5: 0.2}[cfg_index], frac
    err = np.abs(img - want["img"])
    assert err[np.broadcast_to(ok[:, None], img.shape)].max() <= 2e-3
    # PSNR of the whole scene's crop
    full = oracle.render(g, cams, f["mean"], f["quat"], window=win)["img"]
    target = oracle.render(sc.target, cams, window=win)["img"]
    got = render(G, cams, W, H, m, q).cpu().numpy()
    cm = np.broadcast_to(crop[None, None], got.shape)
    psnr = lambda a: -10 * math.log10(np.mean((a[cm] - target[cm]) ** 2))
    assert abs(psnr(got) - psnr(full)) <= 0.05
