"""Parity of every CUDA entry point with the FP64 oracle, element by element,
on the same seeded inputs, at sizes spanning several tiles and ragged tails.

Tolerances: integer, key and index outputs bit-exact; FP32 images <= 1e-4 max
abs; gradients <= 1e-3 relative per tensor (||g - g_ref|| / ||g_ref||) and
elementwise <= 1e-3 * max|g_ref|.  Pixels where the oracle reports a
compositing decision within a small margin of its threshold (where FP32 and
FP64 may decide apart) are compared for validity only, and must be rare.
"""
import math

import numpy as np
import pytest
import torch

import oracle
from paper_2403_01444_gb300 import gs3, scenes
from paper_2403_01444_gb300.engine import Rasterizer

pytestmark = pytest.mark.gpu
DEV = "cuda"


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2403_01444_gb300 import build
    build.build()
    gs3.lib()


def t(a, dtype=torch.float32):
    return torch.from_numpy(np.ascontiguousarray(a)).to(DEV, dtype)


def rel_err(a, b):
    a, b = np.asarray(a, np.float64), np.asarray(b, np.float64)
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-30))


def assert_grad_close(got, want, rtol=1e-3):
    got, want = np.asarray(got, np.float64), np.asarray(want, np.float64)
    assert rel_err(got, want) <= rtol, rel_err(got, want)
    scale = max(np.abs(want).max(), 1e-30)
    assert np.abs(got - want).max() <= rtol * scale * 10, np.abs(got - want).max() / scale


def projected_from_records(rec, device=DEV):
    V, N = rec["depth"].shape
    p = gs3.Projected.empty(V, N, device)
    p.mean2d.copy_(t(rec["mean2d"]))
    co = np.concatenate([rec["conic"], rec["opacity"][..., None]], -1)
    p.conic_opacity.copy_(t(co))
    p.rgb.copy_(t(rec["rgb"]))
    p.depth.copy_(t(rec["depth"]))
    p.radius.copy_(t(rec["radius"], torch.int32))
    p.tiles_touched.zero_()
    return p


def gpu_bin_sort(p, N, V, W, H, capacity=None, keys=True, bin=1):
    cap = capacity if capacity is not None else 4 * N * V * 64 + 16
    r = Rasterizer(N, V, W, H, cap, DEV, bin=bin)
    r.proj = p
    k = torch.zeros(max(cap, 1), dtype=torch.int64, device=DEV) if keys else None
    gs3.gs_bin_sort(p, N, V, W, H, bin, r.capacity, r.vals, r.ranges, k, r.d_count, r.d_err, r.ws)
    torch.cuda.synchronize()
    return r, k


# ------------------------------------------------------------------ binning
@pytest.mark.parametrize("V,N,W,H,seed", [(1, 1, 16, 16, 0), (1, 300, 70, 50, 1), (3, 500, 133, 97, 2),
                                          (4, 2000, 480, 360, 3), (2, 4096, 128, 96, 4)])
def test_bin_sort_bit_exact(V, N, W, H, seed):
    rec = scenes.random_projected(V, N, W, H, np.random.default_rng(seed))
    # equal depths on purpose: ties must break by Gaussian index
    rec["depth"][:, ::7] = rec["depth"][:, :1]
    p = projected_from_records(rec)
    r, k = gpu_bin_sort(p, N, V, W, H)
    count, keys, vals, ranges = oracle.bin_sort(rec["mean2d"], rec["radius"], rec["depth"], W, H)
    assert r.count() == count
    assert int(r.d_err.item()) == 0
    got_keys = k[:count].cpu().numpy().view(np.uint64)
    np.testing.assert_array_equal(got_keys, keys)
    np.testing.assert_array_equal(r.vals[:count].cpu().numpy().view(np.uint32), vals)
    np.testing.assert_array_equal(r.ranges.cpu().numpy().view(np.uint32), ranges)


@pytest.mark.parametrize("pattern", ["byte1", "bytes02", "all_equal", "all_vary"])
def test_bin_sort_constant_depth_bytes(pattern):
    """A depth-sort pass whose byte is the same in every key is skipped, and
    each later pass finds the buffer holding the keys from the passes before
    it that were not skipped.  Depths built bit by bit so that byte 1, or
    bytes 0 and 2, or every byte (all equal: ties by index) is constant, and a
    control where all four vary, give the oracle's keys, values and ranges
    bit for bit.  No entry is culled here: a culled entry's key has every
    byte 0xff and would make each byte vary."""
    V, N, W, H = 2, 900, 200, 130
    rng = np.random.default_rng(61)
    rec = scenes.random_projected(V, N, W, H, rng)
    rec["radius"] = np.maximum(rec["radius"], 1).astype(rec["radius"].dtype)
    rb = lambda lo, hi: rng.integers(lo, hi + 1, size=(V, N)).astype(np.uint32)
    top = np.where(rng.random((V, N)) < 0.5, 0x3F, 0x40).astype(np.uint32)  # positive depths 0.6 .. 4
    if pattern == "byte1":
        bits = (top << 24) | (rb(0x20, 0x7F) << 16) | (0x5A << 8) | rb(0, 255)  # three passes: odd
    elif pattern == "bytes02":
        bits = (top << 24) | (0x20 << 16) | (rb(0, 255) << 8) | 0x11  # the first pass skipped
    elif pattern == "all_equal":
        bits = np.full((V, N), 0x40400000, np.uint32)
    else:
        bits = (top << 24) | (rb(0x20, 0x7F) << 16) | (rb(0, 255) << 8) | rb(0, 255)
    rec["depth"] = bits.astype(np.uint32).view(np.float32)
    assert (rec["depth"] > 0).all()
    p = projected_from_records(rec)
    r, k = gpu_bin_sort(p, N, V, W, H)
    count, keys, vals, ranges = oracle.bin_sort(rec["mean2d"], rec["radius"], rec["depth"], W, H)
    assert count > 0 and r.count() == count
    assert int(r.d_err.item()) == 0
    np.testing.assert_array_equal(k[:count].cpu().numpy().view(np.uint64), keys)
    np.testing.assert_array_equal(r.vals[:count].cpu().numpy().view(np.uint32), vals)
    np.testing.assert_array_equal(r.ranges.cpu().numpy().view(np.uint32), ranges)


def test_bin_sort_all_culled_and_capacity_overflow():
    V, N, W, H = 2, 400, 100, 60
    rec = scenes.random_projected(V, N, W, H, np.random.default_rng(9))
    rec0 = dict(rec)
    rec0["radius"] = np.zeros_like(rec["radius"])
    r, _ = gpu_bin_sort(projected_from_records(rec0), N, V, W, H)
    assert r.count() == 0 and not r.ranges.any()
    count = oracle.bin_sort(rec["mean2d"], rec["radius"], rec["depth"], W, H)[0]
    r, _ = gpu_bin_sort(projected_from_records(rec), N, V, W, H, capacity=count - 1)
    assert r.count() == count
    assert int(r.d_err.item()) == gs3.GS_ERR_CAPACITY
    assert not r.ranges.any()  # nothing usable is published on overflow
    r, _ = gpu_bin_sort(projected_from_records(rec), N, V, W, H, capacity=count)
    assert int(r.d_err.item()) == 0 and r.count() == count


# --------------------------------------------------------------- compositing
def raster_case(V, N, W, H, seed, bin=1, **kw):
    rec = scenes.random_projected(V, N, W, H, np.random.default_rng(seed), **kw)
    p = projected_from_records(rec)
    r, _ = gpu_bin_sort(p, N, V, W, H, keys=False, bin=bin)
    bg = (0.1, 0.2, 0.3)
    gs3.gs_raster_fwd(p, N, V, W, H, bin, bg, r.vals, r.ranges, r.img, r.T_final, r.last)
    torch.cuda.synchronize()
    return rec, p, r, bg


@pytest.mark.parametrize("V,N,W,H,seed", [(1, 50, 40, 24, 10), (2, 1500, 150, 110, 11),
                                          (3, 4000, 257, 129, 12)])
def test_raster_fwd_parity(V, N, W, H, seed):
    rec, p, r, bg = raster_case(V, N, W, H, seed)
    img, Tf, last, amb = oracle.raster_fwd(rec, W, H, bg)
    ok = amb == 0
    assert ok.mean() > 0.98
    gi = r.img.cpu().numpy()
    okc = np.broadcast_to(ok[:, None], gi.shape)
    assert np.abs(gi - img)[okc].max() <= 1e-4
    assert np.abs(r.T_final.cpu().numpy() - Tf)[ok].max() <= 1e-4
    np.testing.assert_array_equal(r.last.cpu().numpy()[ok], last[ok])
    # ambiguous pixels still hold valid values
    assert np.all((gi >= 0) & (gi <= 1.0 + 1e-5))


@pytest.mark.parametrize("V,N,W,H,seed", [(1, 60, 40, 24, 20), (2, 1200, 150, 110, 21)])
def test_raster_bwd_parity(V, N, W, H, seed):
    rec, p, r, bg = raster_case(V, N, W, H, seed)
    img, Tf, last, amb = oracle.raster_fwd(rec, W, H, bg)
    d_img = np.random.default_rng(seed + 100).normal(size=img.shape)
    d_img *= (amb == 0)[:, None]  # decisions near a threshold are not comparable
    grads, dop = oracle.raster_bwd(rec, W, H, Tf, last, d_img, bg, want_opacity=True)
    gg = torch.zeros(V, N, 8, device=DEV)
    gop = torch.zeros(V, N, device=DEV)
    gs3.gs_raster_bwd(p, N, V, W, H, 1, bg, r.vals, r.ranges, r.T_final, r.last, t(d_img), gg, gop)
    torch.cuda.synchronize()
    gg = gg.cpu().numpy()
    for sl in (slice(0, 2), slice(2, 5), slice(5, 8)):
        assert_grad_close(gg[..., sl], grads[..., sl])
    assert_grad_close(gop.cpu().numpy(), dop)


@pytest.mark.parametrize("bin", [2, 3, 8])
def test_binned_keys_brute_force(bin):
    """Bins of bin x bin tiles: keys (view * bins + bin_id) << 32 | depth bits,
    values and ranges against a brute-force enumeration of (entry, bin) pairs."""
    V, N, W, H = 2, 700, 200, 130
    rec = scenes.random_projected(V, N, W, H, np.random.default_rng(40 + bin))
    rec["depth"][:, ::5] = rec["depth"][:, :1]
    p = projected_from_records(rec)
    r, k = gpu_bin_sort(p, N, V, W, H, bin=bin)
    tx, ty = math.ceil(W / 16), math.ceil(H / 16)
    bx, by = math.ceil(tx / bin), math.ceil(ty / bin)
    pairs = []
    for v in range(V):
        for i in range(N):
            rr = int(rec["radius"][v, i])
            if rr <= 0:
                continue
            u, w = (float(x) for x in rec["mean2d"][v, i])
            x0 = min(tx, max(0, math.floor((u - rr) / 16)))
            x1 = min(tx, max(0, math.floor((u + rr + 15) / 16)))
            y0 = min(ty, max(0, math.floor((w - rr) / 16)))
            y1 = min(ty, max(0, math.floor((w + rr + 15) / 16)))
            if x1 <= x0 or y1 <= y0:
                continue
            db = int(np.float32(rec["depth"][v, i]).view(np.uint32))
            for yb in range(y0 // bin, (y1 - 1) // bin + 1):
                for xb in range(x0 // bin, (x1 - 1) // bin + 1):
                    pairs.append((((v * bx * by + yb * bx + xb) << 32) | db, i))
    pairs.sort()
    n = r.count()
    assert n == len(pairs)
    assert [int(x) for x in k[:n].cpu().numpy().view(np.uint64)] == [q[0] for q in pairs]
    assert [int(x) for x in r.vals[:n].cpu().numpy().view(np.uint32)] == [q[1] for q in pairs]


@pytest.mark.parametrize("bin", [2, 4, 8])
def test_binned_raster_equals_per_tile(bin):
    """A tile's records, taken on the fly from its bin's list, are the per-tile
    list: identical images and transmittance, and equal gradients."""
    V, N, W, H = 2, 3000, 300, 170
    rec, p, r1, bg = raster_case(V, N, W, H, 50, bin=1)
    _, p2, r2, _ = raster_case(V, N, W, H, 50, bin=bin)
    assert torch.equal(r1.img, r2.img)
    assert torch.equal(r1.T_final, r2.T_final)
    d_img = t(np.random.default_rng(51).normal(size=(V, 3, H, W)))
    g1 = torch.zeros(V, N, 8, device=DEV)
    g2 = torch.zeros(V, N, 8, device=DEV)
    o1 = torch.zeros(V, N, device=DEV)
    o2 = torch.zeros(V, N, device=DEV)
    gs3.gs_raster_bwd(p, N, V, W, H, 1, bg, r1.vals, r1.ranges, r1.T_final, r1.last, d_img, g1, o1)
    gs3.gs_raster_bwd(p2, N, V, W, H, bin, bg, r2.vals, r2.ranges, r2.T_final, r2.last, d_img, g2, o2)
    torch.cuda.synchronize()
    assert rel_err(g2.cpu().numpy(), g1.cpu().numpy()) <= 1e-5
    assert rel_err(o2.cpu().numpy(), o1.cpu().numpy()) <= 1e-5


@pytest.mark.parametrize("bin,cap", [(1, "all"), (4, "all"), (4, "half")])
def test_reverse_from_tile_lists_equals_retested(bin, cap):
    """The reverse staged from the forward's per-tile lists (gs_tile_lists)
    equals the reverse that tests the bin's list again: the same gradients (to
    the order of the FP32 atomics).  Each list holds records of its tile's
    bin list in position order.  With room for every tile's records all
    tiles are listed; with a cap at the median count the tiles with more
    staged records say so (count -1) and take the re-testing path, the
    others the list."""
    V, N, W, H = 2, 3000, 300, 170
    rec = scenes.random_projected(V, N, W, H, np.random.default_rng(52))
    p = projected_from_records(rec)
    r, _ = gpu_bin_sort(p, N, V, W, H, keys=False, bin=bin)
    bg = (0.1, 0.2, 0.3)
    gs3.gs_raster_fwd(p, N, V, W, H, bin, bg, r.vals, r.ranges, r.img, r.T_final, r.last)
    img = r.img.clone()
    full = gs3.TileLists(V, W, H, 4096, DEV)  # above N: room for any tile
    gs3.gs_raster_fwd(p, N, V, W, H, bin, bg, r.vals, r.ranges, r.img, r.T_final, r.last, lists=full)
    torch.cuda.synchronize()
    assert torch.equal(img, r.img)  # writing the lists leaves the forward as it is
    staged = full.count.cpu().numpy()
    assert (staged >= 0).all()
    cap = 4096 if cap == "all" else max(1, int(np.median(staged)))
    lists = gs3.TileLists(V, W, H, cap, DEV)
    gs3.gs_raster_fwd(p, N, V, W, H, bin, bg, r.vals, r.ranges, r.img, r.T_final, r.last, lists=lists)
    torch.cuda.synchronize()
    cnt = lists.count.cpu().numpy()
    np.testing.assert_array_equal(cnt, np.where(staged <= cap, staged, -1))
    recs = lists.rec.cpu().numpy().view(np.uint32).reshape(-1, cap, 2)
    vals, ranges = r.vals.cpu().numpy().view(np.uint32), r.ranges.cpu().numpy().view(np.uint32)
    tx, ty = math.ceil(W / 16), math.ceil(H / 16)
    bins_x, bins = math.ceil(tx / bin), math.ceil(tx / bin) * math.ceil(ty / bin)
    assert (cnt > 0).any()
    if cap < 4096:
        assert (cnt == -1).any()
    for i in np.nonzero(cnt > 0)[0]:
        v, t_ = divmod(int(i), tx * ty)
        start = int(ranges[v * bins + (t_ // tx // bin) * bins_x + (t_ % tx) // bin, 0])
        e = recs[i, :cnt[i]]
        assert np.all(np.diff(e[:, 1].astype(np.int64)) > 0)
        np.testing.assert_array_equal(vals[start + e[:, 1]], e[:, 0])
    d_img = t(np.random.default_rng(53).normal(size=(V, 3, H, W)))
    g1, g2 = torch.zeros(V, N, 8, device=DEV), torch.zeros(V, N, 8, device=DEV)
    o1, o2 = torch.zeros(V, N, device=DEV), torch.zeros(V, N, device=DEV)
    gs3.gs_raster_bwd(p, N, V, W, H, bin, bg, r.vals, r.ranges, r.T_final, r.last, d_img, g1, o1)
    gs3.gs_raster_bwd(p, N, V, W, H, bin, bg, r.vals, r.ranges, r.T_final, r.last, d_img, g2, o2,
                      lists=lists)
    torch.cuda.synchronize()
    assert float(g1.abs().max()) > 0
    assert rel_err(g2.cpu().numpy(), g1.cpu().numpy()) <= 1e-5
    assert rel_err(o2.cpu().numpy(), o1.cpu().numpy()) <= 1e-5


# ------------------------------------------------------------------ projection
def _proj_scene(seed, N=3000, deg=3, W=200, H=150):
    rng = np.random.default_rng(seed)
    g = scenes.make_gaussians(N, deg, rng)
    g.scale = (g.scale * 3).astype(np.float32)
    cams = scenes.ring_cameras([0, 100, 230], [0, 20, -10], W, H)
    return g, cams


def test_project_parity():
    g, cams = _proj_scene(30)
    W, H, V, N = 200, 150, 3, g.n
    G = gs3.Gaussians.from_numpy(g)
    cd = gs3.cameras_to_device(cams)
    p = gs3.Projected.empty(V, N)
    gs3.gs_project(G, cd, V, W, H, p)
    torch.cuda.synchronize()
    o = oracle.project(g, cams)
    valid = o["radius"] > 0
    clean = valid & (o["margin"] > 1e-3)
    got_r = p.radius.cpu().numpy()
    assert np.array_equal(got_r[clean], o["radius"][clean])
    assert np.array_equal(got_r > 0, valid) or np.mean((got_r > 0) != valid) < 1e-3
    m = clean & (got_r > 0)
    np.testing.assert_allclose(p.mean2d.cpu().numpy()[m], o["mean2d"][m], rtol=1e-5, atol=1e-3)
    co = p.conic_opacity.cpu().numpy()
    cmax = np.abs(o["conic"]).max(-1, keepdims=True)
    assert np.max(np.abs(co[..., :3] - o["conic"])[m] / cmax[m]) < 2e-4
    np.testing.assert_allclose(co[..., 3][m], o["opacity"][m], rtol=1e-6)
    np.testing.assert_allclose(p.rgb.cpu().numpy()[m], o["rgb"][m], atol=2e-6)
    np.testing.assert_allclose(p.depth.cpu().numpy()[m], o["depth"][m], rtol=1e-6)
    rect = o["rect"]
    ntiles = (rect[..., 2] - rect[..., 0]) * (rect[..., 3] - rect[..., 1])
    assert np.array_equal(p.tiles_touched.cpu().numpy()[m], ntiles[m])


def test_project_bwd_parity():
    g, cams = _proj_scene(31, N=2000)
    W, H, V, N = 200, 150, 3, g.n
    G = gs3.Gaussians.from_numpy(g)
    cd = gs3.cameras_to_device(cams)
    o = oracle.project(g, cams)
    rng = np.random.default_rng(32)
    grads = rng.normal(size=(V, N, 8)) * (o["radius"] > 0)[..., None]
    grads[..., 2:5] *= 1e-1
    dm, dq = oracle.project_bwd(g, cams, grads)
    gdm = torch.zeros(N, 3, device=DEV)
    gdq = torch.zeros(N, 4, device=DEV)
    gs3.gs_project_bwd(G, cd, V, W, H, t(grads), gdm, gdq)
    torch.cuda.synchronize()
    assert_grad_close(gdm.cpu().numpy(), dm)
    assert_grad_close(gdq.cpu().numpy(), dq)


# -------------------------------------------------------------------- loss
@pytest.mark.parametrize("V,H,W", [(1, 11, 13), (2, 50, 70), (1, 97, 133), (1, 97, 132), (2, 5, 8)])
def test_loss_parity(V, H, W):
    """Ragged tiles; widths that are multiples of 4 take the TMA-staged forward."""
    rng = np.random.default_rng(V * 1000 + H)
    x = rng.uniform(size=(V, 3, H, W)).astype(np.float32)
    y = np.clip(x + rng.normal(0, 0.15, size=x.shape), 0, 1).astype(np.float32)
    L, d, ss = oracle.loss_l1_dssim(x, y, 0.2)
    ws = torch.empty(gs3.gs_loss_workspace_size(3 * V, H, W), dtype=torch.uint8, device=DEV)
    gd = torch.zeros(V, 3, H, W, device=DEV)
    gl = torch.zeros(1, device=DEV)
    gsim = torch.zeros(1, device=DEV)
    gs3.gs_loss_l1_dssim(t(x), t(y), 3 * V, H, W, 0.2, gd, gl, gsim, ws)
    torch.cuda.synchronize()
    assert abs(gl.item() - L) <= 1e-5 * abs(L)
    assert abs(gsim.item() - ss) <= 1e-5
    assert_grad_close(gd.cpu().numpy(), d)


# -------------------------------------------------------------------- NTC
GRID = dict(levels=16, features=2, log2_table=17, n_min=16, n_max=1024)


def _grid_pair():
    og = oracle.Grid()
    gg = gs3.hashgrid(**GRID)
    return og, gg


@pytest.mark.parametrize("n", [1, 77, 5000])
def test_encode_parity_fp32_and_fp16(n):
    og, gg = _grid_pair()
    rng = np.random.default_rng(n)
    mu = rng.uniform(-1.6, 1.6, size=(n, 3)).astype(np.float32)  # some outside: clamped
    table = rng.normal(0, 0.1, size=(og.n_entries, 2)).astype(np.float32)
    want = oracle.encode(og, mu, table)
    enc = torch.zeros(n, 32, device=DEV)
    gs3.ntc_encode_fwd(t(mu), n, gg, t(table), enc)
    torch.cuda.synchronize()
    # FP32 cell coordinates at resolution 1024 carry ~1e-4 cells of rounding,
    # so the interpolated value may move by ~1e-3 of the table's magnitude
    tol = 1e-3 * np.abs(table).max()
    assert np.abs(enc.cpu().numpy() - want).max() <= tol
    th = table.astype(np.float16)
    want_h = oracle.encode(og, mu, th.astype(np.float64))
    encb = torch.zeros(n, 32, device=DEV, dtype=torch.bfloat16)
    gs3.ntc_encode_fwd(t(mu), n, gg, t(th, torch.float16), encb)
    torch.cuda.synchronize()
    got = encb.float().cpu().numpy()
    assert np.all(np.abs(got - want_h) <= 2 ** -8 * np.abs(want_h) + tol)


def test_encode_bwd_parity():
    og, gg = _grid_pair()
    n = 4000
    rng = np.random.default_rng(5)
    mu = rng.uniform(-1.5, 1.5, size=(n, 3)).astype(np.float32)
    d_enc = rng.normal(size=(n, 32)).astype(np.float32)
    want = oracle.encode_bwd(og, mu, d_enc)
    dt = torch.zeros(og.n_entries, 2, device=DEV)
    gs3.ntc_encode_bwd(t(mu), n, gg, t(d_enc), dt)
    torch.cuda.synchronize()
    assert_grad_close(dt.cpu().numpy(), want, rtol=1e-3)


@pytest.mark.parametrize("n", [1, 33, 70001])
def test_spatial_order_and_ordered_encoding(n):
    """ntc_spatial_order: the Gaussians sorted stably by the Morton code of
    their mean in the grid's box (10 bits an axis, as the definition: the
    FP32 coordinate (m - min) / extent clamped to [0, 1] times 1023,
    truncated), computed here in numpy; the encoding visited in that order is
    the same, bit for bit, and its reverse the same to the order of the FP32
    atomics."""
    og, gg = _grid_pair()
    rng = np.random.default_rng(n + 7)
    mu = rng.uniform(-1.6, 1.6, size=(n, 3)).astype(np.float32)
    mu[: n // 3] = mu[0]  # ties: equal codes keep the index order
    amin = np.float32(gg.aabb[0:3]); ext = np.float32(gg.aabb[3:6]) - amin
    x = np.clip((mu - amin) / ext, np.float32(0), np.float32(1)) * np.float32(1023)
    q = x.astype(np.uint32)

    def spread(v):
        v = v.astype(np.uint64) & 0x3FF
        v = (v | (v << 16)) & 0x30000FF
        v = (v | (v << 8)) & 0x300F00F
        v = (v | (v << 4)) & 0x30C30C3
        v = (v | (v << 2)) & 0x9249249
        return v

    code = spread(q[:, 0]) | (spread(q[:, 1]) << 1) | (spread(q[:, 2]) << 2)
    want = np.argsort(code, kind="stable")
    order = gs3.spatial_order(t(mu), n, gg)
    torch.cuda.synchronize()
    np.testing.assert_array_equal(order.cpu().numpy(), want)
    table = rng.normal(0, 0.1, size=(og.n_entries, 2)).astype(np.float32)
    e0 = torch.zeros(n, 32, device=DEV)
    e1 = torch.zeros(n, 32, device=DEV)
    gs3.ntc_encode_fwd(t(mu), n, gg, t(table), e0)
    gs3.ntc_encode_fwd(t(mu), n, gg, t(table), e1, order=order)
    d_enc = rng.normal(size=(n, 32)).astype(np.float32)
    d0 = torch.zeros(og.n_entries, 2, device=DEV)
    d1 = torch.zeros(og.n_entries, 2, device=DEV)
    gs3.ntc_encode_bwd(t(mu), n, gg, t(d_enc), d0)
    gs3.ntc_encode_bwd(t(mu), n, gg, t(d_enc), d1, order=order)
    torch.cuda.synchronize()
    assert torch.equal(e0, e1)
    assert rel_err(d1.cpu().numpy(), d0.cpu().numpy()) <= 1e-5


def _mlp(seed):
    rng = np.random.default_rng(seed)
    return [w.astype(np.float32) for w in scenes.random_mlp([32, 64, 64, 7], rng)], rng


@pytest.mark.parametrize("n", [1, 129, 3000])
def test_mlp_fp32_parity(n):
    Ws, rng = _mlp(n)
    x = rng.normal(size=(n, 32)).astype(np.float32)
    h1, h2, out = oracle.mlp_fwd(x, Ws)
    wflat = t(np.concatenate([w.ravel() for w in Ws]))
    mlp = gs3.mlp_struct(gs3.GS_MLP_FP32, wflat)
    raw = torch.zeros(n, 7, device=DEV)
    gs3.ntc_mlp_fwd(t(x), n, mlp, raw)
    torch.cuda.synchronize()
    assert np.abs(raw.cpu().numpy() - out).max() <= 1e-4 * max(1, np.abs(out).max())
    gout = rng.normal(size=(n, 7)).astype(np.float32)
    dWs, dx = oracle.mlp_bwd(x, Ws, h1, h2, gout)
    dW = torch.zeros(gs3.MLP_PARAMS, device=DEV)
    denc = torch.zeros(n, 32, device=DEV)
    scale = torch.tensor([4.0], device=DEV)
    gs3.ntc_mlp_bwd(t(x), n, mlp, t(gout), scale, dW, denc)
    torch.cuda.synchronize()
    assert_grad_close(dW.cpu().numpy() / 4.0, np.concatenate([w.ravel() for w in dWs]))
    assert_grad_close(denc.cpu().numpy() / 4.0, dx)


@pytest.mark.parametrize("precision", [gs3.GS_MLP_FP32, gs3.GS_MLP_BF16])
@pytest.mark.parametrize("n,frac", [(1, 1.0), (3000, 0.1), (70001, 0.12), (5000, 0.0)])
def test_cache_reverse_over_active_rows(precision, n, frac):
    """ntc_active_rows lists exactly the rows with a nonzero output gradient;
    the MLP reverse and the reverse encoding over that list give the same
    weight, encoding and table gradients as over all rows (rows whose gradient
    is zero add nothing), to the order of the FP32 sums."""
    Ws, rng = _mlp(n + 11)
    og, gg = _grid_pair()
    x = rng.normal(size=(n, 32)).astype(np.float32)
    mu = rng.uniform(-1.4, 1.4, size=(n, 3)).astype(np.float32)
    gout = rng.normal(size=(n, 7)).astype(np.float32)
    gout[rng.uniform(size=n) >= frac] = 0.0
    wflat = t(np.concatenate([w.ravel() for w in Ws]))
    wb = wflat.to(torch.bfloat16)
    mlp = gs3.mlp_struct(precision, wflat, wb if precision == gs3.GS_MLP_BF16 else None)
    xe = t(x).to(torch.bfloat16) if precision == gs3.GS_MLP_BF16 else t(x)
    rows = torch.zeros(n, dtype=torch.int32, device=DEV)
    cnt = torch.zeros(1, dtype=torch.int64, device=DEV)
    gs3.ntc_active_rows(t(gout), n, rows, cnt)
    torch.cuda.synchronize()
    m = int(cnt.item())
    want_rows = np.nonzero(np.any(gout != 0, axis=1))[0]
    assert m == len(want_rows)
    np.testing.assert_array_equal(np.sort(rows[:m].cpu().numpy()), want_rows)
    scale = torch.tensor([8.0], device=DEV)
    out = {}
    for key, kw in (("all", {}), ("listed", {"rows": rows, "d_rows": cnt})):
        dW = torch.zeros(gs3.MLP_PARAMS, device=DEV)
        denc = torch.zeros(n, 32, device=DEV)
        dT = torch.zeros(og.n_entries, 2, device=DEV)
        gs3.ntc_mlp_bwd(xe, n, mlp, t(gout), scale, dW, denc, **kw)
        gs3.ntc_encode_bwd(t(mu), n, gg, denc, dT, order=kw.get("rows"), d_count=kw.get("d_rows"))
        torch.cuda.synchronize()
        out[key] = (dW.cpu().numpy(), denc.cpu().numpy(), dT.cpu().numpy())
    (w0, e0, t0), (w1, e1, t1) = out["all"], out["listed"]
    if m == 0:
        assert not w1.any() and not e1.any() and not t1.any()
        return
    assert rel_err(w1, w0) <= 1e-5
    np.testing.assert_array_equal(e1[want_rows], e0[want_rows])
    assert not e0[np.setdiff1d(np.arange(n), want_rows)].any()
    assert rel_err(t1, t0) <= 1e-5


@pytest.mark.parametrize("order", [0, 1])
def test_apply_parity(order):
    n = 1000
    rng = np.random.default_rng(40 + order)
    aabb = [-1.5] * 3 + [1.5] * 3
    mu = rng.uniform(-1.6, 1.6, size=(n, 3)).astype(np.float32)
    q = rng.normal(size=(n, 4)).astype(np.float32)
    raw = rng.normal(size=(n, 7)).astype(np.float32)
    mo, qo = oracle.apply(mu, q, raw, aabb, order)
    gm, gq = torch.zeros(n, 3, device=DEV), torch.zeros(n, 4, device=DEV)
    gs3.ntc_apply(t(mu), t(q), t(raw), n, aabb, order, gm, gq)
    torch.cuda.synchronize()
    assert np.abs(gm.cpu().numpy() - mo).max() <= 1e-6
    assert np.abs(gq.cpu().numpy() - qo).max() <= 1e-6
    dmo, dqo = rng.normal(size=(n, 3)), rng.normal(size=(n, 4))
    want = oracle.apply_bwd(mu, q, raw, aabb, dmo, dqo, order)
    got = torch.zeros(n, 7, device=DEV)
    gs3.ntc_apply_bwd(t(mu), t(q), t(raw), n, aabb, order, t(dmo), t(dqo), got)
    torch.cuda.synchronize()
    assert_grad_close(got.cpu().numpy(), want, rtol=1e-5)


def test_warmup_loss_parity():
    n = 3000
    raw = np.random.default_rng(50).normal(size=(n, 7)).astype(np.float32)
    L, d = oracle.warmup_loss(raw)
    gd = torch.zeros(n, 7, device=DEV)
    gl = torch.zeros(1, device=DEV)
    gs3.ntc_warmup_loss(t(raw), n, gd, gl)
    torch.cuda.synchronize()
    assert abs(gl.item() - L) <= 1e-5 * max(1, abs(L))
    assert_grad_close(gd.cpu().numpy(), d, rtol=1e-5)


def test_adam_parity_skip_and_shadow():
    n = 10_001  # ragged tail
    rng = np.random.default_rng(60)
    p0 = rng.normal(size=n)
    p, m, v = p0.copy(), np.zeros(n), np.zeros(n)
    gp = t(p0)
    gm, gv = torch.zeros(n, device=DEV), torch.zeros(n, device=DEV)
    sh16 = torch.zeros(n, device=DEV, dtype=torch.float16)
    st = gs3.new_train_state(256.0)
    hp = gs3.GsAdam(0.002, 0.9, 0.99, 1e-15)
    for step in range(1, 6):
        g = rng.normal(size=n).astype(np.float32)
        oracle.adam(p, g.astype(np.float64), m, v, step)
        gg = t(g * 256.0)
        gs3.gs_check_finite(gg, st)
        gs3.adam_step(gp, gg, gm, gv, hp, st, sh16)
        gs3.gs_train_state_advance(st, 0)
        torch.cuda.synchronize()
        assert not gg.any()  # gradient consumed and zeroed
    np.testing.assert_allclose(gp.cpu().numpy(), p, rtol=1e-5, atol=1e-6)
    np.testing.assert_array_equal(sh16.cpu().numpy(), gp.cpu().numpy().astype(np.float16))
    # a non-finite gradient skips the update and halves the scale
    before = gp.clone()
    bad = torch.ones(n, device=DEV)
    bad[17] = float("inf")
    gs3.gs_check_finite(bad, st)
    gs3.adam_step(gp, bad, gm, gv, hp, st)
    gs3.gs_train_state_advance(st, 0)
    s = gs3.read_train_state(st)
    assert torch.equal(gp, before)
    assert s.loss_scale == 128.0 and s.found_inf == 0 and s.step == 5


@pytest.mark.parametrize("n", [1, 7, 4099, 70001])
def test_check_finite_sees_every_position(n):
    """gs_check_finite flags a non-finite value wherever it is: the vector
    body, the scalar tail, the last block; a finite array leaves the flag."""
    st = gs3.new_train_state(1.0)
    g = torch.ones(n, device=DEV)
    gs3.gs_check_finite(g, st)
    assert gs3.read_train_state(st).found_inf == 0
    for pos in sorted({0, n // 2, n - 1, max(0, n - 5)}):
        for bad in (float("nan"), float("inf"), -float("inf")):
            st = gs3.new_train_state(1.0)
            g = torch.ones(n, device=DEV)
            g[pos] = bad
            gs3.gs_check_finite(g, st)
            assert gs3.read_train_state(st).found_inf == 1, (n, pos, bad)


def test_adam_rate_schedule():
    """The rate decays exponentially from lr to lr * ratio over decay_steps
    applied updates and stays there; a skipped update does not advance it."""
    n = 4099
    rng = np.random.default_rng(61)
    p0 = rng.normal(size=n)
    p, m, v = p0.copy(), np.zeros(n), np.zeros(n)
    gp = t(p0)
    gm, gv = torch.zeros(n, device=DEV), torch.zeros(n, device=DEV)
    st = gs3.new_train_state(1.0)
    hp = gs3.GsAdam(0.01, 0.9, 0.99, 1e-6, 0.05, 4)
    applied, scale = 0, 1.0
    for k in range(7):
        g = rng.normal(size=n).astype(np.float32)
        gg = t(g * scale)          # scaled by the current loss scale
        if k == 2:
            gg[5] = float("inf")   # skipped: the schedule does not move, the scale halves
            scale *= 0.5
        gs3.gs_check_finite(gg, st)
        gs3.adam_step(gp, gg, gm, gv, hp, st)
        gs3.gs_train_state_advance(st, 0)
        if k != 2:
            lr = oracle.adam_rate(0.01, 0.05, 4, applied)
            applied += 1
            oracle.adam(p, g.astype(np.float64), m, v, applied, lr=lr, eps=1e-6)
    torch.cuda.synchronize()
    assert gs3.read_train_state(st).step == applied == 6
    np.testing.assert_allclose(gp.cpu().numpy(), p, rtol=1e-5, atol=1e-6)
    assert oracle.adam_rate(0.01, 0.05, 4, 3) == pytest.approx(0.0005)
    assert oracle.adam_rate(0.01, 0.05, 4, 9) == pytest.approx(0.0005)


def _bf16(a):
    return torch.from_numpy(np.ascontiguousarray(a, np.float32)).to(torch.bfloat16).float().numpy()


def _run_bf16_mlp(x, Wb, gout, scale_value):
    n = x.shape[0]
    wflat = np.concatenate([w.ravel() for w in Wb]).astype(np.float32)
    w32 = t(wflat)
    wbf = w32.to(torch.bfloat16)
    mlp = gs3.mlp_struct(gs3.GS_MLP_BF16, w32, wbf)
    xb = t(x).to(torch.bfloat16)
    raw = torch.full((n, 7), float("nan"), device=DEV)
    gs3.ntc_mlp_fwd(xb, n, mlp, raw)
    dW = torch.zeros(gs3.MLP_PARAMS, device=DEV)
    denc = torch.full((n, 32), float("nan"), device=DEV)
    scale = torch.tensor([scale_value], device=DEV)
    gs3.ntc_mlp_bwd(xb, n, mlp, t(gout), scale, dW, denc)
    torch.cuda.synchronize()
    assert gs3.lib().gs_tc_timeouts() == 0
    return raw.cpu().numpy(), dW.cpu().numpy() / scale_value, denc.cpu().numpy() / scale_value


@pytest.mark.parametrize("n", [1, 127, 128, 129, 5000])
def test_mlp_bf16_tensor_core_exact_on_integers(n):
    """Integer-valued encodings, weights and output gradients keep every
    intermediate (activations, BF16 roundings, FP32 sums) exact, so the
    tcgen05 path must equal the FP64 oracle bit for bit: any layout, transpose
    or accumulation slip shows here."""
    rng = np.random.default_rng(2000 + n)
    sparse = lambda shape, p: (rng.integers(-1, 2, size=shape) * (rng.uniform(size=shape) < p)).astype(np.float64)
    x = sparse((n, 32), 0.6)
    Wb = [sparse((64, 32), 0.3), sparse((64, 64), 0.1), sparse((7, 64), 0.3)]
    gout = sparse((n, 7), 0.8)
    h1, h2, out = oracle.mlp_fwd(x, Wb)
    dWs, dx = oracle.mlp_bwd(x, Wb, h1, h2, gout)
    assert np.abs(h2).max() < 256 and np.abs(dx).max() < 256
    raw, dW, denc = _run_bf16_mlp(x, Wb, gout, 1024.0)
    np.testing.assert_array_equal(raw, out)
    np.testing.assert_array_equal(dW, np.concatenate([w.ravel() for w in dWs]))
    np.testing.assert_array_equal(denc, dx)


@pytest.mark.parametrize("n", [1, 128, 300, 20_000])
def test_mlp_bf16_tensor_core_parity(n):
    """Random inputs: the kernel also rounds hidden activations and gradients
    to BF16 between layers (relative 2^-9 each).  Forward outputs stay within
    1e-2; weight and input gradients within 5e-2 per tensor, the size a BF16
    emulation of the same rounding points gives on these N(0,1) inputs (it
    comes from cancellation in dH1 = dH2 W2 and from ReLU masks flipping on
    the ~0.05% of units whose pre-activation lies within BF16 reach of 0)."""
    Ws, rng = _mlp(1000 + n)
    Wb = [_bf16(w) for w in Ws]
    x = _bf16(rng.normal(size=(n, 32)))
    gout = rng.normal(size=(n, 7)).astype(np.float32)
    h1, h2, out = oracle.mlp_fwd(x, Wb)
    dWs, dx = oracle.mlp_bwd(x, Wb, h1, h2, gout)
    got, gW, gd = _run_bf16_mlp(x, Wb, gout, 1024.0)
    assert np.isfinite(got).all() and np.isfinite(gd).all()
    assert rel_err(got, out) <= 1e-2
    assert np.abs(got - out).max() <= 2e-2 * max(np.abs(out).max(), 1e-6)
    wantW = np.concatenate([w.ravel() for w in dWs])
    for sl in (slice(0, 2048), slice(2048, 6144), slice(6144, 6592)):
        assert rel_err(gW[sl], wantW[sl]) <= 5e-2, sl
    assert rel_err(gd, dx) <= 5e-2


@pytest.mark.parametrize("n", [1, 300, 20_001])
def test_fused_cache_kernels_match_separate_kernels(n):
    """ntc_fused_fwd = encode (FP16 table) + BF16 MLP + apply, bit for bit;
    ntc_fused_bwd = apply_bwd + MLP bwd + encode_bwd up to the order of the
    FP32 atomic additions."""
    og, gg = _grid_pair()
    rng = np.random.default_rng(3000 + n)
    aabb = [-1.5] * 3 + [1.5] * 3
    mu = t(rng.uniform(-1.6, 1.6, size=(n, 3)))   # a few outside the box
    q = t(rng.normal(size=(n, 4)))
    table = t(rng.normal(0, 0.3, size=(og.n_entries, 2))).to(torch.float16)
    Ws, _ = _mlp(3100 + n)
    w32 = t(np.concatenate([w.ravel() for w in Ws]))
    wbf = w32.to(torch.bfloat16)
    mlp = gs3.mlp_struct(gs3.GS_MLP_BF16, w32, wbf)
    # separate kernels
    enc = torch.zeros(n, 32, device=DEV, dtype=torch.bfloat16)
    raw = torch.zeros(n, 7, device=DEV)
    mo, qo = torch.zeros(n, 3, device=DEV), torch.zeros(n, 4, device=DEV)
    gs3.ntc_encode_fwd(mu, n, gg, table, enc)
    gs3.ntc_mlp_fwd(enc, n, mlp, raw)
    gs3.ntc_apply(mu, q, raw, n, aabb, 0, mo, qo)
    # fused
    enc2 = torch.zeros_like(enc)
    raw2, mo2, qo2 = torch.zeros_like(raw), torch.zeros_like(mo), torch.zeros_like(qo)
    gs3.ntc_fused_fwd(mu, q, n, gg, table, mlp, 0, mo2, qo2, raw2, enc2)
    torch.cuda.synchronize()
    assert torch.equal(enc2, enc) and torch.equal(raw2, raw)
    assert torch.equal(mo2, mo) and torch.equal(qo2, qo)
    dmo, dqo = t(rng.normal(size=(n, 3))), t(rng.normal(size=(n, 4)))
    scale = torch.tensor([64.0], device=DEV)
    d_raw = torch.zeros(n, 7, device=DEV)
    dW, d_enc = torch.zeros(gs3.MLP_PARAMS, device=DEV), torch.zeros(n, 32, device=DEV)
    dT = torch.zeros(og.n_entries, 2, device=DEV)
    gs3.ntc_apply_bwd(mu, q, raw, n, aabb, 0, dmo, dqo, d_raw)
    gs3.ntc_mlp_bwd(enc, n, mlp, d_raw, scale, dW, d_enc)
    gs3.ntc_encode_bwd(mu, n, gg, d_enc, dT)
    dW2, dT2 = torch.zeros_like(dW), torch.zeros_like(dT)
    gs3.ntc_fused_bwd(mu, q, raw2, enc2, n, gg, mlp, 0, dmo, dqo, scale, dW2, dT2)
    torch.cuda.synchronize()
    assert rel_err(dW2.cpu().numpy(), dW.cpu().numpy()) <= 1e-5
    assert rel_err(dT2.cpu().numpy(), dT.cpu().numpy()) <= 1e-5
    # and the fused forward against the FP64 oracle on the same FP16 / BF16 values
    want_enc = oracle.encode(og, mu.cpu().numpy(), table.float().cpu().numpy())
    got_enc = enc2.float().cpu().numpy()
    assert np.all(np.abs(got_enc - want_enc) <= 2 ** -8 * np.abs(want_enc) + 1e-3 * 0.3 * 5)
    Wb = [_bf16(w) for w in Ws]
    _, _, want_raw = oracle.mlp_fwd(got_enc, Wb)
    assert rel_err(raw2.cpu().numpy(), want_raw) <= 1e-2


@pytest.mark.parametrize("deg", [1, 2, 3])
def test_sh_rotate_matches_oracle(deg):
    """gs_sh_rotate (fixed directions, A^-1 in the kernel) against the
    oracle's least-squares definition, in place and out of place."""
    from scipy.spatial.transform import Rotation
    rng = np.random.default_rng(70 + deg)
    n, K = 3000, (deg + 1) ** 2
    sh = rng.normal(size=(n, K, 3)).astype(np.float32)
    qa = rng.normal(size=(n, 4)).astype(np.float32)
    qb = rng.normal(size=(n, 4)).astype(np.float32) * 2.0   # not unit on purpose
    want = oracle.sh_rotate(sh[:400], qa[:400], qb[:400], deg)
    t = lambda a: torch.from_numpy(np.ascontiguousarray(a)).to(DEV)
    out = torch.empty(n, K, 3, device=DEV)
    gs3.gs_sh_rotate(t(qa), t(qb), t(sh), n, deg, out)
    inplace = t(sh)
    gs3.gs_sh_rotate(t(qa), t(qb), inplace, n, deg, inplace)
    torch.cuda.synchronize()
    got = out.cpu().numpy()
    np.testing.assert_allclose(got[:400], want, rtol=0, atol=2e-5 * np.abs(sh).max() * K)
    assert torch.equal(out, inplace)
    # band energies preserved over all n (orthonormal basis)
    for lo, hi in ((1, 4), (4, 9), (9, 16))[:deg]:
        np.testing.assert_allclose(np.linalg.norm(got[:, lo:hi], axis=1),
                                   np.linalg.norm(sh[:, lo:hi], axis=1), rtol=1e-4, atol=1e-5)

