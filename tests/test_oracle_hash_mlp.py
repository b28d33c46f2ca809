"""Pins of the oracle's hash encoding, MLP, transformation and warm-up loss
(Section 4.1, Eq. 5 and Eq. 7) against invariants, library routines and
finite differences -- none of them re-derives the oracle's own formula."""
import numpy as np
import pytest

import oracle

def _grid_unit(L=2, Nmin=16, Nmax=32, log2T=10, F=2):
    # box [0,1]^3 and power-of-two resolutions make vertex positions exact
    return oracle.Grid(L=L, F=F, log2T=log2T, Nmin=Nmin, Nmax=Nmax, aabb=(0, 0, 0, 1, 1, 1))


def test_level_resolutions_geometric():
    g = oracle.Grid()
    assert g.res[0] == 16 and g.res[-1] == 1024
    b = (1024 / 16) ** (1 / 15)
    for l in range(16):
        assert abs(g.res[l] - 16 * b ** l) < 1.0
    # the dense/hashed switch: dense exactly when (N+1)^3 fits in T = 2^17
    assert list(g.dense) == [int((n + 1) ** 3 <= 2 ** 17) for n in g.res]
    sizes = [min(2 ** 17, (n + 1) ** 3) for n in g.res]
    assert g.n_entries == sum(sizes)
    assert list(g.offset) == list(np.cumsum([0] + sizes[:-1]))


def test_hash_corners_worked_examples():
    """I-NGP's spatial hash (x*1 xor y*2654435761 xor z*805459861) mod 2^32,
    then mod T = 2^17, worked out in hexadecimal:
      y*0x9E3779B1, z*0x30025795 (mod 2^32), xor, keep the low 17 bits."""
    cases = [
        ((1, 0, 0), 0x1),                       # -> 1
        ((0, 1, 0), 0x9E3779B1 & 0x1FFFF),      # -> 96689
        ((0, 0, 1), 0x30025795 & 0x1FFFF),      # -> 22421
        ((1, 1, 1), 0xAE352E25 & 0x1FFFF),      # 1 ^ 0x9E3779B1 ^ 0x30025795
        ((2, 3, 5), 0x2AADD8F8 & 0x1FFFF),      # 2 ^ 0xDAA66D13 ^ 0xF00BB5E9
        ((1023, 517, 1024), 0x8F56958A & 0x1FFFF),
    ]
    want = [1, 96689, 22421, 77349, 121080, 38282]
    for ((x, y, z), v), w in zip(cases, want):
        assert v == w
        assert oracle.corner_index(100, 0, 17, x, y, z) == w, (x, y, z)


def test_dense_index_bijection():
    n = 7
    idx = {oracle.corner_index(n, 1, 17, x, y, z)
           for x in range(n + 1) for y in range(n + 1) for z in range(n + 1)}
    assert idx == set(range((n + 1) ** 3))


@pytest.mark.parametrize("level", [0, 1])
def test_encoding_at_vertex_equals_entry(level):
    rng = np.random.default_rng(0)
    g = _grid_unit()
    g16 = oracle.Grid(L=2, F=2, log2T=10, Nmin=16, Nmax=32, aabb=(0, 0, 0, 1, 1, 1))
    assert list(g16.res) == [16, 32]
    # level 0: 17^3 = 4913 > 1024 -> hashed; use log2T=13 for a dense level 0
    for log2T in (10, 13):
        g = oracle.Grid(L=2, F=2, log2T=log2T, Nmin=16, Nmax=32, aabb=(0, 0, 0, 1, 1, 1))
        table = rng.normal(size=(g.n_entries, 2))
        n = int(g.res[level])
        for _ in range(20):
            v = rng.integers(0, n, size=3)  # vertex strictly inside (c clamps at n-1)
            mu = (v / n)[None, :]
            enc = oracle.encode(g, mu, table)
            e = g.offset[level] + oracle.corner_index(n, int(g.dense[level]), log2T, *map(int, v))
            np.testing.assert_allclose(enc[0, 2 * level:2 * level + 2], table[e], rtol=0, atol=1e-12)


def test_partition_of_unity():
    rng = np.random.default_rng(1)
    g = oracle.Grid()
    table = np.ones((g.n_entries, 2)) * np.array([0.25, -2.0])
    mu = rng.uniform(-1.5, 1.5, size=(200, 3))
    enc = oracle.encode(g, mu, table)
    np.testing.assert_allclose(enc[:, 0::2], 0.25, atol=1e-12)
    np.testing.assert_allclose(enc[:, 1::2], -2.0, atol=1e-12)


@pytest.mark.parametrize("axis", [0, 1, 2])
def test_linear_along_each_axis_within_a_cell(axis):
    rng = np.random.default_rng(2 + axis)
    g = oracle.Grid()
    table = rng.normal(size=(g.n_entries, 2))
    for _ in range(10):
        base = rng.uniform(-1.4, 1.4, size=3)
        # stay inside one cell of the finest level: step of 1e-5 of the box
        a = base.copy()
        b = base.copy()
        b[axis] += 3.0 * 1e-5
        m = 0.5 * (a + b)
        e = oracle.encode(g, np.stack([a, b, m]), table)
        np.testing.assert_allclose(e[2], 0.5 * (e[0] + e[1]), atol=1e-9)
        # ... but not linear across an axis orthogonal move mixed with this one
    # weights along an axis are affine: f(a + t d) = (1-t) f(a) + t f(a+d)
    n = 16
    g1 = _grid_unit(L=1, Nmin=n, Nmax=n, log2T=14)
    t1 = rng.normal(size=(g1.n_entries, 2))
    p0 = np.array([3 / n, 5 / n, 7 / n])
    p1 = p0.copy()
    p1[axis] += 1 / n
    ts = np.linspace(0, 1, 7)[1:-1]
    pts = np.array([p0 + t * (p1 - p0) for t in ts])
    e = oracle.encode(g1, np.concatenate([p0[None], p1[None] - [0, 0, 0], pts]), t1)
    # p1 is a vertex of the next cell: its value is the table entry there
    for k, t in enumerate(ts):
        np.testing.assert_allclose(e[2 + k], (1 - t) * e[0] + t * e[1], atol=1e-12)


def test_encode_bwd_is_adjoint():
    rng = np.random.default_rng(3)
    g = oracle.Grid()
    mu = rng.uniform(-1.5, 1.5, size=(300, 3))
    table = rng.normal(size=(g.n_entries, 2))
    d_enc = rng.normal(size=(300, 32))
    lhs = np.sum(oracle.encode(g, mu, table) * d_enc)
    rhs = np.sum(table * oracle.encode_bwd(g, mu, d_enc))
    assert abs(lhs - rhs) <= 1e-9 * max(1.0, abs(lhs))


def test_mlp_fwd_matches_numpy():
    rng = np.random.default_rng(4)
    Ws = [rng.normal(size=(64, 32)), rng.normal(size=(64, 64)) / 8, rng.normal(size=(7, 64)) / 8]
    x = rng.normal(size=(50, 32))
    h1, h2, out = oracle.mlp_fwd(x, Ws)
    r1 = np.maximum(x @ Ws[0].T, 0)
    r2 = np.maximum(r1 @ Ws[1].T, 0)
    np.testing.assert_allclose(h1, r1, rtol=1e-12, atol=1e-12)
    np.testing.assert_allclose(h2, r2, rtol=1e-12, atol=1e-12)
    np.testing.assert_allclose(out, r2 @ Ws[2].T, rtol=1e-12, atol=1e-12)


def test_mlp_bwd_matches_torch_autograd():
    torch = pytest.importorskip("torch")
    rng = np.random.default_rng(5)
    Ws = [rng.normal(size=(64, 32)), rng.normal(size=(64, 64)) / 8, rng.normal(size=(7, 64)) / 8]
    x = rng.normal(size=(40, 32))
    gout = rng.normal(size=(40, 7))
    h1, h2, _ = oracle.mlp_fwd(x, Ws)
    dWs, dx = oracle.mlp_bwd(x, Ws, h1, h2, gout)
    tx = torch.tensor(x, requires_grad=True)
    tW = [torch.tensor(w, requires_grad=True) for w in Ws]
    y = torch.relu(torch.relu(tx @ tW[0].T) @ tW[1].T) @ tW[2].T
    (y * torch.tensor(gout)).sum().backward()
    np.testing.assert_allclose(dx, tx.grad.numpy(), rtol=1e-10, atol=1e-10)
    for a, b in zip(dWs, tW):
        np.testing.assert_allclose(a, b.grad.numpy(), rtol=1e-10, atol=1e-10)


def _rot(q):
    from scipy.spatial.transform import Rotation
    q = np.asarray(q, np.float64)
    return Rotation.from_quat(q[[1, 2, 3, 0]] / np.linalg.norm(q)).as_matrix()


def test_qmul_composes_rotations():
    rng = np.random.default_rng(6)
    for _ in range(20):
        a, b = rng.normal(size=4), rng.normal(size=4)
        a /= np.linalg.norm(a)
        b /= np.linalg.norm(b)
        np.testing.assert_allclose(_rot(oracle.qmul(a, b)), _rot(a) @ _rot(b), atol=1e-12)
    # Hamilton unit: i*j = k
    np.testing.assert_allclose(oracle.qmul([0, 1, 0, 0], [0, 0, 1, 0]), [0, 0, 0, 1])


def test_apply_identity_and_unit_norm():
    rng = np.random.default_rng(7)
    aabb = [-1.5, -1.5, -1.5, 1.5, 1.5, 1.5]
    mu = rng.uniform(-1, 1, size=(30, 3))
    q = rng.normal(size=(30, 4))
    raw = np.zeros((30, 7))
    raw[:, 3] = 2.5  # dq = (2.5, 0, 0, 0): identity after normalisation
    mo, qo = oracle.apply(mu, q, raw, aabb)
    np.testing.assert_array_equal(mo, mu)
    np.testing.assert_allclose(qo, q / np.linalg.norm(q, axis=1, keepdims=True), atol=1e-15)
    raw = rng.normal(size=(30, 7))
    for order in (0, 1):
        mo, qo = oracle.apply(mu, q, raw, aabb, order)
        np.testing.assert_allclose(mo, mu + raw[:, :3], atol=1e-15)
        np.testing.assert_allclose(np.linalg.norm(qo, axis=1), 1.0, atol=1e-14)
        for i in range(30):
            Rq, Rd = _rot(q[i]), _rot(raw[i, 3:])
            want = Rq @ Rd if order == 0 else Rd @ Rq
            np.testing.assert_allclose(_rot(qo[i]), want, atol=1e-12)
    # outside the box: mean kept, rotation only normalised
    mu_out = mu.copy()
    mu_out[0] = [2.0, 0, 0]
    mo, qo = oracle.apply(mu_out, q, raw, aabb)
    np.testing.assert_array_equal(mo[0], mu_out[0])
    np.testing.assert_allclose(qo[0], q[0] / np.linalg.norm(q[0]), atol=1e-15)


@pytest.mark.parametrize("order", [0, 1])
def test_apply_bwd_finite_differences(order):
    rng = np.random.default_rng(8 + order)
    aabb = [-1.5, -1.5, -1.5, 1.5, 1.5, 1.5]
    N = 6
    mu = rng.uniform(-1, 1, size=(N, 3))
    q = rng.normal(size=(N, 4))
    raw = rng.normal(size=(N, 7))
    gm, gq = rng.normal(size=(N, 3)), rng.normal(size=(N, 4))

    def f(r):
        mo, qo = oracle.apply(mu, q, r, aabb, order)
        return np.sum(mo * gm) + np.sum(qo * gq)

    d = oracle.apply_bwd(mu, q, raw, aabb, gm, gq, order)
    h = 1e-6
    fd = np.zeros_like(raw)
    for i in range(N):
        for k in range(7):
            rp, rm = raw.copy(), raw.copy()
            rp[i, k] += h
            rm[i, k] -= h
            fd[i, k] = (f(rp) - f(rm)) / (2 * h)
    np.testing.assert_allclose(d, fd, rtol=1e-6, atol=1e-8)


def test_warmup_loss_minimum_and_gradient():
    rng = np.random.default_rng(9)
    raw = np.zeros((5, 7))
    raw[:, 3] = rng.uniform(0.5, 2, size=5) * rng.choice([-1, 1], size=5)
    L, d = oracle.warmup_loss(raw)
    assert abs(L - (-1.0)) < 1e-15  # identity translation and rotation: the minimum
    raw = rng.normal(size=(8, 7))
    L1, _ = oracle.warmup_loss(raw)
    neg = raw.copy()
    neg[:, 3:] *= -1  # double cover: q and -q are the same rotation
    assert abs(oracle.warmup_loss(neg)[0] - L1) < 1e-14
    _, d = oracle.warmup_loss(raw)
    h = 1e-6
    for i in range(8):
        for k in range(7):
            rp, rm = raw.copy(), raw.copy()
            rp[i, k] += h
            rm[i, k] -= h
            fd = (oracle.warmup_loss(rp)[0] - oracle.warmup_loss(rm)[0]) / (2 * h)
            assert abs(fd - d[i, k]) < 1e-7
