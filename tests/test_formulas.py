"""Identities the CUDA kernels rely on where they reorganise the arithmetic
of the method, checked in FP64 against the plain form (no GPU, no shared code
with either side):

  * the 2D-covariance determinant as a sum of non-negative terms
    (Cauchy-Binet), used by the projection (Section 3.2, Eq. 3);
  * the reverse compositing pass carrying the scalar dC . B instead of the
    colour behind B (Eq. 4);
  * the packed row filter of the SSIM loss (Eq. 6): tap pairs times input
    pairs equal the plain 11-tap Gaussian window.
"""
import numpy as np


def test_cauchy_binet_determinant_of_the_dilated_footprint():
    """det(P P^T + 0.3 I) = sum of the squared 2x2 minors of P
    + 0.3 (|P_0|^2 + |P_1|^2) + 0.09 for any 2x3 P; for a needle (P close to
    rank one) a c - b^2 cancels while the sum does not."""
    rng = np.random.default_rng(0)
    for _ in range(200):
        P = rng.normal(size=(2, 3)) * rng.uniform(0.01, 100.0)
        S = P @ P.T + 0.3 * np.eye(2)
        m01 = P[0, 0] * P[1, 1] - P[0, 1] * P[1, 0]
        m02 = P[0, 0] * P[1, 2] - P[0, 2] * P[1, 0]
        m12 = P[0, 1] * P[1, 2] - P[0, 2] * P[1, 1]
        cb = m01 ** 2 + m02 ** 2 + m12 ** 2 + 0.3 * (P[0] @ P[0] + P[1] @ P[1]) + 0.09
        assert abs(cb - np.linalg.det(S)) <= 1e-12 * abs(cb)
    # a needle: long axis 500 px along (1, 1), the others 1e-5 px
    u = np.array([1.0, 1.0, 0.0]) / np.sqrt(2)
    v = np.array([1.0, -1.0, 0.0]) / np.sqrt(2)
    w = np.array([0.0, 0.0, 1.0])
    M = np.stack([500.0 * u, 1e-5 * v, 1e-5 * w], 1)          # R diag(s)
    T = np.array([[1.0, 0.0, 0.0], [0.0, 1.0, 0.0]])
    P = (T @ M).astype(np.float32)
    a, b, c = (np.float32(x) for x in (P[0] @ P[0] + 0.3, P[0] @ P[1], P[1] @ P[1] + 0.3))
    naive = np.float32(a * c - b * b)
    P64 = P.astype(np.float64)
    exact = np.linalg.det(P64 @ P64.T + 0.3 * np.eye(2))
    m = [P[0, i] * P[1, j] - P[0, j] * P[1, i] for i, j in ((0, 1), (0, 2), (1, 2))]
    cb32 = np.float32(sum(np.float32(x) ** 2 for x in m)
                      + np.float32(0.3) * (P[0] @ P[0] + P[1] @ P[1]) + np.float32(0.09))
    assert abs(naive - exact) > 0.01 * exact          # FP32 a c - b^2 is off by > 1 %
    assert abs(cb32 - exact) <= 1e-5 * exact          # the sum keeps FP32 accuracy


def test_reverse_pass_scalar_colour_behind():
    """Back to front over one pixel's contributors, dL/dalpha_i from the colour
    behind B (three channels) equals dL/dalpha_i from S = dC . B alone."""
    rng = np.random.default_rng(1)
    for _ in range(50):
        n = rng.integers(1, 40)
        alpha = rng.uniform(0.004, 0.99, n)
        col = rng.uniform(0.0, 1.0, (n, 3))
        bg = rng.uniform(0.0, 1.0, 3)
        dC = rng.normal(size=3)
        T_final = np.prod(1.0 - alpha)
        # three channels
        T, B, da3 = T_final, bg.copy(), np.zeros(n)
        for i in range(n - 1, -1, -1):
            T = T / (1.0 - alpha[i])
            da3[i] = T * (dC @ (col[i] - B))
            B = alpha[i] * col[i] + (1.0 - alpha[i]) * B
        # the scalar
        T, S, da1 = T_final, dC @ bg, np.zeros(n)
        for i in range(n - 1, -1, -1):
            T = T / (1.0 - alpha[i])
            diff = dC @ col[i] - S
            da1[i] = T * diff
            S = S + alpha[i] * diff
        np.testing.assert_allclose(da1, da3, rtol=1e-10, atol=1e-12)
        # and both are the derivative of the composited colour (central differences)
        def comp(a):
            C, Tr = np.zeros(3), 1.0
            for i in range(n):
                C += col[i] * a[i] * Tr
                Tr *= 1.0 - a[i]
            return dC @ (C + Tr * bg)
        for i in rng.choice(n, size=min(n, 3), replace=False):
            h = 1e-6
            ap, am = alpha.copy(), alpha.copy()
            ap[i] += h
            am[i] -= h
            assert abs((comp(ap) - comp(am)) / (2 * h) - da1[i]) <= 1e-6 * max(1.0, abs(da1[i]))


def _window():
    w = np.exp(-((np.arange(11) - 5) ** 2) / 4.5)
    return w / w.sum()


def test_packed_row_filter_equals_the_11_tap_window():
    """An item's four outputs at columns B + 8 + o (o = 0..3) from the input
    pairs (in_2k, in_2k+1): even o with the shifted tap pairs (w_2i-1, w_2i),
    w_-1 = 0, odd o with (w_2i, w_2i+1) plus the last tap -- the same sums as
    the plain window over in_3+o .. in_13+o."""
    w = _window()
    e = [(w[2 * i], w[2 * i + 1]) for i in range(5)]
    od = [(0.0, w[0])] + [(w[2 * i - 1], w[2 * i]) for i in range(1, 6)]
    rng = np.random.default_rng(2)
    for _ in range(100):
        x = rng.normal(size=18)                         # in_0 .. in_17
        pairs = x.reshape(9, 2)
        for o in range(4):
            if o % 2 == 0:
                got = sum(od[i][0] * pairs[1 + o // 2 + i][0] + od[i][1] * pairs[1 + o // 2 + i][1]
                          for i in range(6))
            else:
                k0 = 2 + (o - 1) // 2                   # pairs from in_3+o
                got = sum(e[i][0] * pairs[k0 + i][0] + e[i][1] * pairs[k0 + i][1]
                          for i in range(5)) + w[10] * x[14 + (o - 1)]
            want = sum(w[t] * x[3 + o + t] for t in range(11))
            assert abs(got - want) <= 1e-14 * max(1.0, abs(want))
