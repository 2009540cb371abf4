"""Pins of oracle.fields: the filter's spectrum, the exact covariance identity,
the sample covariance of many seeds, and bilinear interpolation."""
import numpy as np
import pytest

from oracle import fields, noll


def test_spectrum_is_poisson_sum_of_gaussian():
    # DFT of a Gaussian wrapped on a torus = sampled Gaussian spectrum, itself wrapped
    # (Poisson summation): C1[u] = sqrt(2 pi) (l/s) sum_m exp(-2 pi^2 (l/s)^2 (u/F + m)^2).
    for fh, fw, ell, s in [(16, 32, 6.0, 4), (64, 64, 16.0, 8), (8, 16, 3.0, 1)]:
        g = fields.filter_gain(fh, fw, ell, s)
        def c1(F):
            u = np.arange(F)[:, None] / F + np.arange(-30, 31)[None, :]
            a = ell / s
            return np.sqrt(2 * np.pi) * a * np.exp(-2 * np.pi**2 * a * a * u**2).sum(axis=1)
        ref = np.outer(c1(fh), c1(fw))
        assert np.max(np.abs(g**2 - ref)) < 1e-12 * ref.max()


def test_exact_covariance_of_filter_operator():
    fh, fw, ell, s = 8, 16, 5.0, 2
    g = fields.filter_gain(fh, fw, ell, s)
    n = fh * fw
    G = np.empty((n, n))
    for k in range(n):
        e = np.zeros(n)
        e[k] = 1.0
        G[:, k] = fields.filter_field(e.reshape(fh, fw), g).reshape(-1)
    cov = G @ G.T  # covariance of f = G w for unit white w
    c = fields.kernel_covariance(fh, fw, ell, s)
    yy, xx = np.meshgrid(np.arange(fh), np.arange(fw), indexing="ij")
    yy, xx = yy.reshape(-1), xx.reshape(-1)
    pred = c[(yy[None, :] - yy[:, None]) % fh, (xx[None, :] - xx[:, None]) % fw]
    assert np.max(np.abs(cov - pred)) < 1e-13
    # on a torus much longer than ell the wrapped images vanish: unit variance, Gaussian lags
    c = fields.kernel_covariance(64, 32, 5.0, 2)
    assert abs(c[0, 0] - 1.0) < 1e-14
    assert abs(c[1, 3] - np.exp(-(1 + 9) * 4 / 50.0)) < 1e-14


def test_anchor_and_torus_geometry():
    p = fields.CorrParams(anchor_spacing=8, corr_len_px=(16.0,))
    assert fields.anchor_shape(512, 512, 8) == (65, 65)
    assert p.guard() == 6
    assert fields.torus_shape(512, 512, p) == (128, 128)
    assert fields.anchor_shape(64, 64, 1) == (65, 65)
    assert fields.anchor_shape(1152, 2048, 8) == (145, 257)


def test_sample_covariance_matches_construction():
    p = fields.CorrParams(anchor_spacing=4, corr_len_px=(6.0,))
    h = w = 24
    fh, fw = fields.torus_shape(h, w, p)
    L = noll.cholesky_lower(noll.noll_cov(36))
    n = 2000
    dr0 = 1.7
    a0, a1 = (2, 2), (2, 3)
    s0 = np.empty((n, 35))
    s1 = np.empty((n, 35))
    for i in range(n):
        al = fields.alpha_anchors(10_000 + i, dr0, h, w, p, L)
        s0[i], s1[i] = al[a0], al[a1]
    for d, other in [((0, 0), s0), ((0, 1), s1)]:
        pred = fields.anchor_cross_covariance(d, fh, fw, p, L, dr0)
        emp = s0.T @ other / n
        v0 = fields.anchor_cross_covariance((0, 0), fh, fw, p, L, dr0)
        var = (np.outer(np.diag(v0), np.diag(v0)) + pred**2) / n  # Wishart variance of each entry
        z = np.abs(emp - pred) / np.sqrt(var)
        assert z.max() < 5.5, (d, z.max())


def test_multi_kernel_construction():
    # one kernel per radial order: Cov(alpha_i, alpha_j)(d) = sum_l L_il L_jl c_n(l)[d]
    p = fields.CorrParams(anchor_spacing=2, corr_len_px=(8.0, 7.0, 6.0, 5.0, 4.0, 3.0, 2.0))
    L = noll.cholesky_lower(noll.noll_cov(36))
    fh, fw = fields.torus_shape(16, 16, p)
    c0 = fields.anchor_cross_covariance((0, 0), fh, fw, p, L, 1.0)
    assert np.allclose(c0, noll.noll_cov(36), atol=1e-12)  # every kernel has unit variance
    c1 = fields.anchor_cross_covariance((0, 1), fh, fw, p, L, 1.0)
    # alpha_2 = L_00 f_0 uses the radial-order-1 kernel only: lag of one anchor = s px
    assert abs(c1[0, 0] / c0[0, 0] - np.exp(-4 / (2 * 64.0))) < 1e-12
    assert c1[34, 34] / c0[34, 34] < c1[0, 0] / c0[0, 0]


def test_bilinear_interpolation():
    rng = np.random.default_rng(1)
    s = 4
    aa = rng.normal(size=(5, 6, 3))
    ap = fields.alpha_pixels(aa, 16, 20, s)
    assert np.allclose(ap[::s, ::s], aa[:4, :5])
    assert np.allclose(ap[2, 0], 0.5 * (aa[0, 0] + aa[1, 0]))
    assert np.allclose(ap[1, 3], (3 / 4) * ((1 / 4) * aa[0, 0] + (3 / 4) * aa[0, 1]) + (1 / 4) * ((1 / 4) * aa[1, 0] + (3 / 4) * aa[1, 1]))


def test_dense_draw_equals_explicit_cholesky_of_the_full_matrix():
    """The separable evaluation L_y W L_x^T is the draw chol(Sigma) vec(W) of the full
    A_h A_w x A_h A_w anchor correlation matrix (built and factored explicitly here)."""
    from oracle import fields, philox

    p = fields.CorrParams(8, (16.0,))
    h, w = 33, 41  # 6 x 7 anchors
    ah, aw = fields.anchor_shape(h, w, 8)
    ys, xs = np.meshgrid(np.arange(ah), np.arange(aw), indexing="ij")
    pts = np.stack([ys.ravel(), xs.ravel()], axis=1) * 8.0
    d2 = ((pts[:, None, :] - pts[None, :, :]) ** 2).sum(-1)
    S = np.exp(-d2 / (2 * 16.0 ** 2))
    Lfull = np.linalg.cholesky(S)
    f = fields.dense_fields(99, h, w, p)
    for l in (0, 17, 34):
        wn = philox.normals(99, l, ah * aw)
        np.testing.assert_allclose(f[:, :, l].ravel(), Lfull @ wn, rtol=0, atol=1e-10)


def test_dense_draw_covariance_matches_target():
    """Sample covariance over many seeds: Cov(alpha_i(a), alpha_j(b)) = (D/r0)^(5/3) R_Z[i,j] Sigma[a,b]."""
    from oracle import fields, noll

    p = fields.CorrParams(8, (16.0,))
    R = noll.noll_cov(36)  # J = 2..36
    L = noll.cholesky_lower(noll.noll_cov(36))
    h = w = 17  # 4 x 4 anchors
    n = 2000
    dr = 2.0
    a = np.stack([fields.alpha_anchors(5000 + k, dr, h, w, p, L, method="dense") for k in range(n)])
    # anchors (0, 0) and (0, 1): spatial correlation exp(-64 / 512)
    c01 = np.exp(-64.0 / (2 * 256.0))
    for i, j in ((0, 0), (0, 6), (2, 9), (1, 1)):
        for (ay, ax, by, bx, c) in ((0, 0, 0, 0, 1.0), (0, 0, 0, 1, c01)):
            target = dr ** (5 / 3) * R[i, j] * c
            x, y = a[:, ay, ax, i], a[:, by, bx, j]
            est = np.mean(x * y)
            se = np.sqrt((np.var(x) * np.var(y) + est ** 2) / n)
            assert abs(est - target) < 5 * se + 1e-12, (i, j, ay, ax, by, bx, est, target, se)
