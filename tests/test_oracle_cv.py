"""Pins for the control-variate oracle (oracle/cv.py).

* Radon's 7-point rule integrates every monomial of degree <= 5 exactly on
  a triangle (and not degree 6: it is a degree-5 rule).
* Quadrature of the double-layer potential of f = 1: D[1] = 1 inside a
  closed surface and 0 outside (Gauss); H[1] = -phi on the surface.
* MLP gradients against central finite differences; Adam reduces a loss.
* The residual walk with nu_t = 0 is plain WoB, walk by walk (P9).
* With a constant nu_t = c on a convex mesh every residual walk plus
  D nu_t equals the plain walk (the constant is reproduced exactly by the
  modified series, Sec. 4.1.2, so r = 2 phi g - 2c contributes -c).
* Density walks that start on the boundary reproduce the sphere's
  truncated density series.
"""
import math

import numpy as np
import pytest

import oracle as O
from oracle import cv as C
from paper_2305_04403_gb300 import inputs as I


def _mono_exact(a, b):
    return math.factorial(a) * math.factorial(b) / math.factorial(a + b + 2)


def test_radon7_degree5_exact():
    bp, bw = C.radon7()
    assert abs(bw.sum() - 1.0) < 1e-15
    x, y = bp[:, 1], bp[:, 2]   # reference triangle (0,0), (1,0), (0,1), area 1/2
    for deg in range(7):
        for a in range(deg + 1):
            b = deg - a
            q = 0.5 * np.sum(bw * x ** a * y ** b)
            err = abs(q - _mono_exact(a, b))
            if deg <= 5:
                assert err < 1e-15, (a, b, err)
    # degree 6 is not integrated exactly
    assert abs(0.5 * np.sum(bw * x ** 6) - _mono_exact(6, 0)) > 1e-6


def test_subdivision_partitions_triangle():
    for level in range(4):
        sub = C.subdivide_bary(level)
        assert sub.shape == (4 ** level, 3, 3)
        assert np.allclose(sub.sum(-1), 1.0)
        # sub-triangle areas in barycentric space sum to the whole
        e1 = sub[:, 1, 1:] - sub[:, 0, 1:]
        e2 = sub[:, 2, 1:] - sub[:, 0, 1:]
        assert np.isclose(np.abs(e1[:, 0] * e2[:, 1] - e1[:, 1] * e2[:, 0]).sum(), 1.0)


@pytest.fixture(scope="module")
def sphere_nodes():
    v, f = I.icosphere(3)
    return v, f, C.Nodes(v, f, level=2)


def test_gauss_identities_by_quadrature(sphere_nodes):
    v, f, nodes = sphere_nodes
    ones = nodes.values(lambda p: np.ones(len(p)))
    for x0 in I.ball_queries(20, 0.9, 5):
        assert abs(C.quad_D(nodes, ones, x0) - 1.0) < 2e-5
    for r in (1.2, 2.0):
        assert abs(C.quad_D(nodes, ones, np.array([0.3, -0.2, r]))) < 2e-5
    # H[1] = -phi exactly through the subtraction
    p, prim = I.boundary_points(v, f, 20, 6)
    for j in range(20):
        assert C.quad_H(nodes, ones, p[j], prim[j], 1.0) == -1.0


def test_H_quadrature_converges_under_refinement(sphere_nodes):
    """H[f] for a smooth f: the level-2 near field agrees with a level-4 one
    to 5e-5 (observed 2.9e-5; level 3: 5.6e-6), and on the sphere
    H[z] ~ -z/3 (eigenvalue -1/(2l+1)) up to the O(h^2) polyhedral error."""
    v, f, nodes = sphere_nodes
    fine = C.Nodes(v, f, level=4)
    fz = lambda q: q[:, 2] + 0.3 * q[:, 0] * q[:, 1]
    a, b = nodes.values(fz), fine.values(fz)
    p, prim = I.boundary_points(v, f, 12, 7)
    for j in range(12):
        fx = fz(p[j:j + 1].astype(float))[0]
        ha = C.quad_H(nodes, a, p[j], prim[j], fx)
        hb = C.quad_H(fine, b, p[j], prim[j], fx)
        assert abs(ha - hb) < 5e-5, (ha, hb)
    z = lambda q: q[:, 2]
    vz = nodes.values(z)
    for j in range(12):
        h = C.quad_H(nodes, vz, p[j], prim[j], float(p[j, 2]))
        assert abs(h + p[j, 2] / 3.0) < 2e-2, (h, p[j, 2])


def test_mlp_gradient_finite_differences():
    rng = np.random.default_rng(0)
    params = C.mlp_init(2)
    y = rng.standard_normal((7, 3)) * 0.5
    target = rng.standard_normal(7)
    loss, g = C.mse_grad(params, y, target)
    flat = C.flatten(params)
    idx = rng.choice(len(flat), 40, replace=False)
    for i in idx:
        e = np.zeros_like(flat)
        e[i] = 1e-6
        lp, _ = C.mse_grad(C.unflatten(flat + e), y, target)
        lm, _ = C.mse_grad(C.unflatten(flat - e), y, target)
        fd = (lp - lm) / 2e-6
        assert abs(fd - g[i]) <= 1e-6 * max(1.0, abs(fd)), (i, fd, g[i])
    assert C.N_PARAMS == len(flat) == 18753


def test_features_layout():
    y = np.array([[0.1, -0.2, 0.3]])
    f = C.features(y)
    assert f.shape == (1, 96)
    # column 32 d + 2 k + s
    assert np.isclose(f[0, 32 * 1 + 2 * 4 + 1], math.cos(2 * math.pi * 2 ** (4 / 3) * -0.2))
    assert np.isclose(f[0, 32 * 2 + 2 * 15 + 0], math.sin(2 * math.pi * 32.0 * 0.3))


def test_adam_fits_a_smooth_function():
    rng = np.random.default_rng(1)
    y = rng.standard_normal((2048, 3))
    y /= np.linalg.norm(y, axis=1, keepdims=True)
    target = y[:, 2] * 1.5 + 0.3 * y[:, 0] * y[:, 1]
    params = C.mlp_init(2)
    flat = C.flatten(params)
    opt = C.Adam(len(flat), lr=1e-3)
    loss0, _ = C.mse_grad(params, y, target)
    for it in range(300):
        sel = rng.choice(len(y), 256, replace=False)
        loss, g = C.mse_grad(C.unflatten(flat), y[sel], target[sel])
        flat = opt.step(flat, g)
    loss1, _ = C.mse_grad(C.unflatten(flat), y, target)
    assert loss1 < 0.1 * loss0, (loss0, loss1)


def test_residual_walk_without_cv_is_plain_wob(sphere_nodes):
    v, f, nodes = sphere_nodes
    vs, fs, _ = I.star_mesh(3, 0.3, 6, 3, 0.5)
    q = (I.ball_queries(6, 0.5, 3)).astype(np.float32)
    poly = (0.1, 0.3, -0.2, 0.5, 1.0, -1.0, 0.0, 0.4, 0.0, 0.0)
    S, flag, Dnt = C.cv_walks(vs, fs, q, 32, 5, None, None, None, poly, seed=3)
    r = O.dl_walks(vs, fs, q, 32, 5, seed=3, poly=poly)
    assert np.all(Dnt == 0.0)
    assert np.allclose(S, r["per_walk"], rtol=0, atol=1e-12 * np.abs(r["per_walk"]).max())
    assert np.array_equal(flag, r["flag"].astype(bool))


def test_constant_cv_reproduces_plain_walks_on_convex_mesh(sphere_nodes):
    v, f, nodes = sphere_nodes
    params = C.mlp_init(2)
    params = [(W * 0.0, b * 0.0) for W, b in params]
    c = 0.7
    params[-1] = (params[-1][0], np.array([c]))
    vals = nodes.values(lambda p: np.full(len(p), c))
    q = I.ball_queries(5, 0.8, 9)
    S, flag, Dnt = C.cv_walks(v, f, q, 24, 4, params, nodes, vals, I.POLY_CONFIG1, seed=1)
    r = O.dl_walks(v, f, q, 24, 4, seed=1, poly=I.POLY_CONFIG1)
    ok = ~flag & (r["flag"] == 0)
    assert ok.mean() > 0.9
    assert np.allclose((S + Dnt[:, None])[ok], r["per_walk"][ok], rtol=0, atol=2e-5 * c)


@pytest.mark.parametrize("M", [1, 2, 3])
def test_density_walks_match_sphere_series(sphere_nodes, M):
    v, f, nodes = sphere_nodes
    p, prim = I.boundary_points(v, f, 6, 3)
    n = 40000
    r = O.dl_walks(v, f, p, n, M, poly=(0, 0, 0, 1, 0, 0, 0, 0, 0, 0), query_prim=prim)
    est, var = O.reduce(r["per_walk"])
    lam = -1.0 / 3.0
    # density series (I + H + ... + H^(M-2) + H^(M-1)/2) 2g on mode l = 1
    ratio = 2.0 * sum(lam ** k for k in range(M - 1)) + lam ** (M - 1)
    pred = ratio * p[:, 2].astype(float)
    se = np.sqrt(var / n)
    assert np.all(np.abs(est - pred) <= 5 * se + 5e-3 * abs(ratio)), (est, pred, se)


def test_area_points_are_area_uniform():
    """Training points: on their triangles, triangle frequencies proportional
    to area (chi-square), barycentric coordinates uniform on the simplex
    (each has mean 1/3 and P(b0 > 1/2) = 1/4)."""
    v, f, _ = I.star_mesh(2, 0.3, 6, 3, 0.5)
    n = 200000
    p, pr = O.area_points(v, f, n, seed=3)
    V = v.astype(np.float64)
    a, b, c = V[f[pr, 0]], V[f[pr, 1]], V[f[pr, 2]]
    N = np.cross(b - a, c - a)
    area = 0.5 * np.linalg.norm(N, axis=1)
    assert np.abs(np.einsum("ij,ij->i", p - a, N / (2 * area[:, None]))).max() < 1e-12
    # barycentrics by solving p = a + s (b - a) + t (c - a)
    e1, e2, r = b - a, c - a, p - a
    d11, d12, d22 = (e1 * e1).sum(1), (e1 * e2).sum(1), (e2 * e2).sum(1)
    r1, r2 = (r * e1).sum(1), (r * e2).sum(1)
    det = d11 * d22 - d12 * d12
    s = (d22 * r1 - d12 * r2) / det
    t = (d11 * r2 - d12 * r1) / det
    bary = np.stack([1 - s - t, s, t], 1)
    assert bary.min() > -1e-9
    se = np.sqrt(1 / 18 / n)                      # sd of one coordinate: 1/sqrt(18)
    assert np.all(np.abs(bary.mean(0) - 1 / 3) < 5 * se)
    frac = (bary[:, 0] > 0.5).mean()
    assert abs(frac - 0.25) < 5 * np.sqrt(0.25 * 0.75 / n)
    T = len(f)
    A = 0.5 * np.linalg.norm(np.cross(V[f[:, 1]] - V[f[:, 0]], V[f[:, 2]] - V[f[:, 0]]), axis=1)
    cnt = np.bincount(pr, minlength=T)
    expct = n * A / A.sum()
    chi2 = ((cnt - expct) ** 2 / expct).sum()
    assert abs(chi2 - (T - 1)) < 5 * np.sqrt(2 * (T - 1)), chi2


def test_counter_init_is_he_uniform():
    """Counter-based initial weights: each weight matrix uniform on
    [-sqrt(6/fan_in), sqrt(6/fan_in)] (mean 0, variance lim^2/3, in range),
    biases exactly 0; different seeds give different weights."""
    flat = C.mlp_init_counter(2)
    assert flat.dtype == np.float32 and flat.size == C.N_PARAMS
    o = 0
    for fan_in, fan_out in C.LAYERS:
        W = flat[o:o + fan_in * fan_out].astype(np.float64)
        b = flat[o + fan_in * fan_out:o + fan_in * fan_out + fan_out]
        lim = math.sqrt(6.0 / fan_in)
        assert np.all(np.abs(W) <= lim) and np.all(b == 0.0)
        n = W.size
        assert abs(W.mean()) < 5 * lim / math.sqrt(3 * n)
        assert abs(W.var() / (lim * lim / 3.0) - 1.0) < 5 * math.sqrt(0.8 / n)
        o += fan_in * fan_out + fan_out
    assert o == C.N_PARAMS
    other = C.mlp_init_counter(3)
    assert np.mean(other == flat) < 0.1
