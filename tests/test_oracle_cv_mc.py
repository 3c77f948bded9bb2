"""Pins for the control variate with Monte Carlo integrals (oracle/cv.py,
cv_walks_mc): D nu_t and H nu_t estimated by K independent all-hits lines
per point instead of quadrature (for meshes too large for it).

* nu_t = 0 is plain WoB, walk by walk.
* A constant nu_t = c on a convex mesh: every line from a boundary point
  hits once with s = +1 and every line from an interior point twice, so
  H^ c = -phi c and D^ c = c exactly; then r^ = 2 phi g - 2 c and the walk
  equals the plain walk (the constant is reproduced by the modified series).
* On the sphere, with g of harmonic degree l (interior, phi = 1) the
  density is nu = (2l+1)/(l+1) g and u = D nu; D maps degree l by
  (l+1)/(2l+1) and the truncated series keeps ratio_M(-1/(2l+1)) of it.
  With nu_t = a Y the expectation is therefore
      (l+1)/(2l+1) [a + ratio_M(-1/(2l+1)) ((2l+1)/(l+1) - a)] Y(x0),
  plain WoB at a = 0 and the exact solution at a = (2l+1)/(l+1), at every M.
"""
import numpy as np
import pytest

import oracle as O
from oracle import cv as C
from paper_2305_04403_gb300 import inputs as I
from test_oracle_walks import ratio

Z = (0, 0, 0, 1, 0, 0, 0, 0, 0, 0)
X2Y2 = (0, 0, 0, 0, 1, -1, 0, 0, 0, 0)
QIN = np.array([[0.1, 0.2, 0.6], [0.3, -0.4, 0.3], [-0.2, 0.1, -0.5]], np.float32)


@pytest.fixture(scope="module")
def sphere3():
    return I.icosphere(3)


def test_zero_network_is_plain_wob():
    vs, fs, _ = I.star_mesh(3, 0.3, 6, 3, 0.5)
    q = I.ball_queries(6, 0.5, 3)
    poly = (0.1, 0.3, -0.2, 0.5, 1.0, -1.0, 0.0, 0.4, 0.0, 0.0)
    S, flag = C.cv_walks_mc(vs, fs, q, 32, 5, None, 3, poly, seed=3)
    r = O.dl_walks(vs, fs, q, 32, 5, seed=3, poly=poly)
    assert np.allclose(S, r["per_walk"], rtol=0, atol=1e-12 * np.abs(r["per_walk"]).max())
    assert np.array_equal(flag, r["flag"].astype(bool))


def test_constant_network_reproduces_plain_walks_on_convex_mesh(sphere3):
    v, f = sphere3
    q = I.ball_queries(5, 0.8, 9)
    c = 0.7
    S, flag = C.cv_walks_mc(v, f, q, 24, 4, lambda y: np.full(len(y), c), 2, I.POLY_CONFIG1,
                            seed=1)
    r = O.dl_walks(v, f, q, 24, 4, seed=1, poly=I.POLY_CONFIG1)
    ok = ~flag & (r["flag"] == 0)
    assert ok.mean() > 0.8
    assert np.allclose(S[ok], r["per_walk"][ok], rtol=0, atol=1e-12)


def _closed(a, l, M, y):
    nu = (2 * l + 1) / (l + 1)
    return (l + 1) / (2 * l + 1) * (a + ratio(-1.0 / (2 * l + 1), M) * (nu - a)) * y


@pytest.mark.parametrize("M", [1, 2, 3])
@pytest.mark.parametrize("a", [0.5, 1.0, 1.5])
def test_sphere_closed_form_degree1(sphere3, a, M):
    v, f = sphere3
    S, flag = C.cv_walks_mc(v, f, QIN, 3000, M, lambda y: a * y[:, 2], 2, Z, seed=4)
    est, se = S.mean(1), S.std(1, ddof=1) / np.sqrt(S.shape[1])
    pred = _closed(a, 1, M, QIN[:, 2].astype(float))
    assert np.all(np.abs(est - pred) <= 5 * se + 3e-3), (est, pred, se)


@pytest.mark.parametrize("M", [1, 2])
def test_sphere_closed_form_degree2(sphere3, M):
    v, f = sphere3
    a = 1.0
    S, flag = C.cv_walks_mc(v, f, QIN, 3000, M, lambda y: a * (y[:, 0] ** 2 - y[:, 1] ** 2), 2,
                            X2Y2, seed=5)
    est, se = S.mean(1), S.std(1, ddof=1) / np.sqrt(S.shape[1])
    pred = _closed(a, 2, M, I.poly_eval(X2Y2, QIN))
    assert np.all(np.abs(est - pred) <= 5 * se + 3e-3), (est, pred, se)


def test_exact_density_removes_truncation_bias_and_variance(sphere3):
    """nu_t = 1.5 z (the exact density of u = z): unbiased at M = 1, where
    plain WoB keeps 2/3 of the solution, with smaller per-walk variance."""
    v, f = sphere3
    S, _ = C.cv_walks_mc(v, f, QIN, 3000, 1, lambda y: 1.5 * y[:, 2], 4, Z, seed=6)
    P, _ = C.cv_walks_mc(v, f, QIN, 3000, 1, None, 4, Z, seed=6)
    se = S.std(1, ddof=1) / np.sqrt(S.shape[1])
    assert np.all(np.abs(S.mean(1) - QIN[:, 2]) <= 5 * se + 3e-3)
    assert np.all(np.abs(P.mean(1) - QIN[:, 2]) > 0.05)
    assert S.var(1).mean() < P.var(1).mean()


@pytest.mark.parametrize("mistake", ["H sign", "D without 1/2"])
def test_closed_form_catches_planted_mistakes(sphere3, monkeypatch, mistake):
    """The closed-form pin has the power to see a wrong weight: with the
    sign of H^ flipped, or the 1/2 dropped from D^'s first-step weight, the
    estimate leaves the closed form by far more than 5 standard errors."""
    v, f = sphere3
    orig = C._mc_lines

    def planted(verts, tris, x, excl, qi, wi, vtx, K, nu_t, first, phi, seed, problem, tau):
        acc, flag = orig(verts, tris, x, excl, qi, wi, vtx, K, nu_t, first, phi, seed, problem, tau)
        if mistake == "H sign" and not first:
            acc = -acc
        if mistake == "D without 1/2" and first:
            acc = 2.0 * acc
        return acc, flag

    monkeypatch.setattr(C, "_mc_lines", planted)
    S, _ = C.cv_walks_mc(v, f, QIN, 3000, 2, lambda y: 1.0 * y[:, 2], 2, Z, seed=4)
    est, se = S.mean(1), S.std(1, ddof=1) / np.sqrt(S.shape[1])
    pred = _closed(1.0, 1, 2, QIN[:, 2].astype(float))
    assert np.any(np.abs(est - pred) > 5 * se + 3e-3), (est, pred, se)
