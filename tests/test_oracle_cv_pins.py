"""Closed-form pins of the control-variate oracle's quadrature, residual
walks and optimiser (oracle/cv.py), each with a planted mistake it catches.

* D on the unit sphere: the double-layer potential of the density Y_l is
  (l+1)/(2l+1) r^l Y_l inside (D[1] = 1 is the l = 0 case).  On icosphere
  polyhedra the quadrature follows it to 2.5e-3 h^2 (h the mean edge), at
  two mesh levels, for l = 1 (z) and l = 2 (x^2 - y^2).
* H on the unit sphere: H Y_l = -Y_l / (2l+1) on the surface; for z the
  quadrature is within 0.07 h^2 of -z/3 at two mesh levels.
* Residual walks with quadrature (cv_walks) and nu_t = a Y_l: the
  expectation of D nu_t + (residual walk) is
  (l+1)/(2l+1) [a + ratio_M(-1/(2l+1)) ((2l+1)/(l+1) - a)] Y_l(x0), the
  closed form of the Monte Carlo variant (tests/test_oracle_cv_mc.py).
* Adam (Kingma and Ba 2015): with a constant gradient g the bias-corrected
  moments are g and g^2 at every step, so each step moves by
  lr g / (|g| + eps) exactly; two steps with different gradients equal
  values worked out by hand from the update.
"""
import math

import numpy as np
import pytest

from oracle import cv as C
from paper_2305_04403_gb300 import inputs as I
from test_oracle_cv_mc import _closed

QIN = np.array([[0.1, 0.2, 0.6], [0.3, -0.4, 0.3], [-0.2, 0.1, -0.5]], np.float32)
Z = (0, 0, 0, 1, 0, 0, 0, 0, 0, 0)
X2Y2 = (0, 0, 0, 0, 1, -1, 0, 0, 0, 0)
Y = {1: lambda p: p[:, 2], 2: lambda p: p[:, 0] ** 2 - p[:, 1] ** 2}


@pytest.fixture(scope="module")
def nodes_by_level():
    out = {}
    for lev in (2, 3):
        v, f = I.icosphere(lev)
        out[lev] = (v, f, C.Nodes(v, f, level=2))
    return out


def _D_errors(nodes, l, quad=C.quad_D):
    q = I.ball_queries(20, 0.8, 5).astype(np.float64)
    vals = nodes.values(Y[l])
    d = np.array([quad(nodes, vals, x) for x in q])
    return np.abs(d - (l + 1) / (2 * l + 1) * Y[l](q)).max()


def _H_errors(v, f, nodes, quad=C.quad_H):
    vals = nodes.values(Y[1])
    p, prim = I.boundary_points(v, f, 20, 7)
    h = np.array([quad(nodes, vals, p[j], prim[j], float(p[j, 2])) for j in range(20)])
    return np.abs(h + p[:, 2] / 3.0).max()


@pytest.mark.parametrize("l", [1, 2])
def test_quad_D_sphere_harmonics(nodes_by_level, l):
    errs = []
    for lev, (v, f, nodes) in sorted(nodes_by_level.items()):
        e = _D_errors(nodes, l)
        assert e <= 2.5e-3 * nodes.mean_h ** 2, (lev, e, nodes.mean_h)
        errs.append(e)
    assert errs[1] < 0.4 * errs[0]  # second order: a quarter per halving of h


def test_quad_H_sphere_z(nodes_by_level):
    for lev, (v, f, nodes) in sorted(nodes_by_level.items()):
        e = _H_errors(v, f, nodes)
        assert e <= 0.07 * nodes.mean_h ** 2, (lev, e, nodes.mean_h)


@pytest.mark.parametrize("l,a,M", [(1, 0.5, 1), (1, 1.0, 2), (1, 1.0, 3), (2, 1.0, 2)])
def test_cv_walks_sphere_closed_form(nodes_by_level, l, a, M):
    v, f, nodes = nodes_by_level[3]
    nu_t = lambda y: a * Y[l](y)
    vals = nodes.values(nu_t)
    N = 600
    S, flag, Dnt = C.cv_walks(v, f, QIN, N, M, nu_t, nodes, vals, Z if l == 1 else X2Y2,
                              seed=13 + M)
    est = Dnt + S.mean(1)
    se = S.std(1, ddof=1) / math.sqrt(N)
    pred = _closed(a, l, M, Y[l](QIN.astype(np.float64)))
    assert np.all(np.abs(est - pred) <= 5 * se + 3e-3), (est, pred, se)


def test_adam_constant_gradient_moves_lr_per_step():
    g = np.array([0.5, -2.0, 1e-3, 3.0])
    theta = np.array([1.0, 2.0, 3.0, 4.0])
    opt = C.Adam(4, lr=0.1)
    for t in range(1, 6):
        theta = opt.step(theta, g)
        want = np.array([1.0, 2.0, 3.0, 4.0]) - t * 0.1 * g / (np.abs(g) + 1e-8)
        assert np.allclose(theta, want, rtol=0, atol=1e-12), (t, theta, want)


def test_adam_two_steps_by_hand():
    """theta0 = 1, lr = 0.1, gradients 0.5 then 1.0 (b1 0.9, b2 0.999,
    eps 1e-8), worked out in exact decimal arithmetic.  Step 1: m = 0.05,
    m^ = 0.5, v = 0.00025, v^ = 0.25, theta1 = 1 - 0.1 * 0.5 / 0.50000001 =
    0.90000000199999996.  Step 2: m = 0.145, m^ = 0.145 / 0.19 =
    0.76315789473684211; v = 0.00124975, v^ = 0.00124975 / 0.001999 =
    0.62518759379689845, sqrt = 0.79068805087524780; theta2 = theta1 -
    0.1 m^ / (sqrt(v^) + eps) = 0.80348180063850872."""
    opt = C.Adam(1, lr=0.1)
    th = opt.step(np.array([1.0]), np.array([0.5]))
    assert abs(th[0] - 0.90000000199999996) < 1e-15, th
    th = opt.step(th, np.array([1.0]))
    assert abs(th[0] - 0.80348180063850872) < 1e-15, th


@pytest.mark.parametrize("mistake", ["D without density", "D wrong sign", "H without -phi f(x)",
                                     "H without subtraction", "CV H term sign",
                                     "Adam without bias correction"])
def test_pins_catch_planted_mistakes(nodes_by_level, monkeypatch, mistake):
    """Each plausible mistake, planted by wrapping the oracle's function on
    the CPU, fails the pin that guards it."""
    v, f, nodes = nodes_by_level[3]
    caught = False
    try:
        if mistake == "D without density":
            def quad(nd, vals, x0, near=3.0):
                ones = (np.ones_like(vals[0]), np.ones_like(vals[1]))
                return C.quad_D(nd, ones, x0, near)
            assert _D_errors(nodes, 1, quad) <= 2.5e-3 * nodes.mean_h ** 2
        elif mistake == "D wrong sign":
            quad = lambda nd, vals, x0, near=3.0: -C.quad_D(nd, vals, x0, near)
            assert _D_errors(nodes, 2, quad) <= 2.5e-3 * nodes.mean_h ** 2
        elif mistake == "H without -phi f(x)":
            quad = lambda nd, vals, x, prim, fx, phi=1, near=3.0: (
                C.quad_H(nd, vals, x, prim, fx, phi, near) + phi * fx)
            assert _H_errors(v, f, nodes, quad) <= 0.07 * nodes.mean_h ** 2
        elif mistake == "H without subtraction":
            quad = lambda nd, vals, x, prim, fx, phi=1, near=3.0: (
                C.quad_H(nd, vals, x, prim, 0.0, phi, near) - phi * fx)
            assert _H_errors(v, f, nodes, quad) <= 0.07 * nodes.mean_h ** 2
        elif mistake == "CV H term sign":
            orig = C.quad_H
            monkeypatch.setattr(C, "quad_H", lambda *a, **k: -orig(*a, **k))
            test_cv_walks_sphere_closed_form(nodes_by_level, 1, 1.0, 2)
        else:
            def step(self, flat, grad):
                self.t += 1
                self.m = self.b1 * self.m + (1 - self.b1) * grad
                self.v = self.b2 * self.v + (1 - self.b2) * grad * grad
                return flat - self.lr * self.m / (np.sqrt(self.v) + self.eps)
            monkeypatch.setattr(C.Adam, "step", step)
            test_adam_two_steps_by_hand()
    except AssertionError:
        caught = True
    assert caught, mistake
