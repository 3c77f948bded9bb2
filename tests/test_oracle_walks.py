"""Pins for the oracle's walks against closed forms and special cases.

Truncation closed form (unit sphere).  With M boundary vertices the walk
estimates u_M = D (I + H + ... + H^(M-2) + H^(M-1)/2) 2 phi g  (Sec. 4.1.2),
where H is the operator of the boundary equation.  On the unit sphere every
operator involved is diagonal in spherical harmonics: for x, y on the sphere
r . n_y = r^2 / 2, so dG/dn_y = -G/2 and dG/dn_x = -G/2 (App. A), and the
single layer S = int G . dA has eigenvalue 1/(2l+1).  If b_l is the
eigenvalue of the recursion operator for mode l, mode l of the estimate is
the exact solution times

        ratio_M(b_l) = 1 - b_l^(M-1) (1 + b_l) / 2.

  double layer, interior  (phi = +1):  b_l = -1/(2l+1)
  double layer, exterior  (phi = -1):  b_l = +1/(2l+1)
  single layer Neumann, interior:      b_l = +1/(2l+1)
  single layer Neumann, exterior:      b_l = -1/(2l+1)
  single layer Robin, exterior:        b_l = (2 alpha - 1)/(2l+1)

The polyhedral icosphere deviates from the sphere by O(h^2); the level-3
mesh is close enough that the tests below see only statistical error
(observed: within 2 sigma at level 3 for M = 1..3).
"""
import numpy as np
import pytest
from numpy.polynomial import legendre as Lg

import oracle as O
from paper_2305_04403_gb300 import inputs as I

TAU = 2e-6
Z = (0, 0, 0, 1, 0, 0, 0, 0, 0, 0)
X2Y2 = (0, 0, 0, 0, 1, -1, 0, 0, 0, 0)
ONE = (1, 0, 0, 0, 0, 0, 0, 0, 0, 0)


def ratio(b, M):
    return 1.0 - 0.5 * b ** (M - 1) * (1.0 + b)


def multipole(x0, q, bfun, M, interior, lmax=60):
    """sum_l ratio_M(b_l) h_l(x) for h = 1/|x - x0| expanded about the origin."""
    x0 = np.asarray(x0, float)
    r0 = np.linalg.norm(x0)
    out = np.zeros(len(q))
    for i, p in enumerate(np.asarray(q, float)):
        rho = np.linalg.norm(p)
        cg = p @ x0 / (rho * r0)
        for l in range(lmax):
            c = np.zeros(l + 1)
            c[l] = 1
            h = (rho ** l / r0 ** (l + 1)) if interior else (r0 ** l / rho ** (l + 1))
            out[i] += ratio(bfun(l), M) * h * Lg.legval(cg, c)
    return out


QIN = np.array([[0.1, 0.2, 0.6], [0.3, -0.4, 0.3], [-0.2, 0.1, -0.5]], np.float32)
QOUT = np.array([[1.5, 0.2, 0.3], [0.3, -1.4, 0.6], [-0.2, 0.9, -1.2]], np.float32)


@pytest.fixture(scope="module")
def sphere3():
    return I.icosphere(3)


def _check(est, var, n, pred, k=5.0, slack=0.0):
    se = np.sqrt(var / n)
    assert np.all(np.abs(est - pred) <= k * se + slack), (est, pred, se)


@pytest.mark.parametrize("M", [1, 2, 3])
@pytest.mark.parametrize("poly,l", [(Z, 1), (X2Y2, 2)])
def test_dl_interior_truncation_closed_form(sphere3, M, poly, l):
    v, f = sphere3
    n = 40000
    r = O.dl_walks(v, f, QIN, n, M, mode=O.DATA_POLY, poly=poly, tau=TAU)
    est, var = O.reduce(r["per_walk"])
    _check(est, var, n, ratio(-1.0 / (2 * l + 1), M) * I.poly_eval(poly, QIN))


@pytest.mark.parametrize("M", [1, 2, 3])
def test_dl_interior_point_source_closed_form(sphere3, M):
    v, f = sphere3
    x0 = (2.0, 0.5, -1.0)
    n = 40000
    r = O.dl_walks(v, f, QIN, n, M, mode=O.DATA_POINT, x0=x0, tau=TAU)
    est, var = O.reduce(r["per_walk"])
    _check(est, var, n, multipole(x0, QIN, lambda l: -1.0 / (2 * l + 1), M, True))


@pytest.mark.parametrize("M", [1, 2, 3])
def test_dl_exterior_truncation_closed_form(sphere3, M):
    """Exterior Dirichlet: data z on the sphere, solution z / |x|^3 (decays
    like |x|^-2, the class the double layer represents, Sec. 4.5.1)."""
    v, f = sphere3
    n = 40000
    r = O.dl_walks(v, f, QOUT, n, M, phi=-1, mode=O.DATA_POLY, poly=Z, tau=TAU)
    est, var = O.reduce(r["per_walk"])
    q = QOUT.astype(float)
    exact = q[:, 2] / np.linalg.norm(q, axis=1) ** 3
    _check(est, var, n, ratio(1.0 / 3.0, M) * exact)


def test_convex_walks_equal_algorithm1(sphere3):
    """On a convex mesh the general recursion reduces to Algorithm 1:
    u = 2 g(x1) - 2 g(x2) + ... + (-1)^(M-1) g(xM).  The walk is replayed
    step by step with the oracle's own line query."""
    v, f = sphere3
    M, n = 5, 64
    q = QIN[:2]
    r = O.dl_walks(v, f, q, n, M, mode=O.DATA_POLY, poly=X2Y2, tau=TAU, want_lines=True)
    for qi in range(len(q)):
        for w in range(n):
            x = q[qi].astype(np.float64)
            excl = -1
            trail = []
            flagged = False
            for k in range(M):
                d, _ = O.line_axes(0, 0, [[qi, w, k]])
                res = O.trace_lines(v, f, x[None], d, exclude=[excl], keys=[[qi, w, k]], tau=TAU)
                flagged |= bool(res["flag"][0])
                assert res["m"][0] == (2 if k == 0 else 1)
                assert res["s"][0] == 1
                x = res["y"][0]
                excl = res["prim"][0]
                trail.append(x.copy())
            g = I.poly_eval(X2Y2, np.array(trail))
            alg1 = sum(2 * (-1) ** k * g[k] for k in range(M - 1)) + (-1) ** (M - 1) * g[M - 1]
            assert abs(r["per_walk"][qi, w] - alg1) < 1e-12
            assert r["line_m"][qi, w].tolist() == [2] + [1] * (M - 1)
            assert r["flag"][qi, w] == flagged


@pytest.mark.parametrize("M", [1, 2, 4, 7])
def test_constant_data_is_exact_on_nonconvex_mesh(M):
    """H[1] = -1 on any closed surface (Gauss), so the modified series gives
    E[u] = 1 for every M; each walk is random on a non-convex mesh."""
    v, f, sh = I.star_mesh(3, 0.3, 6, 3, 0.5)
    q = (QIN * 0.6).astype(np.float32)
    n = 20000
    r = O.dl_walks(v, f, q, n, M, mode=O.DATA_POLY, poly=ONE, tau=TAU, want_lines=True)
    assert (r["line_m"] >= 3).any()  # the mesh really is non-convex
    est, var = O.reduce(r["per_walk"])
    if M > 1:
        assert np.all(var > 0)
    _check(est, var, n, np.ones(len(q)), k=5.0, slack=1e-12)


def test_vertex_data_matches_analytic_for_linear_data(sphere3):
    """P1 interpolation reproduces linear data exactly: walk by walk the two
    data modes agree."""
    v, f = sphere3
    lin = (0.3, -1.0, 2.0, 0.5, 0, 0, 0, 0, 0, 0)
    vd = I.poly_eval(lin, v).astype(np.float32)
    a = O.dl_walks(v, f, QIN, 256, 4, mode=O.DATA_POLY, poly=lin, tau=TAU)["per_walk"]
    b = O.dl_walks(v, f, QIN, 256, 4, mode=O.DATA_VERTEX_P1, vertex_data=vd, tau=TAU)["per_walk"]
    assert np.allclose(a, b, rtol=0, atol=1e-5 * np.abs(a).max())


def test_analytic_config1_m6(sphere3):
    """Plain WoB on the first workload's mesh and data (x^2 - y^2 + 0.5 z,
    analytic at the hit), M = 6: the estimate is the exact solution up to
    the closed-form bias and Monte Carlo error."""
    v, f = sphere3
    q = I.ball_queries(8, 0.9, 1)
    poly = (0, 0, 0, 0.5, 1, -1, 0, 0, 0, 0)
    n, M = 8192, 6
    r = O.dl_walks(v, f, q, n, M, mode=O.DATA_POLY, poly=poly, tau=TAU)
    est, var = O.reduce(r["per_walk"])
    qd = q.astype(float)
    pred = (ratio(-1 / 3, M) * 0.5 * qd[:, 2]
            + ratio(-1 / 5, M) * (qd[:, 0] ** 2 - qd[:, 1] ** 2))
    _check(est, var, n, pred)


def test_rmse_decays_as_inverse_sqrt_n(sphere3):
    v, f = sphere3
    q = I.ball_queries(48, 0.8, 4)
    M = 2
    r = O.dl_walks(v, f, q, 4096, M, mode=O.DATA_POLY, poly=Z, tau=TAU)
    pred = ratio(-1 / 3, M) * q[:, 2].astype(float)
    Ns = np.array([16, 64, 256, 1024, 4096])
    rmse = [np.sqrt(np.mean((r["per_walk"][:, :n].mean(1) - pred) ** 2)) for n in Ns]
    slope = np.polyfit(np.log(Ns), np.log(rmse), 1)[0]
    assert -0.6 <= slope <= -0.4, slope


def test_reduce_mean_and_variance():
    rng = np.random.default_rng(0)
    x = rng.standard_normal((5, 37)) * 3 + 1
    est, var = O.reduce(x)
    assert np.allclose(est, x.mean(1), rtol=1e-14)
    assert np.allclose(var, x.var(1, ddof=1), rtol=1e-12)


@pytest.mark.parametrize("M", [1, 2, 3])
def test_sl_interior_neumann_closed_form(sphere3, M):
    v, f = sphere3
    n = 100000
    pw = O.sl_walks(v, f, QIN, n, M, kind=O.KIND_NEUMANN_SL, phi=1, mode=O.DATA_POLY, poly=Z)
    est, var = O.reduce(pw)
    _check(est, var, n, ratio(1 / 3, M) * QIN[:, 2].astype(float))


@pytest.mark.parametrize("M", [1, 2, 3])
def test_sl_exterior_neumann_and_robin_closed_form(sphere3, M):
    v, f = sphere3
    n = 100000
    x0 = (0.1, 0.2, 0.3)
    pw = O.sl_walks(v, f, QOUT, n, M, kind=O.KIND_NEUMANN_SL, phi=-1, mode=O.DATA_POINT, x0=x0)
    est, var = O.reduce(pw)
    _check(est, var, n, multipole(x0, QOUT, lambda l: -1 / (2 * l + 1), M, False))
    alpha = 0.25
    pw = O.sl_walks(v, f, QOUT, n, M, kind=O.KIND_ROBIN_SL, alpha=alpha, phi=-1,
                    mode=O.DATA_POINT, x0=x0)
    est, var = O.reduce(pw)
    _check(est, var, n, multipole(x0, QOUT, lambda l: (2 * alpha - 1) / (2 * l + 1), M, False))


@pytest.mark.parametrize("M", [1, 2, 3])
@pytest.mark.parametrize("poly,l", [(Z, 1), (X2Y2, 2)])
def test_dl_gradient_closed_form(sphere3, M, poly, l):
    """Gradient from the same walks (Sec. 4.1.3): only the first weight
    changes, to -grad_x dG/dn_y / p, so the estimate's expectation is the
    gradient of the truncated solution, ratio_M(b_l) grad h_l, mode by mode."""
    v, f = sphere3
    n = 40000
    r = O.dl_walks(v, f, QIN, n, M, mode=O.DATA_POLY, poly=poly, tau=TAU, want_grad=True)
    q = QIN.astype(float)
    if l == 1:
        gh = np.tile([0.0, 0.0, 1.0], (len(q), 1))
    else:
        gh = np.stack([2 * q[:, 0], -2 * q[:, 1], np.zeros(len(q))], 1)
    pred = ratio(-1.0 / (2 * l + 1), M) * gh
    for c in range(3):
        est, var = O.reduce(r["grad"][c])
        _check(est, var, n, pred[:, c])
    # the value is unchanged by asking for the gradient
    r0 = O.dl_walks(v, f, QIN, 64, M, mode=O.DATA_POLY, poly=poly, tau=TAU)
    assert np.array_equal(r0["per_walk"], r["per_walk"][:, :64])


@pytest.mark.parametrize("M", [1, 2, 3])
def test_sl_mixed_all_dirichlet_closed_form(sphere3, M):
    """Dirichlet parts of a mixed problem (Sec. 4.3): mu = mu - k S mu + k u_D,
    sampled by a move (probability p_k, kernel -(k/p_k) G) or a stay (weight
    1/(1 - p_k)).  In expectation the operator is I - k S, eigenvalue
    b_l = 1 - k/(2l+1) on the sphere; the final step u = S mu divides by
    k/(2l+1), so mode l of the estimate is ratio_M(b_l) h_l."""
    v, f = sphere3
    n = 100000
    bc = np.full(len(f), O.BC_DIRICHLET, np.uint8)
    pw = O.sl_walks(v, f, QIN, n, M, kind=O.KIND_MIXED_SL, phi=1, mode=O.DATA_POLY, poly=Z,
                    bc_type=bc, kmix=1.5, pk=0.75)
    est, var = O.reduce(pw)
    _check(est, var, n, ratio(1.0 - 1.5 / 3.0, M) * QIN[:, 2].astype(float))


def test_sl_mixed_with_one_condition_is_that_problem(sphere3):
    """A mixed problem whose triangles all carry the Neumann (or Robin)
    condition is walk for walk the Neumann (Robin) problem."""
    v, f = sphere3
    for cond, kind, alpha in ((O.BC_NEUMANN, O.KIND_NEUMANN_SL, 0.0),
                              (O.BC_ROBIN, O.KIND_ROBIN_SL, 0.25)):
        bc = np.full(len(f), cond, np.uint8)
        a = O.sl_walks(v, f, QOUT, 64, 4, kind=O.KIND_MIXED_SL, alpha=alpha, phi=-1,
                       mode=O.DATA_POINT, x0=(0.1, 0.2, 0.3), bc_type=bc, kmix=1.0, pk=0.5)
        b = O.sl_walks(v, f, QOUT, 64, 4, kind=kind, alpha=alpha, phi=-1, mode=O.DATA_POINT,
                       x0=(0.1, 0.2, 0.3))
        assert np.array_equal(a, b)


@pytest.mark.parametrize("M", [1, 2, 3])
def test_sl_ris_is_unbiased(sphere3, M):
    """Resampled importance sampling of the next point (16 uniform
    candidates, target |kernel|) keeps the expectation: the same sphere
    closed forms as area sampling, for interior Neumann and exterior Robin."""
    v, f = sphere3
    n = 40000
    pw = O.sl_walks(v, f, QIN, n, M, kind=O.KIND_NEUMANN_SL, phi=1, mode=O.DATA_POLY, poly=Z,
                    ris=16)
    est, var = O.reduce(pw)
    _check(est, var, n, ratio(1 / 3, M) * QIN[:, 2].astype(float))
    alpha, x0 = 0.25, (0.1, 0.2, 0.3)
    pw = O.sl_walks(v, f, QOUT, n, M, kind=O.KIND_ROBIN_SL, alpha=alpha, phi=-1,
                    mode=O.DATA_POINT, x0=x0, ris=16)
    est, var = O.reduce(pw)
    _check(est, var, n, multipole(x0, QOUT, lambda l: (2 * alpha - 1) / (2 * l + 1), M, False))
