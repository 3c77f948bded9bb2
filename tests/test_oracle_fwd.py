"""Pins for the oracle's forward (adjoint) single-layer Neumann paths
(Sec. 4.4.3).  A forward path starts on the boundary and reads the
truncated single-layer series from its source end, connecting every vertex
to every evaluation point; its expectation is that of the backward
single-layer walks, so on the unit sphere mode l of the estimate is
ratio_M(b_l) h_l with b_l = +1/(2l+1) inside and -1/(2l+1) outside (see
test_oracle_walks.py), whatever the start density."""
import numpy as np
import pytest

import oracle as O
from paper_2305_04403_gb300 import inputs as I
from test_oracle_walks import QIN, QOUT, Z, X2Y2, multipole, ratio


@pytest.fixture(scope="module")
def sphere3():
    return I.icosphere(3)


def _check(per_path, pred, k=5.0):
    est, var = O.reduce(per_path)
    se = np.sqrt(var / per_path.shape[1])
    assert np.all(np.abs(est - pred) <= k * se), (est, pred, se)


@pytest.mark.parametrize("start_mode", [0, 1])
@pytest.mark.parametrize("M", [1, 2, 3])
@pytest.mark.parametrize("poly,l", [(Z, 1), (X2Y2, 2)])
def test_forward_interior_closed_form(sphere3, start_mode, M, poly, l):
    v, f = sphere3
    r = O.fwd_paths(v, f, 60000, M, mode=O.DATA_POLY, poly=poly, start_mode=start_mode)
    pp = O.fwd_connect(QIN, r["zpos"], r["zw"])
    _check(pp, ratio(1.0 / (2 * l + 1), M) * I.poly_eval(poly, QIN))


@pytest.mark.parametrize("M", [1, 2, 3])
def test_forward_exterior_closed_form(sphere3, M):
    v, f = sphere3
    x0 = (0.1, 0.2, 0.3)
    r = O.fwd_paths(v, f, 60000, M, phi=-1, mode=O.DATA_POINT, x0=x0, start_mode=1)
    pp = O.fwd_connect(QOUT, r["zpos"], r["zw"])
    _check(pp, multipole(x0, QOUT, lambda l: -1 / (2 * l + 1), M, False))


def test_forward_vertices_and_weights():
    """Structure of a path on a convex mesh: every line from a boundary
    point hits once (m = 1, s = +1), so the weights alternate by phi only
    after the first; the last vertex carries half its weight; positions lie
    on the mesh."""
    v, f = I.icosphere(2)
    r = O.fwd_paths(v, f, 200, 4, mode=O.DATA_POLY, poly=Z, start_mode=0)
    zw, zp = r["zw"], r["zpos"]
    assert np.all(r["flag"] == 0)
    a = zw[:, :3]
    assert np.allclose(a[:, 1:], a[:, :-1], rtol=1e-12)           # phi m s = +1 inside
    assert np.allclose(zw[:, 3], 0.5 * zw[:, 2], rtol=1e-12)
    rad = np.linalg.norm(zp, axis=2)
    assert np.all(rad <= 1.0 + 1e-6) and np.all(rad > 0.95)


def test_boundary_weighted_start_lowers_variance_for_sparse_data():
    """Data concentrated around a few points (the paper's Neumann example):
    starting paths where |q| is large gives the same expectation with far
    less variance than uniform starts."""
    v, f = I.icosphere(3)
    vd = np.zeros(len(v), np.float32)
    for c, s in (((0, 0, 1), 1.0), ((0, 0, -1), -1.0), ((1, 0, 0), 0.7), ((-1, 0, 0), -0.7)):
        d = np.linalg.norm(v - np.array(c, np.float32), axis=1)
        vd += s * np.exp(-(d / 0.15) ** 2).astype(np.float32)
    q = np.array([[0.1, 0.0, 0.5], [0.4, 0.1, 0.0], [-0.3, 0.2, -0.2]], np.float32)
    out = {}
    for sm in (0, 1):
        r = O.fwd_paths(v, f, 40000, 3, mode=O.DATA_VERTEX_P1, vertex_data=vd, start_mode=sm)
        out[sm] = O.reduce(O.fwd_connect(q, r["zpos"], r["zw"]))
    (e0, v0), (e1, v1) = out[0], out[1]
    se = np.sqrt(v0 / 40000 + v1 / 40000)
    assert np.all(np.abs(e0 - e1) <= 5 * se)
    assert np.all(v1 < 0.25 * v0), (v0, v1)
