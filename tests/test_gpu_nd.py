"""GPU parity of the Neumann walks through the direct boundary integral
equation (Sec. 4.2; kind WOB_NEUMANN_DIRECT) against the oracle's nd_walks.

Bars as for the double-layer walks (tests/_parity.py): every walk is
followed line by line and compared whole where its lines agree, flagged or
not -- |gpu - oracle| <= 1e-5 * sum_k |term_k| (the GPU evaluates the
source's data in FP64 from FP32 vertices, G in FP32 from an FP64 distance);
a line where the two sides first differ must be flagged; per query the
mean over the walks compared whole within 1e-4 * the data scale.
"""
import numpy as np
import pytest

import oracle as O
from paper_2305_04403_gb300 import inputs as I
from _parity import compare_walks

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TAU = 2e-6


@pytest.fixture(scope="module")
def wob():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2305_04403_gb300 import build as B
    B.build()
    import paper_2305_04403_gb300 as w
    return w


def _run(wob, v, f, q, N, M, phi=1, mode=O.DATA_POLY, poly=None, x0=None, vd=None, prim=None,
         seed=0, problem=0):
    mesh = wob.build_mesh(v, f)
    bvh = wob.build_bvh(mesh)
    prob = wob.Problem(bvh, kind=wob.NEUMANN_DIRECT, side=phi, data_mode=mode,
                       vertex_data=None if vd is None else torch.from_numpy(vd).cuda(),
                       poly=tuple(poly) if poly is not None else (0.0,) * 10,
                       x0=tuple(x0) if x0 is not None else (0.0, 0.0, 0.0), problem=problem,
                       tau=TAU)
    g = {k: t.cpu().numpy() for k, t in
         wob.solve_debug(prob, q, N, M, seed=seed, query_prim=prim).items()}
    r = O.nd_walks(v, f, q, N, M, seed=seed, problem=problem, phi=phi, mode=mode,
                   vertex_data=vd, poly=poly, x0=x0, tau=TAU, want_lines=True, query_prim=prim)
    return g, r


def _bars(g, r, scale, min_ok):
    same, st = compare_walks(g, r, scale)
    print("direct BIE:", st)
    assert st["walks_compared"] >= min_ok
    return same


def test_nd_interior_sphere_parity(wob):
    v, f = I.icosphere(3)
    q = I.ball_queries(48, 0.85, 2)
    poly = (0.0, 0.3, -0.2, 0.5, 1.0, -1.0, 0.0, 0.4, 0.0, 0.0)
    g, r = _run(wob, v, f, q, 64, 5, poly=poly, seed=3, problem=1)
    ok = _bars(g, r, 2.0, 0.999)
    assert np.all(g["line_m"][ok][:, 0] == 2) and np.all(g["line_m"][ok][:, 1:] == 1)


@pytest.mark.parametrize("phi", [1, -1])
def test_nd_nonconvex_parity(wob, phi):
    v, f, sh = I.star_mesh(4, 0.3, 6, 3, 0.5)
    rng = np.random.default_rng(6)
    d = rng.standard_normal((40, 3))
    d /= np.linalg.norm(d, axis=1, keepdims=True)
    fac = rng.uniform(0.1, 0.7, 40) if phi == 1 else rng.uniform(1.3, 2.0, 40)
    q = (d * (sh.radius(d) * fac)[:, None]).astype(np.float32)
    x0 = (0.05, -0.1, 0.1) if phi == -1 else (3.0, 0.5, -1.0)
    g, r = _run(wob, v, f, q, 64, 8, phi=phi, mode=O.DATA_POINT, x0=x0, seed=7, problem=2)
    _bars(g, r, 1.0 / 0.5, 0.99)
    assert (r["line_m"] >= 3).any()


def test_nd_vertex_data_and_boundary_start(wob):
    v, f, tsh = I.displaced_torus(100, 40)
    p, prim = I.boundary_points(v, f, 32, 9)
    vd = (0.3 * v[:, 0] - 0.2 * v[:, 2] + 0.1).astype(np.float32)  # any P1 flux
    g, r = _run(wob, v, f, p, 64, 6, mode=O.DATA_VERTEX_P1, vd=vd, prim=prim, seed=1)
    _bars(g, r, float(np.abs(vd).max()), 0.99)
    assert np.all(g["line_m"][..., 0] == -1)


def test_nd_solve_and_range_agree(wob):
    v, f = I.icosphere(3)
    q = I.ball_queries(32, 0.9, 4)
    mesh = wob.build_mesh(v, f)
    bvh = wob.build_bvh(mesh)
    prob = wob.Problem(bvh, kind=wob.NEUMANN_DIRECT, data_mode=wob.DATA_POLY, poly=I.POLY_CONFIG1)
    est, var = wob.solve(prob, q, 128, 4, seed=2)
    dbg = wob.solve_debug(prob, q, 128, 4, seed=2, want_lines=False)
    assert torch.equal(est, dbg["est"])
    s = torch.zeros(32, dtype=torch.float64, device="cuda")
    ss = torch.zeros_like(s)
    wob.solve_range(prob, q, 0, 100, 4, s, ss, seed=2)
    wob.solve_range(prob, q, 100, 28, 4, s, ss, seed=2)
    assert torch.allclose(s / 128, est, rtol=1e-12, atol=1e-12)
