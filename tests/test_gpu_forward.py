"""GPU parity of the forward single-layer Neumann paths (Sec. 4.4.3;
wob_solve_forward) against the oracle's fwd_paths / fwd_connect.

Paths: same counter-based draws on both sides, so on paths neither side
flags the vertices agree to 1e-9 (float-float refinement) and the weights
to 2e-6 relative: the start weight 2 phi q(z_0) / p(z_0) takes the data
term in FP32 (rsqrt, products; n . (z_0 - x0) float-float), about five
roundings of up to 2.4e-7 each; the weighted start's CDF is summed in
another order.
Connection: the GPU sums distances and G in FP32 per path, over runs of 32
paths in FP32 and over those runs in FP64: per query within 1e-5 of the
mean of sum_j |w_j| G(x, z_j)."""
import numpy as np
import pytest

import oracle as O
from paper_2305_04403_gb300 import inputs as I

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

Z = (0, 0, 0, 1, 0, 0, 0, 0, 0, 0)


@pytest.fixture(scope="module")
def wob():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2305_04403_gb300 import build as B
    B.build()
    import paper_2305_04403_gb300 as w
    return w


def _abs_connect(q, zpos, zw):
    d = np.linalg.norm(zpos[None, :, :, :] - q[:, None, None, :].astype(np.float64), axis=3)
    return (np.abs(zw)[None] / (4 * np.pi * d)).sum(2).mean(1)


@pytest.mark.parametrize("start_mode", [0, 1])
@pytest.mark.parametrize("phi", [1, -1])
def test_forward_paths_and_connection_parity(wob, start_mode, phi):
    v, f, sh = I.star_mesh(3, 0.3, 6, 3, 0.5)
    mesh = wob.build_mesh(v, f)
    bvh = wob.build_bvh(mesh)
    x0 = (3.0, 0.5, -1.0) if phi == 1 else (0.05, -0.1, 0.1)
    prob = wob.Problem(bvh, kind=wob.NEUMANN_SL, side=phi, data_mode=wob.DATA_POINT, x0=x0,
                       problem=2)
    rng = np.random.default_rng(4)
    d = rng.standard_normal((24, 3))
    d /= np.linalg.norm(d, axis=1, keepdims=True)
    fac = rng.uniform(0.2, 0.7, 24) if phi == 1 else rng.uniform(1.3, 2.0, 24)
    q = (d * (sh.radius(d) * fac)[:, None]).astype(np.float32)
    N, M = 512, 6
    g = {k: t.cpu().numpy() for k, t in
         wob.solve_forward(prob, q, N, M, seed=3, start_mode=start_mode, want_paths=True).items()}
    # the C ABI carries x0 and beta as float32: the oracle gets the same values
    x0_32 = tuple(float(c) for c in np.float32(x0))
    r = O.fwd_paths(v, f, N, M, seed=3, problem=2, phi=phi, mode=O.DATA_POINT, x0=x0_32,
                    start_mode=start_mode, beta=float(np.float32(0.1)))
    ok = (r["flag"] == 0) & (g["flag"] == 0)
    assert ok.mean() > 0.9
    assert np.allclose(g["zpos"][ok], r["zpos"][ok], rtol=0, atol=1e-9)
    scale = np.abs(r["zw"][ok]).max()
    close = np.isclose(g["zw"], r["zw"], rtol=2e-6, atol=1e-12 * scale).all(1)
    bad = np.flatnonzero(ok & ~close)
    assert bad.size == 0, (bad.size, bad[:4], g["zw"][bad[:2]], r["zw"][bad[:2]])
    # connection of the GPU's own paths
    pp = O.fwd_connect(q, g["zpos"], g["zw"])
    e_r, v_r = O.reduce(pp)
    tol = 1e-5 * _abs_connect(q, g["zpos"], g["zw"])
    assert np.all(np.abs(g["est"] - e_r) <= tol)
    assert np.allclose(g["var"], v_r, rtol=1e-3, atol=1e-9)


def test_forward_sphere_closed_form(wob):
    """Interior Neumann with data dh/dn of h = z on icosphere level 4: the
    truncated series scales mode l = 1 by 1 - b^(M-1) (1 + b) / 2, b = 1/3."""
    v, f = I.icosphere(4)
    mesh = wob.build_mesh(v, f)
    bvh = wob.build_bvh(mesh)
    prob = wob.Problem(bvh, kind=wob.NEUMANN_SL, side=1, data_mode=wob.DATA_POLY, poly=Z)
    q = I.ball_queries(64, 0.7, 2)
    M, N = 3, 1 << 16
    g = {k: t.cpu().numpy() for k, t in wob.solve_forward(prob, q, N, M, seed=5).items()}
    b = 1.0 / 3.0
    pred = (1.0 - 0.5 * b ** (M - 1) * (1.0 + b)) * q[:, 2].astype(float)
    se = np.sqrt(g["var"] / N)
    assert np.all(np.abs(g["est"] - pred) <= 5 * se + 2e-3)
