"""GPU parity of the gradient estimator with path reuse (Sec. 4.1.3;
wob_solve_grad) against the oracle's dl_walks(want_grad=True).

The gradient of a walk is its value times the first step's factor
-(n - 3 (w . n) w) / (r (w . n)); the values follow the double-layer bars
(1e-5 * sum |terms| on unflagged walks), the factors (FP64 geometry from the
same FP32 vertices and the same hit) agree to 1e-9 relative."""
import numpy as np
import pytest

import oracle as O
from paper_2305_04403_gb300 import inputs as I

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


@pytest.mark.parametrize("phi", [1, -1])
def test_gradient_parity(wob, phi):
    v, f, sh = I.star_mesh(4, 0.3, 6, 3, 0.5)
    rng = np.random.default_rng(11)
    d = rng.standard_normal((40, 3))
    d /= np.linalg.norm(d, axis=1, keepdims=True)
    fac = rng.uniform(0.1, 0.7, 40) if phi == 1 else rng.uniform(1.3, 2.0, 40)
    q = (d * (sh.radius(d) * fac)[:, None]).astype(np.float32)
    poly = (0.1, 0.3, -0.2, 0.5, 1.0, -1.0, 0.0, 0.4, 0.0, 0.0)
    mesh = wob.build_mesh(v, f)
    bvh = wob.build_bvh(mesh)
    prob = wob.Problem(bvh, side=phi, data_mode=wob.DATA_POLY, poly=poly, problem=4, tau=TAU)
    g = {k: t.cpu().numpy() for k, t in
         wob.solve_grad(prob, q, 64, 6, seed=3, per_walk=True).items()}
    dbg = wob.solve_debug(prob, q, 64, 6, seed=3, want_lines=False)
    pw = dbg["per_walk"].cpu().numpy()
    r = O.dl_walks(v, f, q, 64, 6, seed=3, problem=4, phi=phi, poly=poly, tau=TAU,
                   want_grad=True)
    ok = (dbg["flag"].cpu().numpy() == 0) & (r["flag"] == 0)
    assert ok.mean() > 0.8
    # the gradient walks are the value walks: identical values
    est, _ = wob.solve(prob, q, 64, 6, seed=3)
    assert np.array_equal(g["est"], est.cpu().numpy())
    err = np.abs(pw - r["per_walk"])
    assert np.all(err[ok] <= 1e-5 * r["abs_terms"][ok] + 1e-12)
    big = ok & (np.abs(r["per_walk"]) > 1e-6)
    fg = g["grad"][:, big] / pw[big]
    fr = r["grad"][:, big] / r["per_walk"][big]
    assert np.allclose(fg, fr, rtol=1e-9, atol=0)
    # missed first lines (exterior) give a zero gradient
    zero = np.abs(pw) == 0
    assert np.all(g["grad"][:, zero] == 0)
    # reductions of the per-walk gradients
    for c in range(3):
        e2, v2 = O.reduce(g["grad"][c])
        assert np.allclose(e2, g["grad_est"][c], rtol=1e-12, atol=1e-14)
        assert np.allclose(v2, g["grad_var"][c], rtol=1e-10, atol=1e-14)


def test_gradient_of_linear_field_on_sphere(wob):
    """Large-N check on the GPU against the sphere closed form: h = z has
    grad (0, 0, ratio_M) with ratio_M = 1 - b^(M-1) (1 + b) / 2, b = -1/3."""
    v, f = I.icosphere(4)
    q = I.ball_queries(16, 0.6, 3)
    mesh = wob.build_mesh(v, f)
    bvh = wob.build_bvh(mesh)
    prob = wob.Problem(bvh, data_mode=wob.DATA_POLY, poly=(0, 0, 0, 1, 0, 0, 0, 0, 0, 0))
    M, N = 3, 1 << 16
    g = {k: t.cpu().numpy() for k, t in wob.solve_grad(prob, q, N, M, seed=1).items()}
    b = -1.0 / 3.0
    ratio = 1.0 - 0.5 * b ** (M - 1) * (1.0 + b)
    se = np.sqrt(g["grad_var"] / N)
    pred = np.zeros((3, len(q)))
    pred[2] = ratio
    assert np.all(np.abs(g["grad_est"] - pred) <= 5 * se + 5e-3)
