"""GPU parity for the learned control variate: the BF16 tensor-core network
against the oracle's FP64 network (same weights), density walks, the
quadratures of D and H, and the residual walks.

Bars: network outputs and gradients within 2e-2 (relative, BF16 operands);
quadratures within 5e-5 (FP32 sums against FP64); residual walks with a zero
network equal plain walks (1e-12) and with a constant network reproduce the
plain walks (quadrature error); against the oracle's residual walks with the
same random network, per walk within 3e-2 * M * max|nu_t| (BF16 network).
"""
import numpy as np
import pytest

import oracle as O
from oracle import cv as C
from paper_2305_04403_gb300 import inputs as I
from _parity import compare_walks

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def wob():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2305_04403_gb300 import build as B
    B.build()
    import paper_2305_04403_gb300 as w
    return w


def _params32(seed=2):
    flat = C.flatten(C.mlp_init(seed)).astype(np.float32)
    return flat, C.unflatten(flat.astype(np.float64))


def _sphere_points(n, seed):
    rng = np.random.default_rng(seed)
    y = rng.standard_normal((n, 3))
    return (y / np.linalg.norm(y, axis=1, keepdims=True)).astype(np.float32)


def test_mlp_forward_matches_oracle(wob):
    flat, params = _params32()
    assert wob.mlp_num_params() == flat.size
    y = _sphere_points(3000, 1)
    got = wob.mlp_forward(flat, y).cpu().numpy()
    ref, _ = C.mlp_forward(params, y.astype(np.float64))
    assert np.abs(got - ref).max() <= 2e-2 * np.abs(ref).max(), np.abs(got - ref).max()
    # ragged tails of the 128-row tensor-core tile, and more tiles than CTAs
    for n in (1, 127, 129, 257, 2999):
        g = wob.mlp_forward(flat, y[:n]).cpu().numpy()
        assert np.allclose(g, got[:n], rtol=0, atol=1e-6)
    big = _sphere_points(200_000, 9)
    gb = wob.mlp_forward(flat, big).cpu().numpy()
    rb, _ = C.mlp_forward(params, big[:5000].astype(np.float64))
    assert np.abs(gb[:5000] - rb).max() <= 2e-2 * np.abs(rb).max()
    assert np.allclose(gb[-1000:], wob.mlp_forward(flat, big[-1000:]).cpu().numpy(), rtol=0,
                       atol=1e-6)


def test_mlp_init_matches_oracle(wob):
    for seed in (2, (7 << 32) | 5):
        got = wob.mlp_init(seed).cpu().numpy()
        assert np.array_equal(got, C.mlp_init_counter(seed))


def test_mlp_gradients_match_oracle(wob):
    flat, params = _params32()
    rng = np.random.default_rng(3)
    n = 200
    y = _sphere_points(n, 4)
    target = rng.standard_normal(n).astype(np.float32)
    p = torch.from_numpy(flat).cuda()
    m = torch.zeros_like(p)
    v = torch.zeros_like(p)
    grad = torch.empty_like(p)
    loss = torch.empty(1, dtype=torch.float32, device="cuda")
    wob.mlp_train_step(p, m, v, torch.from_numpy(y).cuda(), torch.from_numpy(target).cuda(),
                       0.0, 1, grad=grad, loss=loss)
    g = grad.cpu().numpy()
    ref_loss, ref = C.mse_grad(params, y.astype(np.float64), target.astype(np.float64))
    assert abs(loss.item() - ref_loss) <= 2e-2 * ref_loss
    o = 0
    for fan_in, fan_out in C.LAYERS:
        for size in (fan_in * fan_out, fan_out):
            a, b = g[o:o + size], ref[o:o + size]
            assert np.linalg.norm(a - b) <= 3e-2 * np.linalg.norm(b) + 1e-7, (o, size)
            o += size
    assert torch.equal(p, torch.from_numpy(flat).cuda())  # lr = 0: no update


def test_mlp_training_reduces_loss(wob):
    flat, _ = _params32()
    y = _sphere_points(8192, 5)
    target = (1.5 * y[:, 2] + 0.3 * y[:, 0] * y[:, 1]).astype(np.float32)
    p = torch.from_numpy(flat).cuda()
    m, v = torch.zeros_like(p), torch.zeros_like(p)
    yd, td = torch.from_numpy(y).cuda(), torch.from_numpy(target).cuda()
    loss = torch.empty(1, dtype=torch.float32, device="cuda")
    wob.mlp_train_step(p, m, v, yd, td, 0.0, 1, loss=loss)
    l0 = loss.item()
    for step in range(1, 401):
        sl = slice((step * 1024) % 8192, (step * 1024) % 8192 + 1024)
        wob.mlp_train_step(p, m, v, yd[sl], td[sl], 1e-3, step)
    wob.mlp_train_step(p, m, v, yd, td, 0.0, 1, loss=loss)
    assert loss.item() < 0.05 * l0, (l0, loss.item())


def test_density_walks_parity(wob):
    v, f, sh = I.star_mesh(4, 0.3, 6, 3, 0.5)
    p, prim = I.boundary_points(v, f, 40, 8)
    poly = (0.1, 0.3, -0.2, 0.5, 1.0, -1.0, 0.0, 0.4, 0.0, 0.0)
    mesh = wob.build_mesh(v, f)
    bvh = wob.build_bvh(mesh)
    prob = wob.Problem(bvh, data_mode=wob.DATA_POLY, poly=poly, tau=O.TAU)
    g = {k: t.cpu().numpy() for k, t in
         wob.solve_debug(prob, p, 48, 6, seed=2, query_prim=prim).items()}
    r = O.dl_walks(v, f, p, 48, 6, seed=2, poly=poly, query_prim=prim, want_lines=True)
    same, st = compare_walks(g, r, 1.0)
    assert st["walks_compared"] > 0.99
    e2, _ = wob.solve_density(prob, p, prim, 48, 6, seed=2)
    assert torch.equal(e2.cpu(), torch.from_numpy(g["est"]))


@pytest.fixture(scope="module")
def sphere_cv(wob):
    v, f = I.icosphere(3)
    mesh = wob.build_mesh(v, f)
    bvh = wob.build_bvh(mesh)
    cvo = wob.ControlVariate(mesh, level=2, near=2.0)
    nodes = C.Nodes(v, f, level=2)
    return v, f, mesh, bvh, cvo, nodes


def test_quadrature_parity(wob, sphere_cv):
    v, f, mesh, bvh, cvo, nodes = sphere_cv
    fz = lambda q: q[..., 2] + 0.3 * q[..., 0] * q[..., 1] - 0.2
    c4, f4 = cvo.nodes()
    cvo.set_node_values(fz(c4[..., :3].astype(np.float64)).astype(np.float32),
                        fz(f4[..., :3].astype(np.float64)).astype(np.float32))
    # node positions and weights agree with the oracle's
    assert np.allclose(c4[..., :3], nodes.coarse_pos, atol=1e-6)
    assert np.allclose(c4[..., 3], nodes.coarse_w, rtol=1e-5)
    vals = nodes.values(fz)
    q = I.ball_queries(64, 0.9, 3)
    gD = cvo.quad_D(q).cpu().numpy()
    rD = np.array([C.quad_D(nodes, vals, x.astype(np.float64), near=2.0) for x in q])
    assert np.abs(gD - rD).max() < 5e-5, np.abs(gD - rD).max()
    p, prim = I.boundary_points(v, f, 64, 4)
    fx = fz(p.astype(np.float64)).astype(np.float32)
    for phi in (1, -1):
        gH = cvo.quad_H(p, prim, fx, phi=phi).cpu().numpy()
        rH = np.array([C.quad_H(nodes, vals, p[j].astype(np.float64), prim[j], float(fx[j]), phi,
                                near=2.0) for j in range(64)])
        assert np.abs(gH - rH).max() < 5e-5, np.abs(gH - rH).max()


def _cv_run(wob, cvo, prob, params, q, walks, M, seed):
    Q = len(q)
    s = torch.zeros(Q, dtype=torch.float64, device="cuda")
    ss = torch.zeros_like(s)
    pw = torch.empty((Q, walks), dtype=torch.float64, device="cuda")
    dnt = torch.empty(Q, dtype=torch.float32, device="cuda")
    cvo.set_network(params)
    cvo.solve_range(prob, params, q, 0, walks, M, s, ss, seed=seed, per_walk=pw, dnt=dnt)
    return pw.cpu().numpy(), dnt.cpu().numpy(), s.cpu().numpy()


def test_cv_zero_network_is_plain_wob(wob, sphere_cv):
    v, f, mesh, bvh, cvo, nodes = sphere_cv
    prob = wob.Problem(bvh, data_mode=wob.DATA_POLY, poly=I.POLY_CONFIG1)
    q = I.ball_queries(32, 0.85, 6)
    zero = np.zeros(wob.mlp_num_params(), np.float32)
    pw, dnt, s = _cv_run(wob, cvo, prob, zero, q, 48, 5, 7)
    plain = wob.solve_debug(prob, q, 48, 5, seed=7, want_lines=False)["per_walk"].cpu().numpy()
    assert np.all(dnt == 0.0)
    assert np.allclose(pw, plain, rtol=0, atol=1e-12 * np.abs(plain).max())
    assert np.allclose(s, pw.sum(1), rtol=1e-12)


def test_cv_constant_network_reproduces_plain_walks(wob, sphere_cv):
    v, f, mesh, bvh, cvo, nodes = sphere_cv
    prob = wob.Problem(bvh, data_mode=wob.DATA_POLY, poly=I.POLY_CONFIG1)
    q = I.ball_queries(32, 0.85, 8)
    c = 0.7
    const = np.zeros(wob.mlp_num_params(), np.float32)
    const[-1] = c
    pw, dnt, _ = _cv_run(wob, cvo, prob, const, q, 48, 4, 9)
    plain = wob.solve_debug(prob, q, 48, 4, seed=9, want_lines=False)["per_walk"].cpu().numpy()
    assert np.allclose(dnt, c, atol=5e-5 * c)
    assert np.allclose(pw + dnt[:, None], plain, rtol=0, atol=1e-4 * c)


def test_cv_random_network_vs_oracle(wob, sphere_cv):
    v, f, mesh, bvh, cvo, nodes = sphere_cv
    prob = wob.Problem(bvh, data_mode=wob.DATA_POLY, poly=I.POLY_CONFIG1, tau=O.TAU)
    flat, params = _params32(5)
    q = I.ball_queries(6, 0.8, 10)
    M, N = 3, 16
    pw, dnt, _ = _cv_run(wob, cvo, prob, flat, q, N, M, 11)
    vals = nodes.values(lambda p: C.mlp_forward(params, p)[0])
    S, flag, Dnt = C.cv_walks(v, f, q, N, M, params, nodes, vals, I.POLY_CONFIG1, seed=11,
                             near=2.0)
    scale = np.abs(np.concatenate(vals[0:1], axis=None)).max()
    ok = ~flag
    assert ok.mean() > 0.8
    assert np.abs(dnt - Dnt).max() <= 3e-2 * scale
    assert np.all(np.abs(pw - S)[ok] <= 3e-2 * M * scale), np.abs(pw - S)[ok].max() / scale


def test_sample_boundary_matches_oracle(wob):
    v, f, _ = I.star_mesh(3, 0.3, 6, 3, 0.5)
    mesh = wob.build_mesh(v, f)
    for n in (1, 1000, 4099):
        p, pr = wob.sample_boundary(mesh, n, seed=3, problem=5)
        rp, rpr = O.area_points(v, f, n, seed=3, problem=5)
        assert np.array_equal(pr.cpu().numpy(), rpr)
        assert np.abs(p.cpu().numpy() - rp).max() <= 2e-7 * np.abs(rp).max()


def _sphere_density_ratio(l, M):
    """Truncated density series on the unit sphere, mode l: 2 sum_{k<M-1}
    lam^k + lam^(M-1), lam = -1/(2l+1) (the eigenvalue of H)."""
    lam = -1.0 / (2 * l + 1)
    return 2.0 * sum(lam ** k for k in range(M - 1)) + lam ** (M - 1)


@pytest.fixture(scope="module")
def trained(wob, sphere_cv):
    v, f, mesh, bvh, cvo, nodes = sphere_cv
    prob = wob.Problem(bvh, data_mode=wob.DATA_POLY, poly=I.POLY_CONFIG1)
    flat, _ = _params32()
    p = torch.from_numpy(flat).cuda()
    m, vv = torch.zeros_like(p), torch.zeros_like(p)
    loss = cvo.train(prob, p, m, vv, points=1 << 20, walks=64, max_len=4, point_seed=3,
                     walk_seed=0, epochs=5, batch=4096, lr=1e-3)
    return prob, p, loss.cpu().numpy()


def test_cv_train_graph_equals_unrolled_steps(wob, sphere_cv):
    """wob_cv_train replays one captured epoch per epoch (step number and
    learning rate in device memory); the parameters and losses equal those
    of the same minibatch steps launched one by one (boundary points, their
    density targets, Adam at the step numbers and the tail epoch's rate)."""
    v, f, mesh, bvh, cvo, nodes = sphere_cv
    prob = wob.Problem(bvh, data_mode=wob.DATA_POLY, poly=I.POLY_CONFIG1)
    flat, _ = _params32()
    n, b, epochs = 1 << 14, 4096, 3
    p = torch.from_numpy(flat).cuda()
    m, vv = torch.zeros_like(p), torch.zeros_like(p)
    loss = cvo.train(prob, p, m, vv, points=n, walks=16, max_len=3, point_seed=3, walk_seed=1,
                     epochs=epochs, batch=b, lr=1e-3, lr_end=2e-4, tail_epochs=1, step0=5)
    pts, prims = wob.sample_boundary(mesh, n, seed=3)
    est, _ = wob.solve_density(prob, pts, prims, 16, 3, seed=1)
    tgt = est.float()
    p2 = torch.from_numpy(flat).cuda()
    m2, v2 = torch.zeros_like(p2), torch.zeros_like(p2)
    l2 = torch.empty((epochs, n // b), dtype=torch.float32, device="cuda")
    step = 5
    for e in range(epochs):
        lr = 2e-4 if e == epochs - 1 else 1e-3
        for j in range(n // b):
            step += 1
            wob.mlp_train_step(p2, m2, v2, pts[j * b:(j + 1) * b], tgt[j * b:(j + 1) * b], lr,
                               step, loss=l2[e, j:j + 1])
    torch.cuda.synchronize()
    assert torch.equal(p, p2) and torch.equal(m, m2) and torch.equal(vv, v2)
    assert torch.equal(loss, l2)


def test_cv_training_fits_the_sphere_density(wob, sphere_cv, trained):
    v, f, mesh, bvh, cvo, nodes = sphere_cv
    prob, p, loss = trained
    assert loss.shape == (5, 256)
    assert loss[-1].mean() < 0.2 * loss[0, 0], (loss[0, 0], loss[-1].mean())
    y, _ = O.area_points(v, f, 4000, seed=9)
    nu = wob.mlp_forward(p, y.astype(np.float32)).cpu().numpy()
    g1, g2 = 0.5 * y[:, 2], y[:, 0] ** 2 - y[:, 1] ** 2
    pred = _sphere_density_ratio(1, 4) * g1 + _sphere_density_ratio(2, 4) * g2
    rel = np.sqrt(np.mean((nu - pred) ** 2) / np.mean(pred ** 2))
    # observed 0.039 (target noise, 5 epochs, and the polyhedron's own density)
    assert rel < 0.06, rel


def test_cv_estimate_is_unbiased_with_lower_variance(wob, sphere_cv, trained):
    v, f, mesh, bvh, cvo, nodes = sphere_cv
    prob, p, _ = trained
    q = I.ball_queries(256, 0.9, 1)
    N, M = 256, 4
    pw, dnt, _ = _cv_run(wob, cvo, prob, p, q, N, M, 0)
    est = dnt + pw.mean(1)
    exact = I.poly_eval(I.POLY_CONFIG1, q.astype(np.float64))
    se = pw.std(1, ddof=1) / np.sqrt(N)
    # residual truncation bias is tiny: |r| is a few percent of 2g
    assert np.all(np.abs(est - exact) <= 5 * se + 2e-3), np.abs(est - exact).max()
    plain = wob.solve_debug(prob, q, N, M, seed=0, want_lines=False)["per_walk"].cpu().numpy()
    ratio = pw.var(1, ddof=1).mean() / plain.var(1, ddof=1).mean()
    assert ratio < 0.05, ratio


# ---- control variate with Monte Carlo integrals (wob_cv_solve_mc) ----------
def _mc_run(wob, prob, params, q, walks, M, K, seed):
    Q = len(q)
    s = torch.zeros(Q, dtype=torch.float64, device="cuda")
    ss = torch.zeros_like(s)
    pw = torch.empty((Q, walks), dtype=torch.float64, device="cuda")
    wob.cv_solve_mc(prob, params, q, 0, walks, M, K, s, ss, seed=seed, per_walk=pw)
    return pw.cpu().numpy(), s.cpu().numpy(), ss.cpu().numpy()


def test_cv_mc_zero_network_is_plain_wob(wob):
    v, f, sh = I.star_mesh(4, 0.3, 6, 3, 0.5)
    bvh = wob.build_bvh(wob.build_mesh(v, f))
    prob = wob.Problem(bvh, data_mode=wob.DATA_POLY, poly=I.POLY_CONFIG1)
    q = I.ball_queries(40, 0.4, 6)
    zero = np.zeros(wob.mlp_num_params(), np.float32)
    pw, s, ss = _mc_run(wob, prob, zero, q, 33, 5, 3, 7)
    plain = wob.solve_debug(prob, q, 33, 5, seed=7, want_lines=False)["per_walk"].cpu().numpy()
    assert np.allclose(pw, plain, rtol=0, atol=1e-12 * np.abs(plain).max())
    assert np.allclose(s, pw.sum(1), rtol=1e-12) and np.allclose(ss, (pw * pw).sum(1), rtol=1e-12)


def test_cv_mc_random_network_vs_oracle(wob, sphere_cv):
    """Same streams, same picks; the GPU network is BF16 (2e-2 relative), so
    each of the 1 + K network values per vertex may differ by that much:
    per walk within 3e-2 x 2 (M + 1) x max|nu_t| on the convex mesh (|P| = 1)."""
    v, f, mesh, bvh, cvo, nodes = sphere_cv
    prob = wob.Problem(bvh, data_mode=wob.DATA_POLY, poly=I.POLY_CONFIG1, tau=O.TAU)
    flat, params = _params32(5)
    q = I.ball_queries(7, 0.8, 12)
    M, N, K = 3, 24, 3
    pw, _, _ = _mc_run(wob, prob, flat, q, N, M, K, 13)
    S, flag = C.cv_walks_mc(v, f, q, N, M, lambda y: C.mlp_forward(params, y)[0], K,
                            I.POLY_CONFIG1, seed=13)
    y, _ = O.area_points(v, f, 2000, seed=1)
    scale = np.abs(C.mlp_forward(params, y)[0]).max()
    ok = ~flag
    assert ok.mean() > 0.8
    err = np.abs(pw - S)[ok]
    assert np.all(err <= 3e-2 * 2 * (M + 1) * scale), err.max() / scale


def test_cv_mc_trained_network_unbiased_with_lower_variance(wob, sphere_cv, trained):
    v, f, mesh, bvh, cvo, nodes = sphere_cv
    prob, p, _ = trained
    q = I.ball_queries(256, 0.9, 1)
    N, M, K = 256, 2, 4
    pw, _, _ = _mc_run(wob, prob, p, q, N, M, K, 0)
    exact = I.poly_eval(I.POLY_CONFIG1, q.astype(np.float64))
    se = pw.std(1, ddof=1) / np.sqrt(N)
    # the network carries the tail: no visible truncation bias at M = 2
    assert np.all(np.abs(pw.mean(1) - exact) <= 5 * se + 3e-3), np.abs(pw.mean(1) - exact).max()
    plain = wob.solve_debug(prob, q, N, M, seed=0, want_lines=False)["per_walk"].cpu().numpy()
    ratio = pw.var(1, ddof=1).mean() / plain.var(1, ddof=1).mean()
    assert ratio < 0.6, ratio
