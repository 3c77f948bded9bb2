"""GPU parity: the CUDA path (through the C ABI) against the CPU oracle on
the same seeded inputs.

Bars:
  * integer / bit work (Philox blocks, line axes, hit counts, picked
    triangle) -- bit-exact on every line the CUDA path does not flag as
    near-degenerate (within 1.25 tau L of a triangle edge, grazing, or a hit
    at |t| < tau L); its flag covers every line the oracle flags (tau L);
  * walks are followed line by line (tests/_parity.py): compared whole
    where every line agrees, flagged or not -- |gpu - oracle| <=
    1e-5 * sum_k |term_k| (the GPU evaluates the data term in FP32, relative
    error ~1e-7 per term, and accumulates in FP64); a line where the sides
    first differ must be flagged;
  * per query -- the mean over the walks compared whole within
    1e-4 * max|g|.
"""
import numpy as np
import pytest

import oracle as O
from paper_2305_04403_gb300 import inputs as I
from _meshes import cube, l_prism, tetrahedron
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


def _axes(n, seed):
    rng = np.random.default_rng(seed)
    d = rng.standard_normal((n, 3))
    return d / np.linalg.norm(d, axis=1, keepdims=True)


def test_philox_bit_exact(wob):
    rng = np.random.default_rng(0)
    n = 1 << 20
    ctr = rng.integers(0, 2 ** 32, size=(n, 4), dtype=np.uint64).astype(np.uint32)
    key = rng.integers(0, 2 ** 32, size=(n, 2), dtype=np.uint64).astype(np.uint32)
    got = wob.philox4x32_10(ctr, key).cpu().numpy().view(np.uint32)
    ref = O.philox4x32_10(ctr, key)
    assert np.array_equal(got, ref)


def test_line_axes_bit_exact(wob):
    n = 200_000
    qws = np.stack([np.arange(n) % 1000, np.arange(n) // 1000, np.arange(n) % 17], 1)
    for seed, problem in ((0, 0), (0xDEADBEEF12345678, 7)):
        got = wob.line_axes(seed, problem, qws).cpu().numpy()
        ref, _ = O.line_axes(seed, problem, qws)
        assert np.array_equal(got.view(np.uint64), ref.view(np.uint64))


def _line_cases():
    rng = np.random.default_rng(3)
    cases = []
    v, f = I.icosphere(3)
    cases.append(("icosphere3", v, f, I.ball_queries(2000, 0.95, 5)))
    v, f, sh = I.star_mesh(4, 0.3, 6, 3, 0.5)
    d = _axes(2000, 4)
    cases.append(("spiky_star4", v, f, (d * (sh.radius(d) * rng.uniform(0.05, 1.6, 2000))[:, None]).astype(np.float32)))
    v, f = l_prism()
    cases.append(("l_prism", v, f, rng.uniform(-1, 5, (2000, 3)).astype(np.float32)))
    v, f, tsh = I.displaced_torus(100, 40)
    cases.append(("torus", v, f, rng.uniform(-1.5, 1.5, (2000, 3)).astype(np.float32)))
    v, f, sh = I.star_mesh(6)
    d = _axes(2000, 6)
    cases.append(("star6", v, f, (d * (sh.radius(d) * rng.uniform(0.0, 1.3, 2000))[:, None]).astype(np.float32)))
    return cases


@pytest.mark.parametrize("case", _line_cases(), ids=lambda c: c[0])
def test_trace_lines_parity(wob, case):
    name, v, f, pts = case
    mesh = wob.build_mesh(v, f)
    bvh = wob.build_bvh(mesh)
    # free points and boundary points (own face excluded)
    bp, prim = I.boundary_points(v, f, len(pts), 9)
    for origins, excl in ((pts.astype(np.float64), None), (bp.astype(np.float64), prim)):
        d = _axes(len(origins), 11)
        g = {k: t.cpu().numpy() for k, t in wob.trace_lines(bvh, origins, d, exclude=excl, tau=TAU).items()}
        r = O.trace_lines(v, f, origins, d, exclude=excl, tau=TAU)
        # the GPU's flag covers every line the oracle flags
        assert not np.any((r["flag"] == 1) & (g["flag"] == 0))
        ok = g["flag"] == 0
        print(f"{name}: oracle flags {r['flag'].mean():.4f}, GPU flags {g['flag'].mean():.4f} of lines")
        assert ok.mean() > 0.95, ok.mean()
        # every line the GPU does not flag agrees exactly
        assert np.array_equal(g["m"][ok], r["m"][ok])
        assert np.array_equal(g["sum_s"][ok], r["sum_s"][ok])
        assert np.array_equal(g["prim"][ok], r["prim"][ok])
        assert np.array_equal(g["s"][ok], r["s"][ok])
        hit = ok & (r["m"] > 0)
        assert np.allclose(g["y"][hit], r["y"][hit], rtol=0, atol=1e-9)
        assert np.allclose(g["t"][hit], r["t"][hit], rtol=0, atol=1e-9)


def _run_dl(wob, v, f, q, N, M, phi=1, mode=O.DATA_POLY, poly=None, x0=None, vd=None,
            seed=0, problem=0):
    mesh = wob.build_mesh(v, f)
    bvh = wob.build_bvh(mesh)
    prob = wob.Problem(bvh, kind=wob.DIRICHLET_DL, side=phi, data_mode=mode,
                       vertex_data=None if vd is None else torch.from_numpy(vd).cuda(),
                       poly=tuple(poly) if poly is not None else (0.0,) * 10,
                       x0=tuple(x0) if x0 is not None else (0.0, 0.0, 0.0), problem=problem,
                       tau=TAU)
    g = {k: t.cpu().numpy() for k, t in wob.solve_debug(prob, q, N, M, seed=seed).items()}
    r = O.dl_walks(v, f, q, N, M, seed=seed, problem=problem, phi=phi, mode=mode,
                   vertex_data=vd, poly=poly, x0=x0, tau=TAU, want_lines=True)
    # the production reduction (from per-block partial sums) equals the
    # oracle's reduction of the GPU's own walks
    e2, v2 = O.reduce(g["per_walk"])
    assert np.allclose(g["est"], e2, rtol=1e-12, atol=1e-14)
    assert np.allclose(g["var"], v2, rtol=1e-9, atol=1e-14)
    return g, r


def test_dl_config1_parity(wob):
    """First workload as written: icosphere level 3, g = x^2 - y^2 + 0.5 z at
    the vertices (linear interpolation), 256 queries, 64 walks, M = 4."""
    v, f = I.icosphere(3)
    vd = I.poly_eval(I.POLY_CONFIG1, v).astype(np.float32)
    q = I.ball_queries(256, 0.9, 1)
    g, r = _run_dl(wob, v, f, q, 64, 4, mode=O.DATA_VERTEX_P1, vd=vd)
    same, st = compare_walks(g, r, np.abs(vd).max())
    print("config 1:", st)
    assert st["walks_compared"] > 0.999
    # every line of a walk on the convex mesh: m = 2 first, then 1
    assert np.all(g["line_m"][same][:, 0] == 2) and np.all(g["line_m"][same][:, 1:] == 1)


@pytest.mark.parametrize("phi", [1, -1])
def test_dl_nonconvex_parity(wob, phi):
    v, f, sh = I.star_mesh(4, 0.3, 6, 3, 0.5)
    rng = np.random.default_rng(2)
    d = _axes(48, 3)
    fac = rng.uniform(0.1, 0.7, 48) if phi == 1 else rng.uniform(1.3, 2.0, 48)
    q = (d * (sh.radius(d) * fac)[:, None]).astype(np.float32)
    poly = (0.1, 0.3, -0.2, 0.5, 1.0, -1.0, 0.0, 0.4, 0.0, 0.0)
    g, r = _run_dl(wob, v, f, q, 64, 8, phi=phi, poly=poly, seed=5, problem=3)
    same, st = compare_walks(g, r, np.abs(I.poly_eval(poly, v)).max())
    print(f"spiky star, phi {phi}:", st)
    assert st["walks_compared"] > 0.99
    assert (r["line_m"] >= 3).any()


def test_dl_headline_parity(wob):
    """The benchmark's mesh, data and walk length: the level-6 star (81,920
    triangles), g = 1 / |x - (3,0,0)|, M = 16; 256 of its slice queries
    (evenly spaced) x 64 walks, every walk followed line by line."""
    v, f, sh = I.star_mesh(6)
    q = I.star_slice_queries(sh, 256)
    q = q[:: len(q) // 256][:256].copy()
    g, r = _run_dl(wob, v, f, q, 64, 16, mode=O.DATA_POINT, x0=(3.0, 0.0, 0.0))
    same, st = compare_walks(g, r, 1.0 / (3.0 - 1.4))
    print("star L6, M 16:", st)
    assert st["walks_compared"] > 0.995


def test_solve_matches_debug_and_range_combines(wob):
    v, f = I.icosphere(3)
    q = I.ball_queries(64, 0.9, 7)
    mesh = wob.build_mesh(v, f)
    bvh = wob.build_bvh(mesh)
    prob = wob.Problem(bvh, data_mode=wob.DATA_POLY, poly=I.POLY_CONFIG1)
    est, var = wob.solve(prob, q, 128, 5, seed=9)
    dbg = wob.solve_debug(prob, q, 128, 5, seed=9, want_lines=False)
    assert torch.equal(est, dbg["est"]) and torch.equal(var, dbg["var"])
    s = torch.zeros(64, dtype=torch.float64, device="cuda")
    ss = torch.zeros_like(s)
    wob.solve_range(prob, q, 0, 50, 5, s, ss, seed=9)
    wob.solve_range(prob, q, 50, 78, 5, s, ss, seed=9)
    assert torch.allclose(s / 128, est, rtol=1e-12, atol=1e-12)
    pw = dbg["per_walk"]
    assert torch.allclose(ss, (pw * pw).sum(1), rtol=1e-12)
    # host entry point: same numbers
    eh, vh = wob.solve_host(prob, q, 128, 5, seed=9)
    assert np.array_equal(eh, est.cpu().numpy()) and np.array_equal(vh, var.cpu().numpy())
    # oracle reduction of the GPU's own walks
    e2, v2 = O.reduce(pw.cpu().numpy())
    assert np.allclose(e2, est.cpu().numpy(), rtol=1e-12, atol=1e-14)
    assert np.allclose(v2, var.cpu().numpy(), rtol=1e-10)


@pytest.mark.parametrize("kind,phi,alpha", [(1, 1, 0.0), (2, -1, 0.25), (1, -1, 0.0)])
def test_sl_parity(wob, kind, phi, alpha):
    v, f = I.icosphere(3)
    q = (I.ball_queries(32, 0.8, 3) if phi == 1 else
         (_axes(32, 4) * np.random.default_rng(1).uniform(1.2, 2, (32, 1))).astype(np.float32))
    mesh = wob.build_mesh(v, f)
    bvh = wob.build_bvh(mesh)
    x0 = (0.1, 0.2, 0.3) if phi == -1 else (0.0, 0.0, 3.0)
    prob = wob.Problem(bvh, kind=kind, side=phi, alpha=alpha, data_mode=wob.DATA_POINT, x0=x0)
    g = wob.solve_debug(prob, q, 256, 6, seed=2, want_lines=False)
    pw, at = O.sl_walks(v, f, q, 256, 6, kind=kind, alpha=alpha, phi=phi, mode=O.DATA_POINT,
                        x0=x0, seed=2, want_abs=True)
    err = np.abs(g["per_walk"].cpu().numpy() - pw)
    assert np.all(err <= 1e-5 * at + 1e-12)


@pytest.mark.parametrize("kind,phi,alpha", [(1, 1, 0.0), (2, -1, 0.5)])
def test_sl_vertex_data_parity(wob, kind, phi, alpha):
    """Single-layer walks with piecewise-linear vertex data (the P1 mode of
    Sec. 4.3's sources): per walk against the oracle."""
    v, f = I.icosphere(3)
    vd = np.random.default_rng(5).standard_normal(len(v)).astype(np.float32)
    q = (I.ball_queries(32, 0.8, 3) if phi == 1 else
         (_axes(32, 4) * np.random.default_rng(1).uniform(1.2, 2, (32, 1))).astype(np.float32))
    bvh = wob.build_bvh(wob.build_mesh(v, f))
    prob = wob.Problem(bvh, kind=kind, side=phi, alpha=alpha, data_mode=wob.DATA_VERTEX_P1,
                       vertex_data=torch.from_numpy(vd).cuda())
    g = wob.solve_debug(prob, q, 128, 6, seed=3, want_lines=False)
    pw, at = O.sl_walks(v, f, q, 128, 6, kind=kind, alpha=alpha, phi=phi,
                        mode=O.DATA_VERTEX_P1, vertex_data=vd, seed=3, want_abs=True)
    err = np.abs(g["per_walk"].cpu().numpy() - pw)
    assert np.all(err <= 1e-5 * at + 1e-12), (err / np.maximum(1e-5 * at, 1e-300)).max()


def _inside_points(v, f, n, seed):
    """n points inside a small closed integer mesh: random points of its box
    kept where the oracle's Gauss invariant (sum of s over a line's hits)
    says inside."""
    rng = np.random.default_rng(seed)
    lo, hi = v.min(0), v.max(0)
    out = []
    while len(out) < n:
        p = rng.uniform(lo + 0.1, hi - 0.1, (4 * n, 3)).astype(np.float32)
        r = O.trace_lines(v, f, p, _axes(len(p), seed + len(out)).astype(np.float32))
        out += list(p[(r["sum_s"] == 2) & (r["flag"] == 0)])
    return np.array(out[:n], np.float32)


@pytest.mark.parametrize("name", ["tetrahedron", "cube", "l_prism"])
def test_small_meshes_parity(wob, name):
    """Meshes of 4, 12 and 20 triangles (integer coordinates; the area-CDF
    guide table has 4 to 32 buckets, the tree one or two levels): double-
    layer walks line by line and single-layer Neumann walks per walk against
    the oracle."""
    v, f = {"tetrahedron": tetrahedron, "cube": cube, "l_prism": l_prism}[name]()
    q = _inside_points(v, f, 24, 3)
    poly = (0.1, 0.3, -0.2, 0.5, 1.0, -1.0, 0.0, 0.4, 0.0, 0.0)
    g, r = _run_dl(wob, v, f, q, 64, 6, poly=poly, seed=4, problem=1)
    same, st = compare_walks(g, r, np.abs(I.poly_eval(poly, v)).max())
    assert st["walks_compared"] > 0.95, st
    bvh = wob.build_bvh(wob.build_mesh(v, f))
    x0 = (10.0, 1.0, -3.0)
    prob = wob.Problem(bvh, kind=wob.NEUMANN_SL, side=1, data_mode=wob.DATA_POINT, x0=x0)
    gs = wob.solve_debug(prob, q, 64, 6, seed=5, want_lines=False)["per_walk"].cpu().numpy()
    pw, at = O.sl_walks(v, f, q, 64, 6, kind=O.KIND_NEUMANN_SL, phi=1, mode=O.DATA_POINT,
                        x0=x0, seed=5, want_abs=True)
    assert np.all(np.abs(gs - pw) <= 1e-5 * at + 1e-12), (np.abs(gs - pw) / at).max()


def test_sl_boundary_queries_torus(wob):
    v, f, tsh = I.displaced_torus(100, 40)
    bp, prim = I.boundary_points(v, f, 32, 3)
    mesh = wob.build_mesh(v, f)
    bvh = wob.build_bvh(mesh)
    prob = wob.Problem(bvh, kind=wob.NEUMANN_SL, side=1, data_mode=wob.DATA_POINT, x0=(0, 0, 5))
    g = wob.solve_debug(prob, bp, 128, 5, seed=4, query_prim=prim, want_lines=False)
    pw, at = O.sl_walks(v, f, bp, 128, 5, kind=1, phi=1, mode=O.DATA_POINT, x0=(0, 0, 5),
                        seed=4, want_abs=True)
    err = np.abs(g["per_walk"].cpu().numpy() - pw)
    assert np.all(err <= 1e-5 * at + 1e-12)


@pytest.mark.parametrize("kind,phi,alpha,x0,inside", [
    (1, 1, 0.0, (0.0, 0.0, 5.0), True),      # interior Neumann
    (2, -1, 2.0, (1.0, 0.0, 0.05), False),   # exterior Robin, alpha 2
])
def test_sl_full_size_torus_sampled(wob, kind, phi, alpha, x0, inside):
    """The single-layer benchmark's mesh and settings, sampled: the
    200,000-triangle displaced torus, M = 24, 8 boundary + 8 off-boundary
    queries x 32 walks (area sampling costs the oracle O(log T) per vertex).
    Per walk |gpu - oracle| <= tol * sum|terms|, tol = max(1e-5, 5e-7 M): the
    GPU forms 1/r, G and dG/dn in FP32 (relative error below 5e-7 per
    weight), so a term after k steps carries up to k such errors."""
    v, f, sh = I.displaced_torus()
    bp, prim = I.boundary_points(v, f, 8, seed=10)
    off = I.torus_queries(sh, 8, inside, seed=20)
    q = np.concatenate([bp, off]).astype(np.float32)
    pr = np.concatenate([prim, np.full(8, -1, np.int32)])
    bvh = wob.build_bvh(wob.build_mesh(v, f))
    prob = wob.Problem(bvh, kind=kind, side=phi, alpha=alpha, data_mode=wob.DATA_POINT, x0=x0,
                       problem=kind - 1)
    M, N = 24, 32
    g = wob.solve_debug(prob, q, N, M, seed=0, query_prim=pr, want_lines=False)
    pw, at = O.sl_walks(v, f, q, N, M, kind=kind, alpha=alpha, phi=phi, mode=O.DATA_POINT,
                        x0=x0, seed=0, problem=kind - 1, want_abs=True)
    err = np.abs(g["per_walk"].cpu().numpy() - pw)
    tol = max(1e-5, 5e-7 * M)
    assert np.all(err <= tol * at + 1e-12), (err / np.maximum(tol * at, 1e-300)).max()


def test_gauss_invariant_on_gpu(wob):
    v, f, sh = I.star_mesh(5, 0.3, 6, 3, 0.5)
    mesh = wob.build_mesh(v, f)
    bvh = wob.build_bvh(mesh)
    d = _axes(100_000, 1)
    r = np.random.default_rng(0).uniform(0.05, 0.9, 100_000)
    pin = d * (sh.radius(d) * r)[:, None]
    out = {k: t.cpu().numpy() for k, t in wob.trace_lines(bvh, pin, _axes(100_000, 2), tau=TAU).items()}
    ok = out["flag"] == 0
    assert ok.mean() > 0.95
    assert np.all(out["sum_s"][ok] == 2)
    bp, prim = I.boundary_points(v, f, 100_000, 3)
    out = {k: t.cpu().numpy() for k, t in wob.trace_lines(bvh, bp, _axes(100_000, 4), exclude=prim, tau=TAU).items()}
    ok = out["flag"] == 0
    assert np.all(out["sum_s"][ok] == 1)


@pytest.mark.parametrize("mesh_kind", ["star5", "torus"])
def test_watertight_every_line(wob, mesh_kind):
    """Every line through an interior point crosses the closed surface with
    sum of s = 2 -- on EVERY line, near-degenerate ones included: two
    triangles that share an edge evaluate it in one canonical form with
    exactly opposite values, so no crossing is counted twice or missed."""
    n = 200_000
    if mesh_kind == "star5":
        v, f, sh = I.star_mesh(5, 0.3, 6, 3, 0.5)
        d = _axes(n, 21)
        pin = d * (sh.radius(d) * np.random.default_rng(1).uniform(0.05, 0.9, n))[:, None]
    else:
        v, f, tsh = I.displaced_torus(200, 80)
        pin = I.torus_queries(tsh, n, True, seed=5).astype(np.float64)
    bvh = wob.build_bvh(wob.build_mesh(v, f))
    out = {k: t.cpu().numpy() for k, t in wob.trace_lines(bvh, pin, _axes(n, 22), tau=TAU).items()}
    print(f"{mesh_kind}: flagged {out['flag'].mean():.4f}, sum_s != 2 on "
          f"{int((out['sum_s'] != 2).sum())} of {n} lines")
    assert np.all(out["sum_s"] == 2)


def test_degenerate_meshes_rejected(wob):
    v, f = I.icosphere(1)
    with pytest.raises(wob.WobError, match="DEGENERATE_MESH"):
        wob.build_mesh(v, f[:, ::-1].copy())  # inward orientation
    bad = v.copy()
    bad[3, 1] = np.nan
    with pytest.raises(wob.WobError, match="DEGENERATE_MESH"):
        wob.build_mesh(bad, f)
    f2 = f.copy()
    f2[5] = (f2[5, 0], f2[5, 0], f2[5, 1])
    with pytest.raises(wob.WobError, match="DEGENERATE_MESH"):
        wob.build_mesh(v, f2)
    f3 = f.copy()
    f3[0, 0] = 10 ** 6
    with pytest.raises(wob.WobError, match="DEGENERATE_MESH"):
        wob.build_mesh(v, f3)


def test_invalid_solve_arguments(wob):
    v, f = I.icosphere(2)
    mesh = wob.build_mesh(v, f)
    bvh = wob.build_bvh(mesh)
    prob = wob.Problem(bvh, data_mode=wob.DATA_POLY, poly=I.POLY_CONFIG1)
    q = I.ball_queries(4, 0.5, 1)
    with pytest.raises(wob.WobError, match="INVALID_ARG"):
        wob.solve(prob, q, 1, 4)
    with pytest.raises(wob.WobError, match="INVALID_ARG"):
        wob.solve(prob, q, 8, 0)
    with pytest.raises(wob.WobError, match="UNSUPPORTED"):
        wob.solve(prob, q, 8, 4, query_prim=np.zeros(4, np.int32))
    bad = wob.Problem(bvh, side=0)
    with pytest.raises(wob.WobError, match="INVALID_ARG"):
        wob.solve(bad, q, 8, 4)
    # an empty query set is a no-op
    est, var = wob.solve(prob, np.zeros((0, 3), np.float32), 8, 4)
    assert est.numel() == 0


def test_single_triangle_leaf_root(wob):
    """A mesh smaller than one leaf (root is a leaf) still traces."""
    v, f = I.icosphere(0)
    v = v[:4] * 0 + np.array([[0, 0, 0], [1, 0, 0], [0, 1, 0], [0, 0, 1]], np.float32)
    f = np.array([[0, 2, 1], [0, 1, 3], [0, 3, 2], [1, 2, 3]], np.int32)
    mesh = wob.build_mesh(v, f)
    bvh = wob.build_bvh(mesh, leaf_size=8)
    pts = np.full((100, 3), 0.2)
    d = _axes(100, 1)
    g = wob.trace_lines(bvh, pts, d, tau=TAU)
    r = O.trace_lines(v, f, pts, d, tau=TAU)
    ok = (g["flag"].cpu().numpy() == 0) & (r["flag"] == 0)
    assert np.array_equal(g["m"].cpu().numpy()[ok], r["m"][ok])
    assert np.all(g["sum_s"].cpu().numpy()[ok] == 2)
