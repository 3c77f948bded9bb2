"""Pins for the oracle's all-hits line query (Sec. 4.4.1 of the paper).

* P7: on integer-coordinate meshes with dyadic line origins and small integer
  axes every signed volume is exact in double, so the oracle's hit set must
  equal an exact integer brute force (Python ints), including which hit
  the minimum-key rule picks and the sign of every hit.
* P1 (Gauss): summed over all hits of a line, s = sign(omega . n) is 2 for
  a point inside a closed surface, 1 for a point on it (own face excluded)
  and 0 outside; this is the solid-angle identity behind c(x) = 1/2 in
  Eq. (cbie).  Checked on convex, non-convex and multiply connected meshes.
* The pick is uniform over the m hits (chi-square over many keys).
"""
import numpy as np
import pytest
from scipy import stats

import oracle as O
from paper_2305_04403_gb300 import inputs as I
from _meshes import cube, l_prism, tetrahedron

TAU = 2e-6


def _exact_hits(v, f, o_num, den, d):
    """Exact brute force: o = o_num / den (ints), d integer, v integer."""
    V = [tuple(int(c) * den for c in row) for row in v.astype(np.int64)]
    O_ = tuple(int(c) for c in o_num)
    D = tuple(int(c) for c in d)
    hits = []
    for j, (a, b, c) in enumerate(f.tolist()):
        P = [tuple(V[i][k] - O_[k] for k in range(3)) for i in (a, b, c)]

        def tri(u, w):
            cx = u[1] * w[2] - u[2] * w[1]
            cy = u[2] * w[0] - u[0] * w[2]
            cz = u[0] * w[1] - u[1] * w[0]
            return D[0] * cx + D[1] * cy + D[2] * cz

        e = (tri(P[0], P[1]), tri(P[1], P[2]), tri(P[2], P[0]))
        if all(x > 0 for x in e) or all(x < 0 for x in e):
            A = P[0]
            e1 = tuple(V[b][k] - V[a][k] for k in range(3))
            e2 = tuple(V[c][k] - V[a][k] for k in range(3))
            N = (e1[1] * e2[2] - e1[2] * e2[1], e1[2] * e2[0] - e1[0] * e2[2],
                 e1[0] * e2[1] - e1[1] * e2[0])
            s = 1 if sum(N[k] * A[k] for k in range(3)) > 0 else -1
            hits.append((j, s))
    return hits


@pytest.mark.parametrize("mesh", [tetrahedron, cube, l_prism])
def test_exact_hit_sets_integer_meshes(mesh):
    v, f = mesh()
    rng = np.random.default_rng(11)
    n = 600
    den = 1024
    o_num = rng.integers(-1 * den, 5 * den, size=(n, 3))
    d = rng.integers(-40, 41, size=(n, 3))
    d[np.all(d == 0, axis=1)] = (1, 2, 3)
    o = o_num / den
    res = O.trace_lines(v, f, o, d.astype(np.float64), tau=TAU)
    for i in range(n):
        hits = _exact_hits(v, f, o_num[i], den, d[i])
        assert res["m"][i] == len(hits)
        assert res["sum_s"][i] == sum(s for _, s in hits)
        if hits:
            keys = []
            for j, s in hits:
                x = O.philox4x32_10(np.array([[i, 0, (0 << 16) | (1 << 12), j]], np.uint32),
                                    np.array([0, 0], np.uint32))[0]
                keys.append(((int(x[0]) << 32) | int(x[1]), j, s))
            kbest = min(keys)
            assert res["prim"][i] == kbest[1]
            assert res["s"][i] == kbest[2]
        else:
            assert res["prim"][i] == -1


def _random_axes(n, seed):
    rng = np.random.default_rng(seed)
    d = rng.standard_normal((n, 3))
    return d / np.linalg.norm(d, axis=1, keepdims=True)


def _meshes_with_points():
    """(name, verts, tris, interior points, exterior points)."""
    out = []
    v, f = I.icosphere(2)
    rng = np.random.default_rng(1)
    pout = _random_axes(300, 2) * rng.uniform(1.2, 3.0, (300, 1))
    out.append(("icosphere2", v, f, I.ball_queries(300, 0.9, 2), pout.astype(np.float32)))
    v, f, sh = I.star_mesh(3, 0.3, 6, 3, 0.5)
    dirs = _random_axes(300, 3)
    r_in = sh.radius(dirs) * rng.uniform(0.05, 0.8, 300)
    r_out = sh.radius(dirs) * rng.uniform(1.3, 2.0, 300)
    out.append(("spiky_star3", v, f, (dirs * r_in[:, None]).astype(np.float32),
                (dirs * r_out[:, None]).astype(np.float32)))
    v, f = l_prism()
    pin = np.concatenate([rng.uniform([0.1, 0.1, 0.1], [3.9, 1.9, 1.9], (150, 3)),
                          rng.uniform([0.1, 0.1, 0.1], [1.9, 3.9, 1.9], (150, 3))])
    pout = rng.uniform([2.1, 2.1, -1], [5, 5, 3], (300, 3))
    out.append(("l_prism", v, f, pin.astype(np.float32), pout.astype(np.float32)))
    v, f, tsh = I.displaced_torus(48, 20)
    phi = rng.uniform(0, 2 * np.pi, 300)
    core = np.stack([np.cos(phi), np.sin(phi), np.zeros(300)], 1)
    jitter = rng.uniform(-0.1, 0.1, (300, 3))
    hole = np.stack([0.3 * np.cos(phi), 0.3 * np.sin(phi), rng.uniform(-1, 1, 300)], 1)
    out.append(("torus", v, f, (core + jitter).astype(np.float32), hole.astype(np.float32)))
    return out


@pytest.mark.parametrize("case", _meshes_with_points(), ids=lambda c: c[0])
def test_gauss_invariant_per_line(case):
    name, v, f, pin, pout = case
    d = _random_axes(len(pin), 5)
    r = O.trace_lines(v, f, pin, d, tau=TAU)
    ok = r["flag"] == 0
    assert ok.mean() > 0.95
    assert np.all(r["sum_s"][ok] == 2)
    # the picked hit's expectation (m/2) s averaged over the pick is sum_s / 2
    assert np.all(r["m"][ok] >= 2) and np.all(r["m"][ok] % 2 == 0)
    r = O.trace_lines(v, f, pout, _random_axes(len(pout), 6), tau=TAU)
    ok = r["flag"] == 0
    assert np.all(r["sum_s"][ok] == 0) and np.all(r["m"][ok] % 2 == 0)
    # boundary points, own face excluded: half the solid angle
    p, prim = I.boundary_points(v, f, 400, 7)
    r = O.trace_lines(v, f, p, _random_axes(400, 8), exclude=prim, tau=TAU)
    ok = r["flag"] == 0
    assert ok.mean() > 0.9
    assert np.all(r["sum_s"][ok] == 1) and np.all(r["m"][ok] % 2 == 1)


def test_gauss_fails_without_exclusion():
    """Without excluding the own face the self hit at t ~ 0 is flagged."""
    v, f = I.icosphere(2)
    p, prim = I.boundary_points(v, f, 200, 9)
    r = O.trace_lines(v, f, p, _random_axes(200, 10), tau=TAU)
    assert r["flag"].mean() > 0.9


def test_pick_is_uniform_over_hits():
    v, f, tsh = I.displaced_torus(48, 20)
    # a line through the hole along x crosses the tube 4 times
    o = np.array([[0.0, 0.0, 0.0]])
    d = np.array([[1.0, 0.013, 0.021]])
    d /= np.linalg.norm(d)
    n = 20000
    keys = np.stack([np.zeros(n), np.arange(n), np.zeros(n)], 1)
    r = O.trace_lines(v, f, np.repeat(o, n, 0), np.repeat(d, n, 0), keys=keys, tau=TAU)
    assert np.all(r["m"] == 4) and np.all(r["flag"] == 0)
    prims, counts = np.unique(r["prim"], return_counts=True)
    assert len(prims) == 4
    assert stats.chisquare(counts).pvalue > 1e-3
    # the two near hits are entering (s=-1) from the hole, the far ones leaving
    assert sorted(np.unique(r["s"]).tolist()) == [-1, 1]
