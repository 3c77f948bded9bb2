"""Synthetic input generators: mesh topology, orientation and shapes."""
import math

import numpy as np

from paper_2305_04403_gb300 import inputs as I
from _meshes import edge_manifold_ok


def _signed_volume(v, f):
    v = v.astype(np.float64)
    a, b, c = v[f[:, 0]], v[f[:, 1]], v[f[:, 2]]
    return np.einsum("ij,ij->i", a, np.cross(b, c)).sum() / 6.0


def test_icosphere_counts_and_closure():
    for level in range(0, 4):
        v, f = I.icosphere(level)
        assert v.shape == (10 * 4 ** level + 2, 3)
        assert f.shape == (20 * 4 ** level, 3)
        assert v.dtype == np.float32 and f.dtype == np.int32
        assert edge_manifold_ok(f)
        assert _signed_volume(v, f) > 0
        assert np.allclose(np.linalg.norm(v, axis=1), 1.0, atol=1e-6)
        # every face normal points away from the origin (convex, outward)
        a, b, c = v[f[:, 0]], v[f[:, 1]], v[f[:, 2]]
        n = np.cross(b - a, c - a)
        assert np.all(np.einsum("ij,ij->i", n, a + b + c) > 0)


def test_real_sph_harm_orthonormal():
    # Gauss-Legendre x trapezoid quadrature, exact for these degrees
    nt, nphi = 24, 48
    x, w = np.polynomial.legendre.leggauss(nt)
    phi = 2 * math.pi * np.arange(nphi) / nphi
    X, PH = np.meshgrid(x, phi, indexing="ij")
    W = np.repeat(w[:, None], nphi, 1) * (2 * math.pi / nphi)
    s = np.sqrt(1 - X ** 2)
    dirs = np.stack([s * np.cos(PH), s * np.sin(PH), X], -1).reshape(-1, 3)
    Y = I.real_sph_harm(6, dirs)
    keys = sorted(Y)
    G = np.array([[np.sum(W.ravel() * Y[a] * Y[b]) for b in keys] for a in keys])
    assert np.allclose(G, np.eye(len(keys)), atol=1e-10)


def test_star_mesh_level6():
    v, f, shape = I.star_mesh(6)
    assert f.shape == (81920, 3) and v.shape == (40962, 3)
    assert edge_manifold_ok(f)
    assert _signed_volume(v, f) > 0
    r = np.linalg.norm(v.astype(np.float64), axis=1)
    assert np.allclose(r, shape.radius(v.astype(np.float64) / r[:, None]), atol=1e-5)


def test_star_slice_queries_inside():
    v, f, shape = I.star_mesh(4)
    q = I.star_slice_queries(shape, 64)
    assert q.shape[1] == 3 and np.all(q[:, 2] == 0)
    rad = np.linalg.norm(q.astype(np.float64), axis=1)
    d = q / rad[:, None]
    assert np.all(rad < shape.radius(d) - 5e-3)
    assert 0.2 < q.shape[0] / 64 ** 2 < 0.8


def test_torus_mesh():
    v, f, shape = I.displaced_torus(40, 16)
    assert f.shape == (2 * 40 * 16, 3)
    assert edge_manifold_ok(f)
    assert _signed_volume(v, f) > 0
    # core circle is inside, centre of the hole is outside
    core = np.array([[1.0, 0, 0], [0, 1.0, 0], [-1.0, 0, 0]])
    assert np.all(I.torus_inside(shape, core, 0.05))
    assert not np.any(I.torus_inside(shape, np.array([[0.0, 0, 0], [0, 0, 0.1]])))


def test_ball_and_boundary_points():
    q = I.ball_queries(1000, 0.9, 1)
    assert q.shape == (1000, 3) and np.all(np.linalg.norm(q, axis=1) <= 0.9 + 1e-6)
    v, f = I.icosphere(2)
    p, prim = I.boundary_points(v, f, 500, 3)
    a, b, c = (v[f[prim, i]].astype(np.float64) for i in range(3))
    n = np.cross(b - a, c - a)
    assert np.allclose(np.einsum("ij,ij->i", n, p - a), 0, atol=1e-6)
