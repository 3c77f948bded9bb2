"""Small closed test meshes with integer vertex coordinates (test helpers)."""
import numpy as np


def orient(v, f):
    v = np.asarray(v, np.float64)
    f = np.asarray(f, np.int64)
    a, b, c = v[f[:, 0]], v[f[:, 1]], v[f[:, 2]]
    vol = np.einsum("ij,ij->i", a, np.cross(b, c)).sum() / 6.0
    if vol < 0:
        f = f[:, ::-1].copy()
    return v.astype(np.float32), f.astype(np.int32)


def tetrahedron():
    v = [(0, 0, 0), (4, 0, 0), (0, 4, 0), (0, 0, 4)]
    f = [(0, 2, 1), (0, 1, 3), (0, 3, 2), (1, 2, 3)]
    return orient(v, f)


def cube(s=4):
    v = [(x, y, z) for z in (0, s) for y in (0, s) for x in (0, s)]
    # vertex index = x/s + 2*y/s + 4*z/s
    quads = [(0, 2, 3, 1), (4, 5, 7, 6), (0, 1, 5, 4), (2, 6, 7, 3), (0, 4, 6, 2), (1, 3, 7, 5)]
    f = []
    for a, b, c, d in quads:
        f += [(a, b, c), (a, c, d)]
    return orient(v, f)


def l_prism():
    """L-shaped prism: polygon (0,0),(4,0),(4,2),(2,2),(2,4),(0,4), z in [0,2].
    Non-convex."""
    P = [(0, 0), (4, 0), (4, 2), (2, 2), (2, 4), (0, 4)]
    n = len(P)
    v = [(x, y, 0) for x, y in P] + [(x, y, 2) for x, y in P]
    # bottom (normal -z): triangulation of the L into 4 triangles
    tri2d = [(0, 1, 2), (0, 2, 3), (0, 3, 4), (0, 4, 5)]
    f = []
    for a, b, c in tri2d:
        f.append((a, c, b))              # bottom, reversed
        f.append((a + n, b + n, c + n))  # top, counter-clockwise from +z
    for i in range(n):
        j = (i + 1) % n
        f += [(i, j, j + n), (i, j + n, i + n)]  # side, outward for a CCW polygon
    return orient(v, f)


def edge_manifold_ok(f):
    """Every directed edge appears once and its reverse once (closed,
    consistently oriented 2-manifold)."""
    f = np.asarray(f)
    e = np.concatenate([f[:, [0, 1]], f[:, [1, 2]], f[:, [2, 0]]], 0)
    s = set(map(tuple, e.tolist()))
    if len(s) != e.shape[0]:
        return False
    return all((b, a) in s for a, b in s)
