"""Seeded synthetic inputs: boundary meshes, query points and boundary data.

This module builds inputs only.  It holds none of the estimator's
arithmetic, and both the CUDA library and the CPU oracle consume the arrays
it returns (float32 vertices, int32 counter-clockwise-from-outside
triangles, float32 query points).

Workloads (sizes as used by the tests and the benchmark):
  * ``icosphere(level)``: unit-sphere icosphere, T = 20*4^L, V = 10*4^L + 2.
  * ``star_mesh``: icosphere of level 6 (81,920 triangles) displaced radially
    by r = 1 + 0.3 * sum of real orthonormal spherical harmonics of degree
    0..6 with N(0,1)/(l+1)^2 coefficients (numpy seed 0); non-convex.
  * ``displaced_torus``: torus R = 1, tube 0.35 modulated by 10% low-order
    Fourier modes (seeded), quad grid nu x nv -> 2*nu*nv triangles.
  * query points uniform in a ball, on a z = 0 slice clipped to the
    interior, or area-uniform on the boundary.
  * ``bump_data``: sparse Neumann data, six signed Gaussian bumps on the
    boundary (the paper's Neumann example with data zero except near six
    points), integrating to zero.
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np

# --------------------------------------------------------------------------
# meshes
# --------------------------------------------------------------------------
_ICO_T = (1.0 + 5.0 ** 0.5) / 2.0
_ICO_V = np.array([(-1, _ICO_T, 0), (1, _ICO_T, 0), (-1, -_ICO_T, 0), (1, -_ICO_T, 0),
                   (0, -1, _ICO_T), (0, 1, _ICO_T), (0, -1, -_ICO_T), (0, 1, -_ICO_T),
                   (_ICO_T, 0, -1), (_ICO_T, 0, 1), (-_ICO_T, 0, -1), (-_ICO_T, 0, 1)],
                  dtype=np.float64)
_ICO_F = np.array([(0, 11, 5), (0, 5, 1), (0, 1, 7), (0, 7, 10), (0, 10, 11), (1, 5, 9),
                   (5, 11, 4), (11, 10, 2), (10, 7, 6), (7, 1, 8), (3, 9, 4), (3, 4, 2),
                   (3, 2, 6), (3, 6, 8), (3, 8, 9), (4, 9, 5), (2, 4, 11), (6, 2, 10),
                   (8, 6, 7), (9, 8, 1)], dtype=np.int64)


def _orient_outward(v: np.ndarray, f: np.ndarray) -> np.ndarray:
    """Flip all faces if the signed volume is negative."""
    a, b, c = v[f[:, 0]], v[f[:, 1]], v[f[:, 2]]
    vol = np.einsum("ij,ij->i", a, np.cross(b, c)).sum() / 6.0
    return f if vol > 0 else f[:, ::-1].copy()


def icosphere_f64(level: int) -> tuple[np.ndarray, np.ndarray]:
    """Unit icosphere in float64 (vertices on the sphere) and int64 faces."""
    v = _ICO_V / np.linalg.norm(_ICO_V, axis=1, keepdims=True)
    f = _ICO_F.copy()
    for _ in range(level):
        e = np.concatenate([f[:, [0, 1]], f[:, [1, 2]], f[:, [2, 0]]], 0)
        e = np.sort(e, axis=1)
        uniq, inv = np.unique(e, axis=0, return_inverse=True)
        inv = inv.reshape(-1)
        mid = v[uniq[:, 0]] + v[uniq[:, 1]]
        mid /= np.linalg.norm(mid, axis=1, keepdims=True)
        base = v.shape[0]
        v = np.concatenate([v, mid], 0)
        nf = f.shape[0]
        ab = base + inv[:nf]
        bc = base + inv[nf:2 * nf]
        ca = base + inv[2 * nf:]
        a, b, c = f[:, 0], f[:, 1], f[:, 2]
        f = np.concatenate([np.stack([a, ab, ca], 1), np.stack([b, bc, ab], 1),
                            np.stack([c, ca, bc], 1), np.stack([ab, bc, ca], 1)], 0)
    f = _orient_outward(v, f)
    return v, f


def icosphere(level: int) -> tuple[np.ndarray, np.ndarray]:
    v, f = icosphere_f64(level)
    return v.astype(np.float32), f.astype(np.int32)


def _assoc_legendre(lmax: int, x: np.ndarray) -> dict:
    """P_l^m(x) for 0 <= m <= l <= lmax (no Condon-Shortley phase), by the
    standard three-term recurrences."""
    P = {}
    s = np.sqrt(np.maximum(0.0, 1.0 - x * x))
    P[(0, 0)] = np.ones_like(x)
    for m in range(1, lmax + 1):
        P[(m, m)] = P[(m - 1, m - 1)] * (2 * m - 1) * s
    for m in range(0, lmax):
        P[(m + 1, m)] = x * (2 * m + 1) * P[(m, m)]
    for m in range(0, lmax + 1):
        for l in range(m + 2, lmax + 1):
            P[(l, m)] = ((2 * l - 1) * x * P[(l - 1, m)] - (l + m - 1) * P[(l - 2, m)]) / (l - m)
    return P


def real_sph_harm(lmax: int, dirs: np.ndarray) -> dict:
    """Real orthonormal spherical harmonics Y_lm (integral of Y^2 over the
    sphere = 1) at unit directions; keys (l, m), -l <= m <= l."""
    x, y, z = dirs[:, 0], dirs[:, 1], dirs[:, 2]
    phi = np.arctan2(y, x)
    P = _assoc_legendre(lmax, np.clip(z, -1.0, 1.0))
    Y = {}
    for l in range(lmax + 1):
        for m in range(0, l + 1):
            norm = math.sqrt((2 * l + 1) / (4 * math.pi) * math.factorial(l - m)
                             / math.factorial(l + m))
            if m == 0:
                Y[(l, 0)] = norm * P[(l, 0)]
            else:
                Y[(l, m)] = math.sqrt(2.0) * norm * P[(l, m)] * np.cos(m * phi)
                Y[(l, -m)] = math.sqrt(2.0) * norm * P[(l, m)] * np.sin(m * phi)
    return Y


@dataclass
class StarShape:
    """Radius function r(dir) = 1 + amp * sum_lm c_lm Y_lm(dir)."""
    coeffs: dict
    amp: float
    lmax: int

    def radius(self, dirs: np.ndarray) -> np.ndarray:
        Y = real_sph_harm(self.lmax, dirs)
        r = np.ones(dirs.shape[0])
        for key, c in self.coeffs.items():
            r += self.amp * c * Y[key]
        return r


def star_shape(amp: float = 0.3, lmax: int = 6, seed: int = 0, decay: float = 2.0) -> StarShape:
    """Coefficients c_lm ~ N(0, 1) / (l + 1)^decay (numpy default_rng(seed))."""
    rng = np.random.default_rng(seed)
    coeffs = {}
    for l in range(lmax + 1):
        for m in range(-l, l + 1):
            coeffs[(l, m)] = rng.standard_normal() / (l + 1) ** decay
    return StarShape(coeffs, amp, lmax)


def star_mesh(level: int = 6, amp: float = 0.3, lmax: int = 6, seed: int = 0,
              decay: float = 2.0):
    """Star-shaped mesh: icosphere displaced radially by the star shape."""
    v, f = icosphere_f64(level)
    shape = star_shape(amp, lmax, seed, decay)
    r = shape.radius(v)
    if np.any(r <= 0.05):
        raise ValueError("star radius not positive")
    v = v * r[:, None]
    f = _orient_outward(v, f)
    return v.astype(np.float32), f.astype(np.int32), shape


@dataclass
class TorusShape:
    R: float
    r: float
    modes: list  # (i, j, a, phase)
    amp: float
    norm: float

    def tube(self, theta: np.ndarray, phi: np.ndarray) -> np.ndarray:
        s = np.zeros(np.broadcast(theta, phi).shape)
        for i, j, a, ph in self.modes:
            s = s + a * np.cos(i * theta + j * phi + ph)
        return self.r * (1.0 + self.amp * s / self.norm)


def torus_shape(R: float = 1.0, r: float = 0.35, amp: float = 0.1, seed: int = 0) -> TorusShape:
    rng = np.random.default_rng(seed)
    modes = []
    for i in range(0, 4):
        for j in range(0, 4):
            if i == 0 and j == 0:
                continue
            modes.append((i, j, rng.standard_normal() / (1 + i + j) ** 2,
                          rng.uniform(0, 2 * math.pi)))
    th = np.linspace(0, 2 * math.pi, 256, endpoint=False)
    TH, PH = np.meshgrid(th, th, indexing="ij")
    s = np.zeros_like(TH)
    for i, j, a, ph in modes:
        s += a * np.cos(i * TH + j * PH + ph)
    norm = float(np.abs(s).max()) * 1.05
    return TorusShape(R, r, modes, amp, norm)


def displaced_torus(nu: int = 500, nv: int = 200, R: float = 1.0, r: float = 0.35,
                    amp: float = 0.1, seed: int = 0):
    """Torus about the z axis; phi (nu samples) around the axis, theta (nv
    samples) around the tube; 2*nu*nv triangles, outward normals."""
    shape = torus_shape(R, r, amp, seed)
    phi = 2 * math.pi * np.arange(nu) / nu
    theta = 2 * math.pi * np.arange(nv) / nv
    PH, TH = np.meshgrid(phi, theta, indexing="ij")
    rho = shape.tube(TH, PH)
    x = (R + rho * np.cos(TH)) * np.cos(PH)
    y = (R + rho * np.cos(TH)) * np.sin(PH)
    z = rho * np.sin(TH)
    v = np.stack([x, y, z], -1).reshape(-1, 3)
    i = np.arange(nu)[:, None]
    j = np.arange(nv)[None, :]
    a = i * nv + j
    b = ((i + 1) % nu) * nv + j
    c = ((i + 1) % nu) * nv + (j + 1) % nv
    d = i * nv + (j + 1) % nv
    f = np.concatenate([np.stack([a, b, c], -1).reshape(-1, 3),
                        np.stack([a, c, d], -1).reshape(-1, 3)], 0)
    f = _orient_outward(v, f)
    return v.astype(np.float32), f.astype(np.int32), shape


def torus_inside(shape: TorusShape, p: np.ndarray, margin: float = 0.0) -> np.ndarray:
    """Point inside the displaced tube by at least ``margin`` (tube-radial)."""
    rho_xy = np.hypot(p[:, 0], p[:, 1])
    phi = np.arctan2(p[:, 1], p[:, 0])
    dx = rho_xy - shape.R
    theta = np.arctan2(p[:, 2], dx)
    dist = np.hypot(dx, p[:, 2])
    return dist < shape.tube(theta, phi) - margin


# --------------------------------------------------------------------------
# queries
# --------------------------------------------------------------------------
def ball_queries(n: int, radius: float = 0.9, seed: int = 1) -> np.ndarray:
    rng = np.random.default_rng(seed)
    g = rng.standard_normal((n, 3))
    g /= np.linalg.norm(g, axis=1, keepdims=True)
    r = radius * rng.random(n) ** (1.0 / 3.0)
    return (g * r[:, None]).astype(np.float32)


def star_slice_queries(shape: StarShape, n_side: int = 256, extent: float = 1.3,
                       margin: float = 1e-2) -> np.ndarray:
    """Cell centres of an n_side^2 grid on [-extent, extent]^2 at z = 0, kept
    where the point is inside the star shape by a radial margin."""
    h = 2 * extent / n_side
    c = -extent + h * (np.arange(n_side) + 0.5)
    X, Y = np.meshgrid(c, c, indexing="ij")
    p = np.stack([X.ravel(), Y.ravel(), np.zeros(X.size)], 1)
    rad = np.linalg.norm(p, axis=1)
    dirs = p / np.maximum(rad, 1e-300)[:, None]
    dirs[rad == 0] = (0.0, 0.0, 1.0)
    keep = rad < shape.radius(dirs) - margin
    return p[keep].astype(np.float32)


def torus_queries(shape: TorusShape, n: int, inside: bool, seed: int = 1,
                  margin: float = 1e-2) -> np.ndarray:
    """n points uniform inside the displaced torus (inside=True) or in the
    box [-2, 2]^2 x [-1, 1] outside it, at least ``margin`` from its tube."""
    rng = np.random.default_rng(seed)
    ext = shape.R + 1.5 * shape.r if inside else 2.0
    zext = 1.5 * shape.r if inside else 1.0
    out = []
    got = 0
    while got < n:
        p = rng.uniform(-1.0, 1.0, (4 * n, 3)) * np.array([ext, ext, zext])
        if inside:
            keep = torus_inside(shape, p, margin)
        else:
            keep = ~torus_inside(shape, p, -margin)
        out.append(p[keep])
        got += int(keep.sum())
    return np.concatenate(out)[:n].astype(np.float32)


def boundary_points(verts: np.ndarray, tris: np.ndarray, n: int, seed: int = 1):
    """Area-uniform points on the mesh and the triangle each lies on."""
    rng = np.random.default_rng(seed)
    v = verts.astype(np.float64)
    a, b, c = v[tris[:, 0]], v[tris[:, 1]], v[tris[:, 2]]
    area = 0.5 * np.linalg.norm(np.cross(b - a, c - a), axis=1)
    prim = rng.choice(tris.shape[0], size=n, p=area / area.sum())
    u1, u2 = rng.random(n), rng.random(n)
    su = np.sqrt(u1)
    p = ((1 - su)[:, None] * a[prim] + (su * (1 - u2))[:, None] * b[prim]
         + (su * u2)[:, None] * c[prim])
    return p.astype(np.float32), prim.astype(np.int32)


# --------------------------------------------------------------------------
# data helpers (harmonic test fields given as plain formulas)
# --------------------------------------------------------------------------
# polynomial coefficient order: 1, x, y, z, x^2, y^2, z^2, xy, yz, zx
POLY_CONFIG1 = (0.0, 0.0, 0.0, 0.5, 1.0, -1.0, 0.0, 0.0, 0.0, 0.0)  # x^2 - y^2 + 0.5 z


def poly_eval(c, p: np.ndarray) -> np.ndarray:
    p = np.asarray(p, np.float64)
    x, y, z = p[..., 0], p[..., 1], p[..., 2]
    return (c[0] + c[1] * x + c[2] * y + c[3] * z + c[4] * x * x + c[5] * y * y + c[6] * z * z
            + c[7] * x * y + c[8] * y * z + c[9] * z * x)


def bump_data(verts: np.ndarray, tris: np.ndarray, n_bumps: int = 6, width: float = 0.05,
              seed: int = 3) -> np.ndarray:
    """Sparse Neumann data as vertex values (P1): zero except for Gaussian
    bumps exp(-(d / width)^2) around ``n_bumps`` area-uniform boundary points
    (seeded) with alternating signs; the negative bumps are scaled so that
    the data integrates to zero over the mesh (a solvable interior Neumann
    problem).  Float32, one value per vertex."""
    c, _ = boundary_points(verts, tris, n_bumps, seed)
    v = verts.astype(np.float64)
    pos = np.zeros(len(v))
    neg = np.zeros(len(v))
    for k in range(n_bumps):
        g = np.exp(-(np.linalg.norm(v - c[k].astype(np.float64), axis=1) / width) ** 2)
        if k % 2 == 0:
            pos += g
        else:
            neg += g
    a, b, cc = v[tris[:, 0]], v[tris[:, 1]], v[tris[:, 2]]
    area = 0.5 * np.linalg.norm(np.cross(b - a, cc - a), axis=1)
    integral = lambda h: float((area * h[tris].mean(axis=1)).sum())
    return (pos - neg * (integral(pos) / integral(neg))).astype(np.float32)


def point_source_eval(x0, p: np.ndarray, scale: float = 1.0) -> np.ndarray:
    p = np.asarray(p, np.float64)
    return scale / np.linalg.norm(p - np.asarray(x0, np.float64), axis=-1)


# --------------------------------------------------------------------------
# many independent problems (the batched workload)
# --------------------------------------------------------------------------
@dataclass
class BatchItem:
    kind: str          # "star" or "torus"
    verts: np.ndarray
    tris: np.ndarray
    queries: np.ndarray
    max_len: int


def _star_points(shape: StarShape, n: int, rng, lo: float = 0.05, hi: float = 0.85):
    g = rng.standard_normal((n, 3))
    g /= np.linalg.norm(g, axis=1, keepdims=True)
    r = shape.radius(g) * (lo + (hi - lo) * rng.random(n))
    return (g * r[:, None]).astype(np.float32)


def _torus_points(shape: TorusShape, n: int, rng, frac: float = 0.8):
    phi = rng.uniform(0, 2 * math.pi, n)
    th = rng.uniform(0, 2 * math.pi, n)
    rho = shape.tube(th, phi) * frac * np.sqrt(rng.random(n))
    x = (shape.R + rho * np.cos(th)) * np.cos(phi)
    y = (shape.R + rho * np.cos(th)) * np.sin(phi)
    return np.stack([x, y, rho * np.sin(th)], 1).astype(np.float32)


def batch_workload(n_problems: int = 512, t_range=(500, 50000), q_range=(64, 16384),
                   m_range=(8, 24), seed: int = 4, q_scale: float = 1.0) -> list:
    """Independent interior Dirichlet problems: each a seeded star-shaped
    icosphere (level nearest to a log-uniform triangle count) or a displaced
    torus (2 nu nv triangles ~ the same target), with a log-uniform number of
    interior query points and a path length uniform in m_range."""
    rng = np.random.default_rng(seed)
    items = []
    for i in range(n_problems):
        kind = "star" if rng.random() < 0.5 else "torus"
        T = math.exp(rng.uniform(math.log(t_range[0]), math.log(t_range[1])))
        Q = max(1, int(round(math.exp(rng.uniform(math.log(q_range[0]), math.log(q_range[1])))
                             * q_scale)))
        M = int(rng.integers(m_range[0], m_range[1] + 1))
        sub = np.random.default_rng([seed, i])
        if kind == "star":
            level = int(min(6, max(2, round(math.log(T / 20.0, 4)))))
            v, f, shape = star_mesh(level, 0.3, 6, int(sub.integers(1 << 30)))
            q = _star_points(shape, Q, sub)
        else:
            nv = max(8, int(round(math.sqrt(T / 5.0))))
            nu = max(8, int(round(2.5 * nv)))
            v, f, shape = displaced_torus(nu, nv, seed=int(sub.integers(1 << 30)))
            q = _torus_points(shape, Q, sub)
        items.append(BatchItem(kind, v, f, q, M))
    return items
