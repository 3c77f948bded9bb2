"""Oracle for the learned control variate -- TEST INFRASTRUCTURE.

Plain FP64 numpy.  Reading of the method (the paper has no control variate;
its nearest ideas are boundary caching, Sec. 3.2, and path reuse, Sec. 5):

  nu = nu_t + rho, where nu solves nu = H nu + 2 phi g (Table 1, Dirichlet,
  source density) and nu_t is a learned approximation; then
      rho = H rho + r,   r = 2 phi g - nu_t + H nu_t,
      u(x0) = D nu_t (x0) + D rho (x0),
  with (H f)(x) = 2 phi int dG/dn_y(x, y) f(y) dA_y on Gamma and
  (D f)(x0) = -int dG/dn_y(x0, y) f(y) dA_y, dG/dn_y = -(r . n_y)/(4 pi r^3)
  (App. A).  D nu_t and H nu_t are computed by quadrature; the walk runs the
  double-layer recursion of Sec. 4.1 with r in place of 2 phi g (and half of
  it on the last vertex, Sec. 4.1.2).  nu_t = 0 gives plain WoB exactly.

Monte Carlo variant (cv_walks_mc, for meshes too large for quadrature):
D nu_t (x0) and H nu_t (x_i) are each the mean of K one-line estimates --
K independent all-hits lines from the point, weights (m/2) s from the query
and -phi m s from a boundary vertex, the walk's own line weights -- so every
term stays unbiased; only the variance grows.

Quadrature: Radon's 7-point rule of degree 5 on every triangle; triangles
whose centroid lies within `near` mesh edge lengths of the target point are
split into 4^level sub-triangles, each with the same rule.  For H at a
boundary point x, nu_t(y) - nu_t(x) is integrated and H[1](x) = -phi is
added back (Gauss: int dG/dn_y dA = -1/2 on a closed surface); the target's
own (flat) triangle contributes nothing.

MLP (nu_t): 16 Fourier frequencies 2^(k/3), k = 0..15, sin and cos of
2 pi f y_d for each coordinate (96 features), four hidden layers of width
64 with SiLU, one linear output; He-uniform weights, zero biases; MSE loss;
Adam.  Weights are stored in the out x in layout.
"""
from __future__ import annotations

import math

import numpy as np

import oracle as O

FREQS = 2.0 ** (np.arange(16) / 3.0)
N_FEAT = 96
WIDTH = 64
LAYERS = [(N_FEAT, WIDTH), (WIDTH, WIDTH), (WIDTH, WIDTH), (WIDTH, WIDTH), (WIDTH, 1)]


# --------------------------------------------------------------------------
# MLP
# --------------------------------------------------------------------------
def features(y: np.ndarray) -> np.ndarray:
    """Column c = 32 d + 2 k + s: s = 0 -> sin, 1 -> cos of 2 pi f_k y_d."""
    y = np.asarray(y, np.float64).reshape(-1, 3)
    out = np.empty((y.shape[0], N_FEAT))
    for d in range(3):
        arg = 2.0 * math.pi * y[:, d:d + 1] * FREQS[None, :]
        out[:, 32 * d + 0:32 * d + 32:2] = np.sin(arg)
        out[:, 32 * d + 1:32 * d + 32:2] = np.cos(arg)
    return out


def mlp_init(seed: int = 2) -> list:
    """[(W (out x in), b (out,)), ...] He-uniform weights, zero biases."""
    rng = np.random.default_rng(seed)
    params = []
    for fan_in, fan_out in LAYERS:
        lim = math.sqrt(6.0 / fan_in)
        params.append((rng.uniform(-lim, lim, (fan_out, fan_in)), np.zeros(fan_out)))
    return params


def mlp_init_counter(seed: int = 2) -> np.ndarray:
    """He-uniform parameters (flat, float32) from the counter-based stream:
    weight i (flat index) of a layer with fan-in f is sqrt(6/f) (2u - 1),
    u = (x >> 8) 2^-24 for x the first word of Philox4x32-10 at counter
    (i, 0, 3 << 12, 0), key (seed_lo, seed_hi); biases 0."""
    n = N_PARAMS
    ctr = np.zeros((n, 4), np.uint32)
    ctr[:, 0] = np.arange(n, dtype=np.uint32)
    ctr[:, 2] = 3 << 12
    key = np.tile(np.array([seed & 0xFFFFFFFF, seed >> 32], np.uint32), (n, 1))
    x = O.philox4x32_10(ctr, key)[:, 0]
    u = (x >> 8).astype(np.float64) * 2.0 ** -24
    flat = np.zeros(n, np.float32)
    o = 0
    for fan_in, fan_out in LAYERS:
        lim = np.float32(math.sqrt(6.0 / fan_in))
        sl = slice(o, o + fan_in * fan_out)
        flat[sl] = lim * (np.float32(2.0) * u[sl].astype(np.float32) - np.float32(1.0))
        o += fan_in * fan_out + fan_out
    return flat


def flatten(params) -> np.ndarray:
    return np.concatenate([np.concatenate([W.ravel(), b.ravel()]) for W, b in params])


def unflatten(flat: np.ndarray) -> list:
    params, o = [], 0
    for fan_in, fan_out in LAYERS:
        W = flat[o:o + fan_in * fan_out].reshape(fan_out, fan_in)
        o += fan_in * fan_out
        b = flat[o:o + fan_out]
        o += fan_out
        params.append((W.astype(np.float64), b.astype(np.float64)))
    return params


N_PARAMS = sum(i * o + o for i, o in LAYERS)


def _silu(a):
    return a / (1.0 + np.exp(-a))


def mlp_forward(params, y, feat=None):
    """Returns (output (n,), cache)."""
    h = features(y) if feat is None else feat
    cache = [h]
    for li, (W, b) in enumerate(params):
        a = h @ W.T + b
        if li < len(params) - 1:
            cache.append(a)
            h = _silu(a)
            cache.append(h)
        else:
            h = a
    return h[:, 0], cache


def mlp_backward(params, cache, dout):
    """Gradients [(dW, db), ...] of sum(dout * output)."""
    grads = [None] * len(params)
    g = dout[:, None]
    n_hidden = len(params) - 1
    for li in range(len(params) - 1, -1, -1):
        W, b = params[li]
        h_in = cache[0] if li == 0 else cache[2 * li]
        grads[li] = (g.T @ h_in, g.sum(0))
        if li == 0:
            break
        gh = g @ W
        a = cache[2 * li - 1]
        s = 1.0 / (1.0 + np.exp(-a))
        g = gh * (s * (1.0 + a * (1.0 - s)))
    assert n_hidden == 4
    return grads


class Adam:
    """Kingma & Ba (2015) with bias correction."""

    def __init__(self, n: int, lr: float = 1e-3, b1: float = 0.9, b2: float = 0.999,
                 eps: float = 1e-8):
        self.m = np.zeros(n)
        self.v = np.zeros(n)
        self.t = 0
        self.lr, self.b1, self.b2, self.eps = lr, b1, b2, eps

    def step(self, flat: np.ndarray, grad: np.ndarray) -> np.ndarray:
        self.t += 1
        self.m = self.b1 * self.m + (1 - self.b1) * grad
        self.v = self.b2 * self.v + (1 - self.b2) * grad * grad
        mh = self.m / (1 - self.b1 ** self.t)
        vh = self.v / (1 - self.b2 ** self.t)
        return flat - self.lr * mh / (np.sqrt(vh) + self.eps)


def mse_grad(params, y, target):
    """Loss = mean (out - target)^2 and its flat gradient."""
    out, cache = mlp_forward(params, y)
    diff = out - target
    grads = mlp_backward(params, cache, 2.0 * diff / len(target))
    flat = np.concatenate([np.concatenate([dW.ravel(), db.ravel()]) for dW, db in grads])
    return float(np.mean(diff * diff)), flat


# --------------------------------------------------------------------------
# quadrature
# --------------------------------------------------------------------------
def radon7():
    """Radon's 7-point degree-5 rule on the triangle: barycentric points
    (3, 7) and weights summing to 1 (multiply by the triangle area)."""
    s15 = math.sqrt(15.0)
    a1, b1 = (6.0 - s15) / 21.0, (9.0 + 2.0 * s15) / 21.0
    a2, b2 = (6.0 + s15) / 21.0, (9.0 - 2.0 * s15) / 21.0
    w1, w2 = (155.0 - s15) / 1200.0, (155.0 + s15) / 1200.0
    pts = [(1 / 3, 1 / 3, 1 / 3),
           (b1, a1, a1), (a1, b1, a1), (a1, a1, b1),
           (b2, a2, a2), (a2, b2, a2), (a2, a2, b2)]
    w = [9.0 / 40.0, w1, w1, w1, w2, w2, w2]
    return np.array(pts), np.array(w)


def subdivide_bary(level: int) -> np.ndarray:
    """Barycentric corners (4^level, 3, 3) of a uniform split."""
    tris = [np.eye(3)]
    for _ in range(level):
        nxt = []
        for T in tris:
            a, b, c = T
            ab, bc, ca = (a + b) / 2, (b + c) / 2, (c + a) / 2
            nxt += [np.array([a, ab, ca]), np.array([b, bc, ab]), np.array([c, ca, bc]),
                    np.array([ab, bc, ca])]
        tris = nxt
    return np.array(tris)


class Nodes:
    """Quadrature nodes of a mesh: coarse (7 per triangle) and fine
    (7 * 4^level per triangle).  Arrays per node: position, weight
    (rule weight x area), owning triangle; per triangle: unit normal,
    centroid, longest edge."""

    def __init__(self, verts, tris, level: int = 2):
        v = np.asarray(verts, np.float64)
        t = np.asarray(tris, np.int64)
        A, B, C = v[t[:, 0]], v[t[:, 1]], v[t[:, 2]]
        N = np.cross(B - A, C - A)
        area = 0.5 * np.linalg.norm(N, axis=1)
        self.normal = N / (2.0 * area[:, None])
        self.centroid = (A + B + C) / 3.0
        self.h = np.max(np.stack([np.linalg.norm(B - A, axis=1), np.linalg.norm(C - B, axis=1),
                                  np.linalg.norm(A - C, axis=1)], 1), 1)
        self.T = len(t)
        bp, bw = radon7()
        corners = np.stack([A, B, C], 1)                      # T, 3, 3
        self.coarse_pos = np.einsum("qk,tkd->tqd", bp, corners)  # T, 7, 3
        self.coarse_w = area[:, None] * bw[None, :]            # T, 7
        sub = subdivide_bary(level)                            # S, 3, 3 (sub corner, bary)
        fine_b = np.einsum("qk,skj->sqj", bp, sub).reshape(-1, 3)   # S*7, 3
        fine_w = np.tile(bw, len(sub)) / len(sub)
        self.fine_pos = np.einsum("qk,tkd->tqd", fine_b, corners)
        self.fine_w = area[:, None] * fine_w[None, :]
        self.mean_h = float(np.mean(self.h))

    def values(self, fn):
        """Evaluate fn at coarse and fine nodes -> (T x 7, T x F)."""
        c = fn(self.coarse_pos.reshape(-1, 3)).reshape(self.T, -1)
        f = fn(self.fine_pos.reshape(-1, 3)).reshape(self.T, -1)
        return c, f


def _kernel_sum(x, pos, w, n, vals):
    """sum over nodes of w (r . n)/(4 pi r^3) vals, r = y - x."""
    r = pos - x[None, :]
    rl = np.linalg.norm(r, axis=1)
    return np.sum(w * np.einsum("ij,ij->i", r, n) / (4.0 * math.pi * rl ** 3) * vals)


def quad_D(nodes: Nodes, vals, x0, near: float = 3.0):
    """(D f)(x0) = -int dG/dn_y f dA = int (r.n)/(4 pi r^3) f dA."""
    cv, fv = vals
    x0 = np.asarray(x0, np.float64)
    dist = np.linalg.norm(nodes.centroid - x0[None, :], axis=1)
    is_near = dist < near * nodes.h
    tot = 0.0
    for sel, pos, w, v in ((~is_near, nodes.coarse_pos, nodes.coarse_w, cv),
                           (is_near, nodes.fine_pos, nodes.fine_w, fv)):
        if not sel.any():
            continue
        k = pos.shape[1]
        tot += _kernel_sum(x0, pos[sel].reshape(-1, 3), w[sel].ravel(),
                           np.repeat(nodes.normal[sel], k, 0), v[sel].ravel())
    return tot


def quad_H(nodes: Nodes, vals, x, prim: int, fx: float, phi: int = 1, near: float = 3.0):
    """(H f)(x) for x on triangle prim: 2 phi int dG/dn_y (f(y) - f(x)) dA - phi f(x)."""
    cv, fv = vals
    x = np.asarray(x, np.float64)
    dist = np.linalg.norm(nodes.centroid - x[None, :], axis=1)
    is_near = dist < near * nodes.h
    own = np.zeros(nodes.T, bool)
    own[prim] = True
    tot = 0.0
    for sel, pos, w, v in ((~is_near & ~own, nodes.coarse_pos, nodes.coarse_w, cv),
                           (is_near & ~own, nodes.fine_pos, nodes.fine_w, fv)):
        if not sel.any():
            continue
        k = pos.shape[1]
        tot += _kernel_sum(x, pos[sel].reshape(-1, 3), w[sel].ravel(),
                           np.repeat(nodes.normal[sel], k, 0), v[sel].ravel() - fx)
    # dG/dn_y = -(r.n)/(4 pi r^3): the sum above is -int dG/dn_y (f - f(x))
    return -2.0 * phi * tot - phi * fx


# --------------------------------------------------------------------------
# walks
# --------------------------------------------------------------------------
def cv_walks(verts, tris, queries, walks: int, max_len: int, params, nodes: Nodes, node_vals,
             poly, seed: int = 0, problem: int = 0, phi: int = 1, tau: float = O.TAU,
             near: float = 3.0):
    """Residual walks for D rho (per walk values, Q x N) and D nu_t per query.
    Data: the harmonic polynomial `poly` evaluated at the walk's vertices.
    `params`: the network's parameters, or a callable nu_t on (n, 3) points
    (node_vals must then hold nu_t at the nodes); None means nu_t = 0 (then
    the walks are plain WoB)."""
    q = np.asarray(queries, np.float32).reshape(-1, 3)
    Q = q.shape[0]
    nw = Q * walks
    qi = np.repeat(np.arange(Q), walks)
    wi = np.tile(np.arange(walks), Q)
    x = q.astype(np.float64)[qi]
    excl = np.full(nw, -1, np.int32)
    S = np.zeros(nw)
    P = np.ones(nw)
    alive = np.ones(nw, bool)
    flag = np.zeros(nw, bool)
    for k in range(max_len):
        idx = np.nonzero(alive)[0]
        if idx.size == 0:
            break
        keys = np.stack([qi[idx], wi[idx], np.full(idx.size, k)], 1)
        d, _ = O.line_axes(seed, problem, keys)
        r = O.trace_lines(verts, tris, x[idx], d, exclude=excl[idx], keys=keys, seed=seed,
                          problem=problem, tau=tau)
        flag[idx] |= r["flag"].astype(bool)
        hit = r["m"] > 0
        dead = idx[~hit]
        alive[dead] = False
        idx, m, s, y, prim = idx[hit], r["m"][hit], r["s"][hit], r["y"][hit], r["prim"][hit]
        ms = m.astype(np.float64) * s
        P[idx] = 0.5 * ms if k == 0 else P[idx] * (-phi * ms)
        g = _poly(poly, y)
        if params is None:
            src = 2.0 * phi * g
        else:
            nt = params(y) if callable(params) else mlp_forward(params, y)[0]
            hn = np.array([quad_H(nodes, node_vals, y[j], prim[j], nt[j], phi, near)
                           for j in range(len(idx))])
            src = 2.0 * phi * g - nt + hn
        c = 0.5 if k == max_len - 1 else 1.0
        S[idx] += P[idx] * c * src
        x[idx] = y
        excl[idx] = prim
    Dnt = np.zeros(Q)
    if params is not None:
        Dnt = np.array([quad_D(nodes, node_vals, q[j].astype(np.float64), near)
                        for j in range(Q)])
    return S.reshape(Q, walks), flag.reshape(Q, walks), Dnt


MC_WALK_BIT = 0x80000000   # walk-index bit of the extra lines' streams


def _mc_lines(verts, tris, x, excl, qi, wi, v, K, nu_t, first, phi, seed, problem, tau):
    """K independent lines from each point x (its own triangle excl), the
    pick y_j and its weight: (m/2) s from a query (first), -phi m s from a
    boundary vertex (Table 1 kernels over the line-pick density, Sec. 4.4.1);
    returns (1/K) sum_j weight_j nu_t(y_j) and the lines' flags."""
    n = x.shape[0]
    acc = np.zeros(n)
    flag = np.zeros(n, bool)
    for j in range(K):
        keys = np.stack([qi, wi | MC_WALK_BIT, np.full(n, v * K + j)], 1).astype(np.uint32)
        d, _ = O.line_axes(seed, problem, keys)
        r = O.trace_lines(verts, tris, x, d, exclude=excl, keys=keys, seed=seed,
                          problem=problem, tau=tau)
        flag |= r["flag"].astype(bool)
        hit = r["m"] > 0
        if not hit.any():
            continue
        ms = r["m"][hit].astype(np.float64) * r["s"][hit]
        wgt = 0.5 * ms if first else -phi * ms
        acc[hit] += wgt * nu_t(r["y"][hit])
    return acc / K, flag


def cv_walks_mc(verts, tris, queries, walks: int, max_len: int, nu_t, K: int, poly,
                seed: int = 0, problem: int = 0, phi: int = 1, tau: float = O.TAU):
    """Residual walks with Monte Carlo estimates of the control variate's
    integrals (no quadrature; for meshes too large for it):
        u(x0) ~ D^ nu_t (x0) + sum_k P_k c_k r^(x_k),
        r^ = 2 phi g - nu_t + H^ nu_t,
    D^ and H^ the means over K independent all-hits lines from the point,
    each an unbiased one-sample estimate of D nu_t resp. H nu_t (the walk's
    own first and later line weights).  The extra lines of vertex v (0 = the
    query) are the streams (query, walk | 2^31, v K + j).  nu_t: callable on
    (n, 3) points, or None for nu_t = 0 (plain WoB).  Returns the per-walk
    values (Q, N) and flags (Q, N) (a walk is flagged if any of its lines,
    its own or an extra one, is near-degenerate)."""
    q = np.asarray(queries, np.float32).reshape(-1, 3)
    Q = q.shape[0]
    nw = Q * walks
    qi = np.repeat(np.arange(Q), walks).astype(np.int64)
    wi = np.tile(np.arange(walks), Q).astype(np.int64)
    x = q.astype(np.float64)[qi]
    excl = np.full(nw, -1, np.int32)
    S = np.zeros(nw)
    P = np.ones(nw)
    alive = np.ones(nw, bool)
    flag = np.zeros(nw, bool)
    zero = nu_t is None
    if not zero:
        S, f0 = _mc_lines(verts, tris, x, excl, qi, wi, 0, K, nu_t, True, phi, seed, problem, tau)
        flag |= f0
    for k in range(max_len):
        idx = np.nonzero(alive)[0]
        if idx.size == 0:
            break
        keys = np.stack([qi[idx], wi[idx], np.full(idx.size, k)], 1)
        d, _ = O.line_axes(seed, problem, keys)
        r = O.trace_lines(verts, tris, x[idx], d, exclude=excl[idx], keys=keys, seed=seed,
                          problem=problem, tau=tau)
        flag[idx] |= r["flag"].astype(bool)
        hit = r["m"] > 0
        alive[idx[~hit]] = False
        idx, m, s, y, prim = idx[hit], r["m"][hit], r["s"][hit], r["y"][hit], r["prim"][hit]
        ms = m.astype(np.float64) * s
        P[idx] = 0.5 * ms if k == 0 else P[idx] * (-phi * ms)
        src = 2.0 * phi * _poly(poly, y)
        if not zero:
            h, fl = _mc_lines(verts, tris, y, prim, qi[idx], wi[idx], k + 1, K, nu_t, False, phi,
                              seed, problem, tau)
            flag[idx] |= fl
            src = src - nu_t(y) + h
        c = 0.5 if k == max_len - 1 else 1.0
        S[idx] += P[idx] * c * src
        x[idx] = y
        excl[idx] = prim
    return S.reshape(Q, walks), flag.reshape(Q, walks)


def _poly(c, p):
    x, y, z = p[:, 0], p[:, 1], p[:, 2]
    return (c[0] + c[1] * x + c[2] * y + c[3] * z + c[4] * x * x + c[5] * y * y + c[6] * z * z
            + c[7] * x * y + c[8] * y * z + c[9] * z * x)
