"""CPU oracle for the walk-on-boundary (WoB) estimator -- TEST INFRASTRUCTURE.

Only ``tests/``, ``__graft_entry__.smoke()`` and the ``cpu_baseline`` /
``--impl reference`` legs of ``bench.py`` may import this package.  The
product (the CUDA library under ``paper_2305_04403_gb300``) never imports,
links or calls it, and this package imports nothing from the product.

The arithmetic lives in ``wob_oracle.c`` (plain C, FP64, brute force, its own
Philox4x32-10); this module only marshals numpy arrays through ctypes and
compiles the C file with gcc on first use (or from ``build()``).

Parity notes: every function follows a passage of the paper (cited in the C
file).  Functions with no independent pin are listed in the module
docstring of the test that covers them; at present every exported function
is pinned (see ``tests/test_oracle_*.py``).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "wob_oracle.c")
_OUT_DIR = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_OUT_DIR, "liboracle.so")
_lock = threading.Lock()
_lib = None

KIND_DIRICHLET_DL = 0
KIND_NEUMANN_SL = 1
KIND_ROBIN_SL = 2
KIND_MIXED_SL = 4
BC_DIRICHLET, BC_NEUMANN, BC_ROBIN = 0, 1, 2
DATA_VERTEX_P1 = 0
DATA_POLY = 1
DATA_POINT = 2

# near-degenerate line thresholds (relative edge distance, grazing |d.n|)
TAU = 2e-6
GRAZE = 1e-4


def build(force: bool = False) -> str:
    """Compile ``wob_oracle.c`` into ``oracle/_build/liboracle.so``.  With
    the environment variable ORACLE_PLANT=k (tests of the pins only) a
    variant with planted mistake k is built into ``oracle/_build/plant_k``."""
    plant = int(os.environ.get("ORACLE_PLANT", "0"))
    out_dir = _OUT_DIR if plant == 0 else os.path.join(_OUT_DIR, f"plant_{plant}")
    lib_path = os.path.join(out_dir, "liboracle.so")
    os.makedirs(out_dir, exist_ok=True)
    if (not force and os.path.exists(lib_path)
            and os.path.getmtime(lib_path) >= os.path.getmtime(_SRC)):
        return lib_path
    tmp = lib_path + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-std=c11", "-fopenmp", "-ffp-contract=off", "-fPIC", "-shared",
           f"-DORACLE_PLANT={plant}", "-o", tmp, _SRC, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, lib_path)
    return lib_path


class _Data(ctypes.Structure):
    _fields_ = [("mode", ctypes.c_int32), ("pad", ctypes.c_int32),
                ("vertex_data", ctypes.c_void_p), ("poly", ctypes.c_double * 10),
                ("x0", ctypes.c_double * 3), ("scale", ctypes.c_double)]


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            P = ctypes.c_void_p
            I64, I32, U32, U64, D = (ctypes.c_int64, ctypes.c_int32, ctypes.c_uint32,
                                     ctypes.c_uint64, ctypes.c_double)
            lib.oracle_num_threads.argtypes = [ctypes.c_int]
            lib.oracle_num_threads.restype = ctypes.c_int
            lib.oracle_philox4x32_10.argtypes = [P, P, I64, P]
            lib.oracle_philox4x64_10.argtypes = [P, P, I64, P]
            lib.oracle_line_axes.argtypes = [U64, U32, P, I64, P, P]
            lib.oracle_uniforms.argtypes = [U64, U32, P, I64, P, P]
            lib.oracle_mesh_stats.argtypes = [P, I64, P, I64, P]
            lib.oracle_mesh_stats.restype = ctypes.c_int
            lib.oracle_area_points.argtypes = [P, I64, P, I64, I64, U64, U32, P, P]
            lib.oracle_area_points.restype = ctypes.c_int
            lib.oracle_trace_lines.argtypes = [P, I64, P, I64, P, P, P, P, I64, U64, U32, D, D,
                                               P, P, P, P, P, P, P, ctypes.c_int]
            lib.oracle_trace_lines.restype = ctypes.c_int
            lib.oracle_dl_walks.argtypes = [P, I64, P, I64, ctypes.POINTER(_Data), I32, P, P, I64,
                                            I64, I64, I32, I32, U64, U32, D, D, P, P, P, P, P, P,
                                            P, ctypes.c_int]
            lib.oracle_dl_walks.restype = ctypes.c_int
            lib.oracle_nd_walks.argtypes = lib.oracle_dl_walks.argtypes[:-2] + [ctypes.c_int]
            lib.oracle_nd_walks.restype = ctypes.c_int
            lib.oracle_fwd_paths.argtypes = [P, I64, P, I64, ctypes.POINTER(_Data), I32, I64, I32,
                                             U64, U32, I32, D, D, D, P, P, P, ctypes.c_int]
            lib.oracle_fwd_paths.restype = ctypes.c_int
            lib.oracle_fwd_connect.argtypes = [P, I64, P, P, I64, I32, P, ctypes.c_int]
            lib.oracle_fwd_connect.restype = None
            lib.oracle_sl_walks.argtypes = [P, I64, P, I64, ctypes.POINTER(_Data), I32, D, I32,
                                            P, I64, I64, I64, I32, I32, U64, U32, P, P,
                                            P, D, D, I32, ctypes.c_int]
            lib.oracle_sl_walks.restype = ctypes.c_int
            lib.oracle_reduce.argtypes = [P, I64, I32, P, P]
            _lib = lib
    return _lib


def _p(a: np.ndarray | None):
    return None if a is None else a.ctypes.data_as(ctypes.c_void_p)


def _c(a, dtype):
    return np.ascontiguousarray(a, dtype=dtype)


def num_threads(n: int = 0) -> int:
    return _load().oracle_num_threads(n)


# --------------------------------------------------------------------------
# random numbers
# --------------------------------------------------------------------------
def philox4x32_10(ctr, key) -> np.ndarray:
    ctr = _c(ctr, np.uint32).reshape(-1, 4)
    key = _c(np.broadcast_to(np.asarray(key, np.uint32), (ctr.shape[0], 2)), np.uint32)
    out = np.empty_like(ctr)
    _load().oracle_philox4x32_10(_p(ctr), _p(key), ctr.shape[0], _p(out))
    return out


def philox4x64_10(ctr, key) -> np.ndarray:
    ctr = _c(ctr, np.uint64).reshape(-1, 4)
    key = _c(np.broadcast_to(np.asarray(key, np.uint64), (ctr.shape[0], 2)), np.uint64)
    out = np.empty_like(ctr)
    _load().oracle_philox4x64_10(_p(ctr), _p(key), ctr.shape[0], _p(out))
    return out


def line_axes(seed: int, problem: int, qws) -> tuple[np.ndarray, np.ndarray]:
    """Line axes for (query, walk, step) triples: (n,3) float64, calls used."""
    qws = _c(qws, np.uint32).reshape(-1, 3)
    d = np.empty((qws.shape[0], 3), np.float64)
    calls = np.empty(qws.shape[0], np.int32)
    _load().oracle_line_axes(seed, problem, _p(qws), qws.shape[0], _p(d), _p(calls))
    return d, calls


def uniforms(seed: int, problem: int, qws) -> tuple[np.ndarray, np.ndarray]:
    qws = _c(qws, np.uint32).reshape(-1, 3)
    u53 = np.empty(qws.shape[0], np.float64)
    u24 = np.empty((qws.shape[0], 2), np.float64)
    _load().oracle_uniforms(seed, problem, _p(qws), qws.shape[0], _p(u53), _p(u24))
    return u53, u24


# --------------------------------------------------------------------------
# geometry
# --------------------------------------------------------------------------
def mesh_stats(verts, tris) -> dict:
    v = _c(verts, np.float32)
    t = _c(tris, np.int32)
    out = np.empty(5, np.float64)
    rc = _load().oracle_mesh_stats(_p(v), v.shape[0], _p(t), t.shape[0], _p(out))
    if rc != 0:
        raise RuntimeError("oracle_mesh_stats failed")
    return dict(L=out[0], area=out[1], volume=out[2], min_area=out[3], max_edge=out[4])


def area_points(verts, tris, n: int, seed: int = 0, problem: int = 0):
    """n area-uniform boundary points (float64 positions, triangle ids):
    point i is the area sample of the stream (i, 0, 0)."""
    v = _c(verts, np.float32)
    t = _c(tris, np.int32)
    pts = np.empty((n, 3), np.float64)
    prims = np.empty(n, np.int32)
    rc = _load().oracle_area_points(_p(v), v.shape[0], _p(t), t.shape[0], n, ctypes.c_uint64(seed),
                                    ctypes.c_uint32(problem), _p(pts), _p(prims))
    if rc != 0:
        raise RuntimeError("oracle_area_points failed")
    return pts, prims


def trace_lines(verts, tris, origins, dirs, exclude=None, keys=None, seed: int = 0,
                problem: int = 0, tau: float = TAU, graze: float = GRAZE,
                nthreads: int = 0) -> dict:
    """All-hits queries of explicit lines.  keys: (n,3) (query, walk, step)
    addressing the hit-selection keys (default: (i, 0, 0))."""
    v = _c(verts, np.float32)
    t = _c(tris, np.int32)
    o = _c(origins, np.float64).reshape(-1, 3)
    d = _c(dirs, np.float64).reshape(-1, 3)
    n = o.shape[0]
    ex = None if exclude is None else _c(exclude, np.int32)
    if keys is None:
        keys = np.stack([np.arange(n), np.zeros(n), np.zeros(n)], 1)
    k = _c(keys, np.uint32).reshape(-1, 3)
    res = dict(m=np.empty(n, np.int32), sum_s=np.empty(n, np.int32), prim=np.empty(n, np.int32),
               s=np.empty(n, np.int32), t=np.empty(n, np.float64), y=np.empty((n, 3), np.float64),
               flag=np.empty(n, np.uint8))
    rc = _load().oracle_trace_lines(_p(v), v.shape[0], _p(t), t.shape[0], _p(o), _p(d), _p(ex),
                                    _p(k), n, seed, problem, tau, graze, _p(res["m"]),
                                    _p(res["sum_s"]), _p(res["prim"]), _p(res["s"]), _p(res["t"]),
                                    _p(res["y"]), _p(res["flag"]), nthreads)
    if rc != 0:
        raise RuntimeError("oracle_trace_lines failed")
    return res


def _data(mode: int, vertex_data=None, poly=None, x0=None, scale: float = 1.0):
    d = _Data()
    d.mode = mode
    keep = None
    if vertex_data is not None:
        keep = _c(vertex_data, np.float32)
        d.vertex_data = keep.ctypes.data
    if poly is not None:
        for i, c in enumerate(poly):
            d.poly[i] = float(c)
    if x0 is not None:
        for i, c in enumerate(x0):
            d.x0[i] = float(c)
    d.scale = float(scale)
    return d, keep


def _line_arrays(Q: int, walks: int, max_len: int, want: bool) -> dict:
    """Per-line outputs of the walk functions: hit count, picked triangle,
    near-degenerate flag (None each when not wanted)."""
    shape = (Q, walks, max_len)
    if not want:
        return dict(line_m=None, line_prim=None, line_flag=None)
    return dict(line_m=np.empty(shape, np.int32), line_prim=np.empty(shape, np.int32),
                line_flag=np.empty(shape, np.uint8))


def dl_walks(verts, tris, queries, walks: int, max_len: int, seed: int = 0, problem: int = 0,
             phi: int = 1, mode: int = DATA_POLY, vertex_data=None, poly=None, x0=None,
             scale: float = 1.0, q_offset: int = 0, walk_begin: int = 0, tau: float = TAU,
             graze: float = GRAZE, want_lines: bool = False, nthreads: int = 0,
             query_prim=None, want_grad: bool = False) -> dict:
    """Double-layer Dirichlet walks; with query_prim (the triangle each query
    lies on) the walks start on the boundary and estimate the density nu
    there.  Returns per_walk (Q,N), flag (Q,N),
    abs_terms (Q,N: sum over the walk's terms of |term|, the scale of its
    rounding error), with want_lines per line the hit count line_m, the
    picked triangle line_prim and the near-degenerate flag line_flag
    (Q,N,M), and with want_grad the per-walk gradient estimates grad (3,Q,N)
    of the same walks."""
    v = _c(verts, np.float32)
    t = _c(tris, np.int32)
    q = _c(queries, np.float32).reshape(-1, 3)
    Q = q.shape[0]
    data, keep = _data(mode, vertex_data, poly, x0, scale)
    per_walk = np.empty((Q, walks), np.float64)
    flag = np.empty((Q, walks), np.uint8)
    lines = _line_arrays(Q, walks, max_len, want_lines)
    abs_terms = np.empty((Q, walks), np.float64)
    qp = None if query_prim is None else _c(query_prim, np.int32)
    grad = np.empty((3, Q, walks), np.float64) if want_grad else None
    rc = _load().oracle_dl_walks(_p(v), v.shape[0], _p(t), t.shape[0], ctypes.byref(data), phi,
                                 _p(q), _p(qp), Q, q_offset, walk_begin, walks, max_len, seed,
                                 problem, tau, graze, _p(per_walk), _p(flag),
                                 *[_p(a) for a in lines.values()], _p(abs_terms), _p(grad),
                                 nthreads)
    del keep
    if rc != 0:
        raise RuntimeError("oracle_dl_walks failed")
    out = dict(per_walk=per_walk, flag=flag, abs_terms=abs_terms)
    if want_lines:
        out.update(lines)
    if want_grad:
        out["grad"] = grad
    return out


def nd_walks(verts, tris, queries, walks: int, max_len: int, seed: int = 0, problem: int = 0,
             phi: int = 1, mode: int = DATA_POLY, vertex_data=None, poly=None, x0=None,
             scale: float = 1.0, q_offset: int = 0, walk_begin: int = 0, tau: float = TAU,
             graze: float = GRAZE, want_lines: bool = False, nthreads: int = 0,
             query_prim=None) -> dict:
    """Neumann walks through the direct boundary integral equation (Sec. 4.2):
    lines for the dG/dn_y term, one area sample per vertex for the G q term,
    q = dh/dn of the field (or the P1 vertex data); with query_prim the walks
    start on the boundary.  Returns per_walk, flag, abs_terms (and, with
    want_lines, line_m, line_prim and line_flag as dl_walks)."""
    v = _c(verts, np.float32)
    t = _c(tris, np.int32)
    q = _c(queries, np.float32).reshape(-1, 3)
    Q = q.shape[0]
    data, keep = _data(mode, vertex_data, poly, x0, scale)
    per_walk = np.empty((Q, walks), np.float64)
    flag = np.empty((Q, walks), np.uint8)
    lines = _line_arrays(Q, walks, max_len, want_lines)
    abs_terms = np.empty((Q, walks), np.float64)
    qp = None if query_prim is None else _c(query_prim, np.int32)
    rc = _load().oracle_nd_walks(_p(v), v.shape[0], _p(t), t.shape[0], ctypes.byref(data), phi,
                                 _p(q), _p(qp), Q, q_offset, walk_begin, walks, max_len, seed,
                                 problem, tau, graze, _p(per_walk), _p(flag),
                                 *[_p(a) for a in lines.values()], _p(abs_terms), nthreads)
    del keep
    if rc != 0:
        raise RuntimeError("oracle_nd_walks failed")
    out = dict(per_walk=per_walk, flag=flag, abs_terms=abs_terms)
    if want_lines:
        out.update(lines)
    return out


def fwd_paths(verts, tris, paths: int, max_len: int, seed: int = 0, problem: int = 0,
              phi: int = 1, mode: int = DATA_POINT, vertex_data=None, poly=None, x0=None,
              scale: float = 1.0, start_mode: int = 0, beta: float = 0.1, tau: float = TAU,
              graze: float = GRAZE, nthreads: int = 0) -> dict:
    """Forward single-layer Neumann paths (Sec. 4.4.3): zpos (N, M, 3) vertex
    positions, zw (N, M) vertex weights c_j a_j (0 after a miss), flag (N).
    start_mode 0: area-uniform starts; 1: weighted by |q| per triangle
    (+ beta times its mean, so that every triangle can start a path)."""
    v = _c(verts, np.float32)
    t = _c(tris, np.int32)
    data, keep = _data(mode, vertex_data, poly, x0, scale)
    zpos = np.empty((paths, max_len, 3), np.float64)
    zw = np.empty((paths, max_len), np.float64)
    flag = np.empty(paths, np.uint8)
    rc = _load().oracle_fwd_paths(_p(v), v.shape[0], _p(t), t.shape[0], ctypes.byref(data), phi,
                                  paths, max_len, seed, problem, start_mode, beta, tau, graze,
                                  _p(zpos), _p(zw), _p(flag), nthreads)
    del keep
    if rc != 0:
        raise RuntimeError("oracle_fwd_paths failed")
    return dict(zpos=zpos, zw=zw, flag=flag)


def fwd_connect(queries, zpos, zw, nthreads: int = 0) -> np.ndarray:
    """Per-path values (Q, N) of forward paths at the query points:
    sum_j zw[p, j] G(x_q, z_pj)."""
    q = _c(queries, np.float32).reshape(-1, 3)
    zp = _c(zpos, np.float64)
    w = _c(zw, np.float64)
    N, M = w.shape
    out = np.empty((q.shape[0], N), np.float64)
    _load().oracle_fwd_connect(_p(q), q.shape[0], _p(zp), _p(w), N, M, _p(out), nthreads)
    return out


def sl_walks(verts, tris, queries, walks: int, max_len: int, kind: int = KIND_NEUMANN_SL,
             alpha: float = 0.0, seed: int = 0, problem: int = 0, phi: int = 1,
             mode: int = DATA_POINT, vertex_data=None, poly=None, x0=None, scale: float = 1.0,
             q_offset: int = 0, walk_begin: int = 0, nthreads: int = 0,
             want_abs: bool = False, bc_type=None, kmix: float = 0.0, pk: float = 0.0,
             ris: int = 0):
    """Single-layer Neumann / Robin / mixed walks; per_walk (Q,N) (and, with
    want_abs, the per-walk sum of |term|).  Mixed (kind KIND_MIXED_SL):
    bc_type (T,) uint8 condition per triangle, constant kmix and branch
    probability pk of the Dirichlet parts.  ris > 1: resampled importance
    sampling of the next point from ris uniform candidates."""
    v = _c(verts, np.float32)
    t = _c(tris, np.int32)
    q = _c(queries, np.float32).reshape(-1, 3)
    Q = q.shape[0]
    data, keep = _data(mode, vertex_data, poly, x0, scale)
    per_walk = np.empty((Q, walks), np.float64)
    abs_terms = np.empty((Q, walks), np.float64)
    bc = None if bc_type is None else _c(bc_type, np.uint8)
    rc = _load().oracle_sl_walks(_p(v), v.shape[0], _p(t), t.shape[0], ctypes.byref(data), kind,
                                 alpha, phi, _p(q), Q, q_offset, walk_begin, walks, max_len,
                                 seed, problem, _p(per_walk), _p(abs_terms), _p(bc), kmix, pk,
                                 ris, nthreads)
    del keep
    if rc != 0:
        raise RuntimeError("oracle_sl_walks failed")
    return (per_walk, abs_terms) if want_abs else per_walk


def reduce(per_walk) -> tuple[np.ndarray, np.ndarray]:
    pw = _c(per_walk, np.float64)
    Q, N = pw.shape
    est = np.empty(Q, np.float64)
    var = np.empty(Q, np.float64)
    _load().oracle_reduce(_p(pw), Q, N, _p(est), _p(var))
    return est, var
