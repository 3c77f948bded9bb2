"""GB300-native walk-on-boundary (WoB) estimator -- Python binding.

Thin ctypes layer over ``libwob.so`` (built from ``csrc/`` for sm_103a by
``paper_2305_04403_gb300.build``); every step of the estimator runs in the
library's CUDA kernels.  Functions take and return torch tensors on the
GPU (torch provides device memory and streams only) and carry the names of
the C entry points in ``include/wob.h``.  If the library is not built the
first call raises; there is no CPU fallback.
"""
from __future__ import annotations

import ctypes
import os
import threading
from dataclasses import dataclass, field

import numpy as np

from . import build as _build

__all__ = [
    "DIRICHLET_DL", "NEUMANN_SL", "ROBIN_SL", "NEUMANN_DIRECT", "MIXED_SL", "BC_DIRICHLET",
    "BC_NEUMANN", "BC_ROBIN", "DATA_VERTEX_P1", "DATA_POLY", "DATA_POINT",
    "WobError", "Mesh", "BVH", "Problem", "Batch", "build_mesh", "build_bvh", "solve", "solve_range",
    "solve_debug", "solve_counted", "solve_host", "solve_noalloc", "solve_density",
    "solve_batched", "get_stats",
    "mlp_num_params", "mlp_forward", "mlp_train_step", "debug_set_tc_wait_limit", "ControlVariate", "trace_lines", "line_axes", "philox4x32_10",
    "library_path", "load_library",
]

DIRICHLET_DL, NEUMANN_SL, ROBIN_SL, NEUMANN_DIRECT, MIXED_SL = 0, 1, 2, 3, 4
BC_DIRICHLET, BC_NEUMANN, BC_ROBIN = 0, 1, 2
DATA_VERTEX_P1, DATA_POLY, DATA_POINT = 0, 1, 2

_ERRORS = {-1: "INVALID_ARG", -2: "CUDA", -3: "OOM", -4: "TIMEOUT", -5: "DEGENERATE_MESH",
           -6: "UNSUPPORTED", -7: "DEVICE_CHECK"}


class WobError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"WOB_ERR_{_ERRORS.get(code, code)}: {msg}")
        self.code = code


class _MeshInfo(ctypes.Structure):
    _fields_ = [("V", ctypes.c_int64), ("T", ctypes.c_int64), ("bbox_lo", ctypes.c_double * 3),
                ("bbox_hi", ctypes.c_double * 3), ("L", ctypes.c_double),
                ("area", ctypes.c_double), ("volume", ctypes.c_double),
                ("max_edge", ctypes.c_double)]


class _BvhParams(ctypes.Structure):
    _fields_ = [("leaf_size", ctypes.c_int32), ("reserved", ctypes.c_int32 * 7)]


class _BvhInfo(ctypes.Structure):
    _fields_ = [("nodes", ctypes.c_int64), ("leaves", ctypes.c_int64), ("depth", ctypes.c_int32),
                ("leaf_size", ctypes.c_int32), ("bytes", ctypes.c_int64)]


class _Problem(ctypes.Structure):
    _fields_ = [("bvh", ctypes.c_void_p), ("kind", ctypes.c_int32), ("side", ctypes.c_int32),
                ("alpha", ctypes.c_float), ("data_mode", ctypes.c_int32),
                ("vertex_data", ctypes.c_void_p), ("poly", ctypes.c_float * 10),
                ("x0", ctypes.c_float * 3), ("scale", ctypes.c_float),
                ("problem", ctypes.c_uint32), ("tau", ctypes.c_float),
                ("bc_type", ctypes.c_void_p), ("k_mix", ctypes.c_float), ("p_k", ctypes.c_float),
                ("ris", ctypes.c_int32), ("iter_limit", ctypes.c_int32)]


class _BatchParams(ctypes.Structure):
    _fields_ = [("tile_rounds", ctypes.c_int32), ("order", ctypes.c_int32),
                ("autotune", ctypes.c_int32), ("reserved", ctypes.c_int32 * 5)]


class _BatchInfo(ctypes.Structure):
    _fields_ = [("P", ctypes.c_int32), ("tile_rounds", ctypes.c_int32), ("order", ctypes.c_int32),
                ("from_cache", ctypes.c_int32), ("queries", ctypes.c_int64),
                ("walks", ctypes.c_int64), ("max_lines", ctypes.c_int64),
                ("tiles", ctypes.c_int64), ("tune_ms", ctypes.c_double * 8)]


class _DebugOut(ctypes.Structure):
    _fields_ = [("per_walk", ctypes.c_void_p), ("walk_flag", ctypes.c_void_p),
                ("line_m", ctypes.c_void_p), ("line_prim", ctypes.c_void_p),
                ("line_flag", ctypes.c_void_p)]


class _CvTrainParams(ctypes.Structure):
    _fields_ = [("points", ctypes.c_int64), ("walks", ctypes.c_int32),
                ("max_len", ctypes.c_int32), ("point_seed", ctypes.c_uint64),
                ("walk_seed", ctypes.c_uint64), ("epochs", ctypes.c_int32),
                ("batch", ctypes.c_int32), ("lr", ctypes.c_float), ("lr_end", ctypes.c_float),
                ("tail_epochs", ctypes.c_int32), ("step0", ctypes.c_int32)]


class _Stats(ctypes.Structure):
    _fields_ = [("lines", ctypes.c_int64), ("node_visits", ctypes.c_int64),
                ("tri_tests", ctypes.c_int64), ("hits", ctypes.c_int64),
                ("flagged", ctypes.c_int64)]


_lock = threading.Lock()
_lib = None


def library_path() -> str:
    return _build.LIB


def load_library() -> ctypes.CDLL:
    """Load libwob.so (raises if it has not been built)."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        if not os.path.exists(_build.LIB):
            raise RuntimeError(f"{_build.LIB} is missing: build it with "
                               "paper_2305_04403_gb300.build.build()")
        lib = ctypes.CDLL(_build.LIB)
        P, I64, I32, U32, U64, F = (ctypes.c_void_p, ctypes.c_int64, ctypes.c_int32,
                                    ctypes.c_uint32, ctypes.c_uint64, ctypes.c_float)
        sig = {
            "wob_version": ([], ctypes.c_int),
            "wob_last_error": ([], ctypes.c_char_p),
            "wob_build_mesh": ([P, I64, P, I64, ctypes.c_int, P, ctypes.POINTER(P)], ctypes.c_int),
            "wob_mesh_get_info": ([P, ctypes.POINTER(_MeshInfo)], ctypes.c_int),
            "wob_destroy_mesh": ([P], None),
            "wob_build_bvh": ([P, ctypes.POINTER(_BvhParams), P, ctypes.POINTER(P)], ctypes.c_int),
            "wob_bvh_get_info": ([P, ctypes.POINTER(_BvhInfo)], ctypes.c_int),
            "wob_destroy_bvh": ([P], None),
            "wob_solve": ([ctypes.POINTER(_Problem), P, P, I64, I32, I32, U64, P, P, P],
                          ctypes.c_int),
            "wob_solve_range": ([ctypes.POINTER(_Problem), P, P, I64, I64, I32, I32, U64, P, P, P],
                                ctypes.c_int),
            "wob_solve_debug": ([ctypes.POINTER(_Problem), P, P, I64, I32, I32, U64, P, P,
                                 ctypes.POINTER(_DebugOut), P], ctypes.c_int),
            "wob_solve_counted": ([ctypes.POINTER(_Problem), P, P, I64, I32, I32, U64, P, P,
                                   ctypes.POINTER(_Stats), P], ctypes.c_int),
            "wob_solve_host": ([ctypes.POINTER(_Problem), P, P, I64, I32, I32, U64, P, P, P],
                               ctypes.c_int),
            "wob_solve_noalloc": ([ctypes.POINTER(_Problem), P, P, I64, I32, I32, U64, P, P, P],
                                  ctypes.c_int),
            "wob_trace_lines": ([P, P, P, P, P, I64, U64, U32, F, P, P, P, P, P, P, P, P],
                                ctypes.c_int),
            "wob_solve_density": ([ctypes.POINTER(_Problem), P, P, I64, I32, I32, U64, P, P, P],
                                  ctypes.c_int),
            "wob_solve_grad": ([ctypes.POINTER(_Problem), P, I64, I32, I32, U64, P, P, P, P, P, P],
                               ctypes.c_int),
            "wob_solve_forward": ([ctypes.POINTER(_Problem), P, I64, I32, I32, U64, I32, F, P, P,
                                   P, P, P, P], ctypes.c_int),
            "wob_mlp_num_params": ([], ctypes.c_int),
            "wob_mlp_init": ([P, U64, P], ctypes.c_int),
            "wob_mlp_forward": ([P, P, I64, P, P], ctypes.c_int),
            "wob_debug_set_tc_wait_limit": ([U32, ctypes.POINTER(U32)], ctypes.c_int),
            "wob_mlp_train_step": ([P, P, P, P, P, I64, F, I32, P, P, P], ctypes.c_int),
            "wob_cv_create": ([P, I32, F, P, ctypes.POINTER(P)], ctypes.c_int),
            "wob_cv_set_network": ([P, P, P], ctypes.c_int),
            "wob_cv_set_node_values": ([P, P, P, P], ctypes.c_int),
            "wob_cv_get_nodes": ([P, P, P, P], ctypes.c_int),
            "wob_cv_get_info": ([P, ctypes.POINTER(I32), ctypes.POINTER(I32),
                                 ctypes.POINTER(I64)], ctypes.c_int),
            "wob_cv_quad_D": ([P, P, I64, P, P], ctypes.c_int),
            "wob_cv_quad_H": ([P, I32, P, P, P, I64, P, P], ctypes.c_int),
            "wob_cv_solve": ([ctypes.POINTER(_Problem), P, P, P, I64, I64, I32, I32, U64, P, P, P,
                              P, P], ctypes.c_int),
            "wob_cv_destroy": ([P], None),
            "wob_probe_l2_read": ([P, I64, I32, P, P], ctypes.c_int),
            "wob_cv_solve_mc": ([ctypes.POINTER(_Problem), P, P, I64, I64, I32, I32, I32, U64, P,
                                 P, P, P], ctypes.c_int),
            "wob_sample_boundary": ([P, I64, U64, U32, P, P, P], ctypes.c_int),
            "wob_cv_train": ([ctypes.POINTER(_Problem), P, ctypes.POINTER(_CvTrainParams), P, P, P,
                              P, P], ctypes.c_int),
            "wob_batch_create": ([P, I32, P, P, P, P, P, P, ctypes.POINTER(_BatchParams), P,
                                  ctypes.POINTER(P)], ctypes.c_int),
            "wob_batch_run": ([P, U64, P], ctypes.c_int),
            "wob_solve_batched": ([P, I32, P, P, P, P, U64, P, P, P], ctypes.c_int),
            "wob_get_stats": ([ctypes.POINTER(_Stats)], ctypes.c_int),
            "wob_batch_get_info": ([P, ctypes.POINTER(_BatchInfo)], ctypes.c_int),
            "wob_batch_destroy": ([P], None),
            "wob_line_axes": ([U64, U32, P, I64, P, P], ctypes.c_int),
            "wob_philox4x32_10": ([P, P, I64, P, P], ctypes.c_int),
        }
        for name, (args, res) in sig.items():
            fn = getattr(lib, name)
            fn.argtypes = args
            fn.restype = res
        _lib = lib
        return lib


def _check(rc: int):
    if rc != 0:
        msg = load_library().wob_last_error()
        raise WobError(rc, msg.decode() if msg else "")


def _stream(stream=None):
    import torch
    s = stream if stream is not None else torch.cuda.current_stream()
    return ctypes.c_void_p(s.cuda_stream)


def _ptr(t):
    return None if t is None else ctypes.c_void_p(t.data_ptr())


def _dev(x, dtype):
    """Contiguous CUDA tensor of dtype from a tensor or array."""
    import torch
    if isinstance(x, torch.Tensor):
        t = x.to(device="cuda", dtype=dtype)
    else:
        t = torch.as_tensor(np.asarray(x), dtype=dtype, device="cuda")
    return t.contiguous()


class Mesh:
    """A device-resident triangle mesh (wob_build_mesh)."""

    def __init__(self, verts, tris, stream=None):
        import torch
        lib = load_library()
        v = _dev(verts, torch.float32).reshape(-1, 3)
        t = _dev(tris, torch.int32).reshape(-1, 3)
        h = ctypes.c_void_p()
        _check(lib.wob_build_mesh(_ptr(v), v.shape[0], _ptr(t), t.shape[0], 1, _stream(stream),
                                  ctypes.byref(h)))
        self._h = h
        self.V, self.T = v.shape[0], t.shape[0]

    @property
    def handle(self):
        return self._h

    def info(self) -> dict:
        i = _MeshInfo()
        _check(load_library().wob_mesh_get_info(self._h, ctypes.byref(i)))
        return dict(V=i.V, T=i.T, bbox_lo=list(i.bbox_lo), bbox_hi=list(i.bbox_hi), L=i.L,
                    area=i.area, volume=i.volume, max_edge=i.max_edge)

    def __del__(self):
        h = getattr(self, "_h", None)
        if h and _lib is not None:
            _lib.wob_destroy_mesh(h)
            self._h = None


class BVH:
    """Bounding-volume hierarchy over a mesh (wob_build_bvh)."""

    def __init__(self, mesh: Mesh, leaf_size: int = 1, stream=None):
        lib = load_library()
        p = _BvhParams()
        p.leaf_size = leaf_size
        h = ctypes.c_void_p()
        _check(lib.wob_build_bvh(mesh.handle, ctypes.byref(p), _stream(stream), ctypes.byref(h)))
        self._h = h
        self.mesh = mesh  # keeps the mesh alive

    @property
    def handle(self):
        return self._h

    def info(self) -> dict:
        i = _BvhInfo()
        _check(load_library().wob_bvh_get_info(self._h, ctypes.byref(i)))
        return dict(nodes=i.nodes, leaves=i.leaves, depth=i.depth, leaf_size=i.leaf_size,
                    bytes=i.bytes)

    def __del__(self):
        h = getattr(self, "_h", None)
        if h and _lib is not None:
            _lib.wob_destroy_bvh(h)
            self._h = None


def build_mesh(verts, tris, stream=None) -> Mesh:
    return Mesh(verts, tris, stream)


def build_bvh(mesh: Mesh, leaf_size: int = 1, stream=None) -> BVH:
    return BVH(mesh, leaf_size, stream)


@dataclass
class Problem:
    """One boundary value problem (the wob_problem struct)."""
    bvh: BVH
    kind: int = DIRICHLET_DL
    side: int = 1
    alpha: float = 0.0
    data_mode: int = DATA_POLY
    vertex_data: object = None          # device float tensor (V,) in P1 mode
    poly: tuple = (0.0,) * 10
    x0: tuple = (0.0, 0.0, 0.0)
    scale: float = 1.0
    problem: int = 0
    tau: float = 0.0
    bc_type: object = None              # device uint8 tensor (T,) for MIXED_SL
    k_mix: float = 0.0
    p_k: float = 0.0
    ris: int = 0
    iter_limit: int = 0                 # 0: automatic traversal bound
    _keep: list = field(default_factory=list, repr=False)

    def _c(self) -> _Problem:
        import torch
        p = _Problem()
        self._keep = []
        p.bvh = self.bvh.handle
        p.kind, p.side, p.alpha, p.data_mode = self.kind, self.side, self.alpha, self.data_mode
        if self.vertex_data is not None:
            vd = _dev(self.vertex_data, torch.float32)
            self._keep.append(vd)
            p.vertex_data = vd.data_ptr()
        for i, c in enumerate(self.poly):
            p.poly[i] = float(c)
        for i, c in enumerate(self.x0):
            p.x0[i] = float(c)
        p.scale, p.problem, p.tau = self.scale, self.problem, self.tau
        if self.bc_type is not None:
            bc = _dev(self.bc_type, torch.uint8)
            self._keep.append(bc)
            p.bc_type = bc.data_ptr()
        p.k_mix, p.p_k, p.ris = self.k_mix, self.p_k, self.ris
        p.iter_limit = self.iter_limit
        return p


class Batch:
    """Many double-layer problems in one graph-captured launch
    (wob_batch_create / wob_batch_run).  `queries` is a list of per-problem
    (Q_p, 3) arrays; est / var are (sum Q_p,) float64 CUDA tensors that every
    run overwrites; `split()` returns them per problem."""

    def __init__(self, problems, queries, walks, max_len, tile_rounds: int | None = None,
                 order: int | None = None, stream=None):
        import torch
        lib = load_library()
        P = len(problems)
        qs = [np.asarray(q, np.float32).reshape(-1, 3) for q in queries]
        self.offsets = np.zeros(P + 1, np.int64)
        self.offsets[1:] = np.cumsum([len(q) for q in qs])
        self.queries = _dev(np.concatenate(qs, 0) if P else np.zeros((0, 3), np.float32),
                            torch.float32)
        Qt = int(self.offsets[-1])
        self.est = torch.empty(Qt, dtype=torch.float64, device="cuda")
        self.var = torch.empty(Qt, dtype=torch.float64, device="cuda")
        self._probs = (_Problem * P)(*[p._c() for p in problems])
        self._keep = problems
        w = np.ascontiguousarray(np.broadcast_to(np.asarray(walks, np.int32), (P,)))
        m = np.ascontiguousarray(np.broadcast_to(np.asarray(max_len, np.int32), (P,)))
        self.walks, self.max_len = w, m
        bp = _BatchParams()
        bp.autotune = 1 if tile_rounds is None else 0
        bp.tile_rounds = tile_rounds or 1
        bp.order = order or 0
        h = ctypes.c_void_p()
        _check(lib.wob_batch_create(self._probs, P, self.offsets.ctypes.data_as(ctypes.c_void_p),
                                    w.ctypes.data_as(ctypes.c_void_p),
                                    m.ctypes.data_as(ctypes.c_void_p), _ptr(self.queries),
                                    _ptr(self.est), _ptr(self.var), ctypes.byref(bp),
                                    _stream(stream), ctypes.byref(h)))
        self._h = h

    def run(self, seed: int = 0, stream=None):
        _check(load_library().wob_batch_run(self._h, seed, _stream(stream)))
        return self.est, self.var

    def info(self) -> dict:
        i = _BatchInfo()
        _check(load_library().wob_batch_get_info(self._h, ctypes.byref(i)))
        return dict(P=i.P, tile_rounds=i.tile_rounds, order=i.order, from_cache=i.from_cache,
                    queries=i.queries, walks=i.walks, max_lines=i.max_lines, tiles=i.tiles,
                    tune_ms=list(i.tune_ms)[:6])

    def split(self):
        e, v = self.est.cpu().numpy(), self.var.cpu().numpy()
        o = self.offsets
        return [(e[o[i]:o[i + 1]], v[o[i]:o[i + 1]]) for i in range(len(o) - 1)]

    def __del__(self):
        h = getattr(self, "_h", None)
        if h and _lib is not None:
            _lib.wob_batch_destroy(h)
            self._h = None


def solve_batched(problems, queries, walks, max_len, seed: int = 0, stream=None):
    """wob_solve_batched: one-shot batched solve of double-layer problems;
    `queries` a list of per-problem (Q_p, 3) arrays, walks / max_len ints or
    per-problem lists.  Returns (est, var) per problem as numpy arrays."""
    import torch
    P = len(problems)
    qs = [np.asarray(q, np.float32).reshape(-1, 3) for q in queries]
    off = np.zeros(P + 1, np.int64)
    off[1:] = np.cumsum([len(q) for q in qs])
    qd = _dev(np.concatenate(qs, 0) if P else np.zeros((0, 3), np.float32), torch.float32)
    est = torch.empty(int(off[-1]), dtype=torch.float64, device="cuda")
    var = torch.empty_like(est)
    probs = (_Problem * P)(*[p._c() for p in problems])
    w = np.ascontiguousarray(np.broadcast_to(np.asarray(walks, np.int32), (P,)))
    m = np.ascontiguousarray(np.broadcast_to(np.asarray(max_len, np.int32), (P,)))
    _check(load_library().wob_solve_batched(probs, P, off.ctypes.data_as(ctypes.c_void_p),
                                            _ptr(qd), w.ctypes.data_as(ctypes.c_void_p),
                                            m.ctypes.data_as(ctypes.c_void_p), seed, _ptr(est),
                                            _ptr(var), _stream(stream)))
    e, v = est.cpu().numpy(), var.cpu().numpy()
    return [(e[off[i]:off[i + 1]], v[off[i]:off[i + 1]]) for i in range(P)]


def get_stats() -> dict:
    """wob_get_stats: counters of this thread's last wob_solve_counted call."""
    st = _Stats()
    _check(load_library().wob_get_stats(ctypes.byref(st)))
    return dict(lines=st.lines, node_visits=st.node_visits, tri_tests=st.tri_tests, hits=st.hits,
                flagged=st.flagged)


def solve(problem: Problem, queries, walks: int, max_len: int, seed: int = 0,
          query_prim=None, stream=None):
    """wob_solve: (est, var) float64 CUDA tensors of length Q."""
    import torch
    q = _dev(queries, torch.float32).reshape(-1, 3)
    qp = None if query_prim is None else _dev(query_prim, torch.int32)
    Q = q.shape[0]
    est = torch.empty(Q, dtype=torch.float64, device="cuda")
    var = torch.empty(Q, dtype=torch.float64, device="cuda")
    pc = problem._c()
    _check(load_library().wob_solve(ctypes.byref(pc), _ptr(q), _ptr(qp), Q, walks, max_len,
                                    seed, _ptr(est), _ptr(var), _stream(stream)))
    return est, var


def solve_noalloc(problem: Problem, queries, walks: int, max_len: int, seed: int = 0,
                  query_prim=None, stream=None):
    """wob_solve_noalloc: wob_solve without any device allocation by the
    library (Q * walks <= 2^20; see include/wob.h).  The est / var tensors
    are allocated here by torch, i.e. by the caller."""
    import torch
    q = _dev(queries, torch.float32).reshape(-1, 3)
    qp = None if query_prim is None else _dev(query_prim, torch.int32)
    Q = q.shape[0]
    est = torch.empty(Q, dtype=torch.float64, device="cuda")
    var = torch.empty(Q, dtype=torch.float64, device="cuda")
    pc = problem._c()
    _check(load_library().wob_solve_noalloc(ctypes.byref(pc), _ptr(q), _ptr(qp), Q, walks,
                                            max_len, seed, _ptr(est), _ptr(var),
                                            _stream(stream)))
    return est, var


def solve_grad(problem: Problem, queries, walks: int, max_len: int, seed: int = 0,
               per_walk: bool = False, stream=None) -> dict:
    """wob_solve_grad: est, var (Q,), grad_est, grad_var (3, Q) and, with
    per_walk, the per-walk gradients (3, Q, walks) of the same walks."""
    import torch
    q = _dev(queries, torch.float32).reshape(-1, 3)
    Q = q.shape[0]
    out = dict(est=torch.empty(Q, dtype=torch.float64, device="cuda"),
               var=torch.empty(Q, dtype=torch.float64, device="cuda"),
               grad_est=torch.empty((3, Q), dtype=torch.float64, device="cuda"),
               grad_var=torch.empty((3, Q), dtype=torch.float64, device="cuda"))
    if per_walk:
        out["grad"] = torch.empty((3, Q, walks), dtype=torch.float64, device="cuda")
    pc = problem._c()
    _check(load_library().wob_solve_grad(ctypes.byref(pc), _ptr(q), Q, walks, max_len, seed,
                                         _ptr(out["est"]), _ptr(out["var"]), _ptr(out["grad_est"]),
                                         _ptr(out["grad_var"]), _ptr(out.get("grad")),
                                         _stream(stream)))
    return out


def solve_forward(problem: Problem, queries, paths: int, max_len: int, seed: int = 0,
                  start_mode: int = 1, beta: float = 0.1, want_paths: bool = False,
                  stream=None) -> dict:
    """wob_solve_forward: est, var (Q,) and, with want_paths, the path
    vertices zpos (paths, max_len, 3), weights zw (paths, max_len) and
    near-degenerate flags (paths,)."""
    import torch
    q = _dev(queries, torch.float32).reshape(-1, 3)
    Q = q.shape[0]
    out = dict(est=torch.empty(Q, dtype=torch.float64, device="cuda"),
               var=torch.empty(Q, dtype=torch.float64, device="cuda"))
    if want_paths:
        out["zpos"] = torch.empty((paths, max_len, 3), dtype=torch.float64, device="cuda")
        out["zw"] = torch.empty((paths, max_len), dtype=torch.float64, device="cuda")
        out["flag"] = torch.empty(paths, dtype=torch.uint8, device="cuda")
    pc = problem._c()
    _check(load_library().wob_solve_forward(ctypes.byref(pc), _ptr(q), Q, paths, max_len, seed,
                                            start_mode, beta, _ptr(out["est"]), _ptr(out["var"]),
                                            _ptr(out.get("zpos")), _ptr(out.get("zw")),
                                            _ptr(out.get("flag")), _stream(stream)))
    return out


def solve_density(problem: Problem, points, prims, walks: int, max_len: int, seed: int = 0,
                  stream=None):
    """wob_solve_density: (est, var) of the density nu at boundary points."""
    import torch
    q = _dev(points, torch.float32).reshape(-1, 3)
    pr = _dev(prims, torch.int32)
    Q = q.shape[0]
    est = torch.empty(Q, dtype=torch.float64, device="cuda")
    var = torch.empty(Q, dtype=torch.float64, device="cuda")
    pc = problem._c()
    _check(load_library().wob_solve_density(ctypes.byref(pc), _ptr(q), _ptr(pr), Q, walks,
                                            max_len, seed, _ptr(est), _ptr(var), _stream(stream)))
    return est, var


def sample_boundary(mesh: Mesh, n: int, seed: int = 0, problem: int = 0, stream=None):
    """wob_sample_boundary: (points (n, 3) float32, prims (n,) int32) on the device."""
    import torch
    pts = torch.empty((n, 3), dtype=torch.float32, device="cuda")
    prims = torch.empty(n, dtype=torch.int32, device="cuda")
    _check(load_library().wob_sample_boundary(mesh.handle, n, seed, problem, _ptr(pts),
                                              _ptr(prims), _stream(stream)))
    return pts, prims


def mlp_num_params() -> int:
    return load_library().wob_mlp_num_params()


def mlp_init(seed: int = 2, stream=None):
    """wob_mlp_init: He-uniform parameters (CUDA float32, n_params)."""
    import torch
    p = torch.empty(mlp_num_params(), dtype=torch.float32, device="cuda")
    _check(load_library().wob_mlp_init(_ptr(p), seed, _stream(stream)))
    return p


def debug_set_tc_wait_limit(polls: int) -> int:
    """wob_debug_set_tc_wait_limit: polls of the first wait on each
    tensor-core product (0: give up at once); returns the previous value."""
    prev = ctypes.c_uint32(0)
    _check(load_library().wob_debug_set_tc_wait_limit(polls, ctypes.byref(prev)))
    return prev.value


def mlp_forward(params, x, stream=None):
    """wob_mlp_forward: the network at points x (n, 3) -> (n,) float32."""
    import torch
    pp = _dev(params, torch.float32)
    xx = _dev(x, torch.float32).reshape(-1, 3)
    out = torch.empty(xx.shape[0], dtype=torch.float32, device="cuda")
    _check(load_library().wob_mlp_forward(_ptr(pp), _ptr(xx), xx.shape[0], _ptr(out),
                                          _stream(stream)))
    return out


def mlp_train_step(params, adam_m, adam_v, x, target, lr: float, step: int, grad=None,
                   loss=None, stream=None):
    """wob_mlp_train_step on CUDA float32 tensors (params / adam_m / adam_v
    updated in place)."""
    _check(load_library().wob_mlp_train_step(
        _ptr(params), _ptr(adam_m), _ptr(adam_v), _ptr(x), _ptr(target), x.shape[0], lr, step,
        _ptr(grad), _ptr(loss), _stream(stream)))


class ControlVariate:
    """Quadrature nodes of a mesh and the residual walks (wob_cv_*)."""

    def __init__(self, mesh: Mesh, level: int = 2, near: float = 2.0, stream=None):
        h = ctypes.c_void_p()
        _check(load_library().wob_cv_create(mesh.handle, level, near, _stream(stream),
                                            ctypes.byref(h)))
        self._h = h
        self.mesh = mesh
        T, F, nc = ctypes.c_int32(), ctypes.c_int32(), ctypes.c_int64()
        _check(load_library().wob_cv_get_info(h, ctypes.byref(T), ctypes.byref(F), ctypes.byref(nc)))
        self.T, self.F, self.candidates = T.value, F.value, nc.value

    def nodes(self):
        """(coarse (T, 7, 4), fine (T, F, 4)) float32 host copies: position, weight."""
        import torch
        c = torch.empty(self.T * 7 * 4, dtype=torch.float32, device="cuda")
        f = torch.empty(self.T * self.F * 4, dtype=torch.float32, device="cuda")
        _check(load_library().wob_cv_get_nodes(self._h, _ptr(c), _ptr(f), _stream(None)))
        return (c.cpu().numpy().reshape(self.T, 7, 4), f.cpu().numpy().reshape(self.T, self.F, 4))

    def set_network(self, params, stream=None):
        import torch
        self._params = _dev(params, torch.float32)
        _check(load_library().wob_cv_set_network(self._h, _ptr(self._params), _stream(stream)))

    def set_node_values(self, coarse, fine, stream=None):
        import torch
        c = _dev(coarse, torch.float32)
        f = _dev(fine, torch.float32)
        _check(load_library().wob_cv_set_node_values(self._h, _ptr(c), _ptr(f), _stream(stream)))
        torch.cuda.synchronize()

    def quad_D(self, points, stream=None):
        import torch
        pts = _dev(points, torch.float32).reshape(-1, 3)
        out = torch.empty(pts.shape[0], dtype=torch.float32, device="cuda")
        _check(load_library().wob_cv_quad_D(self._h, _ptr(pts), pts.shape[0], _ptr(out),
                                            _stream(stream)))
        return out

    def quad_H(self, points, prims, fx, phi: int = 1, stream=None):
        import torch
        pts = _dev(points, torch.float32).reshape(-1, 3)
        pr = _dev(prims, torch.int32)
        f = _dev(fx, torch.float32)
        out = torch.empty(pts.shape[0], dtype=torch.float32, device="cuda")
        _check(load_library().wob_cv_quad_H(self._h, phi, _ptr(pts), _ptr(pr), _ptr(f),
                                            pts.shape[0], _ptr(out), _stream(stream)))
        return out

    def solve_range(self, problem: Problem, params, queries, walk_begin: int, walks: int,
                    max_len: int, sum_, sumsq, seed: int = 0, per_walk=None, dnt=None,
                    stream=None):
        import torch
        pp = _dev(params, torch.float32)
        q = _dev(queries, torch.float32).reshape(-1, 3)
        pc = problem._c()
        _check(load_library().wob_cv_solve(ctypes.byref(pc), self._h, _ptr(pp), _ptr(q),
                                           q.shape[0], walk_begin, walks, max_len, seed,
                                           _ptr(sum_), _ptr(sumsq), _ptr(per_walk), _ptr(dnt),
                                           _stream(stream)))

    def train(self, problem: Problem, params, adam_m, adam_v, points: int = 1 << 20,
              walks: int = 64, max_len: int = 4, point_seed: int = 3, walk_seed: int = 0,
              epochs: int = 1, batch: int = 4096, lr: float = 1e-3, lr_end: float = 1e-4,
              tail_epochs: int = 0, step0: int = 0, want_loss: bool = True, stream=None):
        """wob_cv_train: params / adam_m / adam_v (CUDA float32) updated in
        place; returns the per-step minibatch losses (epochs x steps)."""
        import torch
        steps = -(-points // min(batch, points))
        loss = (torch.empty((epochs, steps), dtype=torch.float32, device="cuda")
                if want_loss else None)
        tp = _CvTrainParams(points, walks, max_len, point_seed, walk_seed, epochs, batch, lr, lr_end,
                            tail_epochs, step0)
        pc = problem._c()
        _check(load_library().wob_cv_train(ctypes.byref(pc), self._h, ctypes.byref(tp),
                                           _ptr(params), _ptr(adam_m), _ptr(adam_v), _ptr(loss),
                                           _stream(stream)))
        self._params = params
        return loss

    def __del__(self):
        h = getattr(self, "_h", None)
        if h and _lib is not None:
            _lib.wob_cv_destroy(h)
            self._h = None


def probe_l2_read(buf, passes: int, out, stream=None):
    """wob_probe_l2_read: `passes` streaming reads of the CUDA tensor buf
    (L1 bypassed); out (CUDA float32 scalar) receives the sum."""
    _check(load_library().wob_probe_l2_read(_ptr(buf), buf.numel() * buf.element_size(), passes,
                                            _ptr(out), _stream(stream)))


def cv_solve_mc(problem: Problem, params, queries, walk_begin: int, walks: int, max_len: int,
                K: int, sum_, sumsq, seed: int = 0, per_walk=None, stream=None):
    """wob_cv_solve_mc: residual walks with Monte Carlo integrals of the
    control variate (K extra lines per point); sum_ / sumsq accumulated."""
    import torch
    pp = _dev(params, torch.float32)
    q = _dev(queries, torch.float32).reshape(-1, 3)
    pc = problem._c()
    _check(load_library().wob_cv_solve_mc(ctypes.byref(pc), _ptr(pp), _ptr(q), q.shape[0],
                                          walk_begin, walks, max_len, K, seed, _ptr(sum_),
                                          _ptr(sumsq), _ptr(per_walk), _stream(stream)))


def solve_range(problem: Problem, queries, walk_begin: int, walks: int, max_len: int,
                sum_, sumsq, seed: int = 0, query_prim=None, stream=None):
    """wob_solve_range: accumulates into the float64 tensors sum_ and sumsq."""
    import torch
    q = _dev(queries, torch.float32).reshape(-1, 3)
    qp = None if query_prim is None else _dev(query_prim, torch.int32)
    pc = problem._c()
    _check(load_library().wob_solve_range(ctypes.byref(pc), _ptr(q), _ptr(qp), q.shape[0],
                                          walk_begin, walks, max_len, seed, _ptr(sum_),
                                          _ptr(sumsq), _stream(stream)))


def solve_debug(problem: Problem, queries, walks: int, max_len: int, seed: int = 0,
                query_prim=None, want_lines: bool = True, stream=None) -> dict:
    """wob_solve_debug: est, var and per-walk values and flags; with
    want_lines also per line the hit count line_m, the picked triangle
    line_prim and the near-degenerate flag line_flag (Q, walks, max_len)."""
    import torch
    q = _dev(queries, torch.float32).reshape(-1, 3)
    qp = None if query_prim is None else _dev(query_prim, torch.int32)
    Q = q.shape[0]
    out = dict(est=torch.empty(Q, dtype=torch.float64, device="cuda"),
               var=torch.empty(Q, dtype=torch.float64, device="cuda"),
               per_walk=torch.empty((Q, walks), dtype=torch.float64, device="cuda"),
               flag=torch.zeros((Q, walks), dtype=torch.uint8, device="cuda"))
    if want_lines:
        shape = (Q, walks, max_len)
        out["line_m"] = torch.empty(shape, dtype=torch.int32, device="cuda")
        out["line_prim"] = torch.empty(shape, dtype=torch.int32, device="cuda")
        out["line_flag"] = torch.zeros(shape, dtype=torch.uint8, device="cuda")
    dbg = _DebugOut(out["per_walk"].data_ptr(), out["flag"].data_ptr(),
                    *((out["line_m"].data_ptr(), out["line_prim"].data_ptr(),
                       out["line_flag"].data_ptr()) if want_lines else (None, None, None)))
    pc = problem._c()
    _check(load_library().wob_solve_debug(ctypes.byref(pc), _ptr(q), _ptr(qp), Q, walks, max_len,
                                          seed, _ptr(out["est"]), _ptr(out["var"]),
                                          ctypes.byref(dbg), _stream(stream)))
    return out


def solve_counted(problem: Problem, queries, walks: int, max_len: int, seed: int = 0,
                  query_prim=None, stream=None):
    """wob_solve_counted: (est, var, stats dict)."""
    import torch
    q = _dev(queries, torch.float32).reshape(-1, 3)
    qp = None if query_prim is None else _dev(query_prim, torch.int32)
    Q = q.shape[0]
    est = torch.empty(Q, dtype=torch.float64, device="cuda")
    var = torch.empty(Q, dtype=torch.float64, device="cuda")
    st = _Stats()
    pc = problem._c()
    _check(load_library().wob_solve_counted(ctypes.byref(pc), _ptr(q), _ptr(qp), Q, walks,
                                            max_len, seed, _ptr(est), _ptr(var),
                                            ctypes.byref(st), _stream(stream)))
    return est, var, dict(lines=st.lines, node_visits=st.node_visits, tri_tests=st.tri_tests,
                          hits=st.hits, flagged=st.flagged)


def solve_host(problem: Problem, queries: np.ndarray, walks: int, max_len: int, seed: int = 0,
               query_prim: np.ndarray | None = None, stream=None):
    """wob_solve_host: host numpy in, host numpy (est, var) out."""
    q = np.ascontiguousarray(queries, np.float32).reshape(-1, 3)
    qp = None if query_prim is None else np.ascontiguousarray(query_prim, np.int32)
    Q = q.shape[0]
    est = np.empty(Q, np.float64)
    var = np.empty(Q, np.float64)
    pc = problem._c()
    _check(load_library().wob_solve_host(
        ctypes.byref(pc), q.ctypes.data_as(ctypes.c_void_p),
        None if qp is None else qp.ctypes.data_as(ctypes.c_void_p), Q, walks, max_len, seed,
        est.ctypes.data_as(ctypes.c_void_p), var.ctypes.data_as(ctypes.c_void_p),
        _stream(stream)))
    return est, var


def trace_lines(bvh: BVH, origins, dirs, exclude=None, keys=None, seed: int = 0,
                problem: int = 0, tau: float = 0.0, stream=None) -> dict:
    """wob_trace_lines on explicit lines; returns CUDA tensors."""
    import torch
    o = _dev(origins, torch.float64).reshape(-1, 3)
    d = _dev(dirs, torch.float64).reshape(-1, 3)
    n = o.shape[0]
    ex = None if exclude is None else _dev(exclude, torch.int32)
    if keys is None:
        keys = np.stack([np.arange(n), np.zeros(n), np.zeros(n)], 1)
    k = _dev(np.asarray(keys, np.int64).astype(np.uint32).view(np.int32), torch.int32).reshape(-1, 3)
    dev = dict(device="cuda")
    out = dict(m=torch.empty(n, dtype=torch.int32, **dev), sum_s=torch.empty(n, dtype=torch.int32, **dev),
               prim=torch.empty(n, dtype=torch.int32, **dev), s=torch.empty(n, dtype=torch.int32, **dev),
               t=torch.empty(n, dtype=torch.float64, **dev), y=torch.empty((n, 3), dtype=torch.float64, **dev),
               flag=torch.empty(n, dtype=torch.uint8, **dev))
    _check(load_library().wob_trace_lines(
        bvh.handle, _ptr(o), _ptr(d), _ptr(ex), _ptr(k), n, seed, problem, tau, _ptr(out["m"]),
        _ptr(out["sum_s"]), _ptr(out["prim"]), _ptr(out["s"]), _ptr(out["t"]), _ptr(out["y"]),
        _ptr(out["flag"]), _stream(stream)))
    return out


def line_axes(seed: int, problem: int, qws, stream=None):
    """wob_line_axes: (n,3) float64 CUDA tensor."""
    import torch
    k = _dev(np.asarray(qws, np.int64).astype(np.uint32).view(np.int32), torch.int32).reshape(-1, 3)
    d = torch.empty((k.shape[0], 3), dtype=torch.float64, device="cuda")
    _check(load_library().wob_line_axes(seed, problem, _ptr(k), k.shape[0], _ptr(d),
                                        _stream(stream)))
    return d


def philox4x32_10(ctr, key, stream=None):
    """wob_philox4x32_10 on (n,4) counters and (n,2) keys (uint32 values)."""
    import torch
    c = _dev(np.asarray(ctr, np.uint64).astype(np.uint32).view(np.int32), torch.int32).reshape(-1, 4)
    kk = np.broadcast_to(np.asarray(key, np.uint64), (c.shape[0], 2))
    k = _dev(np.ascontiguousarray(kk).astype(np.uint32).view(np.int32), torch.int32).reshape(-1, 2)
    out = torch.empty_like(c)
    _check(load_library().wob_philox4x32_10(_ptr(c), _ptr(k), c.shape[0], _ptr(out),
                                            _stream(stream)))
    return out
