"""wob_solve_noalloc, the entry point for callers that cannot allocate
device memory (a process whose GPU memory belongs to its own allocator, or a
path that cannot take an allocation and its synchronisation).  It must give
the same estimates as wob_solve, whose scratch is allocated per call, on two
calls in a row (the second reuses the library's fixed array, which still
holds the first call's values), accept the largest size its fixed array
holds, reject larger ones, and allocate nothing: the device's memory pool
(where the library's stream-ordered allocations come from) keeps its
high-water mark across the call.

Kept in a file pytest collects last so that a run stopping at the first
failure has already run every other test; it also passes on its own.
"""
import ctypes

import numpy as np
import pytest

from paper_2305_04403_gb300 import inputs as I

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

MAX_BLOCKS = 1 << 19  # (query, 32-walk block) partial sums the fixed array holds


@pytest.fixture(scope="module")
def wob():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2305_04403_gb300 import build as B
    B.build()
    import paper_2305_04403_gb300 as w
    return w


def _noalloc(wob, prob, q, walks, max_len, seed, est=None, var=None):
    """Call wob_solve_noalloc through the C ABI with caller-owned outputs."""
    lib = wob.load_library()
    Q = q.shape[0]
    if est is None:
        est = torch.full((Q,), np.nan, dtype=torch.float64, device="cuda")
        var = torch.full((Q,), np.nan, dtype=torch.float64, device="cuda")
    pc = prob._c()
    stream = torch.cuda.current_stream()
    rc = lib.wob_solve_noalloc(ctypes.byref(pc), ctypes.c_void_p(q.data_ptr()), None, Q, walks,
                               max_len, seed, ctypes.c_void_p(est.data_ptr()),
                               ctypes.c_void_p(var.data_ptr()),
                               ctypes.c_void_p(stream.cuda_stream))
    return rc, est, var


def test_noalloc_matches_wob_solve_twice(wob):
    v, f = I.icosphere(3)
    mesh = wob.build_mesh(v, f)
    bvh = wob.build_bvh(mesh)
    prob = wob.Problem(bvh, kind=wob.DIRICHLET_DL, side=1, data_mode=wob.DATA_POLY,
                       poly=I.POLY_CONFIG1)
    scale = float(np.abs(I.poly_eval(I.POLY_CONFIG1, v)).max())
    # two different calls in a row: the second overwrites the shared array
    for n_q, walks, max_len, seed in ((256, 64, 4, 0), (500, 96, 6, 11)):
        q = torch.from_numpy(I.ball_queries(n_q, 0.9, seed + 1)).cuda()
        est_ref, var_ref = wob.solve(prob, q, walks, max_len, seed=seed)
        rc, est, var = _noalloc(wob, prob, q, walks, max_len, seed)
        torch.cuda.synchronize()
        assert rc == 0, wob.load_library().wob_last_error()
        tol = 1e-12 * scale
        assert torch.allclose(est, est_ref, rtol=0, atol=tol)
        assert torch.allclose(var, var_ref, rtol=1e-12, atol=tol)


def test_noalloc_direct_neumann_matches(wob):
    """Every kind takes its own walk kernel here too (the direct-BIE Neumann
    walks, not the single-layer ones)."""
    v, f = I.icosphere(2)
    mesh = wob.build_mesh(v, f)
    bvh = wob.build_bvh(mesh)
    prob = wob.Problem(bvh, kind=wob.NEUMANN_DIRECT, side=1, data_mode=wob.DATA_POLY,
                       poly=(0, 0, 0, 1, 0, 0, 0, 0, 0, 0))
    q = torch.from_numpy(I.ball_queries(96, 0.8, 6)).cuda()
    for seed in (2, 3):
        est_ref, var_ref = wob.solve(prob, q, 64, 3, seed=seed)
        rc, est, var = _noalloc(wob, prob, q, 64, 3, seed)
        torch.cuda.synchronize()
        assert rc == 0
        assert torch.allclose(est, est_ref, rtol=0, atol=1e-12 * est_ref.abs().max().item())


def test_noalloc_single_layer_matches(wob):
    v, f = I.icosphere(2)
    mesh = wob.build_mesh(v, f)
    bvh = wob.build_bvh(mesh)
    prob = wob.Problem(bvh, kind=wob.NEUMANN_SL, side=1, data_mode=wob.DATA_POINT,
                       x0=(0.0, 0.0, 3.0))
    q = torch.from_numpy(I.ball_queries(128, 0.8, 5)).cuda()
    est_ref, var_ref = wob.solve(prob, q, 128, 3, seed=4)
    rc, est, var = _noalloc(wob, prob, q, 128, 3, 4)
    torch.cuda.synchronize()
    assert rc == 0
    assert torch.allclose(est, est_ref, rtol=0, atol=1e-12 * est_ref.abs().max().item())


def test_noalloc_largest_size_and_oversized_work(wob):
    v, f = I.icosphere(1)
    mesh = wob.build_mesh(v, f)
    bvh = wob.build_bvh(mesh)
    prob = wob.Problem(bvh, data_mode=wob.DATA_POLY, poly=I.POLY_CONFIG1)
    # the largest size: Q * ceil(1024 / 32) = 2^19 blocks
    q = torch.from_numpy(I.ball_queries(MAX_BLOCKS // 32, 0.5, 1)).cuda()
    est_ref, _ = wob.solve(prob, q, 1024, 4, seed=3)
    rc, est, var = _noalloc(wob, prob, q, 1024, 4, 3)
    torch.cuda.synchronize()
    assert rc == 0, wob.load_library().wob_last_error()
    assert torch.allclose(est, est_ref, rtol=0, atol=1e-12)
    # one query more does not fit
    q = torch.from_numpy(I.ball_queries(MAX_BLOCKS // 32 + 1, 0.5, 1)).cuda()
    rc, est, var = _noalloc(wob, prob, q, 1024, 4, 0)
    assert rc == -1
    assert b"exceeds" in wob.load_library().wob_last_error()
    torch.cuda.synchronize()
    assert torch.isnan(est).all()  # nothing was launched


class _Pool:
    """High-water mark of the current device's memory pool (the pool that
    stream-ordered allocations draw from), read through the driver API."""

    USED_MEM_HIGH = 8  # CU_MEMPOOL_ATTR_USED_MEM_HIGH

    def __init__(self):
        self.cu = ctypes.CDLL("libcuda.so.1")
        dev = ctypes.c_int()
        assert self.cu.cuCtxGetDevice(ctypes.byref(dev)) == 0
        self.pool = ctypes.c_void_p()
        assert self.cu.cuDeviceGetMemPool(ctypes.byref(self.pool), dev) == 0

    def reset(self):
        zero = ctypes.c_uint64(0)
        assert self.cu.cuMemPoolSetAttribute(self.pool, self.USED_MEM_HIGH, ctypes.byref(zero)) == 0

    def high(self) -> int:
        v = ctypes.c_uint64()
        assert self.cu.cuMemPoolGetAttribute(self.pool, self.USED_MEM_HIGH, ctypes.byref(v)) == 0
        return v.value


def test_noalloc_allocates_nothing(wob):
    v, f = I.icosphere(3)
    mesh = wob.build_mesh(v, f)
    bvh = wob.build_bvh(mesh)
    prob = wob.Problem(bvh, data_mode=wob.DATA_POLY, poly=I.POLY_CONFIG1)
    q = torch.from_numpy(I.ball_queries(512, 0.9, 2)).cuda()
    rc, _, _ = _noalloc(wob, prob, q, 64, 4, 0)  # first call on the device: set-up
    torch.cuda.synchronize()
    assert rc == 0
    pool = _Pool()
    # the detector sees the stream-ordered scratch that wob_solve allocates
    torch.cuda.synchronize()
    pool.reset()
    base = pool.high()
    wob.solve(prob, q, 64, 4, seed=1)
    torch.cuda.synchronize()
    assert pool.high() > base
    # ... and wob_solve_noalloc leaves the high-water mark where it was
    est = torch.empty(512, dtype=torch.float64, device="cuda")
    var = torch.empty_like(est)
    torch.cuda.synchronize()
    pool.reset()
    base = pool.high()
    rc, est, var = _noalloc(wob, prob, q, 64, 4, 1, est, var)
    torch.cuda.synchronize()
    assert rc == 0
    assert pool.high() == base
