"""Edge cases of the newer entry points: empty query sets are no-ops
(nothing launched, accumulators untouched), the largest accepted path
length runs and one beyond is refused, and every problem kind accepts a
walk count that is not a multiple of the 32-walk warp tile; wob_get_stats
returns the last counted solve's counters."""
import numpy as np
import pytest

from paper_2305_04403_gb300 import inputs as I

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


@pytest.fixture(scope="module")
def sphere(wob):
    v, f = I.icosphere(2)
    return wob.build_bvh(wob.build_mesh(v, f))


def test_empty_queries_are_no_ops(wob, sphere):
    none = np.zeros((0, 3), np.float32)
    dl = wob.Problem(sphere, data_mode=wob.DATA_POLY, poly=I.POLY_CONFIG1)
    out = wob.solve_grad(dl, none, 8, 4)
    assert all(t.numel() == 0 for t in out.values() if hasattr(t, "numel"))
    sl = wob.Problem(sphere, kind=wob.NEUMANN_SL, data_mode=wob.DATA_POLY,
                     poly=(0, 0, 0, 1, 0, 0, 0, 0, 0, 0))
    fwd = wob.solve_forward(sl, none, 16, 3, want_paths=True)
    assert fwd["est"].numel() == 0 and torch.isfinite(fwd["zw"]).all()
    s = torch.full((0,), 7.0, dtype=torch.float64, device="cuda")
    wob.cv_solve_mc(dl, np.zeros(wob.mlp_num_params(), np.float32), none, 0, 8, 2, 2, s,
                    s.clone())
    r = torch.full((3,), 7.0, dtype=torch.float64, device="cuda")
    wob.solve_range(dl, none, 0, 8, 4, r[:0], r[:0])
    assert torch.equal(r, torch.full((3,), 7.0, dtype=torch.float64, device="cuda"))


def test_path_length_limits(wob, sphere):
    dl = wob.Problem(sphere, data_mode=wob.DATA_POLY, poly=I.POLY_CONFIG1)
    q = I.ball_queries(3, 0.5, 2)
    est, var = wob.solve(dl, q, 4, 4096)        # the largest accepted length
    assert torch.isfinite(est).all()
    with pytest.raises(wob.WobError, match="INVALID_ARG"):
        wob.solve(dl, q, 4, 4097)
    sl = wob.Problem(sphere, kind=wob.NEUMANN_SL, data_mode=wob.DATA_POLY,
                     poly=(0, 0, 0, 1, 0, 0, 0, 0, 0, 0))
    assert torch.isfinite(wob.solve_forward(sl, q, 4, 1024)["est"]).all()
    with pytest.raises(wob.WobError, match="INVALID_ARG"):
        wob.solve_forward(sl, q, 4, 1025)
    with pytest.raises(wob.WobError, match="INVALID_ARG"):
        wob.solve_forward(sl, q, 1, 3)          # one path has no variance


@pytest.mark.parametrize("kind", ["DIRICHLET_DL", "NEUMANN_SL", "ROBIN_SL", "NEUMANN_DIRECT"])
def test_ragged_walk_counts(wob, sphere, kind):
    """33 walks: one full 32-walk tile and a tile of one; the result equals
    the first 33 walks of a 64-walk solve's per-walk values."""
    k = getattr(wob, kind)
    prob = wob.Problem(sphere, kind=k, side=1 if k != wob.ROBIN_SL else -1, alpha=0.5,
                       data_mode=wob.DATA_POINT, x0=(0.0, 0.0, 3.0) if k != wob.ROBIN_SL
                       else (0.1, 0.0, 0.0))
    q = I.ball_queries(5, 0.5, 4) if k != wob.ROBIN_SL else I.ball_queries(5, 0.5, 4) * 3
    a = wob.solve_debug(prob, q, 33, 3, seed=7, want_lines=False)["per_walk"]
    b = wob.solve_debug(prob, q, 64, 3, seed=7, want_lines=False)["per_walk"]
    assert torch.equal(a, b[:, :33])


def test_get_stats_returns_the_last_counted_solve(wob, sphere):
    """wob_get_stats (through the C ABI) returns the counters of the calling
    thread's last wob_solve_counted call; another thread has its own."""
    import threading
    prob = wob.Problem(sphere, data_mode=wob.DATA_POLY, poly=I.POLY_CONFIG1)
    q = I.ball_queries(40, 0.8, 2)
    _, _, st = wob.solve_counted(prob, q, 64, 4, seed=3)
    assert st["lines"] > 0 and st["node_visits"] > 0 and st["hits"] >= st["lines"]
    assert wob.get_stats() == st
    wob.solve(prob, q, 64, 4, seed=4)  # an uncounted solve leaves them alone
    assert wob.get_stats() == st
    other = {}
    t = threading.Thread(target=lambda: other.update(wob.get_stats()))
    t.start()
    t.join()
    assert other == dict(lines=0, node_visits=0, tri_tests=0, hits=0, flagged=0)
