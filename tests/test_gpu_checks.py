"""Device-side checks without a fault.  The traversal of a line is bounded
(at most iter_limit node visits; the automatic bound is never reached by a
valid tree).  A problem with a tiny bound makes lines give up on purpose:
the solve's check word is set, every estimate of that call is NaN (so
asynchronous callers see it), wob_solve_counted returns
WOB_ERR_DEVICE_CHECK, and the context stays usable -- the next solve with
the automatic bound is exact."""
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


def test_iteration_bound_reports_without_fault(wob):
    v, f, sh = I.star_mesh(4)
    bvh = wob.build_bvh(wob.build_mesh(v, f))
    q = I.ball_queries(64, 0.5, 3)
    good = wob.Problem(bvh, data_mode=wob.DATA_POINT, x0=(3.0, 0.0, 0.0))
    ref, _ = wob.solve(good, q, 32, 6, seed=1)
    bad = wob.Problem(bvh, data_mode=wob.DATA_POINT, x0=(3.0, 0.0, 0.0), iter_limit=2)
    est, var = wob.solve(bad, q, 32, 6, seed=1)
    assert torch.isnan(est).all()          # every line needs more than two node visits
    with pytest.raises(wob.WobError) as e:
        wob.solve_counted(bad, q, 32, 6, seed=1)
    assert "iteration bound" in str(e.value)
    s = torch.zeros(len(q), dtype=torch.float64, device="cuda")
    ss = torch.zeros_like(s)
    wob.solve_range(bad, q, 0, 8, 6, s, ss, seed=1)
    assert torch.isnan(s).all() and torch.isnan(ss).all()
    again, _ = wob.solve(good, q, 32, 6, seed=1)
    assert torch.equal(again, ref)


def test_iteration_bound_in_other_kernels(wob):
    v, f, sh = I.displaced_torus(60, 24)
    bvh = wob.build_bvh(wob.build_mesh(v, f))
    q = I.torus_queries(sh, 32, True, seed=5)
    nd = wob.Problem(bvh, kind=wob.NEUMANN_DIRECT, data_mode=wob.DATA_POINT, x0=(0.0, 0.0, 5.0),
                     iter_limit=2)
    est, _ = wob.solve(nd, q, 16, 4, seed=2)
    assert torch.isnan(est).all()
    sl = wob.Problem(bvh, kind=wob.NEUMANN_SL, data_mode=wob.DATA_POINT, x0=(0.0, 0.0, 5.0),
                     iter_limit=2)
    out = wob.solve_forward(sl, q, 64, 3, seed=2)
    assert torch.isnan(out["est"]).all()
    with pytest.raises(wob.WobError):
        wob.solve(wob.Problem(bvh, iter_limit=-1), q, 4, 2)
