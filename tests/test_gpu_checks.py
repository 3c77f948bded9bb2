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


def test_tensor_core_wait_limit_fails_cleanly(wob):
    """The network kernels' first wait on each tensor-core product gives up
    after a poll limit; forced to 0, every wait gives up at once: the
    kernels drain their products in flight, free their tensor memory and
    write NaN (forward outputs; training gradients and loss), and the
    context stays usable (the next calls reproduce the earlier results)."""
    from oracle import cv as C
    flat = torch.from_numpy(C.flatten(C.mlp_init(2)).astype(np.float32)).cuda()
    y = torch.from_numpy(I.ball_queries(1000, 0.9, 4)).cuda()
    tgt = torch.zeros(1000, dtype=torch.float32, device="cuda")
    ref = wob.mlp_forward(flat, y)
    g_ref = torch.empty_like(flat)
    wob.mlp_train_step(flat.clone(), torch.zeros_like(flat), torch.zeros_like(flat), y, tgt, 0.0,
                       1, grad=g_ref)
    prev = wob.debug_set_tc_wait_limit(0)
    try:
        bad = wob.mlp_forward(flat, y)
        g = torch.empty_like(flat)
        loss = torch.empty(1, dtype=torch.float32, device="cuda")
        wob.mlp_train_step(flat.clone(), torch.zeros_like(flat), torch.zeros_like(flat), y, tgt,
                           0.0, 1, grad=g, loss=loss)
        torch.cuda.synchronize()
    finally:
        wob.debug_set_tc_wait_limit(prev)
    assert torch.isnan(bad).all()
    assert torch.isnan(g).all() and torch.isnan(loss).all()
    assert torch.equal(wob.mlp_forward(flat, y), ref)
    g2 = torch.empty_like(flat)
    wob.mlp_train_step(flat.clone(), torch.zeros_like(flat), torch.zeros_like(flat), y, tgt, 0.0,
                       1, grad=g2)
    assert torch.equal(g2, g_ref)
