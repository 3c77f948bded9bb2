"""GPU parity of the single-layer walks with mixed boundary conditions
(Sec. 4.3; kind WOB_MIXED_SL) and with resampled importance sampling of the
next point (the paper's 16 uniform candidates) against the oracle's sl_walks.

Per walk |gpu - oracle| <= 1e-5 * sum_k |term_k| (+1e-12 * scale): both
sides draw the same candidates, branch decisions and picks from the same
counter-based streams; k and p_k are exact in FP32, so the move / stay
decisions agree."""
import numpy as np
import pytest

import oracle as O
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


def _axes(n, seed):
    rng = np.random.default_rng(seed)
    d = rng.standard_normal((n, 3))
    return d / np.linalg.norm(d, axis=1, keepdims=True)


def _compare(wob, v, f, q, N, M, kind, phi, alpha=0.0, bc=None, kmix=0.0, pk=0.0, ris=0,
             mode=O.DATA_POLY, poly=None, x0=None, seed=0):
    mesh = wob.build_mesh(v, f)
    bvh = wob.build_bvh(mesh)
    prob = wob.Problem(bvh, kind=kind, side=phi, alpha=alpha, data_mode=mode,
                       poly=tuple(poly) if poly is not None else (0.0,) * 10,
                       x0=tuple(x0) if x0 is not None else (0.0, 0.0, 0.0),
                       bc_type=None if bc is None else torch.from_numpy(bc).cuda(),
                       k_mix=kmix, p_k=pk, ris=ris)
    g = wob.solve_debug(prob, q, N, M, seed=seed, want_lines=False)["per_walk"].cpu().numpy()
    pw, at = O.sl_walks(v, f, q, N, M, kind=kind, alpha=alpha, phi=phi, mode=mode, poly=poly,
                        x0=x0, seed=seed, want_abs=True, bc_type=bc, kmix=kmix, pk=pk, ris=ris)
    err = np.abs(g - pw)
    assert np.all(err <= 1e-5 * at + 1e-12), (err / np.maximum(1e-5 * at, 1e-300)).max()
    return g


def test_mixed_random_conditions_parity(wob):
    """Each triangle Dirichlet, Neumann or Robin at random (as the paper's
    mixed examples), interior, harmonic polynomial data."""
    v, f = I.icosphere(3)
    bc = np.random.default_rng(3).integers(0, 3, len(f)).astype(np.uint8)
    q = I.ball_queries(32, 0.8, 4)
    poly = (0.1, 0.3, -0.2, 0.5, 1.0, -1.0, 0.0, 0.4, 0.0, 0.0)
    g = _compare(wob, v, f, q, 128, 6, O.KIND_MIXED_SL, 1, alpha=0.5, bc=bc, kmix=1.5, pk=0.75,
                 poly=poly, seed=5)
    assert np.isfinite(g).all()


def test_mixed_exterior_point_source_parity(wob):
    v, f, sh = I.star_mesh(3, 0.3, 6, 3, 0.5)
    bc = np.random.default_rng(4).integers(0, 3, len(f)).astype(np.uint8)
    q = (_axes(24, 5) * np.random.default_rng(6).uniform(1.4, 2.2, (24, 1))).astype(np.float32)
    _compare(wob, v, f, q, 128, 5, O.KIND_MIXED_SL, -1, alpha=0.25, bc=bc, kmix=1.0, pk=0.5,
             mode=O.DATA_POINT, x0=(0.05, -0.1, 0.1), seed=7)


@pytest.mark.parametrize("kind,phi,alpha", [(1, 1, 0.0), (2, -1, 0.25)])
def test_ris_parity(wob, kind, phi, alpha):
    v, f = I.icosphere(3)
    q = (I.ball_queries(32, 0.8, 3) if phi == 1 else
         (_axes(32, 4) * np.random.default_rng(1).uniform(1.2, 2, (32, 1))).astype(np.float32))
    x0 = (0.1, 0.2, 0.3) if phi == -1 else (0.0, 0.0, 3.0)
    _compare(wob, v, f, q, 128, 5, kind, phi, alpha=alpha, ris=16, mode=O.DATA_POINT, x0=x0,
             seed=2)


def test_ris_and_mixed_together(wob):
    v, f = I.icosphere(3)
    bc = np.random.default_rng(8).integers(0, 3, len(f)).astype(np.uint8)
    q = I.ball_queries(16, 0.7, 9)
    _compare(wob, v, f, q, 64, 4, O.KIND_MIXED_SL, 1, alpha=1.0, bc=bc, kmix=1.5, pk=0.75,
             ris=16, poly=I.POLY_CONFIG1, seed=3)


def test_mixed_rejects_bad_parameters(wob):
    v, f = I.icosphere(1)
    mesh = wob.build_mesh(v, f)
    bvh = wob.build_bvh(mesh)
    bc = torch.zeros(len(f), dtype=torch.uint8, device="cuda")
    q = I.ball_queries(4, 0.5, 1)
    for kw in (dict(bc_type=None, k_mix=1.0, p_k=0.5), dict(bc_type=bc, k_mix=0.0, p_k=0.5),
               dict(bc_type=bc, k_mix=1.0, p_k=1.0), dict(bc_type=bc, k_mix=1.0, p_k=0.5, ris=65)):
        prob = wob.Problem(bvh, kind=wob.MIXED_SL, data_mode=wob.DATA_POLY, **kw)
        with pytest.raises(wob.WobError):
            wob.solve(prob, q, 8, 3)
