"""Walk-by-walk comparison of the CUDA path with the oracle (test helper).

Both sides trace the same lines as long as their walks agree: a walk's line
k starts at the point that line k - 1 picked and its axis comes from the
same counter-based stream.  So each walk is followed line by line and
compared up to the first line where the two sides differ in hit count or
picked triangle; a walk with no such line is compared whole.  The bars:

  * a line where the sides first differ must be near-degenerate: flagged by
    the CUDA path (whose flag covers the oracle's);
  * on every line both sides traced, an oracle flag implies a CUDA flag;
  * walks with no differing line: |gpu - oracle| <= 1e-5 * sum_k |term_k|
    (+ 1e-12 * scale), whatever their flags;
  * per query, the mean over those walks within 1e-4 * scale.

Returns the mask of walks compared whole and the rates for the report:
lines flagged by the oracle, by the CUDA path, lines and walks that
diverged.
"""
import numpy as np


def compare_walks(g: dict, r: dict, scale: float, walk_tol: float = 1e-5) -> tuple:
    gm, gp, gf = g["line_m"], g["line_prim"], g["line_flag"]
    rm, rp, rf = r["line_m"], r["line_prim"], r["line_flag"]
    M = gm.shape[-1]
    diff = (gm != rm) | (gp != rp)
    first = np.where(diff.any(-1), diff.argmax(-1), M)
    same = first == M
    common = np.arange(M)[None, None, :] < first[..., None]
    traced = common & (rm >= 0)
    # the divergent line itself is traced by both sides from the same point
    dq, dw = np.nonzero(~same)
    dk = first[~same]
    div_traced = (rm[dq, dw, dk] >= 0) | (gm[dq, dw, dk] >= 0)
    assert np.all(gf[dq, dw, dk][div_traced] == 1), \
        f"{int((gf[dq, dw, dk][div_traced] == 0).sum())} unflagged lines differ"
    # the CUDA flag covers the oracle's on every line both traced
    both = traced.copy()
    both[dq, dw, dk] = div_traced
    assert not np.any(both & (rf == 1) & (gf == 0)), \
        f"{int((both & (rf == 1) & (gf == 0)).sum())} oracle-flagged lines not flagged on the GPU"
    err = np.abs(g["per_walk"] - r["per_walk"])
    tol = walk_tol * r["abs_terms"] + 1e-12 * scale
    bad = same & (err > tol)
    assert not bad.any(), (f"{int(bad.sum())} walks off", (err / np.maximum(tol, 1e-300))[same].max())
    n = np.maximum(same.sum(1), 1)
    mg = np.where(same, g["per_walk"], 0.0).sum(1) / n
    mr = np.where(same, r["per_walk"], 0.0).sum(1) / n
    assert np.all(np.abs(mg - mr) <= 1e-4 * scale)
    n_lines = max(int(both.sum()), 1)
    stats = dict(lines=int(both.sum()),
                 oracle_flag_rate=float((both & (rf == 1)).sum() / n_lines),
                 gpu_flag_rate=float((both & (gf == 1)).sum() / n_lines),
                 diverged_line_rate=float(div_traced.sum() / n_lines),
                 diverged_walk_rate=float((~same).mean()),
                 walks_compared=float(same.mean()))
    return same, stats
