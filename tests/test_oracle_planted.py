"""The oracle's pins catch plausible mistakes.  For each k, the oracle is
rebuilt with ORACLE_PLANT=k, which compiles one known mistake into it (see
the ORACLE_PLANT switch in oracle/wob_oracle.c), and the pin that guards
that part of the method is run against it in a subprocess: it must fail.
The same checks pass on the oracle itself (k = 0)."""
import os
import subprocess
import sys

import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)

# planted mistake -> pin expected to catch it
CHECKS = {
    1: "W.test_dl_interior_truncation_closed_form(S3, 2, W.Z, 1)",       # no half on the last term
    2: "W.test_dl_interior_truncation_closed_form(S3, 1, W.Z, 1)",       # first weight negated
    3: "W.test_dl_interior_truncation_closed_form(S3, 2, W.Z, 1)",       # recursion sign flipped
    4: "G.test_gauss_invariant_per_line(CASE)",                          # hit sign negated
    5: "W.test_sl_exterior_neumann_and_robin_closed_form(S3, 2)",        # Robin term sign
    6: "N.test_nd_interior_closed_form(S3, 1, N.Z, 1)",                  # no 1/2 on the first line
    7: "N.test_nd_boundary_start_closed_form(S3, 1)",                    # last source not halved
    8: "F.test_forward_interior_closed_form(S3, 0, 1, F.Z, 1)",          # forward start without 2
    9: "F.test_forward_interior_closed_form(S3, 0, 2, F.Z, 1)",          # forward step sign
    10: "F.test_forward_interior_closed_form(S3, 0, 1, F.Z, 1)",         # forward last not halved
    11: "F.test_forward_interior_closed_form(S3, 1, 1, F.Z, 1)",         # weighted start density
}

SCRIPT = """
import sys
sys.path.insert(0, {root!r}); sys.path.insert(0, {here!r})
import test_oracle_walks as W, test_oracle_nd as N, test_oracle_geometry as G
import test_oracle_fwd as F
from paper_2305_04403_gb300 import inputs as I
S3 = I.icosphere(3)
CASE = G._meshes_with_points()[0]
try:
    {check}
except AssertionError:
    print("PIN FAILED")
    sys.exit(0)
print("PIN PASSED")
"""


def _run(k, check):
    env = dict(os.environ, ORACLE_PLANT=str(k))
    r = subprocess.run([sys.executable, "-c", SCRIPT.format(root=ROOT, here=HERE, check=check)],
                       env=env, capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    return r.stdout.strip().splitlines()[-1]


@pytest.mark.parametrize("k", sorted(CHECKS))
def test_planted_mistake_is_caught(k):
    assert _run(k, CHECKS[k]) == "PIN FAILED"


def test_checks_pass_on_the_oracle():
    for check in sorted(set(CHECKS.values())):
        assert _run(0, check) == "PIN PASSED", check
