"""Processes that build the library at the same moment (the ranks of a
multi-GPU run) take turns under the build's file lock: exactly one compiles
and links, the others find the library up to date.  Checked with the compile
step replaced by a stub that records who ran it, in a temporary build
directory (no source or library of the repository is touched)."""
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

CHILD = r"""
import os, sys, time
from paper_2305_04403_gb300 import build as B
tmp = sys.argv[1]
B.OUT = tmp
B.LIB = os.path.join(tmp, "libwob.so")
dep = os.path.join(tmp, "dep.cu")
B._deps = lambda: [dep]
def stub(verbose):
    with open(os.path.join(tmp, "built_by"), "a") as f:
        f.write(f"{os.getpid()}\n")
    time.sleep(2)  # long enough for the other processes to queue on the lock
    open(B.LIB, "w").close()
    return B.LIB
B._build_locked = stub
print(B.build())
"""


def test_concurrent_builds_take_turns(tmp_path):
    (tmp_path / "dep.cu").write_text("")
    procs = [subprocess.Popen([sys.executable, "-c", CHILD, str(tmp_path)], cwd=ROOT,
                              stdout=subprocess.PIPE, stderr=subprocess.PIPE, text=True)
             for _ in range(3)]
    outs = [p.communicate(timeout=120) for p in procs]
    for p, (out, err) in zip(procs, outs):
        assert p.returncode == 0, err
        assert out.strip().endswith("libwob.so")
    builders = (tmp_path / "built_by").read_text().split()
    assert len(builders) == 1, builders
