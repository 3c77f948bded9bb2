"""The C-ABI library builds for sm_103a, loads, and exports every entry point
declared in include/wob.h (no compute calls: no GPU needed)."""
import ctypes
import os
import re

import pytest

from paper_2305_04403_gb300 import build as B

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = []
    for fn in sorted(os.listdir(os.path.join(ROOT, "include"))):
        if not fn.endswith(".h"):
            continue
        src = open(os.path.join(ROOT, "include", fn)).read()
        src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
        names += re.findall(r"^\s*(?:const\s+)?[\w\s\*]+?\b(wob_\w+)\s*\(", src, flags=re.M)
    return sorted(set(names))


@pytest.fixture(scope="module")
def lib_path():
    try:
        return B.build()
    except RuntimeError as e:  # pragma: no cover - no nvcc
        pytest.skip(f"cannot build: {e}")


def test_header_declares_the_entry_points():
    names = _declared()
    for must in ("wob_build_mesh", "wob_build_bvh", "wob_solve", "wob_solve_range",
                 "wob_destroy_mesh", "wob_destroy_bvh", "wob_last_error"):
        assert must in names


def test_library_exports_every_declared_symbol(lib_path):
    lib = ctypes.CDLL(lib_path)
    missing = [n for n in _declared() if not hasattr(lib, n)]
    assert not missing, missing


def test_version_and_error_string_without_gpu(lib_path):
    lib = ctypes.CDLL(lib_path)
    lib.wob_version.restype = ctypes.c_int
    assert lib.wob_version() >= 100
    lib.wob_last_error.restype = ctypes.c_char_p
    # the library may already be loaded in this process with an earlier
    # call's message: a successful call (an empty request, no CUDA) clears it
    lib.wob_philox4x32_10.argtypes = [ctypes.c_void_p] * 2 + [ctypes.c_int64] + [ctypes.c_void_p] * 2
    assert lib.wob_philox4x32_10(None, None, 0, None, None) == 0
    assert lib.wob_last_error() == b""


def test_invalid_arguments_rejected_before_any_cuda_call(lib_path):
    lib = ctypes.CDLL(lib_path)
    lib.wob_build_mesh.argtypes = [ctypes.c_void_p, ctypes.c_int64, ctypes.c_void_p,
                                   ctypes.c_int64, ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p]
    out = ctypes.c_void_p()
    assert lib.wob_build_mesh(None, 3, None, 1, 0, None, ctypes.byref(out)) == -1
    lib.wob_last_error.restype = ctypes.c_char_p
    assert b"invalid" in lib.wob_last_error()
    lib.wob_solve.argtypes = [ctypes.c_void_p] * 3 + [ctypes.c_int64, ctypes.c_int32,
                                                      ctypes.c_int32, ctypes.c_uint64] + [ctypes.c_void_p] * 3
    assert lib.wob_solve(None, None, None, 4, 1, 4, 0, None, None, None) == -1
    P, I64, I32 = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int32
    # forward paths, Monte Carlo control variate, L2 probe: NULL problem,
    # parameters or buffers are refused before anything reaches the GPU
    lib.wob_solve_forward.argtypes = [P, P, I64, I32, I32, ctypes.c_uint64, I32, ctypes.c_float,
                                      P, P, P, P, P, P]
    assert lib.wob_solve_forward(None, None, 4, 64, 3, 0, 1, 0.1, None, None, None, None, None,
                                 None) == -1
    lib.wob_cv_solve_mc.argtypes = [P, P, P, I64, I64, I32, I32, I32, ctypes.c_uint64, P, P, P, P]
    assert lib.wob_cv_solve_mc(None, None, None, 4, 0, 8, 2, 4, 0, None, None, None, None) == -1
    lib.wob_probe_l2_read.argtypes = [P, I64, I32, P, P]
    assert lib.wob_probe_l2_read(None, 1 << 20, 1, None, None) == -1
    assert b"wob_probe_l2_read" in lib.wob_last_error()


# Entry points without a required pointer argument (they succeed without a
# device); every other declared function is in the NULL-argument sweep.
_NO_REQUIRED_POINTER = {"wob_version", "wob_mlp_num_params", "wob_debug_set_tc_wait_limit",
                        "wob_last_error"}

_SWEEP = r"""
import ctypes, json, sys
lib = ctypes.CDLL(sys.argv[1])
lib.wob_last_error.restype = ctypes.c_char_p
kinds = {"p": (ctypes.c_void_p, None), "i64": (ctypes.c_int64, 4), "i32": (ctypes.c_int32, 4),
         "u64": (ctypes.c_uint64, 0), "u32": (ctypes.c_uint32, 0), "f": (ctypes.c_float, 0.5),
         "i": (ctypes.c_int, 0)}
out = {}
for name, ret, args in json.loads(sys.argv[2]):
    f = getattr(lib, name)
    f.argtypes = [kinds[a][0] for a in args]
    f.restype = None if ret == "void" else ctypes.c_int
    rc = f(*[kinds[a][1] for a in args])
    out[name] = [rc, lib.wob_last_error().decode()]
print(json.dumps(out))
"""


def _signatures():
    """(name, return type, argument kinds) of the functions in include/wob.h:
    "p" for pointers and opaque handles, else the integer or float width."""
    src = re.sub(r"/\*.*?\*/", "", open(os.path.join(ROOT, "include", "wob.h")).read(), flags=re.S)
    sigs = []
    for ret, name, params in re.findall(r"^(int|void)\s+(wob_\w+)\s*\(([^;]*?)\)\s*;", src,
                                        flags=re.M | re.S):
        args = []
        for p in " ".join(params.split()).split(","):
            p = p.strip()
            if not p or p == "void":
                continue
            t = p.split()[0] if p.split()[0] != "const" else p.split()[1]
            if "*" in p or t in ("wob_mesh", "wob_bvh", "wob_cv", "wob_batch"):
                args.append("p")
            else:
                args.append({"int64_t": "i64", "int32_t": "i32", "uint64_t": "u64",
                             "uint32_t": "u32", "float": "f", "int": "i"}[t])
        sigs.append((name, ret, args))
    return sigs


def test_every_entry_point_rejects_null_arguments(lib_path):
    """Every declared call given NULL pointers and handles (and small sizes)
    returns WOB_ERR_INVALID_ARG with a message, or for the destroy calls
    returns quietly; -1 rather than WOB_ERR_CUDA on this GPU-less machine
    also shows that the check comes before any CUDA call.  The calls run in
    a child process, so a crash fails this test instead of the session."""
    import json
    import subprocess
    import sys
    sigs = [s for s in _signatures() if s[0] not in _NO_REQUIRED_POINTER]
    assert {s[0] for s in sigs} | _NO_REQUIRED_POINTER == set(_declared())
    r = subprocess.run([sys.executable, "-c", _SWEEP, lib_path, json.dumps(sigs)],
                       capture_output=True, text=True, timeout=120)
    assert r.returncode == 0, r.stderr[-2000:]
    out = json.loads(r.stdout.strip().splitlines()[-1])
    for name, ret, _ in sigs:
        rc, msg = out[name]
        if ret == "void":
            assert rc is None, name
        else:
            assert rc == -1 and msg, (name, rc, msg)
    assert out["wob_solve_batched"][1].startswith("wob_solve_batched")


def _ptxas_functions(log):
    """(function, registers, spill-store bytes) from a ptxas -v log."""
    out = []
    for block in log.split("Function properties for ")[1:]:
        name = block.split()[0]
        spill = re.search(r"(\d+) bytes spill stores", block)
        regs = re.search(r"Used (\d+) registers", block)
        out.append((name, int(regs.group(1)) if regs else 0, int(spill.group(1)) if spill else 0))
    return out


def test_ptxas_register_budget(lib_path):
    """The line-walk kernels (double layer, batched, direct Neumann, forward
    paths) are held to 64 registers (8 blocks of 128 threads per SM); only
    they may keep values in local memory, every other kernel fits in
    registers."""
    log = open(os.path.join(os.path.dirname(lib_path), "ptxas.log")).read()
    funcs = _ptxas_functions(log)
    assert funcs
    for name, regs, spill in funcs:
        if any(k in name for k in ("k_dl_walks", "k_dl_batched", "k_nd_walks", "k_fwd_paths")):
            assert regs <= 64, (name, regs)
        else:
            assert spill == 0, (name, spill)
