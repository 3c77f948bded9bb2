"""Pins for the oracle's random numbers.

* Philox4x32-10 against Triton's independent implementation, run on the CPU
  through Triton's interpreter (a library routine; skipped where Triton is
  absent).
* Philox4x64-10 -- the same round structure at 64 bits -- against numpy's
  Philox bit generator.
* Line axes (Marsaglia 1972) against the properties of the uniform
  distribution on the sphere (Archimedes: z is uniform on [-1, 1]; the
  azimuth is uniform; mean 0; second moment I/3).
* Uniform variates: Kolmogorov-Smirnov and lag-1 correlation.
"""
import json
import os
import subprocess
import sys

import numpy as np
import pytest
from scipy import stats

import oracle as O

_TRITON_SCRIPT = r"""
import os, json, sys
os.environ["TRITON_INTERPRET"] = "1"
import torch, triton, triton.language as tl

@triton.jit
def k(seed, c0p, c1p, c2p, c3p, o0, o1, o2, o3, n: tl.constexpr):
    i = tl.arange(0, n)
    a, b, c, d = tl.philox(seed, tl.load(c0p + i), tl.load(c1p + i), tl.load(c2p + i),
                           tl.load(c3p + i))
    tl.store(o0 + i, a); tl.store(o1 + i, b); tl.store(o2 + i, c); tl.store(o3 + i, d)

req = json.loads(sys.stdin.read())
res = []
for seed, ctrs in req:
    n = len(ctrs)
    cs = [torch.tensor([c[j] for c in ctrs], dtype=torch.int64).to(torch.int32) for j in range(4)]
    outs = [torch.empty(n, dtype=torch.int32) for _ in range(4)]
    k[(1,)](seed, *cs, *outs, n=n)
    res.append([[int(o[i]) & 0xffffffff for o in outs] for i in range(n)])
print(json.dumps(res))
"""


def test_philox4x32_matches_triton_interpreter():
    pytest.importorskip("triton")
    rng = np.random.default_rng(123)
    req = []
    for _ in range(4):
        seed = int(rng.integers(0, 2 ** 63))
        ctrs = rng.integers(0, 2 ** 32, size=(16, 4), dtype=np.uint64).tolist()
        req.append([seed, ctrs])
    env = dict(os.environ, TRITON_INTERPRET="1")
    p = subprocess.run([sys.executable, "-c", _TRITON_SCRIPT], input=json.dumps(req),
                       capture_output=True, text=True, env=env, timeout=600)
    if p.returncode != 0:
        pytest.skip("triton interpreter unavailable: " + p.stderr[-300:])
    ref = json.loads(p.stdout.strip().splitlines()[-1])
    for (seed, ctrs), expect in zip(req, ref):
        key = np.array([seed & 0xFFFFFFFF, seed >> 32], np.uint32)
        got = O.philox4x32_10(np.array(ctrs, np.uint32), key)
        assert got.tolist() == expect


def test_philox4x64_matches_numpy():
    rng = np.random.default_rng(7)
    for _ in range(8):
        key = rng.integers(0, 2 ** 63, size=2, dtype=np.uint64) * np.uint64(2) + np.uint64(1)
        ctr = rng.integers(0, 2 ** 62, size=4, dtype=np.uint64)
        g = np.random.Philox(key=key, counter=ctr)
        raw = g.random_raw(4)
        # numpy advances the counter before producing a block
        nxt = ctr.copy()
        nxt[0] += np.uint64(1)
        got = O.philox4x64_10(nxt, key)[0]
        assert raw.tolist() == got.tolist()


def test_line_axes_uniform_on_sphere():
    n = 200_000
    qws = np.stack([np.arange(n) % 997, np.arange(n) // 997, np.arange(n) % 13], 1)
    d, calls = O.line_axes(0, 0, qws)
    assert np.allclose(np.linalg.norm(d, axis=1), 1.0, atol=1e-15)
    assert calls.min() >= 1 and calls.max() < 20
    # acceptance rate of one attempt is pi/4; two attempts per generator call
    p_call = 1 - (1 - np.pi / 4) ** 2
    assert abs(calls.mean() - 1 / p_call) < 0.01
    sig = 1 / np.sqrt(3 * n)
    assert np.all(np.abs(d.mean(0)) < 5 * sig)
    C = d.T @ d / n
    assert np.allclose(C, np.eye(3) / 3, atol=6e-3)
    assert stats.kstest(d[:, 2], stats.uniform(-1, 2).cdf).pvalue > 1e-3
    az = np.arctan2(d[:, 1], d[:, 0])
    assert stats.kstest(az, stats.uniform(-np.pi, 2 * np.pi).cdf).pvalue > 1e-3
    # distinct (query, walk, step) triples give distinct axes
    assert np.unique(d[:5000], axis=0).shape[0] == 5000


def test_uniforms():
    n = 100_000
    qws = np.stack([np.arange(n), np.full(n, 3), np.zeros(n)], 1)
    u53, u24 = O.uniforms(5, 2, qws)
    for u in (u53, u24[:, 0], u24[:, 1]):
        assert u.min() >= 0 and u.max() < 1
        assert stats.kstest(u, "uniform").pvalue > 1e-3
        assert abs(np.corrcoef(u[:-1], u[1:])[0, 1]) < 5 / np.sqrt(n)
    # 24-bit grid
    assert np.all(u24 * 2 ** 24 == np.floor(u24 * 2 ** 24))
