"""The exact conversions of csrc/bits.cuh, built as plain C++ on the host:
u53_unit(U) must equal the FP64 conversion of the 53-bit integer U times
2^-53, and scale2(t, e) must equal ldexp of t's FP64 conversion, bit for bit
(random U at every leading-one position plus the powers of two and 2^k - 1;
every class of float bit pattern, including zero, subnormals, infinities
and NaN, with shifts from -1200 to 1200 that reach the subnormal and
overflow ranges of FP64).  The area sampling of the single-layer walks takes
its CDF target and its walk terms from these functions."""
import shutil
import subprocess

import pytest

from paper_2305_04403_gb300 import build as B

SRC = r"""
#include <cmath>
#include <cstdint>
#include <cstdio>
#include <cstring>
#include <random>
#include "bits.cuh"
static bool same(double a, double b)
{
    if (std::isnan(a) || std::isnan(b)) return std::isnan(a) && std::isnan(b);
    return std::memcmp(&a, &b, sizeof a) == 0;
}
int main() {
    std::mt19937_64 g(7);
    long n1 = 0, bad1 = 0, n2 = 0, bad2 = 0;
    for (int k = 0; k < 53; ++k) {
        for (int i = 0; i < 20000; ++i, ++n1) {
            uint64_t U = (g() >> 11) >> k;
            if (i == 0) U = 1ull << (52 - k);
            if (i == 1) U = (1ull << (53 - k)) - 1;
            if (!same(wob::u53_unit(U), (double)U * 0x1p-53)) ++bad1;
        }
    }
    ++n1;
    if (!same(wob::u53_unit(0), 0.0)) ++bad1;
    std::uniform_int_distribution<int> wide(-1200, 1200), narrow(-100, 100);
    for (int i = 0; i < 4000000; ++i, ++n2) {
        uint32_t b = (uint32_t)g();
        if (i % 11 == 0) b &= 0x807FFFFFu;                 // zero and subnormals
        if (i % 13 == 0) b |= 0x7F800000u;                 // infinities and NaN
        float t;
        std::memcpy(&t, &b, sizeof t);
        const int e = (i % 7 == 0) ? narrow(g) : wide(g);
        if (!same(wob::scale2(t, e), std::ldexp((double)t, e))) ++bad2;
    }
    printf("%ld %ld %ld %ld\n", n1, bad1, n2, bad2);
    return 0;
}
"""


def test_exact_conversions(tmp_path):
    gxx = shutil.which("g++")
    if not gxx:
        pytest.skip("no host C++ compiler")
    (tmp_path / "t.cpp").write_text(SRC)
    exe = tmp_path / "t"
    subprocess.run([gxx, "-O2", "-std=c++17", "-ffp-contract=off", "-I", B.CSRC,
                    str(tmp_path / "t.cpp"), "-o", str(exe)], check=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout.split()
    n1, bad1, n2, bad2 = map(int, out)
    assert n1 == 53 * 20000 + 1 and n2 == 4000000
    assert bad1 == 0, f"u53_unit differs from the FP64 conversion in {bad1} of {n1} cases"
    assert bad2 == 0, f"scale2 differs from ldexp in {bad2} of {n2} cases"
