"""The compensated FP32 arithmetic of the walk kernels (csrc/ff.cuh), built
as plain C++ on the host without floating-point contraction (the device
build uses the explicitly rounded intrinsics, the same IEEE operations):
Knuth's two-sum and the FMA two-product are exact (checked in double, where
these sums and products are representable); the float-float sum, product,
three-term dot product and square root are within their error bounds of
a long-double reference, including the cancelling r . n of two nearby
points of a surface that the single-layer kernel relies on."""
import shutil
import subprocess

import pytest

from paper_2305_04403_gb300 import build as B

SRC = r"""
#include <cmath>
#include <cstdio>
#include <random>
#include "ff.cuh"
using wob::ff;
static long double val(ff x) { return (long double)x.hi + (long double)x.lo; }
int main() {
    std::mt19937_64 g(5);
    std::uniform_real_distribution<double> m(1.0, 2.0);
    std::uniform_int_distribution<int> ex(-20, 20);
    auto rf = [&]() { float v = (float)std::ldexp(m(g), ex(g)); return (g() & 1) ? -v : v; };
    long n = 0, bad_sum = 0, bad_prod = 0, bad_add = 0, bad_mul = 0, bad_dot = 0, bad_sqrt = 0,
         bad_cancel = 0;
    double worst_add = 0, worst_mul = 0, worst_dot = 0, worst_sqrt = 0, worst_cancel = 0;
    for (int i = 0; i < 1000000; ++i, ++n) {
        const float a = rf(), b = rf();
        const ff s = wob::two_sum(a, b);
        if ((double)s.hi + (double)s.lo != (double)a + (double)b || s.hi != a + b) ++bad_sum;
        const ff p = wob::two_prod(a, b);
        if ((double)p.hi + (double)p.lo != (double)a * (double)b) ++bad_prod;
        // float-float operands: an exact sum of two floats each
        const ff x = wob::two_sum(rf(), rf() * 1e-8f), y = wob::two_sum(rf(), rf() * 1e-8f);
        const long double xa = val(x), ya = val(y);
        const double ea = (double)fabsl(val(wob::ff_add(x, y)) - (xa + ya)) /
                          (double)(fabsl(xa) + fabsl(ya));
        if (ea > 0x1p-44) ++bad_add;
        worst_add = ea > worst_add ? ea : worst_add;
        const double em = (double)fabsl(val(wob::ff_mul(x, y)) / (xa * ya) - 1.0L);
        if (em > 0x1p-44) ++bad_mul;
        worst_mul = em > worst_mul ? em : worst_mul;
        const ff u[3] = {x, y, wob::two_sum(rf(), rf() * 1e-8f)};
        const ff v[3] = {y, wob::two_sum(rf(), rf() * 1e-8f), x};
        long double exact = 0, mag = 0;
        for (int c = 0; c < 3; ++c) {
            exact += val(u[c]) * val(v[c]);
            mag += fabsl(val(u[c]) * val(v[c]));
        }
        const double ed = (double)(fabsl(val(wob::ff_dot3(u, v)) - exact) / mag);
        if (ed > 0x1p-43) ++bad_dot;
        worst_dot = ed > worst_dot ? ed : worst_dot;
        const float q = std::fabs(a);
        const double es = (double)fabsl(val(wob::ff_sqrt(q)) / sqrtl((long double)q) - 1.0L);
        if (es > 0x1p-44) ++bad_sqrt;
        worst_sqrt = es > worst_sqrt ? es : worst_sqrt;
        // r . n for two points of the unit sphere a distance d apart:
        // r . n = -d^2 / 2 at the second point's normal; the float-float
        // dot product keeps it to 2^-40 of |r|^2 however small d is
        const double th = std::ldexp(m(g), -ex(g) % 14 - 4), ph = m(g);
        const double p0[3] = {std::cos(ph), std::sin(ph), 0.0};
        const double p1[3] = {std::cos(ph) * std::cos(th), std::sin(ph) * std::cos(th), std::sin(th)};
        ff r[3], nn[3];
        long double rr = 0, rn = 0;
        for (int c = 0; c < 3; ++c) {
            const float h = (float)(p1[c] - p0[c]);
            r[c] = {h, (float)((p1[c] - p0[c]) - (double)h)};
            const float nh = (float)p0[c];
            nn[c] = {nh, (float)(p0[c] - (double)nh)};
            rr += val(r[c]) * val(r[c]);
            rn += val(r[c]) * val(nn[c]);
        }
        const double ec = (double)(fabsl(val(wob::ff_dot3(nn, r)) - rn) / rr);
        if (ec > 0x1p-40) ++bad_cancel;
        worst_cancel = ec > worst_cancel ? ec : worst_cancel;
    }
    printf("%ld %ld %ld %ld %ld %ld %ld %ld %.3g %.3g %.3g %.3g %.3g\n", n, bad_sum, bad_prod,
           bad_add, bad_mul, bad_dot, bad_sqrt, bad_cancel, worst_add, worst_mul, worst_dot,
           worst_sqrt, worst_cancel);
    return 0;
}
"""


def test_float_float_arithmetic(tmp_path):
    gxx = shutil.which("g++")
    if not gxx:
        pytest.skip("no host C++ compiler")
    (tmp_path / "t.cpp").write_text(SRC)
    exe = tmp_path / "t"
    subprocess.run([gxx, "-O2", "-std=c++17", "-ffp-contract=off", "-I", B.CSRC,
                    str(tmp_path / "t.cpp"), "-o", str(exe)], check=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout.split()
    n, *bad = map(int, out[:8])
    print("cases", n, "worst relative errors (add, mul, dot, sqrt, cancelling dot / r^2):",
          out[8:])
    assert n == 1000000
    assert bad == [0] * 7, dict(zip(["two_sum", "two_prod", "add", "mul", "dot3", "sqrt",
                                     "cancelling r.n"], bad))
