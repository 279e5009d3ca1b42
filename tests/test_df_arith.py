"""Double-float arithmetic of the FP64-accuracy residual stencil (csrc/df.cuh),
checked on the host against exact rational arithmetic: the error-free
transformations are exact, and sums, products and fused multiply-adds stay
within a small multiple of 2^-48 of the operands' magnitudes (the bound the
residual update relies on), including sums that cancel."""
import os
import shutil
import subprocess
from fractions import Fraction

import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "..", "paper_2412_06347_gb300", "csrc")
CUDA_INC = "/usr/local/cuda/include"

PROG = r"""
#include <cstdio>
#include <cstdint>
#include <cmath>
#include "df.cuh"
using mglma::DF;
namespace d = mglma::dfl;
static uint64_t st = 0x9E3779B97F4A7C15ull;
static double urand() {  // [0, 1)
  st = st * 6364136223846793005ull + 1442695040888963407ull;
  return (double)(st >> 11) * (1.0 / 9007199254740992.0);
}
static double val() {
  const double m = 2.0 * urand() - 1.0;
  return m * std::pow(10.0, 6.0 * urand() - 3.0);
}
static void pr(const char* tag, DF x) { std::printf(" %s %a %a", tag, (double)x.hi, (double)x.lo); }
int main() {
  for (int i = 0; i < 4000; ++i) {
    const double a = val(), b = val(), c = val();
    DF x(a), y(b), z(c);
    if (i % 4 == 1) y = -x + DF(val() * 1e-9);   // near-cancelling sums
    if (i % 4 == 2) z = -(x * y) + DF(val() * 1e-7);
    const float fa = (float)a, fb = (float)b;
    std::printf("%a %a %a", a, b, c);
    pr("x", x); pr("y", y); pr("z", z);
    pr("ts", d::two_sum(fa, fb)); pr("tp", d::two_prod(fa, fb));
    pr("add", x + y); pr("mul", x * y); pr("fma", d::fma(x, y, z));
    std::printf(" fab %a %a\n", (double)fa, (double)fb);
  }
  return 0;
}
"""


def _pairs(tokens, tag):
    i = tokens.index(tag)
    return Fraction(float.fromhex(tokens[i + 1])), Fraction(float.fromhex(tokens[i + 2]))


@pytest.fixture(scope="module")
def lines(tmp_path_factory):
    gxx = shutil.which("g++")
    if not gxx or not os.path.isfile(os.path.join(CUDA_INC, "cuda_runtime.h")):
        pytest.skip("g++ or the CUDA headers are missing")
    d = tmp_path_factory.mktemp("df")
    src, exe = d / "df_test.cpp", d / "df_test"
    src.write_text(PROG)
    subprocess.run([gxx, "-std=c++17", "-O2", "-ffp-contract=off", "-I", CSRC, "-I", CUDA_INC, str(src), "-o",
                    str(exe)], check=True, capture_output=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout
    return [ln.split() for ln in out.splitlines()]


def test_error_free_transformations_are_exact(lines):
    for t in lines:
        fa, fb = _pairs(t, "fab")
        s, e = _pairs(t, "ts")
        assert s + e == fa + fb
        p, e = _pairs(t, "tp")
        assert p + e == fa * fb


def test_split_and_normalisation(lines):
    for t in lines:
        a = Fraction(float.fromhex(t[0]))
        hi, lo = _pairs(t, "x")
        assert abs(hi + lo - a) <= abs(a) * Fraction(1, 2**47)
        for tag in ("add", "mul", "fma"):
            h, l = _pairs(t, tag)
            assert abs(l) <= abs(h) * Fraction(1, 2**23) or h == 0


def test_sum_product_fma_bounds(lines):
    eps = Fraction(1, 2**45)
    for t in lines:
        x = sum(_pairs(t, "x"))
        y = sum(_pairs(t, "y"))
        z = sum(_pairs(t, "z"))
        assert abs(sum(_pairs(t, "add")) - (x + y)) <= eps * (abs(x) + abs(y))
        assert abs(sum(_pairs(t, "mul")) - x * y) <= eps * abs(x * y)
        assert abs(sum(_pairs(t, "fma")) - (x * y + z)) <= eps * (abs(x * y) + abs(z))
