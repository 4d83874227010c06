"""Host build of the double-float header (csrc/dfloat.cuh) checked against
its error bounds on random values (CPU; g++)."""
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

PROG = r"""
#include <cstdio>
#include <random>
#include "dfloat.cuh"
using namespace hhg;
int main() {
  std::mt19937_64 rng(12345);
  std::uniform_real_distribution<double> U(-1.0, 1.0);
  std::uniform_int_distribution<int> E(-50, 50);   // supported range: |values| in [2^-74, 2^127]
  double worst_rt = 0, worst_add = 0, worst_mul = 0;
  for (int k = 0; k < 1000000; ++k) {
    const double a = std::ldexp(U(rng), E(rng)), b = std::ldexp(U(rng), E(rng) / 4);
    const dfl x = from_double(a), y = from_double(b);
    if (a != 0) worst_rt = std::fmax(worst_rt, std::fabs(to_double(x) - a) / std::fabs(a));
    const long double sx = (long double)to_double(x), sy = (long double)to_double(y);
    const long double add = sx + sy, mul = sx * sy;
    worst_add = std::fmax(worst_add, (double)(std::fabs((long double)to_double(df_add(x, y)) - add) /
                                              (std::fabs(sx) + std::fabs(sy))));
    if (mul != 0) worst_mul = std::fmax(worst_mul, (double)(std::fabs((long double)to_double(df_mul(x, y)) - mul) / std::fabs(mul)));
  }
  // exact cases
  const double z = to_double(from_double(0.0)), one = to_double(from_double(1.0));
  const double m = to_double(from_double(-0.375)), big = to_double(from_double(3.0e20));
  printf("%.3e %.3e %.3e %g %g %g %g\n", worst_rt, worst_add, worst_mul, z, one, m, big);
  return 0;
}
"""


def test_double_float_error_bounds(tmp_path):
    if not shutil.which("g++"):
        pytest.skip("g++ not available")
    src = tmp_path / "t.cpp"
    src.write_text(PROG)
    exe = tmp_path / "t"
    subprocess.run(["g++", "-O2", "-std=c++17", "-I", os.path.join(ROOT, "paper_1805_10167_gb300", "csrc"),
                    str(src), "-o", str(exe)], check=True)
    out = subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout.split()
    rt, add, mul = (float(v) for v in out[:3])
    # hi is the truncated top 24 bits, lo the next 29 rounded to 24: the pair
    # keeps 48 bits; in a product the cross terms hi*lo (|lo| < ulp(hi)) are
    # each rounded once (2^-47) and lo*lo is dropped
    assert rt <= 1.01 * 2.0 ** -48
    assert add <= 2.0 ** -45         # sloppy addition, absolute in |x| + |y|
    assert mul <= 2.0 ** -44
    assert [float(v) for v in out[3:]] == [0.0, 1.0, -0.375, 3.0e20]
