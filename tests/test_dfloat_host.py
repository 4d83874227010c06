"""Host build of the double-float header (csrc/dfloat.cuh) checked against
its error bounds on random values, and its bit-level binary64 <-> binary32
conversions against the compiler's (CPU; g++)."""
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
  // binary64 -> binary32 (round to nearest even) and back, against the
  // compiler's conversions: random magnitudes, exact ties, overflow, flush
  long bad = 0;
  std::uniform_int_distribution<int> E2(-125, 127);
  std::uniform_int_distribution<uint64_t> M(0, (1ull << 52) - 1);
  for (int k = 0; k < 2000000; ++k) {
    double v = std::ldexp(U(rng), E2(rng));
    if (k % 4 == 1) {   // an exact tie: 24 significant bits followed by a single 1
      uint64_t u = dbits(v) & ~0x1FFFFFFFull;
      u |= 0x10000000ull;
      v = bitsd(u);
    }
    if (k % 4 == 2) v = bitsd((dbits(v) & 0xFFF0000000000000ull) | M(rng));
    if (std::fabs(v) < std::ldexp(1.0, -126)) continue;
    const float want = (float)v;
    if (fbits(d2f_rn(v)) != fbits(want)) ++bad;
    if (f2d_bits(want) != (double)want) ++bad;
  }
  const float mx = d2f_rn(3.4028234663852886e38), ov = d2f_rn(3.5e38), tiny = d2f_rn(1e-40);
  printf("%.3e %.3e %.3e %g %g %g %g %ld %d %g %g\n", worst_rt, worst_add, worst_mul, z, one, m, big, bad,
         (int)(fbits(mx) == 0x7F7FFFFFu), (double)ov, (double)tiny);
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
    assert [float(v) for v in out[3:7]] == [0.0, 1.0, -0.375, 3.0e20]
    # binary64 -> binary32 conversion: bit-identical to the compiler's cast
    # on 2e6 values (a quarter of them exact ties), the largest float kept,
    # overflow to infinity, magnitudes below 2^-126 flushed to zero
    assert int(out[7]) == 0
    assert out[8] == "1" and out[9] == "inf" and float(out[10]) == 0.0
