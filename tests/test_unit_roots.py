"""The compile-time twiddle constants of the register FFT codelets
(csrc/unit_roots.h, Taylor series after exact octant reduction) agree with
the C library's cos / sin to a few units of the last place, for every root
of unity of order <= 512 (checked on the host, compiled with g++)."""
import os
import shutil
import subprocess
import tempfile

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HDR = os.path.join(ROOT, "paper_1812_07357_gb300", "csrc", "unit_roots.h")

SRC = r'''
#include <cmath>
#include <cstdio>
#include "unit_roots.h"
constexpr double c_48_7 = psatd::root_cos(48, 7);   // forces compile-time evaluation
static_assert(c_48_7 > 0.60 && c_48_7 < 0.61, "cos(2 pi 7/48)");
int main() {
  double worst = 0;
  for (int R = 1; R <= 512; ++R)
    for (int m = -R; m < 2 * R; ++m) {
      const long double a = 2.0L * 3.14159265358979323846264338327950288L * m / R;
      const double ec = std::fabs(psatd::root_cos(R, m) - (double)std::cos(a));
      const double es = std::fabs(psatd::root_sin(R, m) - (double)std::sin(a));
      if (ec > worst) worst = ec;
      if (es > worst) worst = es;
    }
  std::printf("%.3e\n", worst);
  return 0;
}
'''


def test_unit_roots_match_libm():
    gxx = shutil.which("g++")
    if not gxx:
        pytest.skip("g++ not available")
    with tempfile.TemporaryDirectory() as d:
        src = os.path.join(d, "t.cpp")
        exe = os.path.join(d, "t")
        open(src, "w").write(SRC)
        subprocess.run([gxx, "-std=c++17", "-O1", "-I", os.path.dirname(HDR), src, "-o", exe],
                       check=True, capture_output=True)
        worst = float(subprocess.run([exe], check=True, capture_output=True, text=True).stdout)
    assert worst < 4.5e-16, worst
