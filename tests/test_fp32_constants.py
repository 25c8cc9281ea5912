"""The FP32 codelets' constants carried to FP64 accuracy (csrc/fft_codelets.cuh,
f32_hi / f32_lo): checked on the host (the header compiled by nvcc, host code
only; no GPU).

* the head + tail pair of every constant the FP32 codelets multiply by
  (sin 2pi/3, cos pi/4, the 5-point DFT's cos / sin of 2pi/5 and 4pi/5, the
  twiddles of the 16- and 32-point composite DFTs) reproduces the FP64
  constant to about 2^-48 relative;
* a product fma(hi, a, lo * a) in FP32 is the correctly rounded c * a up to a
  few 2^-24 ulp, where the nearest-rounded constant alone errs by up to about
  one ulp;
* nearest-rounded (cos, sin) pairs of those roots of unity lie off the unit
  circle by up to ~1e-7 (the per-transform scaling that made long FP32 pushes
  drift), the head + tail pairs by at most ~1e-15."""
import os
import shutil
import subprocess
import tempfile

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_1812_07357_gb300", "csrc")

SRC = r'''
#include <cmath>
#include <cstdio>
#include <random>
#include <vector>
#include "fft_codelets.cuh"
using psatd::f32_hi;
using psatd::f32_lo;
using psatd::root_cos;
using psatd::root_sin;

static double ulp_of(float x) { return (double)std::nextafter(std::fabs(x), INFINITY) - (double)std::fabs(x); }

int main() {
  std::vector<double> cs = {root_sin(3, 1), root_cos(8, 1), root_cos(5, 1), root_cos(5, 2), root_sin(5, 1),
                            root_sin(5, 2)};
  std::vector<std::pair<double, double>> roots;
  for (int R : {16, 32})
    for (int k = 1; k < R; ++k) {
      cs.push_back(root_cos(R, k));
      cs.push_back(root_sin(R, k));
      roots.push_back({root_cos(R, k), root_sin(R, k)});
    }
  std::mt19937_64 g(12345);
  std::uniform_real_distribution<double> e(-10.0, 10.0), u(0.0, 1.0);
  double split = 0, prod_hl = 0, prod_near = 0;
  for (double c : cs) {
    if (c == 0.0) continue;
    const float hi = f32_hi(c), lo = f32_lo(c);
    split = std::fmax(split, std::fabs(((double)hi + (double)lo) - c) / std::fabs(c));
    for (int i = 0; i < 20000; ++i) {
      const float a = (float)((u(g) < 0.5 ? -1.0 : 1.0) * std::exp2(e(g)) * (1.0 + u(g)));
      const double exact = c * (double)a;
      const float p_hl = std::fmaf(hi, a, lo * a);
      const float p_near = hi * a;
      const double ulp = ulp_of((float)exact);
      prod_hl = std::fmax(prod_hl, std::fabs((double)p_hl - exact) / ulp);
      prod_near = std::fmax(prod_near, std::fabs((double)p_near - exact) / ulp);
    }
  }
  double circ_near = 0, circ_hl = 0;
  for (auto& r : roots) {
    const double cn = (double)f32_hi(r.first), sn = (double)f32_hi(r.second);
    const double ch = cn + (double)f32_lo(r.first), sh = sn + (double)f32_lo(r.second);
    circ_near = std::fmax(circ_near, std::fabs(cn * cn + sn * sn - 1.0));
    circ_hl = std::fmax(circ_hl, std::fabs(ch * ch + sh * sh - 1.0));
  }
  std::printf("%.6e %.6e %.6e %.6e %.6e\n", split, prod_hl, prod_near, circ_near, circ_hl);
  return 0;
}
'''


def _nvcc():
    for c in (shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if c and os.path.exists(c):
            return c
    return None


@pytest.fixture(scope="module")
def figures():
    nvcc = _nvcc()
    if not nvcc:
        pytest.skip("nvcc not available")
    with tempfile.TemporaryDirectory() as d:
        src = os.path.join(d, "t.cu")
        exe = os.path.join(d, "t")
        open(src, "w").write(SRC)
        r = subprocess.run([nvcc, "-std=c++17", "-O1", "--expt-relaxed-constexpr",
                            "-gencode", "arch=compute_103a,code=sm_103a", "-I", CSRC, src, "-o", exe],
                           capture_output=True, text=True)
        assert r.returncode == 0, r.stderr
        out = subprocess.run([exe], check=True, capture_output=True, text=True).stdout.split()
    return dict(zip(("split", "prod_hl", "prod_near", "circ_near", "circ_hl"), map(float, out)))


def test_head_and_tail_reproduce_the_fp64_constant(figures):
    assert figures["split"] < 2.0 ** -47, figures


def test_head_tail_product_is_correctly_rounded(figures):
    # fl(hi a + fl(lo a)): one rounding of c a off by at most ~2^-47 |c a|
    assert figures["prod_hl"] <= 0.5 + 2.0 ** -20, figures
    # the nearest-rounded constant alone adds its own error |lo a| ~ 0.5 ulp
    assert figures["prod_near"] > 0.75, figures


def test_rounded_roots_leave_the_unit_circle(figures):
    assert 1e-9 < figures["circ_near"] < 2.0 ** -22, figures
    assert figures["circ_hl"] < 1e-14, figures
