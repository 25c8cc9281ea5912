// Compile-time values of cos(2 pi m / R) and sin(2 pi m / R), used as
// immediate twiddle constants by the register-resident FFT codelets.
//
// Method: the angle is reduced exactly in integer arithmetic to an octant o
// and a remainder phi in [0, pi/4), then the Taylor series of sin / cos at 0
// (17 terms; the first omitted term is below 1e-40 on [0, pi/4]) gives the
// value of phi or of pi/4 - phi, and the octant's symmetry gives the result.
// Plain C++17, no device code: also compiled by the host-side accuracy test.
#pragma once

namespace psatd {

constexpr double kPi = 3.141592653589793238462643383279502884;

constexpr double taylor_sin(double x) {
  double x2 = x * x, t = x, s = x;
  for (int k = 1; k < 17; ++k) {
    t *= -x2 / ((2.0 * k) * (2.0 * k + 1.0));
    s += t;
  }
  return s;
}

constexpr double taylor_cos(double x) {
  double x2 = x * x, t = 1.0, s = 1.0;
  for (int k = 1; k < 17; ++k) {
    t *= -x2 / ((2.0 * k - 1.0) * (2.0 * k));
    s += t;
  }
  return s;
}

// which = 0: cos(2 pi m / R); which = 1: sin(2 pi m / R)
constexpr double unit_root(int R, long long m, int which) {
  m %= R;
  if (m < 0) m += R;
  const long long e = 8LL * m;
  const int o = (int)(e / R);
  const long long r = e - (long long)o * R;          // angle = (o + r/R) pi/4
  const double phi = (kPi / 4) * ((double)r / (double)R);
  const double psi = (kPi / 4) * ((double)(R - r) / (double)R);
  const double cp = taylor_cos(phi), sp = taylor_sin(phi);
  const double cq = taylor_cos(psi), sq = taylor_sin(psi);
  double c = 0, s = 0;
  switch (o) {
    case 0: c = cp; s = sp; break;      // theta = phi
    case 1: c = sq; s = cq; break;      // theta = pi/2 - psi
    case 2: c = -sp; s = cp; break;     // theta = pi/2 + phi
    case 3: c = -cq; s = sq; break;     // theta = pi - psi
    case 4: c = -cp; s = -sp; break;    // theta = pi + phi
    case 5: c = -sq; s = -cq; break;    // theta = 3 pi/2 - psi
    case 6: c = sp; s = -cp; break;     // theta = 3 pi/2 + phi
    default: c = cq; s = -sq; break;    // theta = 2 pi - psi
  }
  return which ? s : c;
}

constexpr double root_cos(int R, long long m) { return unit_root(R, m, 0); }
constexpr double root_sin(int R, long long m) { return unit_root(R, m, 1); }

}  // namespace psatd
