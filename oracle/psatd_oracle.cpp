// FP64 reference implementation ("oracle") of the PSATD Maxwell push, in
// plain C++ with its own FFT.
//
// TEST INFRASTRUCTURE.  Only the test-suite, the smoke check of the package
// entry point and the CPU-baseline leg of the benchmark load this library
// (through oracle/psatd_oracle.py).  It shares no code, header or table with
// the CUDA library, and the CUDA library never loads it.
//
// What one step computes (paper Fig. 1 caption: (i) advance every sub-domain
// with its own FFTs, (ii) exchange guard cells):
//   1. per box, the 3D DFT of every field component over the whole padded box
//      (guards included), the box taken as periodic (Sec. 1.3: local FFTs on
//      sub-domains padded with n_g guard cells);
//   2. per mode, the analytical update of Maxwell's equations in Fourier space
//      (Sec. 1.1: PSATD, exact in time for every mode) with the derivative
//      replaced by the Fourier symbol of an order-p staggered stencil of width
//      p/2 (Sec. 1.1; p = 0 stands for infinite order, the pure spectral
//      derivative) and Yee-staggered component positions;
//   3. the inverse 3D DFT (factor 1/N), real part;
//   4. the guard exchange: every guard cell takes the value of the interior
//      cell that owns the same global position (Fig. 1a/1b, step (ii); for a
//      hybrid group, Sec. 2.1, guards exist on the split axes only).
//
// The paper prints none of the PSATD equations (only the principle, Sec.
// 1.1).  The update used here is the exact solution over one step of
//     dE/dt = c^2 (i K x B) - J/eps0,     dB/dt = -(i K x E),
// with J constant over the step.  With K = |K|, theta = c K dt:
//     C  = cos(theta)
//     Sw = sin(theta)/(c K)     = dt sinc(theta)
//     X1 = (1 - C)/K^2          = (c dt)^2/2 sinc(theta/2)^2
//     X3 = (Sw - dt)/K^2        = c^2 dt^3 (sinc(theta) - 1)/theta^2
//   J form:   E' = C E + X1 K (K.E) + i c^2 Sw K x B - Sw J/eps0 + X3 K (K.J)/eps0
//             B' = C B + X1 K (K.B) - i Sw K x E + i (X1/c^2) K x J/eps0
//   rho form: rho' = rho - i dt K.J (continuity), and
//             E' = C E + i c^2 Sw K x B - Sw J/eps0 + i K (Y1 rho' + Y2 rho)/eps0,
//             Y1 = X3/dt, Y2 = -X1 - X3/dt  (longitudinal E from Gauss's law)
//   vacuum:   the J form with J = 0.
// 1 - C is evaluated as 2 sin^2(theta/2) (through sinc(theta/2)); the bracket
// (sinc(theta) - 1)/theta^2 takes its Taylor series below theta = 0.1.
//
// Fourier convention: forward transform unnormalised with exp(-2 pi i m j/N),
// inverse with 1/N, so a derivative becomes +i K.  Index m of an N-cell axis
// has k = 2 pi m~/(N h), m~ = m for m <= N/2 and m - N above (the Nyquist
// index takes k = +pi/h).  A component sampled at offset s (cells) is centred
// by exp(-i k.s h) before the update and shifted back by exp(+i k.s h).
//
// Order-p staggered stencil: K(k) = sum_{l=1}^{p/2} alpha_l 2 sin((2l-1)kh/2)
// / ((2l-1)h), alpha_l = prod_{j != l} (2j-1)^2 / ((2j-1)^2 - (2l-1)^2) (the
// weights exact to O(h^p)).  Nodal variant (not in the paper, which uses
// staggered stencils): K = sum_l beta_l sin(l k h)/(l h), beta_l = prod_{j != l}
// j^2/(j^2 - l^2), every component at the nodes, and K = 0 at the Nyquist
// index for infinite order.
//
// FFT: recursive mixed-radix decimation in time, radix 4, 2, 3, 5 (a direct
// DFT for any other factor), twiddles cos/sin(2 pi j/N) in double.  The whole
// complex spectrum is computed (no real-to-complex shortcut).
//
// Absorbing layers (PML; the paper only states that the solver supports the
// two-step perfectly matched layer of its reference [shapoval2019two], with
// no equations).  Reading, derived here from Maxwell's equations in vacuum:
// each component is split by derivative direction (Berenger), e.g.
//     E_x = E_xy + E_xz,  dE_xy/dt + s_y E_xy = c^2 dB_z/dy,
//                         dE_xz/dt + s_z E_xz = -c^2 dB_y/dz,
// and likewise for E_y (y-z... parts z, x), E_z (x, y), B_x (y, z), B_y (z, x),
// B_z (x, y) with dB/dt = -curl E.  One step is two exact sub-steps:
//  (1) s = 0: the split parts sum to the usual fields, so E, B take the
//      ordinary PSATD step, and each split part gains the time integral of
//      its own derivative term over the step, which depends on E^n, B^n only.
//      With the mode solution E(t), B(t) of the update above (vacuum),
//        I[E] = int_0^dt E = Sw E - X3 K (K.E) + i X1 K x B,
//        I[B] = int_0^dt B = Sw B - X3 K (K.B) - i (X1/c^2) K x E,
//      so e.g. dE_xy = i c^2 K_y I[B_z], dB_xy = -i K_y I[E_z];
//  (2) each split part along direction d is multiplied by exp(-s_d dt) (the
//      exact solution of dF/dt = -s_d F), and the component is the sum again.
// One split part per component is stored (E_xy, E_yz, E_zx, B_xy, B_yz,
// B_zx); the other is the component minus it.  s_d = s_max,d (xi/w_d)^m at
// depth xi (cells) into a layer of w_d cells on each face of axis d of the
// global domain, evaluated at the component's Yee position; 0 outside the
// layers.  The layers hold no current (vacuum form only).
//
// The push is a template on the arithmetic type.  double is the oracle.  The
// float instantiation (precision 32) carries out the same steps in FP32
// arithmetic and storage, with the twiddles, phases and coefficients computed
// in double and rounded once: a model of the FP32 rounding floor of this
// algorithm, used only to set tolerances, never as a reference.
#include <algorithm>
#include <cmath>
#include <complex>
#include <cstdint>
#include <cstring>
#include <vector>

#ifdef _OPENMP
#include <omp.h>
#endif

namespace {

constexpr double kPi = 3.14159265358979323846264338327950288;

template <typename T>
using cx = std::complex<T>;

// complex product written out (no library call for inf/nan handling)
template <typename T>
inline cx<T> mul(cx<T> a, cx<T> b) {
  return cx<T>(a.real() * b.real() - a.imag() * b.imag(), a.real() * b.imag() + a.imag() * b.real());
}

// ---------------------------------------------------------------------------
// FFT
// ---------------------------------------------------------------------------

// w^j = exp(sign 2 pi i j / N), j < N, computed in double, rounded to T.
template <typename T>
std::vector<cx<T>> unit_roots(int N, int sign) {
  std::vector<cx<T>> w(N);
  for (int j = 0; j < N; ++j) {
    const double a = 2.0 * kPi * (double)j / (double)N;
    w[j] = cx<T>((T)std::cos(a), (T)(sign * std::sin(a)));
  }
  return w;
}

int first_radix(int n) {
  if (n % 4 == 0) return 4;
  for (int r : {2, 3, 5})
    if (n % r == 0) return r;
  return n;  // any other factor: a direct DFT of the whole length
}

// out[k] = sum_{j<n} in[j*is] w_n^{jk}, w_n = W[N/n] (W: the N roots of the
// top-level length).  Decimation in time: the r sub-sequences in[q + r j]
// are transformed into out[q*m .. q*m + m), then for every k < m the r values
// out[q*m + k] w_n^{qk} go through an r-point DFT into out[k + s*m].
template <typename T>
void fft_rec(const cx<T>* in, ptrdiff_t is, cx<T>* out, int n, const cx<T>* W, int N) {
  if (n == 1) {
    out[0] = in[0];
    return;
  }
  const int r = first_radix(n), m = n / r;
  for (int q = 0; q < r; ++q) fft_rec(in + q * is, is * r, out + (ptrdiff_t)q * m, m, W, N);
  const int64_t step = N / n;  // W index of w_n
  cx<T> small[5];
  std::vector<cx<T>> big(r > 5 ? r : 0);
  cx<T>* t = r > 5 ? big.data() : small;
  for (int k = 0; k < m; ++k) {
    for (int q = 0; q < r; ++q) t[q] = mul(out[(ptrdiff_t)q * m + k], W[(q * k * step) % N]);
    for (int s = 0; s < r; ++s) {
      cx<T> acc(0, 0);
      for (int q = 0; q < r; ++q) acc += mul(t[q], W[((int64_t)q * s * m * step) % N]);
      out[k + (ptrdiff_t)s * m] = acc;
    }
  }
}

// In-place unnormalised 3D DFT of a (nz, ny, nx) complex array (x fastest),
// sign -1 forward, +1 inverse; one 1D transform per line, axis by axis.
template <typename T>
void fft3(cx<T>* a, int nx, int ny, int nz, int sign) {
  const int n[3] = {nx, ny, nz};
  const int64_t stride[3] = {1, nx, (int64_t)nx * ny};
  for (int ax = 0; ax < 3; ++ax) {
    const int len = n[ax];
    if (len == 1) continue;
    const std::vector<cx<T>> W = unit_roots<T>(len, sign);
    // lines: every index of the other two axes
    const int o1 = ax == 0 ? 1 : 0, o2 = ax == 2 ? 1 : 2;
    const int64_t nlines = (int64_t)n[o1] * n[o2];
#pragma omp parallel if (nlines * len >= 65536)
    {
      std::vector<cx<T>> src(len), dst(len);
#pragma omp for schedule(static)
      for (int64_t l = 0; l < nlines; ++l) {
        const int64_t i1 = l % n[o1], i2 = l / n[o1];
        cx<T>* base = a + i1 * stride[o1] + i2 * stride[o2];
        for (int j = 0; j < len; ++j) src[j] = base[j * stride[ax]];
        fft_rec(src.data(), 1, dst.data(), len, W.data(), len);
        for (int j = 0; j < len; ++j) base[j * stride[ax]] = dst[j];
      }
    }
  }
}

// ---------------------------------------------------------------------------
// Stencils, wavenumbers and coefficients (all in double)
// ---------------------------------------------------------------------------

// alpha_l (staggered, nodes (2l-1)^2) or beta_l (nodal, nodes l^2), l = 1..p/2:
// the Lagrange basis of the nodes evaluated at 0.
std::vector<double> weights(int p, bool nodal) {
  const int q = p / 2;
  std::vector<double> w(q);
  for (int l = 1; l <= q; ++l) {
    const long double nl = nodal ? (long double)l * l : (long double)(2 * l - 1) * (2 * l - 1);
    long double a = 1;
    for (int j = 1; j <= q; ++j) {
      if (j == l) continue;
      const long double nj = nodal ? (long double)j * j : (long double)(2 * j - 1) * (2 * j - 1);
      a *= nj / (nj - nl);
    }
    w[l - 1] = (double)a;
  }
  return w;
}

// Fourier symbol K(k) of the order-p difference (p = 0: infinite order).
double modified_k(double k, double h, int p, bool nodal, const std::vector<double>& w) {
  if (p == 0) {
    if (nodal && std::fabs(std::fabs(k * h) - kPi) <= 1e-12) return 0.0;
    return k;
  }
  double K = 0;
  for (int l = 1; l <= p / 2; ++l) {
    if (nodal)
      K += w[l - 1] * std::sin(l * k * h) / (l * h);
    else {
      const int m = 2 * l - 1;
      K += w[l - 1] * 2.0 * std::sin(m * k * h / 2.0) / (m * h);
    }
  }
  return K;
}

double true_k(int m, int n, double h) {
  const int mt = m <= n / 2 ? m : m - n;
  return 2.0 * kPi * mt / (n * h);
}

double sinc(double x) { return x == 0.0 ? 1.0 : std::sin(x) / x; }

struct Coef {
  double C, Sw, X1, X3;
};

Coef coefficients(double K2, double c, double dt) {
  const double th = c * dt * std::sqrt(K2);
  Coef r;
  r.C = std::cos(th);
  r.Sw = dt * sinc(th);
  const double s2 = sinc(0.5 * th);
  r.X1 = 0.5 * (c * dt) * (c * dt) * s2 * s2;
  double g;
  if (std::fabs(th) < 0.1) {
    // (sinc(t) - 1)/t^2 = sum_{j>=1} (-1)^j t^(2j-2)/(2j+1)!
    const double t2 = th * th;
    g = -1.0 / 6 + t2 * (1.0 / 120 + t2 * (-1.0 / 5040 + t2 * (1.0 / 362880 + t2 * (-1.0 / 39916800))));
  } else {
    g = (std::sin(th) / th - 1.0) / (th * th);
  }
  r.X3 = c * c * dt * dt * dt * g;
  return r;
}

// Yee offsets (cells) of E_x, E_y, E_z, B_x, B_y, B_z, J_x, J_y, J_z, rho.
const double kYee[10][3] = {{0.5, 0, 0}, {0, 0.5, 0}, {0, 0, 0.5}, {0, 0.5, 0.5}, {0.5, 0, 0.5},
                            {0.5, 0.5, 0}, {0.5, 0, 0}, {0, 0.5, 0}, {0, 0, 0.5}, {0, 0, 0}};

enum Form { kVacuum = 0, kJ = 1, kRho = 2 };

// One mode: centred spectra E, B (J, R) -> E', B' (R').  T arithmetic with
// coefficients given in T.
template <typename T>
struct ModeCoef {
  T K[3], C, Sw, X1, X3, Y1, Y2, cc, ieps, dt, icc;
};

template <typename T>
inline void update_mode(cx<T>* E, cx<T>* B, const cx<T>* J, cx<T>* R, const ModeCoef<T>& m, int form) {
  const T* K = m.K;
  const cx<T> I(0, 1);
  const cx<T> KxB[3] = {K[1] * B[2] - K[2] * B[1], K[2] * B[0] - K[0] * B[2], K[0] * B[1] - K[1] * B[0]};
  const cx<T> KxE[3] = {K[1] * E[2] - K[2] * E[1], K[2] * E[0] - K[0] * E[2], K[0] * E[1] - K[1] * E[0]};
  const cx<T> KdB = K[0] * B[0] + K[1] * B[1] + K[2] * B[2];
  cx<T> Bn[3], En[3];
  for (int d = 0; d < 3; ++d) Bn[d] = m.C * B[d] + m.X1 * K[d] * KdB - mul(I, m.Sw * KxE[d]);
  if (form == kRho) {
    const cx<T> KdJ = K[0] * J[0] + K[1] * J[1] + K[2] * J[2];
    const cx<T> Rn = *R - mul(I, m.dt * KdJ);
    const cx<T> L = m.Y1 * Rn + m.Y2 * (*R);
    for (int d = 0; d < 3; ++d)
      En[d] = m.C * E[d] + mul(I, m.cc * m.Sw * KxB[d]) - m.Sw * J[d] * m.ieps + mul(I, K[d] * L) * m.ieps;
    *R = Rn;
  } else {
    const cx<T> KdE = K[0] * E[0] + K[1] * E[1] + K[2] * E[2];
    for (int d = 0; d < 3; ++d) En[d] = m.C * E[d] + m.X1 * K[d] * KdE + mul(I, m.cc * m.Sw * KxB[d]);
    if (form == kJ) {
      const cx<T> KdJ = K[0] * J[0] + K[1] * J[1] + K[2] * J[2];
      for (int d = 0; d < 3; ++d) En[d] += -m.Sw * J[d] * m.ieps + m.X3 * K[d] * KdJ * m.ieps;
    }
  }
  if (form != kVacuum) {
    const cx<T> KxJ[3] = {K[1] * J[2] - K[2] * J[1], K[2] * J[0] - K[0] * J[2], K[0] * J[1] - K[1] * J[0]};
    for (int d = 0; d < 3; ++d) Bn[d] += mul(I, m.X1 * m.icc * KxJ[d] * m.ieps);
  }
  for (int d = 0; d < 3; ++d) {
    E[d] = En[d];
    B[d] = Bn[d];
  }
}

template <typename T>
ModeCoef<T> mode_coef(const double K[3], double c, double eps0, double dt) {
  const Coef q = coefficients(K[0] * K[0] + K[1] * K[1] + K[2] * K[2], c, dt);
  ModeCoef<T> m;
  for (int d = 0; d < 3; ++d) m.K[d] = (T)K[d];
  m.C = (T)q.C;
  m.Sw = (T)q.Sw;
  m.X1 = (T)q.X1;
  m.X3 = (T)q.X3;
  m.Y1 = (T)(q.X3 / dt);
  m.Y2 = (T)(-q.X1 - q.X3 / dt);
  m.cc = (T)(c * c);
  m.ieps = (T)(1.0 / eps0);
  m.dt = (T)dt;
  m.icc = (T)(1.0 / (c * c));
  return m;
}

// ---------------------------------------------------------------------------
// One PSATD step of one periodic box
// ---------------------------------------------------------------------------

// f: 6 real arrays (E, B) in/out; j: 3 real arrays or nullptr; rho in/out or
// nullptr.  Cells x fastest.  Returns the largest |imaginary part| met in the
// inverse transforms (a real result needs Hermitian spectra).
// Split parts stored per component (PML): E_x along y, E_y along z, E_z
// along x, B_x along y, B_y along z, B_z along x.
const int kSplitDir[6] = {1, 2, 0, 1, 2, 0};

template <typename T>
double push_box(int nx, int ny, int nz, const double h[3], int p, double dt, double c, double eps0, int form,
                bool nodal, T* const* f, const T* const* j, T* rho, T* const* dsplit = nullptr) {
  const int64_t N = (int64_t)nx * ny * nz;
  const int nslots = form == kVacuum ? 6 : form == kJ ? 9 : 10;
  std::vector<std::vector<cx<T>>> S(nslots, std::vector<cx<T>>(N));
  // increments of the stored split parts (centred, then shifted like their
  // components), when asked for
  std::vector<std::vector<cx<T>>> D(dsplit ? 6 : 0, std::vector<cx<T>>(N));
  // slots 0-5: E, B; 6-8: J; 9: rho (component index into kYee)
  for (int s = 0; s < nslots; ++s) {
    const T* src = s < 6 ? f[s] : s < 9 ? j[s - 6] : rho;
#pragma omp parallel for schedule(static) if (N >= 65536)
    for (int64_t i = 0; i < N; ++i) S[s][i] = cx<T>(src[i], 0);
    fft3(S[s].data(), nx, ny, nz, -1);
  }
  const std::vector<double> w = p ? weights(p, nodal) : std::vector<double>();
  std::vector<double> k[3], Kd[3];
  const int n[3] = {nx, ny, nz};
  for (int d = 0; d < 3; ++d) {
    k[d].resize(n[d]);
    Kd[d].resize(n[d]);
    for (int m = 0; m < n[d]; ++m) {
      k[d][m] = true_k(m, n[d], h[d]);
      Kd[d][m] = modified_k(k[d][m], h[d], p, nodal, w);
    }
  }
#pragma omp parallel for schedule(static) if (N >= 16384)
  for (int64_t idx = 0; idx < N; ++idx) {
    const int mx = (int)(idx % nx), my = (int)((idx / nx) % ny), mz = (int)(idx / ((int64_t)nx * ny));
    const double kk[3] = {k[0][mx], k[1][my], k[2][mz]};
    const double KK[3] = {Kd[0][mx], Kd[1][my], Kd[2][mz]};
    cx<T> ph[10];  // exp(-i k.s h) per component (1 on the nodal grid)
    for (int s = 0; s < 10; ++s) {
      if (nodal) {
        ph[s] = cx<T>(1, 0);
        continue;
      }
      const double a = kk[0] * kYee[s][0] * h[0] + kk[1] * kYee[s][1] * h[1] + kk[2] * kYee[s][2] * h[2];
      ph[s] = cx<T>((T)std::cos(a), (T)(-std::sin(a)));
    }
    cx<T> E[3], B[3], J[3], R(0, 0);
    for (int d = 0; d < 3; ++d) {
      E[d] = mul(S[d][idx], ph[d]);
      B[d] = mul(S[3 + d][idx], ph[3 + d]);
      J[d] = form != kVacuum ? mul(S[6 + d][idx], ph[6 + d]) : cx<T>(0, 0);
    }
    if (form == kRho) R = mul(S[9][idx], ph[9]);
    const ModeCoef<T> mc = mode_coef<T>(KK, c, eps0, dt);
    if (dsplit) {
      // time integrals of E and B over the step (vacuum mode solution)
      const T* K = mc.K;
      const cx<T> I(0, 1);
      const cx<T> KdE = K[0] * E[0] + K[1] * E[1] + K[2] * E[2];
      const cx<T> KdB = K[0] * B[0] + K[1] * B[1] + K[2] * B[2];
      const cx<T> KxE[3] = {K[1] * E[2] - K[2] * E[1], K[2] * E[0] - K[0] * E[2], K[0] * E[1] - K[1] * E[0]};
      const cx<T> KxB[3] = {K[1] * B[2] - K[2] * B[1], K[2] * B[0] - K[0] * B[2], K[0] * B[1] - K[1] * B[0]};
      cx<T> IE[3], IB[3];
      for (int d = 0; d < 3; ++d) {
        IE[d] = mc.Sw * E[d] - mc.X3 * K[d] * KdE + mul(I, mc.X1 * KxB[d]);
        IB[d] = mc.Sw * B[d] - mc.X3 * K[d] * KdB - mul(I, mc.X1 * mc.icc * KxE[d]);
      }
      // dE_xy = i c^2 K_y I[B_z], dE_yz = i c^2 K_z I[B_x], dE_zx = i c^2 K_x I[B_y]
      // dB_xy = -i K_y I[E_z],    dB_yz = -i K_z I[E_x],    dB_zx = -i K_x I[E_y]
      const cx<T> d6[6] = {mul(I, mc.cc * K[1] * IB[2]), mul(I, mc.cc * K[2] * IB[0]), mul(I, mc.cc * K[0] * IB[1]),
                           -mul(I, K[1] * IE[2]), -mul(I, K[2] * IE[0]), -mul(I, K[0] * IE[1])};
      for (int q = 0; q < 6; ++q) D[q][idx] = mul(d6[q], std::conj(ph[q]));
    }
    update_mode(E, B, J, &R, mc, form);
    for (int d = 0; d < 3; ++d) {
      S[d][idx] = mul(E[d], std::conj(ph[d]));
      S[3 + d][idx] = mul(B[d], std::conj(ph[3 + d]));
    }
    if (form == kRho) S[9][idx] = mul(R, std::conj(ph[9]));
  }
  double imag = 0;
  const T inv = (T)(1.0 / (double)N);
  for (int s = 0; s < nslots; ++s) {
    if (s >= 6 && s < 9) continue;
    if (s == 9 && form != kRho) continue;
    fft3(S[s].data(), nx, ny, nz, +1);
    T* dst = s < 6 ? f[s] : rho;
    double im = 0;
#pragma omp parallel for schedule(static) reduction(max : im) if (N >= 65536)
    for (int64_t i = 0; i < N; ++i) {
      dst[i] = S[s][i].real() * inv;
      im = std::max(im, (double)std::fabs(S[s][i].imag() * inv));
    }
    imag = std::max(imag, im);
  }
  for (int q = 0; q < (dsplit ? 6 : 0); ++q) {
    fft3(D[q].data(), nx, ny, nz, +1);
#pragma omp parallel for schedule(static) if (N >= 65536)
    for (int64_t i = 0; i < N; ++i) dsplit[q][i] = D[q][i].real() * inv;
  }
  return imag;
}

}  // namespace

// ===========================================================================
// C interface (ctypes)
// ===========================================================================
extern "C" {

typedef struct {
  int32_t n[3], ng_lo[3], ng_hi[3];
  int64_t origin[3];
  int32_t p;
} oracle_box;

// kind: 0 global, 1 local, 2 hybrid, 3 independent (self-periodic boxes)
typedef struct {
  int32_t kind;
  int32_t global_n[3];
  int32_t periodic[3];
  int32_t nbox;
  const oracle_box* boxes;
} oracle_layout;

int oracle_threads(void) {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}

// In-place unnormalised 3D DFT of nz*ny*nx complex values (interleaved re, im;
// x fastest).  sign -1 forward, +1 inverse.  precision 64 (double) or 32 (the
// data is then float).
int oracle_fft3(int nx, int ny, int nz, int sign, int precision, void* data) {
  if (nx < 1 || ny < 1 || nz < 1 || (sign != 1 && sign != -1)) return 1;
  if (precision == 64)
    fft3(static_cast<cx<double>*>(data), nx, ny, nz, sign);
  else if (precision == 32)
    fft3(static_cast<cx<float>*>(data), nx, ny, nz, sign);
  else
    return 1;
  return 0;
}

// Stencil weights alpha_l (nodal = 0) or beta_l (nodal = 1), l = 1..p/2.
int oracle_weights(int p, int nodal, double* out) {
  if (p < 2 || p % 2) return 1;
  const std::vector<double> w = weights(p, nodal != 0);
  std::copy(w.begin(), w.end(), out);
  return 0;
}

// K(k) for n wavenumbers.
int oracle_modified_wavenumber(int64_t n, const double* k, double h, int p, int nodal, double* K) {
  if (p != 0 && (p < 2 || p % 2)) return 1;
  const std::vector<double> w = p ? weights(p, nodal != 0) : std::vector<double>();
  for (int64_t i = 0; i < n; ++i) K[i] = modified_k(k[i], h, p, nodal != 0, w);
  return 0;
}

// C, Sw, X1, X3 for n values of K^2.
int oracle_coefficients(int64_t n, const double* K2, double c, double dt, double* C, double* Sw, double* X1,
                        double* X3) {
  for (int64_t i = 0; i < n; ++i) {
    const Coef q = coefficients(K2[i], c, dt);
    C[i] = q.C;
    Sw[i] = q.Sw;
    X1[i] = q.X1;
    X3[i] = q.X3;
  }
  return 0;
}

// Per-mode update of n centred modes, in place.  E, B: 3 arrays of n complex
// (interleaved); J: 3 arrays or NULL; R: n complex or NULL; K: 3 arrays of n.
int oracle_update_modes(int64_t n, double* const* E, double* const* B, const double* const* J, double* R,
                        const double* const* K, double dt, double c, double eps0, int form) {
  if (form < 0 || form > 2 || (form != kVacuum && !J) || (form == kRho && !R)) return 1;
  for (int64_t i = 0; i < n; ++i) {
    cx<double> e[3], b[3], jj[3], r(0, 0);
    double KK[3];
    for (int d = 0; d < 3; ++d) {
      e[d] = cx<double>(E[d][2 * i], E[d][2 * i + 1]);
      b[d] = cx<double>(B[d][2 * i], B[d][2 * i + 1]);
      jj[d] = form != kVacuum ? cx<double>(J[d][2 * i], J[d][2 * i + 1]) : cx<double>(0, 0);
      KK[d] = K[d][i];
    }
    if (form == kRho) r = cx<double>(R[2 * i], R[2 * i + 1]);
    update_mode(e, b, jj, &r, mode_coef<double>(KK, c, eps0, dt), form);
    for (int d = 0; d < 3; ++d) {
      E[d][2 * i] = e[d].real();
      E[d][2 * i + 1] = e[d].imag();
      B[d][2 * i] = b[d].real();
      B[d][2 * i + 1] = b[d].imag();
    }
    if (form == kRho) {
      R[2 * i] = r.real();
      R[2 * i + 1] = r.imag();
    }
  }
  return 0;
}

}  // extern "C"

namespace {

int64_t cells(const oracle_box& b) { return (int64_t)b.n[0] * b.n[1] * b.n[2]; }

bool has_guards(const oracle_layout* L) {
  for (int i = 0; i < L->nbox; ++i)
    for (int d = 0; d < 3; ++d)
      if (L->boxes[i].ng_lo[d] || L->boxes[i].ng_hi[d]) return true;
  return false;
}

// The global field assembled from the box interiors (which must tile it);
// returns false when they do not.
bool assemble(const oracle_layout* L, const double* data, std::vector<double>& G) {
  const int64_t gx = L->global_n[0], gy = L->global_n[1], gz = L->global_n[2];
  G.assign(gx * gy * gz, 0.0);
  std::vector<uint8_t> cover(G.size(), 0);
  int64_t off = 0;
  for (int i = 0; i < L->nbox; ++i) {
    const oracle_box& b = L->boxes[i];
    int64_t m[3];
    for (int d = 0; d < 3; ++d) m[d] = b.n[d] - b.ng_lo[d] - b.ng_hi[d];
    for (int64_t z = 0; z < m[2]; ++z)
      for (int64_t y = 0; y < m[1]; ++y)
        for (int64_t x = 0; x < m[0]; ++x) {
          const int64_t X = b.origin[0] + x, Y = b.origin[1] + y, Z = b.origin[2] + z;
          if (X < 0 || X >= gx || Y < 0 || Y >= gy || Z < 0 || Z >= gz) return false;
          const int64_t g = X + gx * (Y + gy * Z);
          G[g] = data[off + (x + b.ng_lo[0]) + b.n[0] * ((y + b.ng_lo[1]) + b.n[1] * (z + b.ng_lo[2]))];
          ++cover[g];
        }
    off += cells(b);
  }
  for (uint8_t c : cover)
    if (c != 1) return false;
  return true;
}

// Every padded cell of every box reads the global cell origin - ng_lo + i
// (periodic axes wrap; non-periodic axes give 0 outside the domain).
void sample(const oracle_layout* L, const std::vector<double>& G, double* data) {
  const int64_t gn[3] = {L->global_n[0], L->global_n[1], L->global_n[2]};
  int64_t off = 0;
  for (int i = 0; i < L->nbox; ++i) {
    const oracle_box& b = L->boxes[i];
    for (int64_t z = 0; z < b.n[2]; ++z)
      for (int64_t y = 0; y < b.n[1]; ++y)
        for (int64_t x = 0; x < b.n[0]; ++x) {
          int64_t g[3] = {b.origin[0] - b.ng_lo[0] + x, b.origin[1] - b.ng_lo[1] + y,
                          b.origin[2] - b.ng_lo[2] + z};
          bool outside = false;
          for (int d = 0; d < 3; ++d) {
            if (L->periodic[d])
              g[d] = ((g[d] % gn[d]) + gn[d]) % gn[d];
            else if (g[d] < 0 || g[d] >= gn[d])
              outside = true;
          }
          data[off + x + b.n[0] * (y + b.n[1] * z)] = outside ? 0.0 : G[g[0] + gn[0] * (g[1] + gn[1] * g[2])];
        }
    off += cells(b);
  }
}

// Self-periodic boxes: every padded cell reads the interior cell at
// (i - ng_lo) mod interior (+ ng_lo).
void self_wrap(const oracle_layout* L, double* data) {
  int64_t off = 0;
  for (int i = 0; i < L->nbox; ++i) {
    const oracle_box& b = L->boxes[i];
    const int64_t N = cells(b);
    std::vector<double> src(data + off, data + off + N);
    int64_t m[3];
    for (int d = 0; d < 3; ++d) m[d] = b.n[d] - b.ng_lo[d] - b.ng_hi[d];
    for (int64_t z = 0; z < b.n[2]; ++z)
      for (int64_t y = 0; y < b.n[1]; ++y)
        for (int64_t x = 0; x < b.n[0]; ++x) {
          const int64_t sx = ((x - b.ng_lo[0]) % m[0] + m[0]) % m[0] + b.ng_lo[0];
          const int64_t sy = ((y - b.ng_lo[1]) % m[1] + m[1]) % m[1] + b.ng_lo[1];
          const int64_t sz = ((z - b.ng_lo[2]) % m[2] + m[2]) % m[2] + b.ng_lo[2];
          data[off + x + b.n[0] * (y + b.n[1] * z)] = src[sx + b.n[0] * (sy + b.n[1] * sz)];
        }
    off += N;
  }
}

int exchange(const oracle_layout* L, double* data) {
  if (L->kind == 3) {
    self_wrap(L, data);
    return 0;
  }
  std::vector<double> G;
  if (!assemble(L, data, G)) return 2;
  sample(L, G, data);
  return 0;
}

}  // namespace

extern "C" {
// Absorbing layers on both faces of every axis d with width[d] > 0 (cells):
// conductivity s_max[d] (xi/width[d])^order at depth xi into the layer.
typedef struct {
  int32_t width[3];
  double sigma_max[3];
  int32_t order;
} oracle_pml;
}

namespace {

// s_d at position pos (cells, Yee offset included) of an axis of n cells.
double pml_sigma(const oracle_pml* P, int d, double pos, int64_t n) {
  const double w = P->width[d];
  if (w <= 0) return 0.0;
  double xi = 0.0;
  if (pos < w)
    xi = w - pos;
  else if (pos > n - w)
    xi = pos - (n - w);
  xi = std::min(xi, w);
  return xi > 0 ? P->sigma_max[d] * std::pow(xi / w, (double)P->order) : 0.0;
}

// Step (2) of the PML on the interior cells of box i: add the split-part
// increments, damp both parts, and rebuild the components.
template <typename T>
void pml_damp(const oracle_layout* L, int i, const oracle_pml* P, double dt, T* const* f, const T* const* dsp,
              double* const* split, int64_t off) {
  const oracle_box& b = L->boxes[i];
  for (int q = 0; q < 6; ++q) {
    const int axis = q % 3, sa = kSplitDir[q], sb = 3 - axis - sa;
    const double* yee = kYee[q];
    for (int64_t z = b.ng_lo[2]; z < b.n[2] - b.ng_hi[2]; ++z)
      for (int64_t y = b.ng_lo[1]; y < b.n[1] - b.ng_hi[1]; ++y)
        for (int64_t x = b.ng_lo[0]; x < b.n[0] - b.ng_hi[0]; ++x) {
          const int64_t li = x + b.n[0] * (y + b.n[1] * z);
          const double pos[3] = {b.origin[0] + (x - b.ng_lo[0]) + yee[0], b.origin[1] + (y - b.ng_lo[1]) + yee[1],
                                 b.origin[2] + (z - b.ng_lo[2]) + yee[2]};
          const T ea = (T)std::exp(-pml_sigma(P, sa, pos[sa], L->global_n[sa]) * dt);
          const T eb = (T)std::exp(-pml_sigma(P, sb, pos[sb], L->global_n[sb]) * dt);
          const T ps = (T)split[q][off + li] + dsp[q][li];
          const T po = f[q][li] - ps;
          const T ns = ea * ps, no = eb * po;
          f[q][li] = ns + no;
          split[q][off + li] = (double)ns;
        }
  }
}

template <typename T>
int push_layout(const oracle_layout* L, double* const* fields, double* const* src, const uint8_t* mask,
                int nsteps, const double h[3], double dt, double c, double eps0, int form, bool nodal,
                double* max_imag, const oracle_pml* pml = nullptr, double* const* split = nullptr) {
  const bool guards = has_guards(L);
  double imag = 0;
  int64_t off = 0;
  std::vector<int64_t> offs(L->nbox);
  for (int i = 0; i < L->nbox; ++i) {
    offs[i] = off;
    off += cells(L->boxes[i]);
  }
  for (int step = 0; step < nsteps; ++step) {
    for (int i = 0; i < L->nbox; ++i) {
      if (mask && !mask[i]) continue;
      const oracle_box& b = L->boxes[i];
      const int64_t N = cells(b);
      std::vector<std::vector<T>> f(6, std::vector<T>(N)), jj(3), r;
      for (int s = 0; s < 6; ++s)
        for (int64_t q = 0; q < N; ++q) f[s][q] = (T)fields[s][offs[i] + q];
      if (form != kVacuum)
        for (int s = 0; s < 3; ++s) {
          jj[s].resize(N);
          for (int64_t q = 0; q < N; ++q) jj[s][q] = (T)src[s][offs[i] + q];
        }
      if (form == kRho) {
        r.resize(1, std::vector<T>(N));
        for (int64_t q = 0; q < N; ++q) r[0][q] = (T)src[3][offs[i] + q];
      }
      T* fp[6];
      const T* jp[3] = {nullptr, nullptr, nullptr};
      for (int s = 0; s < 6; ++s) fp[s] = f[s].data();
      if (form != kVacuum)
        for (int s = 0; s < 3; ++s) jp[s] = jj[s].data();
      std::vector<std::vector<T>> dsp(pml ? 6 : 0, std::vector<T>(N));
      T* dp[6];
      for (int q = 0; q < (pml ? 6 : 0); ++q) dp[q] = dsp[q].data();
      imag = std::max(imag, push_box<T>(b.n[0], b.n[1], b.n[2], h, b.p, dt, c, eps0, form, nodal, fp,
                                        form != kVacuum ? jp : nullptr, form == kRho ? r[0].data() : nullptr,
                                        pml ? dp : nullptr));
      if (pml) pml_damp<T>(L, i, pml, dt, fp, dp, split, offs[i]);
      for (int s = 0; s < 6; ++s)
        for (int64_t q = 0; q < N; ++q) fields[s][offs[i] + q] = (double)f[s][q];
      if (form == kRho)
        for (int64_t q = 0; q < N; ++q) src[3][offs[i] + q] = (double)r[0][q];
    }
    if (!mask && guards) {
      for (int s = 0; s < 6; ++s)
        if (int e = exchange(L, fields[s])) return e;
      if (form == kRho)
        if (int e = exchange(L, src[3])) return e;
    }
  }
  if (max_imag) *max_imag = imag;
  return 0;
}

}  // namespace

extern "C" {

// Guard exchange of one component buffer (boxes concatenated in layout
// order, each x fastest), in place.  Returns 2 when the interiors do not tile
// the global domain.
int oracle_exchange(const oracle_layout* L, double* data) {
  if (!L || !data) return 1;
  return exchange(L, data);
}

// Dual-grid coupling (paper Sec. 2.5.2): every cell of every destination box
// takes the value of the source layout's interior cell with the same global
// index.  Returns 2 when the source interiors do not tile the domain, 3 when
// the layouts describe different domains.
int oracle_couple(const oracle_layout* src, const double* src_data, const oracle_layout* dst, double* dst_data) {
  if (!src || !dst || !src_data || !dst_data) return 1;
  for (int d = 0; d < 3; ++d)
    if (src->global_n[d] != dst->global_n[d] || src->periodic[d] != dst->periodic[d]) return 3;
  std::vector<double> G;
  if (!assemble(src, src_data, G)) return 2;
  sample(dst, G, dst_data);
  return 0;
}

// nsteps steps of the push over a layout, in place.  fields: 6 component
// buffers (E_x..B_z); src: J_x, J_y, J_z, rho (NULL for vacuum; rho in/out
// for form 2).  mask: NULL = every box, then the exchange after each step;
// else only the boxes with mask[i] != 0 advance and no exchange runs.
// form: 0 vacuum, 1 J form, 2 rho form.  precision: 64 (the oracle) or 32
// (the FP32 rounding model).  *max_imag (may be NULL): largest imaginary part
// met in an inverse transform.
//
// pml (may be NULL): absorbing layers; then split holds the 6 stored split
// parts (E_xy, E_yz, E_zx, B_xy, B_yz, B_zx; same layout as the fields,
// interior cells in/out) and the form must be vacuum on a global, local or
// hybrid layout (the layers sit on the faces of the global domain).
int oracle_push(const oracle_layout* L, double* const* fields, double* const* src, const uint8_t* mask,
                int nsteps, const double* h, double dt, double c, double eps0, int form, int nodal,
                int precision, double* max_imag, const oracle_pml* pml, double* const* split) {
  if (!L || !fields || !h || nsteps < 0 || form < 0 || form > 2) return 1;
  if (form != kVacuum && (!src || !src[0] || !src[1] || !src[2])) return 1;
  if (form == kRho && !src[3]) return 1;
  if (pml && (!split || form != kVacuum || L->kind == 3 || nodal || pml->order < 0)) return 1;
  if (precision == 64)
    return push_layout<double>(L, fields, src, mask, nsteps, h, dt, c, eps0, form, nodal != 0, max_imag, pml,
                               split);
  if (precision == 32)
    return push_layout<float>(L, fields, src, mask, nsteps, h, dt, c, eps0, form, nodal != 0, max_imag, pml,
                              split);
  return 1;
}

}  // extern "C"
