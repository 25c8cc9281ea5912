// Complex helpers and small-DFT codelets held entirely in registers.
//
// Dft<T, R, DIR>::run(v) replaces v[0..R) by y_k = sum_t v_t exp(DIR 2 pi i t k / R)
// (DIR = -1 forward, +1 inverse, unnormalised).  R in {2,3,4,5,8} are written
// out; the other sizes are composed from two smaller codelets: coprime
// factors by the prime-factor mapping (no twiddles), powers of two by
// decimation in time (R = A*B) with internal twiddles exp(DIR 2 pi i m / R)
// as compile-time constants (unit_roots.h).
#pragma once

#include <cuda_runtime.h>

#include <type_traits>

#include "unit_roots.h"

namespace psatd {

template <typename T>
using cx = typename std::conditional<sizeof(T) == 4, float2, double2>::type;

template <typename T>
__device__ __forceinline__ cx<T> mk(T a, T b) {
  cx<T> r;
  r.x = a;
  r.y = b;
  return r;
}
// FP32 complex sums use the packed two-lane adds of sm_100+ (one instruction
// per complex add; each lane rounds exactly as a scalar add.rn.f32)
__device__ __forceinline__ float2 operator+(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 operator-(float2 a, float2 b) {
  unsigned long long r;
  asm("sub.rn.f32x2 %0, %1, %2;"
      : "=l"(r)
      : "l"(*reinterpret_cast<const unsigned long long*>(&a)), "l"(*reinterpret_cast<const unsigned long long*>(&b)));
  return *reinterpret_cast<const float2*>(&r);
}
// lane-wise product and negation of two-lane FP32 values (the packed update
// keeps the same real quantity of two modes in one float2)
__device__ __forceinline__ float2 operator*(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ float2 operator-(float2 a) { return make_float2(-a.x, -a.y); }
__device__ __forceinline__ double2 operator+(double2 a, double2 b) { return make_double2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ double2 operator-(double2 a, double2 b) { return make_double2(a.x - b.x, a.y - b.y); }

template <typename C>
__device__ __forceinline__ C cmul(C a, C b) {
  C r;
  r.x = a.x * b.x - a.y * b.y;
  r.y = a.x * b.y + a.y * b.x;
  return r;
}
template <typename C>
__device__ __forceinline__ C cmulc(C a, C b) {  // a * conj(b)
  C r;
  r.x = a.x * b.x + a.y * b.y;
  r.y = a.y * b.x - a.x * b.y;
  return r;
}
template <typename C, typename T>
__device__ __forceinline__ C rmul(T s, C a) {
  C r;
  r.x = s * a.x;
  r.y = s * a.y;
  return r;
}
template <typename C>
__device__ __forceinline__ C conjg(C a) {
  a.y = -a.y;
  return a;
}
template <typename C>
__device__ __forceinline__ C times_i(C a) {  // i * a
  C r;
  r.x = -a.y;
  r.y = a.x;
  return r;
}
// multiply by exp(DIR * i pi/2): DIR = -1 -> -i (forward), +1 -> +i (inverse)
template <int DIR, typename C>
__device__ __forceinline__ C rot(C a) {
  C r;
  if (DIR < 0) {
    r.x = a.y;
    r.y = -a.x;
  } else {
    r.x = -a.y;
    r.y = a.x;
  }
  return r;
}
// a * w (forward, w = exp(-i phi) from the table) or a * conj(w) (inverse)
template <int DIR, typename C>
__device__ __forceinline__ C twmul(C a, C w) {
  return DIR < 0 ? cmul(a, w) : cmulc(a, w);
}

// Compile-time loop: f(std::integral_constant<int, I>) for I in [B, E).
template <int B, int E, typename F>
__device__ __forceinline__ void static_for(F&& f) {
  if constexpr (B < E) {
    f(std::integral_constant<int, B>{});
    static_for<B + 1, E>(f);
  }
}

template <typename T, int R, int DIR>
struct Dft;

template <typename T, int DIR>
struct Dft<T, 1, DIR> {
  static __device__ __forceinline__ void run(cx<T>*) {}
};

template <typename T, int DIR>
struct Dft<T, 2, DIR> {
  static __device__ __forceinline__ void run(cx<T>* v) {
    cx<T> a = v[0], b = v[1];
    v[0] = a + b;
    v[1] = a - b;
  }
};

// FP32 products with FP64-accurate constants.  A constant rounded to FP32
// carries a relative error of up to 3e-8 into every product, the same on
// every call: an FFT and its inverse built on such roots of unity scale a mode
// by |w|^2 != 1 per round trip (the FP32 roots of the small DFTs and of the
// composite twiddles lie slightly inside the unit circle), and over the
// hundreds of steps of a push that bias adds up linearly: an FP32 push lost
// ~1e-7 of its amplitude per step.  So in FP32 a constant c = hi + lo (hi its
// FP32 rounding, lo the FP32 rounding of the rest) multiplies as
// fma(hi, a, lo * a): the exact product hi * a and the small lo * a are added
// before the one rounding, which gives the correctly rounded c * a up to the
// rounding of lo * a (adding lo * a after rounding hi * a would lose it: it is
// below half a unit in the last place).  FP64 uses the plain products.
__host__ __device__ constexpr float f32_hi(double v) { return (float)v; }
__host__ __device__ constexpr float f32_lo(double v) { return (float)(v - (double)(float)v); }

// s * x for a real constant s (FP32: head and tail)
template <typename T>
__device__ __forceinline__ T mul_exact(double s, T x) {
  if constexpr (sizeof(T) == 4)
    return __fmaf_rn(f32_hi(s), x, f32_lo(s) * x);
  else
    return T(s) * x;
}
template <typename T, typename C>
__device__ __forceinline__ C rmul_exact(double s, C a) {
  return mk<T>(mul_exact<T>(s, a.x), mul_exact<T>(s, a.y));
}
// a * (c + i s) for FP32 head/tail constants (ch, cl), (sh, sl): the tail
// products first, then the head products, one rounding per fused step
__device__ __forceinline__ float2 cmul_hl(float2 a, float ch, float cl, float sh, float sl) {
  const float re = __fmaf_rn(a.x, ch, __fmaf_rn(-a.y, sh, __fmaf_rn(a.x, cl, -a.y * sl)));
  const float im = __fmaf_rn(a.y, ch, __fmaf_rn(a.x, sh, __fmaf_rn(a.y, cl, a.x * sl)));
  return make_float2(re, im);
}

template <typename T, int DIR>
struct Dft<T, 3, DIR> {
  static __device__ __forceinline__ void run(cx<T>* v) {
    cx<T> s = v[1] + v[2], d = v[1] - v[2];
    cx<T> m = mk<T>(v[0].x - T(0.5) * s.x, v[0].y - T(0.5) * s.y);
    cx<T> r = rmul_exact<T>(0.86602540378443864676, rot<DIR>(d));   // sin(2 pi / 3), FP32 head + tail
    v[0] = v[0] + s;
    v[1] = m + r;
    v[2] = m - r;
  }
};

template <typename T, int DIR>
struct Dft<T, 4, DIR> {
  static __device__ __forceinline__ void run(cx<T>* v) {
    cx<T> t0 = v[0] + v[2], t1 = v[0] - v[2];
    cx<T> t2 = v[1] + v[3], t3 = rot<DIR>(v[1] - v[3]);
    v[0] = t0 + t2;
    v[2] = t0 - t2;
    v[1] = t1 + t3;
    v[3] = t1 - t3;
  }
};

template <typename T, int DIR>
struct Dft<T, 5, DIR> {
  static __device__ __forceinline__ void run(cx<T>* v) {
    constexpr double c1 = 0.30901699437494742410;   // cos(2 pi/5)
    constexpr double c2 = -0.80901699437494742410;  // cos(4 pi/5)
    constexpr double s1 = 0.95105651629515357212;   // sin(2 pi/5)
    constexpr double s2 = 0.58778525229247312917;   // sin(4 pi/5)
    cx<T> a0 = v[0];
    cx<T> p1 = v[1] + v[4], d1 = v[1] - v[4];
    cx<T> p2 = v[2] + v[3], d2 = v[2] - v[3];
    // u x + v y (+ w): the constants' tails first, then their heads (FP32)
    auto dot2 = [](double u, T x, double v, T y, T w) -> T {
      if constexpr (sizeof(T) == 4)
        return __fmaf_rn(f32_hi(u), x, __fmaf_rn(f32_hi(v), y, __fmaf_rn(f32_lo(u), x, __fmaf_rn(f32_lo(v), y, w))));
      else
        return w + u * x + v * y;
    };
    cx<T> m1 = mk<T>(dot2(c1, p1.x, c2, p2.x, a0.x), dot2(c1, p1.y, c2, p2.y, a0.y));
    cx<T> m2 = mk<T>(dot2(c2, p1.x, c1, p2.x, a0.x), dot2(c2, p1.y, c1, p2.y, a0.y));
    cx<T> n1 = mk<T>(dot2(s1, d1.x, s2, d2.x, T(0)), dot2(s1, d1.y, s2, d2.y, T(0)));
    cx<T> n2 = mk<T>(dot2(s2, d1.x, -s1, d2.x, T(0)), dot2(s2, d1.y, -s1, d2.y, T(0)));
    cx<T> r1 = rot<DIR>(n1), r2 = rot<DIR>(n2);
    v[0] = a0 + p1 + p2;
    v[1] = m1 + r1;
    v[4] = m1 - r1;
    v[2] = m2 + r2;
    v[3] = m2 - r2;
  }
};

template <typename T, int DIR>
struct Dft<T, 8, DIR> {
  static __device__ __forceinline__ void run(cx<T>* v) {
    constexpr double r2 = 0.70710678118654752440;   // cos(pi/4), split in FP32 (rmul_exact)
    cx<T> e[4] = {v[0], v[2], v[4], v[6]};
    cx<T> o[4] = {v[1], v[3], v[5], v[7]};
    Dft<T, 4, DIR>::run(e);
    Dft<T, 4, DIR>::run(o);
    // o[k] *= exp(DIR i pi k / 4)
    cx<T> w1, w3;
    if (DIR < 0) {
      w1 = rmul_exact<T>(r2, mk<T>(o[1].x + o[1].y, o[1].y - o[1].x));
      w3 = rmul_exact<T>(r2, mk<T>(o[3].y - o[3].x, -(o[3].x + o[3].y)));
    } else {
      w1 = rmul_exact<T>(r2, mk<T>(o[1].x - o[1].y, o[1].x + o[1].y));
      w3 = rmul_exact<T>(r2, mk<T>(-(o[3].x + o[3].y), o[3].x - o[3].y));
    }
    cx<T> w2 = rot<DIR>(o[2]);
    v[0] = e[0] + o[0];
    v[4] = e[0] - o[0];
    v[1] = e[1] + w1;
    v[5] = e[1] - w1;
    v[2] = e[2] + w2;
    v[6] = e[2] - w2;
    v[3] = e[3] + w3;
    v[7] = e[3] - w3;
  }
};

// R = A * B by decimation in time: n = B n1 + n2, k = k1 + A k2,
// X[k1 + A k2] = sum_n2 w_B^{n2 k2} w_R^{n2 k1} sum_n1 x[B n1 + n2] w_A^{n1 k1}.
template <typename T, int A, int B, int DIR>
struct DftComposite {
  static __device__ __forceinline__ void run(cx<T>* v) {
    constexpr int R = A * B;
    cx<T> u[B][A];
    static_for<0, B>([&](auto n2c) {
      constexpr int n2 = decltype(n2c)::value;
#pragma unroll
      for (int n1 = 0; n1 < A; ++n1) u[n2][n1] = v[B * n1 + n2];
      Dft<T, A, DIR>::run(u[n2]);
      static_for<1, A>([&](auto k1c) {
        constexpr int k1 = decltype(k1c)::value;
        (void)k1;
        if constexpr (n2 > 0) {
          constexpr double c = root_cos(R, n2 * k1);
          constexpr double s = root_sin(R, n2 * k1);
          constexpr double sd = DIR < 0 ? -s : s;
          const cx<T> a = u[n2][k1];
          if constexpr (c == 0.0) {
            // w = +-i
            u[n2][k1] = sd > 0 ? mk<T>(-a.y, a.x) : mk<T>(a.y, -a.x);
          } else if constexpr (c == sd || c == -sd) {
            // w = c (1 + i sd/c): |c| = sqrt(1/2), one head + tail product per lane
            u[n2][k1] = c == sd ? rmul_exact<T>(c, mk<T>(a.x - a.y, a.x + a.y))
                                : rmul_exact<T>(c, mk<T>(a.x + a.y, a.y - a.x));
          } else if constexpr (sizeof(T) == 4) {
            u[n2][k1] = cmul_hl(a, f32_hi(c), f32_lo(c), f32_hi(sd), f32_lo(sd));
          } else {
            u[n2][k1] = cmul(a, mk<T>(T(c), T(sd)));
          }
        }
      });
    });
#pragma unroll
    for (int k1 = 0; k1 < A; ++k1) {
      cx<T> w[B];
#pragma unroll
      for (int n2 = 0; n2 < B; ++n2) w[n2] = u[n2][k1];
      Dft<T, B, DIR>::run(w);
#pragma unroll
      for (int k2 = 0; k2 < B; ++k2) v[k1 + A * k2] = w[k2];
    }
  }
};

// R = A * B with A, B coprime by the prime-factor (Good-Thomas) mapping: with
// input index n = (B n1 + A n2) mod R and output index
// k = (B tB k1 + A tA k2) mod R, tB = B^-1 mod A, tA = A^-1 mod B, the R-point
// DFT is exactly the two-dimensional A x B DFT of the re-indexed input, with
// no twiddle factors (the index maps are compile-time register renamings).
constexpr int inv_mod(int a, int m) {
  int r = 1;
  while ((a * r) % m != 1 % m) ++r;
  return r;
}
constexpr int gcd_int(int a, int b) { return b == 0 ? a : gcd_int(b, a % b); }

template <typename T, int A, int B, int DIR>
struct DftPfa {
  static_assert(gcd_int(A, B) == 1, "prime-factor lengths must be coprime");
  static __device__ __forceinline__ void run(cx<T>* v) {
    constexpr int R = A * B, TB = inv_mod(B % A, A), TA = inv_mod(A % B, B);
    cx<T> u[B][A];
#pragma unroll
    for (int n2 = 0; n2 < B; ++n2) {
#pragma unroll
      for (int n1 = 0; n1 < A; ++n1) u[n2][n1] = v[(B * n1 + A * n2) % R];
      Dft<T, A, DIR>::run(u[n2]);
    }
#pragma unroll
    for (int k1 = 0; k1 < A; ++k1) {
      cx<T> w[B];
#pragma unroll
      for (int n2 = 0; n2 < B; ++n2) w[n2] = u[n2][k1];
      Dft<T, B, DIR>::run(w);
#pragma unroll
      for (int k2 = 0; k2 < B; ++k2) v[(B * TB * k1 + A * TA * k2) % R] = w[k2];
    }
  }
};

template <typename T, int DIR>
struct Dft<T, 6, DIR> : DftPfa<T, 3, 2, DIR> {};
template <typename T, int DIR>
struct Dft<T, 10, DIR> : DftPfa<T, 5, 2, DIR> {};
template <typename T, int DIR>
struct Dft<T, 12, DIR> : DftPfa<T, 4, 3, DIR> {};
template <typename T, int DIR>
struct Dft<T, 16, DIR> : DftComposite<T, 4, 4, DIR> {};
// register-resident lengths of the one-thread-per-line kernels
template <typename T, int DIR>
struct Dft<T, 24, DIR> : DftPfa<T, 8, 3, DIR> {};
template <typename T, int DIR>
struct Dft<T, 30, DIR> : DftPfa<T, 10, 3, DIR> {};
template <typename T, int DIR>
struct Dft<T, 32, DIR> : DftComposite<T, 8, 4, DIR> {};
template <typename T, int DIR>
struct Dft<T, 40, DIR> : DftPfa<T, 8, 5, DIR> {};
template <typename T, int DIR>
struct Dft<T, 48, DIR> : DftPfa<T, 16, 3, DIR> {};
template <typename T, int DIR>
struct Dft<T, 60, DIR> : DftPfa<T, 12, 5, DIR> {};

}  // namespace psatd
