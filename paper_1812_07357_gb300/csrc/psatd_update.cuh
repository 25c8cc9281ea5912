// S2: the per-mode PSATD update shared by the generic and the fast kernels.
//
// Centred spectra (each component shifted by exp(-i k.s h) from its Yee
// offset s), theta = c |K| dt and the coefficient quad (C, Sw, X1, X3) of the
// mode (C = cos theta, Sw = sin theta/(c K), X1 = (1 - C)/K^2,
// X3 = (Sw - dt)/K^2, generated in FP64 at plan time):
//   J form:   E' = C E + X1 K(K.E) + i c^2 Sw K x B - Sw J/eps0 + X3 K(K.J)/eps0
//   rho form: rho' = rho - i dt K.J,
//             E' = C E + i c^2 Sw K x B - Sw J/eps0 + i K (Y1 rho' + Y2 rho)/eps0,
//             Y1 = X3/dt, Y2 = -X1 - X3/dt
//   both:     B' = C B + X1 K(K.B) - i Sw K x E + i (X1/c^2) K x J/eps0
// (the exact solution of Maxwell's equations for one mode over dt with J
// constant over the step; paper Sec. 1.1 states the principle).
#pragma once

#include <type_traits>

#include "fft_codelets.cuh"
#include "psatd_internal.h"

namespace psatd {

template <typename T>
__device__ __forceinline__ const cx<T>* cpool(const DevPlan& P) {
  return reinterpret_cast<const cx<T>*>(P.cpool);
}
template <typename T>
__device__ __forceinline__ const T* rpool(const DevPlan& P) {
  return reinterpret_cast<const T*>(P.rpool);
}

// Quantities of a mode that depend on (mx, my) only: a thread that updates
// several z of one (mx, my) loads them once.
template <typename T>
struct ModeXY {
  T Kx, Ky;
  cx<T> px, py, pxy;
  int64_t qbase;   // coefficient index of (mx, |my|, mz = 0)
};

template <typename T>
__device__ __forceinline__ ModeXY<T> mode_xy(int mx, int my, const ShapeDev& sh, const DevPlan& P) {
  const T* rp = rpool<T>(P);
  const cx<T>* cp = cpool<T>(P);
  const int n1 = sh.n[1];
  const int myr = my <= n1 - my ? my : n1 - my;
  ModeXY<T> r;
  r.Kx = rp[sh.kx + mx];
  r.Ky = rp[sh.ky + my];
  r.px = cp[sh.phx + mx];
  r.py = cp[sh.phy + my];
  r.pxy = cmul(r.px, r.py);
  r.qbase = sh.coef + (int64_t)myr * sh.hx + mx;
  return r;
}

// ---- value types of the update ---------------------------------------------
// The arithmetic below is written once for a real type T and a complex type C:
// (float, float2) and (double, double2) update one mode; (float2, C2) update
// two modes at once, lane 0 and lane 1 of every packed register holding the
// same quantity of mode A and mode B (two-lane FP32 instructions of sm_100+,
// each lane rounded like the scalar instruction).
struct C2 {
  float2 x, y;   // real parts (A, B), imaginary parts (A, B)
};
__device__ __forceinline__ C2 operator+(C2 a, C2 b) { return C2{a.x + b.x, a.y + b.y}; }
__device__ __forceinline__ C2 operator-(C2 a, C2 b) { return C2{a.x - b.x, a.y - b.y}; }
__device__ __forceinline__ C2 cmul(C2 a, C2 b) {
  return C2{__ffma2_rn(a.x, b.x, -(a.y * b.y)), __ffma2_rn(a.x, b.y, a.y * b.x)};
}
__device__ __forceinline__ C2 cmulc(C2 a, C2 b) {   // a * conj(b)
  return C2{__ffma2_rn(a.x, b.x, a.y * b.y), __ffma2_rn(a.y, b.x, -(a.x * b.y))};
}

template <typename T>
__device__ __forceinline__ T bcast(double v) {
  if constexpr (std::is_same<T, float2>::value)
    return make_float2((float)v, (float)v);
  else
    return T(v);
}

// The update of one mode (or of two, with the packed types) in centred form;
// m[0..FIN) holds the field slots of the mode (see Form) in the sampled
// (uncentred) representation and receives E', B' (and rho').
template <typename T, typename C, int FORM>
__device__ __forceinline__ void update_core(C* m, T Kx, T Ky, T Kz, C px, C py, C pz, C pxy, const Coef4<T>& q,
                                            const DevPlan& P) {
  const C pyz = cmul(py, pz), pxz = cmul(px, pz);
  // centred spectra: F~ = exp(-i k.s h) F^
  const C ex = cmulc(m[0], px), ey = cmulc(m[1], py), ez = cmulc(m[2], pz);
  const C bx = cmulc(m[3], pyz), by = cmulc(m[4], pxz), bz = cmulc(m[5], pxy);
  const T cc = bcast<T>(P.cc);
  const T ieps = bcast<T>(P.ieps);
  // K x B, K x E, K.B
  const C kbx = rmul(Ky, bz) - rmul(Kz, by);
  const C kby = rmul(Kz, bx) - rmul(Kx, bz);
  const C kbz = rmul(Kx, by) - rmul(Ky, bx);
  const C kex = rmul(Ky, ez) - rmul(Kz, ey);
  const C key = rmul(Kz, ex) - rmul(Kx, ez);
  const C kez = rmul(Kx, ey) - rmul(Ky, ex);
  const C kdb = rmul(Kx, bx) + rmul(Ky, by) + rmul(Kz, bz);
  const T csw = cc * q.s;
  // B' = C B + X1 K (K.B) - i Sw K x E (+ i X1/c^2 K x J / eps0)
  C nbx = rmul(q.c, bx) + rmul(q.x1 * Kx, kdb) - rmul(q.s, times_i(kex));
  C nby = rmul(q.c, by) + rmul(q.x1 * Ky, kdb) - rmul(q.s, times_i(key));
  C nbz = rmul(q.c, bz) + rmul(q.x1 * Kz, kdb) - rmul(q.s, times_i(kez));
  C nex, ney, nez;
  if (FORM == kRhoForm) {
    const C rho = m[6];
    const C jx = cmulc(m[7], px), jy = cmulc(m[8], py), jz = cmulc(m[9], pz);
    const C kdj = rmul(Kx, jx) + rmul(Ky, jy) + rmul(Kz, jz);
    const T dt = bcast<T>(P.dt);
    const C rhon = rho - rmul(dt, times_i(kdj));
    const T y1 = q.x3 * bcast<T>(P.idt);
    const T y2 = -q.x1 - y1;
    const C g = times_i(rmul(y1, rhon) + rmul(y2, rho));  // i (Y1 rho' + Y2 rho)
    nex = rmul(q.c, ex) + rmul(csw, times_i(kbx)) - rmul(q.s * ieps, jx) + rmul(Kx * ieps, g);
    ney = rmul(q.c, ey) + rmul(csw, times_i(kby)) - rmul(q.s * ieps, jy) + rmul(Ky * ieps, g);
    nez = rmul(q.c, ez) + rmul(csw, times_i(kbz)) - rmul(q.s * ieps, jz) + rmul(Kz * ieps, g);
    const T x2 = q.x1 * bcast<T>(P.icce);
    nbx = nbx + rmul(x2, times_i(rmul(Ky, jz) - rmul(Kz, jy)));
    nby = nby + rmul(x2, times_i(rmul(Kz, jx) - rmul(Kx, jz)));
    nbz = nbz + rmul(x2, times_i(rmul(Kx, jy) - rmul(Ky, jx)));
    m[6] = rhon;
  } else {
    const C kde = rmul(Kx, ex) + rmul(Ky, ey) + rmul(Kz, ez);
    nex = rmul(q.c, ex) + rmul(q.x1 * Kx, kde) + rmul(csw, times_i(kbx));
    ney = rmul(q.c, ey) + rmul(q.x1 * Ky, kde) + rmul(csw, times_i(kby));
    nez = rmul(q.c, ez) + rmul(q.x1 * Kz, kde) + rmul(csw, times_i(kbz));
    if (FORM == kJForm) {
      const C jx = cmulc(m[6], px), jy = cmulc(m[7], py), jz = cmulc(m[8], pz);
      const C kdj = rmul(Kx, jx) + rmul(Ky, jy) + rmul(Kz, jz);
      const T a = q.s * ieps, b = q.x3 * ieps;
      nex = nex - rmul(a, jx) + rmul(b * Kx, kdj);
      ney = ney - rmul(a, jy) + rmul(b * Ky, kdj);
      nez = nez - rmul(a, jz) + rmul(b * Kz, kdj);
      const T x2 = q.x1 * bcast<T>(P.icce);
      nbx = nbx + rmul(x2, times_i(rmul(Ky, jz) - rmul(Kz, jy)));
      nby = nby + rmul(x2, times_i(rmul(Kz, jx) - rmul(Kx, jz)));
      nbz = nbz + rmul(x2, times_i(rmul(Kx, jy) - rmul(Ky, jx)));
    }
  }
  if constexpr (FORM == kPml) {
    // increments of the stored split parts over the step (absorbing layers):
    // the time integrals of the mode solution,
    //   I[E] = Sw E - X3 K (K.E) + i X1 K x B,
    //   I[B] = Sw B - X3 K (K.B) - i (X1/c^2) K x E,
    // give dE_xy = i c^2 K_y I[B_z], dE_yz = i c^2 K_z I[B_x], dE_zx = i c^2 K_x I[B_y],
    //      dB_xy = -i K_y I[E_z],    dB_yz = -i K_z I[E_x],    dB_zx = -i K_x I[E_y]
    const C kde = rmul(Kx, ex) + rmul(Ky, ey) + rmul(Kz, ez);
    const T x1c = q.x1 * bcast<T>(P.icce * P.eps0);
    const C iex = rmul(q.s, ex) - rmul(q.x3 * Kx, kde) + rmul(q.x1, times_i(kbx));
    const C iey = rmul(q.s, ey) - rmul(q.x3 * Ky, kde) + rmul(q.x1, times_i(kby));
    const C iez = rmul(q.s, ez) - rmul(q.x3 * Kz, kde) + rmul(q.x1, times_i(kbz));
    const C ibx = rmul(q.s, bx) - rmul(q.x3 * Kx, kdb) - rmul(x1c, times_i(kex));
    const C iby = rmul(q.s, by) - rmul(q.x3 * Ky, kdb) - rmul(x1c, times_i(key));
    const C ibz = rmul(q.s, bz) - rmul(q.x3 * Kz, kdb) - rmul(x1c, times_i(kez));
    m[6] = cmul(rmul(cc * Ky, times_i(ibz)), px);
    m[7] = cmul(rmul(cc * Kz, times_i(ibx)), py);
    m[8] = cmul(rmul(cc * Kx, times_i(iby)), pz);
    m[9] = cmul(rmul(-Ky, times_i(iez)), pyz);
    m[10] = cmul(rmul(-Kz, times_i(iex)), pxz);
    m[11] = cmul(rmul(-Kx, times_i(iey)), pxy);
  }
  // back to the staggered sample positions: F^ = exp(+i k.s h) F~
  m[0] = cmul(nex, px);
  m[1] = cmul(ney, py);
  m[2] = cmul(nez, pz);
  m[3] = cmul(nbx, pyz);
  m[4] = cmul(nby, pxz);
  m[5] = cmul(nbz, pxy);
}

// One mode (mx, my, mz): md[f * fs] is field slot f.
template <typename T, int FORM>
__device__ __forceinline__ void update_mode_z(cx<T>* md, int fs, const ModeXY<T>& m, int mz, const ShapeDev& sh,
                                              const DevPlan& P) {
  using C = cx<T>;
  const int n1 = sh.n[1], n2 = sh.n[2];
  const T Kz = rpool<T>(P)[sh.kz + mz];
  const C pz = cpool<T>(P)[sh.phz + mz];
  const int mzr = mz <= n2 - mz ? mz : n2 - mz;
  const Coef4<T> q =
      reinterpret_cast<const Coef4<T>*>(P.coef)[m.qbase + (int64_t)mzr * (n1 / 2 + 1) * sh.hx];
  C v[spec_slots(FORM)];
#pragma unroll
  for (int f = 0; f < fields_in(FORM); ++f) v[f] = md[f * fs];
  update_core<T, C, FORM>(v, m.Kx, m.Ky, Kz, m.px, m.py, pz, m.pxy, q, P);
#pragma unroll
  for (int f = 0; f < fields_out(FORM); ++f) md[f * fs] = v[f];
}

// ---- two modes per thread (FP32) --------------------------------------------
// Modes A and B share mz and are adjacent in shared memory (columns t, t + 1
// of a z tile): A = (mxA, myA), B = (mxB, myB).
struct ModeXY2 {
  float2 Kx, Ky;
  C2 px, py, pxy;
  int64_t qa, qb;   // coefficient indices of A and B at mz = 0
};

__device__ __forceinline__ C2 pack2(float2 a, float2 b) { return C2{make_float2(a.x, b.x), make_float2(a.y, b.y)}; }

__device__ __forceinline__ ModeXY2 mode_xy2(int mxa, int mya, int mxb, int myb, const ShapeDev& sh,
                                            const DevPlan& P) {
  const ModeXY<float> a = mode_xy<float>(mxa, mya, sh, P), b = mode_xy<float>(mxb, myb, sh, P);
  ModeXY2 r;
  r.Kx = make_float2(a.Kx, b.Kx);
  r.Ky = make_float2(a.Ky, b.Ky);
  r.px = pack2(a.px, b.px);
  r.py = pack2(a.py, b.py);
  r.pxy = pack2(a.pxy, b.pxy);
  r.qa = a.qbase;
  r.qb = b.qbase;
  return r;
}

// Per-z quantities of modes A and B at mz: K_z, the Yee phase and the
// coefficient quads.
struct ModeZ2 {
  float kz;
  float2 pz;
  Coef4<float2> q;
};

__device__ __forceinline__ ModeZ2 mode_z2(const ModeXY2& m, int mz, const ShapeDev& sh, const DevPlan& P) {
  const int n1 = sh.n[1], n2 = sh.n[2];
  ModeZ2 r;
  r.kz = rpool<float>(P)[sh.kz + mz];
  r.pz = cpool<float>(P)[sh.phz + mz];
  const int mzr = mz <= n2 - mz ? mz : n2 - mz;
  const int64_t zoff = (int64_t)mzr * (n1 / 2 + 1) * sh.hx;
  const float4 qa = reinterpret_cast<const float4*>(P.coef)[m.qa + zoff];
  const float4 qb = reinterpret_cast<const float4*>(P.coef)[m.qb + zoff];
  r.q.c = make_float2(qa.x, qb.x);
  r.q.s = make_float2(qa.y, qb.y);
  r.q.x1 = make_float2(qa.z, qb.z);
  r.q.x3 = make_float2(qa.w, qb.w);
  return r;
}

// A and B of one slot as the 16 bytes at md: (re A, re B, im A, im B) in the
// "re-first" order, (im A, im B, re A, re B) in the "im-first" order, so that
// both two-lane halves are register pairs as loaded.
template <bool IM_FIRST>
__device__ __forceinline__ C2 load2(const float2* md) {
  const float4 w = *reinterpret_cast<const float4*>(md);
  return IM_FIRST ? C2{make_float2(w.z, w.w), make_float2(w.x, w.y)} : C2{make_float2(w.x, w.y), make_float2(w.z, w.w)};
}
template <bool IM_FIRST>
__device__ __forceinline__ void store2(float2* md, C2 v) {
  *reinterpret_cast<float4*>(md) =
      IM_FIRST ? make_float4(v.y.x, v.y.y, v.x.x, v.x.y) : make_float4(v.x.x, v.x.y, v.y.x, v.y.y);
}

// ---- the packed update, written instruction by instruction -----------------
// The same update as update_core for (float2, C2), with every real operation
// a two-lane FMUL / FFMA of sm_100+ and the negated operands formed once per
// mode pair (a subtraction a - b c is fma(-b, c, a)), so that no lane shuffles
// or per-use negations are needed.
__device__ __forceinline__ float2 mul2(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ float2 fma2(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }
__device__ __forceinline__ float2 neg2(float2 a) { return __fmul2_rn(a, make_float2(-1.f, -1.f)); }

// m conj(p) and n p for a phase p with npy = -p.y
__device__ __forceinline__ C2 cmulc_n(C2 m, C2 p, float2 npy) {
  return C2{fma2(m.y, p.y, mul2(m.x, p.x)), fma2(m.x, npy, mul2(m.y, p.x))};
}
__device__ __forceinline__ C2 cmul_n(C2 n, C2 p, float2 npy) {
  return C2{fma2(n.y, npy, mul2(n.x, p.x)), fma2(n.x, p.y, mul2(n.y, p.x))};
}
// a u - b v for real a, b given as (a, -b)
__device__ __forceinline__ C2 cross1(float2 a, C2 u, float2 nb, C2 v) {
  return C2{fma2(nb, v.x, mul2(a, u.x)), fma2(nb, v.y, mul2(a, u.y))};
}
__device__ __forceinline__ C2 dot3(float2 kx, C2 x, float2 ky, C2 y, float2 kz, C2 z) {
  return C2{fma2(kz, z.x, fma2(ky, y.x, mul2(kx, x.x))), fma2(kz, z.y, fma2(ky, y.y, mul2(kx, x.y)))};
}

template <int FORM>
__device__ __forceinline__ void update_core2(C2* m, float2 Kx, float2 Ky, float2 Kz, C2 px, C2 py, C2 pz, C2 pxy,
                                             const Coef4<float2>& q, const DevPlan& P) {
  const float2 npx = neg2(px.y), npy = neg2(py.y), npz = neg2(pz.y), npxy = neg2(pxy.y);
  const C2 pyz = cmul_n(py, pz, npz), pxz = cmul_n(px, pz, npz);
  const float2 npyz = neg2(pyz.y), npxz = neg2(pxz.y);
  const float2 nKx = neg2(Kx), nKy = neg2(Ky), nKz = neg2(Kz);
  // centred spectra
  const C2 ex = cmulc_n(m[0], px, npx), ey = cmulc_n(m[1], py, npy), ez = cmulc_n(m[2], pz, npz);
  const C2 bx = cmulc_n(m[3], pyz, npyz), by = cmulc_n(m[4], pxz, npxz), bz = cmulc_n(m[5], pxy, npxy);
  const float2 cc = bcast<float2>(P.cc);
  // K x B, K x E, K.B
  const C2 kbx = cross1(Ky, bz, nKz, by), kby = cross1(Kz, bx, nKx, bz), kbz = cross1(Kx, by, nKy, bx);
  const C2 kex = cross1(Ky, ez, nKz, ey), key = cross1(Kz, ex, nKx, ez), kez = cross1(Kx, ey, nKy, ex);
  const C2 kdb = dot3(Kx, bx, Ky, by, Kz, bz);
  const float2 x1x = mul2(q.x1, Kx), x1y = mul2(q.x1, Ky), x1z = mul2(q.x1, Kz);
  const float2 S = q.s, nS = neg2(q.s), csw = mul2(cc, q.s), ncsw = neg2(csw), C = q.c;
  // B' = C B + X1 K (K.B) - i Sw K x E      (-i S (u + i v) = S v - i S u)
  auto bnew = [&](C2 b, float2 x1k, C2 ke) {
    return C2{fma2(S, ke.y, fma2(x1k, kdb.x, mul2(C, b.x))), fma2(nS, ke.x, fma2(x1k, kdb.y, mul2(C, b.y)))};
  };
  C2 nbx = bnew(bx, x1x, kex), nby = bnew(by, x1y, key), nbz = bnew(bz, x1z, kez);
  // + i csw K x B                            (i c (u + i v) = -c v + i c u)
  auto ecurl = [&](C2 e, C2 kb) { return C2{fma2(ncsw, kb.y, mul2(C, e.x)), fma2(csw, kb.x, mul2(C, e.y))}; };
  C2 nex = ecurl(ex, kbx), ney = ecurl(ey, kby), nez = ecurl(ez, kbz);
  if (FORM == kRhoForm || FORM == kJForm) {
    constexpr int J0 = FORM == kRhoForm ? 7 : 6;
    const C2 jx = cmulc_n(m[J0], px, npx), jy = cmulc_n(m[J0 + 1], py, npy), jz = cmulc_n(m[J0 + 2], pz, npz);
    const float2 ieps = bcast<float2>(P.ieps);
    const float2 na = neg2(mul2(q.s, ieps));                       // -Sw/eps0
    const C2 kdj = dot3(Kx, jx, Ky, jy, Kz, jz);
    // B' += i (X1/c^2) K x J / eps0
    const float2 x2 = mul2(q.x1, bcast<float2>(P.icce)), nx2 = neg2(x2);
    const C2 kjx = cross1(Ky, jz, nKz, jy), kjy = cross1(Kz, jx, nKx, jz), kjz = cross1(Kx, jy, nKy, jx);
    auto bj = [&](C2 b, C2 kj) { return C2{fma2(nx2, kj.y, b.x), fma2(x2, kj.x, b.y)}; };
    nbx = bj(nbx, kjx);
    nby = bj(nby, kjy);
    nbz = bj(nbz, kjz);
    if (FORM == kRhoForm) {
      // rho' = rho - i dt K.J ; E' += -Sw J/eps0 + i K (Y1 rho' + Y2 rho)/eps0
      const C2 rho = m[6];
      const float2 dt = bcast<float2>(P.dt), ndt = neg2(dt);
      const C2 rhon{fma2(dt, kdj.y, rho.x), fma2(ndt, kdj.x, rho.y)};
      const float2 y1 = mul2(q.x3, bcast<float2>(P.idt));
      const float2 y2 = neg2(q.x1 + y1);
      const C2 t{fma2(y2, rho.x, mul2(y1, rhon.x)), fma2(y2, rho.y, mul2(y1, rhon.y))};   // g = i t
      const float2 kix = mul2(Kx, ieps), kiy = mul2(Ky, ieps), kiz = mul2(Kz, ieps);
      auto er = [&](C2 e, C2 j, float2 ki) {
        return C2{fma2(neg2(ki), t.y, fma2(na, j.x, e.x)), fma2(ki, t.x, fma2(na, j.y, e.y))};
      };
      nex = er(nex, jx, kix);
      ney = er(ney, jy, kiy);
      nez = er(nez, jz, kiz);
      m[6] = rhon;
    } else {
      // E' += X1 K (K.E) - Sw J/eps0 + X3 K (K.J)/eps0
      const C2 kde = dot3(Kx, ex, Ky, ey, Kz, ez);
      const float2 b = mul2(q.x3, ieps);
      const float2 bkx = mul2(b, Kx), bky = mul2(b, Ky), bkz = mul2(b, Kz);
      auto ej = [&](C2 e, C2 j, float2 x1k, float2 bk) {
        return C2{fma2(bk, kdj.x, fma2(na, j.x, fma2(x1k, kde.x, e.x))),
                  fma2(bk, kdj.y, fma2(na, j.y, fma2(x1k, kde.y, e.y)))};
      };
      nex = ej(nex, jx, x1x, bkx);
      ney = ej(ney, jy, x1y, bky);
      nez = ej(nez, jz, x1z, bkz);
    }
  } else {
    // E' += X1 K (K.E)
    const C2 kde = dot3(Kx, ex, Ky, ey, Kz, ez);
    auto eg = [&](C2 e, float2 x1k) { return C2{fma2(x1k, kde.x, e.x), fma2(x1k, kde.y, e.y)}; };
    nex = eg(nex, x1x);
    ney = eg(ney, x1y);
    nez = eg(nez, x1z);
  }
  // back to the staggered sample positions
  m[0] = cmul_n(nex, px, npx);
  m[1] = cmul_n(ney, py, npy);
  m[2] = cmul_n(nez, pz, npz);
  m[3] = cmul_n(nbx, pyz, npyz);
  m[4] = cmul_n(nby, pxz, npxz);
  m[5] = cmul_n(nbz, pxy, npxy);
}

// Modes k and k + NZ/2 of columns A and B, with the last radix-2 stage of the
// forward z FFT before the update and the first stage of the inverse after
// it.  lo / hi: slot 0 of the rows k (re-first order) and NZ/2 + k (im-first
// order).  For slots f < nft those
// rows hold the half-length DFTs of the even and odd z samples, E[k] and
// O[k]; with w = exp(-2 pi i k / NZ) the modes are
//   X[k] = E[k] + w O[k],   X[k + NZ/2] = E[k] - w O[k],
// and after the update the rows receive the inputs of the half-length
// inverse DFTs of the even and odd z samples,
//   E'[k] = X'[k] + X'[k + NZ/2],   O'[k] = conj(w) (X'[k] - X'[k + NZ/2]).
// Slots f >= nft (a cached current spectrum) already hold X in natural z
// order, so rows k and NZ/2 + k are the two modes themselves.
template <int FORM, int NZ>
__device__ __forceinline__ void update_pair_z2(float2* lo, float2* hi, int fs, const ModeXY2& m, int k, float2 w,
                                               int nft, const ShapeDev& sh, const DevPlan& P) {
  constexpr int FIN = fields_in(FORM), FOUT = fields_out(FORM);
  const C2 W{make_float2(w.x, w.x), make_float2(w.y, w.y)};
  C2 a[FIN], b[FIN];
#pragma unroll
  for (int f = 0; f < FIN; ++f) {
    const C2 e = load2<false>(lo + f * fs), o = load2<true>(hi + f * fs);
    if (f < nft) {
      const C2 t = cmul(o, W);
      a[f] = e + t;
      b[f] = e - t;
    } else {
      a[f] = e;
      b[f] = o;
    }
  }
  {
    const ModeZ2 z = mode_z2(m, k, sh, P);
    update_core2<FORM>(a, m.Kx, m.Ky, make_float2(z.kz, z.kz), m.px, m.py, pack2(z.pz, z.pz), m.pxy, z.q, P);
  }
  {
    const ModeZ2 z = mode_z2(m, k + NZ / 2, sh, P);
    update_core2<FORM>(b, m.Kx, m.Ky, make_float2(z.kz, z.kz), m.px, m.py, pack2(z.pz, z.pz), m.pxy, z.q, P);
  }
#pragma unroll
  for (int f = 0; f < FOUT; ++f) {
    store2<false>(lo + f * fs, a[f] + b[f]);
    store2<true>(hi + f * fs, cmulc(a[f] - b[f], W));
  }
}

template <typename T, int FORM>
__device__ __forceinline__ void update_mode(cx<T>* md, int fs, int mx, int my, int mz,
                                            const ShapeDev& sh, const DevPlan& P) {
  update_mode_z<T, FORM>(md, fs, mode_xy<T>(mx, my, sh, P), mz, sh, P);
}

}  // namespace psatd
