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

template <typename T, int FORM>
__device__ __forceinline__ void update_mode_z(cx<T>* md, int fs, const ModeXY<T>& m, int mz, const ShapeDev& sh,
                                              const DevPlan& P) {
  using C = cx<T>;
  const T* rp = rpool<T>(P);
  const C* cp = cpool<T>(P);
  const int n1 = sh.n[1], n2 = sh.n[2];
  const T Kx = m.Kx, Ky = m.Ky, Kz = rp[sh.kz + mz];
  const C px = m.px, py = m.py, pz = cp[sh.phz + mz], pxy = m.pxy;
  const int mzr = mz <= n2 - mz ? mz : n2 - mz;
  const Coef4<T> q =
      reinterpret_cast<const Coef4<T>*>(P.coef)[m.qbase + (int64_t)mzr * (n1 / 2 + 1) * sh.hx];
  const C pyz = cmul(py, pz), pxz = cmul(px, pz);
  // centred spectra: F~ = exp(-i k.s h) F^
  const C ex = cmulc(md[0], px), ey = cmulc(md[fs], py), ez = cmulc(md[2 * fs], pz);
  const C bx = cmulc(md[3 * fs], pyz), by = cmulc(md[4 * fs], pxz), bz = cmulc(md[5 * fs], pxy);
  const T cc = T(P.cc);
  const T ieps = T(P.ieps);
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
    const C rho = md[6 * fs];
    const C jx = cmulc(md[7 * fs], px), jy = cmulc(md[8 * fs], py), jz = cmulc(md[9 * fs], pz);
    const C kdj = rmul(Kx, jx) + rmul(Ky, jy) + rmul(Kz, jz);
    const T dt = T(P.dt);
    const C rhon = rho - rmul(dt, times_i(kdj));
    const T y1 = q.x3 * T(P.idt);
    const T y2 = -q.x1 - y1;
    const C g = times_i(rmul(y1, rhon) + rmul(y2, rho));  // i (Y1 rho' + Y2 rho)
    nex = rmul(q.c, ex) + rmul(csw, times_i(kbx)) - rmul(q.s * ieps, jx) + rmul(Kx * ieps, g);
    ney = rmul(q.c, ey) + rmul(csw, times_i(kby)) - rmul(q.s * ieps, jy) + rmul(Ky * ieps, g);
    nez = rmul(q.c, ez) + rmul(csw, times_i(kbz)) - rmul(q.s * ieps, jz) + rmul(Kz * ieps, g);
    const T x2 = q.x1 * T(P.icce);
    nbx = nbx + rmul(x2, times_i(rmul(Ky, jz) - rmul(Kz, jy)));
    nby = nby + rmul(x2, times_i(rmul(Kz, jx) - rmul(Kx, jz)));
    nbz = nbz + rmul(x2, times_i(rmul(Kx, jy) - rmul(Ky, jx)));
    md[6 * fs] = rhon;
  } else {
    const C kde = rmul(Kx, ex) + rmul(Ky, ey) + rmul(Kz, ez);
    nex = rmul(q.c, ex) + rmul(q.x1 * Kx, kde) + rmul(csw, times_i(kbx));
    ney = rmul(q.c, ey) + rmul(q.x1 * Ky, kde) + rmul(csw, times_i(kby));
    nez = rmul(q.c, ez) + rmul(q.x1 * Kz, kde) + rmul(csw, times_i(kbz));
    if (FORM == kJForm) {
      const C jx = cmulc(md[6 * fs], px), jy = cmulc(md[7 * fs], py), jz = cmulc(md[8 * fs], pz);
      const C kdj = rmul(Kx, jx) + rmul(Ky, jy) + rmul(Kz, jz);
      const T a = q.s * ieps, b = q.x3 * ieps;
      nex = nex - rmul(a, jx) + rmul(b * Kx, kdj);
      ney = ney - rmul(a, jy) + rmul(b * Ky, kdj);
      nez = nez - rmul(a, jz) + rmul(b * Kz, kdj);
      const T x2 = q.x1 * T(P.icce);
      nbx = nbx + rmul(x2, times_i(rmul(Ky, jz) - rmul(Kz, jy)));
      nby = nby + rmul(x2, times_i(rmul(Kz, jx) - rmul(Kx, jz)));
      nbz = nbz + rmul(x2, times_i(rmul(Kx, jy) - rmul(Ky, jx)));
    }
  }
  // back to the staggered sample positions: F^ = exp(+i k.s h) F~
  md[0] = cmul(nex, px);
  md[fs] = cmul(ney, py);
  md[2 * fs] = cmul(nez, pz);
  md[3 * fs] = cmul(nbx, pyz);
  md[4 * fs] = cmul(nby, pxz);
  md[5 * fs] = cmul(nbz, pxy);
}

template <typename T, int FORM>
__device__ __forceinline__ void update_mode(cx<T>* md, int fs, int mx, int my, int mz,
                                            const ShapeDev& sh, const DevPlan& P) {
  update_mode_z<T, FORM>(md, fs, mode_xy<T>(mx, my, sh, P), mz, sh, P);
}

}  // namespace psatd
