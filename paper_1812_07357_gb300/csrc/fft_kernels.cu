// Batched mixed-radix FFT passes and the fused k-space PSATD update.
//
// Spectral layout of one box and one field slot (the "half spectrum"):
//   element (mx, my, mz), mx in [0, n0/2], at mx + hx*(my + n1*mz), hx = n0/2+1.
//
// Passes of one step (S1..S3 of the PSATD push):
//   fwd_x      real rows -> packed complex FFT of length n0/2 -> R2C split
//   col (y)    complex FFT along y for a tile of mx columns of one z plane
//   z_update   complex FFT along z for a tile of mx columns of one y plane, all
//              field slots at once; the per-mode update; inverse FFT along z
//   col (y)    inverse along y (only z planes that hold interior cells)
//   inv_x      C2R merge -> inverse packed FFT -> real rows (interior only)
//
// Every 1D FFT runs in shared memory as a Stockham autosort sequence of radix
// 2/3/4/5/8 passes; a thread keeps its butterflies in registers between the
// read and the write half of a pass.
#include <cuda_runtime.h>

#include <cstdint>
#include <type_traits>

#include "psatd_internal.h"

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
__device__ __forceinline__ float2 operator+(float2 a, float2 b) { return make_float2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ float2 operator-(float2 a, float2 b) { return make_float2(a.x - b.x, a.y - b.y); }
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

// ---------------------------------------------------------------------------
// DFT butterflies of size R, y_k = sum_t a_t exp(DIR 2 pi i t k / R)
// ---------------------------------------------------------------------------
template <typename T, int R, int DIR>
struct Dft;

template <typename T, int DIR>
struct Dft<T, 2, DIR> {
  static __device__ __forceinline__ void run(cx<T>* v) {
    cx<T> a = v[0], b = v[1];
    v[0] = a + b;
    v[1] = a - b;
  }
};

template <typename T, int DIR>
struct Dft<T, 3, DIR> {
  static __device__ __forceinline__ void run(cx<T>* v) {
    const T h = T(0.86602540378443864676);  // sin(2 pi / 3)
    cx<T> s = v[1] + v[2], d = v[1] - v[2];
    cx<T> m = mk<T>(v[0].x - T(0.5) * s.x, v[0].y - T(0.5) * s.y);
    cx<T> r = rmul(h, rot<DIR>(d));
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
    const T c1 = T(0.30901699437494742410);   // cos(2 pi/5)
    const T c2 = T(-0.80901699437494742410);  // cos(4 pi/5)
    const T s1 = T(0.95105651629515357212);   // sin(2 pi/5)
    const T s2 = T(0.58778525229247312917);   // sin(4 pi/5)
    cx<T> a0 = v[0];
    cx<T> p1 = v[1] + v[4], d1 = v[1] - v[4];
    cx<T> p2 = v[2] + v[3], d2 = v[2] - v[3];
    cx<T> m1 = mk<T>(a0.x + c1 * p1.x + c2 * p2.x, a0.y + c1 * p1.y + c2 * p2.y);
    cx<T> m2 = mk<T>(a0.x + c2 * p1.x + c1 * p2.x, a0.y + c2 * p1.y + c1 * p2.y);
    cx<T> n1 = mk<T>(s1 * d1.x + s2 * d2.x, s1 * d1.y + s2 * d2.y);
    cx<T> n2 = mk<T>(s2 * d1.x - s1 * d2.x, s2 * d1.y - s1 * d2.y);
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
    const T r2 = T(0.70710678118654752440);
    cx<T> e[4] = {v[0], v[2], v[4], v[6]};
    cx<T> o[4] = {v[1], v[3], v[5], v[7]};
    Dft<T, 4, DIR>::run(e);
    Dft<T, 4, DIR>::run(o);
    // o[k] *= exp(DIR i pi k / 4)
    cx<T> w1, w3;
    if (DIR < 0) {
      w1 = mk<T>(r2 * (o[1].x + o[1].y), r2 * (o[1].y - o[1].x));
      w3 = mk<T>(r2 * (o[3].y - o[3].x), -r2 * (o[3].x + o[3].y));
    } else {
      w1 = mk<T>(r2 * (o[1].x - o[1].y), r2 * (o[1].x + o[1].y));
      w3 = mk<T>(-r2 * (o[3].x + o[3].y), r2 * (o[3].x - o[3].y));
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

// ---------------------------------------------------------------------------
// One Stockham pass of radix R over `nseq` sequences of length N in smem.
// Element i of sequence s is buf[s*sseq + i*sidx].  INTERLEAVED selects the
// thread mapping: consecutive threads take consecutive sequences (sseq == 1)
// or consecutive butterflies of one sequence (sidx == 1).
// ---------------------------------------------------------------------------
template <typename T, int R, int DIR, bool INTERLEAVED>
__device__ __forceinline__ void stockham_pass(cx<T>* buf, int N, int nseq, int sseq, int sidx,
                                              int Ns, const cx<T>* __restrict__ tw) {
  constexpr int MAXB = (kPointsPerThread + R - 1) / R + 1;
  const int nbf = N / R;
  const int total = nbf * nseq;
  const int tstride = N / (Ns * R);
  cx<T> v[MAXB][R];
  int off[MAXB];
#pragma unroll
  for (int j = 0; j < MAXB; ++j) {
    const int b = threadIdx.x + j * blockDim.x;
    if (b < total) {
      int s, bf;
      if (INTERLEAVED) {
        s = b % nseq;
        bf = b / nseq;
      } else {
        bf = b % nbf;
        s = b / nbf;
      }
      const int k = bf % Ns;
      off[j] = s * sseq + ((bf - k) * R + k) * sidx;
      const cx<T>* src = buf + s * sseq + bf * sidx;
#pragma unroll
      for (int t = 0; t < R; ++t) {
        cx<T> a = src[t * nbf * sidx];
        if (t > 0 && k > 0) {
          cx<T> w = tw[t * k * tstride];
          a = (DIR < 0) ? cmul(a, w) : cmulc(a, w);
        }
        v[j][t] = a;
      }
      Dft<T, R, DIR>::run(v[j]);
    }
  }
  __syncthreads();
#pragma unroll
  for (int j = 0; j < MAXB; ++j) {
    const int b = threadIdx.x + j * blockDim.x;
    if (b < total) {
      cx<T>* dst = buf + off[j];
#pragma unroll
      for (int t = 0; t < R; ++t) dst[t * Ns * sidx] = v[j][t];
    }
  }
  __syncthreads();
}

// Full FFT of `nseq` sequences (chunked so that one chunk holds at most
// kMaxPoints points).  Output in natural order, unnormalised.
template <typename T, int DIR, bool INTERLEAVED>
__device__ void fft_smem(cx<T>* buf, int nseq, int sseq, int sidx, const AxisPlan& ap,
                         const cx<T>* __restrict__ tw) {
  const int N = ap.n;
  if (N <= 1) return;
  int chunk = kMaxPoints / N;
  if (chunk < 1) chunk = 1;
  for (int s0 = 0; s0 < nseq; s0 += chunk) {
    const int ns = min(chunk, nseq - s0);
    cx<T>* b = buf + s0 * sseq;
    int Ns = 1;
    for (int p = 0; p < ap.npass; ++p) {
      const int R = ap.radix[p];
      switch (R) {
        case 2: stockham_pass<T, 2, DIR, INTERLEAVED>(b, N, ns, sseq, sidx, Ns, tw); break;
        case 3: stockham_pass<T, 3, DIR, INTERLEAVED>(b, N, ns, sseq, sidx, Ns, tw); break;
        case 4: stockham_pass<T, 4, DIR, INTERLEAVED>(b, N, ns, sseq, sidx, Ns, tw); break;
        case 5: stockham_pass<T, 5, DIR, INTERLEAVED>(b, N, ns, sseq, sidx, Ns, tw); break;
        default: stockham_pass<T, 8, DIR, INTERLEAVED>(b, N, ns, sseq, sidx, Ns, tw); break;
      }
      Ns *= R;
    }
  }
}

template <typename T>
__device__ __forceinline__ const cx<T>* cpool(const DevPlan& P) {
  return reinterpret_cast<const cx<T>*>(P.cpool);
}
template <typename T>
__device__ __forceinline__ const T* rpool(const DevPlan& P) {
  return reinterpret_cast<const T*>(P.rpool);
}

// ---------------------------------------------------------------------------
// S1, x axis: real rows -> half spectrum (R2C via a packed complex FFT)
// z[m] = x[2m] + i x[2m+1];  Z = FFT_L(z);
// X[k] = (Z[k] + conj Z[L-k])/2 + w^k (Z[k] - conj Z[L-k])/(2i),  w = exp(-2 pi i/n0)
// ---------------------------------------------------------------------------
template <typename T>
__global__ void __launch_bounds__(kThreads) k_fwd_x(DevPlan P, FieldPtrs F, cx<T>* spec,
                                                    int64_t sstride, const RowJob* __restrict__ jobs) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  cx<T>* sm = reinterpret_cast<cx<T>*>(smem_raw);
  const RowJob J = jobs[blockIdx.x];
  const int f = blockIdx.y;
  const BoxDev bx = P.boxes[J.box];
  const ShapeDev& sh = P.shapes[bx.shape];
  const int L = sh.L, hx = sh.hx;
  const cx<T>* in = reinterpret_cast<const cx<T>*>(reinterpret_cast<const T*>(F.p[f]) + bx.foff) +
                    (int64_t)J.r0 * L;
  const int np = J.nr * L;
  for (int e = threadIdx.x; e < np; e += blockDim.x) sm[e] = in[e];
  __syncthreads();
  fft_smem<T, -1, false>(sm, J.nr, L, 1, sh.ax, cpool<T>(P) + sh.ax.tw);
  const cx<T>* post = cpool<T>(P) + sh.post;
  cx<T>* out = spec + f * sstride + bx.soff + (int64_t)J.r0 * hx;
  const int no = J.nr * hx;
  for (int e = threadIdx.x; e < no; e += blockDim.x) {
    const int r = e / hx, k = e - r * hx;
    const cx<T> a = sm[r * L + (k == L ? 0 : k)];
    const cx<T> b = sm[r * L + (k == 0 ? 0 : L - k)];
    const cx<T> A = mk<T>(T(0.5) * (a.x + b.x), T(0.5) * (a.y - b.y));
    const cx<T> Bv = mk<T>(T(0.5) * (a.y + b.y), T(0.5) * (b.x - a.x));
    out[e] = A + cmul(post[k], Bv);
  }
}

// ---------------------------------------------------------------------------
// Column FFT along y (axis 1) or z (axis 2) for one plane and a tile of mx.
// ---------------------------------------------------------------------------
template <typename T, int DIR>
__global__ void __launch_bounds__(kThreads) k_col(DevPlan P, cx<T>* spec, int64_t sstride, int axis,
                                                  const ColJob* __restrict__ jobs) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  cx<T>* sm = reinterpret_cast<cx<T>*>(smem_raw);
  const ColJob J = jobs[blockIdx.x];
  const int f = blockIdx.y;
  const BoxDev bx = P.boxes[J.box];
  const ShapeDev& sh = P.shapes[bx.shape];
  const int hx = sh.hx, n1 = bx.n[1];
  const AxisPlan& ap = axis == 1 ? sh.ay : sh.az;
  const int N = ap.n;
  int64_t base, stride;
  if (axis == 1) {
    base = (int64_t)J.plane * n1 * hx;
    stride = hx;
  } else {
    base = (int64_t)J.plane * hx;
    stride = (int64_t)n1 * hx;
  }
  cx<T>* g = spec + f * sstride + bx.soff + base + J.m0;
  const int nm = J.nm;
  for (int e = threadIdx.x; e < N * nm; e += blockDim.x) {
    const int i = e / nm, t = e - i * nm;
    sm[e] = g[i * stride + t];
  }
  __syncthreads();
  fft_smem<T, DIR, true>(sm, nm, 1, nm, ap, cpool<T>(P) + ap.tw);
  for (int e = threadIdx.x; e < N * nm; e += blockDim.x) {
    const int i = e / nm, t = e - i * nm;
    g[i * stride + t] = sm[e];
  }
}

// ---------------------------------------------------------------------------
// S2: analytical update of one mode (centred spectra; see plan docs).
// md[s * fs] is field slot s of this mode in smem.
// ---------------------------------------------------------------------------
template <typename T, int FORM>
__device__ __forceinline__ void update_mode(cx<T>* md, int fs, int mx, int my, int mz,
                                            const ShapeDev& sh, const DevPlan& P) {
  using C = cx<T>;
  const T* rp = rpool<T>(P);
  const C* cp = cpool<T>(P);
  const int n1 = sh.n[1], n2 = sh.n[2], hx = sh.hx;
  const T Kx = rp[sh.kx + mx], Ky = rp[sh.ky + my], Kz = rp[sh.kz + mz];
  const C px = cp[sh.phx + mx], py = cp[sh.phy + my], pz = cp[sh.phz + mz];
  const int myr = my <= n1 - my ? my : n1 - my;
  const int mzr = mz <= n2 - mz ? mz : n2 - mz;
  const Coef4<T> q = reinterpret_cast<const Coef4<T>*>(P.coef)[sh.coef +
                                                             ((int64_t)mzr * (n1 / 2 + 1) + myr) * hx + mx];
  const C pyz = cmul(py, pz), pxz = cmul(px, pz), pxy = cmul(px, py);
  // centred spectra: F~ = exp(-i k.s h) F^
  const C ex = cmulc(md[0], px), ey = cmulc(md[fs], py), ez = cmulc(md[2 * fs], pz);
  const C bx = cmulc(md[3 * fs], pyz), by = cmulc(md[4 * fs], pxz), bz = cmulc(md[5 * fs], pxy);
  const T cc = T(P.c) * T(P.c);
  const T ieps = T(1.0 / P.eps0);
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
    const T y1 = q.x3 / dt;
    const T y2 = -q.x1 - q.x3 / dt;
    const C g = times_i(rmul(y1, rhon) + rmul(y2, rho));  // i (Y1 rho' + Y2 rho)
    nex = rmul(q.c, ex) + rmul(csw, times_i(kbx)) - rmul(q.s * ieps, jx) + rmul(Kx * ieps, g);
    ney = rmul(q.c, ey) + rmul(csw, times_i(kby)) - rmul(q.s * ieps, jy) + rmul(Ky * ieps, g);
    nez = rmul(q.c, ez) + rmul(csw, times_i(kbz)) - rmul(q.s * ieps, jz) + rmul(Kz * ieps, g);
    const T x2 = q.x1 / cc * ieps;
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
      const T x2 = q.x1 / cc * ieps;
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

// z forward FFT of every slot, update, z inverse FFT of the output slots.
// smem layout [z][slot][t] with t the column inside the tile.
template <typename T, int FORM>
__global__ void __launch_bounds__(kThreads) k_z_update(DevPlan P, cx<T>* spec, int64_t sstride,
                                                       const ColJob* __restrict__ jobs) {
  constexpr int FIN = fields_in(FORM);
  constexpr int FOUT = fields_out(FORM);
  extern __shared__ __align__(16) unsigned char smem_raw[];
  cx<T>* sm = reinterpret_cast<cx<T>*>(smem_raw);
  const ColJob J = jobs[blockIdx.x];
  const BoxDev bx = P.boxes[J.box];
  const ShapeDev& sh = P.shapes[bx.shape];
  const int hx = sh.hx, n1 = bx.n[1], n2 = bx.n[2];
  const int nm = J.nm;
  const int row = FIN * nm;
  const int64_t zstride = (int64_t)n1 * hx;
  cx<T>* g = spec + bx.soff + (int64_t)J.plane * hx + J.m0;
  for (int e = threadIdx.x; e < n2 * row; e += blockDim.x) {
    const int z = e / row, r = e - z * row;
    const int s = r / nm, t = r - s * nm;
    sm[e] = g[s * sstride + z * zstride + t];
  }
  __syncthreads();
  const cx<T>* twz = cpool<T>(P) + sh.az.tw;
  fft_smem<T, -1, true>(sm, row, 1, row, sh.az, twz);
  for (int e = threadIdx.x; e < n2 * nm; e += blockDim.x) {
    const int z = e / nm, t = e - z * nm;
    update_mode<T, FORM>(sm + z * row + t, nm, J.m0 + t, J.plane, z, sh, P);
  }
  __syncthreads();
  fft_smem<T, 1, true>(sm, FOUT * nm, 1, row, sh.az, twz);
  const int rowo = FOUT * nm;
  for (int e = threadIdx.x; e < n2 * rowo; e += blockDim.x) {
    const int z = e / rowo, r = e - z * rowo;
    const int s = r / nm, t = r - s * nm;
    g[s * sstride + z * zstride + t] = sm[z * row + r];
  }
}

// ---------------------------------------------------------------------------
// S3, x axis: half spectrum -> real rows (C2R), with 1/(n0 n1 n2).
// Z'[k] = (X[k] + conj X[L-k]) + i w^-k (X[k] - conj X[L-k]),  k < L
// z = IFFT_L(Z') (unnormalised);  x[2m] = Re z[m], x[2m+1] = Im z[m]
// ---------------------------------------------------------------------------
template <typename T>
__global__ void __launch_bounds__(kThreads) k_inv_x(DevPlan P, FieldPtrs F, const cx<T>* spec,
                                                    int64_t sstride, const RowJob* __restrict__ jobs,
                                                    int interior_only) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  cx<T>* smx = reinterpret_cast<cx<T>*>(smem_raw);
  const RowJob J = jobs[blockIdx.x];
  const int f = blockIdx.y;
  const BoxDev bx = P.boxes[J.box];
  const ShapeDev& sh = P.shapes[bx.shape];
  const int L = sh.L, hx = sh.hx, n0 = bx.n[0];
  cx<T>* smz = smx + J.nr * hx;
  const cx<T>* in = spec + f * sstride + bx.soff + (int64_t)J.r0 * hx;
  for (int e = threadIdx.x; e < J.nr * hx; e += blockDim.x) smx[e] = in[e];
  __syncthreads();
  const cx<T>* post = cpool<T>(P) + sh.post;
  for (int e = threadIdx.x; e < J.nr * L; e += blockDim.x) {
    const int r = e / L, k = e - r * L;
    const cx<T> a = smx[r * hx + k];
    const cx<T> b = conjg(smx[r * hx + L - k]);
    smz[e] = (a + b) + times_i(cmulc(a - b, post[k]));
  }
  __syncthreads();
  fft_smem<T, 1, false>(smz, J.nr, L, 1, sh.ax, cpool<T>(P) + sh.ax.tw);
  const T scale = T(1.0 / ((double)n0 * bx.n[1] * bx.n[2]));
  T* out = reinterpret_cast<T*>(F.p[f]) + bx.foff + (int64_t)J.r0 * n0;
  const int xlo = interior_only ? bx.ng_lo[0] : 0;
  const int xhi = interior_only ? n0 - bx.ng_hi[0] : n0;
  for (int e = threadIdx.x; e < J.nr * n0; e += blockDim.x) {
    const int r = e / n0, x = e - r * n0;
    if (x < xlo || x >= xhi) continue;
    const cx<T> z = smz[r * L + (x >> 1)];
    out[e] = scale * ((x & 1) ? z.y : z.x);
  }
}

// ---------------------------------------------------------------------------
// launchers
// ---------------------------------------------------------------------------
namespace {
constexpr int64_t kMaxGridX = 2147483647LL;
}  // namespace

cudaError_t launch_fwd_x(int prec, const DevPlan& P, const FieldPtrs& f, int nf, void* spec,
                         int64_t sstride, const RowJob* jobs, int64_t njobs, int smem,
                         cudaStream_t st) {
  if (njobs <= 0 || nf <= 0) return cudaSuccess;
  if (njobs > kMaxGridX) return cudaErrorInvalidConfiguration;
  dim3 grid((unsigned)njobs, nf);
  if (prec == 32)
    k_fwd_x<float><<<grid, kThreads, smem, st>>>(P, f, (float2*)spec, sstride, jobs);
  else
    k_fwd_x<double><<<grid, kThreads, smem, st>>>(P, f, (double2*)spec, sstride, jobs);
  return cudaGetLastError();
}

cudaError_t launch_col(int prec, int dir, int axis, const DevPlan& P, void* spec, int64_t sstride,
                       int nf, const ColJob* jobs, int64_t njobs, int smem, cudaStream_t st) {
  if (njobs <= 0 || nf <= 0) return cudaSuccess;
  dim3 grid((unsigned)njobs, nf);
  if (prec == 32) {
    if (dir < 0)
      k_col<float, -1><<<grid, kThreads, smem, st>>>(P, (float2*)spec, sstride, axis, jobs);
    else
      k_col<float, 1><<<grid, kThreads, smem, st>>>(P, (float2*)spec, sstride, axis, jobs);
  } else {
    if (dir < 0)
      k_col<double, -1><<<grid, kThreads, smem, st>>>(P, (double2*)spec, sstride, axis, jobs);
    else
      k_col<double, 1><<<grid, kThreads, smem, st>>>(P, (double2*)spec, sstride, axis, jobs);
  }
  return cudaGetLastError();
}

cudaError_t launch_z_update(int prec, int form, const DevPlan& P, void* spec, int64_t sstride,
                            const ColJob* jobs, int64_t njobs, int smem, cudaStream_t st) {
  if (njobs <= 0) return cudaSuccess;
  dim3 grid((unsigned)njobs);
#define PSATD_ZU(T, C2, FORMV) \
  k_z_update<T, FORMV><<<grid, kThreads, smem, st>>>(P, (C2*)spec, sstride, jobs)
  if (prec == 32) {
    if (form == kVacuum) PSATD_ZU(float, float2, kVacuum);
    else if (form == kJForm) PSATD_ZU(float, float2, kJForm);
    else PSATD_ZU(float, float2, kRhoForm);
  } else {
    if (form == kVacuum) PSATD_ZU(double, double2, kVacuum);
    else if (form == kJForm) PSATD_ZU(double, double2, kJForm);
    else PSATD_ZU(double, double2, kRhoForm);
  }
#undef PSATD_ZU
  return cudaGetLastError();
}

cudaError_t launch_inv_x(int prec, const DevPlan& P, const FieldPtrs& f, int nf, void* spec,
                         int64_t sstride, const RowJob* jobs, int64_t njobs, int smem,
                         int interior_only, cudaStream_t st) {
  if (njobs <= 0 || nf <= 0) return cudaSuccess;
  dim3 grid((unsigned)njobs, nf);
  if (prec == 32)
    k_inv_x<float><<<grid, kThreads, smem, st>>>(P, f, (const float2*)spec, sstride, jobs,
                                                  interior_only);
  else
    k_inv_x<double><<<grid, kThreads, smem, st>>>(P, f, (const double2*)spec, sstride, jobs,
                                                   interior_only);
  return cudaGetLastError();
}

cudaError_t configure_kernels(int prec, int smem) {
  cudaError_t e = cudaSuccess;
#define PSATD_SET(K)                                                                  \
  do {                                                                                \
    cudaError_t r = cudaFuncSetAttribute(K, cudaFuncAttributeMaxDynamicSharedMemorySize, smem); \
    if (r != cudaSuccess) e = r;                                                      \
  } while (0)
  if (prec == 32) {
    PSATD_SET(k_fwd_x<float>);
    PSATD_SET((k_col<float, -1>));
    PSATD_SET((k_col<float, 1>));
    PSATD_SET((k_z_update<float, kVacuum>));
    PSATD_SET((k_z_update<float, kJForm>));
    PSATD_SET((k_z_update<float, kRhoForm>));
    PSATD_SET(k_inv_x<float>);
  } else {
    PSATD_SET(k_fwd_x<double>);
    PSATD_SET((k_col<double, -1>));
    PSATD_SET((k_col<double, 1>));
    PSATD_SET((k_z_update<double, kVacuum>));
    PSATD_SET((k_z_update<double, kJForm>));
    PSATD_SET((k_z_update<double, kRhoForm>));
    PSATD_SET(k_inv_x<double>);
  }
#undef PSATD_SET
  return e;
}

}  // namespace psatd
