// Fast path of the PSATD push for box sizes whose FFT lengths factor as
// N = R1 * R2 with both factors in the register codelet set (list in
// psatd_internal.h, PSATD_FAST_LENGTHS).  Three kernels per step:
//
//   k_plane_fwd   one (box, field, z) plane: real rows -> R2C along x ->
//                 complex FFT along y -> half spectrum plane in HBM.
//   k_z_fast      one (box, y, mx tile): z FFT of every field slot, loaded
//                 straight from HBM into registers; k-space update; inverse z
//                 FFT of the output slots, stored straight to HBM.
//   k_plane_inv   one (box, field, interior z) plane: inverse y FFT -> C2R
//                 along x for interior rows -> interior cells to HBM.
//
// Every 1D FFT is a two-pass ("four-step") transform: pass 1 takes R1
// elements at stride R2, does DFT_R1 in registers and multiplies by
// w_N^(n2 k1); pass 2 takes R2 consecutive pass-1 results and does DFT_R2,
// giving X[k1 + R1 k2] in natural order.  Shared memory holds the data
// between the passes; all index arithmetic inside a pass is compile-time.
#include <cuda_runtime.h>

#include <cstdint>

#include "fft_codelets.cuh"
#include "psatd_internal.h"
#include "psatd_update.cuh"

namespace psatd {

namespace {

template <typename T>
__device__ __forceinline__ const cx<T>* ctab(const DevPlan& P) {
  return reinterpret_cast<const cx<T>*>(P.cpool);
}
template <typename T>
__device__ __forceinline__ const T* rtab(const DevPlan& P) {
  return reinterpret_cast<const T*>(P.rpool);
}

// e / d for 0 <= e < 2^24, d > 0, with inv = 1.0f / d.
__device__ __forceinline__ int div_small(int e, int d, float inv) {
  int q = __float2int_rz((float)e * inv);
  q += (q + 1) * d <= e;
  q -= q * d > e;
  return q;
}

// ---------------------------------------------------------------------------
// pass 1, in place: column c, positions n1*R2 + n2 (n1 < R1); DFT_R1 along
// n1, times w_N^(n2 k1), back to positions k1*R2 + n2.
// CFAST: consecutive threads take consecutive columns (else consecutive n2).
// ---------------------------------------------------------------------------
template <typename T, int R1, int R2, int DIR, bool CFAST>
__device__ __forceinline__ void pass1(cx<T>* buf, int ncol, int cs, int ns, const cx<T>* __restrict__ tw,
                                      float inv_ncol) {
  const int items = ncol * R2;
  for (int it = threadIdx.x; it < items; it += blockDim.x) {
    int c, n2;
    if (CFAST) {
      n2 = div_small(it, ncol, inv_ncol);
      c = it - n2 * ncol;
    } else {
      c = it / R2;
      n2 = it - c * R2;
    }
    cx<T>* p = buf + c * cs + n2 * ns;
    cx<T> v[R1];
#pragma unroll
    for (int j = 0; j < R1; ++j) v[j] = p[j * R2 * ns];
    Dft<T, R1, DIR>::run(v);
    if (n2) {
#pragma unroll
      for (int k = 1; k < R1; ++k) v[k] = twmul<DIR>(v[k], tw[n2 * k]);
    }
#pragma unroll
    for (int j = 0; j < R1; ++j) p[j * R2 * ns] = v[j];
  }
}

// pass 2: column c, R2 consecutive pass-1 results at k1*R2 + n2; DFT_R2;
// st(c, k1 + R1*k2, value) receives the natural-order outputs.
template <typename T, int R1, int R2, int DIR, bool CFAST, typename Store>
__device__ __forceinline__ void pass2(const cx<T>* buf, int ncol, int cs, int ns, float inv_ncol,
                                      Store&& st) {
  const int items = ncol * R1;
  for (int it = threadIdx.x; it < items; it += blockDim.x) {
    int c, k1;
    if (CFAST) {
      k1 = div_small(it, ncol, inv_ncol);
      c = it - k1 * ncol;
    } else {
      c = it / R1;
      k1 = it - c * R1;
    }
    const cx<T>* p = buf + c * cs + k1 * R2 * ns;
    cx<T> u[R2];
#pragma unroll
    for (int j = 0; j < R2; ++j) u[j] = p[j * ns];
    Dft<T, R2, DIR>::run(u);
#pragma unroll
    for (int k2 = 0; k2 < R2; ++k2) st(c, k1 + R1 * k2, u[k2]);
  }
}

// ---------------------------------------------------------------------------
// forward plane: x (R2C) then y
// ---------------------------------------------------------------------------
template <typename T, int R1, int R2>
__device__ __forceinline__ void plane_x_fwd(cx<T>* in, cx<T>* work, const cx<T>* g, int n1, int lp,
                                            int hp, const cx<T>* __restrict__ twx,
                                            const cx<T>* __restrict__ post) {
  constexpr int L = R1 * R2;
  // load: n1 rows of L complex (pairs of reals), contiguous in HBM
  for (int e = threadIdx.x; e < n1 * L; e += blockDim.x) {
    const int y = e / L, x = e - y * L;
    in[y * lp + x] = g[e];
  }
  __syncthreads();
  pass1<T, R1, R2, -1, false>(in, n1, lp, 1, twx, 0.f);
  __syncthreads();
  pass2<T, R1, R2, -1, false>(in, n1, lp, 1, 0.f,
                              [&](int c, int k, cx<T> v) { work[c * hp + k] = v; });
  __syncthreads();
  // R2C split in place, one thread per pair (k, L-k):
  // X[k] = (Z[k] + conj Z[L-k])/2 - i w^k (Z[k] - conj Z[L-k])/2
  constexpr int H = L / 2 + 1;
  for (int e = threadIdx.x; e < n1 * H; e += blockDim.x) {
    const int y = e / H, k = e - y * H;
    cx<T>* row = work + y * hp;
    const cx<T> a = row[k];
    const cx<T> b = row[k == 0 ? 0 : L - k];
    // A = (a + conj b)/2, Bv = (a - conj b)/(2i)
    const cx<T> A = mk<T>(T(0.5) * (a.x + b.x), T(0.5) * (a.y - b.y));
    const cx<T> Bv = mk<T>(T(0.5) * (a.y + b.y), T(0.5) * (b.x - a.x));
    if (k == 0) {
      row[0] = mk<T>(A.x + Bv.x, A.y + Bv.y);
      row[L] = mk<T>(A.x - Bv.x, A.y - Bv.y);
    } else {
      row[k] = A + cmul(post[k], Bv);
      if (2 * k != L) {
        // partner: A' = conj A, Bv' = conj Bv
        row[L - k] = conjg(A) + cmul(post[L - k], conjg(Bv));
      }
    }
  }
}

template <typename T, int R1, int R2>
__device__ __forceinline__ void plane_y_fwd(cx<T>* work, int hx, int hp, cx<T>* out,
                                            const cx<T>* __restrict__ twy) {
  const float inv = 1.0f / hx;
  pass1<T, R1, R2, -1, true>(work, hx, 1, hp, twy, inv);
  __syncthreads();
  pass2<T, R1, R2, -1, true>(work, hx, 1, hp, inv,
                             [&](int c, int k, cx<T> v) { out[k * hx + c] = v; });
}

template <typename T>
__global__ void __launch_bounds__(512, sizeof(T) == 4 ? 2 : 1) k_plane_fwd(DevPlan P, FieldPtrs F, cx<T>* spec, int64_t sstride,
                                                      const int2* __restrict__ jobs) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int2 J = jobs[blockIdx.x];
  const int f = blockIdx.y;
  const BoxDev bx = P.boxes[J.x];
  const ShapeDev& sh = P.shapes[bx.shape];
  const int n1 = bx.n[1], hx = sh.hx, L = sh.L;
  const int lp = sh.lp, hp = sh.hp;
  cx<T>* in = reinterpret_cast<cx<T>*>(smem_raw);
  cx<T>* work = in + n1 * lp;
  const cx<T>* g = reinterpret_cast<const cx<T>*>(reinterpret_cast<const T*>(F.p[f]) + bx.foff) +
                   (int64_t)J.y * n1 * L;
  const cx<T>* twx = ctab<T>(P) + sh.ax.tw;
  const cx<T>* post = ctab<T>(P) + sh.post;
  switch (sh.fx) {
#define PSATD_ARM(code, N, R1, R2) \
  case code: plane_x_fwd<T, R1, R2>(in, work, g, n1, lp, hp, twx, post); break;
    PSATD_FAST_LENGTHS(PSATD_ARM)
#undef PSATD_ARM
    default: break;
  }
  __syncthreads();
  cx<T>* out = spec + f * sstride + bx.soff + (int64_t)J.y * n1 * hx;
  const cx<T>* twy = ctab<T>(P) + sh.ay.tw;
  switch (sh.fy) {
#define PSATD_ARM(code, N, R1, R2) \
  case code: plane_y_fwd<T, R1, R2>(work, hx, hp, out, twy); break;
    PSATD_FAST_LENGTHS(PSATD_ARM)
#undef PSATD_ARM
    default: break;
  }
}

// ---------------------------------------------------------------------------
// inverse plane: y then C2R along x, interior rows and cells only
// ---------------------------------------------------------------------------
template <typename T, int R1, int R2>
__device__ __forceinline__ void plane_y_inv(cx<T>* work, const cx<T>* g, int hx, int hp, cx<T>* out,
                                            int ylo, int yhi, const cx<T>* __restrict__ twy) {
  constexpr int N = R1 * R2;
  const float inv = 1.0f / hx;
  for (int e = threadIdx.x; e < N * hx; e += blockDim.x) {
    const int y = div_small(e, hx, inv), x = e - y * hx;
    work[y * hp + x] = g[e];
  }
  __syncthreads();
  pass1<T, R1, R2, 1, true>(work, hx, 1, hp, twy, inv);
  __syncthreads();
  pass2<T, R1, R2, 1, true>(work, hx, 1, hp, inv, [&](int c, int k, cx<T> v) {
    if (k >= ylo && k < yhi) out[(k - ylo) * hp + c] = v;
  });
}

template <typename T, int R1, int R2>
__device__ __forceinline__ void plane_x_inv(cx<T>* rows, int nrows, int hp, T* gout, int n0,
                                            int xlo, int xhi, T scale, const cx<T>* __restrict__ twx,
                                            const cx<T>* __restrict__ post) {
  constexpr int L = R1 * R2;
  constexpr int H = L / 2 + 1;
  // C2R merge in place, one thread per pair (k, L-k), k < L:
  // Z'[k] = (X[k] + conj X[L-k]) + i w^-k (X[k] - conj X[L-k])
  for (int e = threadIdx.x; e < nrows * H; e += blockDim.x) {
    const int r = e / H, k = e - r * H;
    cx<T>* row = rows + r * hp;
    const cx<T> a = row[k];
    const cx<T> b = row[L - k];
    const cx<T> za = (a + conjg(b)) + times_i(cmulc(a - conjg(b), post[k]));
    if (k != 0 && 2 * k != L) {
      const cx<T> zb = (b + conjg(a)) + times_i(cmulc(b - conjg(a), post[L - k]));
      row[L - k] = zb;
    }
    row[k] = za;
  }
  __syncthreads();
  pass1<T, R1, R2, 1, false>(rows, nrows, hp, 1, twx, 0.f);
  __syncthreads();
  pass2<T, R1, R2, 1, false>(rows, nrows, hp, 1, 0.f, [&](int r, int m, cx<T> v) {
    T* o = gout + (int64_t)r * n0 + 2 * m;
    if (2 * m >= xlo && 2 * m < xhi) o[0] = scale * v.x;
    if (2 * m + 1 >= xlo && 2 * m + 1 < xhi) o[1] = scale * v.y;
  });
}

template <typename T>
__global__ void __launch_bounds__(512, sizeof(T) == 4 ? 2 : 1) k_plane_inv(DevPlan P, FieldPtrs F, const cx<T>* spec,
                                                      int64_t sstride, const int2* __restrict__ jobs) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int2 J = jobs[blockIdx.x];
  const int f = blockIdx.y;
  const BoxDev bx = P.boxes[J.x];
  const ShapeDev& sh = P.shapes[bx.shape];
  const int n0 = bx.n[0], n1 = bx.n[1], hx = sh.hx, hp = sh.hp;
  const int ylo = bx.ng_lo[1], yhi = n1 - bx.ng_hi[1];
  cx<T>* work = reinterpret_cast<cx<T>*>(smem_raw);
  cx<T>* rows = work + n1 * hp;
  const cx<T>* g = spec + f * sstride + bx.soff + (int64_t)J.y * n1 * hx;
  const cx<T>* twy = ctab<T>(P) + sh.ay.tw;
  switch (sh.fy) {
#define PSATD_ARM(code, N, R1, R2) \
  case code: plane_y_inv<T, R1, R2>(work, g, hx, hp, rows, ylo, yhi, twy); break;
    PSATD_FAST_LENGTHS(PSATD_ARM)
#undef PSATD_ARM
    default: break;
  }
  __syncthreads();
  const T scale = T(1.0 / ((double)n0 * n1 * bx.n[2]));
  T* gout = reinterpret_cast<T*>(F.p[f]) + bx.foff + ((int64_t)J.y * n1 + ylo) * n0;
  const cx<T>* twx = ctab<T>(P) + sh.ax.tw;
  const cx<T>* post = ctab<T>(P) + sh.post;
  switch (sh.fx) {
#define PSATD_ARM(code, N, R1, R2)                                                          \
  case code:                                                                                \
    plane_x_inv<T, R1, R2>(rows, yhi - ylo, hp, gout, n0, bx.ng_lo[0], n0 - bx.ng_hi[0], scale, \
                           twx, post);                                                      \
    break;
    PSATD_FAST_LENGTHS(PSATD_ARM)
#undef PSATD_ARM
    default: break;
  }
}

// ---------------------------------------------------------------------------
// z FFT + k-space update + inverse z FFT, all field slots of one mx tile
// ---------------------------------------------------------------------------
template <typename T, int FORM, int TX, int R1, int R2>
__device__ __forceinline__ void z_body(cx<T>* buf, cx<T>* g, int64_t sstride, int64_t zst, int nm, int m0,
                                       int y, const ShapeDev& sh, const DevPlan& P) {
  constexpr int FIN = fields_in(FORM), FOUT = fields_out(FORM);
  constexpr int NCOL = FIN * TX;
  constexpr int NP = NCOL + ((24 - NCOL % 16) % 16);   // row pitch, = 8 (mod 16)
  constexpr int N = R1 * R2;
  const cx<T>* tw = ctab<T>(P) + sh.az.tw;
  // pass 1 straight from HBM: item (c = slot*TX + t, n2)
  for (int it = threadIdx.x; it < NCOL * R2; it += blockDim.x) {
    const int n2 = it / NCOL, c = it - n2 * NCOL;
    const int s = c / TX, t = c - s * TX;
    if (t >= nm) continue;
    const cx<T>* p = g + s * sstride + n2 * zst + t;
    cx<T> v[R1];
#pragma unroll
    for (int j = 0; j < R1; ++j) v[j] = p[j * R2 * zst];
    Dft<T, R1, -1>::run(v);
    if (n2) {
#pragma unroll
      for (int k = 1; k < R1; ++k) v[k] = cmul(v[k], tw[n2 * k]);
    }
#pragma unroll
    for (int j = 0; j < R1; ++j) buf[(j * R2 + n2) * NP + c] = v[j];
  }
  __syncthreads();
  // pass 2 in place: all loads first (registers), then natural-order stores
  {
    constexpr int ITEMS = NCOL * R1;
    constexpr int MAXI = (ITEMS + kThreads - 1) / kThreads;
    cx<T> u[MAXI][R2];
#pragma unroll
    for (int i = 0; i < MAXI; ++i) {
      const int it = threadIdx.x + i * kThreads;
      if (it < ITEMS) {
        const int k1 = it / NCOL, c = it - k1 * NCOL;
#pragma unroll
        for (int j = 0; j < R2; ++j) u[i][j] = buf[(k1 * R2 + j) * NP + c];
        Dft<T, R2, -1>::run(u[i]);
      }
    }
    __syncthreads();
#pragma unroll
    for (int i = 0; i < MAXI; ++i) {
      const int it = threadIdx.x + i * kThreads;
      if (it < ITEMS) {
        const int k1 = it / NCOL, c = it - k1 * NCOL;
#pragma unroll
        for (int k2 = 0; k2 < R2; ++k2) buf[(k1 + R1 * k2) * NP + c] = u[i][k2];
      }
    }
  }
  __syncthreads();
  for (int e = threadIdx.x; e < N * TX; e += blockDim.x) {
    const int z = e / TX, t = e - z * TX;
    if (t < nm) update_mode<T, FORM>(buf + z * NP + t, TX, m0 + t, y, z, sh, P);
  }
  __syncthreads();
  // inverse pass 1 in place on the output slots
  for (int it = threadIdx.x; it < FOUT * TX * R2; it += blockDim.x) {
    const int n2 = it / (FOUT * TX), c = it - n2 * (FOUT * TX);
    cx<T>* p = buf + n2 * NP + c;
    cx<T> v[R1];
#pragma unroll
    for (int j = 0; j < R1; ++j) v[j] = p[j * R2 * NP];
    Dft<T, R1, 1>::run(v);
    if (n2) {
#pragma unroll
      for (int k = 1; k < R1; ++k) v[k] = cmulc(v[k], tw[n2 * k]);
    }
#pragma unroll
    for (int j = 0; j < R1; ++j) p[j * R2 * NP] = v[j];
  }
  __syncthreads();
  // inverse pass 2 straight to HBM
  for (int it = threadIdx.x; it < FOUT * TX * R1; it += blockDim.x) {
    const int k1 = it / (FOUT * TX), c = it - k1 * (FOUT * TX);
    const int s = c / TX, t = c - s * TX;
    if (t >= nm) continue;
    cx<T> u[R2];
#pragma unroll
    for (int j = 0; j < R2; ++j) u[j] = buf[(k1 * R2 + j) * NP + c];
    Dft<T, R2, 1>::run(u);
    cx<T>* p = g + s * sstride + t;
#pragma unroll
    for (int k2 = 0; k2 < R2; ++k2) p[(k1 + R1 * k2) * zst] = u[k2];
  }
}

template <typename T, int FORM, int TX>
__global__ void __launch_bounds__(kThreads, 2) k_z_fast(DevPlan P, cx<T>* spec, int64_t sstride,
                                                        const ColJob* __restrict__ jobs) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  cx<T>* buf = reinterpret_cast<cx<T>*>(smem_raw);
  const ColJob J = jobs[blockIdx.x];
  const BoxDev bx = P.boxes[J.box];
  const ShapeDev& sh = P.shapes[bx.shape];
  const int hx = sh.hx, n1 = bx.n[1];
  const int64_t zst = (int64_t)n1 * hx;
  cx<T>* g = spec + bx.soff + (int64_t)J.plane * hx + J.m0;
  switch (sh.fz) {
#define PSATD_ARM(code, N, R1, R2) \
  case code: z_body<T, FORM, TX, R1, R2>(buf, g, sstride, zst, J.nm, J.m0, J.plane, sh, P); break;
    PSATD_FAST_LENGTHS(PSATD_ARM)
#undef PSATD_ARM
    default: break;
  }
}

}  // namespace

// ---------------------------------------------------------------------------
// launchers
// ---------------------------------------------------------------------------
constexpr int kPlaneThreads = 512;

int fast_tile(int prec) { return prec == 32 ? 8 : 4; }

cudaError_t launch_plane_fwd(int prec, const DevPlan& P, const FieldPtrs& f, int nf, void* spec,
                             int64_t sstride, const int2* jobs, int64_t njobs, int smem, cudaStream_t st) {
  if (njobs <= 0 || nf <= 0) return cudaSuccess;
  dim3 grid((unsigned)njobs, nf);
  if (prec == 32)
    k_plane_fwd<float><<<grid, kPlaneThreads, smem, st>>>(P, f, (float2*)spec, sstride, jobs);
  else
    k_plane_fwd<double><<<grid, kPlaneThreads, smem, st>>>(P, f, (double2*)spec, sstride, jobs);
  return cudaGetLastError();
}

cudaError_t launch_plane_inv(int prec, const DevPlan& P, const FieldPtrs& f, int nf, void* spec,
                             int64_t sstride, const int2* jobs, int64_t njobs, int smem, cudaStream_t st) {
  if (njobs <= 0 || nf <= 0) return cudaSuccess;
  dim3 grid((unsigned)njobs, nf);
  if (prec == 32)
    k_plane_inv<float><<<grid, kPlaneThreads, smem, st>>>(P, f, (const float2*)spec, sstride, jobs);
  else
    k_plane_inv<double><<<grid, kPlaneThreads, smem, st>>>(P, f, (const double2*)spec, sstride, jobs);
  return cudaGetLastError();
}

cudaError_t launch_z_fast(int prec, int form, const DevPlan& P, void* spec, int64_t sstride,
                          const ColJob* jobs, int64_t njobs, int smem, cudaStream_t st) {
  if (njobs <= 0) return cudaSuccess;
  dim3 grid((unsigned)njobs);
#define PSATD_ZF(T, C2, FORMV, TXV) \
  k_z_fast<T, FORMV, TXV><<<grid, kThreads, smem, st>>>(P, (C2*)spec, sstride, jobs)
  if (prec == 32) {
    if (form == kVacuum) PSATD_ZF(float, float2, kVacuum, 8);
    else if (form == kJForm) PSATD_ZF(float, float2, kJForm, 8);
    else PSATD_ZF(float, float2, kRhoForm, 8);
  } else {
    if (form == kVacuum) PSATD_ZF(double, double2, kVacuum, 4);
    else if (form == kJForm) PSATD_ZF(double, double2, kJForm, 4);
    else PSATD_ZF(double, double2, kRhoForm, 4);
  }
#undef PSATD_ZF
  return cudaGetLastError();
}

int z_fast_smem(int prec, int form, int n2) {
  const int tx = fast_tile(prec);
  const int ncol = fields_in(form) * tx;
  const int np = ncol + ((24 - ncol % 16) % 16);
  return n2 * np * (prec == 32 ? 8 : 16);
}

cudaError_t configure_fast_kernels(int prec, int smem) {
  cudaError_t e = cudaSuccess;
#define PSATD_SET(K)                                                                            \
  do {                                                                                          \
    cudaError_t r = cudaFuncSetAttribute(K, cudaFuncAttributeMaxDynamicSharedMemorySize, smem); \
    if (r != cudaSuccess) e = r;                                                                \
  } while (0)
  if (prec == 32) {
    PSATD_SET(k_plane_fwd<float>);
    PSATD_SET(k_plane_inv<float>);
    PSATD_SET((k_z_fast<float, kVacuum, 8>));
    PSATD_SET((k_z_fast<float, kJForm, 8>));
    PSATD_SET((k_z_fast<float, kRhoForm, 8>));
  } else {
    PSATD_SET(k_plane_fwd<double>);
    PSATD_SET(k_plane_inv<double>);
    PSATD_SET((k_z_fast<double, kVacuum, 4>));
    PSATD_SET((k_z_fast<double, kJForm, 4>));
    PSATD_SET((k_z_fast<double, kRhoForm, 4>));
  }
#undef PSATD_SET
  return e;
}

}  // namespace psatd
