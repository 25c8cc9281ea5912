// Fast path of the PSATD push for box sizes whose FFT lengths factor as
// N = R1 * R2 with both factors in the register codelet set (list in
// psatd_internal.h, PSATD_FAST_LENGTHS).  Three kernels per step:
//
//   k_plane_fwd   (box, field, z) planes: real rows -> R2C along x -> complex
//                 FFT along y -> half-spectrum plane in HBM.
//   k_z_fast      (box, y, mx tile): z FFT of every field slot, loaded
//                 straight from HBM into registers; k-space update; inverse z
//                 FFT of the output slots, stored straight to HBM.
//   k_plane_inv   (box, field, interior z) planes: inverse y FFT -> C2R along
//                 x for interior rows -> interior cells to HBM.
//
// Every 1D FFT is a two-pass ("four-step") transform (fft_passes.cuh).
//
// The plane kernels are persistent: each CTA walks the plane list with a
// stride of gridDim.x and loads plane i+1 into its second shared-memory
// buffer with cp.async while it transforms plane i.
#include <cuda_runtime.h>

#include <cstdint>
#include <type_traits>

#include "fft_codelets.cuh"
#include "fft_passes.cuh"
#include "psatd_internal.h"
#include "psatd_update.cuh"

namespace psatd {

namespace {

constexpr int kPlaneThreads = 512;
constexpr int kTileF32 = 8;          // mx columns per z tile (FP32 / FP64)
constexpr int kTileF64 = 4;
constexpr int kMaxPlaneRows = 128;   // largest n1 of a fast box

// Longest x half-length L = n0/2 the plane kernels take (their in-place x
// pass keeps L/4 complex values per thread in registers).
template <typename T>
constexpr int max_plane_x() {
  return sizeof(T) == 4 ? 64 : 48;
}

// pass 2 along rows (ns = 1), in place: every thread first loads and
// transforms its items (at most MAXI), then all store in natural order.
template <typename T, int R1, int R2, int DIR>
__device__ __forceinline__ void pass2_rows_inplace(cx<T>* buf, int nrows, int pitch) {
  constexpr int MAXI = (kMaxPlaneRows * R1 + kPlaneThreads - 1) / kPlaneThreads;
  const int items = nrows * R1;
  cx<T> u[MAXI][R2];
#pragma unroll
  for (int i = 0; i < MAXI; ++i) {
    const int it = threadIdx.x + i * kPlaneThreads;
    if (it < items) {
      const int c = it / R1, k1 = it - c * R1;
      const cx<T>* p = buf + c * pitch + k1 * R2;
#pragma unroll
      for (int j = 0; j < R2; ++j) u[i][j] = p[j];
      Dft<T, R2, DIR>::run(u[i]);
    }
  }
  __syncthreads();
#pragma unroll
  for (int i = 0; i < MAXI; ++i) {
    const int it = threadIdx.x + i * kPlaneThreads;
    if (it < items) {
      const int c = it / R1, k1 = it - c * R1;
      cx<T>* p = buf + c * pitch + k1;
#pragma unroll
      for (int k2 = 0; k2 < R2; ++k2) p[R1 * k2] = u[i][k2];
    }
  }
}

// ---------------------------------------------------------------------------
// forward plane: x (R2C) then y, in place in one buffer of pitch lp >= hx
// ---------------------------------------------------------------------------
template <typename T, int R1, int R2>
__device__ __forceinline__ void plane_x_fwd(cx<T>* buf, int n1, int lp, const cx<T>* __restrict__ twx,
                                            const cx<T>* __restrict__ post) {
  constexpr int L = R1 * R2;
  pass1<T, R1, R2, -1, false>(buf, n1, lp, 1, twx, 0u);
  __syncthreads();
  pass2_rows_inplace<T, R1, R2, -1>(buf, n1, lp);
  __syncthreads();
  // R2C split in place, one thread per pair (k, L-k):
  // X[k] = (Z[k] + conj Z[L-k])/2 - i w^k (Z[k] - conj Z[L-k])/2
  constexpr int H = L / 2 + 1;
  for (int e = threadIdx.x; e < n1 * H; e += blockDim.x) {
    const int y = e / H, k = e - y * H;
    cx<T>* row = buf + y * lp;
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
      // partner: A' = conj A, Bv' = conj Bv
      if (2 * k != L) row[L - k] = conjg(A) + cmul(post[L - k], conjg(Bv));
    }
  }
}

template <typename T, int R1, int R2>
__device__ __forceinline__ void plane_y_fwd(cx<T>* buf, int hx, int lp, cx<T>* out,
                                            const cx<T>* __restrict__ twy) {
  const unsigned inv = magic(hx);
  pass1<T, R1, R2, -1, true>(buf, hx, 1, lp, twy, inv);
  __syncthreads();
  pass2<T, R1, R2, -1, true>(buf, hx, 1, lp, inv,
                             [&](int c, int k, cx<T> v) { out[k * hx + c] = v; });
}

template <typename T>
__device__ __forceinline__ void fwd_issue(const DevPlan& P, const FieldPtrs& F, const int2* jobs, int nplanes,
                                          int j, cx<T>* buf) {
  const int f = j / nplanes;
  const int2 J = jobs[j - f * nplanes];
  const BoxDev bx = P.boxes[J.x];
  const ShapeDev& sh = P.shapes[bx.shape];
  const int n0 = bx.n[0], n1 = bx.n[1];
  const T* g = reinterpret_cast<const T*>(F.p[f]) + bx.foff + (int64_t)J.y * n1 * n0;
  load_rows_async(buf, g, n1, n0 * (int)sizeof(T), sh.lp * (int)sizeof(cx<T>));
}

template <typename T>
__global__ void __launch_bounds__(kPlaneThreads, sizeof(T) == 4 ? 2 : 1)
    k_plane_fwd(DevPlan P, FieldPtrs F, cx<T>* spec, int64_t sstride, const int2* __restrict__ jobs,
                int nplanes, int nf, int bufsz) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  cx<T>* bufs = reinterpret_cast<cx<T>*>(smem_raw);
  const int total = nplanes * nf;
  int j = blockIdx.x;
  if (j >= total) return;
  int cur = 0;
  fwd_issue<T>(P, F, jobs, nplanes, j, bufs);
  cp_commit();
  for (; j < total; j += gridDim.x) {
    const int jn = j + gridDim.x;
    if (jn < total) fwd_issue<T>(P, F, jobs, nplanes, jn, bufs + (cur ^ 1) * bufsz);
    cp_commit();
    cp_wait_prev();
    __syncthreads();
    cx<T>* buf = bufs + cur * bufsz;
    const int f = j / nplanes;
    const int2 J = jobs[j - f * nplanes];
    const BoxDev bx = P.boxes[J.x];
    const ShapeDev& sh = P.shapes[bx.shape];
    const int n1 = bx.n[1], hx = sh.hx, lp = sh.lp;
    const cx<T>* twx = ctab<T>(P) + sh.ax.tw;
    const cx<T>* post = ctab<T>(P) + sh.post;
    switch (sh.fx) {
#define PSATD_ARM(code, N, R1, R2)                                   \
  case code:                                                         \
    if constexpr (N <= max_plane_x<T>()) plane_x_fwd<T, R1, R2>(buf, n1, lp, twx, post); \
    break;
      PSATD_FAST_LENGTHS(PSATD_ARM)
#undef PSATD_ARM
      default: break;
    }
    __syncthreads();
    cx<T>* out = spec + f * sstride + bx.soff + (int64_t)J.y * n1 * hx;
    const cx<T>* twy = ctab<T>(P) + sh.ay.tw;
    switch (sh.fy) {
#define PSATD_ARM(code, N, R1, R2) \
  case code: plane_y_fwd<T, R1, R2>(buf, hx, lp, out, twy); break;
      PSATD_FAST_LENGTHS(PSATD_ARM)
#undef PSATD_ARM
      default: break;
    }
    __syncthreads();
    cur ^= 1;
  }
}

// ---------------------------------------------------------------------------
// inverse plane: y then C2R along x, interior rows and cells only.  The
// spectrum plane is copied as is (pitch hx); interior rows go to a second
// buffer of pitch hp.
// ---------------------------------------------------------------------------
template <typename T, int R1, int R2>
__device__ __forceinline__ void plane_y_inv(cx<T>* buf, int hx, cx<T>* rows, int hp, int ylo, int yhi,
                                            const cx<T>* __restrict__ twy) {
  const unsigned inv = magic(hx);
  pass1<T, R1, R2, 1, true>(buf, hx, 1, hx, twy, inv);
  __syncthreads();
  pass2<T, R1, R2, 1, true>(buf, hx, 1, hx, inv, [&](int c, int k, cx<T> v) {
    if (k >= ylo && k < yhi) rows[(k - ylo) * hp + c] = v;
  });
}

template <typename T, int R1, int R2>
__device__ __forceinline__ void plane_x_inv(cx<T>* rows, int nrows, int hp, T* ibuf, int nxi, int xlo,
                                            T scale, const cx<T>* __restrict__ twx,
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
    if (k != 0 && 2 * k != L) row[L - k] = (b + conjg(a)) + times_i(cmulc(b - conjg(a), post[L - k]));
    row[k] = za;
  }
  __syncthreads();
  pass1<T, R1, R2, 1, false>(rows, nrows, hp, 1, twx, 0u);
  __syncthreads();
  // interior cells of the interior rows -> ibuf (row pitch nxi)
  pass2<T, R1, R2, 1, false>(rows, nrows, hp, 1, 0u, [&](int r, int m, cx<T> v) {
    T* o = ibuf + r * nxi - xlo + 2 * m;
    if (2 * m >= xlo && 2 * m < xlo + nxi) o[0] = scale * v.x;
    if (2 * m + 1 >= xlo && 2 * m + 1 < xlo + nxi) o[1] = scale * v.y;
  });
}

// Copy ny rows of nx elements from shared memory (pitch spitch) to global
// memory (pitch dpitch), in units of V elements, by `nthreads` threads
// numbered `tid`.
template <typename T, int V>
__device__ __forceinline__ void copy_rect(const T* src, int spitch, T* dst, int64_t dpitch, int ny, int nx,
                                          int tid, int nthreads) {
  using Vec = typename std::conditional<V == 1, T, float4>::type;
  const int upr = nx / V;
  const unsigned m = magic(upr);
  for (int u = tid; u < ny * upr; u += nthreads) {
    const int r = fdiv(u, m), c = (u - r * upr) * V;
    *reinterpret_cast<Vec*>(dst + r * dpitch + c) = *reinterpret_cast<const Vec*>(src + r * spitch + c);
  }
}

template <typename T>
__device__ __forceinline__ void inv_issue(const DevPlan& P, const cx<T>* spec, int64_t sstride,
                                          const int2* jobs, int nplanes, int j, cx<T>* buf) {
  const int f = j / nplanes;
  const int2 J = jobs[j - f * nplanes];
  const BoxDev bx = P.boxes[J.x];
  const ShapeDev& sh = P.shapes[bx.shape];
  const int n1 = bx.n[1], hx = sh.hx;
  const cx<T>* g = spec + f * sstride + bx.soff + (int64_t)J.y * n1 * hx;
  const int bytes = n1 * hx * (int)sizeof(cx<T>);
  load_rows_async(buf, g, 1, bytes, bytes);
}

template <typename T>
__global__ void __launch_bounds__(kPlaneThreads, sizeof(T) == 4 ? 2 : 1)
    k_plane_inv(DevPlan P, FieldPtrs F, const cx<T>* spec, int64_t sstride, const int2* __restrict__ jobs,
                int nplanes, int nf, int bufsz, const int* __restrict__ seg_start,
                const GuardSeg* __restrict__ segs) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  cx<T>* bufs = reinterpret_cast<cx<T>*>(smem_raw);
  cx<T>* rows = bufs + 2 * bufsz;
  const int total = nplanes * nf;
  int j = blockIdx.x;
  if (j >= total) return;
  int cur = 0;
  inv_issue<T>(P, spec, sstride, jobs, nplanes, j, bufs);
  cp_commit();
  for (; j < total; j += gridDim.x) {
    const int jn = j + gridDim.x;
    if (jn < total) inv_issue<T>(P, spec, sstride, jobs, nplanes, jn, bufs + (cur ^ 1) * bufsz);
    cp_commit();
    cp_wait_prev();
    __syncthreads();
    cx<T>* buf = bufs + cur * bufsz;
    const int f = j / nplanes;
    const int2 J = jobs[j - f * nplanes];
    const BoxDev bx = P.boxes[J.x];
    const ShapeDev& sh = P.shapes[bx.shape];
    const int n0 = bx.n[0], n1 = bx.n[1], hx = sh.hx, hp = sh.hp;
    const int ylo = bx.ng_lo[1], yhi = n1 - bx.ng_hi[1];
    const cx<T>* twy = ctab<T>(P) + sh.ay.tw;
    switch (sh.fy) {
#define PSATD_ARM(code, N, R1, R2) \
  case code: plane_y_inv<T, R1, R2>(buf, hx, rows, hp, ylo, yhi, twy); break;
      PSATD_FAST_LENGTHS(PSATD_ARM)
#undef PSATD_ARM
      default: break;
    }
    __syncthreads();
    const T scale = T(1.0 / ((double)n0 * n1 * bx.n[2]));
    const int xlo = bx.ng_lo[0], nxi = n0 - bx.ng_lo[0] - bx.ng_hi[0], ni = yhi - ylo;
    T* ibuf = reinterpret_cast<T*>(buf);   // the spectrum plane is no longer needed
    const cx<T>* twx = ctab<T>(P) + sh.ax.tw;
    const cx<T>* post = ctab<T>(P) + sh.post;
    switch (sh.fx) {
#define PSATD_ARM(code, N, R1, R2)                                                       \
  case code:                                                                             \
    if constexpr (N <= max_plane_x<T>())                                                 \
      plane_x_inv<T, R1, R2>(rows, ni, hp, ibuf, nxi, xlo, scale, twx, post);            \
    break;
      PSATD_FAST_LENGTHS(PSATD_ARM)
#undef PSATD_ARM
      default: break;
    }
    __syncthreads();
    // interior cells to this box
    T* fbase = reinterpret_cast<T*>(F.p[f]);
    T* own = fbase + bx.foff + ((int64_t)J.y * n1 + ylo) * n0 + xlo;
    constexpr int V16 = 16 / sizeof(T);
    if (nxi % V16 == 0 && xlo % V16 == 0 && n0 % V16 == 0)
      copy_rect<T, V16>(ibuf, nxi, own, n0, ni, nxi, threadIdx.x, blockDim.x);
    else
      copy_rect<T, 1>(ibuf, nxi, own, n0, ni, nxi, threadIdx.x, blockDim.x);
    // guard cells fed by this plane (fused exchange), one rectangle per warp
    if (seg_start) {
      const int p = j - f * nplanes;
      const int s1 = seg_start[p + 1];
      const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
      for (int si = seg_start[p] + warp; si < s1; si += nw) {
        const GuardSeg g = segs[si];
        const BoxDev db = P.boxes[g.dst_box];
        T* dst = fbase + db.foff + ((int64_t)g.dst_z * db.n[1] + g.dy) * db.n[0] + g.dx;
        const T* src = ibuf + (g.sy - ylo) * nxi + (g.sx - xlo);
        if (g.vec > 1)
          copy_rect<T, V16>(src, nxi, dst, db.n[0], g.ny, g.nx, lane, 32);
        else
          copy_rect<T, 1>(src, nxi, dst, db.n[0], g.ny, g.nx, lane, 32);
      }
    }
    __syncthreads();
    cur ^= 1;
  }
}

template <typename T, int FORM, int TX>
__global__ void __launch_bounds__(kThreads, 2) k_z_fast(DevPlan P, cx<T>* spec, int64_t sstride,
                                                        const ColJob* __restrict__ jobs, int nft) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  cx<T>* buf = reinterpret_cast<cx<T>*>(smem_raw);
  const ColJob J = jobs[blockIdx.x];
  const BoxDev bx = P.boxes[J.box];
  const ShapeDev& sh = P.shapes[bx.shape];
  const int hx = sh.hx, n1 = bx.n[1];
  const int64_t zst = (int64_t)n1 * hx;
  const bool nyq = J.nm < 0;
  const int nm = nyq ? -J.nm : J.nm, ts = nyq ? hx : 1;
  cx<T>* g = spec + bx.soff + (int64_t)J.plane * hx + J.m0;
  switch (sh.fz) {
#define PSATD_ARM(code, N, R1, R2) \
  case code:                                                                                     \
    z_body<T, FORM, TX, R1, R2>(buf, g, sstride, zst, nm, J.m0, J.plane, ts, nyq, bx.ng_lo[2], N - bx.ng_hi[2], nft, \
                                sh, P);                                                                              \
    break;
    PSATD_FAST_LENGTHS(PSATD_ARM)
#undef PSATD_ARM
    default: break;
  }
}



}  // namespace

// ---------------------------------------------------------------------------
// launchers
// ---------------------------------------------------------------------------
int fast_tile(int prec) { return prec == 32 ? kTileF32 : kTileF64; }
int fast_max_x(int prec) { return prec == 32 ? max_plane_x<float>() : max_plane_x<double>(); }
int plane_threads() { return kPlaneThreads; }

cudaError_t launch_plane_fwd(int prec, const DevPlan& P, const FieldPtrs& f, int nf, void* spec,
                             int64_t sstride, const int2* jobs, int64_t nplanes, int bufsz, int smem,
                             int grid, cudaStream_t st) {
  if (nplanes <= 0 || nf <= 0) return cudaSuccess;
  if (prec == 32)
    k_plane_fwd<float><<<grid, kPlaneThreads, smem, st>>>(P, f, (float2*)spec, sstride, jobs, (int)nplanes, nf,
                                                          bufsz);
  else
    k_plane_fwd<double><<<grid, kPlaneThreads, smem, st>>>(P, f, (double2*)spec, sstride, jobs, (int)nplanes,
                                                           nf, bufsz);
  return cudaGetLastError();
}

cudaError_t launch_plane_inv(int prec, const DevPlan& P, const FieldPtrs& f, int nf, void* spec,
                             int64_t sstride, const int2* jobs, int64_t nplanes, int bufsz, int smem,
                             int grid, const int* seg_start, const GuardSeg* segs, cudaStream_t st) {
  if (nplanes <= 0 || nf <= 0) return cudaSuccess;
  if (prec == 32)
    k_plane_inv<float><<<grid, kPlaneThreads, smem, st>>>(P, f, (const float2*)spec, sstride, jobs,
                                                          (int)nplanes, nf, bufsz, seg_start, segs);
  else
    k_plane_inv<double><<<grid, kPlaneThreads, smem, st>>>(P, f, (const double2*)spec, sstride, jobs,
                                                           (int)nplanes, nf, bufsz, seg_start, segs);
  return cudaGetLastError();
}

cudaError_t plane_occupancy(int prec, int smem_fwd, int smem_inv, int* fwd_per_sm, int* inv_per_sm) {
  cudaError_t e;
  if (prec == 32) {
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(fwd_per_sm, k_plane_fwd<float>, kPlaneThreads, smem_fwd);
    if (e == cudaSuccess)
      e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(inv_per_sm, k_plane_inv<float>, kPlaneThreads, smem_inv);
  } else {
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(fwd_per_sm, k_plane_fwd<double>, kPlaneThreads, smem_fwd);
    if (e == cudaSuccess)
      e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(inv_per_sm, k_plane_inv<double>, kPlaneThreads, smem_inv);
  }
  return e;
}

cudaError_t launch_z_fast(int prec, int form, const DevPlan& P, void* spec, int64_t sstride,
                          const ColJob* jobs, int64_t njobs, int smem, int nft, cudaStream_t st) {
  if (njobs <= 0) return cudaSuccess;
  dim3 grid((unsigned)njobs);
#define PSATD_ZF(T, C2, FORMV, TXV) \
  k_z_fast<T, FORMV, TXV><<<grid, kThreads, smem, st>>>(P, (C2*)spec, sstride, jobs, nft)
  if (prec == 32) {
    if (form == kVacuum) PSATD_ZF(float, float2, kVacuum, kTileF32);
    else if (form == kJForm) PSATD_ZF(float, float2, kJForm, kTileF32);
    else PSATD_ZF(float, float2, kRhoForm, kTileF32);
  } else {
    if (form == kVacuum) PSATD_ZF(double, double2, kVacuum, kTileF64);
    else if (form == kJForm) PSATD_ZF(double, double2, kJForm, kTileF64);
    else PSATD_ZF(double, double2, kRhoForm, kTileF64);
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
    PSATD_SET((k_z_fast<float, kVacuum, kTileF32>));
    PSATD_SET((k_z_fast<float, kJForm, kTileF32>));
    PSATD_SET((k_z_fast<float, kRhoForm, kTileF32>));
  } else {
    PSATD_SET(k_plane_fwd<double>);
    PSATD_SET(k_plane_inv<double>);
    PSATD_SET((k_z_fast<double, kVacuum, kTileF64>));
    PSATD_SET((k_z_fast<double, kJForm, kTileF64>));
    PSATD_SET((k_z_fast<double, kRhoForm, kTileF64>));
  }
#undef PSATD_SET
  return e;
}

}  // namespace psatd
