// Pencil path of the PSATD push for boxes whose FFT lengths are two-pass
// lengths (PSATD_PENCIL_LENGTHS, up to 512) but whose planes do not fit the
// plane kernels (n0/2 or n1 above their limits): one kernel per axis pass.
//
//   k_pen_xf   (box, rows, field): real rows -> R2C along x -> half-spectrum
//              rows in HBM (S1, x).
//   k_pen_col  (box, z plane, mx tile, field): complex FFT along y of a tile
//              of consecutive mx columns, in place in HBM (S1 y forward; S3 y
//              inverse on the interior z planes).
//   k_z_pen    (box, y, mx tile): z FFT + k-space update + inverse z FFT of
//              all field slots (S1 z, S2, S3 z), interior z planes stored.
//   k_pen_xi   (box, interior rows, field): C2R along x with 1/N, interior
//              cells to HBM (S3, x).
//
// Every kernel is instantiated per FFT length (its registers and occupancy
// follow that length); the plan groups the jobs of each length and issues
// one launch per group.  The guard exchange (S4) of these boxes is the
// batched copy kernel.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>

#include "fft_codelets.cuh"
#include "fft_passes.cuh"
#include "psatd_internal.h"
#include "psatd_update.cuh"

namespace psatd {

namespace {

constexpr int kPenThreads = 256;
constexpr int kGatherRows = 64;   // row descriptors of the deferred-exchange gather per chunk
constexpr int kPenMaxi = 2;   // rows * R1 <= kPenMaxi * kPenThreads for the x passes

template <typename T>
constexpr int pen_tile() {   // mx columns of a y tile: 128-byte rows
  return sizeof(T) == 4 ? 16 : 8;
}

// longest z length of the pencil z kernel (its pass 2 keeps a few length-R2
// transforms per thread in registers)
template <typename T>
constexpr int pen_max_z() {
  return sizeof(T) == 4 ? 256 : 128;
}

// x row pitch (complex) of the pencil x kernels: >= L + 1, even (16-byte rows)
__host__ __device__ constexpr int pen_x_pitch(int L) { return L + 2; }

// pass 2 along rows (ns = 1), in place: every thread loads and transforms
// its items (at most kPenMaxi), a barrier, then all store in natural order.
template <typename T, int R1, int R2, int DIR>
__device__ __forceinline__ void pen_rows_pass2(cx<T>* buf, int nrows, int pitch) {
  const int items = nrows * R1;
  cx<T> u[kPenMaxi][R2];
#pragma unroll
  for (int i = 0; i < kPenMaxi; ++i) {
    const int it = threadIdx.x + i * kPenThreads;
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
  for (int i = 0; i < kPenMaxi; ++i) {
    const int it = threadIdx.x + i * kPenThreads;
    if (it < items) {
      const int c = it / R1, k1 = it - c * R1;
      cx<T>* p = buf + c * pitch + k1;
#pragma unroll
      for (int k2 = 0; k2 < R2; ++k2) p[R1 * k2] = u[i][k2];
    }
  }
}

// ---------------------------------------------------------------------------
template <typename T, int R1, int R2>
__device__ __forceinline__ void pen_xf_body(cx<T>* buf, int nr, const cx<T>* __restrict__ twx,
                                            const cx<T>* __restrict__ post) {
  constexpr int L = R1 * R2, H = L / 2 + 1, LP = pen_x_pitch(L);
  pass1<T, R1, R2, -1, false>(buf, nr, LP, 1, twx, 0u);
  __syncthreads();
  pen_rows_pass2<T, R1, R2, -1>(buf, nr, LP);
  __syncthreads();
  // R2C split in place, one thread per pair (k, L-k):
  // X[k] = (Z[k] + conj Z[L-k])/2 - i w^k (Z[k] - conj Z[L-k])/2, w = exp(-2 pi i / n0)
  for (int e = threadIdx.x; e < nr * H; e += kPenThreads) {
    const int y = e / H, k = e - y * H;
    cx<T>* row = buf + y * LP;
    const cx<T> a = row[k];
    const cx<T> b = row[k == 0 ? 0 : L - k];
    const cx<T> A = mk<T>(T(0.5) * (a.x + b.x), T(0.5) * (a.y - b.y));
    const cx<T> Bv = mk<T>(T(0.5) * (a.y + b.y), T(0.5) * (b.x - a.x));
    if (k == 0) {
      row[0] = mk<T>(A.x + Bv.x, A.y + Bv.y);
      row[L] = mk<T>(A.x - Bv.x, A.y - Bv.y);
    } else {
      row[k] = A + cmul(post[k], Bv);
      if (2 * k != L) row[L - k] = conjg(A) + cmul(post[L - k], conjg(Bv));
    }
  }
}

template <typename T, int R1, int R2>
__global__ void __launch_bounds__(kPenThreads) k_pen_xf(DevPlan P, FieldPtrs F, cx<T>* spec, int64_t sstride,
                                                        const RowJob* __restrict__ jobs,
                                                        const GatherGrid* __restrict__ ggrid, int ngather) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  cx<T>* buf = reinterpret_cast<cx<T>*>(smem_raw);
  const RowJob J = jobs[blockIdx.x];
  const int f = blockIdx.y;
  const BoxDev bx = P.boxes[J.box];
  const ShapeDev& sh = P.shapes[bx.shape];
  const int n0 = bx.n[0], L = sh.L, hx = sh.hx, LP = pen_x_pitch(L);
  if (ggrid && f < ngather) {
    // deferred exchange: the three x bands of each row from the cells that
    // own them (gather grid of the row's plane); row descriptors in chunks
    constexpr int VE = 16 / (int)sizeof(T);   // elements per 16-byte unit
    __shared__ int64_t rsrc[kGatherRows][3];
    __shared__ int rx[kGatherRows][2];
    const T* fb = reinterpret_cast<const T*>(F.p[f]);
    const int n1 = bx.n[1], upr = n0 / VE;
    const unsigned mu = magic(upr);
    for (int rb = 0; rb < J.nr; rb += kGatherRows) {
      const int nrb = min(kGatherRows, J.nr - rb);
      if (threadIdx.x < nrb) {
        const int r = J.r0 + rb + threadIdx.x;
        const int z = r / n1, y = r - z * n1;
        const GatherGrid& G = ggrid[bx.gplane + z];
        const int iy = (y >= G.y1) + (y >= G.y2);
        const int dy = y - (iy == 0 ? 0 : iy == 1 ? G.y1 : G.y2);
        // element x of band ix is at rsrc[ix] + x
        rsrc[threadIdx.x][0] = G.base[3 * iy] + (int64_t)dy * G.pitch[3 * iy];
        rsrc[threadIdx.x][1] = G.base[3 * iy + 1] + (int64_t)dy * G.pitch[3 * iy + 1] - G.x1;
        rsrc[threadIdx.x][2] = G.base[3 * iy + 2] + (int64_t)dy * G.pitch[3 * iy + 2] - G.x2;
        rx[threadIdx.x][0] = G.x1;
        rx[threadIdx.x][1] = G.x2;
      }
      __syncthreads();
      for (int u = threadIdx.x; u < nrb * upr; u += kPenThreads) {
        const int i = fdiv(u, mu), x = (u - i * upr) * VE;
        const int ix = (x >= rx[i][0]) + (x >= rx[i][1]);
        cp16(reinterpret_cast<char*>(buf) + (size_t)(rb + i) * LP * sizeof(cx<T>) + (size_t)x * sizeof(T),
             fb + rsrc[i][ix] + x);
      }
      __syncthreads();   // the descriptors of the next chunk overwrite these
    }
  } else {
    // rows r0 .. r0+nr-1 are contiguous in the field buffer
    const T* g = reinterpret_cast<const T*>(F.p[f]) + bx.foff + (int64_t)J.r0 * n0;
    load_rows_async(buf, g, J.nr, n0 * (int)sizeof(T), LP * (int)sizeof(cx<T>));
  }
  asm volatile("cp.async.commit_group;\ncp.async.wait_group 0;\n" ::: "memory");
  __syncthreads();
  pen_xf_body<T, R1, R2>(buf, J.nr, ctab<T>(P) + sh.ax.tw, ctab<T>(P) + sh.post);
  __syncthreads();
  // the nr half-spectrum rows are contiguous in the spectrum slot
  cx<T>* out = spec + f * sstride + bx.soff + (int64_t)J.r0 * hx;
  for (int e = threadIdx.x; e < J.nr * hx; e += kPenThreads) {
    const int r = e / hx, k = e - r * hx;
    out[e] = buf[r * LP + k];
  }
}

// ---------------------------------------------------------------------------
// y pass of a tile: columns m0 .. m0+nm-1 of z plane `plane`, all n1 rows.
template <typename T, int DIR, int R1, int R2>
__global__ void __launch_bounds__(kPenThreads) k_pen_col(DevPlan P, cx<T>* spec, int64_t sstride,
                                                         const ColJob* __restrict__ jobs) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  cx<T>* buf = reinterpret_cast<cx<T>*>(smem_raw);   // [y][c], pitch nm
  const ColJob J = jobs[blockIdx.x];
  const int f = blockIdx.y;
  const BoxDev bx = P.boxes[J.box];
  const ShapeDev& sh = P.shapes[bx.shape];
  const int n1 = bx.n[1], hx = sh.hx, nm = J.nm;
  cx<T>* g = spec + f * sstride + bx.soff + (int64_t)J.plane * n1 * hx + J.m0;
  const unsigned mnm = magic(nm);
  for (int e = threadIdx.x; e < n1 * nm; e += kPenThreads) {
    const int y = fdiv(e, mnm), c = e - y * nm;
    buf[e] = g[(int64_t)y * hx + c];
  }
  __syncthreads();
  pass1<T, R1, R2, DIR, true>(buf, nm, 1, nm, ctab<T>(P) + sh.ay.tw, mnm);
  __syncthreads();
  pass2<T, R1, R2, DIR, true>(buf, nm, 1, nm, mnm, [&](int c, int k, cx<T> v) { g[(int64_t)k * hx + c] = v; });
}

// ---------------------------------------------------------------------------
template <typename T, int FORM, int TX, int R1, int R2>
__global__ void __launch_bounds__(kThreads, 1) k_z_pen(DevPlan P, cx<T>* spec, int64_t sstride,
                                                       const ColJob* __restrict__ jobs, int nft) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  cx<T>* buf = reinterpret_cast<cx<T>*>(smem_raw);
  const ColJob J = jobs[blockIdx.x];
  const BoxDev bx = P.boxes[J.box];
  const ShapeDev& sh = P.shapes[bx.shape];
  const int hx = sh.hx, n1 = bx.n[1], N = bx.n[2];
  const int64_t zst = (int64_t)n1 * hx;
  const bool nyq = J.nm < 0;
  const int nm = nyq ? -J.nm : J.nm, ts = nyq ? hx : 1;
  cx<T>* g = spec + bx.soff + (int64_t)J.plane * hx + J.m0;
  z_body<T, FORM, TX, R1, R2>(buf, g, sstride, zst, nm, J.m0, J.plane, ts, nyq, bx.ng_lo[2], N - bx.ng_hi[2], nft,
                              sh, P);
}

// ---------------------------------------------------------------------------
template <typename T, int R1, int R2>
__device__ __forceinline__ void pen_xi_body(cx<T>* buf, int nr, T* out, int n0, int xlo, int nxi, T scale,
                                            const cx<T>* __restrict__ twx, const cx<T>* __restrict__ post) {
  constexpr int L = R1 * R2, H = L / 2 + 1, LP = pen_x_pitch(L);
  // C2R merge in place, one thread per pair (k, L-k):
  // Z'[k] = (X[k] + conj X[L-k]) + i w^-k (X[k] - conj X[L-k])
  for (int e = threadIdx.x; e < nr * H; e += kPenThreads) {
    const int r = e / H, k = e - r * H;
    cx<T>* row = buf + r * LP;
    const cx<T> a = row[k];
    const cx<T> b = row[L - k];
    const cx<T> za = (a + conjg(b)) + times_i(cmulc(a - conjg(b), post[k]));
    if (k != 0 && 2 * k != L) row[L - k] = (b + conjg(a)) + times_i(cmulc(b - conjg(a), post[L - k]));
    row[k] = za;
  }
  __syncthreads();
  pass1<T, R1, R2, 1, false>(buf, nr, LP, 1, twx, 0u);
  __syncthreads();
  // interior cells of each row straight to HBM
  pass2<T, R1, R2, 1, false>(buf, nr, LP, 1, 0u, [&](int r, int m, cx<T> v) {
    T* o = out + (int64_t)r * n0;
    const int x = 2 * m;
    if (x >= xlo && x < xlo + nxi) o[x] = scale * v.x;
    if (x + 1 >= xlo && x + 1 < xlo + nxi) o[x + 1] = scale * v.y;
  });
}

// rows r0 .. r0+nr-1 of one box (consecutive y of one z plane, all interior)
template <typename T, int R1, int R2>
__global__ void __launch_bounds__(kPenThreads) k_pen_xi(DevPlan P, FieldPtrs F, const cx<T>* spec,
                                                        int64_t sstride, const RowJob* __restrict__ jobs) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  cx<T>* buf = reinterpret_cast<cx<T>*>(smem_raw);
  const RowJob J = jobs[blockIdx.x];
  const int f = blockIdx.y;
  const BoxDev bx = P.boxes[J.box];
  const ShapeDev& sh = P.shapes[bx.shape];
  const int n0 = bx.n[0], L = sh.L, hx = sh.hx, LP = pen_x_pitch(L);
  const cx<T>* g = spec + f * sstride + bx.soff + (int64_t)J.r0 * hx;
  for (int e = threadIdx.x; e < J.nr * hx; e += kPenThreads) {
    const int r = e / hx, k = e - r * hx;
    buf[r * LP + k] = g[e];
  }
  __syncthreads();
  const T scale = T(1.0 / ((double)n0 * bx.n[1] * bx.n[2]));
  T* out = reinterpret_cast<T*>(F.p[f]) + bx.foff + (int64_t)J.r0 * n0;
  pen_xi_body<T, R1, R2>(buf, J.nr, out, n0, bx.ng_lo[0], n0 - bx.ng_lo[0] - bx.ng_hi[0], scale,
                         ctab<T>(P) + sh.ax.tw, ctab<T>(P) + sh.post);
}

}  // namespace

// ---------------------------------------------------------------------------
int pen_rows(int prec, int L, int rows, int smem_cap) {
  int r1 = 1;
#define PSATD_R1(code, N, R1, R2) \
  if (L == N) r1 = R1;
  PSATD_PENCIL_LENGTHS(PSATD_R1)
#undef PSATD_R1
  const int row_bytes = pen_x_pitch(L) * (prec == 32 ? 8 : 16);
  int nr = kPenMaxi * kPenThreads / r1;
  nr = std::min(nr, std::max(1, smem_cap / row_bytes));
  return std::max(1, std::min(nr, rows));
}
int pen_z_max(int prec) { return prec == 32 ? pen_max_z<float>() : pen_max_z<double>(); }
int pen_x_smem(int prec, int L, int nr) { return nr * pen_x_pitch(L) * (prec == 32 ? 8 : 16); }
int pen_col_tile(int prec) { return prec == 32 ? pen_tile<float>() : pen_tile<double>(); }
int pen_col_smem(int prec, int n1) { return n1 * pen_col_tile(prec) * (prec == 32 ? 8 : 16); }

// One launch per FFT-length group: `code` is the pencil-length code of the
// axis the kernel transforms (x for the row kernels, y for the column
// kernels, z for the z kernel); every job of the launch has that length.
cudaError_t launch_pen_xf(int prec, int code, const DevPlan& P, const FieldPtrs& f, int nf, void* spec,
                          int64_t sstride, const RowJob* jobs, int64_t njobs, int smem, const GatherGrid* ggrid,
                          int ngather, cudaStream_t st) {
  if (njobs <= 0 || nf <= 0) return cudaSuccess;
  dim3 grid((unsigned)njobs, nf);
  switch (code) {
#define PSATD_ARM(c, N, R1, R2)                                                                       \
  case c:                                                                                             \
    if (prec == 32)                                                                                   \
      k_pen_xf<float, R1, R2><<<grid, kPenThreads, smem, st>>>(P, f, (float2*)spec, sstride, jobs, ggrid, \
                                                               ngather);                              \
    else                                                                                              \
      k_pen_xf<double, R1, R2><<<grid, kPenThreads, smem, st>>>(P, f, (double2*)spec, sstride, jobs, ggrid, \
                                                                ngather);                             \
    break;
    PSATD_PENCIL_LENGTHS(PSATD_ARM)
#undef PSATD_ARM
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

cudaError_t launch_pen_col(int prec, int dir, int code, const DevPlan& P, void* spec, int64_t sstride, int nf,
                           const ColJob* jobs, int64_t njobs, int smem, cudaStream_t st) {
  if (njobs <= 0 || nf <= 0) return cudaSuccess;
  dim3 grid((unsigned)njobs, nf);
  switch (code) {
#define PSATD_ARM(c, N, R1, R2)                                                                        \
  case c:                                                                                              \
    if (prec == 32 && dir < 0)                                                                         \
      k_pen_col<float, -1, R1, R2><<<grid, kPenThreads, smem, st>>>(P, (float2*)spec, sstride, jobs);   \
    else if (prec == 32)                                                                               \
      k_pen_col<float, 1, R1, R2><<<grid, kPenThreads, smem, st>>>(P, (float2*)spec, sstride, jobs);    \
    else if (dir < 0)                                                                                  \
      k_pen_col<double, -1, R1, R2><<<grid, kPenThreads, smem, st>>>(P, (double2*)spec, sstride, jobs); \
    else                                                                                               \
      k_pen_col<double, 1, R1, R2><<<grid, kPenThreads, smem, st>>>(P, (double2*)spec, sstride, jobs);  \
    break;
    PSATD_PENCIL_LENGTHS(PSATD_ARM)
#undef PSATD_ARM
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

template <typename T, typename C2, int R1, int R2>
cudaError_t launch_z_pen_t(int form, const DevPlan& P, void* spec, int64_t sstride, const ColJob* jobs,
                           int64_t njobs, int smem, int nft, cudaStream_t st) {
  constexpr int TX = sizeof(T) == 4 ? 8 : 4;
  if constexpr (R1 * R2 <= pen_max_z<T>()) {
    dim3 grid((unsigned)njobs);
    if (form == kVacuum)
      k_z_pen<T, kVacuum, TX, R1, R2><<<grid, kThreads, smem, st>>>(P, (C2*)spec, sstride, jobs, nft);
    else if (form == kJForm)
      k_z_pen<T, kJForm, TX, R1, R2><<<grid, kThreads, smem, st>>>(P, (C2*)spec, sstride, jobs, nft);
    else
      k_z_pen<T, kRhoForm, TX, R1, R2><<<grid, kThreads, smem, st>>>(P, (C2*)spec, sstride, jobs, nft);
    return cudaGetLastError();
  } else {
    return cudaErrorInvalidValue;
  }
}

cudaError_t launch_z_pen(int prec, int form, int code, const DevPlan& P, void* spec, int64_t sstride,
                         const ColJob* jobs, int64_t njobs, int smem, int nft, cudaStream_t st) {
  if (njobs <= 0) return cudaSuccess;
  switch (code) {
#define PSATD_ARM(c, N, R1, R2)                                                                         \
  case c:                                                                                               \
    return prec == 32 ? launch_z_pen_t<float, float2, R1, R2>(form, P, spec, sstride, jobs, njobs, smem, nft, st) \
                      : launch_z_pen_t<double, double2, R1, R2>(form, P, spec, sstride, jobs, njobs, smem, nft, st);
    PSATD_PENCIL_LENGTHS(PSATD_ARM)
#undef PSATD_ARM
    default: return cudaErrorInvalidValue;
  }
}

cudaError_t launch_pen_xi(int prec, int code, const DevPlan& P, const FieldPtrs& f, int nf, void* spec,
                          int64_t sstride, const RowJob* jobs, int64_t njobs, int smem, cudaStream_t st) {
  if (njobs <= 0 || nf <= 0) return cudaSuccess;
  dim3 grid((unsigned)njobs, nf);
  switch (code) {
#define PSATD_ARM(c, N, R1, R2)                                                                              \
  case c:                                                                                                    \
    if (prec == 32)                                                                                          \
      k_pen_xi<float, R1, R2><<<grid, kPenThreads, smem, st>>>(P, f, (const float2*)spec, sstride, jobs);     \
    else                                                                                                     \
      k_pen_xi<double, R1, R2><<<grid, kPenThreads, smem, st>>>(P, f, (const double2*)spec, sstride, jobs);   \
    break;
    PSATD_PENCIL_LENGTHS(PSATD_ARM)
#undef PSATD_ARM
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

template <typename T, int R1, int R2>
cudaError_t configure_pen_t(int smem) {
  cudaError_t e = cudaSuccess;
  auto set = [&](const void* k) {   // the opt-in maximum less the kernel's static shared memory
    cudaFuncAttributes fa{};
    cudaError_t r = cudaFuncGetAttributes(&fa, k);
    if (r == cudaSuccess)
      r = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, smem - (int)fa.sharedSizeBytes);
    if (r != cudaSuccess) e = r;
  };
  constexpr int TX = sizeof(T) == 4 ? 8 : 4;
  set((const void*)k_pen_xf<T, R1, R2>);
  set((const void*)k_pen_xi<T, R1, R2>);
  set((const void*)k_pen_col<T, -1, R1, R2>);
  set((const void*)k_pen_col<T, 1, R1, R2>);
  if constexpr (R1 * R2 <= pen_max_z<T>()) {
    set((const void*)k_z_pen<T, kVacuum, TX, R1, R2>);
    set((const void*)k_z_pen<T, kJForm, TX, R1, R2>);
    set((const void*)k_z_pen<T, kRhoForm, TX, R1, R2>);
  }
  return e;
}

cudaError_t configure_pen_kernels(int prec, int smem) {
  cudaError_t e = cudaSuccess;
#define PSATD_ARM(c, N, R1, R2)                                                                  \
  {                                                                                              \
    const cudaError_t r = prec == 32 ? configure_pen_t<float, R1, R2>(smem) : configure_pen_t<double, R1, R2>(smem); \
    if (r != cudaSuccess) e = r;                                                                 \
  }
  PSATD_PENCIL_LENGTHS(PSATD_ARM)
#undef PSATD_ARM
  return e;
}

}  // namespace psatd
