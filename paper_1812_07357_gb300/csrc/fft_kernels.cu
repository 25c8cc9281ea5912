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

#include "fft_codelets.cuh"
#include "psatd_internal.h"
#include "psatd_update.cuh"

namespace psatd {

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

// z forward FFT of every slot, update, z inverse FFT of the output slots.
// smem layout [z][slot][t] with t the column inside the tile.
template <typename T, int FORM>
__global__ void __launch_bounds__(kThreads) k_z_update(DevPlan P, cx<T>* spec, int64_t sstride,
                                                       const ColJob* __restrict__ jobs, int nft) {
  constexpr int FIN = fields_in(FORM);
  constexpr int FOUT = fields_out(FORM);
  constexpr int NS = spec_slots(FORM);
  extern __shared__ __align__(16) unsigned char smem_raw[];
  cx<T>* sm = reinterpret_cast<cx<T>*>(smem_raw);
  const ColJob J = jobs[blockIdx.x];
  const BoxDev bx = P.boxes[J.box];
  const ShapeDev& sh = P.shapes[bx.shape];
  const int hx = sh.hx, n1 = bx.n[1], n2 = bx.n[2];
  const int nm = J.nm;
  const int row = NS * nm, rowi = FIN * nm;
  const int64_t zstride = (int64_t)n1 * hx;
  cx<T>* g = spec + bx.soff + (int64_t)J.plane * hx + J.m0;
  for (int e = threadIdx.x; e < n2 * rowi; e += blockDim.x) {
    const int z = e / rowi, r = e - z * rowi;
    const int s = r / nm, t = r - s * nm;
    sm[z * row + r] = g[s * sstride + z * zstride + t];
  }
  __syncthreads();
  const cx<T>* twz = cpool<T>(P) + sh.az.tw;
  // slots >= nft already hold their z spectrum (a cached constant current)
  fft_smem<T, -1, true>(sm, nft * nm, 1, row, sh.az, twz);
  for (int e = threadIdx.x; e < n2 * nm; e += blockDim.x) {
    const int z = e / nm, t = e - z * nm;
    update_mode<T, FORM>(sm + z * row + t, nm, J.m0 + t, J.plane + bx.yoff, z, sh, P);
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
                            const ColJob* jobs, int64_t njobs, int smem, int nft, cudaStream_t st) {
  if (njobs <= 0) return cudaSuccess;
  dim3 grid((unsigned)njobs);
#define PSATD_ZU(T, C2, FORMV) \
  k_z_update<T, FORMV><<<grid, kThreads, smem, st>>>(P, (C2*)spec, sstride, jobs, nft)
  if (prec == 32) {
    if (form == kVacuum) PSATD_ZU(float, float2, kVacuum);
    else if (form == kJForm) PSATD_ZU(float, float2, kJForm);
    else if (form == kPml) PSATD_ZU(float, float2, kPml);
    else PSATD_ZU(float, float2, kRhoForm);
  } else {
    if (form == kVacuum) PSATD_ZU(double, double2, kVacuum);
    else if (form == kJForm) PSATD_ZU(double, double2, kJForm);
    else if (form == kPml) PSATD_ZU(double, double2, kPml);
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
    PSATD_SET((k_z_update<float, kPml>));
    PSATD_SET(k_inv_x<float>);
  } else {
    PSATD_SET(k_fwd_x<double>);
    PSATD_SET((k_col<double, -1>));
    PSATD_SET((k_col<double, 1>));
    PSATD_SET((k_z_update<double, kVacuum>));
    PSATD_SET((k_z_update<double, kJForm>));
    PSATD_SET((k_z_update<double, kRhoForm>));
    PSATD_SET((k_z_update<double, kPml>));
    PSATD_SET(k_inv_x<double>);
  }
#undef PSATD_SET
  return e;
}

}  // namespace psatd
