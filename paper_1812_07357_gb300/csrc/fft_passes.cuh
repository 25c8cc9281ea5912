// Building blocks of the fast and pencil FFT kernels: two-pass ("four-step")
// transforms of columns held in shared memory, asynchronous row copies, and
// the fused z pass (z FFT of every field slot of a tile of mx columns, the
// k-space update, the inverse z FFT of the output slots).
//
// Every 1D FFT of length N = R1 * R2 is done in two passes: pass 1 takes R1
// elements at stride R2, does DFT_R1 in registers and multiplies by
// w_N^(n2 k1); pass 2 takes R2 consecutive pass-1 results and does DFT_R2,
// giving X[k1 + R1 k2] in natural order.  Shared memory holds the data
// between the passes.
#pragma once

#include <cuda_runtime.h>

#include <cstdint>

#include "fft_codelets.cuh"
#include "psatd_internal.h"
#include "psatd_update.cuh"

namespace psatd {
namespace {   // device helpers with internal linkage in every including unit

template <typename T>
__device__ __forceinline__ const cx<T>* ctab(const DevPlan& P) {
  return reinterpret_cast<const cx<T>*>(P.cpool);
}

// Exact e / d for 0 <= e, d < 2^16 with m = magic(d) = floor((2^32 - 1) / d) + 1:
// e*m / 2^32 = e/d + e*(m - 2^32/d)/2^32 and the error term stays below 1/d.
__device__ __forceinline__ unsigned magic(int d) { return 0xFFFFFFFFu / (unsigned)d + 1u; }
// (for d = 1 the constant wraps to 0 and the quotient is e itself)
__device__ __forceinline__ int fdiv(int e, unsigned m) { return m ? (int)__umulhi((unsigned)e, m) : e; }

// asynchronous 16-byte global -> shared copies (bypassing L1)
__device__ __forceinline__ void cp16(void* s, const void* g) {
  const unsigned sa = (unsigned)__cvta_generic_to_shared(s);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(sa), "l"(g) : "memory");
}
__device__ __forceinline__ void cp_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
__device__ __forceinline__ void cp_wait_prev() { asm volatile("cp.async.wait_group 1;\n" ::: "memory"); }

// ---------------------------------------------------------------------------
// pass 1, in place: column c, positions n1*R2 + n2 (n1 < R1); DFT_R1 along
// n1, times w_N^(n2 k1), back to positions k1*R2 + n2.
// CFAST: consecutive threads take consecutive columns (else consecutive n2).
// ---------------------------------------------------------------------------
template <typename T, int R1, int R2, int DIR, bool CFAST>
__device__ __forceinline__ void pass1(cx<T>* buf, int ncol, int cs, int ns, const cx<T>* __restrict__ tw,
                                      unsigned m_ncol) {
  const int items = ncol * R2;
  for (int it = threadIdx.x; it < items; it += blockDim.x) {
    int c, n2;
    if (CFAST) {
      n2 = fdiv(it, m_ncol);
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
__device__ __forceinline__ void pass2(const cx<T>* buf, int ncol, int cs, int ns, unsigned m_ncol,
                                      Store&& st) {
  const int items = ncol * R1;
  for (int it = threadIdx.x; it < items; it += blockDim.x) {
    int c, k1;
    if (CFAST) {
      k1 = fdiv(it, m_ncol);
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

// Issue the cp.async copies of `rows` rows of `row_bytes` (multiple of 16)
// from contiguous global memory into shared rows of `pitch_bytes`.
__device__ __forceinline__ void load_rows_async(void* dst, const void* src, int rows, int row_bytes,
                                                int pitch_bytes) {
  const int upr = row_bytes >> 4;
  const int total = rows * upr;
  const unsigned m = magic(upr);
  for (int u = threadIdx.x; u < total; u += blockDim.x) {
    const int r = rows == 1 ? 0 : fdiv(u, m), x = u - r * upr;
    cp16(static_cast<char*>(dst) + r * pitch_bytes + x * 16, static_cast<const char*>(src) + (size_t)u * 16);
  }
}

// ---------------------------------------------------------------------------
// z FFT + k-space update + inverse z FFT, all field slots of one mx tile
// ---------------------------------------------------------------------------
template <typename T, int FORM, int TX, int R1, int R2>
__device__ __forceinline__ void z_body(cx<T>* buf, cx<T>* g, int64_t sstride, int64_t zst, int nm, int m0,
                                       int y, int tstride, bool nyq, int zlo, int zhi, int nft,
                                       const ShapeDev& sh, const DevPlan& P) {
  // column t of the tile is mode column (mx, my) = (m0 + t, y), or for a
  // Nyquist tile (mx = n0/2 for TX consecutive y) (m0, y + t); its spectrum
  // starts at g + t * tstride.  Only the interior z planes [zlo, zhi) are
  // stored back: the inverse plane pass reads no others.  Slots >= nft
  // already hold their z spectrum (a cached constant current): loaded as is.
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
    const cx<T>* p = g + s * sstride + n2 * zst + t * tstride;
    cx<T> v[R1];
#pragma unroll
    for (int j = 0; j < R1; ++j) v[j] = p[j * R2 * zst];
    if (s < nft) {
      Dft<T, R1, -1>::run(v);
      if (n2) {
#pragma unroll
        for (int k = 1; k < R1; ++k) v[k] = cmul(v[k], tw[n2 * k]);
      }
    }
#pragma unroll
    for (int j = 0; j < R1; ++j) buf[(j * R2 + n2) * NP + c] = v[j];
  }
  __syncthreads();
  // pass 2 in place: all loads first (registers), then natural-order stores
  {
    constexpr int ITEMS = NCOL * R1;
    constexpr int MAXI = (ITEMS + kThreads - 1) / kThreads;
    const int ncolt = nft * TX;   // columns that take the z FFT
    cx<T> u[MAXI][R2];
#pragma unroll
    for (int i = 0; i < MAXI; ++i) {
      const int it = threadIdx.x + i * kThreads;
      if (it < ITEMS && it % NCOL < ncolt) {
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
      if (it < ITEMS && it % NCOL < ncolt) {
        const int k1 = it / NCOL, c = it - k1 * NCOL;
#pragma unroll
        for (int k2 = 0; k2 < R2; ++k2) buf[(k1 + R1 * k2) * NP + c] = u[i][k2];
      }
    }
  }
  __syncthreads();
  static_assert(kThreads % TX == 0, "update threads keep one column");
  {
    const int t = threadIdx.x % TX;
    if (t < nm) {
      const ModeXY<T> xy = mode_xy<T>(nyq ? m0 : m0 + t, nyq ? y + t : y, sh, P);
      for (int z = threadIdx.x / TX; z < N; z += kThreads / TX)
        update_mode_z<T, FORM>(buf + z * NP + t, TX, xy, z, sh, P);
    }
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
    cx<T>* p = g + s * sstride + t * tstride;
#pragma unroll
    for (int k2 = 0; k2 < R2; ++k2) {
      const int z = k1 + R1 * k2;
      if (z >= zlo && z < zhi) p[z * zst] = u[k2];
    }
  }
}

}  // namespace
}  // namespace psatd
