// Helpers shared by the register-resident kernels (plane and z): async and
// L2-hinted copies, division by a run-time constant, compile-time roots of
// unity, shared-memory row pitches and the thread-pair radix-2 join.
#pragma once
#include <cuda_runtime.h>

#include <cstdint>

#include "fft_codelets.cuh"
#include "psatd_internal.h"

namespace psatd {

namespace {

constexpr int kRegThreads = 128;
constexpr int kGatherTab = 64;   // gather rectangles of a plane staged in shared memory

__device__ __forceinline__ void cp16(void* s, const void* g) {
  const unsigned sa = (unsigned)__cvta_generic_to_shared(s);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(sa), "l"(g) : "memory");
}
// global load of one complex value with a 256-byte L2 fetch: the z tiles of
// neighbouring column groups (run by neighbouring CTAs) read the adjacent
// 128-byte pieces of the same spectrum rows
__device__ __forceinline__ float2 ld_l2_256(const float2* p) {
  float2 r;
  asm("ld.global.L2::256B.v2.f32 {%0, %1}, [%2];\n" : "=f"(r.x), "=f"(r.y) : "l"(p));
  return r;
}
__device__ __forceinline__ void cp4(void* s, const void* g) {
  const unsigned sa = (unsigned)__cvta_generic_to_shared(s);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(sa), "l"(g) : "memory");
}
__device__ __forceinline__ void cp_commit_wait_all() {
  asm volatile("cp.async.commit_group;\ncp.async.wait_group 0;\n" ::: "memory");
}

__device__ __forceinline__ unsigned magic(int d) { return 0xFFFFFFFFu / (unsigned)d + 1u; }
__device__ __forceinline__ int fdiv(int e, unsigned m) { return m ? (int)__umulhi((unsigned)e, m) : e; }

// w^k for w = exp(DIR 2 pi i / R), a compile-time constant
template <int R, int K, int DIR>
__device__ __forceinline__ float2 root() {
  constexpr float c = (float)root_cos(R, K);
  constexpr float s = (float)root_sin(R, K);
  return make_float2(c, DIR < 0 ? -s : s);
}

// float row pitch of a plane buffer holding rows of n0 reals or n0/2 + 1
// complex values: >= n0 + 2, a multiple of 4 (16-byte rows) and = 4 (mod 8)
// so that one-row-per-thread 16-byte accesses spread over all banks.
constexpr int row_pitch(int n0) {
  int p = n0 + 2;
  while (p % 8 != 4) ++p;
  return p;
}

// Thread pairs: the two members of a pair are lanes l and l ^ 16 of a warp,
// so that each half-warp touches one row of a shared-memory plane (no bank
// conflicts between the members).  Thread t: half = (t >> 4) & 1 picks the
// even / odd rows, the pair index is (t & 15) + 16 (t >> 5).
__device__ __forceinline__ int pair_half(int t) { return (t >> 4) & 1; }
__device__ __forceinline__ int pair_index(int t) { return (t & 15) + ((t >> 5) << 4); }

// Thread pair -> one length-NY column FFT.  v: the pair member's
// length-NY/2 FFT (in place on entry).  Writes, through st(y, value), the
// outputs y in [k0, k0 + NY/4) and [k0 + NY/2, ...), with k0 = half * NY/4.
template <int NY, int DIR, typename Store>
__device__ __forceinline__ void pair_join(float2* v, int half, Store&& st) {
  constexpr int H = NY / 2, Q = NY / 4;
  static_for<0, Q>([&](auto ic) {
    constexpr int i = decltype(ic)::value;
    // half 0 keeps E[i], sends E[Q+i]; half 1 keeps O[Q+i], sends O[i]
    const float2 send = half ? v[i] : v[Q + i];
    const float2 keep = half ? v[Q + i] : v[i];
    float2 recv;
    recv.x = __shfl_xor_sync(0xffffffffu, send.x, 16);
    recv.y = __shfl_xor_sync(0xffffffffu, send.y, 16);
    const float2 e = half ? recv : keep;
    const float2 o = half ? keep : recv;
    const float2 w0 = root<NY, i, DIR>(), w1 = root<NY, Q + i, DIR>();
    const float2 w = half ? w1 : w0;
    const float2 t = cmul(o, w);
    const int k = i + half * Q;
    st(k, e + t);
    st(k + H, e - t);
  });
}

// Same join, results left in v: v[i] is output row i + half*NY/4 and v[NY/4 + i]
// output row i + half*NY/4 + NY/2.  `mask`: the lanes taking part (both
// members of every pair in it).
// LANEX: the lane distance of the two members (16 by default).
template <int NY, int DIR, int LANEX = 16>
__device__ __forceinline__ void pair_join_inplace(float2* v, int half, unsigned mask = 0xffffffffu) {
  constexpr int Q = NY / 4;
  static_for<0, Q>([&](auto ic) {
    constexpr int i = decltype(ic)::value;
    const float2 send = half ? v[i] : v[Q + i];
    const float2 keep = half ? v[Q + i] : v[i];
    float2 recv;
    recv.x = __shfl_xor_sync(mask, send.x, LANEX);
    recv.y = __shfl_xor_sync(mask, send.y, LANEX);
    const float2 e = half ? recv : keep;
    const float2 o = half ? keep : recv;
    const float2 w0 = root<NY, i, DIR>(), w1 = root<NY, Q + i, DIR>();
    const float2 t = cmul(o, half ? w1 : w0);
    v[i] = e + t;
    v[Q + i] = e - t;
  });
}

// The inverse of the join (decimation in frequency): on entry the member
// holds outputs v[i] = X[i + half*NY/4] and v[NY/4 + i] = X[i + half*NY/4 +
// NY/2] of a length-NY transform; on exit v[k], k < NY/2, holds
// (X[k] + (-1)^half X[k + NY/2]) w^(half k) (w = exp(DIR 2 pi i / NY)), whose
// length-NY/2 DFT (sign DIR) gives the samples 2j + half.
template <int NY, int DIR, int LANEX = 16>
__device__ __forceinline__ void pair_split_inplace(float2* v, int half, unsigned mask = 0xffffffffu) {
  constexpr int Q = NY / 4;
  static_for<0, Q>([&](auto ic) {
    constexpr int i = decltype(ic)::value;
    const float2 a = v[i], b = v[Q + i];
    const float2 w0 = root<NY, i, DIR>(), w1 = root<NY, Q + i, DIR>();
    const float2 a0 = a + b, a1 = cmul(a - b, half ? w1 : w0);
    const float2 send = half ? a0 : a1;
    const float2 keep = half ? a1 : a0;
    float2 recv;
    recv.x = __shfl_xor_sync(mask, send.x, LANEX);
    recv.y = __shfl_xor_sync(mask, send.y, LANEX);
    v[i] = half ? recv : keep;
    v[Q + i] = half ? keep : recv;
  });
}

}  // namespace

}  // namespace psatd
