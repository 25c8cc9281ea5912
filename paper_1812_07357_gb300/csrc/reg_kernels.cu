// Register-resident plane kernels (FP32) for boxes whose x half-length L and
// y length NY have register codelets (L, NY/2 <= 48): every 1D FFT of a
// plane is done inside registers, so a plane costs two block barriers.
//
//   k_plane_fwd_reg  the plane is copied in whole, or, with the deferred guard
//                    exchange, gathered rectangle by rectangle from the cells
//                    that own it;
//                    x: one thread per row: the packed length-L complex FFT
//                    (z[m] = x[2m] + i x[2m+1]) and the R2C split, both in
//                    registers; y: two threads per column, each a length-NY/2
//                    FFT of the even / odd rows, joined by one radix-2 step
//                    whose operands cross between the pair with shuffles.
//   k_plane_inv_reg  the mirror image, keeping interior rows and cells only,
//                    and writing the guard cells the plane feeds (fused S4).
//   k_z_reg          z FFT of every field slot of a tile of columns: a thread
//                    pair per column (loads straight from HBM into registers)
//                    does the half-length DFTs of the even and odd z samples,
//                    the update threads do the radix-2 stage and the k-space
//                    update of every mode in shared memory, then the inverse
//                    radix-2 stage, and the pairs the half-length inverse DFTs
//                    of the output slots back to HBM.
//
// Twiddle factors are compile-time constants (unit_roots.h).
#include <cuda_runtime.h>

#include <cstdint>
#include <type_traits>

#include "fft_codelets.cuh"
#include "psatd_internal.h"
#include "psatd_update.cuh"

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
template <int NY, int DIR>
__device__ __forceinline__ void pair_join_inplace(float2* v, int half, unsigned mask = 0xffffffffu) {
  constexpr int Q = NY / 4;
  static_for<0, Q>([&](auto ic) {
    constexpr int i = decltype(ic)::value;
    const float2 send = half ? v[i] : v[Q + i];
    const float2 keep = half ? v[Q + i] : v[i];
    float2 recv;
    recv.x = __shfl_xor_sync(mask, send.x, 16);
    recv.y = __shfl_xor_sync(mask, send.y, 16);
    const float2 e = half ? recv : keep;
    const float2 o = half ? keep : recv;
    const float2 w0 = root<NY, i, DIR>(), w1 = root<NY, Q + i, DIR>();
    const float2 t = cmul(o, half ? w1 : w0);
    v[i] = e + t;
    v[Q + i] = e - t;
  });
}

// ---------------------------------------------------------------------------
template <int L, int NY>
__global__ void __launch_bounds__(kRegThreads, 4)
    k_plane_fwd_reg(DevPlan P, FieldPtrs F, float2* spec, int64_t sstride, const int2* __restrict__ jobs,
                    const int* __restrict__ gstart, const GatherSeg* __restrict__ gsegs,
                    const GatherGrid* __restrict__ ggrid, int ngather) {
  constexpr int N0 = 2 * L, HX = L + 1, PF = row_pitch(N0);
  static_assert(NY <= kRegThreads && 2 * HX <= kRegThreads, "one thread per row / per half column");
  extern __shared__ __align__(16) unsigned char smem_raw[];
  float* buf = reinterpret_cast<float*>(smem_raw);
  const int2 J = jobs[blockIdx.x];
  const int f = blockIdx.y;
  const BoxDev bx = P.boxes[J.x];
  constexpr int UPR = N0 / 4;
  if (ggrid && f < ngather) {
    // deferred exchange, plane of at most 3 x 3 rectangles: thread t copies
    // the 16-byte column t % UPR of the rows t / UPR + k * RG
    constexpr int RG = kRegThreads / UPR;
    __shared__ GatherGrid gg;
    static_assert(sizeof(GatherGrid) / 4 <= kRegThreads, "one word per thread");
    if (threadIdx.x < sizeof(GatherGrid) / 4)
      reinterpret_cast<int*>(&gg)[threadIdx.x] = reinterpret_cast<const int*>(ggrid + blockIdx.x)[threadIdx.x];
    __syncthreads();
    if (threadIdx.x < RG * UPR) {
      const float* fb = reinterpret_cast<const float*>(F.p[f]);
      const int c = threadIdx.x % UPR, rg = threadIdx.x / UPR, x = 4 * c;
      const int ix = (x >= gg.x1) + (x >= gg.x2);
      const int xo = x - (ix == 0 ? 0 : ix == 1 ? gg.x1 : gg.x2);
#pragma unroll
      for (int iy = 0; iy < 3; ++iy) {   // row bands [ylo, yhi)
        const int ylo = iy == 0 ? 0 : iy == 1 ? gg.y1 : gg.y2;
        const int yhi = iy == 0 ? gg.y1 : iy == 1 ? gg.y2 : NY;
        int r = ylo + (rg - ylo % RG + RG) % RG;   // first row >= ylo with r % RG == rg
        const int pitch = gg.pitch[3 * iy + ix];
        const float* src = fb + gg.base[3 * iy + ix] + (int64_t)(r - ylo) * pitch + xo;
        const int64_t sstep = (int64_t)RG * pitch;
        for (float* dst = buf + r * PF + x; r < yhi; r += RG, src += sstep, dst += RG * PF) cp16(dst, src);
      }
    }
  } else if (gstart && f < ngather) {
    // deferred exchange: every rectangle of the plane from the cells that own
    // it (a neighbour's interior for the guard cells); the plane's rectangle
    // list is staged in shared memory, then all threads copy one rectangle
    // after the other
    __shared__ GatherSeg tab[kGatherTab];
    const float* fb = reinterpret_cast<const float*>(F.p[f]);
    const int s0 = gstart[blockIdx.x], ns = gstart[blockIdx.x + 1] - s0;
    if (threadIdx.x < kGatherTab && threadIdx.x < ns) tab[threadIdx.x] = gsegs[s0 + threadIdx.x];
    __syncthreads();
    for (int i = 0; i < ns; ++i) {
      const GatherSeg gs = i < kGatherTab ? tab[i] : gsegs[s0 + i];
      const float* src = fb + gs.src_off;
      float* dst = buf + gs.dy * PF + gs.dx;
      if (gs.vec) {
        const int upr = gs.nx >> 2;
        const unsigned m = magic(upr);
        for (int u = threadIdx.x; u < gs.ny * upr; u += kRegThreads) {
          const int r = fdiv(u, m), c = 4 * (u - r * upr);
          cp16(dst + r * PF + c, src + (int64_t)r * gs.spitch + c);
        }
      } else {
        const unsigned m = magic(gs.nx);
        for (int u = threadIdx.x; u < gs.ny * gs.nx; u += kRegThreads) {
          const int r = fdiv(u, m), c = u - r * gs.nx;
          cp4(dst + r * PF + c, src + (int64_t)r * gs.spitch + c);
        }
      }
    }
  } else {
    const float* g = reinterpret_cast<const float*>(F.p[f]) + bx.foff + (int64_t)J.y * NY * N0;
    for (int u = threadIdx.x; u < NY * UPR; u += kRegThreads) {
      const int r = u / UPR, x = u - r * UPR;
      cp16(buf + r * PF + 4 * x, g + 4 * u);
    }
  }
  cp_commit_wait_all();
  __syncthreads();
  // x: row r -> half spectrum X[0..L] written back into the same row
  if (threadIdx.x < NY) {
    float* row = buf + threadIdx.x * PF;
    float2 z[L];
#pragma unroll
    for (int j = 0; j < L / 2; ++j) {
      const float4 q = reinterpret_cast<const float4*>(row)[j];
      z[2 * j] = make_float2(q.x, q.y);
      z[2 * j + 1] = make_float2(q.z, q.w);
    }
    Dft<float, L, -1>::run(z);
    float2* xr = reinterpret_cast<float2*>(row);
    // X[k] = (Z[k] + conj Z[L-k])/2 - i w^k (Z[k] - conj Z[L-k])/2, w = exp(-2 pi i / N0)
    static_for<0, L / 2 + 1>([&](auto kc) {
      constexpr int k = decltype(kc)::value;
      const float2 a = z[k % L], b = z[(L - k) % L];
      const float2 A = make_float2(0.5f * (a.x + b.x), 0.5f * (a.y - b.y));
      const float2 Bv = make_float2(0.5f * (a.y + b.y), 0.5f * (b.x - a.x));
      if constexpr (k == 0) {
        xr[0] = make_float2(A.x + Bv.x, A.y + Bv.y);
        xr[L] = make_float2(A.x - Bv.x, A.y - Bv.y);
      } else {
        xr[k] = A + cmul(root<N0, k, -1>(), Bv);
        if constexpr (2 * k != L) xr[L - k] = conjg(A) + cmul(root<N0, L - k, -1>(), conjg(Bv));
      }
    });
  }
  __syncthreads();
  // y: thread pair per column c; threads past the last column repeat it
  {
    const int t = threadIdx.x;
    const int half = pair_half(t);
    const int c = min(pair_index(t), HX - 1);
    const bool live = pair_index(t) < HX;
    const float2* xs = reinterpret_cast<const float2*>(buf);
    float2 v[NY / 2];
#pragma unroll
    for (int m = 0; m < NY / 2; ++m) v[m] = xs[(2 * m + half) * (PF / 2) + c];
    Dft<float, NY / 2, -1>::run(v);
    float2* out = spec + f * sstride + bx.soff + (int64_t)J.y * NY * HX + c;
    pair_join<NY, -1>(v, half, [&](int y, float2 val) {
      if (live) out[y * HX] = val;
    });
  }
}

// ---------------------------------------------------------------------------
template <typename V>
__device__ __forceinline__ void copy_rect_w(const float* src, int spitch, float* dst, int64_t dpitch, int ny,
                                            int nx, int tid, int nthreads) {
  constexpr int W = sizeof(V) / 4;
  const int upr = nx / W;
  const unsigned m = magic(upr);
  for (int u = tid; u < ny * upr; u += nthreads) {
    const int r = fdiv(u, m), c = (u - r * upr) * W;
    *reinterpret_cast<V*>(dst + r * dpitch + c) = *reinterpret_cast<const V*>(src + r * spitch + c);
  }
}

template <int L, int NY>
__global__ void __launch_bounds__(kRegThreads, 4) k_plane_inv_reg(DevPlan P, FieldPtrs F, const float2* spec,
                                                                  int64_t sstride, const int2* __restrict__ jobs,
                                                                  const int* __restrict__ seg_start,
                                                                  const GuardSeg* __restrict__ segs) {
  constexpr int N0 = 2 * L, HX = L + 1, PF = row_pitch(N0), Q = NY / 4;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  // one buffer: first the NY x HX spectrum plane (pitch HX), then, once it is
  // consumed, the interior rows (pitch PF floats): X values, then real cells
  float2* sp = reinterpret_cast<float2*>(smem_raw);
  float* rows = reinterpret_cast<float*>(smem_raw);
  const int2 J = jobs[blockIdx.x];
  const int f = blockIdx.y;
  const BoxDev bx = P.boxes[J.x];
  const int ylo = bx.ng_lo[1], yhi = NY - bx.ng_hi[1], ni = yhi - ylo;
  const int xlo = bx.ng_lo[0], nxi = N0 - bx.ng_lo[0] - bx.ng_hi[0];
  const float2* g = spec + f * sstride + bx.soff + (int64_t)J.y * NY * HX;
  constexpr int UNITS = NY * HX / 2;   // 16-byte units of the contiguous plane
  for (int u = threadIdx.x; u < UNITS; u += kRegThreads) cp16(sp + 2 * u, g + 2 * u);
  cp_commit_wait_all();
  __syncthreads();
  // y: thread pair per column, inverse; outputs kept in v until the plane is consumed
  const int t = threadIdx.x;
  const int half = pair_half(t);
  const int c = min(pair_index(t), HX - 1);
  const bool live = pair_index(t) < HX;
  float2 v[NY / 2];
#pragma unroll
  for (int m = 0; m < NY / 2; ++m) v[m] = sp[(2 * m + half) * HX + c];
  Dft<float, NY / 2, 1>::run(v);
  pair_join_inplace<NY, 1>(v, half);
  __syncthreads();
  if (live) {
    float2* rs = reinterpret_cast<float2*>(rows);
#pragma unroll
    for (int i = 0; i < Q; ++i) {
      const int y1 = i + half * Q, y2 = y1 + NY / 2;
      if (y1 >= ylo && y1 < yhi) rs[(y1 - ylo) * (PF / 2) + c] = v[i];
      if (y2 >= ylo && y2 < yhi) rs[(y2 - ylo) * (PF / 2) + c] = v[Q + i];
    }
  }
  __syncthreads();
  // x: thread per interior row: C2R merge, inverse packed FFT, interior cells
  // written back into the thread's own row
  const float scale = __frcp_rn((float)(N0 * NY * bx.n[2]));   // exact integer < 2^24
  const bool vec_rows = (nxi % 4 == 0) && (xlo % 4 == 0);
  if (threadIdx.x < ni) {
    float* row = rows + threadIdx.x * PF;
    const float2* xr = reinterpret_cast<const float2*>(row);
    float2 z[L];
    // Z'[k] = (X[k] + conj X[L-k]) + i w^-k (X[k] - conj X[L-k]), w = exp(-2 pi i / N0)
    static_for<0, L / 2 + 1>([&](auto kc) {
      constexpr int k = decltype(kc)::value;
      const float2 a = xr[k], b = xr[L - k];
      z[k] = (a + conjg(b)) + times_i(cmul(a - conjg(b), root<N0, k, 1>()));
      if constexpr (k != 0 && 2 * k != L)
        z[L - k] = (b + conjg(a)) + times_i(cmul(b - conjg(a), root<N0, L - k, 1>()));
    });
    Dft<float, L, 1>::run(z);
    float* o = row - xlo;
    if (vec_rows) {
#pragma unroll
      for (int m = 0; m < L; m += 2) {
        const int x = 2 * m;
        if (x >= xlo && x < xlo + nxi)
          *reinterpret_cast<float4*>(o + x) =
              make_float4(scale * z[m].x, scale * z[m].y, scale * z[m + 1].x, scale * z[m + 1].y);
      }
    } else {
#pragma unroll
      for (int m = 0; m < L; ++m) {
        const int x = 2 * m;
        if (x >= xlo && x < xlo + nxi) o[x] = scale * z[m].x;
        if (x + 1 >= xlo && x + 1 < xlo + nxi) o[x + 1] = scale * z[m].y;
      }
    }
  }
  __syncthreads();
  // interior cells to this box, then the guard cells this plane feeds
  float* fbase = reinterpret_cast<float*>(F.p[f]);
  float* own = fbase + bx.foff + ((int64_t)J.y * NY + ylo) * N0 + xlo;
  if (vec_rows)
    copy_rect_w<float4>(rows, PF, own, N0, ni, nxi, threadIdx.x, kRegThreads);
  else
    copy_rect_w<float>(rows, PF, own, N0, ni, nxi, threadIdx.x, kRegThreads);
  if (seg_start) {
    const int p = blockIdx.x;
    const int s1 = seg_start[p + 1];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = kRegThreads >> 5;
    for (int si = seg_start[p] + warp; si < s1; si += nw) {
      const GuardSeg gs = segs[si];
      const BoxDev db = P.boxes[gs.dst_box];
      float* dst = fbase + db.foff + ((int64_t)gs.dst_z * db.n[1] + gs.dy) * db.n[0] + gs.dx;
      const float* src = rows + (gs.sy - ylo) * PF + (gs.sx - xlo);
      if (gs.vec > 1 && vec_rows)
        copy_rect_w<float4>(src, PF, dst, db.n[0], gs.ny, gs.nx, lane, 32);
      else
        copy_rect_w<float>(src, PF, dst, db.n[0], gs.ny, gs.nx, lane, 32);
    }
  }
}

// ---------------------------------------------------------------------------
// exp(-2 pi i k / NZ), k < NZ/2: the twiddles of the radix-2 z stage, rounded
// from the compile-time FP64 roots
template <int NZ>
struct HalfTwiddles {
  float2 w[NZ / 2];
};
template <int NZ>
constexpr HalfTwiddles<NZ> half_twiddles() {
  HalfTwiddles<NZ> t{};
  for (int k = 0; k < NZ / 2; ++k) t.w[k] = float2{(float)root_cos(NZ, k), (float)-root_sin(NZ, k)};
  return t;
}
__constant__ HalfTwiddles<96> kTw96 = half_twiddles<96>();
__constant__ HalfTwiddles<48> kTw48 = half_twiddles<48>();
__constant__ HalfTwiddles<60> kTw60 = half_twiddles<60>();
__constant__ HalfTwiddles<80> kTw80 = half_twiddles<80>();
__constant__ HalfTwiddles<120> kTw120 = half_twiddles<120>();
template <int NZ>
__device__ __forceinline__ float2 half_twiddle(int k) {
  static_assert(NZ == 96 || NZ == 48 || NZ == 60 || NZ == 80 || NZ == 120, "register z lengths");
  if constexpr (NZ == 96) return kTw96.w[k];
  else if constexpr (NZ == 48) return kTw48.w[k];
  else if constexpr (NZ == 60) return kTw60.w[k];
  else if constexpr (NZ == 80) return kTw80.w[k];
  else return kTw120.w[k];
}

// mx columns (or Nyquist-column y rows) per z tile: 16 (128-byte rows of a
// slot) for the 6-slot vacuum form, 8 for the forms with sources
constexpr int z_reg_tile(int form) { return form == kVacuum ? 16 : 8; }

// fields_in * tile (slot, column) FFTs per tile, a thread pair each, rounded
// up to whole warps (the pairs past the last slot compute a copy and store nothing)
template <int FORM>
constexpr int z_reg_threads() {
  return (2 * fields_in(FORM) * z_reg_tile(FORM) + 31) / 32 * 32;
}
// shared-memory pitch (complex) of one z row: >= fields_in * tile, = 8 (mod 16)
constexpr int z_reg_pitch(int form) {
  return fields_in(form) * z_reg_tile(form) + ((24 - (fields_in(form) * z_reg_tile(form)) % 16) % 16);
}
template <int FORM>
constexpr int z_reg_min_blocks() {
  return 2;
}

// ZST > 0: every box of the launch has n1 * (n0/2 + 1) = ZST (the z stride of
// the spectrum), a compile-time constant, so that the z-strided loads and
// stores take immediate offsets.
// L2 prefetch of the input rows of z tile `job` (every slot, every z plane;
// a row of at most TX complex values spans at most two 128-byte lines).
// Nyquist-column tiles (scattered values) are not prefetched.
template <int NZ, int FORM>
__device__ __forceinline__ void prefetch_z_tile(const DevPlan& P, const float2* spec, int64_t sstride,
                                                const ColJob& J) {
  constexpr int FIN = fields_in(FORM), NT = z_reg_threads<FORM>();
  if (J.nm < 0) return;
  const BoxDev bx = P.boxes[J.box];
  const int hx = P.shapes[bx.shape].hx;
  const int64_t zst = (int64_t)bx.n[1] * hx;
  const float2* g = spec + bx.soff + (int64_t)J.plane * hx + J.m0;
  for (int r = threadIdx.x; r < 2 * FIN * NZ; r += NT) {
    const int row = r >> 1, s = row / NZ, z = row - s * NZ;
    const float2* a = g + s * sstride + z * zst + (r & 1) * (J.nm - 1);
    asm volatile("prefetch.global.L2::evict_last [%0];\n" ::"l"(a));
  }
}

template <int NZ, int FORM, int ZST>
__global__ void __launch_bounds__(z_reg_threads<FORM>(), z_reg_min_blocks<FORM>())
    k_z_reg(DevPlan P, float2* spec, int64_t sstride, const ColJob* __restrict__ jobs, int nft, int njobs,
            int pf_dist) {
  constexpr int TX = z_reg_tile(FORM), FIN = fields_in(FORM), FOUT = fields_out(FORM);
  constexpr int NT = z_reg_threads<FORM>(), NP = z_reg_pitch(FORM);
  constexpr int H = NZ / 2;
  static_assert(NT % (2 * TX) == 0, "update threads keep one column");
  extern __shared__ __align__(16) unsigned char smem_raw[];
  float2* buf = reinterpret_cast<float2*>(smem_raw);    // [row][slot * TX + t], pitch NP
  const ColJob J = jobs[blockIdx.x];
  // the tile that a CTA launched about pf_dist blocks later will read: fetched
  // into L2 now, so that its loads hit L2 instead of waiting on HBM
  if (pf_dist > 0 && (int)blockIdx.x + pf_dist < njobs)
    prefetch_z_tile<NZ, FORM>(P, spec, sstride, jobs[blockIdx.x + pf_dist]);
  const BoxDev bx = P.boxes[J.box];
  const ShapeDev& sh = P.shapes[bx.shape];
  const int hx = sh.hx, n1 = bx.n[1];
  const int64_t zst = ZST > 0 ? (int64_t)ZST : (int64_t)n1 * hx;
  // column t: mode column (m0 + t, y), or (m0 = n0/2, y + t) for a Nyquist tile
  const bool nyq = J.nm < 0;
  const int nm = nyq ? -J.nm : J.nm, ts = nyq ? hx : 1;
  float2* g = spec + bx.soff + (int64_t)J.plane * hx + J.m0;
  // thread pair per (slot, column): member `half` holds the z samples 2m + half
  const int tid = threadIdx.x, half = pair_half(tid), col = pair_index(tid);
  const int s = col / TX, t = col - s * TX;
  const bool live = t < nm && s < FIN;
  const int tc = t < nm ? t : 0, sc = s < FIN ? s : FIN - 1;
  float2 v[H];
  {
    const float2* src = g + sc * sstride + (int64_t)tc * ts + half * zst;
#pragma unroll
    for (int m = 0; m < H; ++m) v[m] = ld_l2_256(src + 2 * m * zst);
  }
  // half-length forward DFT of the member's samples into row half * H + k;
  // slots >= nft already hold their z spectrum (a cached constant current) in
  // natural z order and are stored as they are.
  // Shared-memory layout of a row: per slot, per column pair (2j, 2j + 1),
  // the 16 bytes (re 2j, re 2j+1, im 2j, im 2j+1) in rows [0, H) and
  // (im 2j, im 2j+1, re 2j, re 2j+1) in rows [H, NZ): the update threads load
  // the real and imaginary parts of two columns as register pairs, and the
  // two halves of a warp storing rows k and H + k hit disjoint banks.
  float* bw = reinterpret_cast<float*>(buf);
  const int q0 = 2 * s * TX + 4 * (t >> 1) + (t & 1);      // word of re in a re-first row
  if (s < nft) {
    Dft<float, H, -1>::run(v);
    const int re = q0 + 2 * half, im = q0 + 2 - 2 * half;
#pragma unroll
    for (int k = 0; k < H; ++k) {
      bw[(half * H + k) * 2 * NP + re] = v[k].x;
      bw[(half * H + k) * 2 * NP + im] = v[k].y;
    }
  } else if (s < FIN) {
#pragma unroll
    for (int m = 0; m < H; ++m) {
      const int z = 2 * m + half, sw = 2 * m >= H ? 2 : 0;
      bw[z * 2 * NP + q0 + sw] = v[m].x;
      bw[z * 2 * NP + q0 + 2 - sw] = v[m].y;
    }
  }
  __syncthreads();
  // k-space update of the column pair (2 tp, 2 tp + 1), tp = tid % (TX/2),
  // modes k and k + H for k = tid / (TX/2) + i NT/(TX/2) (unrolled), with the
  // radix-2 stages of both z transforms.  A pair whose second column is past
  // the tile computes it on dead data (clamped table indices) and only writes
  // dead shared memory.
  {
    constexpr int TP = TX / 2, ZS = NT / TP, NIT = (H + ZS - 1) / ZS;
    static_assert(TX % 2 == 0 && NT % TP == 0, "column pairs");
    const int tp = tid % TP, k0 = tid / TP;
    const int ta = 2 * tp;
    if (ta < nm) {
      const int mxa = nyq ? J.m0 : J.m0 + ta, mya = nyq ? J.plane + ta : J.plane;
      const int mxb = nyq ? J.m0 : mxa + 1, myb = nyq ? min(mya + 1, n1 - 1) : J.plane;
      const ModeXY2 xy = mode_xy2(mxa, mya, mxb, myb, sh, P);
#pragma unroll
      for (int it = 0; it < NIT; ++it) {
        const int k = k0 + it * ZS;
        if (H % ZS == 0 || k < H) {
          const float2 w = half_twiddle<NZ>(k);   // exp(-2 pi i k / NZ)
          update_pair_z2<FORM, NZ>(buf + k * NP + ta, buf + (k + H) * NP + ta, TX, xy, k, w, nft, sh, P);
        }
      }
    }
  }
  __syncthreads();
  // half-length inverse DFTs: member `half` gives the z samples 2m + half of
  // the output slots; threads of the remaining slots repeat the last output
  // slot and store nothing.  Only interior z planes are stored: the inverse
  // plane pass reads no others.
  {
    const int so = s < FOUT ? s : FOUT - 1;
    const int qo = 2 * so * TX + 4 * (t >> 1) + (t & 1);
    const int re = qo + 2 * half, im = qo + 2 - 2 * half;
#pragma unroll
    for (int k = 0; k < H; ++k) v[k] = make_float2(bw[(half * H + k) * 2 * NP + re], bw[(half * H + k) * 2 * NP + im]);
  }
  Dft<float, H, 1>::run(v);
  if (live && s < FOUT) {
    const int zlo = bx.ng_lo[2], zhi = NZ - bx.ng_hi[2];
    float2* dst = g + s * sstride + (int64_t)t * ts + half * zst;
#pragma unroll
    for (int m = 0; m < H; ++m) {
      const int z = 2 * m + half;
      if (z >= zlo && z < zhi) dst[2 * m * zst] = v[m];
    }
  }
}

}  // namespace

// z lengths with a register z kernel: X(NZ)
#define PSATD_REG_Z(X) X(96) X(48) X(60) X(80) X(120)

int z_reg_ok(int n2) {
#define PSATD_ZC(NZV) \
  if (n2 == NZV) return 1;
  PSATD_REG_Z(PSATD_ZC)
#undef PSATD_ZC
  return 0;
}

int z_reg_smem(int form, int n2) { return n2 * z_reg_pitch(form) * 8; }

int z_reg_tile_width(int form) { return z_reg_tile(form); }

// z strides with their own instantiation: the register plane shape 96 x 96
constexpr int kRegZst = 96 * 49;

cudaError_t launch_z_reg(int form, const DevPlan& P, void* spec, int64_t sstride, const ColJob* jobs,
                         int64_t njobs, int n2, int zst, int nft, int pf_dist, cudaStream_t st) {
  if (njobs <= 0) return cudaSuccess;
  dim3 grid((unsigned)njobs);
  const int smem = z_reg_smem(form, n2);
#define PSATD_ZF(NZV, F, ZS)                                                                      \
  k_z_reg<NZV, F, ZS><<<grid, z_reg_threads<F>(), smem, st>>>(P, (float2*)spec, sstride, jobs, nft, \
                                                               (int)njobs, pf_dist)
#define PSATD_ZL(NZV)                                                    \
  if (n2 == NZV) {                                                      \
    if (form == kVacuum) {                                              \
      if (zst == kRegZst)                                               \
        PSATD_ZF(NZV, kVacuum, kRegZst);                                \
      else                                                              \
        PSATD_ZF(NZV, kVacuum, 0);                                      \
    } else if (form == kJForm) {                                        \
      if (zst == kRegZst)                                               \
        PSATD_ZF(NZV, kJForm, kRegZst);                                 \
      else                                                              \
        PSATD_ZF(NZV, kJForm, 0);                                       \
    } else {                                                            \
      if (zst == kRegZst)                                               \
        PSATD_ZF(NZV, kRhoForm, kRegZst);                               \
      else                                                              \
        PSATD_ZF(NZV, kRhoForm, 0);                                     \
    }                                                                   \
  }
  PSATD_REG_Z(PSATD_ZL)
#undef PSATD_ZL
#undef PSATD_ZF
  return cudaGetLastError();
}

// Register-resident plane shapes: X(code, L, NY)
#define PSATD_REG_SHAPES(X) X(0, 48, 96)

int reg_shape_code(int L, int n1) {
#define PSATD_RC(code, LV, NYV) \
  if (L == LV && n1 == NYV) return code;
  PSATD_REG_SHAPES(PSATD_RC)
#undef PSATD_RC
  return -1;
}

int reg_fwd_smem(int code) {
#define PSATD_RS(code_, LV, NYV) \
  if (code == code_) return NYV * row_pitch(2 * LV) * 4;
  PSATD_REG_SHAPES(PSATD_RS)
#undef PSATD_RS
  return 0;
}

// the spectrum plane, or at most NY interior rows of pitch row_pitch(n0)
int reg_inv_smem(int code) {
#define PSATD_RS(code_, LV, NYV) \
  if (code == code_) return NYV * (LV + 1) * 8 > NYV * row_pitch(2 * LV) * 4 ? NYV * (LV + 1) * 8 \
                                                                            : NYV * row_pitch(2 * LV) * 4;
  PSATD_REG_SHAPES(PSATD_RS)
#undef PSATD_RS
  return 0;
}

cudaError_t launch_plane_fwd_reg(int code, const DevPlan& P, const FieldPtrs& f, int nf, void* spec,
                                 int64_t sstride, const int2* jobs, int64_t nplanes, const int* gstart,
                                 const GatherSeg* gsegs, const GatherGrid* ggrid, int ngather, cudaStream_t st) {
  if (nplanes <= 0 || nf <= 0) return cudaSuccess;
  dim3 grid((unsigned)nplanes, nf);
#define PSATD_RL(code_, LV, NYV)                                                                        \
  if (code == code_)                                                                                   \
    k_plane_fwd_reg<LV, NYV><<<grid, kRegThreads, reg_fwd_smem(code_), st>>>(P, f, (float2*)spec, sstride, \
                                                                           jobs, gstart, gsegs, ggrid, ngather);
  PSATD_REG_SHAPES(PSATD_RL)
#undef PSATD_RL
  return cudaGetLastError();
}

cudaError_t launch_plane_inv_reg(int code, const DevPlan& P, const FieldPtrs& f, int nf, void* spec,
                                 int64_t sstride, const int2* jobs, int64_t nplanes, const int* seg_start,
                                 const GuardSeg* segs, cudaStream_t st) {
  if (nplanes <= 0 || nf <= 0) return cudaSuccess;
  dim3 grid((unsigned)nplanes, nf);
#define PSATD_RL(code_, LV, NYV)                                                                   \
  if (code == code_)                                                                              \
    k_plane_inv_reg<LV, NYV><<<grid, kRegThreads, reg_inv_smem(code_), st>>>(                         \
        P, f, (const float2*)spec, sstride, jobs, seg_start, segs);
  PSATD_REG_SHAPES(PSATD_RL)
#undef PSATD_RL
  return cudaGetLastError();
}

// Dynamic shared memory limits of the register kernels: what each launch
// asks for (the gather table of the forward kernel is static shared memory
// on top of it); `smem` is the device's opt-in maximum.
cudaError_t configure_reg_kernels(int smem) {
  cudaError_t e = cudaSuccess;
#define PSATD_RC(code, LV, NYV)                                                                          \
  if (reg_fwd_smem(code) <= smem && reg_inv_smem(code) <= smem) {                                        \
    cudaError_t r = cudaFuncSetAttribute(k_plane_fwd_reg<LV, NYV>,                                        \
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, reg_fwd_smem(code)); \
    if (r != cudaSuccess) e = r;                                                                         \
    r = cudaFuncSetAttribute(k_plane_inv_reg<LV, NYV>, cudaFuncAttributeMaxDynamicSharedMemorySize,       \
                             reg_inv_smem(code));                                                        \
    if (r != cudaSuccess) e = r;                                                                         \
  }
  PSATD_REG_SHAPES(PSATD_RC)
#undef PSATD_RC
#define PSATD_ZA(NZV, F, ZS)                                                                      \
  if (z_reg_smem(F, NZV) <= smem) {                                                               \
    const cudaError_t r = cudaFuncSetAttribute(k_z_reg<NZV, F, ZS>,                               \
                                               cudaFuncAttributeMaxDynamicSharedMemorySize,       \
                                               z_reg_smem(F, NZV));                               \
    if (r != cudaSuccess) e = r;                                                                  \
  }
#define PSATD_ZS(NZV)                 \
  PSATD_ZA(NZV, kVacuum, 0)           \
  PSATD_ZA(NZV, kJForm, 0)            \
  PSATD_ZA(NZV, kRhoForm, 0)          \
  PSATD_ZA(NZV, kVacuum, kRegZst)     \
  PSATD_ZA(NZV, kJForm, kRegZst)      \
  PSATD_ZA(NZV, kRhoForm, kRegZst)
  PSATD_REG_Z(PSATD_ZS)
#undef PSATD_ZS
#undef PSATD_ZA
  return e;
}

}  // namespace psatd
