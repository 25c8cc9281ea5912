// Register-resident z kernels (FP32):
//
//   k_z_reg          z FFT of every field slot of a tile of columns: a thread
//                    pair per column (loads straight from HBM into registers)
//                    does the half-length DFTs of the even and odd z samples,
//                    the update threads do the radix-2 stage and the k-space
//                    update of every mode in shared memory, then the inverse
//                    radix-2 stage, and the pairs the half-length inverse DFTs
//                    of the output slots back to HBM.
//   k_z_reg_multi    the same tiles for boxes of several z lengths in one
//                    persistent launch.
//
// Twiddle factors are compile-time constants (unit_roots.h).  This file also
// dispatches the register plane kernels (reg_planes.cuh) by shape code.
#include <cuda_runtime.h>

#include <cstdint>
#include <type_traits>

#include "fft_codelets.cuh"
#include "psatd_internal.h"
#include "psatd_update.cuh"
#include "reg_common.cuh"
#include "reg_planes.cuh"

namespace psatd {

namespace {
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
__constant__ HalfTwiddles<128> kTw128 = half_twiddles<128>();
__constant__ HalfTwiddles<192> kTw192 = half_twiddles<192>();
template <int NZ>
__device__ __forceinline__ float2 half_twiddle(int k) {
  static_assert(NZ == 96 || NZ == 48 || NZ == 60 || NZ == 80 || NZ == 120 || NZ == 128 || NZ == 192,
                "register z lengths");
  if constexpr (NZ == 96) return kTw96.w[k];
  else if constexpr (NZ == 48) return kTw48.w[k];
  else if constexpr (NZ == 60) return kTw60.w[k];
  else if constexpr (NZ == 80) return kTw80.w[k];
  else if constexpr (NZ == 120) return kTw120.w[k];
  else if constexpr (NZ == 128) return kTw128.w[k];
  else return kTw192.w[k];
}

// mx columns (or Nyquist-column y rows) per z tile: 16 (128-byte rows of a
// slot) for the 6-slot vacuum form, 8 for the forms with sources
constexpr int z_reg_tile(int form) { return form == kVacuum ? 16 : 8; }

// fields_in * tile (slot, column) FFTs per tile, a thread pair each, rounded
// up to whole warps; the forms with sources (8-column tiles, 144 or 160 pair
// threads) take 192 threads, so that the update stage's (column pair, k)
// items divide evenly among them for the z lengths 48 and 96 (one and two per
// thread) and 6 warps are resident per CTA.  The pairs past the last slot
// skip the transforms.
template <int FORM>
constexpr int z_reg_threads() {
  return FORM == kVacuum ? (2 * fields_in(FORM) * z_reg_tile(FORM) + 31) / 32 * 32 : 192;
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
template <int NZ, int FORM, int NT = z_reg_threads<FORM>()>
__device__ __forceinline__ void prefetch_z_tile(const DevPlan& P, const float2* spec, int64_t sstride,
                                                const ColJob& J) {
  constexpr int FIN = fields_in(FORM);
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

// k-space update of one z tile held in shared memory as the half-length
// spectra of the even z samples (rows [0, NZ/2)) and of the odd ones (rows
// [NZ/2, NZ)), pitch NP: column pair (2 tp, 2 tp + 1), tp = tid % (TX/2),
// modes k and k + H for k = tid / (TX/2) + i NT/(TX/2) (unrolled), with the
// radix-2 stages of both z transforms.  A pair whose second column is past
// the tile computes it on dead data (clamped table indices) and only writes
// dead shared memory.
template <int NZ, int FORM, int TX, int NT, int NP>
__device__ __forceinline__ void z_tile_update(const DevPlan& P, float2* buf, const ColJob& J, bool nyq, int nm, int n1,
                                              const ShapeDev& sh, int nft) {
  constexpr int H = NZ / 2, TP = TX / 2, ZS = NT / TP, NIT = (H + ZS - 1) / ZS;
  static_assert(TX % 2 == 0 && NT % TP == 0, "column pairs");
  const int tid = threadIdx.x;
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

// One z tile (job J): the body of the register z kernels, for z length NZ.
template <int NZ, int FORM, int ZST>
__device__ __forceinline__ void z_reg_tile_job(const DevPlan& P, float2* spec, int64_t sstride, const ColJob& J,
                                               int nft, unsigned char* smem_raw) {
  constexpr int TX = z_reg_tile(FORM), FIN = fields_in(FORM), FOUT = fields_out(FORM);
  constexpr int NT = z_reg_threads<FORM>(), NP = z_reg_pitch(FORM);
  constexpr int H = NZ / 2;
  static_assert(NT % (2 * TX) == 0, "update threads keep one column");
  float2* buf = reinterpret_cast<float2*>(smem_raw);    // [row][slot * TX + t], pitch NP
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
  z_tile_update<NZ, FORM, TX, NT, NP>(P, buf, J, nyq, nm, n1, sh, nft);
  __syncthreads();
  // half-length inverse DFTs: member `half` gives the z samples 2m + half of
  // the output slots; threads of the remaining slots have nothing to do.
  // Only interior z planes are stored: the inverse plane pass reads no others.
  if (s < FOUT) {
    const int qo = 2 * s * TX + 4 * (t >> 1) + (t & 1);
    const int re = qo + 2 * half, im = qo + 2 - 2 * half;
#pragma unroll
    for (int k = 0; k < H; ++k) v[k] = make_float2(bw[(half * H + k) * 2 * NP + re], bw[(half * H + k) * 2 * NP + im]);
    Dft<float, H, 1>::run(v);
    if (live) {
      const int zlo = bx.ng_lo[2], zhi = NZ - bx.ng_hi[2];
      float2* dst = g + s * sstride + (int64_t)t * ts + half * zst;
#pragma unroll
      for (int m = 0; m < H; ++m) {
        const int z = 2 * m + half;
        if (z >= zlo && z < zhi) dst[2 * m * zst] = v[m];
      }
    }
  }
}

// One CTA per z tile, every box of the launch with z length NZ.
template <int NZ, int FORM, int ZST>
__global__ void __launch_bounds__(z_reg_threads<FORM>(), z_reg_min_blocks<FORM>())
    k_z_reg(DevPlan P, float2* spec, int64_t sstride, const ColJob* __restrict__ jobs, int nft, int njobs,
            int pf_dist) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const ColJob J = jobs[blockIdx.x];
  // the tile that a CTA launched about pf_dist blocks later will read: fetched
  // into L2 now, so that its loads hit L2 instead of waiting on HBM
  if (pf_dist > 0 && (int)blockIdx.x + pf_dist < njobs)
    prefetch_z_tile<NZ, FORM>(P, spec, sstride, jobs[blockIdx.x + pf_dist]);
  z_reg_tile_job<NZ, FORM, ZST>(P, spec, sstride, J, nft, smem_raw);
}

// z lengths with a register z kernel: X(NZ)
#define PSATD_REG_Z(X) X(96) X(48) X(60) X(80) X(120)

// Persistent form for a batch of boxes of several z lengths (the uneven
// batch): one launch, every CTA takes the jobs blockIdx.x, blockIdx.x +
// gridDim.x, ... in turn (no waiting between CTAs), dispatching on the job's
// z length, and prefetches into L2 the tile of its next job.
template <int FORM>
__global__ void __launch_bounds__(z_reg_threads<FORM>(), z_reg_min_blocks<FORM>())
    k_z_reg_multi(DevPlan P, float2* spec, int64_t sstride, const ColJob* __restrict__ jobs, int nft,
                  int njobs, int prefetch) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  for (int j = blockIdx.x; j < njobs; j += gridDim.x) {
    if (j != (int)blockIdx.x) __syncthreads();   // the previous job's shared-memory reads are done
    const ColJob J = jobs[j];
    const int nz = P.boxes[J.box].n[2];
    if (prefetch && j + (int)gridDim.x < njobs) {
      const ColJob Jn = jobs[j + gridDim.x];
      const int nzn = P.boxes[Jn.box].n[2];
#define PSATD_ZPF(NZV) \
  if (nzn == NZV) prefetch_z_tile<NZV, FORM>(P, spec, sstride, Jn);
      PSATD_REG_Z(PSATD_ZPF)
#undef PSATD_ZPF
    }
#define PSATD_ZJ(NZV) \
  if (nz == NZV) z_reg_tile_job<NZV, FORM, 0>(P, spec, sstride, J, nft, smem_raw);
    PSATD_REG_Z(PSATD_ZJ)
#undef PSATD_ZJ
  }
}


// ---------------------------------------------------------------------------
// Quad register z kernel, for z lengths whose half-length DFT is too long for
// one thread's registers (128, 192): four threads per (slot, column), lanes
// l, l ^ 8, l ^ 16, l ^ 24 of a warp (half = lane bit 4: even / odd z; sub =
// lane bit 3), each holding the samples 4j + 2 sub + half and running their
// length-NZ/4 DFT; the two sub members join their transforms by shuffles into
// the half-length spectrum of their half (rows of the pair kernel's layout),
// the update stage is the pair kernel's, and the inverse mirrors the forward
// (split by shuffles, length-NZ/4 inverse DFTs, interior z planes stored).
#define PSATD_REG_Z4(X) X(128) X(192)
// columns per tile: 8 (the 6-slot vacuum form), 4 with sources
constexpr int z_reg4_tile(int form) { return form == kVacuum ? 8 : 4; }
template <int FORM>
constexpr int z_reg4_threads() {
  return (4 * fields_in(FORM) * z_reg4_tile(FORM) + 31) / 32 * 32;
}
constexpr int z_reg4_pitch(int form) {
  return fields_in(form) * z_reg4_tile(form) + ((24 - (fields_in(form) * z_reg4_tile(form)) % 16) % 16);
}

template <int NZ, int FORM>
__device__ __forceinline__ void z_reg4_tile_job(const DevPlan& P, float2* spec, int64_t sstride, const ColJob& J,
                                                int nft, unsigned char* smem_raw) {
  constexpr int TX = z_reg4_tile(FORM), FIN = fields_in(FORM), FOUT = fields_out(FORM);
  constexpr int NT = z_reg4_threads<FORM>(), NP = z_reg4_pitch(FORM);
  constexpr int H = NZ / 2, Q = NZ / 4, Q2 = NZ / 8;
  static_assert(NZ % 8 == 0 && NT % (2 * TX) == 0, "quad z tile");
  float2* buf = reinterpret_cast<float2*>(smem_raw);    // [row][slot * TX + t], pitch NP
  const BoxDev bx = P.boxes[J.box];
  const ShapeDev& sh = P.shapes[bx.shape];
  const int hx = sh.hx, n1 = bx.n[1];
  const int64_t zst = (int64_t)n1 * hx;
  const bool nyq = J.nm < 0;
  const int nm = nyq ? -J.nm : J.nm, ts = nyq ? hx : 1;
  float2* g = spec + bx.soff + (int64_t)J.plane * hx + J.m0;
  const int tid = threadIdx.x, lane = tid & 31;
  const int half = (lane >> 4) & 1, sub = (lane >> 3) & 1, quad = (lane & 7) + ((tid >> 5) << 3);
  const int s = quad / TX, t = quad - s * TX;
  const bool live = t < nm && s < FIN;
  const int tc = t < nm ? t : 0, sc = s < FIN ? s : FIN - 1;
  const int zoff = 2 * sub + half;   // the member's samples: z = 4m + zoff
  float2 v[Q];
  {
    const float2* src = g + sc * sstride + (int64_t)tc * ts + zoff * zst;
#pragma unroll
    for (int m = 0; m < Q; ++m) v[m] = ld_l2_256(src + 4 * m * zst);
  }
  // forward: length-Q DFT, join of the two sub members into the half-length
  // spectrum rows half * H + k, k in {sub Q2 + i, sub Q2 + i + Q}; slots >= nft
  // hold a cached z spectrum in natural z order, stored as they are
  float* bw = reinterpret_cast<float*>(buf);
  const int q0 = 2 * s * TX + 4 * (t >> 1) + (t & 1);      // word of re in a re-first row
  // the lanes that transform (both sub members of a quad share s): the
  // shuffles of the join name exactly these
  const unsigned fmask = __ballot_sync(0xffffffffu, s < nft);
  if (s < nft) {
    Dft<float, Q, -1>::run(v);
    pair_join_inplace<H, -1, 8>(v, sub, fmask);
    const int re = q0 + 2 * half, im = q0 + 2 - 2 * half;
#pragma unroll
    for (int i = 0; i < Q2; ++i) {
      const int k1 = sub * Q2 + i, k2 = k1 + Q;
      bw[(half * H + k1) * 2 * NP + re] = v[i].x;
      bw[(half * H + k1) * 2 * NP + im] = v[i].y;
      bw[(half * H + k2) * 2 * NP + re] = v[Q2 + i].x;
      bw[(half * H + k2) * 2 * NP + im] = v[Q2 + i].y;
    }
  } else if (s < FIN) {
#pragma unroll
    for (int m = 0; m < Q; ++m) {
      const int z = 4 * m + zoff, sw = z >= H ? 2 : 0;
      bw[z * 2 * NP + q0 + sw] = v[m].x;
      bw[z * 2 * NP + q0 + 2 - sw] = v[m].y;
    }
  }
  __syncthreads();
  z_tile_update<NZ, FORM, TX, NT, NP>(P, buf, J, nyq, nm, n1, sh, nft);
  __syncthreads();
  // inverse: the member's rows of its half, split by shuffles, length-Q
  // inverse DFT -> the samples 4m + zoff of the output slots
  {
    const int so = s < FOUT ? s : FOUT - 1;
    const int qo = 2 * so * TX + 4 * (t >> 1) + (t & 1);
    const int re = qo + 2 * half, im = qo + 2 - 2 * half;
#pragma unroll
    for (int i = 0; i < Q2; ++i) {
      const int k1 = sub * Q2 + i, k2 = k1 + Q;
      v[i] = make_float2(bw[(half * H + k1) * 2 * NP + re], bw[(half * H + k1) * 2 * NP + im]);
      v[Q2 + i] = make_float2(bw[(half * H + k2) * 2 * NP + re], bw[(half * H + k2) * 2 * NP + im]);
    }
  }
  pair_split_inplace<H, 1, 8>(v, sub);
  Dft<float, Q, 1>::run(v);
  if (live && s < FOUT) {
    const int zlo = bx.ng_lo[2], zhi = NZ - bx.ng_hi[2];
    float2* dst = g + s * sstride + (int64_t)t * ts + zoff * zst;
#pragma unroll
    for (int m = 0; m < Q; ++m) {
      const int z = 4 * m + zoff;
      if (z >= zlo && z < zhi) dst[4 * m * zst] = v[m];
    }
  }
}

template <int NZ, int FORM>
__global__ void __launch_bounds__(z_reg4_threads<FORM>(), 2)
    k_z_reg4(DevPlan P, float2* spec, int64_t sstride, const ColJob* __restrict__ jobs, int nft, int njobs,
             int pf_dist) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const ColJob J = jobs[blockIdx.x];
  if (pf_dist > 0 && (int)blockIdx.x + pf_dist < njobs)
    prefetch_z_tile<NZ, FORM, z_reg4_threads<FORM>()>(P, spec, sstride, jobs[blockIdx.x + pf_dist]);
  z_reg4_tile_job<NZ, FORM>(P, spec, sstride, J, nft, smem_raw);
}

// ---------------------------------------------------------------------------
// z-only forward FFT in natural z order of `ns` slots (from slot 0 of `spec`)
// over z tiles of boxes with a thread-pair register z length: the spectrum of
// a constant current, computed once per push.  Thread pair per (slot,
// column): member `half` holds the samples 2m + half, runs their half-length
// DFT, and the pair joins by shuffles (lanes l, l ^ 16) into the outputs
// i + half NZ/4 and i + half NZ/4 + NZ/2, stored to every z plane.
constexpr int kZfwdTile = 8;   // columns per tile: the job lists' width with sources
template <int NZ>
__global__ void __launch_bounds__(64) k_z_fwd_pair(DevPlan P, float2* spec, int64_t sstride,
                                                   const ColJob* __restrict__ jobs, int ns) {
  constexpr int H = NZ / 2, Q = NZ / 4;
  static_assert(NZ % 4 == 0, "pair join");
  const ColJob J = jobs[blockIdx.x];
  const BoxDev bx = P.boxes[J.box];
  const int hx = P.shapes[bx.shape].hx;
  const int64_t zst = (int64_t)bx.n[1] * hx;
  const bool nyq = J.nm < 0;
  const int nm = nyq ? -J.nm : J.nm, ts = nyq ? hx : 1;
  float2* g = spec + bx.soff + (int64_t)J.plane * hx + J.m0;
  const int tid = threadIdx.x, half = pair_half(tid), col = pair_index(tid);
  const int s = col / kZfwdTile, t = col - s * kZfwdTile;
  const bool live = t < nm && s < ns;
  const int tc = t < nm ? t : 0, sc = s < ns ? s : ns - 1;
  float2 v[H];
  const float2* src = g + sc * sstride + (int64_t)tc * ts + half * zst;
#pragma unroll
  for (int m = 0; m < H; ++m) v[m] = src[2 * m * zst];
  Dft<float, H, -1>::run(v);
  pair_join_inplace<NZ, -1>(v, half);
  if (live) {
    float2* dst = g + s * sstride + (int64_t)t * ts;
#pragma unroll
    for (int i = 0; i < Q; ++i) {
      dst[(i + half * Q) * zst] = v[i];
      dst[(i + half * Q + H) * zst] = v[Q + i];
    }
  }
}
}  // namespace

static bool z_reg_quad(int n2) {
#define PSATD_ZC(NZV) \
  if (n2 == NZV) return true;
  PSATD_REG_Z4(PSATD_ZC)
#undef PSATD_ZC
  return false;
}

int z_reg_ok(int n2) {
#define PSATD_ZC(NZV) \
  if (n2 == NZV) return 1;
  PSATD_REG_Z(PSATD_ZC)
#undef PSATD_ZC
  return z_reg_quad(n2) ? 1 : 0;
}

int z_reg_multi_ok(int n2) {
#define PSATD_ZC(NZV) \
  if (n2 == NZV) return 1;
  PSATD_REG_Z(PSATD_ZC)
#undef PSATD_ZC
  return 0;
}

cudaError_t launch_z_fwd_pair(const DevPlan& P, void* spec, int64_t sstride, const ColJob* jobs, int64_t njobs,
                              int n2, int tile, int ns, cudaStream_t st) {
  if (njobs <= 0) return cudaSuccess;
  if (tile != kZfwdTile || ns < 1 || 2 * ns * kZfwdTile > 64) return cudaErrorInvalidValue;
  bool hit = false;
#define PSATD_ZW(NZV)                                                                                       \
  if (n2 == NZV) {                                                                                         \
    k_z_fwd_pair<NZV><<<(unsigned)njobs, 64, 0, st>>>(P, (float2*)spec, sstride, jobs, ns);                  \
    hit = true;                                                                                            \
  }
  PSATD_REG_Z(PSATD_ZW)
#undef PSATD_ZW
  return hit ? cudaGetLastError() : cudaErrorInvalidValue;
}

int z_reg_smem(int form, int n2) { return n2 * (z_reg_quad(n2) ? z_reg4_pitch(form) : z_reg_pitch(form)) * 8; }

int z_reg_tile_width(int form, int n2) { return z_reg_quad(n2) ? z_reg4_tile(form) : z_reg_tile(form); }

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
#define PSATD_ZL(NZV)                                                                                     \
  if (n2 == NZV) {                                                                                       \
    if (form == kVacuum)                                                                                 \
      k_z_reg4<NZV, kVacuum><<<grid, z_reg4_threads<kVacuum>(), smem, st>>>(P, (float2*)spec, sstride, jobs, \
                                                                            nft, (int)njobs, pf_dist);    \
    else if (form == kJForm)                                                                             \
      k_z_reg4<NZV, kJForm><<<grid, z_reg4_threads<kJForm>(), smem, st>>>(P, (float2*)spec, sstride, jobs,   \
                                                                          nft, (int)njobs, pf_dist);      \
    else                                                                                                 \
      k_z_reg4<NZV, kRhoForm><<<grid, z_reg4_threads<kRhoForm>(), smem, st>>>(P, (float2*)spec, sstride,     \
                                                                              jobs, nft, (int)njobs, pf_dist); \
  }
  PSATD_REG_Z4(PSATD_ZL)
#undef PSATD_ZL
  return cudaGetLastError();
}

cudaError_t launch_z_reg_multi(int form, const DevPlan& P, void* spec, int64_t sstride, const ColJob* jobs,
                               int64_t njobs, int grid, int prefetch, int nft, cudaStream_t st) {
  if (njobs <= 0) return cudaSuccess;
  int smem = 0;
#define PSATD_ZM(NZV) smem = smem > z_reg_smem(form, NZV) ? smem : z_reg_smem(form, NZV);
  PSATD_REG_Z(PSATD_ZM)
#undef PSATD_ZM
  const unsigned g = (unsigned)(grid < njobs ? grid : njobs);
  if (form == kVacuum)
    k_z_reg_multi<kVacuum><<<g, z_reg_threads<kVacuum>(), smem, st>>>(P, (float2*)spec, sstride, jobs, nft,
                                                                      (int)njobs, prefetch);
  else if (form == kJForm)
    k_z_reg_multi<kJForm><<<g, z_reg_threads<kJForm>(), smem, st>>>(P, (float2*)spec, sstride, jobs, nft,
                                                                    (int)njobs, prefetch);
  else
    k_z_reg_multi<kRhoForm><<<g, z_reg_threads<kRhoForm>(), smem, st>>>(P, (float2*)spec, sstride, jobs, nft,
                                                                        (int)njobs, prefetch);
  return cudaGetLastError();
}

int z_reg_multi_smem(int form) {
  int smem = 0;
#define PSATD_ZM(NZV) smem = smem > z_reg_smem(form, NZV) ? smem : z_reg_smem(form, NZV);
  PSATD_REG_Z(PSATD_ZM)
#undef PSATD_ZM
  return smem;
}

int reg_shape_code(int L, int n1) {
#define PSATD_RC(code, LV, NYV, PART) \
  if (L == LV && n1 == NYV) return code;
  PSATD_REG_SHAPES(PSATD_RC)
#undef PSATD_RC
  return -1;
}

// bytes of dynamic shared memory of the forward plane kernel: the real plane
int reg_fwd_smem(int code) {
#define PSATD_RS(code_, LV, NYV, PART) \
  if (code == code_) return NYV * row_pitch(2 * LV) * 4;
  PSATD_REG_SHAPES(PSATD_RS)
#undef PSATD_RS
  return 0;
}

// the spectrum plane, or at most NY interior rows of pitch row_pitch(n0)
int reg_inv_smem(int code) {
#define PSATD_RS(code_, LV, NYV, PART) \
  if (code == code_) return NYV * (LV + 1) * 8 > NYV * row_pitch(2 * LV) * 4 ? NYV * (LV + 1) * 8 \
                                                                            : NYV * row_pitch(2 * LV) * 4;
  PSATD_REG_SHAPES(PSATD_RS)
#undef PSATD_RS
  return 0;
}

static int reg_plane_part(int code) {
#define PSATD_RP(code_, LV, NYV, PART) \
  if (code == code_) return PART;
  PSATD_REG_SHAPES(PSATD_RP)
#undef PSATD_RP
  return -1;
}

cudaError_t launch_plane_fwd_reg(int code, const DevPlan& P, const FieldPtrs& f, int nf, void* spec,
                                 int64_t sstride, const int2* jobs, int64_t nplanes, const int* gstart,
                                 const GatherSeg* gsegs, const GatherGrid* ggrid, int ngather, cudaStream_t st) {
  switch (reg_plane_part(code)) {
    case 0: return plane_part0::launch_fwd(code, P, f, nf, spec, sstride, jobs, nplanes, gstart, gsegs, ggrid, ngather, st);
    case 1: return plane_part1::launch_fwd(code, P, f, nf, spec, sstride, jobs, nplanes, gstart, gsegs, ggrid, ngather, st);
    case 2: return plane_part2::launch_fwd(code, P, f, nf, spec, sstride, jobs, nplanes, gstart, gsegs, ggrid, ngather, st);
    case 3: return plane_part3::launch_fwd(code, P, f, nf, spec, sstride, jobs, nplanes, gstart, gsegs, ggrid, ngather, st);
    default: return cudaErrorInvalidValue;
  }
}

cudaError_t launch_plane_inv_reg(int code, const DevPlan& P, const FieldPtrs& f, int nf, void* spec,
                                 int64_t sstride, const int2* jobs, int64_t nplanes, const int* seg_start,
                                 const GuardSeg* segs, cudaStream_t st) {
  switch (reg_plane_part(code)) {
    case 0: return plane_part0::launch_inv(code, P, f, nf, spec, sstride, jobs, nplanes, seg_start, segs, st);
    case 1: return plane_part1::launch_inv(code, P, f, nf, spec, sstride, jobs, nplanes, seg_start, segs, st);
    case 2: return plane_part2::launch_inv(code, P, f, nf, spec, sstride, jobs, nplanes, seg_start, segs, st);
    case 3: return plane_part3::launch_inv(code, P, f, nf, spec, sstride, jobs, nplanes, seg_start, segs, st);
    default: return cudaErrorInvalidValue;
  }
}

// Dynamic shared memory limits of the register kernels: what each launch
// asks for (the gather table of the forward kernel is static shared memory
// on top of it); `smem` is the device's opt-in maximum.
cudaError_t configure_reg_kernels(int smem) {
  cudaError_t e = cudaSuccess;
  for (cudaError_t r : {plane_part0::configure(smem), plane_part1::configure(smem), plane_part2::configure(smem),
                        plane_part3::configure(smem)})
    if (r != cudaSuccess) e = r;
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
#define PSATD_ZA(NZV, F)                                                                                  \
  if (z_reg_smem(F, NZV) <= smem) {                                                                       \
    const cudaError_t r =                                                                                 \
        cudaFuncSetAttribute(k_z_reg4<NZV, F>, cudaFuncAttributeMaxDynamicSharedMemorySize, z_reg_smem(F, NZV)); \
    if (r != cudaSuccess) e = r;                                                                          \
  }
#define PSATD_ZS(NZV) PSATD_ZA(NZV, kVacuum) PSATD_ZA(NZV, kJForm) PSATD_ZA(NZV, kRhoForm)
  PSATD_REG_Z4(PSATD_ZS)
#undef PSATD_ZS
#undef PSATD_ZA
#define PSATD_ZMA(F)                                                                                \
  if (z_reg_multi_smem(F) <= smem) {                                                               \
    const cudaError_t r = cudaFuncSetAttribute(k_z_reg_multi<F>, cudaFuncAttributeMaxDynamicSharedMemorySize, \
                                               z_reg_multi_smem(F));                               \
    if (r != cudaSuccess) e = r;                                                                   \
  }
  PSATD_ZMA(kVacuum)
  PSATD_ZMA(kJForm)
  PSATD_ZMA(kRhoForm)
#undef PSATD_ZMA
  return e;
}

}  // namespace psatd
