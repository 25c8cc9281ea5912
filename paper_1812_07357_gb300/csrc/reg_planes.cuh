// Register-resident plane kernels (FP32) for boxes whose x half-length L and
// y length NY have register codelets (L, NY/2 in the codelet set, L <= 63,
// NY <= 128): every 1D FFT of a plane is done inside registers, so a plane
// costs two block barriers.
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
//
//   k_plane_*_wide   planes too wide for those (n0/2 > 60 or NY > 120): 2
//                    threads per row and 2 or 4 per column, each a register
//                    DFT of every 2nd (4th) sample, combined through shared
//                    memory.
//
// The shapes are instantiated in four translation units (reg_planes_<part>.cu,
// PSATD_PLANE_PART = part), each taking its share of PSATD_REG_SHAPES.
#pragma once
#include <cooperative_groups.h>

#include "reg_common.cuh"

namespace psatd {

// Register plane shapes X(code, L, NY, part): x half-lengths 24, 30, 40, 48, 60
// by y lengths 48, 60, 80, 96, 120 (code 0: the 96 x 96 plane of 96^3 boxes),
// and the wide planes 128 x 128 and 192 x 192 (k_plane_*_wide)
#define PSATD_REG_SHAPES(X)                                                                        \
  X(0, 48, 96, 0) X(1, 24, 48, 0) X(2, 24, 60, 0) X(3, 24, 80, 0) X(4, 24, 96, 0) X(5, 24, 120, 0) \
  X(6, 30, 48, 1) X(7, 30, 60, 1) X(8, 30, 80, 1) X(9, 30, 96, 1) X(10, 30, 120, 1)               \
  X(11, 40, 48, 1) X(12, 40, 60, 1) X(13, 40, 80, 1) X(14, 40, 96, 1) X(15, 40, 120, 1)           \
  X(16, 48, 48, 2) X(17, 48, 60, 2) X(18, 48, 80, 2) X(19, 48, 120, 2)                            \
  X(20, 60, 48, 2) X(21, 60, 60, 2) X(22, 60, 80, 2) X(23, 60, 96, 2) X(24, 60, 120, 2)                     \
  X(25, 64, 128, 3) X(26, 96, 192, 3)

namespace {

// Threads of the narrow plane kernels: one per row of the plane (x) and a
// pair per complex column of the y pass, where the two real columns (mx = 0
// and the x Nyquist column mx = L) share one complex column, so L columns
// take 2 L threads; rounded up to whole warps.
template <int L, int NY>
constexpr int reg_plane_threads() {
  return ((NY > 2 * L ? NY : 2 * L) + 31) / 32 * 32;
}
// register budget per thread: 128 up to the 96 x 96 plane, 168 above; the
// resident CTAs per SM that budget allows (at most 8)
template <int L, int NY>
constexpr int reg_plane_regs() {
  return (L <= 48 && NY <= 96) ? 128 : 168;
}
template <int L, int NY>
constexpr int reg_plane_min_blocks() {
  return 65536 / (reg_plane_threads<L, NY>() * reg_plane_regs<L, NY>()) < 8
             ? 65536 / (reg_plane_threads<L, NY>() * reg_plane_regs<L, NY>())
             : 8;
}

// The real N0 x NY plane J.y of field f into shared memory (pitch
// row_pitch(N0) floats), by NT threads: copied in whole from the box, or, with
// the deferred guard exchange, gathered from the cells that own it (a 3 x 3
// grid of rectangles, or the plane's rectangle list).  Ends with a barrier.
template <int N0, int NY, int NT>
__device__ __forceinline__ void plane_load(const DevPlan& P, const FieldPtrs& F, float* buf, const int2& J, int f,
                                           const BoxDev& bx, const int* __restrict__ gstart,
                                           const GatherSeg* __restrict__ gsegs, const GatherGrid* __restrict__ ggrid,
                                           int ngather) {
  constexpr int PF = row_pitch(N0);
  constexpr int UPR = N0 / 4;
  if (ggrid && f < ngather) {
    // deferred exchange, plane of at most 3 x 3 rectangles: thread t copies
    // the 16-byte column t % UPR of the rows t / UPR + k * RG
    constexpr int RG = NT / UPR;
    __shared__ GatherGrid gg;
    static_assert(sizeof(GatherGrid) / 4 <= NT, "one word per thread");
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
        for (int u = threadIdx.x; u < gs.ny * upr; u += NT) {
          const int r = fdiv(u, m), c = 4 * (u - r * upr);
          cp16(dst + r * PF + c, src + (int64_t)r * gs.spitch + c);
        }
      } else {
        const unsigned m = magic(gs.nx);
        for (int u = threadIdx.x; u < gs.ny * gs.nx; u += NT) {
          const int r = fdiv(u, m), c = u - r * gs.nx;
          cp4(dst + r * PF + c, src + (int64_t)r * gs.spitch + c);
        }
      }
    }
  } else {
    const float* g = reinterpret_cast<const float*>(F.p[f]) + bx.foff + (int64_t)J.y * NY * N0;
    for (int u = threadIdx.x; u < NY * UPR; u += NT) {
      const int r = u / UPR, x = u - r * UPR;
      cp16(buf + r * PF + 4 * x, g + 4 * u);
    }
  }
  cp_commit_wait_all();
  __syncthreads();
}

// ---------------------------------------------------------------------------
template <int L, int NY>
__global__ void __launch_bounds__(reg_plane_threads<L, NY>(), reg_plane_min_blocks<L, NY>())
    k_plane_fwd_reg(DevPlan P, FieldPtrs F, float2* spec, int64_t sstride, const int2* __restrict__ jobs,
                    const int* __restrict__ gstart, const GatherSeg* __restrict__ gsegs,
                    const GatherGrid* __restrict__ ggrid, int ngather) {
  constexpr int N0 = 2 * L, HX = L + 1, PF = row_pitch(N0), NT = reg_plane_threads<L, NY>();
  static_assert(NY <= NT && 2 * L <= NT, "one thread per row / per half column");
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ float2 wsc[NY];   // y transform of the packed real columns
  float* buf = reinterpret_cast<float*>(smem_raw);
  const int2 J = jobs[blockIdx.x];
  const int f = blockIdx.y;
  const BoxDev bx = P.boxes[J.x];
  plane_load<N0, NY, NT>(P, F, buf, J, f, bx, gstart, gsegs, ggrid, ngather);
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
        // X[0] and X[L] of a real row are real: stored together as the
        // complex value X[0] + i X[L] of column 0 (the y pass transforms the
        // two real columns as one complex column)
        xr[0] = make_float2(A.x + Bv.x, A.x - Bv.x);
      } else {
        xr[k] = A + cmul(root<N0, k, -1>(), Bv);
        if constexpr (2 * k != L) xr[L - k] = conjg(A) + cmul(root<N0, L - k, -1>(), conjg(Bv));
      }
    });
  }
  __syncthreads();
  // y: thread pair per complex column c in [0, L), column 0 holding the two
  // real columns X[.][0] + i X[.][L]; pairs past L repeat column 0 and store
  // nothing.  The packed pair stores its transform in shared memory.
  {
    const int t = threadIdx.x;
    const int half = pair_half(t), p = pair_index(t);
    const bool packed = p == 0, live = p < L;
    const int c = live ? p : 0;
    const float2* xs = reinterpret_cast<const float2*>(buf);
    float2 v[NY / 2];
#pragma unroll
    for (int m = 0; m < NY / 2; ++m) v[m] = xs[(2 * m + half) * (PF / 2) + c];
    Dft<float, NY / 2, -1>::run(v);
    float2* out = spec + f * sstride + bx.soff + (int64_t)J.y * NY * HX;
    float2* dst = packed ? wsc : out + c;
    const int ds = packed ? 1 : HX;
    pair_join<NY, -1>(v, half, [&](int y, float2 val) {
      if (live) dst[y * ds] = val;
    });
    // the packed pair is lanes 0 and 16 of warp 0: warp 0 splits its transform
    // W = F0 + i FL into the spectra of the two real columns,
    // F0[k] = (W[k] + conj W[-k])/2, FL[k] = (W[k] - conj W[-k])/(2i)
    if (t < 32) {
      __syncwarp();
      for (int k = t; k < NY; k += 32) {
        const float2 a = wsc[k], b = wsc[k == 0 ? 0 : NY - k];
        out[k * HX] = make_float2(0.5f * (a.x + b.x), 0.5f * (a.y - b.y));
        out[k * HX + L] = make_float2(0.5f * (a.y + b.y), 0.5f * (b.x - a.x));
      }
    }
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

// The interior cells of a plane (rows: ni interior rows of pitch
// row_pitch(N0) floats in shared memory, the first interior cell at xlo) to
// field f of their box, then the guard rectangles this plane feeds in other
// boxes (seg_start: CSR of the guard segments per plane job), by NT threads.
template <int N0, int NY, int NT>
__device__ __forceinline__ void plane_store(const DevPlan& P, const FieldPtrs& F, const float* rows, const int2& J,
                                            int f, const BoxDev& bx, int ylo, int ni, int xlo, int nxi,
                                            bool vec_rows, const int* __restrict__ seg_start,
                                            const GuardSeg* __restrict__ segs) {
  constexpr int PF = row_pitch(N0);
  // interior cells to this box, then the guard cells this plane feeds
  float* fbase = reinterpret_cast<float*>(F.p[f]);
  float* own = fbase + bx.foff + ((int64_t)J.y * NY + ylo) * N0 + xlo;
  if (vec_rows)
    copy_rect_w<float4>(rows, PF, own, N0, ni, nxi, threadIdx.x, NT);
  else
    copy_rect_w<float>(rows, PF, own, N0, ni, nxi, threadIdx.x, NT);
  if (seg_start) {
    const int p = blockIdx.x;
    const int s1 = seg_start[p + 1];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = NT >> 5;
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

template <int L, int NY>
__global__ void __launch_bounds__(reg_plane_threads<L, NY>(), reg_plane_min_blocks<L, NY>())
    k_plane_inv_reg(DevPlan P, FieldPtrs F, const float2* spec, int64_t sstride, const int2* __restrict__ jobs,
                    const int* __restrict__ seg_start, const GuardSeg* __restrict__ segs) {
  constexpr int N0 = 2 * L, HX = L + 1, PF = row_pitch(N0), Q = NY / 4, NT = reg_plane_threads<L, NY>();
  static_assert(NY <= NT && 2 * L <= NT, "one thread per row / per half column");
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
  for (int u = threadIdx.x; u < UNITS; u += NT) cp16(sp + 2 * u, g + 2 * u);
  cp_commit_wait_all();
  __syncthreads();
  // column 0 <- X[.][0] + i X[.][L]: the two columns whose y transforms are
  // real (Hermitian in y), transformed as one complex column
  if (threadIdx.x < NY) {
    const float2 a = sp[threadIdx.x * HX], b = sp[threadIdx.x * HX + L];
    sp[threadIdx.x * HX] = make_float2(a.x - b.y, a.y + b.x);
  }
  __syncthreads();
  // y: thread pair per complex column c in [0, L), inverse (column 0: the
  // real and imaginary parts of its result are the two real columns, left
  // packed as x0 + i xL); pairs past L repeat column 0 and store nothing.
  // Outputs kept in v until the plane is consumed.
  const int t = threadIdx.x;
  const int half = pair_half(t), p = pair_index(t);
  const bool live = p < L;
  const int c = live ? p : 0;
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
    // Z'[k] = (X[k] + conj X[L-k]) + i w^-k (X[k] - conj X[L-k]), w = exp(-2 pi i / N0);
    // k = 0 from the real X[0], X[L] packed in column 0: Z'[0] = (X0 + XL) + i (X0 - XL)
    static_for<0, L / 2 + 1>([&](auto kc) {
      constexpr int k = decltype(kc)::value;
      if constexpr (k == 0) {
        const float2 a = xr[0];
        z[0] = make_float2(a.x + a.y, a.x - a.y);
      } else {
        const float2 a = xr[k], b = xr[L - k];
        z[k] = (a + conjg(b)) + times_i(cmul(a - conjg(b), root<N0, k, 1>()));
        if constexpr (2 * k != L) z[L - k] = (b + conjg(a)) + times_i(cmul(b - conjg(a), root<N0, L - k, 1>()));
      }
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
  plane_store<N0, NY, NT>(P, F, rows, J, f, bx, ylo, ni, xlo, nxi, vec_rows, seg_start, segs);
}

// ---------------------------------------------------------------------------
// Wide register plane kernels: planes too wide for one thread per row
// (n0/2 > 60) or a thread pair per column (n1 > 120).  GX threads share a row
// and GY a column; each does the length-L/GX (NY/GY) register DFT of every
// GX-th (GY-th) sample, twiddled, and the GX- (GY-) point combination of the
// partial transforms goes through shared memory (decimation in time:
// X[k + (R/G) p] = sum_q w_R^{q k} w_G^{q p} DFT_{R/G}(x[G j + q])[k]).
template <int L, int NY>
constexpr bool plane_is_wide() {
  return L > 60 || NY > 120;
}
template <int L, int NY>
constexpr int wide_gx() {
  return L > 60 ? 2 : 1;
}
template <int L, int NY>
constexpr int wide_gy() {
  return NY > 120 ? 4 : 2;
}
template <int L, int NY>
constexpr int wide_threads() {
  constexpr int a = NY * wide_gx<L, NY>(), b = (L + 1) * wide_gy<L, NY>();
  return ((a > b ? a : b) + 31) / 32 * 32;
}
// one CTA per SM above 113 KB of shared memory, else two
template <int L, int NY>
constexpr int wide_min_blocks() {
  return NY * row_pitch(2 * L) * 4 > 113 * 1024 ? 1 : 2;
}
// threads of a plane CTA of either kind
template <int L, int NY>
constexpr int plane_threads() {
  if constexpr (plane_is_wide<L, NY>())
    return wide_threads<L, NY>();
  else
    return kRegThreads;
}

// w_R^(q K) (sign DIR) for a run-time q < G <= 4 and a compile-time K
template <int R, int K, int G, int DIR>
__device__ __forceinline__ float2 root_q(int q) {
  float2 w = make_float2(1.f, 0.f);
  if constexpr (G > 1) w = q == 1 ? root<R, K % R, DIR>() : w;
  if constexpr (G > 2) w = q == 2 ? root<R, (2 * K) % R, DIR>() : w;
  if constexpr (G > 3) w = q == 3 ? root<R, (3 * K) % R, DIR>() : w;
  return w;
}

template <int L, int NY>
__global__ void __launch_bounds__(wide_threads<L, NY>(), wide_min_blocks<L, NY>())
    k_plane_fwd_wide(DevPlan P, FieldPtrs F, float2* spec, int64_t sstride, const int2* __restrict__ jobs,
                     const int* __restrict__ gstart, const GatherSeg* __restrict__ gsegs,
                     const GatherGrid* __restrict__ ggrid, int ngather) {
  constexpr int N0 = 2 * L, HX = L + 1, PF = row_pitch(N0), PC = PF / 2;
  constexpr int GX = wide_gx<L, NY>(), GY = wide_gy<L, NY>(), NT = wide_threads<L, NY>();
  constexpr int LX = L / GX, LY = NY / GY, LXP = GX > 1 ? LX + 1 : LX;
  static_assert(L % GX == 0 && NY % GY == 0 && LY % GY == 0 && GX * LXP <= PC, "wide plane shape");
  extern __shared__ __align__(16) unsigned char smem_raw[];
  float* buf = reinterpret_cast<float*>(smem_raw);
  float2* cb = reinterpret_cast<float2*>(smem_raw);
  const int2 J = jobs[blockIdx.x];
  const int f = blockIdx.y;
  const BoxDev bx = P.boxes[J.x];
  plane_load<N0, NY, NT>(P, F, buf, J, f, bx, gstart, gsegs, ggrid, ngather);
  const int t = threadIdx.x;
  // x, stage 1: thread (row r, q): DFT of the packed samples z[q + GX j]
  // (z[m] = x[2m] + i x[2m+1]), twiddled; back into the row at q * LXP + k
  {
    const int r = t / GX, q = t - r * GX;
    const bool live = r < NY;
    float2 v[LX];
    if (live) {
      const float2* row = cb + r * PC;
#pragma unroll
      for (int j = 0; j < LX; ++j) v[j] = row[q + GX * j];
      Dft<float, LX, -1>::run(v);
      static_for<1, LX>([&](auto kc) {
        constexpr int k = decltype(kc)::value;
        v[k] = cmul(v[k], root_q<L, k, GX, -1>(q));
      });
    }
    __syncthreads();
    if (live) {
      float2* row = cb + r * PC + q * LXP;
#pragma unroll
      for (int k = 0; k < LX; ++k) row[k] = v[k];
    }
  }
  __syncthreads();
  // x, stage 2: Z[k] = sum_p w_GX^{p (k / LX)} Z_p[k mod LX], then the R2C
  // split X[k] = (Z[k] + conj Z[L-k])/2 - i w^k (Z[k] - conj Z[L-k])/2
  // (w = exp(-2 pi i / N0)) for k = q + GX j <= L/2 and its partner L - k
  {
    const int r = t / GX, q = t - r * GX;
    const bool live = r < NY;
    constexpr int NK = (L / 2 + GX) / GX;   // k = q + GX j, j < NK (some past L/2)
    float2 lo[NK], hi[NK];
    if (live) {
      const float2* row = cb + r * PC;
      auto zval = [&](int k) {   // Z[k], 0 <= k < L
        const int kk = k % LX, p = k / LX;
        float2 a[GX];
#pragma unroll
        for (int s = 0; s < GX; ++s) a[s] = row[s * LXP + kk];
        float2 z = a[0];
#pragma unroll
        for (int s = 1; s < GX; ++s) {
          // w_GX^{s p}: GX <= 2 here, so +-1
          z = (s * p) % 2 ? z - a[s] : z + a[s];
        }
        return z;
      };
      static_for<0, NK>([&](auto jc) {
        constexpr int j = decltype(jc)::value;
        const int k = q + GX * j;
        if (k <= L / 2) {
          const float2 a = zval(k), b = zval((L - k) % L);
          const float2 A = make_float2(0.5f * (a.x + b.x), 0.5f * (a.y - b.y));
          const float2 Bv = make_float2(0.5f * (a.y + b.y), 0.5f * (b.x - a.x));
          // w^k and w^(L-k) for k = GX j + q (q < GX <= 2)
          const float2 wk = GX > 1 && q == 1 ? root<N0, GX * j + 1, -1>() : root<N0, GX * j, -1>();
          const float2 wl = GX > 1 && q == 1 ? root<N0, L - GX * j - 1, -1>() : root<N0, L - GX * j, -1>();
          if (k == 0) {
            lo[j] = make_float2(A.x + Bv.x, A.y + Bv.y);
            hi[j] = make_float2(A.x - Bv.x, A.y - Bv.y);
          } else {
            lo[j] = A + cmul(wk, Bv);
            hi[j] = conjg(A) + cmul(wl, conjg(Bv));
          }
        }
      });
    }
    static_assert(GX <= 2, "the x combination handles GX <= 2");
    __syncthreads();
    if (live) {
      float2* row = cb + r * PC;
      static_for<0, NK>([&](auto jc) {
        constexpr int j = decltype(jc)::value;
        const int k = q + GX * j;
        if (k <= L / 2) {
          row[k] = lo[j];
          if (k == 0) row[L] = hi[j];
          else if (2 * k != L) row[L - k] = hi[j];
        }
      });
    }
  }
  __syncthreads();
  // y, stage 1: thread (column c, q): DFT of the rows q + GY j, twiddled;
  // back into rows q * LY + k
  {
    const int q = t / HX, c = t - q * HX;
    const bool live = q < GY;
    float2 v[LY];
    if (live) {
#pragma unroll
      for (int j = 0; j < LY; ++j) v[j] = cb[(q + GY * j) * PC + c];
      Dft<float, LY, -1>::run(v);
      static_for<1, LY>([&](auto kc) {
        constexpr int k = decltype(kc)::value;
        v[k] = cmul(v[k], root_q<NY, k, GY, -1>(q));
      });
    }
    __syncthreads();
    if (live) {
#pragma unroll
      for (int k = 0; k < LY; ++k) cb[(q * LY + k) * PC + c] = v[k];
    }
  }
  __syncthreads();
  // y, stage 2: thread (c, q) combines k in [q LY/GY, (q+1) LY/GY) over the
  // GY partial transforms and stores rows k + LY p of the spectrum plane
  {
    const int q = t / HX, c = t - q * HX;
    if (q < GY) {
      float2* out = spec + f * sstride + bx.soff + (int64_t)J.y * NY * HX + c;
      constexpr int KQ = LY / GY;
#pragma unroll
      for (int i = 0; i < KQ; ++i) {
        const int k = q * KQ + i;
        float2 a[GY];
#pragma unroll
        for (int p = 0; p < GY; ++p) a[p] = cb[(p * LY + k) * PC + c];
        Dft<float, GY, -1>::run(a);
#pragma unroll
        for (int p = 0; p < GY; ++p) out[(k + LY * p) * HX] = a[p];
      }
    }
  }
}

template <int L, int NY>
__global__ void __launch_bounds__(wide_threads<L, NY>(), wide_min_blocks<L, NY>())
    k_plane_inv_wide(DevPlan P, FieldPtrs F, const float2* spec, int64_t sstride, const int2* __restrict__ jobs,
                     const int* __restrict__ seg_start, const GuardSeg* __restrict__ segs) {
  constexpr int N0 = 2 * L, HX = L + 1, PF = row_pitch(N0), PC = PF / 2;
  constexpr int GX = wide_gx<L, NY>(), GY = wide_gy<L, NY>(), NT = wide_threads<L, NY>();
  constexpr int LX = L / GX, LY = NY / GY, LXP = GX > 1 ? LX + 1 : LX;
  static_assert(GX <= 2 && LX % GX == 0 && LY % GY == 0 && GX * LXP <= PC, "wide plane shape");
  extern __shared__ __align__(16) unsigned char smem_raw[];
  // one buffer: first the NY x HX spectrum plane (pitch HX), then the interior
  // rows (pitch PF floats)
  float2* sp = reinterpret_cast<float2*>(smem_raw);
  float2* cb = reinterpret_cast<float2*>(smem_raw);
  float* rows = reinterpret_cast<float*>(smem_raw);
  const int2 J = jobs[blockIdx.x];
  const int f = blockIdx.y;
  const BoxDev bx = P.boxes[J.x];
  const int ylo = bx.ng_lo[1], yhi = NY - bx.ng_hi[1], ni = yhi - ylo;
  const int xlo = bx.ng_lo[0], nxi = N0 - bx.ng_lo[0] - bx.ng_hi[0];
  {
    const float2* g = spec + f * sstride + bx.soff + (int64_t)J.y * NY * HX;
    constexpr int UNITS = NY * HX / 2;   // 16-byte units of the contiguous plane
    for (int u = threadIdx.x; u < UNITS; u += NT) cp16(sp + 2 * u, g + 2 * u);
    cp_commit_wait_all();
    __syncthreads();
  }
  const int t = threadIdx.x;
  // y, stage 1 (inverse): thread (c, q): DFT of rows q + GY j, twiddled
  {
    const int q = t / HX, c = t - q * HX;
    const bool live = q < GY;
    float2 v[LY];
    if (live) {
#pragma unroll
      for (int j = 0; j < LY; ++j) v[j] = sp[(q + GY * j) * HX + c];
      Dft<float, LY, 1>::run(v);
      static_for<1, LY>([&](auto kc) {
        constexpr int k = decltype(kc)::value;
        v[k] = cmul(v[k], root_q<NY, k, GY, 1>(q));
      });
    }
    __syncthreads();
    if (live) {
#pragma unroll
      for (int k = 0; k < LY; ++k) sp[(q * LY + k) * HX + c] = v[k];
    }
  }
  __syncthreads();
  // y, stage 2: combination; interior rows kept in registers until the plane
  // is consumed, then stored as rows of pitch PF floats
  {
    const int q = t / HX, c = t - q * HX;
    const bool live = q < GY;
    constexpr int KQ = LY / GY;
    float2 a[KQ][GY];
    if (live) {
#pragma unroll
      for (int i = 0; i < KQ; ++i) {
        const int k = q * KQ + i;
#pragma unroll
        for (int p = 0; p < GY; ++p) a[i][p] = sp[(p * LY + k) * HX + c];
        Dft<float, GY, 1>::run(a[i]);
      }
    }
    __syncthreads();
    if (live) {
#pragma unroll
      for (int i = 0; i < KQ; ++i) {
#pragma unroll
        for (int p = 0; p < GY; ++p) {
          const int y = q * KQ + i + LY * p;
          if (y >= ylo && y < yhi) cb[(y - ylo) * PC + c] = a[i][p];
        }
      }
    }
  }
  __syncthreads();
  // x, stage 1 (interior rows): thread (r, q): C2R merge
  // Z'[k] = (X[k] + conj X[L-k]) + i w^-k (X[k] - conj X[L-k]) at k = q + GX j,
  // inverse DFT over j, twiddled; back into the row at q * LXP + k
  {
    const int r = t / GX, q = t - r * GX;
    const bool live = r < ni;
    float2 v[LX];
    if (live) {
      const float2* xr = cb + r * PC;
      static_for<0, LX>([&](auto jc) {
        constexpr int j = decltype(jc)::value;
        const int k = q + GX * j;
        const float2 a = xr[k], b = xr[L - k];
        const float2 w = GX > 1 && q == 1 ? root<N0, GX * j + 1, 1>() : root<N0, GX * j, 1>();
        v[j] = (a + conjg(b)) + times_i(cmul(a - conjg(b), w));
      });
      Dft<float, LX, 1>::run(v);
      static_for<1, LX>([&](auto kc) {
        constexpr int k = decltype(kc)::value;
        v[k] = cmul(v[k], root_q<L, k, GX, 1>(q));
      });
    }
    __syncthreads();
    if (live) {
      float2* row = cb + r * PC + q * LXP;
#pragma unroll
      for (int k = 0; k < LX; ++k) row[k] = v[k];
    }
  }
  __syncthreads();
  // x, stage 2: z[m + LX p] = sum_s w_GX^{s p} Z_s[m] for m in the thread's
  // share; cells 2m, 2m+1 (interior ones) written back into the row from x = 0
  const float scale = __frcp_rn((float)(N0 * NY * bx.n[2]));   // exact integer < 2^24
  {
    const int r = t / GX, q = t - r * GX;
    const bool live = r < ni;
    constexpr int MQ = LX / GX;
    float2 z[MQ][GX];
    if (live) {
      const float2* row = cb + r * PC;
#pragma unroll
      for (int i = 0; i < MQ; ++i) {
        const int m = q * MQ + i;
        float2 a[GX];
#pragma unroll
        for (int s = 0; s < GX; ++s) a[s] = row[s * LXP + m];
        Dft<float, GX, 1>::run(a);
#pragma unroll
        for (int p = 0; p < GX; ++p) z[i][p] = a[p];
      }
    }
    __syncthreads();
    if (live) {
      float* o = rows + r * PF - xlo;
#pragma unroll
      for (int i = 0; i < MQ; ++i) {
#pragma unroll
        for (int p = 0; p < GX; ++p) {
          const int x = 2 * (q * MQ + i + LX * p);
          if (x >= xlo && x < xlo + nxi) o[x] = scale * z[i][p].x;
          if (x + 1 >= xlo && x + 1 < xlo + nxi) o[x + 1] = scale * z[i][p].y;
        }
      }
    }
  }
  __syncthreads();
  const bool vec_rows = (nxi % 4 == 0) && (xlo % 4 == 0);
  plane_store<N0, NY, NT>(P, F, rows, J, f, bx, ylo, ni, xlo, nxi, vec_rows, seg_start, segs);
}


// ---------------------------------------------------------------------------
// Split wide forward plane kernel (planes above 113 KB: the 192 x 192 plane):
// a cluster of two CTAs per plane, CTA rank h holding rows [h NY/2, (h+1) NY/2)
// in its shared memory (half the plane, so that two CTAs fit an SM and one
// CTA's loads overlap the other's transforms).  Each CTA does the x pass of
// its rows; after a cluster barrier, the y pass of its half of the columns,
// reading the other half of the rows from the peer CTA's shared memory
// (distributed shared memory); a second cluster barrier before the buffers
// are reused for the y combination.
template <int L, int NY>
constexpr bool plane_is_split() {
  return plane_is_wide<L, NY>() && NY * row_pitch(2 * L) * 4 > 113 * 1024;
}
template <int L, int NY>
constexpr int split_cols() {   // columns of rank 0 (rank 1: the rest)
  return (L + 2) / 2;
}
template <int L, int NY>
constexpr int split_threads() {
  constexpr int a = (NY / 2) * wide_gx<L, NY>(), b = split_cols<L, NY>() * wide_gy<L, NY>();
  return ((a > b ? a : b) + 31) / 32 * 32;
}
template <int L, int NY>
constexpr int split_smem() {
  constexpr int rows = (NY / 2) * row_pitch(2 * L) * 4, cols = NY * split_cols<L, NY>() * 8;
  return rows > cols ? rows : cols;
}

// Rows [r0, r0 + NR) of the real N0 x NY plane J.y of field f into shared
// memory (row r at buf + (r - r0) * row_pitch(N0)), by NT threads, as
// plane_load (pj: the plane job's index in the gather tables).
template <int N0, int NY, int NT, int NR>
__device__ __forceinline__ void plane_load_rows(const FieldPtrs& F, float* buf, const int2& J, int f,
                                                const BoxDev& bx, int pj, int r0,
                                                const int* __restrict__ gstart, const GatherSeg* __restrict__ gsegs,
                                                const GatherGrid* __restrict__ ggrid, int ngather) {
  constexpr int PF = row_pitch(N0);
  constexpr int UPR = N0 / 4;
  const int r1 = r0 + NR;
  if (ggrid && f < ngather) {
    constexpr int RG = NT / UPR;
    __shared__ GatherGrid gg;
    static_assert(sizeof(GatherGrid) / 4 <= NT, "one word per thread");
    if (threadIdx.x < sizeof(GatherGrid) / 4)
      reinterpret_cast<int*>(&gg)[threadIdx.x] = reinterpret_cast<const int*>(ggrid + pj)[threadIdx.x];
    __syncthreads();
    if (threadIdx.x < RG * UPR) {
      const float* fb = reinterpret_cast<const float*>(F.p[f]);
      const int c = threadIdx.x % UPR, rg = threadIdx.x / UPR, x = 4 * c;
      const int ix = (x >= gg.x1) + (x >= gg.x2);
      const int xo = x - (ix == 0 ? 0 : ix == 1 ? gg.x1 : gg.x2);
#pragma unroll
      for (int iy = 0; iy < 3; ++iy) {   // row bands [ylo, yhi), clipped to [r0, r1)
        const int ylo = iy == 0 ? 0 : iy == 1 ? gg.y1 : gg.y2;
        const int yhi = iy == 0 ? gg.y1 : iy == 1 ? gg.y2 : NY;
        const int a = max(ylo, r0), b = min(yhi, r1);
        int r = a + (rg - a % RG + RG) % RG;   // first row >= a with r % RG == rg
        const int pitch = gg.pitch[3 * iy + ix];
        const float* src = fb + gg.base[3 * iy + ix] + (int64_t)(r - ylo) * pitch + xo;
        const int64_t sstep = (int64_t)RG * pitch;
        for (float* dst = buf + (r - r0) * PF + x; r < b; r += RG, src += sstep, dst += RG * PF) cp16(dst, src);
      }
    }
  } else if (gstart && f < ngather) {
    __shared__ GatherSeg tab[kGatherTab];
    const float* fb = reinterpret_cast<const float*>(F.p[f]);
    const int s0 = gstart[pj], ns = gstart[pj + 1] - s0;
    if (threadIdx.x < kGatherTab && threadIdx.x < ns) tab[threadIdx.x] = gsegs[s0 + threadIdx.x];
    __syncthreads();
    for (int i = 0; i < ns; ++i) {
      const GatherSeg gs = i < kGatherTab ? tab[i] : gsegs[s0 + i];
      const int a = max(gs.dy, r0), b = min(gs.dy + gs.ny, r1);
      if (a >= b) continue;
      const int ny = b - a;
      const float* src = fb + gs.src_off + (int64_t)(a - gs.dy) * gs.spitch;
      float* dst = buf + (a - r0) * PF + gs.dx;
      if (gs.vec) {
        const int upr = gs.nx >> 2;
        const unsigned m = magic(upr);
        for (int u = threadIdx.x; u < ny * upr; u += NT) {
          const int r = fdiv(u, m), c = 4 * (u - r * upr);
          cp16(dst + r * PF + c, src + (int64_t)r * gs.spitch + c);
        }
      } else {
        const unsigned m = magic(gs.nx);
        for (int u = threadIdx.x; u < ny * gs.nx; u += NT) {
          const int r = fdiv(u, m), c = u - r * gs.nx;
          cp4(dst + r * PF + c, src + (int64_t)r * gs.spitch + c);
        }
      }
    }
  } else {
    const float* g = reinterpret_cast<const float*>(F.p[f]) + bx.foff + ((int64_t)J.y * NY + r0) * N0;
    for (int u = threadIdx.x; u < NR * UPR; u += NT) {
      const int r = u / UPR, x = u - r * UPR;
      cp16(buf + r * PF + 4 * x, g + 4 * u);
    }
  }
  cp_commit_wait_all();
  __syncthreads();
}

template <int L, int NY>
__global__ void __cluster_dims__(2, 1, 1) __launch_bounds__(split_threads<L, NY>(), 2)
    k_plane_fwd_split(DevPlan P, FieldPtrs F, float2* spec, int64_t sstride, const int2* __restrict__ jobs,
                      const int* __restrict__ gstart, const GatherSeg* __restrict__ gsegs,
                      const GatherGrid* __restrict__ ggrid, int ngather) {
  constexpr int N0 = 2 * L, HX = L + 1, PF = row_pitch(N0), PC = PF / 2;
  constexpr int GX = wide_gx<L, NY>(), GY = wide_gy<L, NY>(), NT = split_threads<L, NY>();
  constexpr int LX = L / GX, LY = NY / GY, LXP = GX > 1 ? LX + 1 : LX;
  constexpr int NH = NY / 2, C0 = split_cols<L, NY>(), CP = C0;
  static_assert(GX == 2 && NY % (2 * GY) == 0 && LY % GY == 0 && GX * LXP <= PC && LY % 2 == 0,
                "split wide plane shape");
  namespace cg = cooperative_groups;
  cg::cluster_group cluster = cg::this_cluster();
  extern __shared__ __align__(16) unsigned char smem_raw[];
  float* buf = reinterpret_cast<float*>(smem_raw);
  float2* cb = reinterpret_cast<float2*>(smem_raw);
  const int h = (int)cluster.block_rank();
  const int pj = blockIdx.x >> 1;
  const int2 J = jobs[pj];
  const int f = blockIdx.y;
  const BoxDev bx = P.boxes[J.x];
  plane_load_rows<N0, NY, NT, NH>(F, buf, J, f, bx, pj, h * NH, gstart, gsegs, ggrid, ngather);
  const int t = threadIdx.x;
  // x, stage 1 on the CTA's rows (as k_plane_fwd_wide)
  {
    const int r = t / GX, q = t - r * GX;
    const bool live = r < NH;
    float2 v[LX];
    if (live) {
      const float2* row = cb + r * PC;
#pragma unroll
      for (int j = 0; j < LX; ++j) v[j] = row[q + GX * j];
      Dft<float, LX, -1>::run(v);
      static_for<1, LX>([&](auto kc) {
        constexpr int k = decltype(kc)::value;
        v[k] = cmul(v[k], root_q<L, k, GX, -1>(q));
      });
    }
    __syncthreads();
    if (live) {
      float2* row = cb + r * PC + q * LXP;
#pragma unroll
      for (int k = 0; k < LX; ++k) row[k] = v[k];
    }
  }
  __syncthreads();
  // x, stage 2: combination and R2C split (as k_plane_fwd_wide)
  {
    const int r = t / GX, q = t - r * GX;
    const bool live = r < NH;
    constexpr int NK = (L / 2 + GX) / GX;
    float2 lo[NK], hi[NK];
    if (live) {
      const float2* row = cb + r * PC;
      auto zval = [&](int k) {
        const int kk = k % LX, p = k / LX;
        const float2 a0 = row[kk], a1 = row[LXP + kk];
        return p ? a0 - a1 : a0 + a1;
      };
      static_for<0, NK>([&](auto jc) {
        constexpr int j = decltype(jc)::value;
        const int k = q + GX * j;
        if (k <= L / 2) {
          const float2 a = zval(k), b = zval((L - k) % L);
          const float2 A = make_float2(0.5f * (a.x + b.x), 0.5f * (a.y - b.y));
          const float2 Bv = make_float2(0.5f * (a.y + b.y), 0.5f * (b.x - a.x));
          const float2 wk = q == 1 ? root<N0, GX * j + 1, -1>() : root<N0, GX * j, -1>();
          const float2 wl = q == 1 ? root<N0, L - GX * j - 1, -1>() : root<N0, L - GX * j, -1>();
          if (k == 0) {
            lo[j] = make_float2(A.x + Bv.x, A.y + Bv.y);
            hi[j] = make_float2(A.x - Bv.x, A.y - Bv.y);
          } else {
            lo[j] = A + cmul(wk, Bv);
            hi[j] = conjg(A) + cmul(wl, conjg(Bv));
          }
        }
      });
    }
    __syncthreads();
    if (live) {
      float2* row = cb + r * PC;
      static_for<0, NK>([&](auto jc) {
        constexpr int j = decltype(jc)::value;
        const int k = q + GX * j;
        if (k <= L / 2) {
          row[k] = lo[j];
          if (k == 0) row[L] = hi[j];
          else if (2 * k != L) row[L - k] = hi[j];
        }
      });
    }
  }
  // every row of both halves transformed along x
  cluster.sync();
  // y, stage 1: thread (column c of this CTA's half, q): rows q + GY j, the
  // first NH/GY of them in rank 0's buffer, the rest in rank 1's
  const int c0 = h * C0, ncols = h ? HX - C0 : C0;
  const int q = t / CP, cl = t - q * CP;
  const bool ylive = q < GY && cl < ncols;
  float2 v[LY];
  {
    const float2* half0 = cluster.map_shared_rank(cb, 0);
    const float2* half1 = cluster.map_shared_rank(cb, 1);
    const int c = c0 + (ylive ? cl : 0);
    if (q < GY) {
#pragma unroll
      for (int j = 0; j < LY; ++j) {
        const int rr = q + GY * j;   // compile-time owner: rows < NH in rank 0
        v[j] = (j < LY / 2 ? half0 : half1)[(j < LY / 2 ? rr : rr - NH) * PC + c];
      }
      Dft<float, LY, -1>::run(v);
      static_for<1, LY>([&](auto kc) {
        constexpr int k = decltype(kc)::value;
        v[k] = cmul(v[k], root_q<NY, k, GY, -1>(q));
      });
    }
  }
  // both CTAs have read what they need of the other's rows
  cluster.sync();
  if (ylive) {
#pragma unroll
    for (int k = 0; k < LY; ++k) cb[(q * LY + k) * CP + cl] = v[k];
  }
  __syncthreads();
  // y, stage 2: combination, rows k + LY p of the spectrum plane, this CTA's columns
  if (ylive) {
    float2* out = spec + f * sstride + bx.soff + (int64_t)J.y * NY * HX + c0 + cl;
    constexpr int KQ = LY / GY;
#pragma unroll
    for (int i = 0; i < KQ; ++i) {
      const int k = q * KQ + i;
      float2 a[GY];
#pragma unroll
      for (int p = 0; p < GY; ++p) a[p] = cb[(p * LY + k) * CP + cl];
      Dft<float, GY, -1>::run(a);
#pragma unroll
      for (int p = 0; p < GY; ++p) out[(k + LY * p) * HX] = a[p];
    }
  }
}

}  // namespace

// ---------------------------------------------------------------------------
// The launchers of one part (PSATD_PLANE_PART): every shape of the part, by code.
#ifdef PSATD_PLANE_PART
#define PSATD_PART_CAT2(a, b) a##b
#define PSATD_PART_CAT(a, b) PSATD_PART_CAT2(a, b)
namespace {

// bytes of dynamic shared memory: the real plane with its row pitch (forward);
// the spectrum plane or the interior rows, whichever is larger (inverse)
template <int L, int NY>
constexpr int plane_fwd_bytes() {
  return NY * row_pitch(2 * L) * 4;
}
template <int L, int NY>
constexpr int plane_inv_bytes() {
  return NY * (L + 1) * 8 > NY * row_pitch(2 * L) * 4 ? NY * (L + 1) * 8 : NY * row_pitch(2 * L) * 4;
}

template <int CODE, int L, int NY, int PART>
bool plane_fwd_shape(int code, dim3 grid, const DevPlan& P, const FieldPtrs& f, void* spec, int64_t sstride,
                     const int2* jobs, const int* gstart, const GatherSeg* gsegs, const GatherGrid* ggrid,
                     int ngather, cudaStream_t st) {
  if constexpr (PART == PSATD_PLANE_PART) {
    if (code != CODE) return false;
    if constexpr (plane_is_split<L, NY>())
      k_plane_fwd_split<L, NY><<<dim3(2 * grid.x, grid.y), split_threads<L, NY>(), split_smem<L, NY>(), st>>>(
          P, f, (float2*)spec, sstride, jobs, gstart, gsegs, ggrid, ngather);
    else if constexpr (plane_is_wide<L, NY>())
      k_plane_fwd_wide<L, NY><<<grid, wide_threads<L, NY>(), plane_fwd_bytes<L, NY>(), st>>>(
          P, f, (float2*)spec, sstride, jobs, gstart, gsegs, ggrid, ngather);
    else
      k_plane_fwd_reg<L, NY><<<grid, reg_plane_threads<L, NY>(), plane_fwd_bytes<L, NY>(), st>>>(
          P, f, (float2*)spec, sstride, jobs, gstart, gsegs, ggrid, ngather);
    return true;
  } else {
    return false;
  }
}

template <int CODE, int L, int NY, int PART>
bool plane_inv_shape(int code, dim3 grid, const DevPlan& P, const FieldPtrs& f, void* spec, int64_t sstride,
                     const int2* jobs, const int* seg_start, const GuardSeg* segs, cudaStream_t st) {
  if constexpr (PART == PSATD_PLANE_PART) {
    if (code != CODE) return false;
    if constexpr (plane_is_wide<L, NY>())
      k_plane_inv_wide<L, NY><<<grid, wide_threads<L, NY>(), plane_inv_bytes<L, NY>(), st>>>(
          P, f, (const float2*)spec, sstride, jobs, seg_start, segs);
    else
      k_plane_inv_reg<L, NY><<<grid, reg_plane_threads<L, NY>(), plane_inv_bytes<L, NY>(), st>>>(
          P, f, (const float2*)spec, sstride, jobs, seg_start, segs);
    return true;
  } else {
    return false;
  }
}

template <int L, int NY, int PART>
void plane_configure_shape(int smem, cudaError_t* e) {
  if constexpr (PART == PSATD_PLANE_PART) {
    if (plane_fwd_bytes<L, NY>() > smem || plane_inv_bytes<L, NY>() > smem) return;
    cudaError_t r, r2;
    if constexpr (plane_is_split<L, NY>()) {
      r = cudaFuncSetAttribute(k_plane_fwd_split<L, NY>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                               split_smem<L, NY>());
      r2 = cudaFuncSetAttribute(k_plane_inv_wide<L, NY>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                plane_inv_bytes<L, NY>());
    } else if constexpr (plane_is_wide<L, NY>()) {
      r = cudaFuncSetAttribute(k_plane_fwd_wide<L, NY>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                               plane_fwd_bytes<L, NY>());
      r2 = cudaFuncSetAttribute(k_plane_inv_wide<L, NY>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                plane_inv_bytes<L, NY>());
    } else {
      r = cudaFuncSetAttribute(k_plane_fwd_reg<L, NY>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                               plane_fwd_bytes<L, NY>());
      r2 = cudaFuncSetAttribute(k_plane_inv_reg<L, NY>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                plane_inv_bytes<L, NY>());
      // the whole unified L1 as shared memory: room for every CTA the
      // register budget allows
      if (r == cudaSuccess)
        r = cudaFuncSetAttribute(k_plane_fwd_reg<L, NY>, cudaFuncAttributePreferredSharedMemoryCarveout, 100);
      if (r2 == cudaSuccess)
        r2 = cudaFuncSetAttribute(k_plane_inv_reg<L, NY>, cudaFuncAttributePreferredSharedMemoryCarveout, 100);
    }
    if (r != cudaSuccess) *e = r;
    if (r2 != cudaSuccess) *e = r2;
  }
}

}  // namespace

namespace PSATD_PART_CAT(plane_part, PSATD_PLANE_PART) {

cudaError_t launch_fwd(int code, const DevPlan& P, const FieldPtrs& f, int nf, void* spec, int64_t sstride,
                       const int2* jobs, int64_t nplanes, const int* gstart, const GatherSeg* gsegs,
                       const GatherGrid* ggrid, int ngather, cudaStream_t st) {
  if (nplanes <= 0 || nf <= 0) return cudaSuccess;
  const dim3 grid((unsigned)nplanes, nf);
#define PSATD_RL(c, LV, NYV, PART) \
  ||plane_fwd_shape<c, LV, NYV, PART>(code, grid, P, f, spec, sstride, jobs, gstart, gsegs, ggrid, ngather, st)
  const bool hit = false PSATD_REG_SHAPES(PSATD_RL);
#undef PSATD_RL
  return hit ? cudaGetLastError() : cudaErrorInvalidValue;
}

cudaError_t launch_inv(int code, const DevPlan& P, const FieldPtrs& f, int nf, void* spec, int64_t sstride,
                       const int2* jobs, int64_t nplanes, const int* seg_start, const GuardSeg* segs,
                       cudaStream_t st) {
  if (nplanes <= 0 || nf <= 0) return cudaSuccess;
  const dim3 grid((unsigned)nplanes, nf);
#define PSATD_RL(c, LV, NYV, PART) \
  ||plane_inv_shape<c, LV, NYV, PART>(code, grid, P, f, spec, sstride, jobs, seg_start, segs, st)
  const bool hit = false PSATD_REG_SHAPES(PSATD_RL);
#undef PSATD_RL
  return hit ? cudaGetLastError() : cudaErrorInvalidValue;
}

cudaError_t configure(int smem) {
  cudaError_t e = cudaSuccess;
#define PSATD_RC(c, LV, NYV, PART) plane_configure_shape<LV, NYV, PART>(smem, &e);
  PSATD_REG_SHAPES(PSATD_RC)
#undef PSATD_RC
  return e;
}

}  // namespace plane_part<PSATD_PLANE_PART>
#undef PSATD_PART_CAT
#undef PSATD_PART_CAT2
#endif  // PSATD_PLANE_PART

}  // namespace psatd
