// S4: guard-cell exchange between batched boxes (paper Fig. 1, step (ii)),
// and the dual-grid coupling copies between two layouts (paper Sec. 2.5.2).
//
// The host precomputes copy blocks, each a 3D region of guard cells of one
// box whose values live in the interior of one source box (or outside a
// non-periodic domain: zero).  A tile is a run of rows of one block; a row is
// ext[0] consecutive cells in both the source and the destination box.  Reads
// touch interior cells only and writes guard cells only, so tiles never race.
// Where both rows start on 16-byte boundaries and ext[0] fills whole 16-byte
// units, a thread moves 16 bytes at a time (XTile::vec > 1).
#include <cuda_runtime.h>

#include <algorithm>
#include <type_traits>

#include "psatd_internal.h"

namespace psatd {

namespace {

// Exact e / d for 0 <= e, d < 2^16 with m = floor((2^32 - 1)/d) + 1; for
// d = 1 that constant wraps to 0 and the quotient is e itself.
__device__ __forceinline__ int fdiv(int e, unsigned m) { return m ? (int)__umulhi((unsigned)e, m) : e; }

constexpr int kBatch = 4;   // units loaded before any is stored (bytes in flight)

template <typename T, int V>
__device__ __forceinline__ void copy_tile(T* dbase, const T* sbase, const CopyBlk& b, const XTile& t, const BoxDev& db,
                                          int64_t sfoff, int64_t sn0, int64_t sn1) {
  using Vec = typename std::conditional<V == 1, T, float4>::type;
  const int ex = b.ext[0], ey = b.ext[1];
  const int upr = ex / V;
  const unsigned m_upr = 0xFFFFFFFFu / (unsigned)upr + 1u, m_ey = 0xFFFFFFFFu / (unsigned)ey + 1u;
  const int64_t dn0 = db.n[0], dn1 = db.n[1];
  const int units = t.nrows * upr;
  const bool zero = b.src_box < 0;
  for (int u0 = threadIdx.x; u0 < units; u0 += kBatch * blockDim.x) {
    Vec v[kBatch];
    int64_t d[kBatch];
#pragma unroll
    for (int i = 0; i < kBatch; ++i) {
      const int u = u0 + i * blockDim.x;
      d[i] = -1;
      if (u < units) {
        const int rr = fdiv(u, m_upr);
        const int x = (u - rr * upr) * V;
        const int r = t.row0 + rr;
        const int rz = fdiv(r, m_ey);
        const int ry = r - rz * ey;
        d[i] = db.foff + ((int64_t)(b.dst_lo[2] + rz) * dn1 + (b.dst_lo[1] + ry)) * dn0 + b.dst_lo[0] + x;
        if (zero) {
          v[i] = Vec{};
        } else {
          const int64_t s = sfoff + ((int64_t)(b.src_lo[2] + rz) * sn1 + (b.src_lo[1] + ry)) * sn0 +
                            b.src_lo[0] + x;
          v[i] = *reinterpret_cast<const Vec*>(sbase + s);
        }
      }
    }
#pragma unroll
    for (int i = 0; i < kBatch; ++i)
      if (d[i] >= 0) *reinterpret_cast<Vec*>(dbase + d[i]) = v[i];
  }
}

// dst and src boxes may belong to two layouts (the plan's boxes for the
// guard exchange; the two grids of a dual-grid coupling); field slot
// blockIdx.y is read from S.p and written to Dst.p.
template <typename T>
__global__ void __launch_bounds__(256) k_exchange(const BoxDev* __restrict__ dboxes, const BoxDev* __restrict__ sboxes,
                                                  FieldPtrs Dst, FieldPtrs S, const CopyBlk* __restrict__ blocks,
                                                  const XTile* __restrict__ tiles) {
  const XTile t = tiles[blockIdx.x];
  const CopyBlk b = blocks[t.blk];
  T* dbase = reinterpret_cast<T*>(Dst.p[blockIdx.y]);
  const T* sbase = reinterpret_cast<const T*>(S.p[blockIdx.y]);
  const BoxDev db = dboxes[b.dst_box];
  int64_t sfoff = 0, sn0 = 0, sn1 = 0;
  if (b.src_box >= 0) {
    const BoxDev sb = sboxes[b.src_box];
    sfoff = sb.foff;
    sn0 = sb.n[0];
    sn1 = sb.n[1];
  }
  if (t.vec > 1)
    copy_tile<T, 16 / sizeof(T)>(dbase, sbase, b, t, db, sfoff, sn0, sn1);
  else
    copy_tile<T, 1>(dbase, sbase, b, t, db, sfoff, sn0, sn1);
}

// Absorbing layers, step (2) (the split-field PML: each component is the sum
// of two parts, one per derivative direction; the part along direction d
// decays by exp(-s_d dt) over the step).  For component q the stored part is
// along kStored[q] and the other part along the remaining direction; with
// the step's increment of the stored part (slot 6 + q of f):
//   stored* = stored + increment,  other* = component - stored*,
//   stored' = e_stored stored*,    other' = e_other other*,
//   component = stored' + other'.
// Grid: x strides over the interior cells of box blockIdx.y of the list.
__constant__ int kStored[6] = {1, 2, 0, 1, 2, 0};    // E_xy, E_yz, E_zx, B_xy, B_yz, B_zx
// Yee offset of component q along axis d, in half cells (0 or 1)
__constant__ int kYeeHalf[6][3] = {{1, 0, 0}, {0, 1, 0}, {0, 0, 1}, {0, 1, 1}, {1, 0, 1}, {1, 1, 0}};

template <typename T>
__global__ void __launch_bounds__(256) k_pml_damp(DevPlan P, FieldPtrs F, FieldPtrs S, const PmlBox* __restrict__ boxes,
                                                  const T* __restrict__ tab, PmlTab t) {
  const PmlBox pb = boxes[blockIdx.y];
  const BoxDev bx = P.boxes[pb.box];
  const int m0 = bx.n[0] - bx.ng_lo[0] - bx.ng_hi[0], m1 = bx.n[1] - bx.ng_lo[1] - bx.ng_hi[1];
  const int m2 = bx.n[2] - bx.ng_lo[2] - bx.ng_hi[2];
  const int64_t cells = (int64_t)m0 * m1 * m2;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < cells; e += (int64_t)gridDim.x * blockDim.x) {
    const int x = (int)(e % m0), y = (int)((e / m0) % m1), z = (int)(e / ((int64_t)m0 * m1));
    const int g[3] = {pb.origin[0] + x, pb.origin[1] + y, pb.origin[2] + z};
    const int64_t li =
        bx.foff + ((int64_t)(z + bx.ng_lo[2]) * bx.n[1] + (y + bx.ng_lo[1])) * bx.n[0] + (x + bx.ng_lo[0]);
#pragma unroll
    for (int q = 0; q < 6; ++q) {
      const int axis = q % 3, sa = kStored[q], sb = 3 - axis - sa;
      const T ea = tab[t.off[sa][kYeeHalf[q][sa]] + g[sa]];
      const T eb = tab[t.off[sb][kYeeHalf[q][sb]] + g[sb]];
      T* f = reinterpret_cast<T*>(F.p[q]) + li;
      T* sp = reinterpret_cast<T*>(S.p[q]) + li;
      const T ps = *sp + reinterpret_cast<const T*>(F.p[6 + q])[li];
      const T po = *f - ps;
      const T ns = ea * ps;
      *f = ns + eb * po;
      *sp = ns;
    }
  }
}

// Copy of whole field buffers in 16-byte units, slot blockIdx.y: the host
// path's copies between page-locked host memory (device-mapped) and the
// device staging buffers, driven by the SMs instead of the copy engines.
__global__ void __launch_bounds__(256) k_copy_fields(FieldPtrs dst, FieldPtrs src, int64_t n16) {
  const float4* s = reinterpret_cast<const float4*>(src.p[blockIdx.y]);
  float4* d = reinterpret_cast<float4*>(dst.p[blockIdx.y]);
  constexpr int kU = 4;   // units in flight per thread
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n16; i += kU * stride) {
    float4 v[kU];
#pragma unroll
    for (int u = 0; u < kU; ++u)
      if (i + u * stride < n16) v[u] = s[i + u * stride];
#pragma unroll
    for (int u = 0; u < kU; ++u)
      if (i + u * stride < n16) d[i + u * stride] = v[u];
  }
}

}  // namespace

cudaError_t launch_copy_fields(const FieldPtrs& dst, const FieldPtrs& src, int nf, int64_t bytes, int blocks,
                               cudaStream_t st) {
  if (nf <= 0 || bytes <= 0) return cudaSuccess;
  if (bytes % 16) return cudaErrorInvalidValue;
  dim3 grid((unsigned)std::max(1, blocks), (unsigned)nf);
  k_copy_fields<<<grid, 256, 0, st>>>(dst, src, bytes / 16);
  return cudaGetLastError();
}

cudaError_t launch_pml_damp(int prec, const DevPlan& P, const FieldPtrs& f, const FieldPtrs& parts,
                            const PmlBox* boxes, int nboxes, const void* tab, const PmlTab& t, cudaStream_t st) {
  for (int b0 = 0; b0 < nboxes; b0 += 65535) {
    dim3 grid(64, (unsigned)std::min(65535, nboxes - b0));
    if (prec == 32)
      k_pml_damp<float><<<grid, 256, 0, st>>>(P, f, parts, boxes + b0, (const float*)tab, t);
    else
      k_pml_damp<double><<<grid, 256, 0, st>>>(P, f, parts, boxes + b0, (const double*)tab, t);
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

cudaError_t launch_exchange(int prec, const DevPlan& P, const FieldPtrs& f, int nf,
                            const CopyBlk* blocks, const XTile* tiles, int64_t ntiles,
                            cudaStream_t st) {
  return launch_copy_blocks(prec, P.boxes, P.boxes, f, f, nf, blocks, tiles, ntiles, st);
}

cudaError_t launch_copy_blocks(int prec, const BoxDev* dboxes, const BoxDev* sboxes, const FieldPtrs& dst,
                               const FieldPtrs& src, int nf, const CopyBlk* blocks, const XTile* tiles,
                               int64_t ntiles, cudaStream_t st) {
  if (ntiles <= 0 || nf <= 0) return cudaSuccess;
  dim3 grid((unsigned)ntiles, nf);
  if (prec == 32)
    k_exchange<float><<<grid, 256, 0, st>>>(dboxes, sboxes, dst, src, blocks, tiles);
  else
    k_exchange<double><<<grid, 256, 0, st>>>(dboxes, sboxes, dst, src, blocks, tiles);
  return cudaGetLastError();
}

}  // namespace psatd
