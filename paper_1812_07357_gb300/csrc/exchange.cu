// S4: guard-cell exchange between batched boxes (paper Fig. 1, step (ii)).
//
// The host precomputes copy blocks, each a 3D region of guard cells of one
// box whose values live in the interior of one source box (or outside a
// non-periodic domain: zero).  A tile is a run of rows of one block; a row is
// ext[0] consecutive cells in both the source and the destination box.  Reads
// touch interior cells only and writes guard cells only, so tiles never race.
#include <cuda_runtime.h>

#include "psatd_internal.h"

namespace psatd {

template <typename T>
__global__ void __launch_bounds__(256) k_exchange(DevPlan P, FieldPtrs F,
                                                  const CopyBlk* __restrict__ blocks,
                                                  const XTile* __restrict__ tiles) {
  const XTile t = tiles[blockIdx.x];
  const CopyBlk b = blocks[t.blk];
  T* base = reinterpret_cast<T*>(F.p[blockIdx.y]);
  const BoxDev db = P.boxes[b.dst_box];
  const int ex = b.ext[0], ey = b.ext[1];
  const int64_t dn0 = db.n[0], dn1 = db.n[1];
  int64_t sfoff = 0, sn0 = 0, sn1 = 0;
  if (b.src_box >= 0) {
    const BoxDev sb = P.boxes[b.src_box];
    sfoff = sb.foff;
    sn0 = sb.n[0];
    sn1 = sb.n[1];
  }
  const int count = t.nrows * ex;
  for (int e = threadIdx.x; e < count; e += blockDim.x) {
    const int rr = e / ex;
    const int x = e - rr * ex;
    const int r = t.row0 + rr;
    const int ry = r % ey, rz = r / ey;
    const int64_t d = db.foff + ((int64_t)(b.dst_lo[2] + rz) * dn1 + (b.dst_lo[1] + ry)) * dn0 +
                      b.dst_lo[0] + x;
    T v = T(0);
    if (b.src_box >= 0) {
      const int64_t s = sfoff + ((int64_t)(b.src_lo[2] + rz) * sn1 + (b.src_lo[1] + ry)) * sn0 +
                        b.src_lo[0] + x;
      v = base[s];
    }
    base[d] = v;
  }
}

cudaError_t launch_exchange(int prec, const DevPlan& P, const FieldPtrs& f, int nf,
                            const CopyBlk* blocks, const XTile* tiles, int64_t ntiles,
                            cudaStream_t st) {
  if (ntiles <= 0 || nf <= 0) return cudaSuccess;
  dim3 grid((unsigned)ntiles, nf);
  if (prec == 32)
    k_exchange<float><<<grid, 256, 0, st>>>(P, f, blocks, tiles);
  else
    k_exchange<double><<<grid, 256, 0, st>>>(P, f, blocks, tiles);
  return cudaGetLastError();
}

}  // namespace psatd
