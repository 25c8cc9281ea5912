// Internal structures shared by the host plan (plan.cpp) and the CUDA kernels.
// Everything here is plain old data copied to the device as-is.
#pragma once

#include <cstdint>
#include <vector>

#include <cuda_runtime.h>

#include "../../include/psatd.h"

namespace psatd {

constexpr int kMaxPass = 16;       // radix passes of one axis (2^10 needs <= 4 with radix 8)
constexpr int kThreads = 256;      // threads per CTA of every FFT kernel
constexpr int kPointsPerThread = 16;
constexpr int kMaxPoints = kThreads * kPointsPerThread;  // points of one FFT chunk in smem

// Equation form of the k-space update (slot layout of the fields):
//   kVacuum: E 0-2, B 3-5                      (6 in, 6 out)
//   kJForm : E 0-2, B 3-5, J 6-8               (9 in, 6 out)
//   kRhoForm: E 0-2, B 3-5, rho 6, J 7-9       (10 in, 7 out)
//   kPml   : E 0-2, B 3-5 in; E, B and the increments of the stored split
//            parts E_xy, E_yz, E_zx, B_xy, B_yz, B_zx in 6-11 out (vacuum
//            with absorbing layers; generic kernels only)
enum Form { kVacuum = 0, kJForm = 1, kRhoForm = 2, kPml = 3 };

constexpr int fields_in(int form) { return form == kVacuum || form == kPml ? 6 : form == kJForm ? 9 : 10; }
constexpr int fields_out(int form) { return form == kRhoForm ? 7 : form == kPml ? 12 : 6; }
// spectrum slots a step needs (inputs and outputs share them)
constexpr int spec_slots(int form) { return fields_in(form) > fields_out(form) ? fields_in(form) : fields_out(form); }

// Radix schedule of one complex FFT length.
struct AxisPlan {
  int32_t n;
  int32_t npass;
  int64_t tw;                     // offset of the n-entry twiddle table (complex pool)
  uint8_t radix[kMaxPass];
};

// Tables of one box shape (n0, n1, n2, p); offsets index the typed pools.
struct ShapeDev {
  int32_t n[3];
  int32_t L;                      // n0/2: length of the packed complex FFT along x
  int32_t hx;                     // n0/2 + 1: half-spectrum length along x
  int32_t p;
  AxisPlan ax, ay, az;            // x: length L; y: n1; z: n2
  int64_t post;                   // hx entries exp(-2 pi i k / n0)         (complex pool)
  int64_t kx, ky, kz;             // modified wavenumbers, hx / n1 / n2      (real pool)
  int64_t phx, phy, phz;          // exp(i k h / 2), hx / n1 / n2            (complex pool)
  int64_t coef;                   // hx*(n1/2+1)*(n2/2+1) coefficient quads (coef pool)
  int32_t fx, fy, fz;             // fast-length codes of L, n1, n2 (-1: not a fast length)
  int32_t px, py, pz;             // pencil-length codes of L, n1, n2 (-1: none)
  int32_t lp, hp;                 // smem row pitches (complex) of the fast plane kernels
};

// Lengths with a two-pass register FFT, N = R1 * R2: X(code, N, R1, R2).
#define PSATD_FAST_LENGTHS(X)                                                          \
  X(0, 24, 8, 3) X(1, 30, 6, 5) X(2, 32, 8, 4) X(3, 40, 8, 5) X(4, 48, 8, 6)              \
  X(5, 60, 12, 5) X(6, 64, 8, 8) X(7, 80, 10, 8) X(8, 96, 12, 8) X(9, 120, 12, 10)       \
  X(10, 128, 16, 8)

// Lengths of the pencil kernels (boxes too large for the plane kernels):
// the same two-pass factorizations, extended to 512.  Codes 0-10 coincide
// with PSATD_FAST_LENGTHS.
#define PSATD_PENCIL_LENGTHS(X)                                                         \
  PSATD_FAST_LENGTHS(X)                                                                \
  X(11, 144, 12, 12) X(12, 160, 16, 10) X(13, 192, 16, 12) X(14, 240, 24, 10)            \
  X(15, 256, 16, 16) X(16, 320, 32, 10) X(17, 384, 24, 16) X(18, 512, 32, 16)

inline int pencil_code(int n) {
#define PSATD_CODE(code, N, R1, R2) \
  if (n == N) return code;
  PSATD_PENCIL_LENGTHS(PSATD_CODE)
#undef PSATD_CODE
  return -1;
}

inline int fast_code(int n) {
#define PSATD_CODE(code, N, R1, R2) \
  if (n == N) return code;
  PSATD_FAST_LENGTHS(PSATD_CODE)
#undef PSATD_CODE
  return -1;
}

struct BoxDev {
  int32_t n[3];
  int32_t ng_lo[3];
  int32_t ng_hi[3];
  int32_t shape;
  int32_t gplane;                 // index of the box's plane z = 0 in the gather grids
  int32_t yoff;                   // global index of the box's spectrum row my = 0 (rows of a distributed group)
  int64_t foff;                   // element offset in every field buffer
  int64_t soff;                   // complex-element offset in every spectrum slot
};

// rows r0 .. r0+nr-1 of one box, row r = y + n1*z (x-axis passes)
struct RowJob {
  int32_t box, r0, nr, pad;
};

// columns m0 .. m0+nm-1 of one plane (y-axis passes: plane = z; z-axis: plane = y).
// Fast z tiles with nm < 0 hold the Nyquist column mx = m0 = n0/2 of the -nm
// planes y = plane .. plane-nm-1.
struct ColJob {
  int32_t box, plane, m0, nm;
};

struct CopyBlk {
  int32_t dst_box, src_box;
  int32_t dst_lo[3], src_lo[3], ext[3];
};

// rows [row0, row0+nrows) of one copy block, row = ry + ext1*rz; vec > 1:
// rows are copied in 16-byte units of `vec` elements
struct XTile {
  int32_t blk, row0, nrows, vec;
};

// A rectangle of one interior source plane that feeds guard cells of a box:
// source rows sy.., columns sx.. (box-local) -> destination (dst_box, dst_z,
// dy.., dx..).  vec: rows can move in 16-byte units.
struct GuardSeg {
  int32_t dst_box, dst_z;
  int32_t sy, sx, ny, nx;
  int32_t dy, dx;
  int32_t vec, pad;
};

// Deferred guard exchange: rows [dy, dy + ny) x columns [dx, dx + nx) of a
// forward plane buffer are read from the field elements src_off + r * spitch
// + c (the owning box's interior, or the box's own cells).
struct GatherSeg {
  int64_t src_off;
  int32_t spitch, dy, dx, ny, nx, vec;
};

// The same gather when the plane splits into at most 3 x 3 rectangles at
// columns x1 <= x2 and rows y1 <= y2 (guard faces of a local or hybrid box),
// every rectangle copied in 16-byte units: rectangle (iy, ix) starts at field
// element base[3 iy + ix], row pitch pitch[3 iy + ix].
struct alignas(16) GatherGrid {
  int64_t base[9];
  int32_t pitch[9];
  int32_t x1, x2, y1, y2;
  int32_t pad[3];
};

// Up to 12 field slots (see Form).
struct FieldPtrs {
  void* p[12];
};

template <typename T>
struct alignas(4 * sizeof(T)) Coef4 {
  T c;    // cos(theta)
  T s;    // sin(theta)/(c K)
  T x1;   // (1 - cos theta)/K^2
  T x3;   // (sin(theta)/(c K) - dt)/K^2
};

// Device view of a plan, passed by value to every kernel.
struct DevPlan {
  const BoxDev* boxes;
  const ShapeDev* shapes;
  const void* rpool;              // T[]
  const void* cpool;              // T2[]
  const void* coef;               // Coef4<T>[]
  double c, eps0, dt;
  double cc, ieps, idt, icce;     // c^2, 1/eps0, 1/dt, 1/(c^2 eps0)
};

inline void set_constants(DevPlan& P, double c, double eps0, double dt) {
  P.c = c;
  P.eps0 = eps0;
  P.dt = dt;
  P.cc = c * c;
  P.ieps = 1.0 / eps0;
  P.idt = 1.0 / dt;
  P.icce = 1.0 / (c * c * eps0);
}

// ---- kernel launchers (fft_kernels.cu, exchange.cu) ----------------------

// Forward R2C along x of `nf` field slots into spectrum slots (stride sstride).
cudaError_t launch_fwd_x(int prec, const DevPlan& P, const FieldPtrs& f, int nf, void* spec,
                         int64_t sstride, const RowJob* jobs, int64_t njobs, int smem,
                         cudaStream_t st);
// Complex FFT along y (axis 1) or z (axis 2), in place on spectrum slots.
cudaError_t launch_col(int prec, int dir, int axis, const DevPlan& P, void* spec,
                       int64_t sstride, int nf, const ColJob* jobs, int64_t njobs, int smem,
                       cudaStream_t st);
// z forward FFT + k-space update + z inverse FFT, all slots of `form`.
// nft: field slots transformed along z (the others hold a cached z spectrum)
cudaError_t launch_z_update(int prec, int form, const DevPlan& P, void* spec, int64_t sstride,
                            const ColJob* jobs, int64_t njobs, int smem, int nft, cudaStream_t st);
// C2R inverse along x with 1/(n0 n1 n2) into field slots; interior_only skips guards.
cudaError_t launch_inv_x(int prec, const DevPlan& P, const FieldPtrs& f, int nf, void* spec,
                         int64_t sstride, const RowJob* jobs, int64_t njobs, int smem,
                         int interior_only, cudaStream_t st);
// Guard exchange of `nf` field slots.
// Absorbing layers, step (2): one box of the layers' list.  Damping table
// (type T): for axis d and Yee offset o (0: cell, 1: half cell), entry
// tab[d][o] + g = exp(-s_d(g + o/2) dt) for global index g.
struct PmlBox {
  int32_t box;
  int32_t origin[3];
};
struct PmlTab {
  int64_t off[3][2];
};
// f: the 6 components (updated in place) and, in slots 6-11, the increments of
// the stored split parts; parts: the 6 stored split parts (in place); every
// interior cell of every listed box.
cudaError_t launch_pml_damp(int prec, const DevPlan& P, const FieldPtrs& f, const FieldPtrs& parts,
                            const PmlBox* boxes, int nboxes, const void* tab, const PmlTab& t, cudaStream_t st);

// Copy nf whole buffers of `bytes` (a multiple of 16) from src.p[i] to
// dst.p[i] with `blocks` x nf CTAs (16-byte aligned pointers).
cudaError_t launch_copy_fields(const FieldPtrs& dst, const FieldPtrs& src, int nf, int64_t bytes, int blocks,
                               cudaStream_t st);

cudaError_t launch_exchange(int prec, const DevPlan& P, const FieldPtrs& f, int nf,
                            const CopyBlk* blocks, const XTile* tiles, int64_t ntiles,
                            cudaStream_t st);
// Copy blocks whose destination boxes (dboxes, buffers dst) and source boxes
// (sboxes, buffers src) may belong to two different layouts.
cudaError_t launch_copy_blocks(int prec, const BoxDev* dboxes, const BoxDev* sboxes, const FieldPtrs& dst,
                               const FieldPtrs& src, int nf, const CopyBlk* blocks, const XTile* tiles,
                               int64_t ntiles, cudaStream_t st);
// Maximum dynamic shared memory opt-in for all kernels of a precision.
cudaError_t configure_kernels(int prec, int smem_bytes);

// ---- fast path (fast_kernels.cu): boxes whose three FFT lengths are fast --
// jobs: (box, z plane); forward writes every plane, inverse takes interior z.
// Persistent kernels: `grid` CTAs walk nplanes x nf planes; bufsz is the
// complex-element size of one plane buffer (two per CTA).
cudaError_t launch_plane_fwd(int prec, const DevPlan& P, const FieldPtrs& f, int nf, void* spec,
                             int64_t sstride, const int2* jobs, int64_t nplanes, int bufsz, int smem,
                             int grid, cudaStream_t st);
// The inverse kernel also writes the guard cells its interior plane feeds
// (segments seg_start[p] .. seg_start[p+1] of plane p; NULL: none).
cudaError_t launch_plane_inv(int prec, const DevPlan& P, const FieldPtrs& f, int nf, void* spec,
                             int64_t sstride, const int2* jobs, int64_t nplanes, int bufsz, int smem,
                             int grid, const int* seg_start, const GuardSeg* segs, cudaStream_t st);
// Resident CTAs per SM of the plane kernels at the given shared memory.
cudaError_t plane_occupancy(int prec, int smem_fwd, int smem_inv, int* fwd_per_sm, int* inv_per_sm);
cudaError_t launch_z_fast(int prec, int form, const DevPlan& P, void* spec, int64_t sstride,
                          const ColJob* jobs, int64_t njobs, int smem, int nft, cudaStream_t st);
int fast_tile(int prec);                        // mx columns per k_z_fast job
int fast_max_x(int prec);                       // longest n0/2 of a fast-path box
int z_fast_smem(int prec, int form, int n2);    // bytes of shared memory of k_z_fast
cudaError_t configure_fast_kernels(int prec, int smem_bytes);

// ---- register-resident plane kernels (reg_kernels.cu), FP32 -----------------
// code >= 0 when the plane shape (n0/2, n1) has register kernels
int reg_shape_code(int L, int n1);
int reg_fwd_smem(int code);
int reg_inv_smem(int code);
cudaError_t launch_plane_fwd_reg(int code, const DevPlan& P, const FieldPtrs& f, int nf, void* spec,
                                 int64_t sstride, const int2* jobs, int64_t nplanes, const int* gstart,
                                 const GatherSeg* gsegs, const GatherGrid* ggrid, int ngather, cudaStream_t st);
cudaError_t launch_plane_inv_reg(int code, const DevPlan& P, const FieldPtrs& f, int nf, void* spec,
                                 int64_t sstride, const int2* jobs, int64_t nplanes, const int* seg_start,
                                 const GuardSeg* segs, cudaStream_t st);
cudaError_t configure_reg_kernels(int smem_bytes);
// the plane shapes are instantiated in four translation units
// (reg_planes_<part>.cu); each exports its launchers in namespace plane_part<part>
#define PSATD_DECLARE_PLANE_PART(NS)                                                                       \
  namespace NS {                                                                                           \
  cudaError_t launch_fwd(int code, const DevPlan& P, const FieldPtrs& f, int nf, void* spec, int64_t sstride,  \
                         const int2* jobs, int64_t nplanes, const int* gstart, const GatherSeg* gsegs,      \
                         const GatherGrid* ggrid, int ngather, cudaStream_t st);                           \
  cudaError_t launch_inv(int code, const DevPlan& P, const FieldPtrs& f, int nf, void* spec, int64_t sstride,  \
                         const int2* jobs, int64_t nplanes, const int* seg_start, const GuardSeg* segs,     \
                         cudaStream_t st);                                                                 \
  cudaError_t configure(int smem_bytes);                                                                   \
  }
PSATD_DECLARE_PLANE_PART(plane_part0)
PSATD_DECLARE_PLANE_PART(plane_part1)
PSATD_DECLARE_PLANE_PART(plane_part2)
PSATD_DECLARE_PLANE_PART(plane_part3)
#undef PSATD_DECLARE_PLANE_PART
// register z kernel (FP32, tiles of z_reg_tile_width(form, n2) columns) for z
// length n2 (thread pairs per column; thread quads for 128 and 192)
int z_reg_ok(int n2);
int z_reg_multi_ok(int n2);   // a length the persistent multi-length kernel takes
int z_reg_smem(int form, int n2);
int z_reg_tile_width(int form, int n2);
// z-only forward FFT (natural z order) of slots [0, ns) of `spec` over the z
// tiles `jobs` (tile columns `tile`, 8 required; n2 a thread-pair register z
// length; 2 * ns * tile <= 64)
cudaError_t launch_z_fwd_pair(const DevPlan& P, void* spec, int64_t sstride, const ColJob* jobs, int64_t njobs,
                              int n2, int tile, int ns, cudaStream_t st);
// zst: n1 * (n0/2 + 1) shared by every box of the job list, else 0
// pf_dist > 0: every CTA first prefetches into L2 the tile of the CTA
// launched pf_dist blocks after it
cudaError_t launch_z_reg(int form, const DevPlan& P, void* spec, int64_t sstride, const ColJob* jobs,
                         int64_t njobs, int n2, int zst, int nft, int pf_dist, cudaStream_t st);
// The register z pass of boxes of several z lengths (every one z_reg_ok) in
// one persistent launch of at most `grid` CTAs; prefetch != 0: every CTA
// prefetches into L2 the tile of its next job.
cudaError_t launch_z_reg_multi(int form, const DevPlan& P, void* spec, int64_t sstride, const ColJob* jobs,
                               int64_t njobs, int grid, int prefetch, int nft, cudaStream_t st);
int z_reg_multi_smem(int form);

// ---- pencil kernels (pencil_kernels.cu): boxes of two-pass lengths too large
// for the plane kernels; the z pass takes fast_tile(prec) mx columns per tile
int pen_rows(int prec, int L, int rows, int smem_cap);   // x rows per CTA
int pen_x_smem(int prec, int L, int nr);
int pen_z_max(int prec);                                  // longest n2 of a pencil box
int pen_col_tile(int prec);                               // mx columns of a y tile
int pen_col_smem(int prec, int n1);
// one launch per length group: `code` = pencil code of the transformed axis
// ggrid (deferred exchange): the gather grid of every plane, box b's plane z
// at boxes[b].gplane + z, used for the slots f < ngather; null: plain rows
cudaError_t launch_pen_xf(int prec, int code, const DevPlan& P, const FieldPtrs& f, int nf, void* spec,
                          int64_t sstride, const RowJob* jobs, int64_t njobs, int smem, const GatherGrid* ggrid, int ngather, cudaStream_t st);
cudaError_t launch_pen_col(int prec, int dir, int code, const DevPlan& P, void* spec, int64_t sstride, int nf,
                           const ColJob* jobs, int64_t njobs, int smem, cudaStream_t st);
cudaError_t launch_z_pen(int prec, int form, int code, const DevPlan& P, void* spec, int64_t sstride,
                         const ColJob* jobs, int64_t njobs, int smem, int nft, cudaStream_t st);
cudaError_t launch_pen_xi(int prec, int code, const DevPlan& P, const FieldPtrs& f, int nf, void* spec,
                          int64_t sstride, const RowJob* jobs, int64_t njobs, int smem, cudaStream_t st);
cudaError_t configure_pen_kernels(int prec, int smem_bytes);

// ---- host helpers (plan.cpp) ------------------------------------------------
// Radix schedule of a complex FFT length (false if it is not 5-smooth).
bool radix_plan(int n, AxisPlan& ap);
// Weights alpha_l, l = 1..p/2, of the order-p staggered difference
// (nodal: beta_l of the centred collocated difference).
std::vector<double> stencil_alpha(int p, bool nodal = false);
// Text returned by psatd_last_error(NULL) on this thread.
void set_thread_error(const char* msg);

// ---- FP64 table generators (tables.cu) ------------------------------------
cudaError_t gen_twiddles(double2* out, int n, cudaStream_t st);
cudaError_t gen_post(double2* out, int n0, cudaStream_t st);
cudaError_t gen_axis(double* K, double2* ph, int count, int n, double h, int q,
                     const double* alpha_dev, int nodal, cudaStream_t st);
cudaError_t gen_coef(Coef4<double>* out, int hx, int n1, int n2, const double* kx,
                     const double* ky, const double* kz, double c, double dt, cudaStream_t st);
cudaError_t convert_pools(const double* r64, float* r32, int64_t nr, const double2* c64,
                          float2* c32, int64_t nc, const Coef4<double>* q64, Coef4<float>* q32,
                          int64_t nq, cudaStream_t st);

}  // namespace psatd
