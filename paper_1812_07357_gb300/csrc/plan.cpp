// Host side of the PSATD library: description validation, the guard-exchange
// protocol (copy blocks from box-overlap geometry, computed once before any
// step, as the paper's Sec. 2.6 does for its two grids), work lists,
// device tables, and the C ABI entry points declared in include/psatd.h.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <map>
#include <string>
#include <tuple>
#include <vector>

#include "psatd_internal.h"

using namespace psatd;

namespace {

thread_local std::string g_thread_error = "no error";

void set_msg(char* msg, size_t len, const std::string& s) {
  if (msg && len) {
    size_t n = std::min(len - 1, s.size());
    std::memcpy(msg, s.data(), n);
    msg[n] = 0;
  }
}

std::string fmt(const char* f, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, f);
  std::vsnprintf(buf, sizeof buf, f, ap);
  va_end(ap);
  return buf;
}

bool five_smooth(int n) {
  if (n <= 0) return false;
  for (int f : {2, 3, 5})
    while (n % f == 0) n /= f;
  return n == 1;
}

int64_t align_up(int64_t v, int64_t a) { return (v + a - 1) / a * a; }

struct Err {
  psatd_status st;
  std::string msg;
};

// ---------------------------------------------------------------------------
// validation
// ---------------------------------------------------------------------------
Err validate(const psatd_plan_desc* d) {
  if (!d) return {PSATD_ERR_INVALID_ARG, "desc is NULL"};
  if (d->num_boxes < 1 || !d->boxes) return {PSATD_ERR_INVALID_ARG, "no boxes"};
  if (d->precision != 32 && d->precision != 64)
    return {PSATD_ERR_INVALID_ARG, fmt("precision %d is not 32 or 64", d->precision)};
  if (!(std::isfinite(d->dt)) || d->dt == 0.0) return {PSATD_ERR_INVALID_ARG, "dt must be finite and nonzero"};
  if (!(d->c > 0.0) || !std::isfinite(d->c)) return {PSATD_ERR_INVALID_ARG, "c must be > 0"};
  if (!(d->eps0 > 0.0) || !std::isfinite(d->eps0)) return {PSATD_ERR_INVALID_ARG, "eps0 must be > 0"};
  for (int a = 0; a < 3; ++a)
    if (!(d->dx[a] > 0.0) || !std::isfinite(d->dx[a])) return {PSATD_ERR_INVALID_ARG, "dx must be > 0"};
  const uint32_t known =
      PSATD_VACUUM | PSATD_RHO_CONTINUITY | PSATD_J_CONSTANT | PSATD_NO_GRAPH | PSATD_GENERIC_KERNELS |
      PSATD_PENCIL_KERNELS | PSATD_PLANE_KERNELS | PSATD_NODAL | PSATD_EAGER_EXCHANGE;
  if (d->flags & ~known) return {PSATD_ERR_INVALID_ARG, "unknown flag bits"};
  if ((d->flags & PSATD_VACUUM) && (d->flags & PSATD_RHO_CONTINUITY))
    return {PSATD_ERR_INVALID_ARG, "PSATD_VACUUM and PSATD_RHO_CONTINUITY exclude each other"};
  if (d->decomp < PSATD_DECOMP_GLOBAL || d->decomp > PSATD_DECOMP_INDEPENDENT)
    return {PSATD_ERR_INVALID_ARG, "unknown decomposition"};
  for (int i = 0; i < d->num_boxes; ++i) {
    const psatd_box& b = d->boxes[i];
    for (int a = 0; a < 3; ++a) {
      const int lim = a == 0 ? 1024 : 512;
      if (b.n[a] < 4 || b.n[a] % 2 || !five_smooth(b.n[a]) || b.n[a] > lim)
        return {PSATD_ERR_UNSUPPORTED_SIZE,
                fmt("box %d: n[%d] = %d must be even, 5-smooth, in [4, %d]", i, a, b.n[a], lim)};
      if (b.ng_lo[a] < 0 || b.ng_hi[a] < 0 || b.ng_lo[a] + b.ng_hi[a] >= b.n[a])
        return {PSATD_ERR_INVALID_ARG,
                fmt("box %d: guards %d + %d leave no interior on axis %d", i, b.ng_lo[a], b.ng_hi[a], a)};
    }
    if (!(b.order_p == 0 || (b.order_p >= 2 && b.order_p <= 256 && b.order_p % 2 == 0)))
      return {PSATD_ERR_UNSUPPORTED_ORDER, fmt("box %d: order %d is not 0 or even in [2, 256]", i, b.order_p)};
  }
  if (d->tuning) {
    int i = 0;
    for (; i < 16 && d->tuning[2 * i] != 0; ++i) {
      const int32_t k = d->tuning[2 * i], v = d->tuning[2 * i + 1];
      const bool ok = (k == PSATD_TUNE_Z_PREFETCH && v >= 0 && v <= (1 << 20)) ||
                      (k == PSATD_TUNE_PENCIL_ROWS_KB && v >= 8 && v <= 200) ||
                      (k == PSATD_TUNE_Z_TILE && v >= 1 && v <= fast_tile(d->precision == 64 ? 64 : 32)) ||
                      (k == PSATD_TUNE_HOST_COPY && (v == 0 || v == 1)) ||
                      (k == PSATD_TUNE_PENCIL_REG_Z && (v == 0 || v == 1)) ||
                      (k == PSATD_TUNE_Z_ONE_LAUNCH && (v == 0 || v == 1)) ||
                      (k == PSATD_TUNE_REG_PLANES && (v == 0 || v == 1));
      if (!ok) return {PSATD_ERR_INVALID_ARG, fmt("tuning knob %d: value %d unknown or out of range", k, v)};
    }
    if (i == 16 && d->tuning[32] != 0) return {PSATD_ERR_INVALID_ARG, "more than 16 tuning pairs"};
  }
  if (d->pml) {
    if (!(d->flags & PSATD_VACUUM)) return {PSATD_ERR_INVALID_ARG, "absorbing layers need PSATD_VACUUM"};
    if (d->flags & PSATD_NODAL) return {PSATD_ERR_INVALID_ARG, "absorbing layers need the staggered grid"};
    if (d->decomp == PSATD_DECOMP_INDEPENDENT)
      return {PSATD_ERR_INVALID_ARG, "absorbing layers need a global domain"};
    if (d->pml->order < 0 || d->pml->order > 16) return {PSATD_ERR_INVALID_ARG, "PML order not in [0, 16]"};
    for (int a = 0; a < 3; ++a) {
      if (d->pml->width[a] < 0 || 2 * d->pml->width[a] > d->global_n[a])
        return {PSATD_ERR_INVALID_ARG, fmt("PML width %d not in [0, global_n/2] on axis %d", d->pml->width[a], a)};
      if (!(d->pml->sigma_max[a] >= 0.0) || !std::isfinite(d->pml->sigma_max[a]))
        return {PSATD_ERR_INVALID_ARG, "PML sigma_max must be finite and >= 0"};
    }
  }
  if (d->decomp == PSATD_DECOMP_INDEPENDENT) return {PSATD_OK, ""};
  for (int a = 0; a < 3; ++a) {
    if (d->global_n[a] < 1) return {PSATD_ERR_INVALID_ARG, "global_n must be >= 1"};
    if (d->periodic[a] != 0 && d->periodic[a] != 1) return {PSATD_ERR_INVALID_ARG, "periodic must be 0 or 1"};
  }
  if (d->decomp == PSATD_DECOMP_GLOBAL) {
    if (d->num_boxes != 1) return {PSATD_ERR_INVALID_ARG, "global decomposition takes one box"};
    const psatd_box& b = d->boxes[0];
    for (int a = 0; a < 3; ++a)
      if (b.ng_lo[a] || b.ng_hi[a] || b.n[a] != d->global_n[a] || b.origin[a] != 0)
        return {PSATD_ERR_INVALID_ARG, "global box must equal the domain, without guards"};
  }
  // interiors must tile the domain: inside, volumes add up, no overlaps
  int64_t vol = 0;
  for (int i = 0; i < d->num_boxes; ++i) {
    const psatd_box& b = d->boxes[i];
    int64_t v = 1;
    for (int a = 0; a < 3; ++a) {
      const int64_t m = b.n[a] - b.ng_lo[a] - b.ng_hi[a];
      if (b.origin[a] < 0 || b.origin[a] + m > d->global_n[a])
        return {PSATD_ERR_INVALID_ARG, fmt("box %d interior leaves the domain on axis %d", i, a)};
      v *= m;
    }
    vol += v;
  }
  const int64_t gv = (int64_t)d->global_n[0] * d->global_n[1] * d->global_n[2];
  if (vol != gv) return {PSATD_ERR_INVALID_ARG, "box interiors do not cover the domain exactly"};
  for (int i = 0; i < d->num_boxes; ++i)
    for (int j = i + 1; j < d->num_boxes; ++j) {
      const psatd_box &p = d->boxes[i], &q = d->boxes[j];
      bool overlap = true;
      for (int a = 0; a < 3; ++a) {
        const int64_t pl = p.origin[a], ph = pl + p.n[a] - p.ng_lo[a] - p.ng_hi[a];
        const int64_t ql = q.origin[a], qh = ql + q.n[a] - q.ng_lo[a] - q.ng_hi[a];
        if (ph <= ql || qh <= pl) overlap = false;
      }
      if (overlap) return {PSATD_ERR_INVALID_ARG, fmt("box interiors %d and %d overlap", i, j)};
    }
  return {PSATD_OK, ""};
}

// ---------------------------------------------------------------------------
// guard-exchange protocol
// ---------------------------------------------------------------------------
struct Seg {
  int64_t dst, g, len;
  bool outside;
};

// Split the padded range [a, a+n) of one axis into pieces that map onto the
// global axis [0, N) (periodic: wrap; otherwise pieces outside are flagged).
std::vector<Seg> axis_segments(int64_t a, int64_t n, int64_t N, bool periodic) {
  std::vector<Seg> out;
  int64_t pos = a;
  const int64_t end = a + n;
  while (pos < end) {
    if (periodic) {
      const int64_t w = ((pos % N) + N) % N;
      const int64_t l = std::min(end - pos, N - w);
      out.push_back({pos - a, w, l, false});
      pos += l;
    } else if (pos < 0) {
      const int64_t l = std::min(end, (int64_t)0) - pos;
      out.push_back({pos - a, 0, l, true});
      pos += l;
    } else if (pos >= N) {
      out.push_back({pos - a, 0, end - pos, true});
      pos = end;
    } else {
      const int64_t l = std::min(end, N) - pos;
      out.push_back({pos - a, pos, l, false});
      pos += l;
    }
  }
  return out;
}

std::vector<CopyBlk> build_blocks(const psatd_plan_desc* d) {
  std::vector<CopyBlk> out;
  const bool indep = d->decomp == PSATD_DECOMP_INDEPENDENT;
  for (int b = 0; b < d->num_boxes; ++b) {
    const psatd_box& B = d->boxes[b];
    bool guards = false;
    for (int a = 0; a < 3; ++a) guards |= B.ng_lo[a] || B.ng_hi[a];
    if (!guards) continue;
    int64_t N[3], org[3];
    bool per[3];
    for (int a = 0; a < 3; ++a) {
      const int64_t m = B.n[a] - B.ng_lo[a] - B.ng_hi[a];
      N[a] = indep ? m : d->global_n[a];
      org[a] = indep ? 0 : B.origin[a];
      per[a] = indep ? true : d->periodic[a] != 0;
    }
    std::vector<Seg> s[3];
    for (int a = 0; a < 3; ++a) s[a] = axis_segments(org[a] - B.ng_lo[a], B.n[a], N[a], per[a]);
    for (const Seg& sz : s[2])
      for (const Seg& sy : s[1])
        for (const Seg& sx : s[0]) {
          const Seg* sg[3] = {&sx, &sy, &sz};
          if (sx.outside || sy.outside || sz.outside) {
            CopyBlk c{};
            c.dst_box = b;
            c.src_box = -1;
            for (int a = 0; a < 3; ++a) {
              c.dst_lo[a] = (int32_t)sg[a]->dst;
              c.src_lo[a] = 0;
              c.ext[a] = (int32_t)sg[a]->len;
            }
            out.push_back(c);
            continue;
          }
          const int s0 = indep ? b : 0, s1 = indep ? b + 1 : d->num_boxes;
          for (int sb = s0; sb < s1; ++sb) {
            const psatd_box& S = d->boxes[sb];
            int64_t lo[3], hi[3];
            bool empty = false;
            for (int a = 0; a < 3; ++a) {
              const int64_t so = indep ? 0 : S.origin[a];
              const int64_t sm = S.n[a] - S.ng_lo[a] - S.ng_hi[a];
              lo[a] = std::max(sg[a]->g, so);
              hi[a] = std::min(sg[a]->g + sg[a]->len, so + sm);
              if (hi[a] <= lo[a]) empty = true;
            }
            if (empty) continue;
            CopyBlk c{};
            c.dst_box = b;
            c.src_box = sb;
            bool same = sb == b;
            for (int a = 0; a < 3; ++a) {
              const int64_t so = indep ? 0 : S.origin[a];
              c.dst_lo[a] = (int32_t)(sg[a]->dst + (lo[a] - sg[a]->g));
              c.src_lo[a] = (int32_t)(lo[a] - so + S.ng_lo[a]);
              c.ext[a] = (int32_t)(hi[a] - lo[a]);
              same = same && c.dst_lo[a] == c.src_lo[a];
            }
            if (!same) out.push_back(c);
          }
        }
  }
  return out;
}

}  // namespace

// ---------------------------------------------------------------------------
// helpers shared with the no-allocation single-box variant (static_push.cu)
// ---------------------------------------------------------------------------
namespace psatd {

// Radix schedule: 8s first (4,4 instead of 8,2), then 4 / 2, 3s and 5s.
bool radix_plan(int n, AxisPlan& ap) {
  ap.n = n;
  ap.npass = 0;
  int e2 = 0, v = n;
  while (v % 2 == 0) v /= 2, ++e2;
  std::vector<int> r;
  int n8 = e2 / 3, rem = e2 % 3;
  if (rem == 1 && n8 > 0) {
    --n8;
    rem = 4;
  }
  for (int i = 0; i < n8; ++i) r.push_back(8);
  if (rem == 4) r.push_back(4), r.push_back(4);
  if (rem == 2) r.push_back(4);
  if (rem == 1) r.push_back(2);
  while (v % 5 == 0) v /= 5, r.push_back(5);
  while (v % 3 == 0) v /= 3, r.push_back(3);
  if (v != 1 || (int)r.size() > kMaxPass) return false;
  for (size_t i = 0; i < r.size(); ++i) ap.radix[i] = (uint8_t)r[i];
  ap.npass = (int)r.size();
  return true;
}


// Order-p staggered stencil weights (see tables.cu for their use):
std::vector<double> stencil_alpha(int p, bool nodal) {
  // staggered: alpha_l = prod_{j != l} (2j-1)^2 / ((2j-1)^2 - (2l-1)^2), l = 1..p/2
  // nodal:     beta_l  = prod_{j != l} j^2 / (j^2 - l^2)
  const int q = p / 2;
  std::vector<double> a(q);
  for (int l = 1; l <= q; ++l) {
    double v = 1.0;
    const double xl = nodal ? (double)l * l : (double)(2 * l - 1) * (2 * l - 1);
    for (int j = 1; j <= q; ++j) {
      if (j == l) continue;
      const double xj = nodal ? (double)j * j : (double)(2 * j - 1) * (2 * j - 1);
      v *= xj / (xj - xl);
    }
    a[l - 1] = v;
  }
  return a;
}

void set_thread_error(const char* msg) { g_thread_error = msg; }

}  // namespace psatd

// ---------------------------------------------------------------------------
// the plan
// ---------------------------------------------------------------------------
struct psatd_coupling;
static void destroy_global_coupling(psatd_coupling* c);

struct psatd_plan {
  psatd_plan_desc desc{};
  std::vector<psatd_box> boxes;
  int prec = 32;
  int form = kVacuum;
  size_t csize = 8;  // bytes of one complex element
  size_t rsize = 4;

  std::vector<BoxDev> hboxes;
  std::vector<ShapeDev> hshapes;
  std::vector<RowJob> rows_all, rows_int;
  std::vector<ColJob> ycols_all, ycols_int, zcols;           // every box (standalone FFTs)
  std::vector<RowJob> g_rows, g_rows_int;                     // push, generic boxes
  std::vector<ColJob> g_ycols, g_ycols_int, g_zcols;
  std::vector<int2> plane_fwd, plane_inv;                     // push, fast boxes
  std::vector<ColJob> zfast;
  int fast_boxes = 0;
  std::vector<RowJob> pen_rows, pen_rows_int;                 // push, pencil boxes
  std::vector<ColJob> pen_ycols, pen_ycols_int, zpen;
  struct PenGroup {
    int code;                 // pencil-length code of the transformed axis
    int64_t start, count;     // jobs of the list
  };
  std::vector<PenGroup> grp_rows, grp_rows_int, grp_ycols, grp_ycols_int, grp_z;
  std::vector<ColJob> zpen_reg;              // boxes of several z lengths whose z pass runs on the register z kernel
  std::vector<PenGroup> grp_zreg;            // ... grouped by z length (code = n2)
  std::vector<PenGroup> grp_pf, grp_pi;      // register plane jobs grouped by plane shape (code: reg_shape_code)
  // one group spread over ranks (psatd_plan_distribute): the rank's z slab
  // [z0, z1) and spectrum rows [y0, y1), the plan's boxes followed by the slab
  // box (every y, the slab's planes, the global n2 for the 1/N factor) and the
  // rows box (y1 - y0 rows, every z, yoff = y0), and their job lists
  struct Dist {
    int world = 0, rank = 0, z0 = 0, z1 = 0, y0 = 0, y1 = 0;
    BoxDev* d_boxes = nullptr;
    RowJob* d_rows = nullptr;
    ColJob *d_ycols = nullptr, *d_zcols = nullptr;
    int64_t nrows = 0, nycols = 0, nzcols = 0;
    int64_t s_slab = 0, s_rows = 0;   // complex elements per component of the slab spectrum / the rows
  } dist;
  int pen_reg_z = 1;                         // tuning: register z kernel for those boxes where one exists
  bool pen_reg_z_used = false;               // ... and whether the plan has such boxes
  int reg_planes = 1;                        // tuning: register plane kernels for the boxes whose shape has them
  bool reg_planes_used = false;              // ... and whether the plan has such boxes
  bool zreg_multi = false;                   // every length of zpen_reg has the persistent multi-length kernel
  int z_one_launch = 0;                      // tuning: those boxes' z pass in one persistent launch (measured
                                             // slower on the 300-box uneven batch: 7.07 against 5.11 ms)
  int sms = 0;                               // multiprocessors of the plan's device
  int pen_boxes = 0;
  std::vector<CopyBlk> blocks;
  std::vector<XTile> tiles;                                   // every block (psatd_guard_exchange)
  std::vector<XTile> step_tiles;                              // blocks not fused into the inverse
  std::vector<int> seg_start;                                 // fused exchange, CSR per plane_inv
  std::vector<GuardSeg> segs;
  bool deferred = false;                                      // deferred exchange (gather in S1)
  std::vector<int> gseg_start;                                // its CSR per plane_fwd
  std::vector<GatherSeg> gsegs;
  std::vector<GatherGrid> ggrid;                              // or one 3 x 3 grid per plane_fwd

  int64_t field_total = 0;  // elements per field buffer
  int64_t spec_total = 0;   // complex elements per spectrum slot
  int smem_fx = 0, smem_y = 0, smem_z = 0, smem_zonly = 0, smem_ix = 0;
  int smem_pf = 0, smem_pi = 0, smem_zf = 0;
  int smem_penx = 0, smem_penxi = 0, smem_penc = 0, smem_penz = 0;
  int buf_pf = 0, buf_pi = 0, rows_pi = 0;     // complex elements per plane buffer
  int grid_pf = 0, grid_pi = 0;                // persistent grid sizes
  int reg_z = 0;                               // register z kernel length (0: none)
  int reg_zst = 0;                             // n1 * (n0/2 + 1) of every register-z box, else 0
  int z_prefetch = 64;                         // register z kernel: L2 prefetch distance in CTAs (64: measured
                                               // best of 0 .. 1216 on 512 boxes of 96^3)
  int pen_rows_kb = 64;                        // pencil x pass: shared memory for one CTA's rows
  int host_copy = 1;                           // host path: 1 = SM copy kernel on mapped memory, 0 = copy engines
  int z_tile = 0;                              // plane/pencil z tile columns (0: the kernel maximum)
  // absorbing layers (form kPml): the description, boxes with layer cells,
  // damping table, stored split parts and their per-step increments
  psatd_pml pml{};
  std::vector<PmlBox> pml_boxes;
  PmlTab pml_tab{};
  PmlBox* d_pml_boxes = nullptr;
  void* d_pml_tab = nullptr;
  void* pml_parts[6] = {};
  void* pml_inc[6] = {};

  // device memory
  std::vector<void*> allocs;
  BoxDev* d_boxes = nullptr;
  ShapeDev* d_shapes = nullptr;
  RowJob *d_rows_all = nullptr, *d_rows_int = nullptr;
  ColJob *d_ycols_all = nullptr, *d_ycols_int = nullptr, *d_zcols = nullptr;
  RowJob *d_g_rows = nullptr, *d_g_rows_int = nullptr;
  ColJob *d_g_ycols = nullptr, *d_g_ycols_int = nullptr, *d_g_zcols = nullptr, *d_zfast = nullptr;
  int2 *d_plane_fwd = nullptr, *d_plane_inv = nullptr;
  RowJob *d_pen_rows = nullptr, *d_pen_rows_int = nullptr;
  ColJob *d_pen_ycols = nullptr, *d_pen_ycols_int = nullptr, *d_zpen = nullptr, *d_zpen_reg = nullptr;
  CopyBlk* d_blocks = nullptr;
  XTile* d_tiles = nullptr;
  XTile* d_step_tiles = nullptr;
  int* d_seg_start = nullptr;
  GuardSeg* d_segs = nullptr;
  int* d_gseg_start = nullptr;
  GatherSeg* d_gsegs = nullptr;
  GatherGrid* d_ggrid = nullptr;
  void *d_rpool = nullptr, *d_cpool = nullptr, *d_coef = nullptr;
  void* d_ws = nullptr;
  size_t plan_bytes = 0;

  std::string last_error = "no error";
  cudaStream_t last_stream = nullptr;
  int64_t last_launches = 0;

  // multi-step pushes replay captured steps (CUDA graphs) per field set, one
  // per step variant: 2 * (forward gathers) + (inverse writes the guards)
  cudaGraphExec_t graph_exec[4] = {};
  cudaStream_t cap_stream = nullptr;   // capture only; never executes work
  // host-buffer push: device staging fields and one copy stream per component;
  // the global-array variant also keeps the whole domain on the device and a
  // coupling of the plan's boxes with one box covering the domain
  void* global_stage[6] = {};
  psatd_coupling* global_coupling = nullptr;
  void* host_stage[6] = {};
  cudaStream_t copy_stream = nullptr;   // host paths: the copies (highest priority)
  cudaEvent_t copy_events[7] = {};
  FieldPtrs graph_fp{};
  int graph_nf = 0;
  int64_t graph_launches[4] = {};

  // per-kernel timing (diagnostics)
  bool timing = false;
  std::vector<cudaEvent_t> ev_pool;
  struct Rec {
    int kind;
    cudaEvent_t a, b;
  };
  std::vector<Rec> recs;

  DevPlan dev() const {
    DevPlan P;
    P.boxes = d_boxes;
    P.shapes = d_shapes;
    P.rpool = d_rpool;
    P.cpool = d_cpool;
    P.coef = d_coef;
    set_constants(P, desc.c, desc.eps0, desc.dt);
    return P;
  }

  ~psatd_plan() {
    cudaDeviceSynchronize();
    for (cudaGraphExec_t g : graph_exec)
      if (g) cudaGraphExecDestroy(g);
    if (cap_stream) cudaStreamDestroy(cap_stream);
    destroy_global_coupling(global_coupling);
    if (copy_stream) cudaStreamDestroy(copy_stream);
    for (cudaEvent_t e : copy_events)
      if (e) cudaEventDestroy(e);
    for (void* p : allocs) cudaFree(p);
    for (auto& r : recs) {
      ev_pool.push_back(r.a);
      ev_pool.push_back(r.b);
    }
    for (cudaEvent_t e : ev_pool) cudaEventDestroy(e);
  }

  cudaEvent_t take_event() {
    if (!ev_pool.empty()) {
      cudaEvent_t e = ev_pool.back();
      ev_pool.pop_back();
      return e;
    }
    cudaEvent_t e = nullptr;
    cudaEventCreate(&e);
    return e;
  }
};

namespace {

psatd_status fail(psatd_plan* p, psatd_status st, const std::string& m) {
  if (p)
    p->last_error = m;
  else
    g_thread_error = m;
  return st;
}

#define CK(plan, expr)                                                                          \
  do {                                                                                          \
    cudaError_t _e = (expr);                                                                    \
    if (_e != cudaSuccess) {                                                                    \
      psatd_status _s = _e == cudaErrorMemoryAllocation ? PSATD_ERR_OUT_OF_MEMORY : PSATD_ERR_CUDA; \
      return fail(plan, _s, fmt("%s: %s (%s:%d)", #expr, cudaGetErrorString(_e), __FILE__, __LINE__)); \
    }                                                                                           \
  } while (0)

template <typename V>
cudaError_t upload(psatd_plan* p, const std::vector<V>& h, V** d) {
  *d = nullptr;
  if (h.empty()) return cudaSuccess;
  cudaError_t e = cudaMalloc((void**)d, h.size() * sizeof(V));
  if (e != cudaSuccess) return e;
  p->allocs.push_back(*d);
  p->plan_bytes += h.size() * sizeof(V);
  return cudaMemcpy(*d, h.data(), h.size() * sizeof(V), cudaMemcpyHostToDevice);
}

cudaError_t dalloc(psatd_plan* p, size_t bytes, void** d) {
  *d = nullptr;
  if (!bytes) return cudaSuccess;
  cudaError_t e = cudaMalloc(d, bytes);
  if (e != cudaSuccess) return e;
  p->allocs.push_back(*d);
  p->plan_bytes += bytes;
  return cudaSuccess;
}


// Gather rectangles of plane z of box b for the deferred guard exchange: the
// rectangles of the exchange blocks that feed b's plane z (read from the
// owning interiors), then the cells no block feeds (interior, and guards
// outside a non-periodic domain) from b itself, consecutive equal rows merged.
// foff: element offset of every box in a field buffer; by_dst: the blocks
// (with a source box) of every destination box; v16: elements per 16 bytes.
static void plane_segs(const std::vector<psatd_box>& boxes, const std::vector<int64_t>& foff,
                       const std::vector<CopyBlk>& blocks, const std::vector<std::vector<int>>& by_dst, int b, int z,
                       int v16, std::vector<GatherSeg>* out) {
  auto emit = [&](int64_t src_off, int spitch, int dy, int dx, int ny, int nx) {
    GatherSeg g{};
    g.src_off = src_off;
    g.spitch = spitch;
    g.dy = dy;
    g.dx = dx;
    g.ny = ny;
    g.nx = nx;
    g.vec = nx % v16 == 0 && dx % v16 == 0 && src_off % v16 == 0 && spitch % v16 == 0;
    out->push_back(g);
  };
  const psatd_box& B = boxes[b];
  const int n0 = B.n[0], n1 = B.n[1];
  // covered[y]: x intervals of row y fed by a block
  std::vector<std::vector<std::pair<int, int>>> covered(n1);
  for (int bi : by_dst[b]) {
    const CopyBlk& c = blocks[bi];
    if (z < c.dst_lo[2] || z >= c.dst_lo[2] + c.ext[2]) continue;
    const psatd_box& S = boxes[c.src_box];
    const int64_t off =
        foff[c.src_box] + ((int64_t)(c.src_lo[2] + z - c.dst_lo[2]) * S.n[1] + c.src_lo[1]) * S.n[0] + c.src_lo[0];
    emit(off, S.n[0], c.dst_lo[1], c.dst_lo[0], c.ext[1], c.ext[0]);
    for (int y = c.dst_lo[1]; y < c.dst_lo[1] + c.ext[1]; ++y) covered[y].push_back({c.dst_lo[0], c.dst_lo[0] + c.ext[0]});
  }
  auto gaps = [&](int y) {
    auto iv = covered[y];
    std::sort(iv.begin(), iv.end());
    std::vector<std::pair<int, int>> g;
    int x = 0;
    for (const auto& v : iv) {
      if (v.first > x) g.push_back({x, v.first});
      x = std::max(x, v.second);
    }
    if (x < n0) g.push_back({x, n0});
    return g;
  };
  const int64_t base = foff[b] + (int64_t)z * n1 * n0;
  int y0 = 0;
  std::vector<std::pair<int, int>> cur = gaps(0);
  for (int y = 1; y <= n1; ++y) {
    std::vector<std::pair<int, int>> nx = y < n1 ? gaps(y) : std::vector<std::pair<int, int>>{{-1, -1}};
    if (y < n1 && nx == cur) continue;
    for (const auto& g : cur) emit(base + (int64_t)y0 * n0 + g.first, n0, y0, g.first, y - y0, g.second - g.first);
    y0 = y;
    cur.swap(nx);
  }
}

// The 3 x 3 grid form of a plane's rectangles (n0 x n1 plane), or false when
// the plane splits into more bands or a rectangle is not in 16-byte units.
static bool plane_grid(const GatherSeg* segs, int ns, int n0, int n1, GatherGrid* out) {
  std::vector<int> xs{0, n0}, ys{0, n1};
  for (int i = 0; i < ns; ++i) {
    if (!segs[i].vec) return false;
    xs.push_back(segs[i].dx);
    xs.push_back(segs[i].dx + segs[i].nx);
    ys.push_back(segs[i].dy);
    ys.push_back(segs[i].dy + segs[i].ny);
  }
  for (auto* v : {&xs, &ys}) {
    std::sort(v->begin(), v->end());
    v->erase(std::unique(v->begin(), v->end()), v->end());
  }
  if (xs.size() > 4 || ys.size() > 4) return false;
  while (xs.size() < 4) xs.push_back(n0);
  while (ys.size() < 4) ys.push_back(n1);
  GatherGrid gg{};
  gg.x1 = xs[1];
  gg.x2 = xs[2];
  gg.y1 = ys[1];
  gg.y2 = ys[2];
  for (int iy = 0; iy < 3; ++iy)
    for (int ix = 0; ix < 3; ++ix) {
      if (ys[iy] == ys[iy + 1] || xs[ix] == xs[ix + 1]) continue;   // empty cell
      bool found = false;
      for (int i = 0; i < ns && !found; ++i) {
        const GatherSeg& g = segs[i];
        if (g.dy <= ys[iy] && ys[iy + 1] <= g.dy + g.ny && g.dx <= xs[ix] && xs[ix + 1] <= g.dx + g.nx) {
          gg.base[3 * iy + ix] = g.src_off + (int64_t)(ys[iy] - g.dy) * g.spitch + (xs[ix] - g.dx);
          gg.pitch[3 * iy + ix] = g.spitch;
          found = true;
        }
      }
      if (!found) return false;
    }
  *out = gg;
  return true;
}

// Deferred guard exchange.  When every box runs on the register plane kernels
// (every guard block fed by an inverse plane pass) or every box on the pencil
// kernels (guard blocks stored by the step's exchange kernel), a step need
// not store its guard cells: the next step's forward x pass reads every guard
// cell straight from the interior cell that owns it, which is the value the
// exchange would have stored there, and only the last step of a push stores
// the guards.  Register plane plans keep rectangle lists where a plane is not
// a 3 x 3 grid; pencil plans take the grid form only.
static void build_gather(psatd_plan* P, const std::vector<char>& box_fast, uint32_t flags) {
  P->deferred = false;
  const int nb = (int)P->boxes.size();
  const bool reg = !P->grp_pf.empty() && P->grp_pf.front().code >= 0 && !P->segs.empty() && P->step_tiles.empty() &&
                   P->g_rows.empty() && P->pen_rows.empty() &&
                   std::all_of(box_fast.begin(), box_fast.end(), [](char f) { return f != 0; });
  const bool pen = P->pen_boxes == nb && !P->step_tiles.empty();
  if ((flags & PSATD_EAGER_EXCHANGE) || !(reg || pen)) return;
  std::vector<int64_t> foff(nb);
  for (int b = 0; b < nb; ++b) foff[b] = P->hboxes[b].foff;
  std::vector<std::vector<int>> by_dst(nb);
  for (int i = 0; i < (int)P->blocks.size(); ++i)
    if (P->blocks[i].src_box >= 0) by_dst[P->blocks[i].dst_box].push_back(i);
  const int v16 = 16 / (int)P->rsize;
  // every plane of every box: for register plane plans in the order of the
  // forward plane jobs (grouped by plane shape), else box-major
  std::vector<int2> planes;
  if (reg) {
    planes = P->plane_fwd;
  } else {
    for (int b = 0; b < nb; ++b)
      for (int z = 0; z < P->boxes[b].n[2]; ++z) planes.push_back(make_int2(b, z));
  }
  std::vector<GatherSeg> segs;
  std::vector<int> start{0};
  std::vector<GatherGrid> grids;
  bool all_grid = true;
  for (const int2& pl : planes) {
    const int b = pl.x, z = pl.y;
    plane_segs(P->boxes, foff, P->blocks, by_dst, b, z, v16, &segs);
    GatherGrid gg{};
    if (all_grid)
      all_grid = plane_grid(segs.data() + start.back(), (int)segs.size() - start.back(), P->boxes[b].n[0],
                            P->boxes[b].n[1], &gg);
    grids.push_back(gg);
    start.push_back((int)segs.size());
  }
  if (all_grid) {
    P->ggrid.swap(grids);
  } else if (reg) {
    P->gseg_start.swap(start);
    P->gsegs.swap(segs);
  } else {
    return;
  }
  P->deferred = true;
}

psatd_status build(psatd_plan* P, cudaStream_t st) {
  const psatd_plan_desc& d = P->desc;
  const int FIN = fields_in(P->form);
  // ---- shapes and table pool layout
  std::map<std::tuple<int, int, int, int>, int> shape_of;
  std::map<int, int64_t> tw_of;  // length -> complex pool offset
  int64_t rtot = 0, ctot = 0, qtot = 0;
  auto tw_offset = [&](int n) -> int64_t {
    auto it = tw_of.find(n);
    if (it != tw_of.end()) return it->second;
    const int64_t o = ctot;
    ctot += align_up(n, 2);
    tw_of[n] = o;
    return o;
  };
  for (const psatd_box& b : P->boxes) {
    auto key = std::make_tuple(b.n[0], b.n[1], b.n[2], b.order_p);
    if (shape_of.count(key)) continue;
    ShapeDev s{};
    for (int a = 0; a < 3; ++a) s.n[a] = b.n[a];
    s.L = b.n[0] / 2;
    s.hx = s.L + 1;
    s.p = b.order_p;
    if (!radix_plan(s.L, s.ax) || !radix_plan(b.n[1], s.ay) || !radix_plan(b.n[2], s.az))
      return fail(nullptr, PSATD_ERR_UNSUPPORTED_SIZE, "no radix schedule");
    s.ax.tw = tw_offset(s.L);
    s.ay.tw = tw_offset(b.n[1]);
    s.az.tw = tw_offset(b.n[2]);
    s.post = ctot;
    ctot += align_up(s.hx, 2);
    s.phx = ctot;
    ctot += align_up(s.hx, 2);
    s.phy = ctot;
    ctot += align_up(b.n[1], 2);
    s.phz = ctot;
    ctot += align_up(b.n[2], 2);
    s.kx = rtot;
    rtot += align_up(s.hx, 4);
    s.ky = rtot;
    rtot += align_up(b.n[1], 4);
    s.kz = rtot;
    rtot += align_up(b.n[2], 4);
    s.coef = qtot;
    qtot += (int64_t)s.hx * (b.n[1] / 2 + 1) * (b.n[2] / 2 + 1);
    s.fx = fast_code(s.L);
    s.fy = fast_code(b.n[1]);
    s.fz = fast_code(b.n[2]);
    s.px = pencil_code(s.L);
    s.py = pencil_code(b.n[1]);
    s.pz = pencil_code(b.n[2]);
    // x-pass row pitch = R2 (mod 16) and work pitch = 1 (mod 16) keep the
    // shared-memory accesses of the plane kernels free of most bank conflicts
    int r2x = 1;
#define PSATD_R2(code, N, R1, R2) if (s.fx == code) r2x = R2;
    PSATD_FAST_LENGTHS(PSATD_R2)
#undef PSATD_R2
    // forward plane buffer: even pitch >= hx (16-byte rows for cp.async),
    // close to R2 (mod 16); inverse row buffer: pitch >= hx, = 1 (mod 16)
    s.lp = s.hx;
    while (s.lp % 2 || (s.lp % 16 != r2x % 16 && s.lp % 16 != (r2x + 1) % 16)) ++s.lp;
    s.hp = s.hx + (int)((1 - s.hx % 16 + 32) % 16);
    shape_of[key] = (int)P->hshapes.size();
    P->hshapes.push_back(s);
  }
  // ---- boxes
  int64_t foff = 0, soff = 0;
  int32_t gplane = 0;
  for (const psatd_box& b : P->boxes) {
    BoxDev x{};
    for (int a = 0; a < 3; ++a) {
      x.n[a] = b.n[a];
      x.ng_lo[a] = b.ng_lo[a];
      x.ng_hi[a] = b.ng_hi[a];
    }
    x.shape = shape_of[std::make_tuple(b.n[0], b.n[1], b.n[2], b.order_p)];
    x.gplane = gplane;
    gplane += b.n[2];
    x.foff = foff;
    x.soff = soff;
    foff += align_up((int64_t)b.n[0] * b.n[1] * b.n[2], 64);
    soff += align_up((int64_t)(b.n[0] / 2 + 1) * b.n[1] * b.n[2], 32);
    P->hboxes.push_back(x);
  }
  P->field_total = foff;
  P->spec_total = soff;
  // ---- work lists
  const int csz = (int)P->csize;
  const int zbudget = 100 * 1024;
  int dev = 0, optin = 0;
  CK(P, cudaGetDevice(&dev));
  CK(P, cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev));
  CK(P, cudaDeviceGetAttribute(&P->sms, cudaDevAttrMultiProcessorCount, dev));
  const int tile = P->z_tile > 0 ? std::min(P->z_tile, fast_tile(P->prec)) : fast_tile(P->prec);
  // Kernel family of each box: plane kernels (x+y per z plane) for the boxes
  // whose plane shape has register-resident plane kernels (FP32, one launch
  // per shape); otherwise the pencil kernels (one launch per axis and FFT
  // length) take the boxes they accept, which measured faster than the
  // shared-memory plane kernels on mixed batches; the rest run on the
  // generic kernels.  PSATD_PENCIL_KERNELS and PSATD_PLANE_KERNELS
  // prefer one family outright, PSATD_GENERIC_KERNELS the generic kernels.
  auto plane_ok = [&](const psatd_box& b, const ShapeDev& sh) {
    const int L = b.n[0] / 2, n1 = b.n[1], n2 = b.n[2], hx = L + 1;
    const int ni = n1 - b.ng_lo[1] - b.ng_hi[1];
    const int sm_pf = 2 * n1 * sh.lp * csz, sm_pi = (2 * n1 * hx + ni * sh.hp) * csz;
    return !(d.flags & PSATD_GENERIC_KERNELS) && P->form != kPml && sh.fx >= 0 && sh.fy >= 0 && sh.fz >= 0 &&
           L <= fast_max_x(P->prec) && sm_pf <= optin && sm_pi <= optin &&
           z_fast_smem(P->prec, P->form, n2) <= optin;
  };
  // register plane shape of a box, or -1
  // register plane shape of a box, or -1: a shape with register plane
  // kernels and a z-pass kernel for its z length (register z, shared-memory
  // plane z or pencil z)
  auto reg_code_of = [&](const psatd_box& b, const ShapeDev& sh) {
    if (P->prec != 32 || (d.flags & PSATD_GENERIC_KERNELS) || P->form == kPml) return -1;
    const int c = reg_shape_code(sh.L, b.n[1]);
    if (c < 0 || reg_fwd_smem(c) > optin || reg_inv_smem(c) > optin) return -1;
    const int n2 = b.n[2], szf = z_fast_smem(P->prec, P->form, n2);
    const bool zr = z_reg_ok(n2) && z_reg_smem(P->form, n2) <= optin;
    const bool zf = sh.fz >= 0 && szf <= optin;
    const bool zp = sh.pz >= 0 && n2 <= pen_z_max(P->prec) && szf <= optin;
    if (!(zr || zf || zp)) return -1;
    P->reg_planes_used = true;
    return P->reg_planes ? c : -1;
  };
  std::vector<int> box_reg(P->boxes.size(), -1);
  for (int bi = 0; bi < (int)P->boxes.size(); ++bi) {
    const psatd_box& b = P->boxes[bi];
    const int n0 = b.n[0], n1 = b.n[1], n2 = b.n[2];
    const int L = n0 / 2, hx = L + 1;
    const ShapeDev& sh = P->hshapes[P->hboxes[bi].shape];
    const int ni = n1 - b.ng_lo[1] - b.ng_hi[1];
    const int sm_pf = 2 * n1 * sh.lp * csz, sm_pi = (2 * n1 * hx + ni * sh.hp) * csz;
    const int sm_zf = z_fast_smem(P->prec, P->form, n2);
    const bool fast_ok = plane_ok(b, sh);
    const int rows = n1 * n2;
    const int nr = std::max(1, std::min(rows, kMaxPoints / L));
    for (int r = 0; r < rows; r += nr) P->rows_all.push_back({bi, r, std::min(nr, rows - r), 0});
    for (int z = b.ng_lo[2]; z < n2 - b.ng_hi[2]; ++z) {
      const int y0 = b.ng_lo[1], y1 = n1 - b.ng_hi[1];
      for (int y = y0; y < y1; y += nr) P->rows_int.push_back({bi, z * n1 + y, std::min(nr, y1 - y), 0});
    }
    const bool pencil_ok = !(d.flags & PSATD_GENERIC_KERNELS) && P->form != kPml && sh.px >= 0 && sh.py >= 0 &&
                           sh.pz >= 0 &&
                           n2 <= pen_z_max(P->prec) && sm_zf <= optin && pen_col_smem(P->prec, n1) <= optin;
    box_reg[bi] = reg_code_of(b, sh);
    const bool prefer_pencil =
        (d.flags & PSATD_PENCIL_KERNELS) || (!(d.flags & PSATD_PLANE_KERNELS) && box_reg[bi] < 0);
    const bool fast = (fast_ok || box_reg[bi] >= 0) && !(pencil_ok && prefer_pencil);
    const bool pencil = !fast && pencil_ok;
    const bool generic = !fast && !pencil;   // the generic Stockham kernels
    if (fast) {
      ++P->fast_boxes;
      for (int z = 0; z < n2; ++z) {
        P->plane_fwd.push_back(make_int2(bi, z));
        if (z >= b.ng_lo[2] && z < n2 - b.ng_hi[2]) P->plane_inv.push_back(make_int2(bi, z));
      }
      // z pass: the shared-memory plane z kernel (or the register z kernel,
      // chosen below) where the z length has one, else the pencil z kernel
      const bool zf = sh.fz >= 0 && sm_zf <= optin;
      std::vector<ColJob>& zl = zf ? P->zfast : P->zpen;
      for (int y = 0; y < n1; ++y)
        for (int m = 0; m < L; m += tile) zl.push_back({bi, y, m, std::min(tile, L - m)});
      // the Nyquist column mx = L in tiles of consecutive y (negative count)
      for (int y = 0; y < n1; y += tile) zl.push_back({bi, y, L, -std::min(tile, n1 - y)});
      if (zf)
        P->smem_zf = std::max(P->smem_zf, sm_zf);
      else
        P->smem_penz = std::max(P->smem_penz, sm_zf);
      if (fast_ok) {   // buffers of the shared-memory plane kernels
        P->buf_pf = std::max(P->buf_pf, n1 * sh.lp);
        P->buf_pi = std::max(P->buf_pi, n1 * hx);
        P->rows_pi = std::max(P->rows_pi, ni * sh.hp);
      }
    } else if (pencil) {
      // pencil kernels: x rows, y tiles, z tiles (+ update), y tiles, x rows
      ++P->pen_boxes;
      const int pr = pen_rows(P->prec, L, rows, P->pen_rows_kb * 1024);
      for (int r = 0; r < rows; r += pr) P->pen_rows.push_back({bi, r, std::min(pr, rows - r), 0});
      const int y0 = b.ng_lo[1], y1 = n1 - b.ng_hi[1];
      const int pri = pen_rows(P->prec, L, y1 - y0, P->pen_rows_kb * 1024);
      for (int z = b.ng_lo[2]; z < n2 - b.ng_hi[2]; ++z)
        for (int y = y0; y < y1; y += pri) P->pen_rows_int.push_back({bi, z * n1 + y, std::min(pri, y1 - y), 0});
      const int ct = pen_col_tile(P->prec);
      for (int z = 0; z < n2; ++z)
        for (int m = 0; m < hx; m += ct) {
          const ColJob j{bi, z, m, std::min(ct, hx - m)};
          P->pen_ycols.push_back(j);
          if (z >= b.ng_lo[2] && z < n2 - b.ng_hi[2]) P->pen_ycols_int.push_back(j);
        }
      for (int y = 0; y < n1; ++y)
        for (int m = 0; m < L; m += tile) P->zpen.push_back({bi, y, m, std::min(tile, L - m)});
      for (int y = 0; y < n1; y += tile) P->zpen.push_back({bi, y, L, -std::min(tile, n1 - y)});
      P->smem_penx = std::max(P->smem_penx, pen_x_smem(P->prec, L, pr));
      P->smem_penxi = std::max(P->smem_penxi, pen_x_smem(P->prec, L, pri));
      P->smem_penc = std::max(P->smem_penc, pen_col_smem(P->prec, n1));
      P->smem_penz = std::max(P->smem_penz, sm_zf);
    } else {
      for (int r = 0; r < rows; r += nr) P->g_rows.push_back({bi, r, std::min(nr, rows - r), 0});
      for (int z = b.ng_lo[2]; z < n2 - b.ng_hi[2]; ++z) {
        const int y0 = b.ng_lo[1], y1 = n1 - b.ng_hi[1];
        for (int y = y0; y < y1; y += nr) P->g_rows_int.push_back({bi, z * n1 + y, std::min(nr, y1 - y), 0});
      }
    }
    P->smem_fx = std::max(P->smem_fx, nr * L * csz);
    P->smem_ix = std::max(P->smem_ix, nr * (hx + L) * csz);
    int ny = std::max(1, kMaxPoints / n1);
    if (ny >= 8) ny = ny / 8 * 8;
    ny = std::min(ny, hx);
    for (int z = 0; z < n2; ++z) {
      const bool inner = z >= b.ng_lo[2] && z < n2 - b.ng_hi[2];
      for (int m = 0; m < hx; m += ny) {
        ColJob j{bi, z, m, std::min(ny, hx - m)};
        P->ycols_all.push_back(j);
        if (inner) P->ycols_int.push_back(j);
        if (generic) {
          P->g_ycols.push_back(j);
          if (inner) P->g_ycols_int.push_back(j);
        }
      }
    }
    P->smem_y = std::max(P->smem_y, n1 * ny * csz);
    int nz = std::max(1, zbudget / (n2 * spec_slots(P->form) * csz));
    if (nz >= 4) nz = nz / 4 * 4;
    nz = std::min(nz, hx);
    for (int y = 0; y < n1; ++y)
      for (int m = 0; m < hx; m += nz) {
        P->zcols.push_back({bi, y, m, std::min(nz, hx - m)});
        if (generic) P->g_zcols.push_back({bi, y, m, std::min(nz, hx - m)});
      }
    P->smem_z = std::max(P->smem_z, n2 * spec_slots(P->form) * nz * csz);
    P->smem_zonly = std::max(P->smem_zonly, n2 * nz * csz);
  }
  // pencil jobs grouped by the FFT length of the axis each kernel transforms
  // (one launch per group; boxes keep their order inside a group)
  auto group = [&](auto& list, auto code_of, std::vector<psatd_plan::PenGroup>& groups) {
    std::stable_sort(list.begin(), list.end(),
                     [&](const auto& a, const auto& b) { return code_of(a) < code_of(b); });
    for (int64_t i = 0; i < (int64_t)list.size(); ++i) {
      const int c = code_of(list[i]);
      if (groups.empty() || groups.back().code != c) groups.push_back({c, i, 0});
      ++groups.back().count;
    }
  };
  auto shape_of_box = [&](int box) -> const ShapeDev& { return P->hshapes[P->hboxes[box].shape]; };
  // FP32 pencil boxes whose z length has a register z kernel: that kernel
  // does their z pass (z FFT, update, inverse z FFT), its jobs re-tiled to
  // its own tile width; the shared-memory pencil z kernel keeps the rest
  if (P->prec == 32 && !P->zpen.empty()) P->pen_reg_z_used = true;
  if (P->prec == 32 && P->pen_reg_z && !P->zpen.empty()) {
    std::vector<ColJob> keep;
    std::vector<char> done(P->boxes.size(), 0);
    for (const ColJob& j : P->zpen) {
      const psatd_box& b = P->boxes[j.box];
      if (!(z_reg_ok(b.n[2]) && z_reg_smem(P->form, b.n[2]) <= optin && z_reg_multi_smem(P->form) <= optin)) {
        keep.push_back(j);
        continue;
      }
      if (done[j.box]) continue;
      done[j.box] = 1;
      const int L = b.n[0] / 2, n1 = b.n[1], rt = z_reg_tile_width(P->form, b.n[2]);
      for (int y = 0; y < n1; ++y)
        for (int m = 0; m < L; m += rt) P->zpen_reg.push_back({j.box, y, m, std::min(rt, L - m)});
      for (int y = 0; y < n1; y += rt) P->zpen_reg.push_back({j.box, y, L, -std::min(rt, n1 - y)});
    }
    P->zpen.swap(keep);
  }
  if (P->fast_boxes && P->prec == 32) {
    // register plane kernels for the fast boxes with a register shape: the
    // plane jobs grouped by shape (one launch each), box order kept in a
    // group; the other fast boxes (code -1, first) on the shared-memory plane
    // kernels
    const bool all_reg = std::all_of(P->plane_fwd.begin(), P->plane_fwd.end(),
                                     [&](const int2& j) { return box_reg[j.x] >= 0; });
    const bool any_reg = std::any_of(P->plane_fwd.begin(), P->plane_fwd.end(),
                                     [&](const int2& j) { return box_reg[j.x] >= 0; });
    if (any_reg) {
      group(P->plane_fwd, [&](const int2& j) { return box_reg[j.x]; }, P->grp_pf);
      group(P->plane_inv, [&](const int2& j) { return box_reg[j.x]; }, P->grp_pi);
    }
    // one register z length for every fast box: its own launch (below);
    // several lengths, each with a register z kernel: the z jobs join the
    // register z list of the pencil boxes
    int nz = -2;
    for (const ColJob& j : P->zfast) {
      const int n2 = P->boxes[j.box].n[2];
      nz = (nz == -2 || nz == n2) ? n2 : -1;
      if (nz == -1) break;
    }
    const bool zreg_all = std::all_of(P->zfast.begin(), P->zfast.end(), [&](const ColJob& j) {
      const int n2 = P->boxes[j.box].n[2];
      return z_reg_ok(n2) && z_reg_smem(P->form, n2) <= optin && z_reg_multi_smem(P->form) <= optin;
    });
    if (nz == -1 && all_reg && zreg_all) P->pen_reg_z_used = true;
    if (nz == -1 && all_reg && zreg_all && P->pen_reg_z) {
      int last = -1;
      for (const ColJob& j : P->zfast) {
        if (j.box == last) continue;
        last = j.box;
        const int L = P->boxes[j.box].n[0] / 2, n1 = P->boxes[j.box].n[1];
        const int rt = z_reg_tile_width(P->form, P->boxes[j.box].n[2]);
        for (int y = 0; y < n1; ++y)
          for (int m = 0; m < L; m += rt) P->zpen_reg.push_back({j.box, y, m, std::min(rt, L - m)});
        for (int y = 0; y < n1; y += rt) P->zpen_reg.push_back({j.box, y, L, -std::min(rt, n1 - y)});
      }
      P->zfast.clear();
    }
  }
  group(P->zpen_reg, [&](const ColJob& j) { return P->boxes[j.box].n[2]; }, P->grp_zreg);
  P->zreg_multi = !P->zpen_reg.empty() && std::all_of(P->grp_zreg.begin(), P->grp_zreg.end(), [](const auto& g) {
    return z_reg_multi_ok(g.code) != 0;
  });
  group(P->pen_rows, [&](const RowJob& j) { return shape_of_box(j.box).px; }, P->grp_rows);
  group(P->pen_rows_int, [&](const RowJob& j) { return shape_of_box(j.box).px; }, P->grp_rows_int);
  group(P->pen_ycols, [&](const ColJob& j) { return shape_of_box(j.box).py; }, P->grp_ycols);
  group(P->pen_ycols_int, [&](const ColJob& j) { return shape_of_box(j.box).py; }, P->grp_ycols_int);
  group(P->zpen, [&](const ColJob& j) { return shape_of_box(j.box).pz; }, P->grp_z);
  if (P->fast_boxes && P->prec == 32 && !P->zfast.empty()) {
    // one register z length for every fast box, or none
    int nz = -2;
    for (const ColJob& j : P->zfast) {
      const int n2 = P->boxes[j.box].n[2];
      nz = (nz == -2 || nz == n2) ? n2 : -1;
      if (nz == -1) break;
    }
    if (nz > 0 && z_reg_ok(nz) && z_reg_smem(P->form, nz) <= optin) P->reg_z = nz;
    // the z stride, when every fast box shares it
    for (const ColJob& j : P->zfast) {
      const int zs = P->boxes[j.box].n[1] * (P->boxes[j.box].n[0] / 2 + 1);
      if (&j == &P->zfast.front())
        P->reg_zst = zs;
      else if (zs != P->reg_zst)
        P->reg_zst = 0;
    }
    // the register z kernel has its own tile width: re-tile (jobs are grouped by box)
    const int rt = P->reg_z ? z_reg_tile_width(P->form, P->reg_z) : tile;
    if (P->reg_z && rt != tile) {
      std::vector<ColJob> zt;
      int last = -1;
      for (const ColJob& j : P->zfast) {
        if (j.box == last) continue;
        last = j.box;
        const int L = P->boxes[j.box].n[0] / 2, n1 = P->boxes[j.box].n[1];
        for (int y = 0; y < n1; ++y)
          for (int m = 0; m < L; m += rt) zt.push_back({j.box, y, m, std::min(rt, L - m)});
        for (int y = 0; y < n1; y += rt) zt.push_back({j.box, y, L, -std::min(rt, n1 - y)});
      }
      P->zfast.swap(zt);
    }
  }
  if (P->fast_boxes) {
    P->smem_pf = 2 * P->buf_pf * csz;
    P->smem_pi = (2 * P->buf_pi + P->rows_pi) * csz;
    if (P->smem_pf > optin || P->smem_pi > optin)
      return fail(P, PSATD_ERR_UNSUPPORTED_SIZE, "plane buffers exceed shared memory");
  }
  // ---- exchange protocol
  P->blocks = build_blocks(&d);
  // Guard rectangles fed by fast boxes are written by the inverse plane
  // kernel itself (fused exchange); the step's exchange kernel keeps the
  // blocks whose source box runs on the generic kernels.  Blocks outside a
  // non-periodic domain (zero fill) keep the value written by the explicit
  // psatd_guard_exchange: no step writes those cells.
  std::vector<char> box_fast(P->boxes.size(), 0);
  std::map<std::pair<int, int>, int> plane_index;  // (box, z) -> plane_inv index
  for (int i = 0; i < (int)P->plane_inv.size(); ++i) {
    box_fast[P->plane_inv[i].x] = 1;
    plane_index[{P->plane_inv[i].x, P->plane_inv[i].y}] = i;
  }
  std::vector<std::vector<GuardSeg>> per_plane(P->plane_inv.size());
  const int v16 = 16 / (int)P->rsize;
  for (const CopyBlk& c : P->blocks) {
    if (c.src_box < 0 || !box_fast[c.src_box]) continue;
    const psatd_box& sb = P->boxes[c.src_box];
    const psatd_box& db = P->boxes[c.dst_box];
    const int nxi = sb.n[0] - sb.ng_lo[0] - sb.ng_hi[0];
    const bool vec = c.ext[0] % v16 == 0 && (c.src_lo[0] - sb.ng_lo[0]) % v16 == 0 && nxi % v16 == 0 &&
                     c.dst_lo[0] % v16 == 0 && db.n[0] % v16 == 0;
    for (int k = 0; k < c.ext[2]; ++k) {
      GuardSeg g{};
      g.dst_box = c.dst_box;
      g.dst_z = c.dst_lo[2] + k;
      g.sy = c.src_lo[1];
      g.sx = c.src_lo[0];
      g.ny = c.ext[1];
      g.nx = c.ext[0];
      g.dy = c.dst_lo[1];
      g.dx = c.dst_lo[0];
      g.vec = vec ? v16 : 1;
      per_plane[plane_index.at({c.src_box, c.src_lo[2] + k})].push_back(g);
    }
  }
  P->seg_start.assign(P->plane_inv.size() + 1, 0);
  for (size_t i = 0; i < per_plane.size(); ++i) {
    P->seg_start[i + 1] = P->seg_start[i] + (int)per_plane[i].size();
    P->segs.insert(P->segs.end(), per_plane[i].begin(), per_plane[i].end());
  }
  for (int i = 0; i < (int)P->blocks.size(); ++i) {
    const CopyBlk& c = P->blocks[i];
    const bool fused = c.src_box >= 0 && box_fast[c.src_box];
    const bool stepwise = c.src_box >= 0 && !fused;
    const int rows = c.ext[1] * c.ext[2];
    // 16-byte units when both rows start on 16-byte boundaries (box offsets
    // are 64-element aligned, so the row pitch and x offsets decide)
    const psatd_box& db = P->boxes[c.dst_box];
    bool vec = c.ext[0] % v16 == 0 && c.dst_lo[0] % v16 == 0 && db.n[0] % v16 == 0;
    if (c.src_box >= 0) vec = vec && c.src_lo[0] % v16 == 0 && P->boxes[c.src_box].n[0] % v16 == 0;
    const int unit = vec ? v16 : 1;
    const int per = std::max(1, 2048 * unit / std::max(1, c.ext[0]));
    for (int r = 0; r < rows; r += per) {
      P->tiles.push_back({i, r, std::min(per, rows - r), vec ? v16 : 1});
      if (stepwise) P->step_tiles.push_back({i, r, std::min(per, rows - r), vec ? v16 : 1});
    }
  }
  build_gather(P, box_fast, d.flags);
  // ---- device memory
  CK(P, upload(P, P->hboxes, &P->d_boxes));
  CK(P, upload(P, P->hshapes, &P->d_shapes));
  CK(P, upload(P, P->rows_all, &P->d_rows_all));
  CK(P, upload(P, P->rows_int, &P->d_rows_int));
  CK(P, upload(P, P->ycols_all, &P->d_ycols_all));
  CK(P, upload(P, P->ycols_int, &P->d_ycols_int));
  CK(P, upload(P, P->zcols, &P->d_zcols));
  CK(P, upload(P, P->g_rows, &P->d_g_rows));
  CK(P, upload(P, P->g_rows_int, &P->d_g_rows_int));
  CK(P, upload(P, P->g_ycols, &P->d_g_ycols));
  CK(P, upload(P, P->g_ycols_int, &P->d_g_ycols_int));
  CK(P, upload(P, P->g_zcols, &P->d_g_zcols));
  CK(P, upload(P, P->zfast, &P->d_zfast));
  CK(P, upload(P, P->plane_fwd, &P->d_plane_fwd));
  CK(P, upload(P, P->plane_inv, &P->d_plane_inv));
  CK(P, upload(P, P->pen_rows, &P->d_pen_rows));
  CK(P, upload(P, P->pen_rows_int, &P->d_pen_rows_int));
  CK(P, upload(P, P->pen_ycols, &P->d_pen_ycols));
  CK(P, upload(P, P->pen_ycols_int, &P->d_pen_ycols_int));
  CK(P, upload(P, P->zpen, &P->d_zpen));
  CK(P, upload(P, P->zpen_reg, &P->d_zpen_reg));
  CK(P, upload(P, P->blocks, &P->d_blocks));
  CK(P, upload(P, P->tiles, &P->d_tiles));
  CK(P, upload(P, P->step_tiles, &P->d_step_tiles));
  CK(P, upload(P, P->seg_start, &P->d_seg_start));
  CK(P, upload(P, P->segs, &P->d_segs));
  CK(P, upload(P, P->gseg_start, &P->d_gseg_start));
  CK(P, upload(P, P->gsegs, &P->d_gsegs));
  CK(P, upload(P, P->ggrid, &P->d_ggrid));
  CK(P, dalloc(P, (size_t)rtot * P->rsize, &P->d_rpool));
  CK(P, dalloc(P, (size_t)ctot * P->csize, &P->d_cpool));
  CK(P, dalloc(P, (size_t)qtot * 4 * P->rsize, &P->d_coef));
  CK(P, dalloc(P, (size_t)spec_slots(P->form) * P->spec_total * P->csize, &P->d_ws));
  // ---- FP64 tables
  double *r64 = nullptr, *alpha = nullptr;
  double2* c64 = nullptr;
  Coef4<double>* q64 = nullptr;
  std::vector<void*> tmp;
  auto tmp_alloc = [&](size_t bytes, void** ptr) -> cudaError_t {
    cudaError_t e = cudaMalloc(ptr, std::max<size_t>(bytes, 16));
    if (e == cudaSuccess) tmp.push_back(*ptr);
    return e;
  };
  auto free_tmp = [&]() {
    cudaStreamSynchronize(st);
    for (void* t : tmp) cudaFree(t);
    tmp.clear();
  };
  cudaError_t e = cudaSuccess;
  if (P->prec == 32) {
    e = tmp_alloc((size_t)rtot * 8, (void**)&r64);
    if (e == cudaSuccess) e = tmp_alloc((size_t)ctot * 16, (void**)&c64);
    if (e == cudaSuccess) e = tmp_alloc((size_t)qtot * 32, (void**)&q64);
  } else {
    r64 = (double*)P->d_rpool;
    c64 = (double2*)P->d_cpool;
    q64 = (Coef4<double>*)P->d_coef;
  }
  // stencil weights of every order used
  std::map<int, int64_t> alpha_of;
  std::vector<double> halpha;
  for (const ShapeDev& s : P->hshapes) {
    if (s.p == 0 || alpha_of.count(s.p)) continue;
    alpha_of[s.p] = (int64_t)halpha.size();
    auto a = stencil_alpha(s.p, (d.flags & PSATD_NODAL) != 0);
    halpha.insert(halpha.end(), a.begin(), a.end());
  }
  if (e == cudaSuccess) e = tmp_alloc(halpha.size() * 8, (void**)&alpha);
  if (e == cudaSuccess && !halpha.empty())
    e = cudaMemcpy(alpha, halpha.data(), halpha.size() * 8, cudaMemcpyHostToDevice);
  for (auto& kv : tw_of)
    if (e == cudaSuccess) e = gen_twiddles(c64 + kv.second, kv.first, st);
  for (const ShapeDev& s : P->hshapes) {
    if (e != cudaSuccess) break;
    const int q = s.p / 2;
    const double* al = q ? alpha + alpha_of[s.p] : alpha;
    e = gen_post(c64 + s.post, s.n[0], st);
    const int nodal = (d.flags & PSATD_NODAL) != 0;
    if (e == cudaSuccess) e = gen_axis(r64 + s.kx, c64 + s.phx, s.hx, s.n[0], d.dx[0], q, al, nodal, st);
    if (e == cudaSuccess) e = gen_axis(r64 + s.ky, c64 + s.phy, s.n[1], s.n[1], d.dx[1], q, al, nodal, st);
    if (e == cudaSuccess) e = gen_axis(r64 + s.kz, c64 + s.phz, s.n[2], s.n[2], d.dx[2], q, al, nodal, st);
    if (e == cudaSuccess)
      e = gen_coef(q64 + s.coef, s.hx, s.n[1], s.n[2], r64 + s.kx, r64 + s.ky, r64 + s.kz, d.c, d.dt, st);
  }
  if (e == cudaSuccess && P->prec == 32)
    e = convert_pools(r64, (float*)P->d_rpool, rtot, c64, (float2*)P->d_cpool, ctot, q64,
                      (Coef4<float>*)P->d_coef, qtot, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  free_tmp();
  CK(P, e);
  const int smem = std::max({P->smem_fx, P->smem_y, P->smem_z, P->smem_zonly, P->smem_ix, P->smem_pf,
                             P->smem_pi, P->smem_zf, P->smem_penx, P->smem_penxi, P->smem_penc, P->smem_penz});
  if (smem > optin) return fail(P, PSATD_ERR_UNSUPPORTED_SIZE, fmt("needs %d B shared memory", smem));
  // The attribute is a per-kernel cap shared by every plan: raise it to the
  // device maximum so that no plan lowers it below another plan's need.
  CK(P, configure_kernels(P->prec, optin));
  CK(P, configure_fast_kernels(P->prec, optin));
  CK(P, configure_pen_kernels(P->prec, optin));
  if (P->prec == 32) CK(P, configure_reg_kernels(optin));
  if (P->fast_boxes) {
    int sms = 0, occ_f = 0, occ_i = 0;
    CK(P, cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    CK(P, plane_occupancy(P->prec, P->smem_pf, P->smem_pi, &occ_f, &occ_i));
    if (occ_f < 1 || occ_i < 1) return fail(P, PSATD_ERR_UNSUPPORTED_SIZE, "plane kernels do not fit an SM");
    const int FINv = fields_in(P->form), FOUTv = fields_out(P->form);
    P->grid_pf = (int)std::min<int64_t>((int64_t)occ_f * sms, (int64_t)P->plane_fwd.size() * FINv);
    P->grid_pi = (int)std::min<int64_t>((int64_t)occ_i * sms, (int64_t)P->plane_inv.size() * FOUTv);
  }
  return PSATD_OK;
}

// Absorbing layers: the boxes whose interiors reach into a layer, the
// damping table exp(-s_d(g + o/2) dt) per axis d, Yee offset o and global
// index g (FP64, rounded once), the stored split parts (zero) and the
// buffers of their per-step increments.
psatd_status build_pml(psatd_plan* P, cudaStream_t st) {
  if (P->form != kPml) return PSATD_OK;
  const psatd_plan_desc& d = P->desc;
  for (int i = 0; i < (int)P->boxes.size(); ++i) {
    const psatd_box& b = P->boxes[i];
    bool touches = false;
    for (int a = 0; a < 3; ++a) {
      const int64_t w = P->pml.width[a], m = b.n[a] - b.ng_lo[a] - b.ng_hi[a];
      if (w > 0 && (b.origin[a] < w || b.origin[a] + m > d.global_n[a] - w)) touches = true;
    }
    if (touches)
      P->pml_boxes.push_back(PmlBox{i, {(int32_t)b.origin[0], (int32_t)b.origin[1], (int32_t)b.origin[2]}});
  }
  std::vector<double> tab;
  for (int a = 0; a < 3; ++a)
    for (int o = 0; o < 2; ++o) {
      P->pml_tab.off[a][o] = (int64_t)tab.size();
      const double N = d.global_n[a], w = P->pml.width[a];
      for (int g = 0; g < d.global_n[a]; ++g) {
        const double pos = g + 0.5 * o;
        double xi = 0.0;
        if (w > 0 && pos < w)
          xi = w - pos;
        else if (w > 0 && pos > N - w)
          xi = pos - (N - w);
        xi = std::min(xi, w);
        const double sig = xi > 0 ? P->pml.sigma_max[a] * std::pow(xi / w, (double)P->pml.order) : 0.0;
        tab.push_back(std::exp(-sig * d.dt));
      }
    }
  if (P->prec == 32) {
    std::vector<float> t32(tab.begin(), tab.end());
    float* dt32 = nullptr;
    CK(P, upload(P, t32, &dt32));
    P->d_pml_tab = dt32;
  } else {
    double* dt64 = nullptr;
    CK(P, upload(P, tab, &dt64));
    P->d_pml_tab = dt64;
  }
  CK(P, upload(P, P->pml_boxes, &P->d_pml_boxes));
  const size_t bytes = (size_t)P->field_total * P->rsize;
  for (int q = 0; q < 6; ++q) {
    CK(P, dalloc(P, bytes, &P->pml_parts[q]));
    CK(P, dalloc(P, bytes, &P->pml_inc[q]));
    CK(P, cudaMemsetAsync(P->pml_parts[q], 0, bytes, st));
    CK(P, cudaMemsetAsync(P->pml_inc[q], 0, bytes, st));
  }
  CK(P, cudaStreamSynchronize(st));
  return PSATD_OK;
}

bool aligned16(const void* p) { return ((uintptr_t)p & 15u) == 0; }

// Run one launch, bracketed by events when the plan records kernel times.
template <typename F>
cudaError_t timed(psatd_plan* P, int kind, cudaStream_t st, F&& launch) {
  if (!P->timing) return launch();
  cudaEvent_t a = P->take_event(), b = P->take_event();
  if (!a || !b) return cudaErrorMemoryAllocation;
  cudaError_t e = cudaEventRecord(a, st);
  if (e == cudaSuccess) e = launch();
  if (e == cudaSuccess) e = cudaEventRecord(b, st);
  P->recs.push_back({kind, a, b});
  return e;
}

}  // namespace

// ===========================================================================
// C ABI
// ===========================================================================
// ---------------------------------------------------------------------------
// dual-grid coupling (paper Sec. 2.5.2): copy blocks between two layouts of
// one global domain.  Every cell of every destination box (guards included)
// reads the source-layout interior cell with the same global index.
// ---------------------------------------------------------------------------
namespace {

std::vector<CopyBlk> coupling_blocks(const std::vector<psatd_box>& dst, const std::vector<psatd_box>& src,
                                     const int64_t N[3], const bool per[3]) {
  std::vector<CopyBlk> out;
  for (int b = 0; b < (int)dst.size(); ++b) {
    const psatd_box& B = dst[b];
    std::vector<Seg> sg3[3];
    for (int a = 0; a < 3; ++a) sg3[a] = axis_segments(B.origin[a] - B.ng_lo[a], B.n[a], N[a], per[a]);
    for (const Seg& sz : sg3[2])
      for (const Seg& sy : sg3[1])
        for (const Seg& sx : sg3[0]) {
          const Seg* sg[3] = {&sx, &sy, &sz};
          if (sx.outside || sy.outside || sz.outside) {
            CopyBlk c{};
            c.dst_box = b;
            c.src_box = -1;
            for (int a = 0; a < 3; ++a) {
              c.dst_lo[a] = (int32_t)sg[a]->dst;
              c.ext[a] = (int32_t)sg[a]->len;
            }
            out.push_back(c);
            continue;
          }
          for (int sb = 0; sb < (int)src.size(); ++sb) {
            const psatd_box& S = src[sb];
            int64_t lo[3], hi[3];
            bool empty = false;
            for (int a = 0; a < 3; ++a) {
              const int64_t sm = S.n[a] - S.ng_lo[a] - S.ng_hi[a];
              lo[a] = std::max(sg[a]->g, S.origin[a]);
              hi[a] = std::min(sg[a]->g + sg[a]->len, S.origin[a] + sm);
              if (hi[a] <= lo[a]) empty = true;
            }
            if (empty) continue;
            CopyBlk c{};
            c.dst_box = b;
            c.src_box = sb;
            for (int a = 0; a < 3; ++a) {
              c.dst_lo[a] = (int32_t)(sg[a]->dst + (lo[a] - sg[a]->g));
              c.src_lo[a] = (int32_t)(lo[a] - S.origin[a] + S.ng_lo[a]);
              c.ext[a] = (int32_t)(hi[a] - lo[a]);
            }
            out.push_back(c);
          }
        }
  }
  return out;
}

// Tiles of up to ~2048 units (16-byte units where both rows allow them).
std::vector<XTile> block_tiles(const std::vector<CopyBlk>& blocks, const std::vector<psatd_box>& dst,
                               const std::vector<psatd_box>& src, int v16) {
  std::vector<XTile> tiles;
  for (int i = 0; i < (int)blocks.size(); ++i) {
    const CopyBlk& c = blocks[i];
    const int rows = c.ext[1] * c.ext[2];
    bool vec = c.ext[0] % v16 == 0 && c.dst_lo[0] % v16 == 0 && dst[c.dst_box].n[0] % v16 == 0;
    if (c.src_box >= 0) vec = vec && c.src_lo[0] % v16 == 0 && src[c.src_box].n[0] % v16 == 0;
    const int unit = vec ? v16 : 1;
    const int per = std::max(1, 2048 * unit / std::max(1, c.ext[0]));
    for (int r = 0; r < rows; r += per) tiles.push_back({i, r, std::min(per, rows - r), vec ? v16 : 1});
  }
  return tiles;
}

// G1 boxes: positive interiors inside the domain that tile it exactly.
Err validate_g1(const psatd_plan_desc& d, int32_t n, const psatd_box* g1) {
  if (d.decomp == PSATD_DECOMP_INDEPENDENT) return {PSATD_ERR_INVALID_ARG, "independent boxes share no domain"};
  if (n <= 0 || !g1) return {PSATD_ERR_INVALID_ARG, "no G1 boxes"};
  int64_t vol = 0;
  for (int b = 0; b < n; ++b) {
    int64_t v = 1;
    for (int a = 0; a < 3; ++a) {
      const psatd_box& B = g1[b];
      const int64_t m = (int64_t)B.n[a] - B.ng_lo[a] - B.ng_hi[a];
      if (B.ng_lo[a] < 0 || B.ng_hi[a] < 0 || m < 1)
        return {PSATD_ERR_INVALID_ARG, fmt("G1 box %d: empty interior or negative guards", b)};
      if (B.origin[a] < 0 || B.origin[a] + m > d.global_n[a])
        return {PSATD_ERR_INVALID_ARG, fmt("G1 box %d: interior outside the domain", b)};
      v *= m;
    }
    vol += v;
  }
  if (vol != (int64_t)d.global_n[0] * d.global_n[1] * d.global_n[2])
    return {PSATD_ERR_INVALID_ARG, "G1 interiors do not tile the domain"};
  for (int b = 0; b < n; ++b)
    for (int c = b + 1; c < n; ++c) {
      bool overlap = true;
      for (int a = 0; a < 3; ++a) {
        const psatd_box &B = g1[b], &C = g1[c];
        const int64_t mb = B.n[a] - B.ng_lo[a] - B.ng_hi[a], mc = C.n[a] - C.ng_lo[a] - C.ng_hi[a];
        overlap = overlap && B.origin[a] < C.origin[a] + mc && C.origin[a] < B.origin[a] + mb;
      }
      if (overlap) return {PSATD_ERR_INVALID_ARG, fmt("G1 boxes %d and %d overlap", b, c)};
    }
  return {PSATD_OK, ""};
}

void domain_of(const psatd_plan_desc& d, int64_t N[3], bool per[3]) {
  for (int a = 0; a < 3; ++a) {
    N[a] = d.global_n[a];
    per[a] = d.periodic[a] != 0;
  }
}

}  // namespace

struct psatd_coupling {
  psatd_plan* plan = nullptr;
  std::vector<psatd_box> g1;
  std::vector<BoxDev> hg1;
  int64_t field_total = 0;
  std::vector<CopyBlk> blk[2];
  std::vector<XTile> tiles[2];
  BoxDev* d_g1 = nullptr;
  CopyBlk* d_blk[2] = {nullptr, nullptr};
  XTile* d_tiles[2] = {nullptr, nullptr};
  std::vector<void*> allocs;
  ~psatd_coupling() {
    cudaDeviceSynchronize();
    for (void* q : allocs) cudaFree(q);
  }
  template <typename V>
  cudaError_t up(const std::vector<V>& h, V** dptr) {
    *dptr = nullptr;
    if (h.empty()) return cudaSuccess;
    cudaError_t e = cudaMalloc((void**)dptr, h.size() * sizeof(V));
    if (e != cudaSuccess) return e;
    allocs.push_back(*dptr);
    return cudaMemcpy(*dptr, h.data(), h.size() * sizeof(V), cudaMemcpyHostToDevice);
  }
};

static void destroy_global_coupling(psatd_coupling* c) { delete c; }

extern "C" {

psatd_status psatd_plan_validate(const psatd_plan_desc* desc, char* msg, size_t msg_len) {
  try {
    Err e = validate(desc);
    set_msg(msg, msg_len, e.st == PSATD_OK ? "ok" : e.msg);
    if (e.st != PSATD_OK) g_thread_error = e.msg;
    return e.st;
  } catch (...) {
    return PSATD_ERR_INVALID_ARG;
  }
}

psatd_status psatd_exchange_blocks(const psatd_plan_desc* desc, psatd_copy_block* out, int64_t cap,
                                   int64_t* count) {
  try {
    if (!count || cap < 0 || (cap > 0 && !out)) return fail(nullptr, PSATD_ERR_INVALID_ARG, "bad output arguments");
    Err e = validate(desc);
    if (e.st != PSATD_OK) return fail(nullptr, e.st, e.msg);
    std::vector<CopyBlk> b = build_blocks(desc);
    *count = (int64_t)b.size();
    for (int64_t i = 0; i < std::min<int64_t>(cap, (int64_t)b.size()); ++i) {
      psatd_copy_block& o = out[i];
      o.dst_box = b[i].dst_box;
      o.src_box = b[i].src_box;
      for (int a = 0; a < 3; ++a) {
        o.dst_lo[a] = b[i].dst_lo[a];
        o.src_lo[a] = b[i].src_lo[a];
        o.ext[a] = b[i].ext[a];
      }
    }
    return PSATD_OK;
  } catch (...) {
    return fail(nullptr, PSATD_ERR_INVALID_ARG, "internal error");
  }
}

psatd_status psatd_plane_gather(const psatd_plan_desc* desc, int32_t box, int32_t z, int32_t* src_box,
                                int64_t* src_cell, int32_t* is_grid) {
  try {
    if (!src_box || !src_cell || !is_grid) return fail(nullptr, PSATD_ERR_INVALID_ARG, "NULL output");
    Err e = validate(desc);
    if (e.st != PSATD_OK) return fail(nullptr, e.st, e.msg);
    if (box < 0 || box >= desc->num_boxes || z < 0 || z >= desc->boxes[box].n[2])
      return fail(nullptr, PSATD_ERR_INVALID_ARG, "box or plane out of range");
    const int nb = desc->num_boxes;
    const std::vector<psatd_box> boxes(desc->boxes, desc->boxes + nb);
    // box offsets in a field buffer, as the plan lays them out
    std::vector<int64_t> foff(nb + 1, 0);
    for (int b = 0; b < nb; ++b)
      foff[b + 1] = foff[b] + align_up((int64_t)boxes[b].n[0] * boxes[b].n[1] * boxes[b].n[2], 64);
    const std::vector<CopyBlk> blocks = build_blocks(desc);
    std::vector<std::vector<int>> by_dst(nb);
    for (int i = 0; i < (int)blocks.size(); ++i)
      if (blocks[i].src_box >= 0) by_dst[blocks[i].dst_box].push_back(i);
    std::vector<GatherSeg> segs;
    plane_segs(boxes, foff, blocks, by_dst, box, z, desc->precision == 32 ? 4 : 2, &segs);
    const int n0 = boxes[box].n[0], n1 = boxes[box].n[1];
    GatherGrid gg{};
    const bool grid = plane_grid(segs.data(), (int)segs.size(), n0, n1, &gg);
    *is_grid = grid ? 1 : 0;
    for (int y = 0; y < n1; ++y)
      for (int x = 0; x < n0; ++x) {
        int64_t off = -1;
        if (grid) {
          const int iy = (y >= gg.y1) + (y >= gg.y2), ix = (x >= gg.x1) + (x >= gg.x2);
          const int ylo = iy == 0 ? 0 : iy == 1 ? gg.y1 : gg.y2, xlo = ix == 0 ? 0 : ix == 1 ? gg.x1 : gg.x2;
          off = gg.base[3 * iy + ix] + (int64_t)(y - ylo) * gg.pitch[3 * iy + ix] + (x - xlo);
        } else {
          for (const GatherSeg& g : segs)
            if (y >= g.dy && y < g.dy + g.ny && x >= g.dx && x < g.dx + g.nx) {
              off = g.src_off + (int64_t)(y - g.dy) * g.spitch + (x - g.dx);
              break;
            }
        }
        if (off < 0) return fail(nullptr, PSATD_ERR_INVALID_ARG, "internal error: uncovered cell");
        const int sb = (int)(std::upper_bound(foff.begin(), foff.end(), off) - foff.begin()) - 1;
        src_box[(int64_t)y * n0 + x] = sb;
        src_cell[(int64_t)y * n0 + x] = off - foff[sb];
      }
    return PSATD_OK;
  } catch (...) {
    return fail(nullptr, PSATD_ERR_INVALID_ARG, "internal error");
  }
}

psatd_status psatd_plan_create(const psatd_plan_desc* desc, void* stream, psatd_plan** out) {
  if (!out) return fail(nullptr, PSATD_ERR_INVALID_ARG, "out is NULL");
  *out = nullptr;
  psatd_plan* P = nullptr;
  try {
    Err v = validate(desc);
    if (v.st != PSATD_OK) return fail(nullptr, v.st, v.msg);
    P = new psatd_plan();
    P->desc = *desc;
    P->boxes.assign(desc->boxes, desc->boxes + desc->num_boxes);
    P->desc.boxes = P->boxes.data();
    P->prec = desc->precision;
    P->csize = P->prec == 32 ? 8 : 16;
    P->rsize = P->prec == 32 ? 4 : 8;
    P->form = (desc->flags & PSATD_VACUUM) ? kVacuum : (desc->flags & PSATD_RHO_CONTINUITY) ? kRhoForm : kJForm;
    if (desc->pml) {
      P->pml = *desc->pml;
      P->desc.pml = &P->pml;
      P->form = kPml;
    }
    P->desc.tuning = nullptr;   // read here only
    for (int i = 0; desc->tuning && i < 16 && desc->tuning[2 * i] != 0; ++i) {
      const int32_t k = desc->tuning[2 * i], v = desc->tuning[2 * i + 1];
      if (k == PSATD_TUNE_Z_PREFETCH) P->z_prefetch = v;
      if (k == PSATD_TUNE_PENCIL_ROWS_KB) P->pen_rows_kb = v;
      if (k == PSATD_TUNE_Z_TILE) P->z_tile = v;
      if (k == PSATD_TUNE_HOST_COPY) P->host_copy = v;
      if (k == PSATD_TUNE_PENCIL_REG_Z) P->pen_reg_z = v;
      if (k == PSATD_TUNE_Z_ONE_LAUNCH) P->z_one_launch = v;
      if (k == PSATD_TUNE_REG_PLANES) P->reg_planes = v;
    }
    int dev = 0;
    cudaError_t ce = cudaGetDevice(&dev);
    if (ce != cudaSuccess) {
      std::string m = fmt("no CUDA device: %s", cudaGetErrorString(ce));
      delete P;
      return fail(nullptr, PSATD_ERR_CUDA, m);
    }
    psatd_status s = build(P, (cudaStream_t)stream);
    if (s == PSATD_OK) s = build_pml(P, (cudaStream_t)stream);
    if (s != PSATD_OK) {
      std::string m = P->last_error != "no error" ? P->last_error : g_thread_error;
      delete P;
      return fail(nullptr, s, m);
    }
    P->last_stream = (cudaStream_t)stream;
    *out = P;
    return PSATD_OK;
  } catch (const std::bad_alloc&) {
    delete P;
    return fail(nullptr, PSATD_ERR_OUT_OF_MEMORY, "host allocation failed");
  } catch (...) {
    delete P;
    return fail(nullptr, PSATD_ERR_INVALID_ARG, "internal error");
  }
}

psatd_status psatd_plan_destroy(psatd_plan* plan) {
  delete plan;
  return PSATD_OK;
}

psatd_status psatd_plan_layout(const psatd_plan* p, int32_t box, int64_t* off, int64_t* elems) {
  if (!p || !off || !elems) return PSATD_ERR_INVALID_ARG;
  if (box < 0 || box >= (int32_t)p->hboxes.size()) return PSATD_ERR_INVALID_ARG;
  const BoxDev& b = p->hboxes[box];
  *off = b.foff;
  *elems = (int64_t)b.n[0] * b.n[1] * b.n[2];
  return PSATD_OK;
}

psatd_status psatd_plan_spectrum_layout(const psatd_plan* p, int32_t box, int64_t* off,
                                        int64_t* elems) {
  if (!p || !off || !elems) return PSATD_ERR_INVALID_ARG;
  if (box < 0 || box >= (int32_t)p->hboxes.size()) return PSATD_ERR_INVALID_ARG;
  const BoxDev& b = p->hboxes[box];
  *off = b.soff;
  *elems = (int64_t)(b.n[0] / 2 + 1) * b.n[1] * b.n[2];
  return PSATD_OK;
}

psatd_status psatd_plan_memory(const psatd_plan* p, size_t* field_bytes, size_t* workspace_bytes) {
  if (!p) return PSATD_ERR_INVALID_ARG;
  if (field_bytes) *field_bytes = (size_t)p->field_total * p->rsize;
  if (workspace_bytes) *workspace_bytes = p->plan_bytes;
  return PSATD_OK;
}

static psatd_status gather_fields(psatd_plan* P, const psatd_fields* f, const psatd_sources* s,
                                  bool with_sources_for_form, FieldPtrs* fp, int* nf) {
  if (!f) return fail(P, PSATD_ERR_INVALID_ARG, "fields is NULL");
  std::memset(fp, 0, sizeof *fp);
  for (int a = 0; a < 3; ++a) {
    fp->p[a] = f->E[a];
    fp->p[3 + a] = f->B[a];
  }
  int n = 6;
  if (with_sources_for_form) {
    if (P->form == kJForm) {
      if (!s) return fail(P, PSATD_ERR_INVALID_ARG, "sources required (plan is not PSATD_VACUUM)");
      for (int a = 0; a < 3; ++a) fp->p[6 + a] = const_cast<void*>(s->J[a]);
      n = 9;
    } else if (P->form == kRhoForm) {
      if (!s) return fail(P, PSATD_ERR_INVALID_ARG, "sources required (plan is not PSATD_VACUUM)");
      fp->p[6] = s->rho;
      for (int a = 0; a < 3; ++a) fp->p[7 + a] = const_cast<void*>(s->J[a]);
      n = 10;
    }
  } else if (s) {
    for (int a = 0; a < 3; ++a) fp->p[6 + a] = const_cast<void*>(s->J[a]);
    n = 9;
    if (s->rho) fp->p[n++] = s->rho;
  }
  for (int i = 0; i < n; ++i) {
    if (!fp->p[i]) return fail(P, PSATD_ERR_INVALID_ARG, fmt("field slot %d is NULL", i));
    if (!aligned16(fp->p[i])) return fail(P, PSATD_ERR_INVALID_ARG, fmt("field slot %d not 16-byte aligned", i));
  }
  if (P->form == kPml && with_sources_for_form)   // the inverse pass writes the split-part increments there
    for (int q = 0; q < 6; ++q) fp->p[6 + q] = P->pml_inc[q];
  *nf = n;
  return PSATD_OK;
}

psatd_status psatd_guard_exchange(psatd_plan* P, const psatd_fields* f, const psatd_sources* s,
                                  void* stream) {
  if (!P) return PSATD_ERR_INVALID_ARG;
  try {
    FieldPtrs fp;
    int nf = 0;
    psatd_status r = gather_fields(P, f, s, false, &fp, &nf);
    if (r != PSATD_OK) return r;
    cudaStream_t st = (cudaStream_t)stream;
    P->last_stream = st;
    CK(P, launch_exchange(P->prec, P->dev(), fp, nf, P->d_blocks, P->d_tiles, (int64_t)P->tiles.size(), st));
    return PSATD_OK;
  } catch (...) {
    return fail(P, PSATD_ERR_INVALID_ARG, "internal error");
  }
}

// S1 along x and y of the field slots fp.p[0..nf) into spectrum slots
// spec + f * spec_total, on every kernel family; adds the launches.
static psatd_status forward_xy(psatd_plan* P, const DevPlan& D, const FieldPtrs& fp, int nf, void* spec,
                               cudaStream_t st, int64_t* launches_out, bool gather = false) {
  const int64_t S = P->spec_total;
  int64_t launches = 0;
  // fast boxes: one plane kernel; generic: x rows, y columns; pencil: x rows, y tiles
  if (!P->grp_pf.empty()) {
    // one launch per register plane shape; the gather tables are indexed by plane_fwd position
    for (const auto& g : P->grp_pf) {
      if (g.code < 0) {
        CK(P, timed(P, 0, st, [&] {
             return launch_plane_fwd(P->prec, D, fp, nf, spec, S, P->d_plane_fwd + g.start, g.count, P->buf_pf,
                                     P->smem_pf, P->grid_pf, st);
           }));
        ++launches;
        continue;
      }
      CK(P, timed(P, 0, st, [&] {
           return launch_plane_fwd_reg(g.code, D, fp, nf, spec, S, P->d_plane_fwd + g.start, g.count,
                                       gather && !P->gseg_start.empty() ? P->d_gseg_start + g.start : nullptr,
                                       P->d_gsegs, gather && !P->ggrid.empty() ? P->d_ggrid + g.start : nullptr,
                                       fields_out(P->form), st);
         }));
      ++launches;
    }
  } else if (!P->plane_fwd.empty()) {
    CK(P, timed(P, 0, st, [&] {
         return launch_plane_fwd(P->prec, D, fp, nf, spec, S, P->d_plane_fwd, (int64_t)P->plane_fwd.size(),
                                 P->buf_pf, P->smem_pf, P->grid_pf, st);
       }));
    ++launches;
  }
  if (!P->g_rows.empty()) {
    CK(P, timed(P, 0, st, [&] {
         return launch_fwd_x(P->prec, D, fp, nf, spec, S, P->d_g_rows, (int64_t)P->g_rows.size(), P->smem_fx, st);
       }));
    CK(P, timed(P, 1, st, [&] {
         return launch_col(P->prec, -1, 1, D, spec, S, nf, P->d_g_ycols, (int64_t)P->g_ycols.size(), P->smem_y, st);
       }));
    launches += 2;
  }
  for (const auto& g : P->grp_rows) {
    CK(P, timed(P, 0, st, [&] {
         return launch_pen_xf(P->prec, g.code, D, fp, nf, spec, S, P->d_pen_rows + g.start, g.count, P->smem_penx,
                              gather && P->deferred && !P->ggrid.empty() ? P->d_ggrid : nullptr, fields_out(P->form),
                              st);
       }));
    ++launches;
  }
  for (const auto& g : P->grp_ycols) {
    CK(P, timed(P, 1, st, [&] {
         return launch_pen_col(P->prec, -1, g.code, D, spec, S, nf, P->d_pen_ycols + g.start, g.count,
                               P->smem_penc, st);
       }));
    ++launches;
  }
  *launches_out += launches;
  return PSATD_OK;
}

// Field slots each step transforms: with PSATD_J_CONSTANT the current's
// three slots (the last ones) keep the spectrum computed once per push.
static int step_slots(const psatd_plan* P) {
  const int FIN = fields_in(P->form);
  return (P->desc.flags & PSATD_J_CONSTANT) && P->form != kVacuum ? FIN - 3 : FIN;
}

// The whole 3D spectrum of the (constant) current into its workspace slots.
static psatd_status transform_current(psatd_plan* P, const DevPlan& D, const FieldPtrs& fp, cudaStream_t st,
                                      int64_t* launches_out) {
  const int nft = step_slots(P);
  FieldPtrs fj{};
  for (int a = 0; a < 3; ++a) fj.p[a] = fp.p[nft + a];
  void* spec = static_cast<char*>(P->d_ws) + (size_t)nft * P->spec_total * P->csize;
  const psatd_status r = forward_xy(P, D, fj, 3, spec, st, launches_out);
  if (r != PSATD_OK) return r;
  // z: the register z-forward kernel over the step's register z tiles when
  // every box's z pass is a thread-pair register z kernel with 8-column tiles,
  // else the generic column kernel
  const int rt = z_reg_tile_width(P->form, P->reg_z ? P->reg_z : 48);
  const bool zreg = P->prec == 32 && P->zpen.empty() && P->g_zcols.empty() && rt == 8 &&
                    (P->zfast.empty() || (P->reg_z && z_reg_multi_ok(P->reg_z))) &&
                    std::all_of(P->grp_zreg.begin(), P->grp_zreg.end(),
                                [](const auto& g) { return z_reg_multi_ok(g.code) != 0; }) &&
                    (!P->zfast.empty() || !P->zpen_reg.empty());
  if (zreg) {
    for (const auto& g : P->grp_zreg) {
      CK(P, timed(P, 2, st, [&] {
           return launch_z_fwd_pair(D, spec, P->spec_total, P->d_zpen_reg + g.start, g.count, g.code, rt, 3, st);
         }));
      ++*launches_out;
    }
    if (!P->zfast.empty()) {
      CK(P, timed(P, 2, st, [&] {
           return launch_z_fwd_pair(D, spec, P->spec_total, P->d_zfast, (int64_t)P->zfast.size(), P->reg_z, rt, 3,
                                    st);
         }));
      ++*launches_out;
    }
    return PSATD_OK;
  }
  CK(P, timed(P, 2, st, [&] {
       return launch_col(P->prec, -1, 2, D, spec, P->spec_total, 3, P->d_zcols, (int64_t)P->zcols.size(),
                         P->smem_zonly, st);
     }));
  ++*launches_out;
  return PSATD_OK;
}

// S1 (z) + S2 + S3 (z) of one step: every register-z, pencil and generic z
// pass, on the plan's spectrum workspace.
static psatd_status z_step(psatd_plan* P, const DevPlan& D, cudaStream_t st, int64_t* launches_out) {
  const int NFT = step_slots(P);
  const int64_t S = P->spec_total;
  int64_t launches = 0;
  const bool one_launch = P->z_one_launch && P->zreg_multi;
  if (one_launch) {
    // every register-z length in one persistent launch, 2 CTAs per SM
    CK(P, timed(P, 2, st, [&] {
         return launch_z_reg_multi(P->form, D, P->d_ws, S, P->d_zpen_reg, (int64_t)P->zpen_reg.size(),
                                   2 * std::max(1, P->sms), P->z_prefetch > 0, NFT, st);
       }));
    ++launches;
  }
  for (const auto& g : one_launch ? std::vector<psatd_plan::PenGroup>() : P->grp_zreg) {
    CK(P, timed(P, 2, st, [&] {
         return launch_z_reg(P->form, D, P->d_ws, S, P->d_zpen_reg + g.start, g.count, g.code, 0, NFT, P->z_prefetch,
                             st);
       }));
    ++launches;
  }
  for (const auto& g : P->grp_z) {
    CK(P, timed(P, 2, st, [&] {
         return launch_z_pen(P->prec, P->form, g.code, D, P->d_ws, S, P->d_zpen + g.start, g.count, P->smem_penz,
                             NFT, st);
       }));
    ++launches;
  }
  if (!P->zfast.empty() && P->reg_z) {
    CK(P, timed(P, 2, st, [&] {
         return launch_z_reg(P->form, D, P->d_ws, S, P->d_zfast, (int64_t)P->zfast.size(), P->reg_z, P->reg_zst,
                             NFT, P->z_prefetch, st);
       }));
    ++launches;
  } else if (!P->zfast.empty()) {
    CK(P, timed(P, 2, st, [&] {
         return launch_z_fast(P->prec, P->form, D, P->d_ws, S, P->d_zfast, (int64_t)P->zfast.size(), P->smem_zf, NFT,
                              st);
       }));
    ++launches;
  }
  if (!P->g_zcols.empty()) {
    CK(P, timed(P, 2, st, [&] {
         return launch_z_update(P->prec, P->form, D, P->d_ws, S, P->d_g_zcols, (int64_t)P->g_zcols.size(), P->smem_z,
                                NFT, st);
       }));
    ++launches;
  }
  *launches_out += launches;
  return PSATD_OK;
}

// S3 of one step for the output slots [0, nout) of fp, whose spectra start
// at `spec` (slot f at spec + f * spec_total), then the absorbing layers'
// damping and the eager guard exchange (with `guards`).  The kernels use the
// slot index only to offset the field and spectrum pointers, so one slot c
// alone is inverted by passing its field pointer as slot 0 and its spectrum.
static psatd_status inverse_step(psatd_plan* P, const DevPlan& D, const FieldPtrs& fp, int nout, void* spec,
                                 cudaStream_t st, int64_t* launches_out, bool guards) {
  const int64_t S = P->spec_total;
  int64_t launches = 0;
  // S3: inverse y+x, interior cells only
  if (!P->grp_pi.empty()) {
    // one launch per register plane shape; the guard segments are indexed by plane_inv position
    for (const auto& g : P->grp_pi) {
      if (g.code < 0) {
        CK(P, timed(P, 4, st, [&] {
             return launch_plane_inv(P->prec, D, fp, nout, spec, S, P->d_plane_inv + g.start, g.count, P->buf_pi,
                                     P->smem_pi, P->grid_pi, P->segs.empty() ? nullptr : P->d_seg_start + g.start,
                                     P->d_segs, st);
           }));
        ++launches;
        continue;
      }
      CK(P, timed(P, 4, st, [&] {
           return launch_plane_inv_reg(g.code, D, fp, nout, spec, S, P->d_plane_inv + g.start, g.count,
                                       P->segs.empty() || !guards ? nullptr : P->d_seg_start + g.start, P->d_segs,
                                       st);
         }));
      ++launches;
    }
  } else if (!P->plane_inv.empty()) {
    CK(P, timed(P, 4, st, [&] {
         return launch_plane_inv(P->prec, D, fp, nout, spec, S, P->d_plane_inv, (int64_t)P->plane_inv.size(),
                                 P->buf_pi, P->smem_pi, P->grid_pi, P->segs.empty() ? nullptr : P->d_seg_start,
                                 P->d_segs, st);
       }));
    ++launches;
  }
  if (!P->g_rows.empty()) {
    CK(P, timed(P, 3, st, [&] {
         return launch_col(P->prec, 1, 1, D, spec, S, nout, P->d_g_ycols_int, (int64_t)P->g_ycols_int.size(), P->smem_y, st);
       }));
    CK(P, timed(P, 4, st, [&] {
         return launch_inv_x(P->prec, D, fp, nout, spec, S, P->d_g_rows_int, (int64_t)P->g_rows_int.size(), P->smem_ix, 1, st);
       }));
    launches += 2;
  }
  for (const auto& g : P->grp_ycols_int) {
    CK(P, timed(P, 3, st, [&] {
         return launch_pen_col(P->prec, 1, g.code, D, spec, S, nout, P->d_pen_ycols_int + g.start, g.count,
                               P->smem_penc, st);
       }));
    ++launches;
  }
  for (const auto& g : P->grp_rows_int) {
    CK(P, timed(P, 4, st, [&] {
         return launch_pen_xi(P->prec, g.code, D, fp, nout, spec, S, P->d_pen_rows_int + g.start, g.count,
                              P->smem_penxi, st);
       }));
    ++launches;
  }
  if (P->form == kPml && !P->pml_boxes.empty()) {
    // absorbing layers, step (2): damp the split parts, rebuild the components
    FieldPtrs parts{};
    for (int q = 0; q < 6; ++q) parts.p[q] = P->pml_parts[q];
    CK(P, timed(P, 4, st, [&] {
         return launch_pml_damp(P->prec, D, fp, parts, P->d_pml_boxes, (int)P->pml_boxes.size(), P->d_pml_tab,
                                P->pml_tab, st);
       }));
    ++launches;
  }
  if (!P->step_tiles.empty() && guards) {
    const int nex = P->form == kPml ? 6 : nout;   // components only, not the increments
    CK(P, timed(P, 5, st, [&] {
         return launch_exchange(P->prec, D, fp, nex, P->d_blocks, P->d_step_tiles, (int64_t)P->step_tiles.size(),
                                st);
       }));
    ++launches;
  }
  *launches_out += launches;
  return PSATD_OK;
}

// One step S1..S4 of every box on `st`; adds the launches to *launches.
// gather: the forward pass reads guard cells from their owners (deferred
// exchange); guards: the inverse pass stores the guard cells.
static psatd_status push_step(psatd_plan* P, const DevPlan& D, const FieldPtrs& fp, cudaStream_t st,
                              int64_t* launches_out, bool gather = false, bool guards = true) {
  // S1: forward x+y of the slots transformed every step
  psatd_status r = forward_xy(P, D, fp, step_slots(P), P->d_ws, st, launches_out, gather);
  if (r != PSATD_OK) return r;
  r = z_step(P, D, st, launches_out);
  if (r != PSATD_OK) return r;
  // S3: inverse y+x, interior cells only
  return inverse_step(P, D, fp, fields_out(P->form), P->d_ws, st, launches_out, guards);
}

// Capture one step of variant v (2 * gather + guards, see push_step) into a
// CUDA graph for the field set fp (kept until the field pointers change).
// The capture runs on a plan-owned stream (nothing executes during capture),
// so the graph can then be launched on any stream, the legacy default stream
// included.  Returns false, with nothing captured, when the caller's stream
// is itself being captured or capture fails; the push then launches the
// kernels directly.
static bool step_graph(psatd_plan* P, const DevPlan& D, const FieldPtrs& fp, int nf, cudaStream_t st, int v) {
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  if (cudaStreamIsCapturing(st, &cs) != cudaSuccess || cs != cudaStreamCaptureStatusNone) {
    cudaGetLastError();
    return false;
  }
  const bool same = nf == P->graph_nf && std::memcmp(&fp, &P->graph_fp, sizeof(FieldPtrs)) == 0;
  if (same && P->graph_exec[v]) return true;
  if (!same) {
    for (cudaGraphExec_t& g : P->graph_exec)
      if (g) {
        cudaGraphExecDestroy(g);
        g = nullptr;
      }
    P->graph_fp = fp;
    P->graph_nf = nf;
  }
  if (!P->cap_stream && cudaStreamCreateWithFlags(&P->cap_stream, cudaStreamNonBlocking) != cudaSuccess) {
    P->cap_stream = nullptr;
    cudaGetLastError();
    return false;
  }
  if (cudaStreamBeginCapture(P->cap_stream, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  int64_t n = 0;
  const psatd_status r = push_step(P, D, fp, P->cap_stream, &n, (v & 2) != 0, (v & 1) != 0);
  cudaGraph_t g = nullptr;
  const cudaError_t e = cudaStreamEndCapture(P->cap_stream, &g);
  cudaGraphExec_t x = nullptr;
  const bool ok = r == PSATD_OK && e == cudaSuccess && g && cudaGraphInstantiate(&x, g, 0) == cudaSuccess;
  if (g) cudaGraphDestroy(g);
  if (!ok) {
    cudaGetLastError();
    if (x) cudaGraphExecDestroy(x);
    return false;
  }
  P->graph_exec[v] = x;
  P->graph_launches[v] = n;
  return true;
}

psatd_status psatd_push(psatd_plan* P, const psatd_fields* f, const psatd_sources* s, int32_t nsteps,
                        void* stream) {
  if (!P) return PSATD_ERR_INVALID_ARG;
  if (nsteps < 0) return fail(P, PSATD_ERR_INVALID_ARG, "nsteps < 0");
  try {
    FieldPtrs fp{};
    int nf = 0;
    psatd_status r = gather_fields(P, f, s, true, &fp, &nf);
    if (r != PSATD_OK) return r;
    cudaStream_t st = (cudaStream_t)stream;
    P->last_stream = st;
    const DevPlan D = P->dev();
    int64_t launches = 0;
    if (nsteps > 0 && step_slots(P) < fields_in(P->form)) {
      r = transform_current(P, D, fp, st, &launches);
      if (r != PSATD_OK) return r;
    }
    // with the deferred exchange the first step reads the caller's guards,
    // later ones gather them, and the last one stores them
    const bool use_graph = nsteps > 1 && !(P->desc.flags & PSATD_NO_GRAPH) && !P->timing;
    for (int step = 0; step < nsteps; ++step) {
      const bool gather = P->deferred && step > 0;
      const bool guards = !P->deferred || step == nsteps - 1;
      const int v = 2 * gather + guards;
      if (use_graph && step_graph(P, D, fp, nf, st, v)) {
        CK(P, cudaGraphLaunch(P->graph_exec[v], st));
        launches += P->graph_launches[v];
      } else {
        r = push_step(P, D, fp, st, &launches, gather, guards);
        if (r != PSATD_OK) return r;
      }
    }
    P->last_launches = launches;
    return PSATD_OK;
  } catch (...) {
    return fail(P, PSATD_ERR_INVALID_ARG, "internal error");
  }
}

static psatd_status make_copy_stream(psatd_plan* P) {
  if (!P->copy_stream) {
    // highest priority: a copy kernel's blocks take the SM slots that free up
    // before the waiting blocks of the transforms running beside it
    int least = 0, greatest = 0;
    CK(P, cudaDeviceGetStreamPriorityRange(&least, &greatest));
    CK(P, cudaStreamCreateWithPriority(&P->copy_stream, cudaStreamNonBlocking, greatest));
    for (cudaEvent_t& e : P->copy_events) CK(P, cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
  }
  return PSATD_OK;
}

// Whether the six host buffers take the copy kernel (the plan's mode allows
// it, each is page-locked and mapped, both sides 16-byte aligned and bytes %
// 16 == 0); their device addresses in hp, the device buffers in dp.
static bool host_mapped(const psatd_plan* P, void* const host[6], void* const devb[6], size_t bytes, FieldPtrs& hp,
                        FieldPtrs& dp) {
  bool mapped = P->host_copy == 1 && bytes % 16 == 0;
  for (int c = 0; c < 6 && mapped; ++c) {
    void* a = nullptr;
    if (cudaHostGetDevicePointer(&a, host[c], 0) != cudaSuccess || !aligned16(a) || !aligned16(devb[c])) {
      cudaGetLastError();
      mapped = false;
      break;
    }
    hp.p[c] = a;
    dp.p[c] = devb[c];
  }
  return mapped;
}

// The host paths' transfers and push, component by component.  Component c
// is copied between the host buffer src[c] / dst[c] and the device buffer
// stage[c] (nbytes) on a side stream, by the copy kernel through the host
// buffers' device mapping when the plan's mode allows it (host_mapped), else
// by the copy engines; with a coupling, stage[c] is the whole domain,
// scattered into the padded boxes P->host_stage[c] (guards included) and
// gathered back from their interiors, else stage[c] is host_stage[c].
static psatd_status host_pipeline(psatd_plan* P, void* const src[6], void* const dst[6], void* const stage[6],
                                  size_t nbytes, psatd_coupling* coupling, const psatd_sources* s, int nsteps,
                                  cudaStream_t st) {
  psatd_status r = make_copy_stream(P);
  if (r != PSATD_OK) return r;
  FieldPtrs hin{}, hout{}, dev_g{};
  const bool mapped = host_mapped(P, src, stage, nbytes, hin, dev_g) &&
                      host_mapped(P, dst, stage, nbytes, hout, dev_g);
  int sms = 0, gpu = 0;
  CK(P, cudaGetDevice(&gpu));
  CK(P, cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, gpu));
  // Component by component, the host copies on a side stream overlap the
  // scatter into the boxes and the forward x, y transforms of the previous
  // component (and, on the way back, the inverse y, x transforms and the
  // gather of the next one): component c's copy is ordered after the copy
  // of c - 1 on the side stream, the work on c after its copy.  The forward
  // and inverse passes go component by component for the vacuum form
  // without sources (per-kernel timing off); otherwise psatd_push runs
  // between the scatters and the gathers.
  const bool split = P->form == kVacuum && !s && !P->timing && nsteps >= 1;
  const DevPlan D = P->dev();
  FieldPtrs fp{};
  for (int c = 0; c < 6; ++c) fp.p[c] = P->host_stage[c];
  const size_t sbytes = (size_t)P->spec_total * P->csize;   // the spectrum of one slot
  auto slot_fields = [&](int c) {
    FieldPtrs f1{};
    f1.p[0] = P->host_stage[c];
    return f1;
  };
  auto slot_spec = [&](int c) { return static_cast<void*>(static_cast<char*>(P->d_ws) + c * sbytes); };
  cudaStream_t cs = P->copy_stream;
  auto copy_one = [&](int c, bool to_dev) -> cudaError_t {
    if (mapped) {
      FieldPtrs h1{}, d1{};
      h1.p[0] = to_dev ? hin.p[c] : hout.p[c];
      d1.p[0] = stage[c];
      return launch_copy_fields(to_dev ? d1 : h1, to_dev ? h1 : d1, 1, (int64_t)nbytes, 2 * sms, cs);
    }
    return cudaMemcpyAsync(to_dev ? stage[c] : dst[c], to_dev ? src[c] : stage[c], nbytes,
                           to_dev ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToHost, cs);
  };
  int64_t launches = 0;   // kernels of this call: copy kernels, scatters, transforms, gathers
  CK(P, cudaEventRecord(P->copy_events[6], st));
  CK(P, cudaStreamWaitEvent(cs, P->copy_events[6], 0));
  for (int c = 0; c < 6; ++c) {
    // component c to the device (with a coupling, scattered into the padded
    // boxes, guards included), and (split) its forward x, y transforms of the
    // first step
    CK(P, copy_one(c, true));
    CK(P, cudaEventRecord(P->copy_events[c], cs));
    CK(P, cudaStreamWaitEvent(st, P->copy_events[c], 0));
    if (coupling) {
      r = psatd_couple(coupling, PSATD_G1_TO_G2, &stage[c], &P->host_stage[c], 1, st);
      if (r != PSATD_OK) return r;
      launches += P->last_launches;
    }
    launches += mapped ? 1 : 0;
    if (split) {
      r = forward_xy(P, D, slot_fields(c), 1, slot_spec(c), st, &launches, false);
      if (r != PSATD_OK) return r;
    }
  }
  if (split) {
    // the steps as psatd_push runs them (the first step reads the guards
    // the scatter filled; with the deferred exchange later steps gather
    // them and the last one stores them), but for the first step's forward
    // pass, done above, and the last step's inverse pass, done below
    for (int step = 0; step < nsteps; ++step) {
      if (step > 0) {
        r = forward_xy(P, D, fp, 6, P->d_ws, st, &launches, P->deferred);
        if (r != PSATD_OK) return r;
      }
      r = z_step(P, D, st, &launches);
      if (r != PSATD_OK) return r;
      if (step < nsteps - 1) {
        r = inverse_step(P, D, fp, 6, P->d_ws, st, &launches, !P->deferred);
        if (r != PSATD_OK) return r;
      }
    }
    P->last_stream = st;
  } else {
    psatd_fields dev{};
    for (int a = 0; a < 3; ++a) {
      dev.E[a] = P->host_stage[a];
      dev.B[a] = P->host_stage[3 + a];
    }
    r = psatd_push(P, &dev, s, nsteps, st);
    if (r != PSATD_OK) return r;
    launches += P->last_launches;
  }
  for (int c = 0; c < 6; ++c) {
    // (split) the last step's inverse y, x transforms of component c, storing
    // the guard cells; (with a coupling) its box interiors gathered back into
    // the domain; to the host
    if (split) {
      r = inverse_step(P, D, slot_fields(c), 1, slot_spec(c), st, &launches, true);
      if (r != PSATD_OK) return r;
    }
    if (coupling) {
      r = psatd_couple(coupling, PSATD_G2_TO_G1, &stage[c], &P->host_stage[c], 1, st);
      if (r != PSATD_OK) return r;
      launches += P->last_launches;
    }
    launches += mapped ? 1 : 0;
    CK(P, cudaEventRecord(P->copy_events[c], st));
    CK(P, cudaStreamWaitEvent(cs, P->copy_events[c], 0));
    CK(P, copy_one(c, false));
  }
  CK(P, cudaEventRecord(P->copy_events[6], cs));
  CK(P, cudaStreamWaitEvent(st, P->copy_events[6], 0));
  P->last_launches = launches;
  P->last_stream = st;
  return PSATD_OK;
}

psatd_status psatd_push_host(psatd_plan* P, const psatd_fields* in, const psatd_fields* out,
                             const psatd_sources* s, int32_t nsteps, void* stream) {
  if (!P) return PSATD_ERR_INVALID_ARG;
  if (!in || !out) return fail(P, PSATD_ERR_INVALID_ARG, "host field sets must not be NULL");
  for (int a = 0; a < 3; ++a)
    if (!in->E[a] || !in->B[a] || !out->E[a] || !out->B[a])
      return fail(P, PSATD_ERR_INVALID_ARG, "a host field pointer is NULL");
  if (nsteps < 0) return fail(P, PSATD_ERR_INVALID_ARG, "nsteps < 0");
  try {
    cudaStream_t st = (cudaStream_t)stream;
    const size_t bytes = (size_t)P->field_total * P->rsize;
    if (!P->host_stage[0])
      for (int c = 0; c < 6; ++c) CK(P, dalloc(P, bytes, &P->host_stage[c]));
    void* src[6] = {in->E[0], in->E[1], in->E[2], in->B[0], in->B[1], in->B[2]};
    void* dst[6] = {out->E[0], out->E[1], out->E[2], out->B[0], out->B[1], out->B[2]};
    return host_pipeline(P, src, dst, P->host_stage, bytes, nullptr, s, nsteps, st);
  } catch (...) {
    return fail(P, PSATD_ERR_INVALID_ARG, "internal error");
  }
}

psatd_status psatd_push_host_global(psatd_plan* P, const psatd_fields* in, const psatd_fields* out,
                                    const psatd_sources* s, int32_t nsteps, void* stream) {
  if (!P) return PSATD_ERR_INVALID_ARG;
  if (P->desc.decomp == PSATD_DECOMP_INDEPENDENT)
    return fail(P, PSATD_ERR_STATE, "independent boxes have no global domain");
  if (!in || !out) return fail(P, PSATD_ERR_INVALID_ARG, "host field sets must not be NULL");
  for (int a = 0; a < 3; ++a)
    if (!in->E[a] || !in->B[a] || !out->E[a] || !out->B[a])
      return fail(P, PSATD_ERR_INVALID_ARG, "a host field pointer is NULL");
  if (nsteps < 0) return fail(P, PSATD_ERR_INVALID_ARG, "nsteps < 0");
  try {
    cudaStream_t st = (cudaStream_t)stream;
    const psatd_plan_desc& d = P->desc;
    const size_t gcells = (size_t)d.global_n[0] * d.global_n[1] * d.global_n[2];
    const size_t gbytes = gcells * P->rsize, bytes = (size_t)P->field_total * P->rsize;
    if (!P->global_coupling) {
      psatd_box g{};
      for (int a = 0; a < 3; ++a) g.n[a] = d.global_n[a];
      g.order_p = P->boxes[0].order_p;
      psatd_coupling* c = nullptr;
      const psatd_status r = psatd_coupling_create(P, 1, &g, &c);
      if (r != PSATD_OK) return r;
      P->global_coupling = c;
      for (int q = 0; q < 6; ++q) CK(P, dalloc(P, (gbytes + 255) / 256 * 256, &P->global_stage[q]));
    }
    if (!P->host_stage[0])
      for (int c = 0; c < 6; ++c) CK(P, dalloc(P, bytes, &P->host_stage[c]));
    void* src[6] = {in->E[0], in->E[1], in->E[2], in->B[0], in->B[1], in->B[2]};
    void* dst[6] = {out->E[0], out->E[1], out->E[2], out->B[0], out->B[1], out->B[2]};
    return host_pipeline(P, src, dst, P->global_stage, gbytes, P->global_coupling, s, nsteps, st);
  } catch (...) {
    return fail(P, PSATD_ERR_INVALID_ARG, "internal error");
  }
}

psatd_status psatd_forward_fft(psatd_plan* P, const void* field, void* spectrum, void* stream) {
  if (!P) return PSATD_ERR_INVALID_ARG;
  if (!field || !spectrum || !aligned16(field) || !aligned16(spectrum))
    return fail(P, PSATD_ERR_INVALID_ARG, "field/spectrum NULL or not 16-byte aligned");
  FieldPtrs fp{};
  fp.p[0] = const_cast<void*>(field);
  cudaStream_t st = (cudaStream_t)stream;
  P->last_stream = st;
  const DevPlan D = P->dev();
  const int64_t S = P->spec_total;
  CK(P, launch_fwd_x(P->prec, D, fp, 1, spectrum, S, P->d_rows_all, (int64_t)P->rows_all.size(), P->smem_fx, st));
  CK(P, launch_col(P->prec, -1, 1, D, spectrum, S, 1, P->d_ycols_all, (int64_t)P->ycols_all.size(), P->smem_y, st));
  CK(P, launch_col(P->prec, -1, 2, D, spectrum, S, 1, P->d_zcols, (int64_t)P->zcols.size(), P->smem_zonly, st));
  P->last_launches = 3;
  return PSATD_OK;
}

psatd_status psatd_inverse_fft(psatd_plan* P, void* spectrum, void* field, void* stream) {
  if (!P) return PSATD_ERR_INVALID_ARG;
  if (!field || !spectrum || !aligned16(field) || !aligned16(spectrum))
    return fail(P, PSATD_ERR_INVALID_ARG, "field/spectrum NULL or not 16-byte aligned");
  FieldPtrs fp{};
  fp.p[0] = field;
  cudaStream_t st = (cudaStream_t)stream;
  P->last_stream = st;
  const DevPlan D = P->dev();
  const int64_t S = P->spec_total;
  CK(P, launch_col(P->prec, 1, 2, D, spectrum, S, 1, P->d_zcols, (int64_t)P->zcols.size(), P->smem_zonly, st));
  CK(P, launch_col(P->prec, 1, 1, D, spectrum, S, 1, P->d_ycols_all, (int64_t)P->ycols_all.size(), P->smem_y, st));
  CK(P, launch_inv_x(P->prec, D, fp, 1, spectrum, S, P->d_rows_all, (int64_t)P->rows_all.size(), P->smem_ix, 0, st));
  P->last_launches = 3;
  return PSATD_OK;
}

// ---------------------------------------------------------------------------
// One group spread over ranks (paper Sec. 2.4.1 distributed FFT, Sec. 2.6
// spectrum kept in the transposed layout): the rank's device work on its z
// slab and its spectrum rows; the caller moves the spectrum between them.
// ---------------------------------------------------------------------------
namespace {
// [0, n) split into `parts` ranges, sizes differing by at most one, the
// larger ones first: range `i`
void even_range(int n, int parts, int i, int* lo, int* hi) {
  const int q = n / parts, r = n % parts;
  *lo = i * q + std::min(i, r);
  *hi = *lo + q + (i < r ? 1 : 0);
}
}  // namespace

psatd_status psatd_plan_distribute(psatd_plan* P, int32_t world, int32_t rank) {
  if (!P) return PSATD_ERR_INVALID_ARG;
  try {
    if (P->dist.world) return fail(P, PSATD_ERR_STATE, "the plan is already distributed");
    if (P->boxes.size() != 1) return fail(P, PSATD_ERR_INVALID_ARG, "a distributed group is a plan of one box");
    if (P->form == kPml) return fail(P, PSATD_ERR_INVALID_ARG, "absorbing layers are not distributed");
    const psatd_box& b = P->boxes[0];
    if (b.ng_lo[1] || b.ng_hi[1] || b.ng_lo[2] || b.ng_hi[2])
      return fail(P, PSATD_ERR_INVALID_ARG, "a distributed group has guards on its x faces only");
    const int n0 = b.n[0], n1 = b.n[1], n2 = b.n[2], L = n0 / 2, hx = L + 1;
    if (world < 1 || rank < 0 || rank >= world || world > n1 || world > n2)
      return fail(P, PSATD_ERR_INVALID_ARG,
                  fmt("rank %d of %d: need 0 <= rank < world <= min(n1, n2) = %d", rank, world, std::min(n1, n2)));
    auto& d = P->dist;
    even_range(n2, world, rank, &d.z0, &d.z1);
    even_range(n1, world, rank, &d.y0, &d.y1);
    const int nz = d.z1 - d.z0, ny = d.y1 - d.y0;
    d.s_slab = (int64_t)nz * n1 * hx;
    d.s_rows = (int64_t)n2 * ny * hx;
    std::vector<BoxDev> hb = P->hboxes;
    BoxDev slab = hb[0], rows = hb[0];
    slab.ng_lo[1] = slab.ng_lo[2] = slab.ng_hi[1] = slab.ng_hi[2] = 0;
    slab.foff = slab.soff = 0;
    slab.yoff = 0;
    rows = slab;
    rows.n[1] = ny;
    rows.yoff = d.y0;
    const int ib = (int)hb.size();
    hb.push_back(slab);
    hb.push_back(rows);
    // the tile sizes of the plan's generic kernels (its shared-memory limits hold)
    const int csz = (int)P->csize;
    std::vector<RowJob> rj;
    const int nr = std::max(1, std::min(nz * n1, kMaxPoints / L));
    for (int r = 0; r < nz * n1; r += nr) rj.push_back({ib, r, std::min(nr, nz * n1 - r), 0});
    std::vector<ColJob> yc, zc;
    int tyc = std::max(1, kMaxPoints / n1);
    if (tyc >= 8) tyc = tyc / 8 * 8;
    tyc = std::min(tyc, hx);
    for (int z = 0; z < nz; ++z)
      for (int m = 0; m < hx; m += tyc) yc.push_back({ib, z, m, std::min(tyc, hx - m)});
    int tzc = std::max(1, 100 * 1024 / (n2 * spec_slots(P->form) * csz));
    if (tzc >= 4) tzc = tzc / 4 * 4;
    tzc = std::min(tzc, hx);
    for (int y = 0; y < ny; ++y)
      for (int m = 0; m < hx; m += tzc) zc.push_back({ib + 1, y, m, std::min(tzc, hx - m)});
    if (nr * L * csz > P->smem_fx || nr * (hx + L) * csz > P->smem_ix || n1 * tyc * csz > P->smem_y ||
        n2 * spec_slots(P->form) * tzc * csz > P->smem_z)
      return fail(P, PSATD_ERR_UNSUPPORTED_SIZE, "slab tiles exceed the plan's shared memory");
    CK(P, upload(P, hb, &d.d_boxes));
    CK(P, upload(P, rj, &d.d_rows));
    CK(P, upload(P, yc, &d.d_ycols));
    CK(P, upload(P, zc, &d.d_zcols));
    d.nrows = (int64_t)rj.size();
    d.nycols = (int64_t)yc.size();
    d.nzcols = (int64_t)zc.size();
    d.world = world;
    d.rank = rank;
    return PSATD_OK;
  } catch (...) {
    return fail(P, PSATD_ERR_OUT_OF_MEMORY, "host allocation failed");
  }
}

psatd_status psatd_dist_bounds(const psatd_plan* P, int32_t* z0, int32_t* z1, int32_t* y0, int32_t* y1) {
  if (!P || !P->dist.world) return PSATD_ERR_INVALID_ARG;
  if (z0) *z0 = P->dist.z0;
  if (z1) *z1 = P->dist.z1;
  if (y0) *y0 = P->dist.y0;
  if (y1) *y1 = P->dist.y1;
  return PSATD_OK;
}

psatd_status psatd_dist_forward_xy(psatd_plan* P, const psatd_fields* slab, const psatd_sources* src,
                                   void* slab_spectrum, void* stream) {
  if (!P) return PSATD_ERR_INVALID_ARG;
  if (!P->dist.world) return fail(P, PSATD_ERR_STATE, "psatd_plan_distribute first");
  if (!slab_spectrum || !aligned16(slab_spectrum))
    return fail(P, PSATD_ERR_INVALID_ARG, "slab spectrum NULL or not 16-byte aligned");
  FieldPtrs fp{};
  int nf = 0;
  psatd_status r = gather_fields(P, slab, src, true, &fp, &nf);
  if (r != PSATD_OK) return r;
  cudaStream_t st = (cudaStream_t)stream;
  P->last_stream = st;
  DevPlan D = P->dev();
  D.boxes = P->dist.d_boxes;
  const auto& d = P->dist;
  CK(P, launch_fwd_x(P->prec, D, fp, nf, slab_spectrum, d.s_slab, d.d_rows, d.nrows, P->smem_fx, st));
  CK(P, launch_col(P->prec, -1, 1, D, slab_spectrum, d.s_slab, nf, d.d_ycols, d.nycols, P->smem_y, st));
  P->last_launches = 2;
  return PSATD_OK;
}

psatd_status psatd_dist_z_update(psatd_plan* P, void* rows, void* stream) {
  if (!P) return PSATD_ERR_INVALID_ARG;
  if (!P->dist.world) return fail(P, PSATD_ERR_STATE, "psatd_plan_distribute first");
  if (!rows || !aligned16(rows)) return fail(P, PSATD_ERR_INVALID_ARG, "rows NULL or not 16-byte aligned");
  cudaStream_t st = (cudaStream_t)stream;
  P->last_stream = st;
  DevPlan D = P->dev();
  D.boxes = P->dist.d_boxes;
  const auto& d = P->dist;
  CK(P, launch_z_update(P->prec, P->form, D, rows, d.s_rows, d.d_zcols, d.nzcols, P->smem_z, fields_in(P->form),
                        st));
  P->last_launches = 1;
  return PSATD_OK;
}

psatd_status psatd_dist_inverse_yx(psatd_plan* P, void* slab_spectrum, const psatd_fields* slab,
                                   const psatd_sources* src, void* stream) {
  if (!P) return PSATD_ERR_INVALID_ARG;
  if (!P->dist.world) return fail(P, PSATD_ERR_STATE, "psatd_plan_distribute first");
  if (!slab_spectrum || !aligned16(slab_spectrum))
    return fail(P, PSATD_ERR_INVALID_ARG, "slab spectrum NULL or not 16-byte aligned");
  FieldPtrs fp{};
  int nf = 0;
  psatd_status r = gather_fields(P, slab, src, true, &fp, &nf);
  if (r != PSATD_OK) return r;
  const int FOUT = fields_out(P->form);
  cudaStream_t st = (cudaStream_t)stream;
  P->last_stream = st;
  DevPlan D = P->dev();
  D.boxes = P->dist.d_boxes;
  const auto& d = P->dist;
  CK(P, launch_col(P->prec, 1, 1, D, slab_spectrum, d.s_slab, FOUT, d.d_ycols, d.nycols, P->smem_y, st));
  CK(P, launch_inv_x(P->prec, D, fp, FOUT, slab_spectrum, d.s_slab, d.d_rows, d.nrows, P->smem_ix, 1, st));
  P->last_launches = 2;
  return PSATD_OK;
}

psatd_status psatd_sync_status(psatd_plan* P) {
  if (!P) return PSATD_ERR_INVALID_ARG;
  cudaError_t e = cudaStreamSynchronize(P->last_stream);
  if (e == cudaSuccess) e = cudaGetLastError();
  if (e != cudaSuccess) return fail(P, PSATD_ERR_CUDA, fmt("device error: %s", cudaGetErrorString(e)));
  return PSATD_OK;
}

const char* psatd_status_string(psatd_status s) {
  switch (s) {
    case PSATD_OK: return "ok";
    case PSATD_ERR_INVALID_ARG: return "invalid argument";
    case PSATD_ERR_UNSUPPORTED_SIZE: return "unsupported box size";
    case PSATD_ERR_UNSUPPORTED_ORDER: return "unsupported stencil order";
    case PSATD_ERR_OUT_OF_MEMORY: return "out of device memory";
    case PSATD_ERR_CUDA: return "CUDA error";
    case PSATD_ERR_TIMEOUT: return "device-side wait timed out";
    case PSATD_ERR_STATE: return "invalid plan state";
  }
  return "unknown status";
}

const char* psatd_last_error(const psatd_plan* p) {
  return p ? p->last_error.c_str() : g_thread_error.c_str();
}

psatd_status psatd_plan_pml_part(const psatd_plan* p, int32_t q, void** part) {
  if (!p || !part || q < 0 || q >= 6) return PSATD_ERR_INVALID_ARG;
  if (p->form != kPml) return PSATD_ERR_STATE;
  *part = p->pml_parts[q];
  return PSATD_OK;
}

int64_t psatd_last_launch_count(const psatd_plan* p) { return p ? p->last_launches : 0; }

int32_t psatd_plan_fast_boxes(const psatd_plan* p) { return p ? p->fast_boxes : -1; }

int32_t psatd_plan_pencil_boxes(const psatd_plan* p) { return p ? p->pen_boxes : -1; }

int32_t psatd_plan_deferred_exchange(const psatd_plan* p) { return p ? (p->deferred ? 1 : 0) : -1; }

psatd_status psatd_plan_tune(psatd_plan* P, int32_t knob, int32_t value) {
  if (!P) return PSATD_ERR_INVALID_ARG;
  switch (knob) {
    case PSATD_TUNE_Z_PREFETCH:
      if (value < 0 || value > (1 << 20)) return fail(P, PSATD_ERR_INVALID_ARG, "prefetch distance out of range");
      P->z_prefetch = value;
      break;
    case PSATD_TUNE_HOST_COPY:
      if (value != 0 && value != 1) return fail(P, PSATD_ERR_INVALID_ARG, "host copy mode is 0 or 1");
      P->host_copy = value;
      return PSATD_OK;   // not part of any captured graph
    case PSATD_TUNE_Z_ONE_LAUNCH:
      if (value != 0 && value != 1) return fail(P, PSATD_ERR_INVALID_ARG, "one-launch z pass is 0 or 1");
      P->z_one_launch = value;
      break;
    case PSATD_TUNE_PENCIL_ROWS_KB:
    case PSATD_TUNE_Z_TILE:
    case PSATD_TUNE_PENCIL_REG_Z:
    case PSATD_TUNE_REG_PLANES:
      return fail(P, PSATD_ERR_INVALID_ARG, "this knob is set at plan creation only");
    default:
      return fail(P, PSATD_ERR_INVALID_ARG, "unknown tuning knob");
  }
  // captured graphs hold the old launch parameters
  for (cudaGraphExec_t& g : P->graph_exec)
    if (g) {
      cudaGraphExecDestroy(g);
      g = nullptr;
    }
  return PSATD_OK;
}

int32_t psatd_plan_tuning(const psatd_plan* P, int32_t knob) {
  if (!P) return -1;
  switch (knob) {
    case PSATD_TUNE_Z_PREFETCH:
      return P->reg_z || !P->zpen_reg.empty() ? P->z_prefetch : -1;
    case PSATD_TUNE_PENCIL_ROWS_KB:
      return P->pen_boxes ? P->pen_rows_kb : -1;
    case PSATD_TUNE_HOST_COPY:
      return P->host_copy;
    case PSATD_TUNE_PENCIL_REG_Z:
      return P->pen_reg_z_used ? P->pen_reg_z : -1;
    case PSATD_TUNE_REG_PLANES:
      return P->reg_planes_used ? P->reg_planes : -1;
    case PSATD_TUNE_Z_ONE_LAUNCH:
      return P->zreg_multi ? P->z_one_launch : -1;
    case PSATD_TUNE_Z_TILE:
      return (P->pen_boxes || (P->fast_boxes && !P->reg_z))
                 ? (P->z_tile > 0 ? std::min(P->z_tile, fast_tile(P->prec)) : fast_tile(P->prec))
                 : -1;
    default:
      return -1;
  }
}

psatd_status psatd_plan_set_timing(psatd_plan* P, int32_t enable) {
  if (!P) return PSATD_ERR_INVALID_ARG;
  P->timing = enable != 0;
  return PSATD_OK;
}

psatd_status psatd_plan_kernel_times(psatd_plan* P, double* ms, int64_t* launches, int32_t n) {
  if (!P || n < 0) return PSATD_ERR_INVALID_ARG;
  cudaError_t e = cudaStreamSynchronize(P->last_stream);
  if (e != cudaSuccess) return fail(P, PSATD_ERR_CUDA, fmt("device error: %s", cudaGetErrorString(e)));
  for (auto& r : P->recs) {
    float t = 0.f;
    if (r.kind < n) {
      e = cudaEventElapsedTime(&t, r.a, r.b);
      if (e != cudaSuccess) return fail(P, PSATD_ERR_CUDA, fmt("event timing: %s", cudaGetErrorString(e)));
      if (ms) ms[r.kind] += t;
      if (launches) launches[r.kind] += 1;
    }
    P->ev_pool.push_back(r.a);
    P->ev_pool.push_back(r.b);
  }
  P->recs.clear();
  return PSATD_OK;
}

psatd_status psatd_coupling_blocks(const psatd_plan_desc* g2, int32_t num_g1_boxes, const psatd_box* g1_boxes,
                                   int32_t direction, psatd_copy_block* out, int64_t cap, int64_t* count) {
  try {
    if (!count || cap < 0 || (cap > 0 && !out) || (direction != PSATD_G1_TO_G2 && direction != PSATD_G2_TO_G1))
      return fail(nullptr, PSATD_ERR_INVALID_ARG, "bad arguments");
    Err e = validate(g2);
    if (e.st == PSATD_OK) e = validate_g1(*g2, num_g1_boxes, g1_boxes);
    if (e.st != PSATD_OK) return fail(nullptr, e.st, e.msg);
    const std::vector<psatd_box> a(g2->boxes, g2->boxes + g2->num_boxes), b(g1_boxes, g1_boxes + num_g1_boxes);
    int64_t N[3];
    bool per[3];
    domain_of(*g2, N, per);
    const std::vector<CopyBlk> blocks =
        direction == PSATD_G1_TO_G2 ? coupling_blocks(a, b, N, per) : coupling_blocks(b, a, N, per);
    *count = (int64_t)blocks.size();
    for (int64_t i = 0; i < std::min<int64_t>(cap, (int64_t)blocks.size()); ++i) {
      out[i].dst_box = blocks[i].dst_box;
      out[i].src_box = blocks[i].src_box;
      for (int k = 0; k < 3; ++k) {
        out[i].dst_lo[k] = blocks[i].dst_lo[k];
        out[i].src_lo[k] = blocks[i].src_lo[k];
        out[i].ext[k] = blocks[i].ext[k];
      }
    }
    return PSATD_OK;
  } catch (...) {
    return fail(nullptr, PSATD_ERR_INVALID_ARG, "internal error");
  }
}

psatd_status psatd_coupling_create(psatd_plan* plan, int32_t num_g1_boxes, const psatd_box* g1_boxes,
                                   psatd_coupling** out) {
  if (!out) return fail(nullptr, PSATD_ERR_INVALID_ARG, "out is NULL");
  *out = nullptr;
  if (!plan) return fail(nullptr, PSATD_ERR_INVALID_ARG, "plan is NULL");
  try {
    Err e = validate_g1(plan->desc, num_g1_boxes, g1_boxes);
    if (e.st != PSATD_OK) return fail(plan, e.st, e.msg);
    auto* C = new psatd_coupling();
    C->plan = plan;
    C->g1.assign(g1_boxes, g1_boxes + num_g1_boxes);
    int64_t foff = 0;
    for (const psatd_box& b : C->g1) {
      BoxDev x{};
      for (int a = 0; a < 3; ++a) {
        x.n[a] = b.n[a];
        x.ng_lo[a] = b.ng_lo[a];
        x.ng_hi[a] = b.ng_hi[a];
      }
      x.foff = foff;
      foff += align_up((int64_t)b.n[0] * b.n[1] * b.n[2], 64);
      C->hg1.push_back(x);
    }
    C->field_total = foff;
    int64_t N[3];
    bool per[3];
    domain_of(plan->desc, N, per);
    const int v16 = 16 / (int)plan->rsize;
    C->blk[PSATD_G1_TO_G2] = coupling_blocks(plan->boxes, C->g1, N, per);
    C->blk[PSATD_G2_TO_G1] = coupling_blocks(C->g1, plan->boxes, N, per);
    C->tiles[PSATD_G1_TO_G2] = block_tiles(C->blk[PSATD_G1_TO_G2], plan->boxes, C->g1, v16);
    C->tiles[PSATD_G2_TO_G1] = block_tiles(C->blk[PSATD_G2_TO_G1], C->g1, plan->boxes, v16);
    cudaError_t ce = C->up(C->hg1, &C->d_g1);
    for (int d = 0; d < 2 && ce == cudaSuccess; ++d) {
      ce = C->up(C->blk[d], &C->d_blk[d]);
      if (ce == cudaSuccess) ce = C->up(C->tiles[d], &C->d_tiles[d]);
    }
    if (ce != cudaSuccess) {
      delete C;
      return fail(plan, ce == cudaErrorMemoryAllocation ? PSATD_ERR_OUT_OF_MEMORY : PSATD_ERR_CUDA,
                  fmt("coupling: %s", cudaGetErrorString(ce)));
    }
    *out = C;
    return PSATD_OK;
  } catch (...) {
    return fail(plan, PSATD_ERR_INVALID_ARG, "internal error");
  }
}

psatd_status psatd_coupling_destroy(psatd_coupling* c) {
  delete c;
  return PSATD_OK;
}

psatd_status psatd_coupling_layout(const psatd_coupling* c, int32_t box, int64_t* off, int64_t* elems) {
  if (!c || !off || !elems || box < 0 || box >= (int32_t)c->g1.size()) return PSATD_ERR_INVALID_ARG;
  const psatd_box& b = c->g1[box];
  *off = c->hg1[box].foff;
  *elems = (int64_t)b.n[0] * b.n[1] * b.n[2];
  return PSATD_OK;
}

psatd_status psatd_couple(psatd_coupling* c, int32_t direction, void* const* g1_fields, void* const* g2_fields,
                          int32_t nfields, void* stream) {
  if (!c) return PSATD_ERR_INVALID_ARG;
  psatd_plan* P = c->plan;
  if ((direction != PSATD_G1_TO_G2 && direction != PSATD_G2_TO_G1) || nfields < 1 || nfields > 10 || !g1_fields ||
      !g2_fields)
    return fail(P, PSATD_ERR_INVALID_ARG, "bad direction, field count or field arrays");
  FieldPtrs f1{}, f2{};
  for (int i = 0; i < nfields; ++i) {
    f1.p[i] = g1_fields[i];
    f2.p[i] = g2_fields[i];
    if (!f1.p[i] || !f2.p[i] || !aligned16(f1.p[i]) || !aligned16(f2.p[i]))
      return fail(P, PSATD_ERR_INVALID_ARG, fmt("field %d NULL or not 16-byte aligned", i));
  }
  cudaStream_t st = (cudaStream_t)stream;
  P->last_stream = st;
  const bool to_fft = direction == PSATD_G1_TO_G2;
  CK(P, launch_copy_blocks(P->prec, to_fft ? P->d_boxes : c->d_g1, to_fft ? c->d_g1 : P->d_boxes,
                           to_fft ? f2 : f1, to_fft ? f1 : f2, nfields, c->d_blk[direction], c->d_tiles[direction],
                           (int64_t)c->tiles[direction].size(), st));
  P->last_launches = c->tiles[direction].empty() ? 0 : 1;
  return PSATD_OK;
}

}  // extern "C"
