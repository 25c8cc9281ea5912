// psatd_push_box_static: the PSATD push of one periodic FP32 box without any
// device allocation.
//
// Who needs it: callers that are not allowed to allocate device memory
// themselves or through a library, for example code that runs inside a host
// framework that owns every device allocation (and forbids cudaMalloc behind
// its back), fixed-memory real-time loops, or plug-ins that may only touch the
// buffers they are handed.  psatd_plan_create allocates its workspace and
// tables with cudaMalloc, so those callers cannot use it; this entry point
// takes the caller's field buffers and keeps everything else (spectral
// workspace, FFT and PSATD tables, work lists) in one file-scope __device__
// array that the CUDA driver reserves when the library's module is loaded.
//
// The array is kStaticScratchBytes = PSATD_STATIC_SCRATCH_BYTES (64 MiB) and
// stays reserved on every GPU that loads this library until the process
// exits.  All calls on one device share it: a call rewrites every byte it
// later reads (work lists, tables, then the spectra), so nothing needs to be
// cleared between calls, but two calls that overlap on the GPU (different
// streams, or different host threads without ordering) race on the array and
// corrupt each other's results.
//
// The first call on a device looks up the array's device address with
// cudaGetSymbolAddress, reads the device's opt-in shared-memory maximum and
// raises the kernels' shared-memory limit to it; make that first call before
// any stream capture.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <vector>

#include "psatd_internal.h"

namespace psatd {
namespace {

constexpr size_t kStaticScratchBytes = PSATD_STATIC_SCRATCH_BYTES;

// The scratch arena.  Host code must never pass this name to a kernel: on the
// host it denotes a shadow object, not device memory.  Its device address is
// obtained once per device with cudaGetSymbolAddress.
static __device__ __align__(256) unsigned char g_static_scratch[kStaticScratchBytes];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
unsigned char* g_arena[kMaxDevices] = {};
bool g_configured[kMaxDevices] = {};
int g_optin[kMaxDevices] = {};

size_t up(size_t v, size_t a) { return (v + a - 1) / a * a; }

psatd_status err(psatd_status s, const char* fmt, ...) {
  char buf[256];
  va_list ap;
  va_start(ap, fmt);
  std::vsnprintf(buf, sizeof buf, fmt, ap);
  va_end(ap);
  set_thread_error(buf);
  return s;
}

bool smooth_even(int n, int lo, int hi) {
  if (n < lo || n > hi || n % 2) return false;
  for (int f : {2, 3, 5})
    while (n % f == 0) n /= f;
  return n == 1;
}

}  // namespace
}  // namespace psatd

using namespace psatd;

extern "C" psatd_status psatd_push_box_static(const int32_t n[3], int32_t order_p, const double dx[3],
                                              double dt, double c, const psatd_fields* fields,
                                              int32_t nsteps, void* stream) {
  // ---- arguments (nothing touches the GPU before they are all checked)
  if (!n || !dx || !fields) return err(PSATD_ERR_INVALID_ARG, "NULL argument");
  if (nsteps < 0) return err(PSATD_ERR_INVALID_ARG, "nsteps < 0");
  for (int a = 0; a < 3; ++a) {
    if (!smooth_even(n[a], 4, a == 0 ? 1024 : 512))
      return err(PSATD_ERR_UNSUPPORTED_SIZE, "n[%d] = %d must be even, 5-smooth, in [4, %d]", a, n[a],
                 a == 0 ? 1024 : 512);
    if (!(dx[a] > 0.0)) return err(PSATD_ERR_INVALID_ARG, "dx must be > 0");
  }
  if (!(order_p == 0 || (order_p >= 2 && order_p <= 256 && order_p % 2 == 0)))
    return err(PSATD_ERR_UNSUPPORTED_ORDER, "order %d is not 0 or even in [2, 256]", order_p);
  if (!(dt != 0.0) || !(c > 0.0)) return err(PSATD_ERR_INVALID_ARG, "dt must be nonzero and c > 0");
  FieldPtrs fp{};
  for (int a = 0; a < 3; ++a) {
    fp.p[a] = fields->E[a];
    fp.p[3 + a] = fields->B[a];
  }
  for (int i = 0; i < 6; ++i)
    if (!fp.p[i] || ((uintptr_t)fp.p[i] & 15u))
      return err(PSATD_ERR_INVALID_ARG, "field %d is NULL or not 16-byte aligned", i);

  // ---- host description of the one box (same tables and work lists as a plan)
  const int n0 = n[0], n1 = n[1], n2 = n[2];
  const int L = n0 / 2, hx = L + 1, FIN = fields_in(kVacuum);
  ShapeDev s{};
  s.fx = s.fy = s.fz = s.px = s.py = s.pz = -1;   // generic kernels only
  for (int a = 0; a < 3; ++a) s.n[a] = n[a];
  s.L = L;
  s.hx = hx;
  s.p = order_p;
  if (!radix_plan(L, s.ax) || !radix_plan(n1, s.ay) || !radix_plan(n2, s.az))
    return err(PSATD_ERR_UNSUPPORTED_SIZE, "no radix schedule");
  int64_t ctot = 0, rtot = 0;
  auto ctake = [&](int64_t k) {
    const int64_t o = ctot;
    ctot += (k + 1) / 2 * 2;
    return o;
  };
  auto rtake = [&](int64_t k) {
    const int64_t o = rtot;
    rtot += (k + 3) / 4 * 4;
    return o;
  };
  s.ax.tw = ctake(L);
  s.ay.tw = ctake(n1);
  s.az.tw = ctake(n2);
  s.post = ctake(hx);
  s.phx = ctake(hx);
  s.phy = ctake(n1);
  s.phz = ctake(n2);
  s.kx = rtake(hx);
  s.ky = rtake(n1);
  s.kz = rtake(n2);
  s.coef = 0;
  const int64_t qtot = (int64_t)hx * (n1 / 2 + 1) * (n2 / 2 + 1);
  BoxDev b{};
  for (int a = 0; a < 3; ++a) b.n[a] = n[a];
  const int64_t spec = (int64_t)hx * n1 * n2;
  std::vector<RowJob> rows;
  std::vector<ColJob> ycols, zcols;
  const int nr = std::max(1, std::min(n1 * n2, kMaxPoints / L));
  for (int r = 0; r < n1 * n2; r += nr) rows.push_back({0, r, std::min(nr, n1 * n2 - r), 0});
  int ny = std::max(1, kMaxPoints / n1);
  if (ny >= 8) ny = ny / 8 * 8;
  ny = std::min(ny, hx);
  for (int z = 0; z < n2; ++z)
    for (int m = 0; m < hx; m += ny) ycols.push_back({0, z, m, std::min(ny, hx - m)});
  int nz = std::max(1, 100 * 1024 / (n2 * FIN * 8));
  if (nz >= 4) nz = nz / 4 * 4;
  nz = std::min(nz, hx);
  for (int y = 0; y < n1; ++y)
    for (int m = 0; m < hx; m += nz) zcols.push_back({0, y, m, std::min(nz, hx - m)});
  const int smem = std::max({nr * L * 8, n1 * ny * 8, n2 * FIN * nz * 8, nr * (hx + L) * 8});
  const std::vector<double> alpha = order_p ? stencil_alpha(order_p) : std::vector<double>(1, 0.0);

  // ---- carve the arena: [box][shape][rows][ycols][zcols][alpha][r32][c32][q32][r64][c64][q64][spectra]
  size_t off = 0;
  auto carve = [&](size_t bytes) {
    off = up(off, 256);
    const size_t o = off;
    off += bytes;
    return o;
  };
  const size_t o_box = carve(sizeof(BoxDev)), o_shape = carve(sizeof(ShapeDev));
  const size_t o_rows = carve(rows.size() * sizeof(RowJob));
  const size_t o_ycols = carve(ycols.size() * sizeof(ColJob));
  const size_t o_zcols = carve(zcols.size() * sizeof(ColJob));
  const size_t o_alpha = carve(alpha.size() * sizeof(double));
  const size_t o_r32 = carve(rtot * 4), o_c32 = carve(ctot * 8), o_q32 = carve(qtot * 16);
  const size_t o_r64 = carve(rtot * 8), o_c64 = carve(ctot * 16), o_q64 = carve(qtot * 32);
  const size_t o_ws = carve((size_t)FIN * spec * 8);
  if (off > kStaticScratchBytes)
    return err(PSATD_ERR_UNSUPPORTED_SIZE,
               "box %dx%dx%d needs %zu bytes of static scratch; the limit is %zu bytes", n0, n1, n2, off,
               kStaticScratchBytes);

  // ---- per-device set-up: address of the arena, shared-memory opt-in
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return err(PSATD_ERR_CUDA, "cudaGetDevice: %s", cudaGetErrorString(e));
  if (dev < 0 || dev >= kMaxDevices) return err(PSATD_ERR_CUDA, "device %d out of range", dev);
  unsigned char* A = nullptr;
  int optin = 0;
  {
    std::lock_guard<std::mutex> lk(g_mu);
    if (!g_arena[dev]) {
      void* p = nullptr;
      e = cudaGetSymbolAddress(&p, g_static_scratch);
      if (e != cudaSuccess || !p)
        return err(PSATD_ERR_CUDA, "cudaGetSymbolAddress: %s", cudaGetErrorString(e));
      g_arena[dev] = static_cast<unsigned char*>(p);
    }
    if (!g_optin[dev]) {
      // the device's per-block opt-in shared-memory maximum bounds both the
      // size check below and the kernels' dynamic shared-memory attribute
      e = cudaDeviceGetAttribute(&g_optin[dev], cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
      if (e != cudaSuccess || g_optin[dev] <= 0) {
        g_optin[dev] = 0;
        return err(PSATD_ERR_CUDA, "cudaDeviceGetAttribute: %s", cudaGetErrorString(e));
      }
    }
    optin = g_optin[dev];
    if (smem > optin)
      return err(PSATD_ERR_UNSUPPORTED_SIZE, "box needs %d B of shared memory per block; the device allows %d B",
                 smem, optin);
    if (!g_configured[dev]) {
      e = configure_kernels(32, optin);
      if (e != cudaSuccess) return err(PSATD_ERR_CUDA, "cudaFuncSetAttribute: %s", cudaGetErrorString(e));
      g_configured[dev] = true;
    }
    A = g_arena[dev];
  }
  cudaStream_t st = (cudaStream_t)stream;
  // ---- work lists and descriptors (copied from host memory; no allocation)
#define PSATD_CK(x)                                                                   \
  do {                                                                                \
    cudaError_t _e = (x);                                                             \
    if (_e != cudaSuccess) return err(PSATD_ERR_CUDA, "%s: %s", #x, cudaGetErrorString(_e)); \
  } while (0)
  PSATD_CK(cudaMemcpyAsync(A + o_box, &b, sizeof b, cudaMemcpyHostToDevice, st));
  PSATD_CK(cudaMemcpyAsync(A + o_shape, &s, sizeof s, cudaMemcpyHostToDevice, st));
  PSATD_CK(cudaMemcpyAsync(A + o_rows, rows.data(), rows.size() * sizeof(RowJob), cudaMemcpyHostToDevice, st));
  PSATD_CK(cudaMemcpyAsync(A + o_ycols, ycols.data(), ycols.size() * sizeof(ColJob), cudaMemcpyHostToDevice, st));
  PSATD_CK(cudaMemcpyAsync(A + o_zcols, zcols.data(), zcols.size() * sizeof(ColJob), cudaMemcpyHostToDevice, st));
  PSATD_CK(cudaMemcpyAsync(A + o_alpha, alpha.data(), alpha.size() * sizeof(double), cudaMemcpyHostToDevice, st));
  // ---- FP64 tables, rounded once to FP32
  double* r64 = reinterpret_cast<double*>(A + o_r64);
  double2* c64 = reinterpret_cast<double2*>(A + o_c64);
  Coef4<double>* q64 = reinterpret_cast<Coef4<double>*>(A + o_q64);
  const double* al = reinterpret_cast<const double*>(A + o_alpha);
  const int q = order_p / 2;
  PSATD_CK(gen_twiddles(c64 + s.ax.tw, L, st));
  PSATD_CK(gen_twiddles(c64 + s.ay.tw, n1, st));
  PSATD_CK(gen_twiddles(c64 + s.az.tw, n2, st));
  PSATD_CK(gen_post(c64 + s.post, n0, st));
  PSATD_CK(gen_axis(r64 + s.kx, c64 + s.phx, hx, n0, dx[0], q, al, 0, st));
  PSATD_CK(gen_axis(r64 + s.ky, c64 + s.phy, n1, n1, dx[1], q, al, 0, st));
  PSATD_CK(gen_axis(r64 + s.kz, c64 + s.phz, n2, n2, dx[2], q, al, 0, st));
  PSATD_CK(gen_coef(q64, hx, n1, n2, r64 + s.kx, r64 + s.ky, r64 + s.kz, c, dt, st));
  PSATD_CK(convert_pools(r64, reinterpret_cast<float*>(A + o_r32), rtot, c64,
                         reinterpret_cast<float2*>(A + o_c32), ctot, q64,
                         reinterpret_cast<Coef4<float>*>(A + o_q32), qtot, st));
  // ---- the push: S1 forward FFT, S2 update, S3 inverse FFT (no guards)
  DevPlan P;
  P.boxes = reinterpret_cast<const BoxDev*>(A + o_box);
  P.shapes = reinterpret_cast<const ShapeDev*>(A + o_shape);
  P.rpool = A + o_r32;
  P.cpool = A + o_c32;
  P.coef = A + o_q32;
  set_constants(P, c, 1.0, dt);
  void* ws = A + o_ws;
  const RowJob* drows = reinterpret_cast<const RowJob*>(A + o_rows);
  const ColJob* dy = reinterpret_cast<const ColJob*>(A + o_ycols);
  const ColJob* dz = reinterpret_cast<const ColJob*>(A + o_zcols);
  for (int step = 0; step < nsteps; ++step) {
    PSATD_CK(launch_fwd_x(32, P, fp, FIN, ws, spec, drows, (int64_t)rows.size(), nr * L * 8, st));
    PSATD_CK(launch_col(32, -1, 1, P, ws, spec, FIN, dy, (int64_t)ycols.size(), n1 * ny * 8, st));
    PSATD_CK(launch_z_update(32, kVacuum, P, ws, spec, dz, (int64_t)zcols.size(), n2 * FIN * nz * 8, FIN, st));
    PSATD_CK(launch_col(32, 1, 1, P, ws, spec, FIN, dy, (int64_t)ycols.size(), n1 * ny * 8, st));
    PSATD_CK(launch_inv_x(32, P, fp, FIN, ws, spec, drows, (int64_t)rows.size(), nr * (hx + L) * 8, 1, st));
  }
#undef PSATD_CK
  return PSATD_OK;
}
