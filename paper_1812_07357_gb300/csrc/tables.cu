// FP64 generation of the plan's tables on the device (run once per plan):
// FFT twiddles, the R2C split factors, the order-p staggered modified
// wavenumbers K(k) (Sec. 1.1: stencil of width p/2, p -> infinity gives
// K = k), the Yee half-cell phase factors and the per-mode PSATD
// coefficients.  The FP32 path uses these values rounded once to float.
#include <cuda_runtime.h>

#include "psatd_internal.h"

namespace psatd {

// tw[j] = exp(-2 pi i j / n)
__global__ void g_twiddles(double2* out, int n) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= n) return;
  double s, c;
  sincospi(-2.0 * (double)j / (double)n, &s, &c);
  out[j] = make_double2(c, s);
}

// post[k] = exp(-2 pi i k / n0), k = 0 .. n0/2
__global__ void g_post(double2* out, int n0) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k > n0 / 2) return;
  double s, c;
  sincospi(-2.0 * (double)k / (double)n0, &s, &c);
  out[k] = make_double2(c, s);
}

// Index m of an n-point axis has k = 2 pi mt/(n h), mt = m (m <= n/2) else m - n.
// K(k) = sum_l alpha_l 2 sin((2l-1) k h/2)/((2l-1) h)   (q = p/2 terms), or k (q = 0).
// ph = exp(i k h/2).
// nodal = 0: staggered K = sum_l alpha_l 2 sin((2l-1) k h/2) / ((2l-1) h) and the
// half-cell phase exp(i k h/2); nodal = 1: collocated K = sum_l beta_l
// sin(l k h) / (l h) and no phase (weights in `alpha`).
__global__ void g_axis(double* K, double2* ph, int count, int n, double h, int q,
                       const double* __restrict__ alpha, int nodal) {
  const int m = blockIdx.x * blockDim.x + threadIdx.x;
  if (m >= count) return;
  const int mt = (2 * m <= n) ? m : m - n;
  double k;
  if (q == 0) {
    // collocated infinite order: the Nyquist index is its own mirror image,
    // only K = 0 keeps the derivative of a real field real
    k = (nodal && 2 * mt == n) ? 0.0 : 2.0 * M_PI * (double)mt / ((double)n * h);
  } else {
    k = 0.0;
    for (int l = 1; l <= q; ++l) {
      if (nodal) {
        k += alpha[l - 1] * sinpi((double)(2 * l * mt) / (double)n) / ((double)l * h);
      } else {
        const int o = 2 * l - 1;
        k += alpha[l - 1] * 2.0 * sinpi((double)(o * mt) / (double)n) / ((double)o * h);
      }
    }
  }
  K[m] = k;
  if (nodal) {
    ph[m] = make_double2(1.0, 0.0);
  } else {
    double s, c;
    sincospi((double)mt / (double)n, &s, &c);
    ph[m] = make_double2(c, s);
  }
}

// theta = c dt |K|:  C = cos theta,  Sw = dt sin(theta)/theta,
// X1 = (c dt)^2/2 (sin(theta/2)/(theta/2))^2  (= (1 - C)/K^2 without cancellation),
// X3 = c^2 dt^3 (sin(theta)/theta - 1)/theta^2 (Taylor series below theta = 0.1).
__global__ void g_coef(Coef4<double>* out, int hx, int n1, int n2, const double* __restrict__ kx,
                       const double* __restrict__ ky, const double* __restrict__ kz, double c,
                       double dt) {
  const int h1 = n1 / 2 + 1, h2 = n2 / 2 + 1;
  const int64_t total = (int64_t)hx * h1 * h2;
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= total) return;
  const int mx = (int)(i % hx);
  const int my = (int)((i / hx) % h1);
  const int mz = (int)(i / ((int64_t)hx * h1));
  const double k2 = kx[mx] * kx[mx] + ky[my] * ky[my] + kz[mz] * kz[mz];
  const double th = c * dt * sqrt(k2);
  const double cth = cos(th);
  const double sinc = th == 0.0 ? 1.0 : sin(th) / th;
  const double hth = 0.5 * th;
  const double sinch = hth == 0.0 ? 1.0 : sin(hth) / hth;
  double g;
  if (fabs(th) < 0.1) {
    const double t2 = th * th;
    g = -1.0 / 6 + t2 * (1.0 / 120 + t2 * (-1.0 / 5040 + t2 * (1.0 / 362880 + t2 * (-1.0 / 39916800))));
  } else {
    g = (sinc - 1.0) / (th * th);
  }
  Coef4<double> r;
  r.c = cth;
  r.s = dt * sinc;
  r.x1 = 0.5 * (c * dt) * (c * dt) * sinch * sinch;
  r.x3 = c * c * dt * dt * dt * g;
  out[i] = r;
}

__global__ void g_convert(const double* r64, float* r32, int64_t nr, const double2* c64, float2* c32,
                          int64_t nc, const Coef4<double>* q64, Coef4<float>* q32, int64_t nq) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < nr) r32[i] = (float)r64[i];
  if (i < nc) c32[i] = make_float2((float)c64[i].x, (float)c64[i].y);
  if (i < nq) {
    Coef4<float> o;
    o.c = (float)q64[i].c;
    o.s = (float)q64[i].s;
    o.x1 = (float)q64[i].x1;
    o.x3 = (float)q64[i].x3;
    q32[i] = o;
  }
}

static unsigned nblk(int64_t n) { return (unsigned)((n + 255) / 256); }

cudaError_t gen_twiddles(double2* out, int n, cudaStream_t st) {
  g_twiddles<<<nblk(n), 256, 0, st>>>(out, n);
  return cudaGetLastError();
}
cudaError_t gen_post(double2* out, int n0, cudaStream_t st) {
  g_post<<<nblk(n0 / 2 + 1), 256, 0, st>>>(out, n0);
  return cudaGetLastError();
}
cudaError_t gen_axis(double* K, double2* ph, int count, int n, double h, int q,
                     const double* alpha_dev, int nodal, cudaStream_t st) {
  g_axis<<<nblk(count), 256, 0, st>>>(K, ph, count, n, h, q, alpha_dev, nodal);
  return cudaGetLastError();
}
cudaError_t gen_coef(Coef4<double>* out, int hx, int n1, int n2, const double* kx, const double* ky,
                     const double* kz, double c, double dt, cudaStream_t st) {
  const int64_t total = (int64_t)hx * (n1 / 2 + 1) * (n2 / 2 + 1);
  g_coef<<<nblk(total), 256, 0, st>>>(out, hx, n1, n2, kx, ky, kz, c, dt);
  return cudaGetLastError();
}
cudaError_t convert_pools(const double* r64, float* r32, int64_t nr, const double2* c64,
                          float2* c32, int64_t nc, const Coef4<double>* q64, Coef4<float>* q32,
                          int64_t nq, cudaStream_t st) {
  int64_t n = nr > nc ? nr : nc;
  if (nq > n) n = nq;
  if (n == 0) return cudaSuccess;
  g_convert<<<nblk(n), 256, 0, st>>>(r64, r32, nr, c64, c32, nc, q64, q32, nq);
  return cudaGetLastError();
}

}  // namespace psatd
