// Retarded-cumulant spectral function (Sec. "Numerical GW+C scheme").
//
//   beta_j = |Im Sigma_n(eps_n + w_j)| / pi
//   C~(t)  = sum_j q_j beta_j / w_j^2 (e^{-i w_j t} - 1)        (Eq. landau_cumulant_truncated)
//   G^C(t) = G^QP(t) e^{C~(t)}                                   (Eq. cumulant_propagator_numerical_time)
//   A(eps^QP + nu) = (1/pi) Re int_0^T e^{i nu t - eta t} e^{C~(t)} dt    (Eq. eq:AGWC)
//
// The transform of e^{C~(t)} followed by the convolution with G^QP (Eqs.
// cumulant_propagator_fourier, cumulant_propagator_convolution) is done as ONE damped
// transform (convolution theorem): g_k = w_k e^{C~(t_k) - eta t_k}, t_k = k dt, w_0 = 1/2,
// X_j = dt sum_k g_k e^{2 pi i jk/n}, A_j = Re X_j / pi on nu_j = 2 pi j/(n dt).
// The sum over k is a batched radix-2 Stockham FFT in FP64 (Stockham autosort form as in
// E. Bainville, "OpenCL Fast Fourier Transform", 2010), one pass per kernel.
#include "gwc_internal.h"

namespace gwc {

namespace {

// coef[c][j] = q_j beta_j / w_j^2 with trapezoid weights q_j of the per-core grid.
__global__ void cumulant_coef_kernel(const double* __restrict__ omega_rel, int n_w, const double* __restrict__ im_sigma,
                                     int n_core, double* __restrict__ coef) {
  int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= n_core * n_w) return;
  int c = t / n_w, j = t % n_w;
  const double* w = omega_rel + (size_t)c * n_w;
  double q = 0.0;
  if (j > 0) q += 0.5 * (w[j] - w[j - 1]);
  if (j < n_w - 1) q += 0.5 * (w[j + 1] - w[j]);
  double wj = w[j];
  double beta = fabs(im_sigma[t]) * (1.0 / 3.14159265358979323846);
  coef[t] = wj == 0.0 ? 0.0 : q * beta / (wj * wj);
}

// g[c][k] = w_k exp(C~(t_k) - eta t_k), C~ summed over the grid in FP64. Each thread takes KT consecutive
// times: per grid point one sincos at its first time and one for the step w_j dt, then the phase advances
// by that rotation (FP64 sincos runs at the FP64 rate, 1/64 of FP32 on this part; the rotation drifts by
// ~KT ulp over a block).
constexpr int KT = 32;

__global__ void cumulant_time_kernel(const double* __restrict__ omega_rel, int n_w, const double* __restrict__ coef,
                                     int n_core, int n_t, double dt, double eta, double2* __restrict__ g) {
  extern __shared__ double sh[];  // [2][n_w]
  double* sw = sh;
  double* sc = sh + n_w;
  const int c = blockIdx.y;
  for (int j = threadIdx.x; j < n_w; j += blockDim.x) {
    sw[j] = omega_rel[(size_t)c * n_w + j];
    sc[j] = coef[(size_t)c * n_w + j];
  }
  __syncthreads();
  const int k0 = (blockIdx.x * blockDim.x + threadIdx.x) * KT;
  if (k0 >= n_t) return;
  double re[KT], im[KT];
#pragma unroll
  for (int q = 0; q < KT; ++q) re[q] = im[q] = 0.0;
  const double t0 = dt * k0;
  for (int j = 0; j < n_w; ++j) {
    const double cj = sc[j];
    if (cj == 0.0) continue;
    double sn, cs, sd, cd;
    sincos(sw[j] * t0, &sn, &cs);
    sincos(sw[j] * dt, &sd, &cd);
#pragma unroll
    for (int q = 0; q < KT; ++q) {
      re[q] += cj * (cs - 1.0);
      im[q] -= cj * sn;
      const double c2 = cs * cd - sn * sd;  // angle + w_j dt
      sn = sn * cd + cs * sd;
      cs = c2;
    }
  }
#pragma unroll
  for (int q = 0; q < KT; ++q) {
    const int k = k0 + q;
    if (k >= n_t) break;
    const double t = dt * k;
    const double mag = exp(re[q] - eta * t) * (k == 0 ? 0.5 : 1.0);
    double sn, cs;
    sincos(im[q], &sn, &cs);
    g[(size_t)c * n_t + k] = make_double2(mag * cs, mag * sn);
  }
}

__global__ void twiddle_kernel(int n, double2* __restrict__ tw) {
  int m = blockIdx.x * blockDim.x + threadIdx.x;
  if (m >= n / 2) return;
  double sn, cs;
  sincospi(2.0 * (double)m / (double)n, &sn, &cs);  // e^{+2 pi i m / n}
  tw[m] = make_double2(cs, sn);
}

// One radix-2 Stockham pass with span p (1, 2, ..., n/2); X_j = sum_k x_k e^{+2 pi i jk/n}.
__global__ void stockham_pass_kernel(const double2* __restrict__ x, double2* __restrict__ y, int n, int p,
                                     const double2* __restrict__ tw, int n_batch) {
  long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  int half = n >> 1;
  if (t >= (long long)half * n_batch) return;
  int b = (int)(t / half), i = (int)(t % half);
  const double2* xb = x + (size_t)b * n;
  double2* yb = y + (size_t)b * n;
  int k = i & (p - 1);
  double2 u0 = xb[i], u1 = xb[i + half];
  double2 w = tw[k * (half / p)];  // e^{+i pi k / p}
  double2 v = make_double2(u1.x * w.x - u1.y * w.y, u1.x * w.y + u1.y * w.x);
  int j = (i << 1) - k;
  yb[j] = make_double2(u0.x + v.x, u0.y + v.y);
  yb[j + p] = make_double2(u0.x - v.x, u0.y - v.y);
}

__global__ void spectrum_out_kernel(const double2* __restrict__ X, int n, int n_core, double dt, double* __restrict__ a,
                                    double* __restrict__ nu) {
  long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (t >= (long long)n * n_core) return;
  int c = (int)(t / n), o = (int)(t % n);
  int j = (o + n / 2) & (n - 1);  // ascending nu: o = 0 <-> j = n/2 (most negative)
  a[t] = dt * X[(size_t)c * n + j].x * (1.0 / 3.14159265358979323846);
  if (nu && c == 0) nu[o] = 2.0 * 3.14159265358979323846 * (double)(o - n / 2) / ((double)n * dt);
}

}  // namespace

int launch_cumulant_spectrum(const double* omega_rel, int n_w, const double* im_sigma, int n_core, int n_t, double t_max,
                             double eta, double* work_a, double* work_b, double* coef, double* twiddle, double* a_out,
                             double* nu_out, cudaStream_t s) {
  int launches = 0;
  const double dt = t_max / n_t;
  int tot = n_core * n_w;
  cumulant_coef_kernel<<<(tot + 255) / 256, 256, 0, s>>>(omega_rel, n_w, im_sigma, n_core, coef);
  ++launches;
  size_t sm = sizeof(double) * 2 * (size_t)n_w;
  if (sm > 48 * 1024) {
    if (cudaFuncSetAttribute(cumulant_time_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm) != cudaSuccess)
      return -1;
  }
  dim3 g((n_t + 256 * KT - 1) / (256 * KT), n_core);
  cumulant_time_kernel<<<g, 256, sm, s>>>(omega_rel, n_w, coef, n_core, n_t, dt, eta, (double2*)work_a);
  ++launches;
  twiddle_kernel<<<(n_t / 2 + 255) / 256, 256, 0, s>>>(n_t, (double2*)twiddle);
  ++launches;
  double2* src = (double2*)work_a;
  double2* dst = (double2*)work_b;
  long long work = (long long)(n_t / 2) * n_core;
  for (int p = 1; p < n_t; p <<= 1) {
    stockham_pass_kernel<<<(int)((work + 255) / 256), 256, 0, s>>>(src, dst, n_t, p, (const double2*)twiddle, n_core);
    ++launches;
    double2* tmp = src;
    src = dst;
    dst = tmp;
  }
  long long outn = (long long)n_t * n_core;
  spectrum_out_kernel<<<(int)((outn + 255) / 256), 256, 0, s>>>(src, n_t, n_core, dt, a_out, nu_out);
  ++launches;
  return cudaPeekAtLastError() == cudaSuccess ? launches : -1;
}

}  // namespace gwc
