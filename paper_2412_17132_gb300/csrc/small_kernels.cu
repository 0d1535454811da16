// Small element-wise kernels of the self-energy path: transition energies, the
// frequency factor table D_ia(z), precision copies of O_ov, right-hand-side gathers,
// the exchange self-energy and output conversion.
#include "gwc_internal.h"

namespace gwc {

namespace {

__global__ void delta_kernel(const double* __restrict__ eps, int n_occ, int n_virt, double* __restrict__ delta) {
  long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  long long n = (long long)n_occ * n_virt;
  if (t >= n) return;
  int i = (int)(t / n_virt), a = (int)(t % n_virt);
  delta[t] = eps[n_occ + a] - eps[i];
}

// D_ia(z) = 2[1/(z - Delta) - 1/(z + Delta)] = 4 Delta / (z^2 - Delta^2), z = x + i y.
// (Sec. "Self-energy evaluation": the RI polarizability of the CD method.)
template <typename T>
__global__ void dtable_kernel(const double* __restrict__ z, int F, const double* __restrict__ delta, int n_ov, int ld,
                              T* __restrict__ out) {
  int f = blockIdx.y;
  int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (f >= F || k >= ld) return;
  T* re = out + (size_t)f * 2 * ld;
  T* im = re + ld;
  if (k >= n_ov) {
    re[k] = (T)0;
    im[k] = (T)0;
    return;
  }
  double x = z[2 * f], y = z[2 * f + 1], dl = delta[k];
  double a = (x - dl) * (x + dl) - y * y;  // Re(z^2 - Delta^2)
  double b = 2.0 * x * y;                  // Im(z^2 - Delta^2)
  double s = 4.0 * dl / (a * a + b * b);
  re[k] = (T)(s * a);
  im[k] = (T)(-s * b);
}

__global__ void split_o_kernel(const double* __restrict__ o, int n_aux, int n_ov, int n_aux_pad, int n_ov_pad,
                               __nv_bfloat16* __restrict__ hi, __nv_bfloat16* __restrict__ lo, float* __restrict__ f32) {
  long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  long long total = (long long)n_aux_pad * n_ov_pad;
  if (t >= total) return;
  int p = (int)(t / n_ov_pad), k = (int)(t % n_ov_pad);
  double v = (p < n_aux && k < n_ov) ? o[(size_t)p * n_ov + k] : 0.0;
  __nv_bfloat16 h = __double2bfloat16(v);
  double r = v - (double)__bfloat162float(h);
  hi[t] = h;
  lo[t] = __double2bfloat16(r);
  f32[t] = (float)v;
}

template <typename S>
__global__ void rhs_gather_kernel(const double* __restrict__ src, long long src_row_stride, const int* __restrict__ row_of,
                                  int r, int n_aux, S* __restrict__ dst, long long ldr, long long rhs_stride,
                                  double* __restrict__ bnorm2) {
  int f = blockIdx.y, q = blockIdx.x;
  int row = row_of[f * r + q];
  const double* s = src + (size_t)row * src_row_stride;
  S* d = dst + f * rhs_stride + q * ldr;
  double acc = 0.0;
  for (int p = threadIdx.x; p < n_aux; p += blockDim.x) {
    double v = s[p];
    d[p] = sfrom<S>(v, 0.0);
    acc += v * v;
  }
  __shared__ double red[32];
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += red[w];
    bnorm2[f * r + q] = t;
  }
}

// Sigma^x_n = -sum_{i occ} (n i | i n) = -sum_{i occ} sum_P (O^P_{n i})^2  (Eq. sigma_x)
__global__ void sigma_x_kernel(const double* __restrict__ o_core, int n_occ, int n_core, int n_aux, double* __restrict__ sx) {
  int c = blockIdx.x;
  double acc = 0.0;
  long long total = (long long)n_occ * n_aux;
  for (long long t = threadIdx.x; t < total; t += blockDim.x) {
    int i = (int)(t / n_aux), p = (int)(t % n_aux);
    double v = o_core[((size_t)i * n_core + c) * n_aux + p];
    acc += v * v;
  }
  __shared__ double red[32];
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += red[w];
    sx[c] = -t;
  }
}

__global__ void fill_z_pairs_kernel(const double* __restrict__ eps, const int* __restrict__ pair_m,
                                    const double* __restrict__ pair_w, int n_pairs, double eta, double* __restrict__ z) {
  int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= n_pairs) return;
  z[2 * p] = fabs(eps[pair_m[p]] - pair_w[p]);
  z[2 * p + 1] = eta;
}

template <typename S>
__global__ void mat_to_c128_kernel(const S* __restrict__ m, int n, long long ldm, long long stride, double* __restrict__ out) {
  int f = blockIdx.z;
  int q = blockIdx.x * blockDim.x + threadIdx.x;
  int p = blockIdx.y;
  if (q >= n) return;
  int r = p >= q ? p : q, c = p >= q ? q : p;  // lower triangle holds the data
  S v = m[f * stride + (long long)r * ldm + c];
  double* o = out + (((size_t)f * n + p) * n + q) * 2;
  o[0] = sre(v);
  o[1] = sim(v);
}

inline int grid1(long long n, int b) { return (int)((n + b - 1) / b); }

}  // namespace

int launch_delta(const double* eps, int n_occ, int n_virt, double* delta, cudaStream_t s) {
  long long n = (long long)n_occ * n_virt;
  delta_kernel<<<grid1(n, 256), 256, 0, s>>>(eps, n_occ, n_virt, delta);
  return cudaPeekAtLastError() == cudaSuccess ? 1 : -1;
}

int launch_dtable(const double* z, int F, const double* delta, int n_ov, int ld, bool fp32, void* out, cudaStream_t s) {
  dim3 g(grid1(ld, 256), F);
  if (fp32)
    dtable_kernel<float><<<g, 256, 0, s>>>(z, F, delta, n_ov, ld, (float*)out);
  else
    dtable_kernel<double><<<g, 256, 0, s>>>(z, F, delta, n_ov, ld, (double*)out);
  return cudaPeekAtLastError() == cudaSuccess ? 1 : -1;
}

int launch_split_o(const double* o_ov, int n_aux, int n_ov, int n_aux_pad, int n_ov_pad, __nv_bfloat16* hi,
                   __nv_bfloat16* lo, float* f32, cudaStream_t s) {
  long long n = (long long)n_aux_pad * n_ov_pad;
  split_o_kernel<<<grid1(n, 256), 256, 0, s>>>(o_ov, n_aux, n_ov, n_aux_pad, n_ov_pad, hi, lo, f32);
  return cudaPeekAtLastError() == cudaSuccess ? 1 : -1;
}

int launch_rhs_gather(MatKind kind, const double* src, long long src_row_stride, const int* row_of, int F, int r,
                      int n_aux, void* dst, long long ldr, long long rhs_stride, double* bnorm2, cudaStream_t s) {
  dim3 g(r, F);
  switch (kind) {
    case MatKind::RealF32:
      rhs_gather_kernel<float><<<g, 128, 0, s>>>(src, src_row_stride, row_of, r, n_aux, (float*)dst, ldr, rhs_stride, bnorm2);
      break;
    case MatKind::CplxF32:
      rhs_gather_kernel<float2><<<g, 128, 0, s>>>(src, src_row_stride, row_of, r, n_aux, (float2*)dst, ldr, rhs_stride, bnorm2);
      break;
    case MatKind::RealF64:
      rhs_gather_kernel<double><<<g, 128, 0, s>>>(src, src_row_stride, row_of, r, n_aux, (double*)dst, ldr, rhs_stride, bnorm2);
      break;
    case MatKind::CplxF64:
      rhs_gather_kernel<double2><<<g, 128, 0, s>>>(src, src_row_stride, row_of, r, n_aux, (double2*)dst, ldr, rhs_stride, bnorm2);
      break;
  }
  return cudaPeekAtLastError() == cudaSuccess ? 1 : -1;
}

int launch_sigma_x(const double* o_core, int n_occ, int n_core, int n_aux, double* sx, cudaStream_t s) {
  sigma_x_kernel<<<n_core, 256, 0, s>>>(o_core, n_occ, n_core, n_aux, sx);
  return cudaPeekAtLastError() == cudaSuccess ? 1 : -1;
}

int launch_fill_z_pairs(const double* eps, const int* pair_m, const double* pair_w, int n_pairs, double eta, double* z,
                        cudaStream_t s) {
  if (n_pairs <= 0) return 0;
  fill_z_pairs_kernel<<<grid1(n_pairs, 128), 128, 0, s>>>(eps, pair_m, pair_w, n_pairs, eta, z);
  return cudaPeekAtLastError() == cudaSuccess ? 1 : -1;
}

int launch_mat_to_c128(MatKind kind, const void* mats, int n, long long ldm, long long stride, int F, double* out,
                       cudaStream_t s) {
  dim3 g(grid1(n, 128), n, F);
  switch (kind) {
    case MatKind::RealF32: mat_to_c128_kernel<float><<<g, 128, 0, s>>>((const float*)mats, n, ldm, stride, out); break;
    case MatKind::CplxF32: mat_to_c128_kernel<float2><<<g, 128, 0, s>>>((const float2*)mats, n, ldm, stride, out); break;
    case MatKind::RealF64: mat_to_c128_kernel<double><<<g, 128, 0, s>>>((const double*)mats, n, ldm, stride, out); break;
    case MatKind::CplxF64: mat_to_c128_kernel<double2><<<g, 128, 0, s>>>((const double2*)mats, n, ldm, stride, out); break;
  }
  return cudaPeekAtLastError() == cudaSuccess ? 1 : -1;
}

}  // namespace gwc
