// SIMT polarizability build (FP64 for the plain FP64 path, FP32 for the FP32 mode).
//
//   Pi_PQ(z_f) = sum_k O_Pk D_f(k) O_Qk,   k = (i, a) occupied-virtual pair
//
// (RI polarizability of the contour-deformation self-energy, Sec. "Self-energy
// evaluation"). One CTA computes one 64x64 lower-triangle tile (P-tile >= Q-tile) for
// one frequency; the D_f(k) scaling is applied to the Q operand as it is read from
// shared memory, so O is read once per tile and frequency part. The epilogue writes
// alpha*Pi + beta*I into the dielectric matrix buffer (alpha = -1, beta = 1 gives
// eps = 1 - Pi directly).
#include "gwc_internal.h"

namespace gwc {

namespace {

constexpr int kTile = 64;
constexpr int kKc = 16;

__device__ __forceinline__ void tile_pair(int t, int& ip, int& iq) {
  int a = (int)((sqrt(8.0 * t + 1.0) - 1.0) * 0.5);
  while ((a + 1) * (a + 2) / 2 <= t) ++a;
  while (a * (a + 1) / 2 > t) --a;
  ip = a;
  iq = t - a * (a + 1) / 2;
}

template <typename S> __device__ __forceinline__ S make_out(double re, double im);
template <> __device__ __forceinline__ float make_out<float>(double re, double) { return (float)re; }
template <> __device__ __forceinline__ double make_out<double>(double re, double) { return re; }
template <> __device__ __forceinline__ float2 make_out<float2>(double re, double im) { return make_float2((float)re, (float)im); }
template <> __device__ __forceinline__ double2 make_out<double2>(double re, double im) { return make_double2(re, im); }

template <typename T, typename S, bool CPLX>
__global__ void __launch_bounds__(256) chi0_simt_kernel(const T* __restrict__ o, int ldo, int n_aux, int n_ov,
                                                         const T* __restrict__ dtab, int ld_dtab, double alpha,
                                                         double beta, S* __restrict__ out, long long ldm,
                                                         long long mat_stride, int full, const int* __restrict__ active) {
  const int f = blockIdx.y;
  if (active && !active[f]) return;
  int ip, iq;
  tile_pair(blockIdx.x, ip, iq);
  const int p0 = ip * kTile, q0 = iq * kTile;
  const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;

  __shared__ T ps[kKc][kTile];
  __shared__ T qs[kKc][kTile];
  __shared__ T dre[kKc];
  __shared__ T dim_[kKc];

  T acc_re[4][4], acc_im[4][4];
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int b = 0; b < 4; ++b) {
      acc_re[a][b] = (T)0;
      acc_im[a][b] = (T)0;
    }

  const T* dr = dtab + (size_t)f * 2 * ld_dtab;
  const T* di = dr + ld_dtab;

  for (int k0 = 0; k0 < n_ov; k0 += kKc) {
#pragma unroll
    for (int e = 0; e < 4; ++e) {
      int idx = tid + 256 * e;
      int row = idx >> 4, kk = idx & 15;
      int k = k0 + kk;
      int p = p0 + row, q = q0 + row;
      ps[kk][row] = (p < n_aux && k < n_ov) ? o[(size_t)p * ldo + k] : (T)0;
      qs[kk][row] = (q < n_aux && k < n_ov) ? o[(size_t)q * ldo + k] : (T)0;
    }
    if (tid < kKc) {
      int k = k0 + tid;
      dre[tid] = k < n_ov ? dr[k] : (T)0;
      dim_[tid] = (CPLX && k < n_ov) ? di[k] : (T)0;
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < kKc; ++kk) {
      T a[4], br[4], bi[4];
#pragma unroll
      for (int u = 0; u < 4; ++u) a[u] = ps[kk][ty + 16 * u];
      T sr = dre[kk], si = dim_[kk];
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        T qv = qs[kk][tx + 16 * u];
        br[u] = qv * sr;
        if (CPLX) bi[u] = qv * si;
      }
#pragma unroll
      for (int x = 0; x < 4; ++x)
#pragma unroll
        for (int y = 0; y < 4; ++y) {
          acc_re[x][y] = fma(a[x], br[y], acc_re[x][y]);
          if (CPLX) acc_im[x][y] = fma(a[x], bi[y], acc_im[x][y]);
        }
    }
    __syncthreads();
  }

  S* m = out + f * mat_stride;
#pragma unroll
  for (int x = 0; x < 4; ++x)
#pragma unroll
    for (int y = 0; y < 4; ++y) {
      int p = p0 + ty + 16 * x, q = q0 + tx + 16 * y;
      if (p >= n_aux || q >= n_aux) continue;
      if (p < q && !full) continue;
      double re = alpha * (double)acc_re[x][y] + (p == q ? beta : 0.0);
      double im = CPLX ? alpha * (double)acc_im[x][y] : 0.0;
      S v = make_out<S>(re, im);
      m[(long long)p * ldm + q] = v;
      if (full && ip != iq) m[(long long)q * ldm + p] = v;
    }
}

}  // namespace

int launch_chi0_simt(MatKind kind, const void* o_ov, int ldo, int n_aux, int n_ov, const void* dtab, int ld_dtab, int F,
                     double alpha, double beta, void* out, long long ldm, long long mat_stride, int full,
                     const int* active, cudaStream_t s) {
  int nt = (n_aux + kTile - 1) / kTile;
  dim3 g(nt * (nt + 1) / 2, F);
  switch (kind) {
    case MatKind::RealF64:
      chi0_simt_kernel<double, double, false><<<g, 256, 0, s>>>((const double*)o_ov, ldo, n_aux, n_ov, (const double*)dtab,
                                                               ld_dtab, alpha, beta, (double*)out, ldm, mat_stride, full, active);
      break;
    case MatKind::CplxF64:
      chi0_simt_kernel<double, double2, true><<<g, 256, 0, s>>>((const double*)o_ov, ldo, n_aux, n_ov, (const double*)dtab,
                                                               ld_dtab, alpha, beta, (double2*)out, ldm, mat_stride, full, active);
      break;
    case MatKind::RealF32:
      chi0_simt_kernel<float, float, false><<<g, 256, 0, s>>>((const float*)o_ov, ldo, n_aux, n_ov, (const float*)dtab,
                                                             ld_dtab, alpha, beta, (float*)out, ldm, mat_stride, full, active);
      break;
    case MatKind::CplxF32:
      chi0_simt_kernel<float, float2, true><<<g, 256, 0, s>>>((const float*)o_ov, ldo, n_aux, n_ov, (const float*)dtab,
                                                             ld_dtab, alpha, beta, (float2*)out, ldm, mat_stride, full, active);
      break;
  }
  return cudaPeekAtLastError() == cudaSuccess ? 1 : -1;
}

}  // namespace gwc
