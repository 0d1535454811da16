// Batched dielectric factorisation eps = L D L^T (no pivoting) and the screened
// contraction W^c = b^T (eps^-1 - 1) b = y^T D^-1 y - b^T b with y = L^-1 b.
//
// eps(i xi) is real symmetric positive definite (Pi(i xi) is negative semidefinite), so
// there this is a Cholesky-type factorisation; eps(x + i eta) is complex SYMMETRIC (not
// Hermitian), so no conjugation appears anywhere. Without pivoting a zero pivot is
// possible in exact arithmetic only; it is detected (|d| below a floor) and reported
// through the status word, and the pivot is replaced by 1 so the batch stays finite.
//
// Storage after the factorisation (matrix [n][ldm], row-major):
//   strictly lower part  W = L D   (W_ij = L_ij d_j, j < i)
//   diagonal             d
//   strictly upper part  L^T       (A[j][i] = L_ij; scratch used by the trailing updates)
//
// One CTA factors one matrix, right-looking and blocked:
//   * 64-wide panels, each factored as two 32-wide halves: the two 32 x 32 diagonal blocks in
//     shared memory, then every row below in one pass by one thread (solve against block 1,
//     apply block 1 to its block-2 columns, solve against block 2), storing W (lower) and L
//     (upper).
//   * the trailing lower triangle is updated with the rank-64 product W_panel L_panel^T, in
//     64 x 64 tiles (4 x 4 per thread); both operands are staged through shared memory by
//     cp.async in 32-deep chunks, double-buffered across chunks and tiles.
#include <algorithm>

#include "gwc_internal.h"
#include "ldlt_simt.cuh"

namespace gwc {

namespace {

template <typename S>
__global__ void __launch_bounds__(256) ldlt_kernel(S* __restrict__ mats, int n, int nrow, long long ldm, long long stride,
                                                    const int* __restrict__ active, unsigned* __restrict__ status) {
  const int f = blockIdx.x;
  if (active && !active[f]) return;
  S* A = mats + f * stride;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  // the panel scratch and the update stages alias (the phases alternate)
  const PanelSmem<S, kSimtThreads> ps(smem_raw);
  S* stages = reinterpret_cast<S*>(smem_raw);
  __shared__ int sing;
  if (threadIdx.x == 0) sing = 0;

  for (int k0 = 0; k0 < n; k0 += PW) {
    const int kb = min(PW, n - k0);
    factor_panel<S, kSimtThreads>(A, n, nrow, ldm, k0, ps, sing);
    // rank-kb trailing update of the lower triangle beyond the panel (and of appended rows)
    if (k0 + kb < n) update_region(A, nrow, ldm, k0 + kb, k0 + kb, n, k0, kb, stages);
  }
  __syncthreads();
  if (threadIdx.x == 0 && sing) atomicOr(status, kStatSingular);
}

// Forward substitution with the W storage, for a block of SR right-hand sides (in place):
//   y_i = b_i - sum_{l<i} W_il u_l,  u_l = y_l / d_l   (since L_il = W_il / d_l)
//   w_q = sum_i y_i^2 / d_i - |b_q|^2 = sum_i u_i^2 d_i - |b_q|^2.
// The right-hand-side buffer ends up holding u. Grid: (matrix f, RHS block). Per 64-row panel:
//   * update: acc = -W[panel rows][0 .. k0) U[0 .. k0)[block], a product in 32-deep chunks staged through
//     shared memory, 4 x 4 outputs per thread (rows strided by 16 so that a warp reads distinct rows);
//   * panel: the 64 x 64 diagonal block by four threads per right-hand side (strided partial sums of the
//     row, two shuffles), u_i = (b_i + acc_i - sum_{l<i} W_il u_l) / d_i, u_i^2 d_i summed in FP64.
constexpr int SB = 64;  // panel rows
constexpr int SR = 64;  // right-hand sides per CTA
constexpr int SK = 32;  // depth of the staged update chunks

template <typename S>
struct SolveSmem {
  // update phase: ls[SB][SK + 1], us[SK][SR + 1]; panel phase: acc (then u) [SB][SR + 1], wd [SB][SB + 1], dv [SB]
  static constexpr size_t upd = (size_t)SB * (SK + 1) + (size_t)SK * (SR + 1);
  static constexpr size_t pan = (size_t)SB * (SR + 1) + (size_t)SB * (SB + 1) + SB;
  static constexpr size_t elems = upd > pan ? upd : pan;
  static size_t bytes() { return elems * sizeof(S); }
};

template <typename S>
__global__ void __launch_bounds__(256) ldlt_solve_kernel(const S* __restrict__ mats, int n, long long ldm, long long stride,
                                                          S* __restrict__ rhs, int r, long long ldr, long long rhs_stride,
                                                          const double* __restrict__ bnorm2, double* __restrict__ w,
                                                          long long w_stride, const int* __restrict__ active) {
  const int f = blockIdx.x;
  if (active && !active[f]) return;
  const int q0 = blockIdx.y * SR;
  const int nq = min(SR, r - q0);
  const S* L = mats + f * stride;
  S* Y = rhs + f * rhs_stride + (long long)q0 * ldr;
  const int tid = threadIdx.x;

  extern __shared__ __align__(16) unsigned char smem_raw[];
  S(*ls)[SK + 1] = reinterpret_cast<S(*)[SK + 1]>(smem_raw);
  S(*us)[SR + 1] = reinterpret_cast<S(*)[SR + 1]>(smem_raw + sizeof(S) * SB * (SK + 1));
  S(*acc_s)[SR + 1] = reinterpret_cast<S(*)[SR + 1]>(smem_raw);
  S(*wd)[SB + 1] = reinterpret_cast<S(*)[SB + 1]>(smem_raw + sizeof(S) * SB * (SR + 1));
  S* dv = reinterpret_cast<S*>(smem_raw + sizeof(S) * (SB * (SR + 1) + SB * (SB + 1)));

  const int tr = tid & 15, tc = tid >> 4;         // update: rows tr + 16 a, columns 4 tc + b
  const int cq = tid >> 2, cp = tid & 3;           // panel: right-hand side cq, quarter cp of each row sum
  double wr = 0.0, wi = 0.0;                       // sum u_i^2 d_i of right-hand side cq (kept by cp == 0)
  for (int k0 = 0; k0 < n; k0 += SB) {
    const int kb = min(SB, n - k0);
    S acc[4][4];
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
      for (int b = 0; b < 4; ++b) acc[a][b] = szero<S>();
    for (int l0 = 0; l0 < k0; l0 += SK) {
      for (int e = tid; e < SB * SK; e += 256) {
        const int i = e / SK, l = e % SK;
        ls[i][l] = i < kb ? L[(long long)(k0 + i) * ldm + l0 + l] : szero<S>();
      }
      for (int e = tid; e < SR * SK; e += 256) {
        const int q = e / SK, l = e % SK;
        us[l][q] = q < nq ? Y[(long long)q * ldr + l0 + l] : szero<S>();
      }
      __syncthreads();
#pragma unroll 4
      for (int l = 0; l < SK; ++l) {
        S av[4], bv[4];
#pragma unroll
        for (int a = 0; a < 4; ++a) av[a] = ls[tr + 16 * a][l];
#pragma unroll
        for (int b = 0; b < 4; ++b) bv[b] = us[l][4 * tc + b];
#pragma unroll
        for (int a = 0; a < 4; ++a)
#pragma unroll
          for (int b = 0; b < 4; ++b) acc[a][b] = sfnms(av[a], bv[b], acc[a][b]);
      }
      __syncthreads();
    }
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
      for (int b = 0; b < 4; ++b) acc_s[tr + 16 * a][4 * tc + b] = acc[a][b];
    for (int e = tid; e < SB * SB; e += 256) {
      const int i = e / SB, l = e % SB;
      wd[i][l] = (i < kb && l < i) ? L[(long long)(k0 + i) * ldm + k0 + l] : szero<S>();
    }
    if (tid < SB) dv[tid] = tid < kb ? L[(long long)(k0 + tid) * ldm + k0 + tid] : sfrom<S>(1.0, 0.0);
    __syncthreads();
    // the panel's rows in order; the four threads of a right-hand side are consecutive lanes of one warp
    for (int i = 0; i < kb; ++i) {
      S part = szero<S>();
      for (int l = cp; l < i; l += 4) part = sadd(part, smul(wd[i][l], acc_s[l][cq]));
      part = sadd(part, shfl_xor_s(part, 1));
      part = sadd(part, shfl_xor_s(part, 2));
      if (cp == 0 && cq < nq) {
        const S v = ssub(sadd(Y[(long long)cq * ldr + k0 + i], acc_s[i][cq]), part);
        const S u = smul(v, sinv(dv[i]));
        acc_s[i][cq] = u;
        Y[(long long)cq * ldr + k0 + i] = u;
        const S t = smul(smul(u, u), dv[i]);
        wr += sre(t);
        wi += sim(t);
      }
      __syncwarp();
    }
    __syncthreads();
  }
  if (cp == 0 && cq < nq) {
    double* o = w + f * w_stride + (long long)(q0 + cq) * 2;
    o[0] = wr - bnorm2[(long long)f * r + q0 + cq];
    o[1] = wi;
  }
}

template <typename S>
size_t solve_smem() {
  return SolveSmem<S>::bytes();
}

template <typename S>
int run_ldlt(S* mats, int n, int nrow, long long ldm, long long stride, int F, const int* active, unsigned* status,
             cudaStream_t s) {
  static bool attr = false;
  const size_t sm = std::max(FactorSmem<S>::bytes(), PanelSmem<S, kSimtThreads>::bytes());
  if (!attr) {
    if (cudaFuncSetAttribute(ldlt_kernel<S>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm) != cudaSuccess) return -1;
    attr = true;
  }
  ldlt_kernel<S><<<F, 256, sm, s>>>(mats, n, nrow, ldm, stride, active, status);
  return cudaPeekAtLastError() == cudaSuccess ? 1 : -1;
}

template <typename S>
int run_solve(const S* mats, int n, long long ldm, long long stride, S* rhs, int r, long long ldr, long long rhs_stride,
              const double* bnorm2, int F, double* w, long long w_stride, const int* active, cudaStream_t s) {
  static bool attr = false;
  const size_t sm = solve_smem<S>();
  if (!attr) {
    if (cudaFuncSetAttribute(ldlt_solve_kernel<S>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm) != cudaSuccess)
      return -1;
    attr = true;
  }
  dim3 g(F, (r + SR - 1) / SR);
  ldlt_solve_kernel<S><<<g, 256, sm, s>>>(mats, n, ldm, stride, rhs, r, ldr, rhs_stride, bnorm2, w, w_stride, active);
  return cudaPeekAtLastError() == cudaSuccess ? 1 : -1;
}

}  // namespace

int launch_ldlt(MatKind kind, void* mats, int n, int nrow, long long ldm, long long stride, int F, const int* active,
                unsigned* status, cudaStream_t s) {
  // 16-byte staging needs even leading dimensions and 16-byte aligned matrices
  if ((ldm % 4) || (stride % 4) || (reinterpret_cast<uintptr_t>(mats) & 15) || nrow < n) return -1;
  switch (kind) {
    case MatKind::RealF32: return run_ldlt((float*)mats, n, nrow, ldm, stride, F, active, status, s);
    case MatKind::CplxF32: return run_ldlt((float2*)mats, n, nrow, ldm, stride, F, active, status, s);
    case MatKind::RealF64: return run_ldlt((double*)mats, n, nrow, ldm, stride, F, active, status, s);
    default: return run_ldlt((double2*)mats, n, nrow, ldm, stride, F, active, status, s);
  }
}

// ---- appended right-hand-side rows ("bordered" matrix) -------------------------------------------
// With the r vectors b_q appended as rows n..n+r-1 of the lower triangle, the factorisation's row
// solves give W[n+q][k] = (L^-1 b_q)_k = y_k, so W^c_q = sum_k y_k^2 / d_k - |b_q|^2 follows from
// the factored rows without a separate forward substitution.
template <typename S>
__global__ void border_rows_kernel(S* __restrict__ mats, int n, long long ldm, long long stride,
                                   const double* __restrict__ src, long long src_row_stride, const int* __restrict__ row_of,
                                   int r, double* __restrict__ bnorm2) {
  const int f = blockIdx.y, q = blockIdx.x;
  const double* b = src + (size_t)row_of[f * r + q] * src_row_stride;
  S* row = mats + f * stride + (long long)(n + q) * ldm;
  double acc = 0.0;
  for (int k = threadIdx.x; k < n; k += blockDim.x) {
    const double v = b[k];
    row[k] = sfrom<S>(v, 0.0);
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

template <typename S>
__global__ void border_w_kernel(const S* __restrict__ mats, int n, long long ldm, long long stride, int r,
                                const double* __restrict__ bnorm2, double* __restrict__ w, long long w_stride,
                                const int* __restrict__ active) {
  const int f = blockIdx.y, q = blockIdx.x;
  if (active && !active[f]) return;
  const S* A = mats + f * stride;
  const S* y = A + (long long)(n + q) * ldm;
  double sr = 0.0, si = 0.0;
  for (int k = threadIdx.x; k < n; k += blockDim.x) {
    const S yk = y[k];
    const S t = smul(smul(yk, yk), sinv(A[(long long)k * ldm + k]));
    sr += sre(t);
    si += sim(t);
  }
  __shared__ double red[2][32];
  for (int o = 16; o > 0; o >>= 1) {
    sr += __shfl_down_sync(0xffffffffu, sr, o);
    si += __shfl_down_sync(0xffffffffu, si, o);
  }
  if ((threadIdx.x & 31) == 0) {
    red[0][threadIdx.x >> 5] = sr;
    red[1][threadIdx.x >> 5] = si;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double a = 0.0, b = 0.0;
    for (int v = 0; v < (int)(blockDim.x >> 5); ++v) {
      a += red[0][v];
      b += red[1][v];
    }
    double* o = w + f * w_stride + (long long)q * 2;
    o[0] = a - bnorm2[(long long)f * r + q];
    o[1] = b;
  }
}

int launch_border_rows(MatKind kind, void* mats, int n, long long ldm, long long stride, const double* src,
                       long long src_row_stride, const int* row_of, int F, int r, double* bnorm2, cudaStream_t s) {
  dim3 g(r, F);
  switch (kind) {
    case MatKind::CplxF32:
      border_rows_kernel<float2><<<g, 256, 0, s>>>((float2*)mats, n, ldm, stride, src, src_row_stride, row_of, r, bnorm2);
      break;
    case MatKind::CplxF64:
      border_rows_kernel<double2><<<g, 256, 0, s>>>((double2*)mats, n, ldm, stride, src, src_row_stride, row_of, r, bnorm2);
      break;
    case MatKind::RealF32:
      border_rows_kernel<float><<<g, 256, 0, s>>>((float*)mats, n, ldm, stride, src, src_row_stride, row_of, r, bnorm2);
      break;
    default:
      border_rows_kernel<double><<<g, 256, 0, s>>>((double*)mats, n, ldm, stride, src, src_row_stride, row_of, r, bnorm2);
      break;
  }
  return cudaPeekAtLastError() == cudaSuccess ? 1 : -1;
}

int launch_border_w(MatKind kind, const void* mats, int n, long long ldm, long long stride, int F, int r,
                    const double* bnorm2, double* w, long long w_stride, const int* active, cudaStream_t s) {
  dim3 g(r, F);
  switch (kind) {
    case MatKind::CplxF32:
      border_w_kernel<float2><<<g, 256, 0, s>>>((const float2*)mats, n, ldm, stride, r, bnorm2, w, w_stride, active);
      break;
    case MatKind::CplxF64:
      border_w_kernel<double2><<<g, 256, 0, s>>>((const double2*)mats, n, ldm, stride, r, bnorm2, w, w_stride, active);
      break;
    case MatKind::RealF32:
      border_w_kernel<float><<<g, 256, 0, s>>>((const float*)mats, n, ldm, stride, r, bnorm2, w, w_stride, active);
      break;
    default:
      border_w_kernel<double><<<g, 256, 0, s>>>((const double*)mats, n, ldm, stride, r, bnorm2, w, w_stride, active);
      break;
  }
  return cudaPeekAtLastError() == cudaSuccess ? 1 : -1;
}

int launch_ldlt_solve_w(MatKind kind, const void* mats, int n, long long ldm, long long stride, void* rhs, int r,
                        long long ldr, long long rhs_stride, const double* bnorm2, int F, double* w, long long w_stride,
                        const int* active, cudaStream_t s) {
  switch (kind) {
    case MatKind::RealF32:
      return run_solve((const float*)mats, n, ldm, stride, (float*)rhs, r, ldr, rhs_stride, bnorm2, F, w, w_stride, active, s);
    case MatKind::CplxF32:
      return run_solve((const float2*)mats, n, ldm, stride, (float2*)rhs, r, ldr, rhs_stride, bnorm2, F, w, w_stride, active, s);
    case MatKind::RealF64:
      return run_solve((const double*)mats, n, ldm, stride, (double*)rhs, r, ldr, rhs_stride, bnorm2, F, w, w_stride, active, s);
    default:
      return run_solve((const double2*)mats, n, ldm, stride, (double2*)rhs, r, ldr, rhs_stride, bnorm2, F, w, w_stride, active,
                       s);
  }
}

}  // namespace gwc
