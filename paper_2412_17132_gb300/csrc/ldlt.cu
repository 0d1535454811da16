// Batched dielectric factorisation eps = L D L^T (no pivoting) and the screened
// contraction W^c = b^T (eps^-1 - 1) b = y^T D^-1 y - b^T b with y = L^-1 b.
//
// eps(i xi) is real symmetric positive definite (Pi(i xi) is negative semidefinite), so
// there this is a Cholesky-type factorisation; eps(x + i eta) is complex SYMMETRIC (not
// Hermitian), so no conjugation appears anywhere. Without pivoting a zero pivot is
// possible in exact arithmetic only; it is detected (|d| below a floor) and reported
// through the status word, and the pivot is replaced by 1 so the batch stays finite.
//
// One CTA factors one matrix, right-looking and blocked (panel width NB = 32):
//   1. the NB x NB diagonal block is factored in shared memory,
//   2. every row below solves against it (one thread per row),
//   3. the trailing lower triangle is updated tile by tile (64 x 64 tiles, 4 x 4 per thread)
//      with the rank-NB product (L D)_panel L_panel^T staged through shared memory.
#include "gwc_internal.h"

namespace gwc {

namespace {

constexpr int NB = 32;
constexpr int TT = 64;

template <typename S>
__global__ void __launch_bounds__(256) ldlt_kernel(S* __restrict__ mats, int n, long long ldm, long long stride,
                                                    const int* __restrict__ active, unsigned* __restrict__ status) {
  const int f = blockIdx.x;
  if (active && !active[f]) return;
  S* A = mats + f * stride;
  const int tid = threadIdx.x;

  extern __shared__ __align__(16) unsigned char smem_raw[];
  S(*lkk)[NB + 1] = reinterpret_cast<S(*)[NB + 1]>(smem_raw);
  S* dinv = reinterpret_cast<S*>(smem_raw + sizeof(S) * NB * (NB + 1));
  S(*ws)[TT + 1] = reinterpret_cast<S(*)[TT + 1]>(smem_raw + sizeof(S) * (NB * (NB + 1) + NB));  // (L D) of tile I
  S(*ls)[TT + 1] = ws + NB;  // L rows of tile J, transposed: ls[l][jj]
  __shared__ int sing;
  if (tid == 0) sing = 0;

  for (int k0 = 0; k0 < n; k0 += NB) {
    const int kb = min(NB, n - k0);
    // ---- 1. diagonal block -------------------------------------------------------------
    __syncthreads();
    for (int e = tid; e < NB * NB; e += 256) {
      int i = e / NB, j = e % NB;
      lkk[i][j] = (i < kb && j <= i) ? A[(long long)(k0 + i) * ldm + (k0 + j)] : szero<S>();
    }
    __syncthreads();
    for (int j = 0; j < kb; ++j) {
      S d = lkk[j][j];
      if (sabs2(d) < 1e-60) {
        if (tid == 0) sing = 1;
        d = sfrom<S>(1.0, 0.0);
      }
      S inv = sinv(d);
      // trailing update inside the block with the unscaled column j
      int m = kb - 1 - j;
      for (int e = tid; e < m * m; e += 256) {
        int i = j + 1 + e / m, l = j + 1 + e % m;
        if (l <= i) lkk[i][l] = sfnms(smul(lkk[i][j], inv), lkk[l][j], lkk[i][l]);
      }
      __syncthreads();
      if (tid == 0) {
        lkk[j][j] = d;
        dinv[j] = inv;
      }
      for (int i = j + 1 + tid; i < kb; i += 256) lkk[i][j] = smul(lkk[i][j], inv);
      __syncthreads();
    }
    for (int e = tid; e < kb * kb; e += 256) {
      int i = e / kb, j = e % kb;
      if (j <= i) A[(long long)(k0 + i) * ldm + (k0 + j)] = lkk[i][j];
    }
    // ---- 2. panel rows: L_i = A_i L_kk^-T D^-1 ------------------------------------------
    for (int i = k0 + kb + tid; i < n; i += 256) {
      S w[NB];
      S* row = A + (long long)i * ldm + k0;
#pragma unroll
      for (int j = 0; j < NB; ++j) w[j] = j < kb ? row[j] : szero<S>();
#pragma unroll
      for (int j = 0; j < NB; ++j) {
        if (j < kb) {
          S acc = w[j];
#pragma unroll
          for (int l = 0; l < j; ++l) acc = sfnms(w[l], lkk[j][l], acc);
          w[j] = acc;
        }
      }
#pragma unroll
      for (int j = 0; j < NB; ++j)
        if (j < kb) row[j] = smul(w[j], dinv[j]);
    }
    __syncthreads();
    // ---- 3. trailing update: A_ij -= sum_l L_il d_l L_jl, i >= j >= k0 + kb ----------------
    const int r0 = k0 + kb;
    const int mrows = n - r0;
    if (mrows <= 0) break;
    const int nt = (mrows + TT - 1) / TT;
    const int tx = tid & 15, ty = tid >> 4;
    for (int tI = 0; tI < nt; ++tI) {
      for (int tJ = 0; tJ <= tI; ++tJ) {
        const int i0 = r0 + tI * TT, j0 = r0 + tJ * TT;
        for (int e = tid; e < TT * NB; e += 256) {
          int rr = e / NB, l = e % NB;
          int gi = i0 + rr, gj = j0 + rr;
          S li = (gi < n && l < kb) ? A[(long long)gi * ldm + k0 + l] : szero<S>();
          S lj = (gj < n && l < kb) ? A[(long long)gj * ldm + k0 + l] : szero<S>();
          ws[l][rr] = (l < kb) ? smul(li, lkk[l][l]) : szero<S>();
          ls[l][rr] = lj;
        }
        __syncthreads();
        S acc[4][4];
#pragma unroll
        for (int a = 0; a < 4; ++a)
#pragma unroll
          for (int b = 0; b < 4; ++b) acc[a][b] = szero<S>();
#pragma unroll 4
        for (int l = 0; l < kb; ++l) {
          S wa[4], lb[4];
#pragma unroll
          for (int a = 0; a < 4; ++a) wa[a] = ws[l][ty + 16 * a];
#pragma unroll
          for (int b = 0; b < 4; ++b) lb[b] = ls[l][tx + 16 * b];
#pragma unroll
          for (int a = 0; a < 4; ++a)
#pragma unroll
            for (int b = 0; b < 4; ++b) acc[a][b] = sfnms(wa[a], lb[b], acc[a][b]);
        }
#pragma unroll
        for (int a = 0; a < 4; ++a)
#pragma unroll
          for (int b = 0; b < 4; ++b) {
            int gi = i0 + ty + 16 * a, gj = j0 + tx + 16 * b;
            if (gi < n && gj < n && gj <= gi) {
              S* p = A + (long long)gi * ldm + gj;
              *p = sadd(*p, acc[a][b]);
            }
          }
        __syncthreads();
      }
    }
  }
  __syncthreads();
  if (tid == 0 && sing) atomicOr(status, kStatSingular);
}

// Forward substitution y = L^-1 b for a block of RB right-hand sides (in place), then
// w_q = sum_i y_i^2 / d_i - |b_q|^2.  Grid: (matrix f, RHS block).
constexpr int RB = 32;

template <typename S>
__global__ void __launch_bounds__(256) ldlt_solve_kernel(const S* __restrict__ mats, int n, long long ldm, long long stride,
                                                          S* __restrict__ rhs, int r, long long ldr, long long rhs_stride,
                                                          const double* __restrict__ bnorm2, double* __restrict__ w,
                                                          long long w_stride, const int* __restrict__ active) {
  const int f = blockIdx.x;
  if (active && !active[f]) return;
  const int q0 = blockIdx.y * RB;
  const int nq = min(RB, r - q0);
  const S* L = mats + f * stride;
  S* Y = rhs + f * rhs_stride + (long long)q0 * ldr;
  const int tid = threadIdx.x;

  extern __shared__ __align__(16) unsigned char smem_raw[];
  S(*ls)[NB + 1] = reinterpret_cast<S(*)[NB + 1]>(smem_raw);                             // L[k0+i][l0+l]
  S(*ys)[RB + 1] = reinterpret_cast<S(*)[RB + 1]>(smem_raw + sizeof(S) * NB * (NB + 1));  // y[l0+l][q]
  S(*accs)[RB + 1] = ys + NB;                                                              // panel partial sums

  const int ii = tid & 31, qg = tid >> 5;  // row in panel, group of 4 rhs
  for (int k0 = 0; k0 < n; k0 += NB) {
    const int kb = min(NB, n - k0);
    S acc[4];
#pragma unroll
    for (int u = 0; u < 4; ++u) acc[u] = szero<S>();
    for (int l0 = 0; l0 < k0; l0 += NB) {
      for (int e = tid; e < NB * NB; e += 256) {
        int i = e / NB, l = e % NB;
        ls[i][l] = (i < kb) ? L[(long long)(k0 + i) * ldm + l0 + l] : szero<S>();
      }
      for (int e = tid; e < NB * RB; e += 256) {
        int q = e / NB, l = e % NB;
        ys[l][q] = (q < nq) ? Y[(long long)q * ldr + l0 + l] : szero<S>();
      }
      __syncthreads();
#pragma unroll 8
      for (int l = 0; l < NB; ++l) {
        S a = ls[ii][l];
#pragma unroll
        for (int u = 0; u < 4; ++u) acc[u] = sfnms(a, ys[l][qg * 4 + u], acc[u]);
      }
      __syncthreads();
    }
#pragma unroll
    for (int u = 0; u < 4; ++u) accs[ii][qg * 4 + u] = acc[u];
    // diagonal block of the panel
    for (int e = tid; e < NB * NB; e += 256) {
      int i = e / NB, l = e % NB;
      ls[i][l] = (i < kb && l < i) ? L[(long long)(k0 + i) * ldm + k0 + l] : szero<S>();
    }
    __syncthreads();
    if (tid < nq) {
      const int q = tid;
      S* y = Y + (long long)q * ldr + k0;
      for (int i = 0; i < kb; ++i) {
        S v = sadd(y[i], accs[i][q]);
        for (int l = 0; l < i; ++l) v = sfnms(ls[i][l], ys[l][q], v);
        ys[i][q] = v;
        y[i] = v;
      }
    }
    __syncthreads();
  }
  // w_q = sum_i y_i^2 / d_i - |b|^2  (FP64 accumulation)
  for (int q = 0; q < nq; ++q) {
    double sr = 0.0, si = 0.0;
    const S* y = Y + (long long)q * ldr;
    for (int i = tid; i < n; i += 256) {
      S yi = y[i];
      S t = smul(smul(yi, yi), sinv(L[(long long)i * ldm + i]));
      sr += sre(t);
      si += sim(t);
    }
    for (int o = 16; o > 0; o >>= 1) {
      sr += __shfl_down_sync(0xffffffffu, sr, o);
      si += __shfl_down_sync(0xffffffffu, si, o);
    }
    __shared__ double red[2][8];
    if ((tid & 31) == 0) {
      red[0][tid >> 5] = sr;
      red[1][tid >> 5] = si;
    }
    __syncthreads();
    if (tid == 0) {
      double a = 0.0, b = 0.0;
      for (int u = 0; u < 8; ++u) {
        a += red[0][u];
        b += red[1][u];
      }
      double* o = w + f * w_stride + (long long)(q0 + q) * 2;
      o[0] = a - bnorm2[(long long)f * r + q0 + q];
      o[1] = b;
    }
    __syncthreads();
  }
}

template <typename S>
size_t ldlt_smem() {
  return sizeof(S) * (NB * (NB + 1) + NB + 2 * NB * (TT + 1));
}
template <typename S>
size_t solve_smem() {
  return sizeof(S) * (NB * (NB + 1) + 2 * NB * (RB + 1));
}

template <typename S>
int run_ldlt(S* mats, int n, long long ldm, long long stride, int F, const int* active, unsigned* status, cudaStream_t s) {
  static bool attr = false;
  size_t sm = ldlt_smem<S>();
  if (!attr) {
    if (cudaFuncSetAttribute(ldlt_kernel<S>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm) != cudaSuccess) return -1;
    attr = true;
  }
  ldlt_kernel<S><<<F, 256, sm, s>>>(mats, n, ldm, stride, active, status);
  return cudaPeekAtLastError() == cudaSuccess ? 1 : -1;
}

template <typename S>
int run_solve(const S* mats, int n, long long ldm, long long stride, S* rhs, int r, long long ldr, long long rhs_stride,
              const double* bnorm2, int F, double* w, long long w_stride, const int* active, cudaStream_t s) {
  static bool attr = false;
  size_t sm = solve_smem<S>();
  if (!attr) {
    if (cudaFuncSetAttribute(ldlt_solve_kernel<S>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm) != cudaSuccess)
      return -1;
    attr = true;
  }
  dim3 g(F, (r + RB - 1) / RB);
  ldlt_solve_kernel<S><<<g, 256, sm, s>>>(mats, n, ldm, stride, rhs, r, ldr, rhs_stride, bnorm2, w, w_stride, active);
  return cudaPeekAtLastError() == cudaSuccess ? 1 : -1;
}

}  // namespace

int launch_ldlt(MatKind kind, void* mats, int n, long long ldm, long long stride, int F, const int* active,
                unsigned* status, cudaStream_t s) {
  switch (kind) {
    case MatKind::RealF32: return run_ldlt((float*)mats, n, ldm, stride, F, active, status, s);
    case MatKind::CplxF32: return run_ldlt((float2*)mats, n, ldm, stride, F, active, status, s);
    case MatKind::RealF64: return run_ldlt((double*)mats, n, ldm, stride, F, active, status, s);
    default: return run_ldlt((double2*)mats, n, ldm, stride, F, active, status, s);
  }
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
