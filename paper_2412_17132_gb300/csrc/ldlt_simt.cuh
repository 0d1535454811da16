// Blocked SIMT pieces of the complex-symmetric LDL^T (no pivoting), shared by the SIMT kernel
// and the tensor-core kernel: sub-panel factorisation (32 x 32 diagonal block in shared memory,
// then one thread per row solving against it) and the tiled rank-k update of a region of the
// lower triangle. Both run on warps 0-7 (256 threads) and synchronise with named barrier 1.
//
// Storage (matrix [nrow][ldm], row-major): strictly lower W = L D, diagonal d, strictly upper
// L^T; rows n..nrow-1 are appended right-hand sides (lower part only).
#pragma once
#include "gwc_internal.h"

namespace gwc {
namespace {

constexpr int NB = 32;   // sub-panel width (diagonal block)
constexpr int PW = 64;   // panel width
constexpr int TT = 64;   // trailing tile
constexpr int KC = 32;   // staged K chunk

constexpr int kSimtThreads = 256;  // threads of the blocked SIMT routines (warps 0-7 of the CTA)

// Barrier over warps 0-7 only (named barrier 1), so a CTA may carry further warps with other roles.
__device__ __forceinline__ void grp_sync() { asm volatile("bar.sync 1, 256;" ::: "memory"); }

__device__ __forceinline__ void cp_async16(void* dst, const void* src, bool valid) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(static_cast<uint32_t>(__cvta_generic_to_shared(dst))),
               "l"(src), "r"(valid ? 16 : 0)
               : "memory");
}
__device__ __forceinline__ void cp_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_wait() {
  asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory");
}

// Shared-memory layout of the factor kernel (element type S):
//   lkk [NB][NB+1], dinv [NB], then 2 stages of { X [TT][KC + PADX], Y [KC][TT] }, then the
//   prefetched target tile C [TT][TT] of the read-modify-write
template <typename S>
struct FactorSmem {
  static constexpr int PADX = 16 / (int)sizeof(S);
  static constexpr int XS = TT * (KC + PADX);
  static constexpr int YS = KC * TT;
  static constexpr int STAGE = XS + YS;
  static constexpr int CS = TT * TT;
  static constexpr size_t LKK_BYTES = ((sizeof(S) * (NB * (NB + 1) + NB)) + 15) / 16 * 16;
  static constexpr size_t bytes() { return LKK_BYTES + sizeof(S) * (2 * STAGE + CS); }
};

// A[i][j] -= sum_{l in [k0, k0+klen)} W[i][l] L[j][l] for rows [r0, n), columns [c0, c1), j <= i
// (n counts every row, including appended right-hand-side rows; c1 never exceeds the factored
// columns). W is read from the lower part (row i), L from the upper part (row l, column j).
template <typename S>
__device__ void update_region(S* __restrict__ A, int n, long long ldm, int r0, int c0, int c1, int k0, int klen,
                              S* __restrict__ stages) {
  using SM = FactorSmem<S>;
  constexpr int PER = 16 / (int)sizeof(S);  // elements per 16-byte copy
  const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
  const int n_ti = (n - r0 + TT - 1) / TT;
  const int nk = (klen + KC - 1) / KC;
  // tiles (tI, tJ): row tile i0 = r0 + TT*tI, column tile j0 = c0 + TT*tJ with j0 <= i0 + TT - 1;
  // every row tile has at least one column tile because c0 == r0 or c1 - c0 <= TT.
  auto cnt_of = [&](int tI) {
    const int jmax = min(c1, r0 + TT * tI + TT);
    return jmax > c0 ? (jmax - c0 + TT - 1) / TT : 0;
  };
  int n_tiles = 0;
  for (int tI = 0; tI < n_ti; ++tI) n_tiles += cnt_of(tI);
  const int total = n_tiles * nk;
  if (total == 0) return;

  struct It {
    int tI, tJ, cnt, chunk;
  };
  auto advance = [&](It& it) {
    if (++it.chunk == nk) {
      it.chunk = 0;
      if (++it.tJ == it.cnt) {
        it.tJ = 0;
        ++it.tI;
        it.cnt = it.tI < n_ti ? cnt_of(it.tI) : 0;
      }
    }
  };

  S* Cs = stages + 2 * SM::STAGE;  // target tile, prefetched with the tile's last chunk (nk > 1)
  auto issue = [&](const It& it, S* buf) {
    const int i0 = r0 + TT * it.tI, j0 = c0 + TT * it.tJ;
    const int kc = k0 + it.chunk * KC;
    S* X = buf;
    S* Y = buf + SM::XS;
    if (nk > 1 && it.chunk == nk - 1) {
      // C[ii][jj] = A[i0+ii][j0+jj]; the previous tile's read-modify-write is complete (it ended
      // before this tile's first chunk was computed), so the single buffer is free
      constexpr int CPR = TT / PER;
      for (int e = tid; e < TT * CPR; e += kSimtThreads) {
        const int ii = e / CPR, jj = (e % CPR) * PER;
        const int gi = i0 + ii, gj = j0 + jj;
        const bool ok = gi < n && gj < c1;
        const S* src = ok ? A + (long long)gi * ldm + gj : A;
        cp_async16(Cs + ii * TT + jj, src, ok);
      }
    }
    // X[ii][l] = A[i0+ii][kc+l]   (TT rows x KC, 16-byte pieces along l)
    constexpr int XPR = KC / PER;  // pieces per row
    for (int e = tid; e < TT * XPR; e += kSimtThreads) {
      const int ii = e / XPR, l = (e % XPR) * PER;
      const int gi = i0 + ii;
      const bool ok = gi < n && (kc + l) < k0 + klen;
      const S* src = ok ? A + (long long)gi * ldm + kc + l : A;
      cp_async16(X + ii * (KC + SM::PADX) + l, src, ok);
    }
    // Y[l][jj] = A[kc+l][j0+jj]  (upper part: L^T rows), 16-byte pieces along jj
    constexpr int YPR = TT / PER;
    for (int e = tid; e < KC * YPR; e += kSimtThreads) {
      const int l = e / YPR, jj = (e % YPR) * PER;
      const int gj = j0 + jj;
      const bool ok = (kc + l) < k0 + klen && gj < c1;
      const S* src = ok ? A + (long long)(kc + l) * ldm + gj : A;
      cp_async16(Y + l * TT + jj, src, ok);
    }
  };

  S acc[4][4];
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int b = 0; b < 4; ++b) acc[a][b] = szero<S>();

  It it_issue{0, 0, cnt_of(0), 0};
  It it_comp = it_issue;
  issue(it_issue, stages);
  cp_commit();
  advance(it_issue);
  for (int s = 0; s < total; ++s) {
    S* buf = stages + (s & 1) * SM::STAGE;
    if (s + 1 < total) {
      issue(it_issue, stages + ((s + 1) & 1) * SM::STAGE);
      cp_commit();
      advance(it_issue);
      cp_wait<1>();
    } else {
      cp_wait<0>();
    }
    grp_sync();
    const int kc = k0 + it_comp.chunk * KC;
    const int lmax = min(KC, k0 + klen - kc);
    const S* X = buf;
    const S* Y = buf + SM::XS;
#pragma unroll 4
    for (int l = 0; l < lmax; ++l) {
      S xa[4], yb[4];
#pragma unroll
      for (int a = 0; a < 4; ++a) xa[a] = X[(ty + 16 * a) * (KC + SM::PADX) + l];
#pragma unroll
      for (int b = 0; b < 4; ++b) yb[b] = Y[l * TT + tx + 16 * b];
#pragma unroll
      for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int b = 0; b < 4; ++b) acc[a][b] = sfnms(xa[a], yb[b], acc[a][b]);
    }
    if (it_comp.chunk == nk - 1) {
      const int i0 = r0 + TT * it_comp.tI, j0 = c0 + TT * it_comp.tJ;
#pragma unroll
      for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int b = 0; b < 4; ++b) {
          const int gi = i0 + ty + 16 * a, gj = j0 + tx + 16 * b;
          if (gi < n && gj < c1 && gj <= gi) {
            S* p = A + (long long)gi * ldm + gj;
            const S c = nk > 1 ? Cs[(ty + 16 * a) * TT + tx + 16 * b] : *p;
            *p = sadd(c, acc[a][b]);
          }
          acc[a][b] = szero<S>();
        }
    }
    advance(it_comp);
    grp_sync();
  }
}

// Factor the NB-wide sub-panel starting at column c0 (its columns already hold the Schur
// complement): diagonal block, then W (lower) and L^T (upper) for the rows below.
template <typename S>
__device__ void factor_subpanel(S* __restrict__ A, int n, int nrow, long long ldm, int c0, S (*lkk)[NB + 1], S* dinv,
                                int& sing) {
  const int tid = threadIdx.x;
  const int kb = min(NB, n - c0);
  grp_sync();
  for (int e = tid; e < NB * NB; e += kSimtThreads) {
    const int i = e / NB, j = e % NB;
    lkk[i][j] = (i < kb && j <= i) ? A[(long long)(c0 + i) * ldm + (c0 + j)] : szero<S>();
  }
  grp_sync();
  for (int j = 0; j < kb; ++j) {
    S d = lkk[j][j];
    if (sabs2(d) < 1e-60) {
      if (tid == 0) sing = 1;
      d = sfrom<S>(1.0, 0.0);
    }
    const S inv = sinv(d);
    const int m = kb - 1 - j;
    for (int e = tid; e < m * m; e += kSimtThreads) {
      const int i = j + 1 + e / m, l = j + 1 + e % m;
      if (l <= i) lkk[i][l] = sfnms(smul(lkk[i][j], inv), lkk[l][j], lkk[i][l]);
    }
    grp_sync();
    if (tid == 0) {
      lkk[j][j] = d;
      dinv[j] = inv;
    }
    for (int i = j + 1 + tid; i < kb; i += kSimtThreads) lkk[i][j] = smul(lkk[i][j], inv);
    grp_sync();
  }
  // diagonal block: W = L d below the diagonal, d on it, L^T above it
  for (int e = tid; e < kb * kb; e += kSimtThreads) {
    const int i = e / kb, j = e % kb;
    if (j < i) {
      A[(long long)(c0 + i) * ldm + (c0 + j)] = smul(lkk[i][j], lkk[j][j]);
      A[(long long)(c0 + j) * ldm + (c0 + i)] = lkk[i][j];
    } else if (j == i) {
      A[(long long)(c0 + i) * ldm + (c0 + i)] = lkk[i][i];
    }
  }
  // rows below: w = a L_kk^-T (= W row), L row = w D^-1
  for (int i = c0 + kb + tid; i < nrow; i += kSimtThreads) {
    S w[NB];
    S* row = A + (long long)i * ldm + c0;
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
      if (j < kb) {
        row[j] = w[j];
        if (i < n) A[(long long)(c0 + j) * ldm + i] = smul(w[j], dinv[j]);
      }
  }
  grp_sync();
}

}  // namespace
}  // namespace gwc
