// Blocked SIMT pieces of the complex-symmetric LDL^T (no pivoting), shared by the SIMT kernel
// and the tensor-core kernel: the 64-wide panel factorisation (two 32 x 32 diagonal blocks in
// shared memory, then one thread per row solving against both) and the tiled rank-k update of a
// region of the lower triangle. Both run on warps 0-7 (256 threads) and synchronise with named barrier 1.
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
// element-sized asynchronous copy (4, 8 or 16 bytes)
template <int BYTES>
__device__ __forceinline__ void cp_async_elem(void* dst, const void* src) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], %2;" ::"r"(static_cast<uint32_t>(__cvta_generic_to_shared(dst))),
               "l"(src), "n"(BYTES)
               : "memory");
}
__device__ __forceinline__ void cp_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_wait() {
  asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory");
}

// Shared memory of the tiled update (element type S): 2 stages of { X [TT][KC + PADX], Y [KC][TT] },
// then the prefetched target tile C [TT][TT] of the read-modify-write
template <typename S>
struct FactorSmem {
  static constexpr int PADX = 16 / (int)sizeof(S);
  static constexpr int XS = TT * (KC + PADX);
  static constexpr int YS = KC * TT;
  static constexpr int STAGE = XS + YS;
  static constexpr int CS = TT * TT;
  static constexpr size_t bytes() { return sizeof(S) * (2 * STAGE + CS); }
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

// Barrier over the first NT threads of the CTA (named barrier 1).
template <int NT>
__device__ __forceinline__ void grp_sync_n() {
  asm volatile("bar.sync 1, %0;" ::"n"(NT) : "memory");
}

// Shared memory of the panel factorisation (NT threads): the two diagonal blocks (factored in
// place: unit L below the diagonal, d on it), their inverse pivots, W / L of the second block's
// rows against the first block (for the Schur complement of the second block), and per-thread row
// scratch.
template <typename S, int NT>
struct PanelSmem {
  S (*lkk1)[NB + 1];
  S (*lkk2)[NB + 1];
  S (*w1s)[NB + 1];
  S (*l1s)[NB + 1];
  S* dinv1;
  S* dinv2;
  S* arow;  // [NB][NT]: block-2 part of each thread's current row
  static constexpr size_t bytes() { return sizeof(S) * (4 * NB * (NB + 1) + 2 * NB + NB * NT); }
  __device__ explicit PanelSmem(void* base) {
    S* p = reinterpret_cast<S*>(base);
    lkk1 = reinterpret_cast<S(*)[NB + 1]>(p);
    lkk2 = reinterpret_cast<S(*)[NB + 1]>(p + NB * (NB + 1));
    w1s = reinterpret_cast<S(*)[NB + 1]>(p + 2 * NB * (NB + 1));
    l1s = reinterpret_cast<S(*)[NB + 1]>(p + 3 * NB * (NB + 1));
    dinv1 = p + 4 * NB * (NB + 1);
    dinv2 = dinv1 + NB;
    arow = dinv2 + NB;
  }
};

// In-place LDL^T of the kb x kb block held (lower triangle) in lkk, by one warp (lane i owns row
// i; no block-wide barrier per column); a zero pivot is replaced by 1 and flagged.
template <typename S>
__device__ void factor_diag_warp(S (*lkk)[NB + 1], S* dinv, int kb, int& sing) {
  const int i = threadIdx.x & 31;
  for (int j = 0; j < kb; ++j) {
    __syncwarp();
    S d = lkk[j][j];
    const bool zero = sabs2(d) < 1e-60;
    if (zero) d = sfrom<S>(1.0, 0.0);
    const S inv = sinv(d);
    S lij = szero<S>();
    if (i > j && i < kb) {
      // row i of the Schur complement: a_il -= (a_ij / d_j) a_lj for j < l <= i (column j unscaled)
      lij = smul(lkk[i][j], inv);
      for (int l = j + 1; l <= i; ++l) lkk[i][l] = sfnms(lij, lkk[l][j], lkk[i][l]);
    }
    __syncwarp();
    if (i > j && i < kb) lkk[i][j] = lij;
    if (i == j) {
      lkk[j][j] = d;
      dinv[j] = inv;
      if (zero) sing = 1;
    }
  }
  __syncwarp();
}

// diagonal block at (c0, c0): W = L d below the diagonal, d on it, L^T above it
template <typename S, int NT>
__device__ void store_diag(S* __restrict__ A, long long ldm, int c0, int kb, S (*lkk)[NB + 1]) {
  for (int e = threadIdx.x; e < kb * kb; e += NT) {
    const int i = e / kb, j = e % kb;
    if (j < i) {
      A[(long long)(c0 + i) * ldm + (c0 + j)] = smul(lkk[i][j], lkk[j][j]);
      A[(long long)(c0 + j) * ldm + (c0 + i)] = lkk[i][j];
    } else if (j == i) {
      A[(long long)(c0 + i) * ldm + (c0 + i)] = lkk[i][i];
    }
  }
}

// w <- w L_kk^-T (unit lower L of the factored block): the W values of one row (two partial
// sums per element to halve the dependent FMA chain)
template <typename S>
__device__ __forceinline__ void solve_row(S (&w)[NB], S (*lkk)[NB + 1], int kb) {
#pragma unroll
  for (int j = 0; j < NB; ++j) {
    if (j < kb) {
      S a0 = w[j], a1 = szero<S>();
#pragma unroll
      for (int l = 0; l + 1 < j; l += 2) {
        a0 = sfnms(w[l], lkk[j][l], a0);
        a1 = sfnms(w[l + 1], lkk[j][l + 1], a1);
      }
      if (j & 1) a0 = sfnms(w[j - 1], lkk[j][j - 1], a0);
      w[j] = sadd(a0, a1);
    }
  }
}

// Factor the panel [k0, k0 + min(PW, n - k0)) (its columns already hold the Schur complement) as
// two NB-wide halves, on the first NT threads: the diagonal blocks in shared memory (one warp each),
// then every row below in one pass by one thread: solve against block 1, apply block 1 to its
// block-2 columns, solve against block 2, and store W (lower) and L^T (upper). Rows >= n are
// appended right-hand sides (W only).
template <typename S, int NT>
__device__ void factor_panel(S* __restrict__ A, int n, int nrow, long long ldm, int k0, const PanelSmem<S, NT>& ps,
                             int& sing) {
  const int tid = threadIdx.x;
  const int kb = min(PW, n - k0);
  const int kb1 = min(NB, kb), kb2 = kb - kb1;
  const int c2 = k0 + NB;
  grp_sync_n<NT>();
  for (int e = tid; e < NB * NB; e += NT) {
    const int i = e / NB, j = e % NB;
    ps.lkk1[i][j] = (i < kb1 && j <= i) ? A[(long long)(k0 + i) * ldm + (k0 + j)] : szero<S>();
  }
  grp_sync_n<NT>();
  if (tid < 32) factor_diag_warp(ps.lkk1, ps.dinv1, kb1, sing);
  grp_sync_n<NT>();
  store_diag<S, NT>(A, ldm, k0, kb1, ps.lkk1);
  if (kb2 > 0) {
    // rows of block 2 against block 1
    for (int r = tid; r < kb2; r += NT) {
      const int i = c2 + r;
      S* row = A + (long long)i * ldm + k0;
      S w[NB];
#pragma unroll
      for (int j = 0; j < NB; ++j) w[j] = j < kb1 ? row[j] : szero<S>();
      solve_row(w, ps.lkk1, kb1);
#pragma unroll
      for (int j = 0; j < NB; ++j) {
        const S l = smul(w[j], ps.dinv1[j]);
        row[j] = w[j];
        A[(long long)(k0 + j) * ldm + i] = l;
        ps.w1s[r][j] = w[j];
        ps.l1s[r][j] = l;
      }
    }
    grp_sync_n<NT>();
    // Schur complement of block 2
    for (int e = tid; e < NB * NB; e += NT) {
      const int r = e / NB, c = e % NB;
      S v = szero<S>();
      if (r < kb2 && c <= r) {
        v = A[(long long)(c2 + r) * ldm + (c2 + c)];
#pragma unroll 8
        for (int j = 0; j < NB; ++j) v = sfnms(ps.w1s[r][j], ps.l1s[c][j], v);
      }
      ps.lkk2[r][c] = v;
    }
    grp_sync_n<NT>();
    if (tid < 32) factor_diag_warp(ps.lkk2, ps.dinv2, kb2, sing);
    grp_sync_n<NT>();
    store_diag<S, NT>(A, ldm, c2, kb2, ps.lkk2);
  }
  // every row below the panel
  for (int i = k0 + kb + tid; i < nrow; i += NT) {
    S* row = A + (long long)i * ldm + k0;
    // block-2 values of the row into this thread's scratch, in flight while block 1 is solved
    S* as = ps.arow + tid;
    for (int c = 0; c < kb2; ++c) cp_async_elem<(int)sizeof(S)>(as + c * NT, row + NB + c);
    cp_commit();
    S w[NB];
#pragma unroll
    for (int j = 0; j < NB; ++j) w[j] = j < kb1 ? row[j] : szero<S>();
    solve_row(w, ps.lkk1, kb1);
#pragma unroll
    for (int j = 0; j < NB; ++j)
      if (j < kb1) {
        row[j] = w[j];
        if (i < n) A[(long long)(k0 + j) * ldm + i] = smul(w[j], ps.dinv1[j]);
      }
    if (kb2 > 0) {
      // block-2 columns: a = (row - L1 w) L_22^-T, one column at a time; a is kept per thread in
      // shared memory (column-major over the threads: conflict-free) so w stays in registers
      cp_wait<0>();
#pragma unroll 1
      for (int c = 0; c < kb2; ++c) {
        S v0 = as[c * NT], v1 = szero<S>(), v2 = szero<S>(), v3 = szero<S>();
#pragma unroll
        for (int j = 0; j < NB; j += 4) {
          v0 = sfnms(w[j], ps.l1s[c][j], v0);
          v1 = sfnms(w[j + 1], ps.l1s[c][j + 1], v1);
          v2 = sfnms(w[j + 2], ps.l1s[c][j + 2], v2);
          v3 = sfnms(w[j + 3], ps.l1s[c][j + 3], v3);
        }
        int l = 0;
        for (; l + 1 < c; l += 2) {
          v0 = sfnms(as[l * NT], ps.lkk2[c][l], v0);
          v1 = sfnms(as[(l + 1) * NT], ps.lkk2[c][l + 1], v1);
        }
        if (l < c) v2 = sfnms(as[l * NT], ps.lkk2[c][l], v2);
        const S v = sadd(sadd(v0, v1), sadd(v2, v3));
        as[c * NT] = v;
        row[NB + c] = v;
        if (i < n) A[(long long)(c2 + c) * ldm + i] = smul(v, ps.dinv2[c]);
      }
    }
  }
  grp_sync_n<NT>();
}

}  // namespace
}  // namespace gwc
