// Tensor-core LDL^T of complex-symmetric FP32 dielectric matrices (sm_103a: tcgen05 + TMEM).
//
// Same factorisation, storage and panel order as the SIMT kernel (eps = L D L^T without pivoting;
// W = L D below the diagonal, d on it, L^T above it; appended rows n..nrow-1 become L^-1 b), with
// the rank-64 trailing update of every panel moved to the tensor cores:
//
//   C[i][j] -= sum_l W[i][l] L[j][l],   l in the panel, i >= j beyond the panel.
//
// Complex products as real GEMMs over split planes. With A = W rows (Ar, Ai) and B = L rows
// (Lr, Li) stored as the 128-row window [Lr ; Li], two accumulators of N = 128 columns take
//     P = Ar [Lr ; Li]^T = [Ar Lr^T | Ar Li^T],   Q = Ai [Lr ; Li]^T = [Ai Lr^T | Ai Li^T],
// and the epilogue forms Re = Ar Lr^T - Ai Li^T and Im = Ar Li^T + Ai Lr^T from them (N = 128 MMAs
// run at full rate; N = 64 ones at about 60 %).
//
// FP32 accuracy from TF32 operands (kind::tf32): every value v is split into hi = tf32(v) and
// lo = tf32(v - hi) (3xTF32; Henry, Tang & Heinecke 2019 for the BF16 analogue): each accumulator
// takes hi*hi + hi*lo + lo*hi, and the epilogue forms C - (P and Q terms) in round-to-nearest FP32.
//
// Roles (416 threads, one CTA per matrix):
//   warps 0-11  panel factorisation (factor_panel_tc below, named barrier 1)
//   warps 4-7   operand transform: global memory (L2) -> hi/lo planes in the 128-byte-swizzled
//               K-major layout. The A operand (W rows of a 128-row tile, all 64 panel columns)
//               stays resident while the tile row's column tiles pass; the B operand (L rows of a
//               64-column tile) streams through two stages of 32 panel columns, the global loads
//               of a stage issued before the wait for its buffer.
//   warp 12     TMEM allocation (512 columns: two tiles in flight x {D1, D2}) and the MMA issuer
//   warps 0-3,  epilogue: one thread per tile row and half of the tile's columns, the target values
//   8-11        read and written with 16-byte accesses, the next chunk's values loaded ahead
// The panel scratch aliases the operand buffers (the phases alternate).
// Every mbarrier wait is bounded (one second); on expiry the CTA records kStatTimeout, stops,
// drains the MMAs it issued and frees TMEM.
#include <algorithm>
#include <cstring>

#include "gwc_internal.h"
#include "ldlt_simt.cuh"
#include "tc_common.cuh"

namespace gwc {

namespace {

constexpr int TM = 128;                                  // rows per trailing tile (MMA M)
constexpr int TN = 64;                                   // complex columns per tile (MMA N per part)
constexpr int KH = 32;                                   // panel columns per stage (128-byte plane rows)
constexpr int A_PLANE = TM * 128;                        // 16 KB: [half][Ar, Ai, Ar_lo, Ai_lo]
constexpr int A_BYTES = 8 * A_PLANE;                     // 128 KB: the resident A operand
constexpr int B_PLANE = TN * 128;                        // 8 KB: Lr, Li, Lr_lo, Li_lo
constexpr int B_STAGE = 4 * B_PLANE;                     // 32 KB
constexpr int NSTAGE = 2;
constexpr int NT_TC = 416;                               // 13 warps
constexpr int MMA_WARP = 12;
constexpr int N_EPI = 256;                               // epilogue threads (warps 0-3, 8-11)
constexpr int META_BYTES = 128;
constexpr int OPS_BYTES = A_BYTES + NSTAGE * B_STAGE;    // 192 KB
constexpr int SMEM_TC = 1024 + OPS_BYTES + META_BYTES;
static_assert(PW == 2 * KH, "one panel is two stages");
constexpr int NT_PANEL = 384;                            // warps 0-11 factor the panels

// kind::tf32 instruction descriptor: D = F32, A = B = TF32, both K-major, N = 2 TN, M = TM.
constexpr uint32_t kIdescTf32 =
    (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(2 * TN >> 3) << 17) | ((uint32_t)(TM >> 4) << 24);

__device__ __forceinline__ void mma_tf32(uint32_t d_tmem, uint64_t a, uint64_t b, uint32_t accum) {
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "setp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}" ::"r"(d_tmem),
      "l"(a), "l"(b), "n"(kIdescTf32), "r"(accum));
}

// round to the nearest TF32 value (10 explicit mantissa bits), kept in an FP32 container
__device__ __forceinline__ float tf32_rn(float x) {
  uint32_t r;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
  return __uint_as_float(r);
}

__device__ __forceinline__ void split4(const float (&v)[4], float4& hi, float4& lo) {
  float h[4], l[4];
#pragma unroll
  for (int e = 0; e < 4; ++e) {
    h[e] = tf32_rn(v[e]);
    l[e] = tf32_rn(v[e] - h[e]);
  }
  hi = make_float4(h[0], h[1], h[2], h[3]);
  lo = make_float4(l[0], l[1], l[2], l[3]);
}

// ---- panel factorisation (warps 0-11) -----------------------------------------------------------
// The kb x kb diagonal block (kb <= 64) is factored right-looking by all 384 threads, one barrier per
// step, and the same kb steps form X = L^-1 of its unit lower factor. Every element (i, c <= i) of
// the lower triangle is owned by one thread and held in a register: while c > j it is the Schur
// complement entry, a_ic -= W_ij d_j^-1 W_cj, final after step c - 1 and then published to shared
// memory as W_ic (d_i on the diagonal); from step c on the same register accumulates
// X_ic -= l_ij X_jc (c <= j < i, X_jj = 1, l_ij = W_ij / d_j), published after step i - 1. Step j
// reads only column j of W and row j of X, both published before the barrier that opens it.
// The rows below then need no dependent chain: W_rows = A_rows X^T (a product over the panel
// columns, X^T upper triangular) and L^T_rows = (W_rows D^-1)^T.
struct PanelInv {
  static constexpr int LDP = PW + 1;                  // padded row (conflict-free column access)
  static constexpr int CH = 16 * (NT_PANEL / 32);     // 192 staged rows: 6 blocks of 32 x 2 group pairs
  float2 (*dm)[LDP];   // [64][65] W below the diagonal, d on it
  float2 (*xg)[PW];    // [64][64] xg[l][c] = X_cl (zero for c < l), 16-byte rows for broadcast loads
  float2* dinv;        // [64] 1 / d
  float2* dpiv;        // [64] d (a zero pivot replaced by 1)
  float2 (*xr)[LDP];   // [64][65] X by rows while the block is factored ...
  float2 (*ach)[LDP];  // [CH][65] ... then, aliased, the staged rows below the panel
  static constexpr size_t bytes() {
    return sizeof(float2) * ((size_t)PW * LDP + PW * PW + 2 * PW + (size_t)CH * LDP);
  }
  __device__ explicit PanelInv(void* base) {
    float2* p = reinterpret_cast<float2*>(base);
    dm = reinterpret_cast<float2(*)[LDP]>(p);
    p += PW * LDP;
    xg = reinterpret_cast<float2(*)[PW]>(p);
    p += PW * PW;
    dinv = p;
    dpiv = p + PW;
    p += 2 * PW;
    xr = reinterpret_cast<float2(*)[LDP]>(p);
    ach = reinterpret_cast<float2(*)[LDP]>(p);
  }
};
static_assert(PanelInv::bytes() <= (size_t)OPS_BYTES, "panel scratch fits in the operand buffers");
static_assert(PW * PW <= PanelInv::CH * PanelInv::LDP, "X by rows fits in the staging rows");

__device__ __forceinline__ void panel_sync() { grp_sync_n<NT_PANEL>(); }

// diagonal block [k0, k0 + kb): W / d / L^T stored to A; dinv and xg left in shared memory
__device__ void factor_diag_block(float2* __restrict__ A, long long ldm, int k0, int kb, const PanelInv& ps,
                                  int* sing) {
  constexpr int MAXS = (PW * (PW + 1) / 2 + NT_PANEL - 1) / NT_PANEL;
  const int tid = threadIdx.x;
  panel_sync();  // the previous phase's use of the scratch is over
  for (int e = tid; e < PW * PW; e += NT_PANEL) {
    const int i = e >> 6, c = e & 63;
    ps.dm[i][c] = (i < kb && c <= i) ? A[(long long)(k0 + i) * ldm + (k0 + c)] : make_float2(0.f, 0.f);
    ps.xr[i][c] = make_float2(i == c ? 1.f : 0.f, 0.f);
  }
  panel_sync();
  int si[MAXS], sc[MAXS];
  float2 v[MAXS];
  const int tot = kb * (kb + 1) / 2;
#pragma unroll
  for (int s = 0; s < MAXS; ++s) {
    const int e = tid + s * NT_PANEL;
    int i = -1, c = 0;
    if (e < tot) {
      i = (int)((sqrtf(8.f * (float)e + 1.f) - 1.f) * 0.5f);
      while (i * (i + 1) / 2 > e) --i;
      while ((i + 1) * (i + 2) / 2 <= e) ++i;
      c = e - i * (i + 1) / 2;
      v[s] = ps.dm[i][c];
    } else {
      v[s] = make_float2(0.f, 0.f);
    }
    si[s] = i;
    sc[s] = c;
  }
  for (int j = 0; j < kb; ++j) {
    float2 d = ps.dm[j][j];
    const bool zero = fabsf(d.x) + fabsf(d.y) < 1e-30f;
    if (zero) d = make_float2(1.f, 0.f);
    const float2 inv = sinv(d);
    if (tid == 0) {
      ps.dinv[j] = inv;
      ps.dpiv[j] = d;
      if (zero) *sing = 1;
    }
#pragma unroll
    for (int s = 0; s < MAXS; ++s) {
      const int i = si[s], c = sc[s];
      if (i > j) {
        const float2 wij = ps.dm[i][j];
        if (c > j) {
          v[s] = sfnms(wij, smul(inv, ps.dm[c][j]), v[s]);
          if (c == j + 1) ps.dm[i][c] = v[s];
        } else {
          if (c == j) v[s] = make_float2(0.f, 0.f);
          v[s] = sfnms(wij, smul(inv, ps.xr[j][c]), v[s]);
          if (i == j + 1) ps.xr[i][c] = v[s];
        }
      }
    }
    panel_sync();
  }
  for (int e = tid; e < PW * PW; e += NT_PANEL) {
    const int l = e >> 6, c = e & 63;
    ps.xg[l][c] = (c >= l && c < kb) ? ps.xr[c][l] : make_float2(0.f, 0.f);
  }
  for (int e = tid; e < kb * kb; e += NT_PANEL) {
    const int i = e / kb, c = e % kb;
    if (c < i) {
      const float2 w = ps.dm[i][c];
      A[(long long)(k0 + i) * ldm + (k0 + c)] = w;
      A[(long long)(k0 + c) * ldm + (k0 + i)] = smul(w, ps.dinv[c]);
    } else if (c == i) {
      A[(long long)(k0 + i) * ldm + (k0 + i)] = ps.dpiv[i];
    }
  }
  panel_sync();  // xg, dinv complete; xr may be overwritten by the staged rows
}

// One warp's share of a staged chunk: rows r0 .. r0 + 31 (one per lane), the 16 columns of group g,
// w_c = sum_{l <= c} a_l X_cl in packed FP32 pairs (re and im of X per product), then W (row-major,
// lower part) and L^T (transposed, coalesced over the lanes) stored.
__device__ __forceinline__ void panel_rows_group(float2* __restrict__ A, int n, long long ldm, int k0, int kb,
                                                 const PanelInv& ps, int r, int i, bool row_ok, int g) {
  const int cb = 16 * g, ncol = min(16, kb - cb);
  const float2* arow = ps.ach[r];
  float2* rowp = A + (long long)i * ldm + k0 + cb;
  // two passes of 8 columns (c0 = 0, 8): 16 float2 accumulators per pass keep the loop in registers
#pragma unroll 1
  for (int c0 = 0; c0 < 16; c0 += 8) {
    if (c0 >= ncol) break;
    const int lmax = min(cb + c0 + 8, kb);  // X_cl = 0 for l > c
    float2 pr[8], pi[8];  // pr[c] = sum a.re (X re, X im), pi[c] = sum a.im (X re, X im)
#pragma unroll
    for (int c = 0; c < 8; ++c) {
      pr[c] = make_float2(0.f, 0.f);
      pi[c] = make_float2(0.f, 0.f);
    }
#pragma unroll 4
    for (int l = 0; l < lmax; ++l) {
      const float2 a = arow[l];
      const float2 ar = make_float2(a.x, a.x), ai = make_float2(a.y, a.y);
      const float4* xp = reinterpret_cast<const float4*>(&ps.xg[l][cb + c0]);
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const float4 x = xp[q];
        const float2 x0 = make_float2(x.x, x.y), x1 = make_float2(x.z, x.w);
        pr[2 * q] = __ffma2_rn(ar, x0, pr[2 * q]);
        pi[2 * q] = __ffma2_rn(ai, x0, pi[2 * q]);
        pr[2 * q + 1] = __ffma2_rn(ar, x1, pr[2 * q + 1]);
        pi[2 * q + 1] = __ffma2_rn(ai, x1, pi[2 * q + 1]);
      }
    }
    if (!row_ok) continue;
    float2 w[8];
#pragma unroll
    for (int c = 0; c < 8; ++c) w[c] = make_float2(pr[c].x - pi[c].y, pr[c].y + pi[c].x);
    const int nc8 = min(8, ncol - c0);
    if (nc8 == 8) {
#pragma unroll
      for (int q = 0; q < 4; ++q)
        *reinterpret_cast<float4*>(rowp + c0 + 2 * q) = make_float4(w[2 * q].x, w[2 * q].y, w[2 * q + 1].x, w[2 * q + 1].y);
    } else {
#pragma unroll
      for (int c = 0; c < 8; ++c)
        if (c < nc8) rowp[c0 + c] = w[c];
    }
    if (i < n) {
#pragma unroll
      for (int c = 0; c < 8; ++c)
        if (c < nc8) A[(long long)(k0 + cb + c0 + c) * ldm + i] = smul(w[c], ps.dinv[cb + c0 + c]);
    }
  }
}

// Panel [k0, k0 + kb): the diagonal block, then every row below (appended right-hand-side rows
// n..nrow-1 included, W only) in chunks of CH staged rows; warp w takes the 32-row block w / 2 of a
// chunk and the column groups {0, 3} or {1, 2} (equal work: the triangle of X).
__device__ void factor_panel_tc(float2* __restrict__ A, int n, int nrow, long long ldm, int k0, const PanelInv& ps,
                                int* sing) {
  const int kb = min(PW, n - k0);
  factor_diag_block(A, ldm, k0, kb, ps, sing);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int r = 32 * (warp >> 1) + lane;
  const int g0 = (warp & 1) ? 1 : 0, g1 = (warp & 1) ? 2 : 3;
  for (int base = k0 + kb; base < nrow; base += PanelInv::CH) {
    for (int e = tid; e < PanelInv::CH * PW; e += NT_PANEL) {
      const int rr = e >> 6, l = e & 63, i = base + rr;
      if (i < nrow && l < kb) cp_async_elem<8>(&ps.ach[rr][l], A + (long long)i * ldm + k0 + l);
    }
    cp_commit();
    cp_wait<0>();
    panel_sync();
    const int i = base + r;
    const bool row_ok = i < nrow;
    if (base + 32 * (warp >> 1) < nrow) {  // warp-uniform: the block has rows
      if (16 * g0 < kb) panel_rows_group(A, n, ldm, k0, kb, ps, r, i, row_ok, g0);
      if (16 * g1 < kb) panel_rows_group(A, n, ldm, k0, kb, ps, r, i, row_ok, g1);
    }
    panel_sync();  // the staging rows are free
  }
}

// column tiles of row tile tI: j0 = R0 + TN tJ < min(n, i0 + TM)
__device__ __forceinline__ int tile_cols(int R0, int n, int tI) {
  const int jmax = min(n, R0 + TM * tI + TM);
  return (jmax - R0 + TN - 1) / TN;
}

struct TcSmem {
  uint8_t* base;  // A operand, then the B stages
  uint64_t *a_full, *a_empty, *b_full, *b_empty, *tfull, *tempty, *mma_done;
  uint32_t* tmem_slot;
  volatile int* abort_flag;
  int* sing;
  unsigned long long wait_ns;  // bound of every mbarrier wait
};

// Iterates the (row tile, column tile, half) stages of one panel in issue order.
struct StageIt {
  int R0, n, n_ti;
  int tI, tJ, h, nc;
  __device__ void init(int R0_, int n_, int n_ti_) {
    R0 = R0_;
    n = n_;
    n_ti = n_ti_;
    tI = 0;
    tJ = 0;
    h = 0;
    nc = tile_cols(R0, n, 0);
  }
  __device__ bool valid() const { return tI < n_ti; }
  __device__ void next() {
    if (++h == 2) {
      h = 0;
      if (++tJ == nc) {
        tJ = 0;
        ++tI;
        nc = tI < n_ti ? tile_cols(R0, n, tI) : 0;
      }
    }
  }
};

// B operand values of one stage for this thread: L^T[k0 + KH h + 16 lh + e][j0 + jj], e < 16
__device__ __forceinline__ void load_b(float2 (&bv)[16], const float2* A, int n, long long ldm, int k0,
                                       const StageIt& it, int tt) {
  const int jj = tt & 63, lh = tt >> 6, j = it.R0 + TN * it.tJ + jj;
  const bool jv = j < n;
  const float2* colp = A + (long long)(k0 + KH * it.h + 16 * lh) * ldm + (jv ? j : 0);
#pragma unroll
  for (int e = 0; e < 16; ++e) bv[e] = jv ? colp[(long long)e * ldm] : make_float2(0.f, 0.f);
}

// ---- operand transform (warps 4-7) --------------------------------------------------------------
// (A is written by this kernel: plain coherent loads, no read-only path)
__device__ void transform_role(const TcSmem& sm, const float2* A, int n, int nrow, long long ldm, int k0, int R0,
                               int n_ti, int seq, int rt) {
  const int tt = threadIdx.x - 128;  // 0..127
  StageIt it;
  it.init(R0, n, n_ti);
  float2 bv[16];
  load_b(bv, A, n, ldm, k0, it, tt);
  bool ok = true;
  for (int tI = 0; tI < n_ti && ok; ++tI, ++rt) {
    // A operand of row tile tI: W[i0 + row][k0 .. k0 + 64), four threads per row (64 bytes each)
    if (!mbar_wait(smem_u32(sm.a_empty), (rt & 1) ^ 1, sm.abort_flag, sm.wait_ns)) break;
    {
      const int rq = tt & 3, rr = tt >> 2;
      const int i0 = R0 + TM * tI;
#pragma unroll 1
      for (int hp = 0; hp < 4; ++hp) {  // (half, pair of row passes)
        const int h = hp >> 1;
        float4 av[8];
#pragma unroll
        for (int pp = 0; pp < 2; ++pp) {
          const int i = i0 + rr + 32 * (2 * (hp & 1) + pp);
          const float4* src =
              reinterpret_cast<const float4*>(A + (long long)(i < nrow ? i : 0) * ldm + k0 + KH * h + 8 * rq);
#pragma unroll
          for (int c = 0; c < 4; ++c) av[4 * pp + c] = i < nrow ? src[c] : make_float4(0.f, 0.f, 0.f, 0.f);
        }
#pragma unroll
        for (int pp = 0; pp < 2; ++pp) {
          const int r = rr + 32 * (2 * (hp & 1) + pp), sw = r & 7;
          uint8_t* rowp = sm.base + h * 4 * A_PLANE + r * 128;
#pragma unroll
          for (int e = 0; e < 2; ++e) {  // chunk 2 rq + e: complex l = 8 rq + 4 e .. + 3
            const float4 v0 = av[4 * pp + 2 * e], v1 = av[4 * pp + 2 * e + 1];
            const float re[4] = {v0.x, v0.z, v1.x, v1.z};
            const float im[4] = {v0.y, v0.w, v1.y, v1.w};
            float4 rh, rl, ih, il;
            split4(re, rh, rl);
            split4(im, ih, il);
            const int off = ((2 * rq + e) ^ sw) << 4;
            *reinterpret_cast<float4*>(rowp + off) = rh;
            *reinterpret_cast<float4*>(rowp + A_PLANE + off) = ih;
            *reinterpret_cast<float4*>(rowp + 2 * A_PLANE + off) = rl;
            *reinterpret_cast<float4*>(rowp + 3 * A_PLANE + off) = il;
          }
        }
      }
    }
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    mbar_arrive(smem_u32(sm.a_full));
    // B operand stages of this row tile
    const int nc = tile_cols(R0, n, tI);
    for (int q = 0; q < 2 * nc; ++q, ++seq) {
      const int s = seq & 1, us = seq >> 1;
      if (!mbar_wait(smem_u32(&sm.b_empty[s]), (us & 1) ^ 1, sm.abort_flag, sm.wait_ns)) {
        ok = false;
        break;
      }
      const int jj = tt & 63, lh = tt >> 6, sw = jj & 7;
      uint8_t* rowp = sm.base + A_BYTES + s * B_STAGE + jj * 128;
#pragma unroll
      for (int c = 0; c < 4; ++c) {
        float lr[4], li[4];
#pragma unroll
        for (int e = 0; e < 4; ++e) {
          lr[e] = bv[4 * c + e].x;
          li[e] = bv[4 * c + e].y;
        }
        float4 rh, rl, ih, il;
        split4(lr, rh, rl);
        split4(li, ih, il);
        const int off = ((4 * lh + c) ^ sw) << 4;
        *reinterpret_cast<float4*>(rowp + off) = rh;
        *reinterpret_cast<float4*>(rowp + B_PLANE + off) = ih;
        *reinterpret_cast<float4*>(rowp + 2 * B_PLANE + off) = rl;
        *reinterpret_cast<float4*>(rowp + 3 * B_PLANE + off) = il;
      }
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      mbar_arrive(smem_u32(&sm.b_full[s]));
      // the next stage's loads travel while this thread waits for that stage's buffer
      it.next();
      if (it.valid()) load_b(bv, A, n, ldm, k0, it, tt);
    }
  }
}

// ---- MMA issuer (one thread of warp 8) ----------------------------------------------------------
__device__ void mma_role(const TcSmem& sm, uint32_t tmem_base, int n, int R0, int n_ti, int seq, int tcount, int rt) {
  bool ok = true;
  const uint32_t abase = smem_u32(sm.base);
  for (int tI = 0; tI < n_ti && ok; ++tI, ++rt) {
    if (!mbar_wait(smem_u32(sm.a_full), rt & 1, sm.abort_flag, sm.wait_ns)) break;
    tc_fence_after();
    const int nc = tile_cols(R0, n, tI);
    for (int tJ = 0; tJ < nc && ok; ++tJ, ++tcount) {
      const int b = tcount & 1, ub = tcount >> 1;
      if (!mbar_wait(smem_u32(&sm.tempty[b]), (ub & 1) ^ 1, sm.abort_flag, sm.wait_ns)) {
        ok = false;
        break;
      }
      tc_fence_after();
      const uint32_t dp = tmem_base + (uint32_t)(b * 256), dq = dp + 128;  // P and Q accumulators
      for (int h = 0; h < 2; ++h, ++seq) {
        const int s = seq & 1, us = seq >> 1;
        if (!mbar_wait(smem_u32(&sm.b_full[s]), us & 1, sm.abort_flag, sm.wait_ns)) {
          ok = false;
          break;
        }
        tc_fence_after();
        const uint32_t ah = abase + h * 4 * A_PLANE;
        const uint32_t ar = ah, ai = ah + A_PLANE, arl = ah + 2 * A_PLANE, ail = ah + 3 * A_PLANE;
        const uint32_t bb = abase + A_BYTES + s * B_STAGE;
        const uint32_t br = bb, bi = bb + B_PLANE, brl = bb + 2 * B_PLANE, bil = bb + 3 * B_PLANE;
        // descriptors once per stage; a k step moves the start address by 32 bytes = 2 units of the
        // 16-byte address field (few instructions per MMA for the issuing thread)
        const uint64_t dar = sdesc(ar), dai = sdesc(ai), darl = sdesc(arl), dail = sdesc(ail);
        const uint64_t dbr = sdesc(br), dbi = sdesc(bi), dbrl = sdesc(brl), dbil = sdesc(bil);
#pragma unroll
        for (int k = 0; k < KH / 8; ++k) {
          const uint64_t o = 2u * k;  // 8 TF32 values = 32 bytes along K inside the 128-B row
          const uint32_t acc = (h == 0 && k == 0) ? 0u : 1u;
          const uint64_t a_r = dar + o, a_i = dai + o, a_rl = darl + o, a_il = dail + o;
          const uint64_t bh = dbr + o, bl = dbrl + o;  // [Lr ; Li] hi and lo windows (N = 128)
          mma_tf32(dp, a_r, bh, acc);
          mma_tf32(dp, a_r, bl, 1u);
          mma_tf32(dp, a_rl, bh, 1u);
          mma_tf32(dq, a_i, bh, acc);
          mma_tf32(dq, a_i, bl, 1u);
          mma_tf32(dq, a_il, bh, 1u);
        }
        mma_commit(smem_u32(&sm.b_empty[s]));
      }
      if (!ok) break;
      mma_commit(smem_u32(&sm.tfull[b]));
    }
    if (!ok) break;
    mma_commit(smem_u32(sm.a_empty));  // the row tile's A operand is free once its MMAs complete
  }
}

// ---- epilogue (warps 0-3 and 8-11): C -= D1 + D2 -----------------------------------------------
// Warp w serves TMEM lanes 32 (w % 4) .. +31 (rows of the tile) and, with its partner w ^ 8, half
// of the tile's 64 columns: two 16-column chunks. Each thread owns one row; the target values of
// its next chunk are loaded (16-byte loads) while the current one is formed.
// TMEM loads without the implicit wait, so the accumulator slices of a chunk share one wait
__device__ __forceinline__ void tmem_ld16_nw(uint32_t taddr, uint32_t (&r)[16]) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]),
        "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
      : "r"(taddr));
}

// this thread's chunks in issue order: (row tile, column tile, chunk cc0 or cc0 + 1)
struct ChunkIt {
  int R0, n, nrow, n_ti, r, cc0;
  int tI, tJ, cc, nc, i, jlim;
  __device__ void set_row() {
    i = R0 + TM * tI + r;
    jlim = i < nrow ? (i < n ? min(n, i + 1) : n) : 0;  // j <= i inside the factored block
  }
  __device__ void init(int R0_, int n_, int nrow_, int n_ti_, int r_, int cc0_) {
    R0 = R0_;
    n = n_;
    nrow = nrow_;
    n_ti = n_ti_;
    r = r_;
    cc0 = cc0_;
    tI = 0;
    tJ = 0;
    cc = cc0;
    nc = tile_cols(R0, n, 0);
    set_row();
  }
  __device__ bool valid() const { return tI < n_ti; }
  __device__ int jb() const { return R0 + TN * tJ + 16 * cc; }
  __device__ bool full() const { return valid() && jb() + 16 <= jlim; }
  __device__ void next() {
    if (++cc == cc0 + 2) {
      cc = cc0;
      if (++tJ == nc) {
        tJ = 0;
        ++tI;
        nc = tI < n_ti ? tile_cols(R0, n, tI) : 0;
        set_row();
      }
    }
  }
};

__device__ void epilogue_role(const TcSmem& sm, uint32_t tmem_base, float2* __restrict__ A, int n, int nrow,
                              long long ldm, int R0, int n_ti, int tcount) {
  const int warp = threadIdx.x >> 5, q = warp & 3, cc0 = 2 * (warp >> 3);
  const int r = 32 * q + (threadIdx.x & 31);
  const uint32_t lane_base = tmem_base + ((uint32_t)(32 * q) << 16);
  ChunkIt it;
  it.init(R0, n, nrow, n_ti, r, cc0);
  float4 nxt[8];
  if (it.full()) {
    const float2* p = A + (long long)it.i * ldm + it.jb();
#pragma unroll
    for (int e = 0; e < 8; ++e) nxt[e] = *reinterpret_cast<const float4*>(p + 2 * e);
  }
  bool ok = true;
  for (int tI = 0; tI < n_ti && ok; ++tI) {
    const int nc = tile_cols(R0, n, tI);
    for (int tJ = 0; tJ < nc; ++tJ, ++tcount) {
      const int b = tcount & 1, ub = tcount >> 1;
      ok = mbar_wait(smem_u32(&sm.tfull[b]), ub & 1, sm.abort_flag, sm.wait_ns);
      ok = __all_sync(0xffffffffu, ok);
      if (!ok) break;
      tc_fence_after();
#pragma unroll 1
      for (int cc = cc0; cc < cc0 + 2; ++cc) {
        const bool full = it.full();
        const int jb = it.jb(), jlim = it.jlim, i = it.i;
        float4 cur[8];
#pragma unroll
        for (int e = 0; e < 8; ++e) cur[e] = nxt[e];
        it.next();
        if (it.full()) {  // the next chunk's target values, in flight while this one is formed
          const float2* pn = A + (long long)it.i * ldm + it.jb();
#pragma unroll
          for (int e = 0; e < 8; ++e) nxt[e] = *reinterpret_cast<const float4*>(pn + 2 * e);
        }
        float2* p = A + (long long)i * ldm + jb;
        const bool part = !full && jb < jlim;
        if (part) {  // ragged chunk: the valid columns only
#pragma unroll
          for (int e = 0; e < 8; ++e) {
            const float2 u = jb + 2 * e < jlim ? p[2 * e] : make_float2(0.f, 0.f);
            const float2 v = jb + 2 * e + 1 < jlim ? p[2 * e + 1] : make_float2(0.f, 0.f);
            cur[e] = make_float4(u.x, u.y, v.x, v.y);
          }
        }
        // Re = Ar Lr^T - Ai Li^T: P columns 16 cc.., Q columns 64 + 16 cc..
        const uint32_t col = lane_base + (uint32_t)(b * 256 + 16 * cc);
        uint32_t t1[16], t2[16];
        tmem_ld16_nw(col, t1);
        tmem_ld16_nw(col + 128 + 64, t2);
        asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
        for (int e = 0; e < 8; ++e) {
          cur[e].x = cur[e].x - __uint_as_float(t1[2 * e]) + __uint_as_float(t2[2 * e]);
          cur[e].z = cur[e].z - __uint_as_float(t1[2 * e + 1]) + __uint_as_float(t2[2 * e + 1]);
        }
        // Im = Ar Li^T + Ai Lr^T: P columns 64 + 16 cc.., Q columns 16 cc..
        tmem_ld16_nw(col + 64, t1);
        tmem_ld16_nw(col + 128, t2);
        asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
        for (int e = 0; e < 8; ++e) {
          cur[e].y = cur[e].y - __uint_as_float(t1[2 * e]) - __uint_as_float(t2[2 * e]);
          cur[e].w = cur[e].w - __uint_as_float(t1[2 * e + 1]) - __uint_as_float(t2[2 * e + 1]);
        }
        if (full) {
#pragma unroll
          for (int e = 0; e < 8; ++e) *reinterpret_cast<float4*>(p + 2 * e) = cur[e];
        } else if (part) {
#pragma unroll
          for (int e = 0; e < 8; ++e) {
            if (jb + 2 * e < jlim) p[2 * e] = make_float2(cur[e].x, cur[e].y);
            if (jb + 2 * e + 1 < jlim) p[2 * e + 1] = make_float2(cur[e].z, cur[e].w);
          }
        }
      }
      tc_fence_before();
      mbar_arrive(smem_u32(&sm.tempty[b]));
    }
  }
}

// The factorisation of one matrix A (n columns, nrow rows) by one CTA.
__device__ __forceinline__ void ldlt_tc_matrix(float2* __restrict__ A, int n, int nrow, long long ldm,
                                               unsigned* __restrict__ status, unsigned long long wait_ns) {
  extern __shared__ uint8_t smem_raw[];
  TcSmem sm;
  sm.base = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~(uintptr_t)1023);
  uint64_t* bars = reinterpret_cast<uint64_t*>(sm.base + OPS_BYTES);
  sm.a_full = bars;
  sm.a_empty = bars + 1;
  sm.b_full = bars + 2;
  sm.b_empty = bars + 4;
  sm.tfull = bars + 6;
  sm.tempty = bars + 8;
  sm.mma_done = bars + 10;
  sm.tmem_slot = reinterpret_cast<uint32_t*>(bars + 11);
  sm.abort_flag = reinterpret_cast<volatile int*>(sm.tmem_slot + 1);
  sm.sing = reinterpret_cast<int*>(sm.tmem_slot + 2);
  sm.wait_ns = wait_ns;
  const PanelInv ps(sm.base);  // aliases the operand buffers (the phases alternate)

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (threadIdx.x == 0) {
    mbar_init(smem_u32(sm.a_full), 128);
    mbar_init(smem_u32(sm.a_empty), 1);
    for (int i = 0; i < 2; ++i) {
      mbar_init(smem_u32(&sm.b_full[i]), 128);
      mbar_init(smem_u32(&sm.b_empty[i]), 1);
      mbar_init(smem_u32(&sm.tfull[i]), 1);
      mbar_init(smem_u32(&sm.tempty[i]), N_EPI);
    }
    mbar_init(smem_u32(sm.mma_done), 1);
    *sm.abort_flag = 0;
    *sm.sing = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == MMA_WARP) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], 512;" ::"r"(smem_u32(sm.tmem_slot)));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem_base = *sm.tmem_slot;

  // B stages, tiles and row tiles issued so far; every role advances them alike
  int seq = 0, tcount = 0, rt = 0;
  for (int k0 = 0; k0 < n; k0 += PW) {
    const int kb = min(PW, n - k0);
    if (warp < NT_PANEL / 32) factor_panel_tc(A, n, nrow, ldm, k0, ps, sm.sing);
    __syncthreads();  // panel W / L^T in global memory; the panel scratch is free
    const int R0 = k0 + kb;
    if (R0 < n) {
      const int n_ti = (nrow - R0 + TM - 1) / TM;
      if (warp == MMA_WARP) {
        if (lane == 0) mma_role(sm, tmem_base, n, R0, n_ti, seq, tcount, rt);
        __syncwarp();
      } else if (warp >= 4 && warp < 8) {
        transform_role(sm, A, n, nrow, ldm, k0, R0, n_ti, seq, rt);
      } else {
        epilogue_role(sm, tmem_base, A, n, nrow, ldm, R0, n_ti, tcount);
      }
      int nt = 0;
      for (int tI = 0; tI < n_ti; ++tI) nt += tile_cols(R0, n, tI);
      seq += 2 * nt;
      tcount += nt;
      rt += n_ti;
    }
    tc_fence_before();
    __syncthreads();  // every tile of the panel is written back; the operand buffers are free
    tc_fence_after();
    if (*sm.abort_flag) break;
  }
  // every MMA issued has completed before TMEM is freed (immediate unless a wait gave up)
  if (warp == MMA_WARP) {
    if (lane == 0) {
      mma_commit(smem_u32(sm.mma_done));
      mbar_drain(smem_u32(sm.mma_done), 0);
    }
    __syncwarp();
  }
  tc_fence_before();
  __syncthreads();
  if (threadIdx.x == 0) {
    if (*sm.abort_flag) atomicOr(status, kStatTimeout);
    if (*sm.sing) atomicOr(status, kStatSingular);
  }
  if (warp == MMA_WARP) {
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, 512;" ::"r"(tmem_base));
  }
}

__global__ void __launch_bounds__(NT_TC, 1)
    ldlt_tc_kernel(float2* __restrict__ mats, int n, int nrow, long long ldm, long long stride,
                   const int* __restrict__ active, unsigned* __restrict__ status, unsigned long long wait_ns) {
  const int f = blockIdx.x;
  if (active && !active[f]) return;  // uniform across the CTA, before any barrier or TMEM use
  ldlt_tc_matrix(mats + f * stride, n, nrow, ldm, status, wait_ns);
}

// Grouped: CTA b factors matrix b - cta0 of the group whose CTA range holds b (groups ascending in cta0).
__global__ void __launch_bounds__(NT_TC, 1)
    ldlt_tc_grouped_kernel(const LdltGroup* __restrict__ gs, int n_groups, unsigned* __restrict__ status,
                           unsigned long long wait_ns) {
  int lo = 0, hi = n_groups - 1;
  while (lo < hi) {  // last group with cta0 <= blockIdx.x
    const int mid = (lo + hi + 1) / 2;
    if (gs[mid].cta0 <= (int)blockIdx.x) lo = mid; else hi = mid - 1;
  }
  const LdltGroup& G = gs[lo];
  const int f = blockIdx.x - G.cta0;
  if (f >= G.F) return;
  if (G.active && !G.active[f]) return;  // uniform across the CTA, before any barrier or TMEM use
  ldlt_tc_matrix(G.mats + f * G.stride, G.n, G.nrow, G.ldm, status, wait_ns);
}

// ---- split factorisation: one panel launch and one batched tensor-core update per panel --------------
// The kernel above gives each matrix one CTA for its whole factorisation, and its tensor phase waits on
// the per-thread global loads of one SM (a 4500-wide matrix takes ~190 ms). Here every panel is three
// launches over all matrices of the batch:
//   ldlt_panel_kernel   the panel [k0, k0 + 64) of every matrix (one CTA each: factor_panel_tc);
//   ldlt_planes_kernel  the panel's W columns (rows below it) and L rows (row k0 + l of the L^T stored above
//                       the diagonal, the columns beyond the panel) as TF32 hi / lo planes, K-major;
//   ldlt_update_kernel  C[i][j] -= sum_l W[i][l] L[j][l] over the trailing 128 x 64 tiles of every matrix,
//                       one tile per CTA, two CTAs per SM: TMA-fed planes, the P and Q accumulators of the
//                       one-CTA kernel, and the target tile staged through shared memory by TMA (128-byte
//                       swizzle, clipped at column n and row nrow; the part of a diagonal tile above the
//                       diagonal holds nothing yet and is overwritten when its own panel is factored).
// Panels go in pairs with a one-panel lookahead: panel p's update is first applied to panel p + 1's 64
// columns only, panel p + 1 is factored, and then one rank-128 update (K = 128: both panels' planes side by
// side) covers the trailing matrix, which is thus read and written once per two panels.

constexpr int UP_A = TM * 128;                   // one A plane chunk: 128 rows x 32 FP32 = 16 KB
constexpr int UP_B = TN * 128;                   // one B plane chunk: 64 rows x 32 FP32 = 8 KB
constexpr int UP_STAGE = 4 * UP_A + 4 * UP_B;    // Ar, Ai, Ar_lo, Ai_lo | Lr, Li, Lr_lo, Li_lo: 96 KB
constexpr int UP_SMEM = 1024 + UP_STAGE + 128;
constexpr int UP_THREADS = 256;                  // warp 0 TMA, 1 MMA, 2 TMEM, 4-7 epilogue
constexpr int PANEL_SCRATCH = (int)PanelInv::bytes();
constexpr int PANEL_SMEM = 1024 + PANEL_SCRATCH + 64;
static_assert(TM * TN * 8 <= UP_STAGE, "the target tile fits in the stage");

constexpr int KW = 2 * PW;  // K width of the planes: two panels

struct UpParams {
  CUtensorMap a[4];  // Ar_hi, Ai_hi, Ar_lo, Ai_lo  [F * nrow][KW]
  CUtensorMap b[4];  // Lr_hi, Li_hi, Lr_lo, Li_lo  [F * n][KW]
  CUtensorMap c;     // targets: (2n FP32 along a row, nrow rows, F matrices)
  int n, nrow, R0, F, tiles;
  int nkc;           // 32-wide K chunks of this update (2: one panel, 4: two)
  int one_col;       // lookahead: only the column tile [R0, R0 + 64)
  const int* active;
  unsigned* status;
  unsigned long long wait_ns;
};

__device__ __forceinline__ void tma_load_3d(uint32_t dst, const CUtensorMap* tm, int x, int y, int z, uint32_t bar) {
  asm volatile(
      "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], [%5];" ::"r"(dst),
      "l"(reinterpret_cast<uint64_t>(tm)), "r"(x), "r"(y), "r"(z), "r"(bar)
      : "memory");
}

__device__ __forceinline__ void tma_store_3d(const CUtensorMap* tm, int x, int y, int z, uint32_t src) {
  asm volatile("cp.async.bulk.tensor.3d.global.shared::cta.bulk_group [%0, {%1, %2, %3}], [%4];" ::"l"(
                   reinterpret_cast<uint64_t>(tm)),
               "r"(x), "r"(y), "r"(z), "r"(src)
               : "memory");
}

__global__ void __launch_bounds__(NT_PANEL, 1)
    ldlt_panel_kernel(float2* __restrict__ mats, int n, int nrow, long long ldm, long long stride, int k0,
                      const int* __restrict__ active, unsigned* __restrict__ status) {
  const int f = blockIdx.x;
  if (active && !active[f]) return;
  extern __shared__ uint8_t smem_raw[];
  uint8_t* base = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~(uintptr_t)1023);
  const PanelInv ps(base);
  int* sing = reinterpret_cast<int*>(base + PANEL_SCRATCH);
  if (threadIdx.x == 0) *sing = 0;
  __syncthreads();
  factor_panel_tc(mats + f * stride, n, nrow, ldm, k0, ps, sing);
  __syncthreads();
  if (threadIdx.x == 0 && *sing) atomicOr(status, kStatSingular);
}

// blockIdx.y = matrix; blocks 0 .. nA-1: four rows i of W each; blocks nA ..: 32 columns j of L each
__global__ void __launch_bounds__(256)
    ldlt_planes_kernel(const float2* __restrict__ mats, int n, int nrow, long long ldm, long long stride, int k0, int koff,
                       int nA, const int* __restrict__ active, float* __restrict__ ap, float* __restrict__ bp) {
  const int f = blockIdx.y;
  if (active && !active[f]) return;
  const float2* A = mats + f * stride;
  const int kb = min(PW, n - k0), R0 = k0 + kb;
  const size_t a_plane = (size_t)gridDim.y * nrow * KW, b_plane = (size_t)gridDim.y * n * KW;
  if ((int)blockIdx.x < nA) {
    const int i = R0 + 4 * blockIdx.x + (threadIdx.x >> 6), l = threadIdx.x & 63;
    if (i >= nrow) return;
    const float2 v = l < kb ? A[(long long)i * ldm + k0 + l] : make_float2(0.f, 0.f);
    const size_t o = ((size_t)f * nrow + i) * KW + koff + l;
    const float rh = tf32_rn(v.x), ih = tf32_rn(v.y);
    ap[o] = rh;
    ap[a_plane + o] = ih;
    ap[2 * a_plane + o] = tf32_rn(v.x - rh);
    ap[3 * a_plane + o] = tf32_rn(v.y - ih);
    return;
  }
  __shared__ float2 tile[PW][33];
  const int j0 = R0 + 32 * (blockIdx.x - nA);
  for (int e = threadIdx.x; e < PW * 32; e += 256) {
    const int l = e >> 5, jj = e & 31, j = j0 + jj;
    tile[l][jj] = (l < kb && j < n) ? A[(long long)(k0 + l) * ldm + j] : make_float2(0.f, 0.f);
  }
  __syncthreads();
  for (int e = threadIdx.x; e < PW * 32; e += 256) {
    const int jj = e >> 6, l = e & 63, j = j0 + jj;
    if (j >= n) continue;
    const float2 v = tile[l][jj];
    const size_t o = ((size_t)f * n + j) * KW + koff + l;
    const float rh = tf32_rn(v.x), ih = tf32_rn(v.y);
    bp[o] = rh;
    bp[b_plane + o] = ih;
    bp[2 * b_plane + o] = tf32_rn(v.x - rh);
    bp[3 * b_plane + o] = tf32_rn(v.y - ih);
  }
}

__global__ void __launch_bounds__(UP_THREADS, 2) ldlt_update_kernel(const __grid_constant__ UpParams p) {
  extern __shared__ uint8_t smem_raw[];
  uint8_t* base = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~(uintptr_t)1023);
  uint64_t* full = reinterpret_cast<uint64_t*>(base + UP_STAGE);
  uint64_t* empty = full + 1;
  uint64_t* done = full + 2;
  uint64_t* c_full = full + 3;
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(full + 4);
  volatile int* abort_flag = reinterpret_cast<volatile int*>(tmem_slot + 1);

  const int f = blockIdx.x / p.tiles;
  int t = blockIdx.x - f * p.tiles;
  if (f >= p.F || (p.active && !p.active[f])) return;  // uniform, before any barrier or TMEM use
  int tI = 0;
  if (p.one_col) {  // lookahead: row tile t, the column tile [R0, R0 + 64)
    tI = t;
    t = 0;
  } else {
    for (;;) {  // (row tile, column tile) of tile t of the trailing lower part
      const int nc = tile_cols(p.R0, p.n, tI);
      if (t < nc) break;
      t -= nc;
      ++tI;
    }
  }
  const int i0 = p.R0 + TM * tI, j0 = p.R0 + TN * t;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;

  if (threadIdx.x == 0) {
    mbar_init(smem_u32(full), 1);
    mbar_init(smem_u32(empty), 1);
    mbar_init(smem_u32(done), 1);
    mbar_init(smem_u32(c_full), 1);
    *abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 2) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], 256;" ::"r"(smem_u32(tmem_slot)));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tmem_slot;

  if (warp == 0) {
    if (lane == 0) {
      int issued = 0;
      for (int kc = 0; kc < p.nkc; ++kc) {  // one stage, reused by every chunk
        if (kc > 0 && !mbar_wait(smem_u32(empty), (uint32_t)(kc - 1) & 1, abort_flag, p.wait_ns)) break;
        mbar_expect_tx(smem_u32(full), UP_STAGE);
        const int ay = f * p.nrow + i0, by = f * p.n + j0;
        for (int q = 0; q < 4; ++q) tma_load_2d(smem_u32(base + q * UP_A), &p.a[q], KH * kc, ay, smem_u32(full));
        for (int q = 0; q < 4; ++q) tma_load_2d(smem_u32(base + 4 * UP_A + q * UP_B), &p.b[q], KH * kc, by, smem_u32(full));
        issued = kc + 1;
      }
      if (issued > 0) mbar_drain(smem_u32(full), (uint32_t)(issued - 1) & 1);
    }
  } else if (warp == 1) {
    if (lane == 0) {
      const uint32_t st = smem_u32(base);
      const uint64_t dar = sdesc(st), dai = sdesc(st + UP_A), darl = sdesc(st + 2 * UP_A), dail = sdesc(st + 3 * UP_A);
      const uint64_t dbh = sdesc(st + 4 * UP_A), dbl = sdesc(st + 4 * UP_A + 2 * UP_B);  // [Lr; Li] hi, lo
      const uint32_t dp = tmem, dq = tmem + 128;
      bool committed = false;  // `done` takes exactly one commit (a second would flip its phase back)
      for (int kc = 0; kc < p.nkc; ++kc) {
        if (!mbar_wait(smem_u32(full), (uint32_t)kc & 1, abort_flag, p.wait_ns)) break;
        tc_fence_after();
#pragma unroll
        for (int k = 0; k < KH / 8; ++k) {
          const uint64_t o = 2u * k;
          const uint32_t acc = (kc == 0 && k == 0) ? 0u : 1u;
          mma_tf32(dp, dar + o, dbh + o, acc);
          mma_tf32(dp, dar + o, dbl + o, 1u);
          mma_tf32(dp, darl + o, dbh + o, 1u);
          mma_tf32(dq, dai + o, dbh + o, acc);
          mma_tf32(dq, dai + o, dbl + o, 1u);
          mma_tf32(dq, dail + o, dbh + o, 1u);
        }
        if (kc + 1 < p.nkc) {
          mma_commit(smem_u32(empty));
        } else {
          mma_commit(smem_u32(done));
          committed = true;
        }
      }
      if (!committed) mma_commit(smem_u32(done));  // after an early stop: fires once the issued MMAs complete
    }
  } else if (warp >= 4) {
    // ---- epilogue: C -= (P_re - Q_im, P_im + Q_re) through shared memory -------------------------
    const int q = warp & 3, r = 32 * q + lane;
    const bool ok = __all_sync(0xffffffffu, mbar_wait(smem_u32(done), 0, abort_flag, p.wait_ns));
    tc_fence_after();
    bool landed = false;
    if (ok && !*abort_flag) {
      if (threadIdx.x == 128) {
        mbar_expect_tx(smem_u32(c_full), TM * TN * 8);
        for (int b = 0; b < 4; ++b) tma_load_3d(smem_u32(base + b * UP_A), &p.c, 2 * j0 + 32 * b, i0, f, smem_u32(c_full));
      }
      landed = __all_sync(0xffffffffu, mbar_wait(smem_u32(c_full), 0, abort_flag, p.wait_ns));
      if (landed) {
        const uint32_t lb = tmem + ((uint32_t)(32 * q) << 16);
        for (int c4 = 0; c4 < 4; ++c4) {  // complex columns 16 c4 .. + 15: box c4 of the staged tile
          uint32_t pr[16], pi[16], qr[16], qi[16];
          tmem_ld16_nw(lb + 16 * c4, pr);        // Ar Lr^T
          tmem_ld16_nw(lb + 64 + 16 * c4, pi);   // Ar Li^T
          tmem_ld16_nw(lb + 128 + 16 * c4, qr);  // Ai Lr^T
          tmem_ld16_nw(lb + 192 + 16 * c4, qi);  // Ai Li^T
          asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
          uint8_t* rowp = base + c4 * UP_A + r * 128;
#pragma unroll
          for (int ch = 0; ch < 8; ++ch) {  // 16-byte chunk ch: complex columns 2 ch, 2 ch + 1
            float4* cp = reinterpret_cast<float4*>(rowp + ((ch ^ (r & 7)) << 4));
            float4 v = *cp;
            const int e0 = 2 * ch, e1 = 2 * ch + 1;
            v.x -= __uint_as_float(pr[e0]) - __uint_as_float(qi[e0]);
            v.y -= __uint_as_float(pi[e0]) + __uint_as_float(qr[e0]);
            v.z -= __uint_as_float(pr[e1]) - __uint_as_float(qi[e1]);
            v.w -= __uint_as_float(pi[e1]) + __uint_as_float(qr[e1]);
            *cp = v;
          }
        }
      }
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    }
    asm volatile("bar.sync 1, 128;" ::: "memory");  // every epilogue warp, whatever its waits gave
    if (threadIdx.x == 128) {
      if (landed && !*abort_flag) {
        for (int b = 0; b < 4; ++b) tma_store_3d(&p.c, 2 * j0 + 32 * b, i0, f, smem_u32(base + b * UP_A));
        asm volatile("cp.async.bulk.commit_group;" ::: "memory");
        asm volatile("cp.async.bulk.wait_group.read 0;" ::: "memory");
      } else if (ok) {
        mbar_drain(smem_u32(c_full), 0);
      }
    }
  }
  if (warp == 2) {
    if (lane == 0) mbar_drain(smem_u32(done), 0);
    __syncwarp();
  }
  tc_fence_before();
  __syncthreads();
  if (threadIdx.x == 0 && *abort_flag) atomicOr(p.status, kStatTimeout);
  if (warp == 2) {
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, 256;" ::"r"(tmem));
  }
}

int host_tile_cols(int R0, int n, int tI) {
  const int jmax = std::min(n, R0 + TM * tI + TM);
  return (jmax - R0 + TN - 1) / TN;
}

}  // namespace

int launch_ldlt_tc_grouped(const LdltGroup* d_groups, int n_groups, int n_ctas, unsigned* status,
                           unsigned long long wait_ns, cudaStream_t s) {
  if (!tc_supported()) return -2;
  if (n_groups < 1 || n_ctas < 1) return -1;
  static bool attr = false;
  if (!attr) {
    if (cudaFuncSetAttribute(ldlt_tc_grouped_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, SMEM_TC) != cudaSuccess)
      return -1;
    attr = true;
  }
  ldlt_tc_grouped_kernel<<<n_ctas, NT_TC, SMEM_TC, s>>>(d_groups, n_groups, status, wait_ns);
  return cudaPeekAtLastError() == cudaSuccess ? 1 : -1;
}

// Returns 1 (launches), -1 on a launch error or bad layout, -2 if the device has no tcgen05.
int launch_ldlt_tc(void* mats, int n, int nrow, long long ldm, long long stride, int F, const int* active,
                   unsigned* status, unsigned long long wait_ns, cudaStream_t s) {
  if (!tc_supported()) return -2;
  // 16-byte loads and stores: ldm and the matrix stride multiples of 4 complex values (32 B)
  if ((ldm % 4) || (stride % 4) || (reinterpret_cast<uintptr_t>(mats) & 15) || nrow < n || n < 1) return -1;
  static bool attr = false;
  if (!attr) {
    if (cudaFuncSetAttribute(ldlt_tc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, SMEM_TC) != cudaSuccess)
      return -1;
    attr = true;
  }
  ldlt_tc_kernel<<<F, NT_TC, SMEM_TC, s>>>(reinterpret_cast<float2*>(mats), n, nrow, ldm, stride, active, status,
                                                wait_ns);
  return cudaPeekAtLastError() == cudaSuccess ? 1 : -1;
}

size_t ldlt_split_bytes(int n, int nrow, int F) { return (size_t)16 * F * KW * ((size_t)nrow + n) + 1024; }

// Returns the launches, -1 on a launch error or bad layout, -2 if unsupported.
int launch_ldlt_split(void* mats, int n, int nrow, long long ldm, long long stride, int F, const int* active,
                      unsigned* status, unsigned long long wait_ns, void* work, size_t work_bytes, cudaStream_t s) {
  if (!tc_supported()) return -2;
  if ((ldm % 4) || (stride % 4) || (reinterpret_cast<uintptr_t>(mats) & 15) || nrow < n || n < 1 || F < 1) return -1;
  if (ldlt_split_bytes(n, nrow, F) > work_bytes || (reinterpret_cast<uintptr_t>(work) & 15)) return -2;
  static bool attr = false;
  if (!attr) {
    if (cudaFuncSetAttribute(ldlt_panel_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, PANEL_SMEM) != cudaSuccess ||
        cudaFuncSetAttribute(ldlt_update_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, UP_SMEM) != cudaSuccess)
      return -1;
    attr = true;
  }
  float* ap = static_cast<float*>(work);
  float* bp = ap + (size_t)4 * F * nrow * KW;
  UpParams p;
  std::memset(static_cast<void*>(&p), 0, sizeof(p));
  for (int q = 0; q < 4; ++q) {
    if (!make_map(&p.a[q], ap + (size_t)q * F * nrow * KW, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 4, F * nrow, KW, KH, TM) ||
        !make_map(&p.b[q], bp + (size_t)q * F * n * KW, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 4, F * n, KW, KH, TN))
      return -2;
  }
  {
    EncodeTiledFn enc = encoder();
    if (!enc) return -2;
    cuuint64_t dims[3] = {(cuuint64_t)2 * n, (cuuint64_t)nrow, (cuuint64_t)F};
    cuuint64_t strides[2] = {(cuuint64_t)ldm * 8, (cuuint64_t)stride * 8};
    cuuint32_t box[3] = {32, (cuuint32_t)TM, 1};
    cuuint32_t es[3] = {1, 1, 1};
    if (enc(&p.c, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, mats, dims, strides, box, es, CU_TENSOR_MAP_INTERLEAVE_NONE,
            CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
      return -2;
  }
  p.n = n;
  p.nrow = nrow;
  p.F = F;
  p.active = active;
  p.status = status;
  p.wait_ns = wait_ns;
  float2* A = reinterpret_cast<float2*>(mats);
  int launches = 0;
  auto panel = [&](int k0) {
    ldlt_panel_kernel<<<F, NT_PANEL, PANEL_SMEM, s>>>(A, n, nrow, ldm, stride, k0, active, status);
    ++launches;
  };
  auto planes = [&](int k0, int koff) {
    const int R0 = k0 + std::min(PW, n - k0);
    const int nA = (nrow - R0 + 3) / 4, nB = (n - R0 + 31) / 32;
    ldlt_planes_kernel<<<dim3(nA + nB, F), 256, 0, s>>>(A, n, nrow, ldm, stride, k0, koff, nA, active, ap, bp);
    ++launches;
  };
  auto update = [&](int R0, int nkc, bool one_col) {
    const int n_ti = (nrow - R0 + TM - 1) / TM;
    int tiles = 0;
    if (one_col) {
      tiles = n_ti;
    } else {
      for (int tI = 0; tI < n_ti; ++tI) tiles += host_tile_cols(R0, n, tI);
    }
    p.R0 = R0;
    p.tiles = tiles;
    p.nkc = nkc;
    p.one_col = one_col ? 1 : 0;
    ldlt_update_kernel<<<F * tiles, UP_THREADS, UP_SMEM, s>>>(p);
    ++launches;
  };
  for (int k0 = 0; k0 < n;) {
    // panel p at k0, with the planes of its W columns and L rows in K columns 0..63
    const int R0 = k0 + std::min(PW, n - k0);
    panel(k0);
    if (R0 >= n) break;
    planes(k0, 0);
    // lookahead: panel p's update of panel p + 1's columns only, then panel p + 1
    update(R0, PW / KH, true);
    panel(R0);
    const int R1 = R0 + std::min(PW, n - R0);
    if (R1 < n) {
      planes(R0, PW);
      update(R1, KW / KH, false);  // both panels: K = 128
    }
    if (cudaPeekAtLastError() != cudaSuccess) return -1;
    k0 = R1;
  }
  if (cudaPeekAtLastError() != cudaSuccess) return -1;
  return launches;
}

}  // namespace gwc
