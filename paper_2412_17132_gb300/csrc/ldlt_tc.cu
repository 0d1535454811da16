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
//   warps 0-11  panel factorisation (the shared SIMT routine, named barrier 1)
//   warps 4-7   operand transform: global memory (L2) -> hi/lo planes in the 128-byte-swizzled
//               K-major layout. The A operand (W rows of a 128-row tile, all 64 panel columns)
//               stays resident while the tile row's column tiles pass; the B operand (L rows of a
//               64-column tile) streams through two stages of 32 panel columns, the global loads
//               of a stage issued before the wait for its buffer.
//   warp 12     TMEM allocation (512 columns: two tiles in flight x {D1, D2}) and the MMA issuer
//   warps 0-3,  epilogue: one thread per tile row and half of the tile's columns, the target values
//   8-11        read and written with 16-byte accesses, the next chunk's values loaded ahead
// The panel scratch of the SIMT routine aliases the operand buffers (the phases alternate).
// Every mbarrier wait is bounded (one second); on expiry the CTA records kStatTimeout, stops,
// drains the MMAs it issued and frees TMEM.
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
static_assert(PanelSmem<float2, NT_PANEL>::bytes() <= (size_t)OPS_BYTES, "panel scratch fits in the operand buffers");

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
    if (!mbar_wait(smem_u32(sm.a_empty), (rt & 1) ^ 1, sm.abort_flag)) break;
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
      if (!mbar_wait(smem_u32(&sm.b_empty[s]), (us & 1) ^ 1, sm.abort_flag)) {
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
    if (!mbar_wait(smem_u32(sm.a_full), rt & 1, sm.abort_flag)) break;
    tc_fence_after();
    const int nc = tile_cols(R0, n, tI);
    for (int tJ = 0; tJ < nc && ok; ++tJ, ++tcount) {
      const int b = tcount & 1, ub = tcount >> 1;
      if (!mbar_wait(smem_u32(&sm.tempty[b]), (ub & 1) ^ 1, sm.abort_flag)) {
        ok = false;
        break;
      }
      tc_fence_after();
      const uint32_t dp = tmem_base + (uint32_t)(b * 256), dq = dp + 128;  // P and Q accumulators
      for (int h = 0; h < 2; ++h, ++seq) {
        const int s = seq & 1, us = seq >> 1;
        if (!mbar_wait(smem_u32(&sm.b_full[s]), us & 1, sm.abort_flag)) {
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
      ok = mbar_wait(smem_u32(&sm.tfull[b]), ub & 1, sm.abort_flag);
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

__global__ void __launch_bounds__(NT_TC, 1)
    ldlt_tc_kernel(float2* __restrict__ mats, int n, int nrow, long long ldm, long long stride,
                   const int* __restrict__ active, unsigned* __restrict__ status) {
  const int f = blockIdx.x;
  if (active && !active[f]) return;  // uniform across the CTA, before any barrier or TMEM use
  float2* A = mats + f * stride;
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
  const PanelSmem<float2, NT_PANEL> ps(sm.base);  // aliases the operand buffers (the phases alternate)

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
    if (warp < NT_PANEL / 32) factor_panel<float2, NT_PANEL>(A, n, nrow, ldm, k0, ps, *sm.sing);
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

}  // namespace

// Returns 1 (launches), -1 on a launch error or bad layout, -2 if the device has no tcgen05.
int launch_ldlt_tc(void* mats, int n, int nrow, long long ldm, long long stride, int F, const int* active,
                   unsigned* status, cudaStream_t s) {
  if (!tc_supported()) return -2;
  // 16-byte loads and stores: ldm and the matrix stride multiples of 4 complex values (32 B)
  if ((ldm % 4) || (stride % 4) || (reinterpret_cast<uintptr_t>(mats) & 15) || nrow < n || n < 1) return -1;
  static bool attr = false;
  if (!attr) {
    if (cudaFuncSetAttribute(ldlt_tc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, SMEM_TC) != cudaSuccess)
      return -1;
    attr = true;
  }
  ldlt_tc_kernel<<<F, NT_TC, SMEM_TC, s>>>(reinterpret_cast<float2*>(mats), n, nrow, ldm, stride, active, status);
  return cudaPeekAtLastError() == cudaSuccess ? 1 : -1;
}

}  // namespace gwc
