// Tensor-core polarizability build for sm_103a (tcgen05 + TMEM + TMA).
//
//   Pi_PQ(z_f) = sum_k O_Pk D_f(k) O_Qk      (RI polarizability, Sec. "Self-energy evaluation")
//
// One CTA computes one 128 x 128 lower-triangle tile (P-tile >= Q-tile) for two frequency
// parts: the real and imaginary parts of D at one complex z, or two points of the imaginary
// axis. The contraction index k = (i, a) runs over the occupied-virtual pairs in 64-wide chunks.
//
//   * TMA brings, per chunk, the B operand O[Q-tile][chunk] (BF16 hi, and lo in split mode,
//     SWIZZLE_128B, K-major), the FP32 rows O[P-tile][chunk] and the two 64-value slices of
//     the D(z) table into two-stage rings.
//   * 8 transform warps form the A operand O[P][k] D_p(k) (the D scaling is fused into the
//     operand load): two threads per row, each scaling 32 of its 64 values, split them into
//     BF16 hi and lo = bf16(v - hi) and write them in the swizzled K-major layout the MMA reads.
//   * One thread issues tcgen05.mma (kind::f16, BF16 x BF16 -> FP32 in TMEM): per part and
//     16-wide k step hi*hi (+ hi*lo + lo*hi in split mode; Henry, Tang & Heinecke 2019).
//   * Segmented accumulation: the FP32 accumulator of the tensor core rounds toward zero, a
//     bias that grows with the number of accumulations into one accumulator. Each part
//     therefore accumulates only kSeg chunks into a "fresh" TMEM accumulator; 4 fold warps
//     then add it (round-to-nearest FP32) into a running sum kept in TMEM and release the
//     accumulator. Each part has its own segment and fold barriers: the fold of part 0 runs
//     while the MMAs of part 1 finish the chunk, and the fold of part 1 while the next
//     segment's part-0 MMAs run, so the tensor pipe does not wait for a whole fold. The last
//     fold writes alpha * Pi + beta * I (eps = 1 - Pi for alpha = -1, beta = 1) to global memory.
//
// Every wait on an mbarrier is bounded (one second unless the context sets another bound); on expiry the CTA records kStatTimeout,
// stops issuing work, drains the copies and MMAs it issued and frees TMEM.
#include <cuda.h>

#include <algorithm>
#include <cstdio>
#include <cstring>
#include <mutex>

#include "gwc_internal.h"
#include "tc_common.cuh"

namespace gwc {

namespace {

constexpr int BM = 128, BN = 128, BK = 64;
constexpr int kParts = 2;                  // frequency parts per CTA
constexpr int kSeg = 8;                    // chunks accumulated per fresh accumulator
constexpr int NB_ST = 2;                   // B ring / raw-A ring stages
constexpr int NA_ST = 3;                   // scaled-A slots (one part each)
constexpr int TILE = BM * BK * 2;          // 16 KB: one BF16 128 x 64 operand tile
constexpr int RAW = BM * BK * 4;           // 32 KB: FP32 128 x 64 rows (two 128-B swizzled halves)
constexpr int DSL = kParts * BK * 4;       // 512 B: D slices of one chunk
constexpr int NTHREADS = 512;              // warp 0 TMA, 1 MMA, 2 TMEM then transform, 12-15 fold
// Transform warps: none on the MMA warp's scheduler (warp % 4 == 1). A single issuing thread
// shares its sub-partition's issue slots with the warps there, and ALU-heavy neighbours starve
// it (measured: 322 instead of 64 cycles per 128x128x16 MMA beside two FMA-bound warps).
__device__ __forceinline__ int transform_rank(int warp) {
  switch (warp) {
    case 2: return 0;
    case 3: return 1;
    case 4: return 2;
    case 6: return 3;
    case 7: return 4;
    case 8: return 5;
    case 10: return 6;
    case 11: return 7;
    default: return -1;
  }
}
constexpr int NXF = 256;                   // transform threads (two per row of the P tile)
constexpr int NFOLD = 128;                 // fold threads
constexpr int SMEM_BYTES = 1024 + NB_ST * 2 * TILE + NB_ST * RAW + NA_ST * 2 * TILE + NB_ST * DSL + 256;

// One group of work: one molecule's frequency batch (its O copies, D table and output matrices). A
// launch processes the items (lower 128 x 128 tile, frequency group) of one or several groups.
struct Chi0Group {
  CUtensorMap tm_hi, tm_lo, tm_raw;  // B operand (BF16 hi, lo) and FP32 rows of the A operand
  const float* dtab;
  void* out;
  const int* active;      // per frequency, or null
  long long ldm, mat_stride;
  int ld_dtab;
  int n_aux;
  int n_kc;               // number of 64-wide chunks
  int F;
  int ppf;                // parts per frequency (1 real, 2 complex)
  int fpc;                // frequencies per item (kParts / ppf)
  int n_tiles;            // lower 128-tiles of the matrix
  int item0;              // index of the group's first item in the launch
  int n_items;            // n_tiles * ceil(F / fpc)
  int split3;
  int out64;              // matrices in FP64 (double / double2) instead of FP32
  float alpha, beta;
};

struct TcParams {
  const Chi0Group* groups;  // grouped launch: descriptors in global memory (else the kernel's own group)
  int n_groups;
  int n_items;
  unsigned* status;
  unsigned long long wait_ns;  // bound of every mbarrier wait
};

// Instruction descriptor, kind::f16: D = F32, A = B = BF16, both K-major, M = 128, N = 128.
constexpr uint32_t kIdesc = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(BN >> 3) << 17) | ((uint32_t)(BM >> 4) << 24);

__device__ __forceinline__ void mma_bf16(uint32_t d_tmem, uint64_t a, uint64_t b, uint32_t accum) {
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "setp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(d_tmem),
      "l"(a), "l"(b), "r"(kIdesc), "r"(accum));
}

__device__ __forceinline__ void tile_pair(int t, int& ip, int& iq) {
  int a = (int)((sqrt(8.0 * t + 1.0) - 1.0) * 0.5);
  while ((a + 1) * (a + 2) / 2 <= t) ++a;
  while (a * (a + 1) / 2 > t) --a;
  ip = a;
  iq = t - a * (a + 1) / 2;
}

// TMEM load without the implicit wait: several loads share one tcgen05.wait::ld
__device__ __forceinline__ void tmem_ld16_async(uint32_t taddr, uint32_t (&r)[16]) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]),
        "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
      : "r"(taddr));
}

__device__ __forceinline__ void tmem_wait_ld() { asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory"); }

__device__ __forceinline__ uint32_t pack_bf16x2(float a, float b) {
  __nv_bfloat162 h = __floats2bfloat162_rn(a, b);
  return *reinterpret_cast<uint32_t*>(&h);
}

// Item `it` of the launch: its group (groups are ordered by item0; g only moves forward), tile and
// frequency range; false if every frequency of the item is masked out (all roles skip it alike).
struct Item {
  int g, P0, Q0, f0, nf, n_parts;
};

__device__ __forceinline__ bool decode_item(const Chi0Group* gs, int n_groups, int it, int& g, Item& x) {
  while (g + 1 < n_groups && it >= gs[g + 1].item0) ++g;
  const Chi0Group& G = gs[g];
  const int local = it - G.item0;
  const int t = local % G.n_tiles, fgi = local / G.n_tiles;
  int ip, iq;
  tile_pair(t, ip, iq);
  x.g = g;
  x.P0 = ip * BM;
  x.Q0 = iq * BN;
  x.f0 = fgi * G.fpc;
  x.nf = min(G.fpc, G.F - x.f0);
  x.n_parts = x.nf * G.ppf;
  if (G.active) {
    int any = 0;
    for (int u = 0; u < x.nf; ++u) any |= G.active[x.f0 + u];
    if (!any) return false;
  }
  return true;
}

// Every role walks the same items in the same order (it = blockIdx.x, + gridDim.x, ...) and keeps running
// counters across them (chunks, A slots, segments per part), from which the mbarrier phases follow; a
// launch with one item per CTA and a persistent launch over many items run the same code.
template <bool CPLX, bool GROUPED>
__global__ void __launch_bounds__(NTHREADS, 1)
    chi0_tc_kernel(const __grid_constant__ Chi0Group g_own, TcParams p) {
  extern __shared__ uint8_t smem_raw[];
  uint8_t* base = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~(uintptr_t)1023);
  uint8_t* b_ring = base;                            // NB_ST x [hi | lo]
  uint8_t* r_ring = b_ring + NB_ST * 2 * TILE;       // NB_ST x [k 0..31 | k 32..63] FP32, swizzled
  uint8_t* a_ring = r_ring + NB_ST * RAW;            // NA_ST x [hi | lo]
  float* d_ring = reinterpret_cast<float*>(a_ring + NA_ST * 2 * TILE);  // NB_ST x [part][64]
  uint64_t* bars = reinterpret_cast<uint64_t*>(d_ring + NB_ST * kParts * BK);
  uint64_t* b_full = bars;
  uint64_t* b_empty = b_full + NB_ST;
  uint64_t* r_full = b_empty + NB_ST;
  uint64_t* r_empty = r_full + NB_ST;
  uint64_t* a_full = r_empty + NB_ST;
  uint64_t* a_empty = a_full + NA_ST;
  uint64_t* seg_full = a_empty + NA_ST;      // [part]: the part's fresh accumulator is complete
  uint64_t* fold_done = seg_full + kParts;   // [part]: the part's fresh accumulator is folded
  uint64_t* mma_done = fold_done + kParts;
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(mma_done + 1);
  volatile int* abort_flag = reinterpret_cast<volatile int*>(tmem_slot + 1);

  const Chi0Group* gs = GROUPED ? p.groups : &g_own;
  const int n_groups = GROUPED ? p.n_groups : 1;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (blockIdx.x >= p.n_items) return;  // uniform across the CTA, before any barrier or TMEM use

  if (threadIdx.x == 0) {
    for (int i = 0; i < NB_ST; ++i) {
      mbar_init(smem_u32(&b_full[i]), 1);
      mbar_init(smem_u32(&b_empty[i]), 1);
      mbar_init(smem_u32(&r_full[i]), 1);
      mbar_init(smem_u32(&r_empty[i]), NXF);
    }
    for (int i = 0; i < NA_ST; ++i) {
      mbar_init(smem_u32(&a_full[i]), NXF);
      mbar_init(smem_u32(&a_empty[i]), 1);
    }
    for (int i = 0; i < kParts; ++i) {
      mbar_init(smem_u32(&seg_full[i]), 1);
      mbar_init(smem_u32(&fold_done[i]), NFOLD);
    }
    mbar_init(smem_u32(mma_done), 1);
    *abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 2) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], 512;" ::"r"(smem_u32(tmem_slot)));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem_base = *tmem_slot;

  if (warp == 0) {
    // ---------------- TMA producer --------------------------------------------------------
    if (lane == 0) {
      long long C = 0, issued = 0;  // chunks whose copies were issued (all of them / at least the B copy)
      bool ok = true;
      int g = 0;
      for (int it = blockIdx.x; it < p.n_items && ok; it += gridDim.x) {
        Item x;
        if (!decode_item(gs, n_groups, it, g, x)) continue;
        const Chi0Group& G = gs[x.g];
        const uint32_t b_bytes = G.split3 ? 2 * TILE : TILE;
        for (int kc = 0; kc < G.n_kc; ++kc, ++C) {
          const int s = (int)(C % NB_ST);
          const uint32_t u = (uint32_t)(C / NB_ST);
          if (!mbar_wait(smem_u32(&b_empty[s]), (u & 1) ^ 1, abort_flag, p.wait_ns)) {
            ok = false;
            break;
          }
          mbar_expect_tx(smem_u32(&b_full[s]), b_bytes);
          uint8_t* bd = b_ring + s * 2 * TILE;
          tma_load_2d(smem_u32(bd), &G.tm_hi, kc * BK, x.Q0, smem_u32(&b_full[s]));
          if (G.split3) tma_load_2d(smem_u32(bd + TILE), &G.tm_lo, kc * BK, x.Q0, smem_u32(&b_full[s]));
          issued = C + 1;
          if (!mbar_wait(smem_u32(&r_empty[s]), (u & 1) ^ 1, abort_flag, p.wait_ns)) {
            ok = false;  // the B copy of this chunk is in flight
            break;
          }
          mbar_expect_tx(smem_u32(&r_full[s]), RAW + x.n_parts * BK * 4);
          uint8_t* rd = r_ring + s * RAW;
          tma_load_2d(smem_u32(rd), &G.tm_raw, kc * BK, x.P0, smem_u32(&r_full[s]));
          tma_load_2d(smem_u32(rd + RAW / 2), &G.tm_raw, kc * BK + 32, x.P0, smem_u32(&r_full[s]));
          for (int part = 0; part < x.n_parts; ++part) {
            const int f = x.f0 + part / G.ppf, comp = part % G.ppf;
            bulk_load(smem_u32(d_ring + (s * kParts + part) * BK), G.dtab + ((size_t)f * 2 + comp) * G.ld_dtab + kc * BK,
                      BK * 4, smem_u32(&r_full[s]));
          }
        }
      }
      // no copy may still be writing shared memory when the CTA exits
      for (long long c = issued > NB_ST ? issued - NB_ST : 0; c < issued; ++c) {
        mbar_drain(smem_u32(&b_full[c % NB_ST]), (uint32_t)(c / NB_ST) & 1);
        mbar_drain(smem_u32(&r_full[c % NB_ST]), (uint32_t)(c / NB_ST) & 1);
      }
    }
  } else if (warp == 1) {
    // ---------------- MMA issuer ------------------------------------------------------------
    if (lane == 0) {
      long long C = 0, a = 0;
      long long segc0 = 0, segc1 = 0;  // segments started per part (scalars: no local-memory array)
      bool ok = true;
      int g = 0;
      for (int it = blockIdx.x; it < p.n_items && ok; it += gridDim.x) {
        Item x;
        if (!decode_item(gs, n_groups, it, g, x)) continue;
        const Chi0Group& G = gs[x.g];
        const bool split3 = G.split3 != 0;
        for (int kc = 0; kc < G.n_kc && ok; ++kc, ++C) {
          const int s = (int)(C % NB_ST);
          const uint32_t u = (uint32_t)(C / NB_ST);
          if (!mbar_wait(smem_u32(&b_full[s]), u & 1, abort_flag, p.wait_ns)) {
            ok = false;
            break;
          }
          tc_fence_after();
          const uint32_t bh = smem_u32(b_ring + s * 2 * TILE), bl = bh + TILE;
          const bool seg_start = (kc % kSeg) == 0;
          const bool seg_end = (kc % kSeg) == kSeg - 1 || kc == G.n_kc - 1;
          for (int part = 0; part < x.n_parts; ++part, ++a) {
            const int t = (int)(a % NA_ST);
            const uint32_t ua = (uint32_t)(a / NA_ST);
            // a new segment overwrites this part's fresh accumulator: its previous fold must be done
            if (seg_start) {
              const long long sc = part ? segc1 : segc0;
              if (sc > 0 && !mbar_wait(smem_u32(&fold_done[part]), (uint32_t)(sc - 1) & 1, abort_flag, p.wait_ns)) {
                ok = false;
                break;
              }
              if (part) ++segc1; else ++segc0;
            }
            if (!mbar_wait(smem_u32(&a_full[t]), ua & 1, abort_flag, p.wait_ns)) {
              ok = false;
              break;
            }
            tc_fence_after();
            const uint32_t ah = smem_u32(a_ring + t * 2 * TILE), al = ah + TILE;
            const uint32_t d = tmem_base + (uint32_t)(part * BN);  // fresh accumulator of this part
            // descriptors once; a k step moves the start address by 32 bytes = 2 units of the
            // 16-byte address field (few instructions per MMA for the issuing thread)
            const uint64_t dah = sdesc(ah), dal = sdesc(al), dbh = sdesc(bh), dbl = sdesc(bl);
#pragma unroll
            for (int k = 0; k < BK / 16; ++k) {
              const uint64_t o = 2u * k;  // 16 BF16 = 32 bytes along K inside the 128-B row
              const uint32_t acc = (seg_start && k == 0) ? 0u : 1u;
              mma_bf16(d, dah + o, dbh + o, acc);
              if (split3) {
                mma_bf16(d, dah + o, dbl + o, 1u);
                mma_bf16(d, dal + o, dbh + o, 1u);
              }
            }
            mma_commit(smem_u32(&a_empty[t]));
            if (seg_end) mma_commit(smem_u32(&seg_full[part]));  // the fold of this part may start
          }
          if (!ok) break;
          mma_commit(smem_u32(&b_empty[s]));
        }
      }
      mma_commit(smem_u32(mma_done));  // fires when every MMA issued above has completed
    }
  } else if (transform_rank(warp) >= 0) {
    // ---------------- transform: A = O[P][k] D_p(k), split into BF16 hi / lo -------------------
    const int tt = 32 * transform_rank(warp) + lane;
    const int r = tt & 127, h = tt >> 7;  // row of the P tile, half of the 64-wide chunk
    long long C = 0, a = 0;
    bool ok = true;
    int g = 0;
    for (int it = blockIdx.x; it < p.n_items && ok; it += gridDim.x) {
      Item x;
      if (!decode_item(gs, n_groups, it, g, x)) continue;
      const Chi0Group& G = gs[x.g];
      for (int kc = 0; kc < G.n_kc; ++kc, ++C) {
        const int s = (int)(C % NB_ST);
        const uint32_t u = (uint32_t)(C / NB_ST);
        if (!mbar_wait(smem_u32(&r_full[s]), u & 1, abort_flag, p.wait_ns)) {
          ok = false;
          break;
        }
        float raw[32];
        const uint8_t* rrow = r_ring + s * RAW + h * (RAW / 2) + r * 128;
#pragma unroll
        for (int c = 0; c < 8; ++c) {  // 16-byte chunk c (4 floats) of this half, swizzled by row%8
          float4 v = *reinterpret_cast<const float4*>(rrow + ((c ^ (r & 7)) << 4));
          raw[4 * c] = v.x;
          raw[4 * c + 1] = v.y;
          raw[4 * c + 2] = v.z;
          raw[4 * c + 3] = v.w;
        }
        for (int part = 0; part < x.n_parts; ++part, ++a) {
          const int t = (int)(a % NA_ST);
          const uint32_t ua = (uint32_t)(a / NA_ST);
          if (!mbar_wait(smem_u32(&a_empty[t]), (ua & 1) ^ 1, abort_flag, p.wait_ns)) {
            ok = false;
            break;
          }
          const float4* ds = reinterpret_cast<const float4*>(d_ring + (s * kParts + part) * BK + 32 * h);  // broadcast
          uint8_t* ah = a_ring + t * 2 * TILE + r * 128;
          uint8_t* al = ah + TILE;
#pragma unroll
          for (int c = 0; c < 4; ++c) {  // 16-byte chunk 4h + c = 8 BF16 values k = 32h + 8c .. +7
            const float4 d0 = ds[2 * c], d1 = ds[2 * c + 1];
            const float v[8] = {raw[8 * c] * d0.x,     raw[8 * c + 1] * d0.y, raw[8 * c + 2] * d0.z, raw[8 * c + 3] * d0.w,
                                raw[8 * c + 4] * d1.x, raw[8 * c + 5] * d1.y, raw[8 * c + 6] * d1.z, raw[8 * c + 7] * d1.w};
            uint32_t hw[4], lw[4];
#pragma unroll
            for (int e = 0; e < 4; ++e) {
              hw[e] = pack_bf16x2(v[2 * e], v[2 * e + 1]);
              __nv_bfloat162 hb = *reinterpret_cast<__nv_bfloat162*>(&hw[e]);
              float2 hf = __bfloat1622float2(hb);
              lw[e] = pack_bf16x2(v[2 * e] - hf.x, v[2 * e + 1] - hf.y);
            }
            const int chunk = (4 * h + c) ^ (r & 7);  // SWIZZLE_128B: 16-B chunk index XOR row%8
            *reinterpret_cast<uint4*>(ah + chunk * 16) = make_uint4(hw[0], hw[1], hw[2], hw[3]);
            if (G.split3) *reinterpret_cast<uint4*>(al + chunk * 16) = make_uint4(lw[0], lw[1], lw[2], lw[3]);
          }
          asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
          mbar_arrive(smem_u32(&a_full[t]));
        }
        if (!ok) break;
        mbar_arrive(smem_u32(&r_empty[s]));  // raw rows and D slices of this stage are consumed
      }
    }
  } else if (warp >= 12) {
    // ---------------- fold + epilogue: running += fresh (FP32, round to nearest) -------------
    const int q = warp & 3;
    const int row = 32 * q + lane;
    const uint32_t lane_base = tmem_base + ((uint32_t)(32 * q) << 16);
    long long segf0 = 0, segf1 = 0;  // segments folded per part
    bool ok = true;
    int g = 0;
    for (int it = blockIdx.x; it < p.n_items && ok; it += gridDim.x) {
      Item x;
      if (!decode_item(gs, n_groups, it, g, x)) continue;
      const Chi0Group& G = gs[x.g];
      const int P = x.P0 + row;
      const int n_seg = (G.n_kc + kSeg - 1) / kSeg;
      for (int seg = 0; seg < n_seg && ok; ++seg) {
        const bool last = seg == n_seg - 1;
        if (!last) {
          for (int part = 0; part < x.n_parts; ++part) {
            ok = mbar_wait(smem_u32(&seg_full[part]), (uint32_t)(part ? segf1 : segf0) & 1, abort_flag, p.wait_ns);
            ok = __all_sync(0xffffffffu, ok);
            if (!ok) break;
            tc_fence_after();
            // 32 columns per round trip: the fresh and running slices are loaded, then one wait
            for (int cc = 0; cc < BN / 16; cc += 2) {
              const uint32_t fa = lane_base + (uint32_t)(part * BN + cc * 16), ra = fa + (uint32_t)(2 * BN);
              uint32_t f0[16], f1[16];
              float s0[16], s1[16];
              tmem_ld16_async(fa, f0);
              tmem_ld16_async(fa + 16, f1);
              if (seg > 0) {
                uint32_t r0[16], r1[16];
                tmem_ld16_async(ra, r0);
                tmem_ld16_async(ra + 16, r1);
                tmem_wait_ld();
#pragma unroll
                for (int i = 0; i < 16; ++i) {
                  s0[i] = __uint_as_float(f0[i]) + __uint_as_float(r0[i]);
                  s1[i] = __uint_as_float(f1[i]) + __uint_as_float(r1[i]);
                }
              } else {
                tmem_wait_ld();
#pragma unroll
                for (int i = 0; i < 16; ++i) {
                  s0[i] = __uint_as_float(f0[i]);
                  s1[i] = __uint_as_float(f1[i]);
                }
              }
              tmem_st16(ra, s0);
              tmem_st16(ra + 16, s1);
            }
            tmem_wait_st();
            tc_fence_before();
            mbar_arrive(smem_u32(&fold_done[part]));
            if (part) ++segf1; else ++segf0;
          }
        } else {
          for (int part = 0; part < x.n_parts && ok; ++part) {
            ok = mbar_wait(smem_u32(&seg_full[part]), (uint32_t)(part ? segf1 : segf0) & 1, abort_flag, p.wait_ns);
            ok = __all_sync(0xffffffffu, ok);
          }
          if (!ok) break;
          tc_fence_after();
          // final fold fused with the store: per frequency, 16 columns at a time, 16-byte stores
          const int nfl = x.n_parts / G.ppf;
          for (int fl = 0; fl < nfl; ++fl) {
            const int f = x.f0 + fl;
            const bool write = (!G.active || G.active[f]) && P < G.n_aux;
            for (int cc = 0; cc < BN / 16; ++cc) {
              float v[CPLX ? 2 : 1][16];
              {  // the fresh (and running) slices of both parts, then one wait
                uint32_t fr[CPLX ? 2 : 1][16];
                const uint32_t fa = lane_base + (uint32_t)(fl * G.ppf * BN + cc * 16);
#pragma unroll
                for (int comp = 0; comp < (CPLX ? 2 : 1); ++comp) tmem_ld16_async(fa + (uint32_t)(comp * BN), fr[comp]);
                if (seg > 0) {
                  uint32_t rn[CPLX ? 2 : 1][16];
#pragma unroll
                  for (int comp = 0; comp < (CPLX ? 2 : 1); ++comp)
                    tmem_ld16_async(fa + (uint32_t)((2 + comp) * BN), rn[comp]);
                  tmem_wait_ld();
#pragma unroll
                  for (int comp = 0; comp < (CPLX ? 2 : 1); ++comp)
#pragma unroll
                    for (int i = 0; i < 16; ++i) v[comp][i] = __uint_as_float(fr[comp][i]) + __uint_as_float(rn[comp][i]);
                } else {
                  tmem_wait_ld();
#pragma unroll
                  for (int comp = 0; comp < (CPLX ? 2 : 1); ++comp)
#pragma unroll
                    for (int i = 0; i < 16; ++i) v[comp][i] = __uint_as_float(fr[comp][i]);
                }
              }
              if (!write) continue;
              const int qb = x.Q0 + cc * 16;
              const bool full = qb + 15 < G.n_aux && qb + 15 <= P;  // every column of the chunk is stored
#pragma unroll
              for (int i = 0; i < 16; ++i) {
                const float dg = (P == qb + i) ? G.beta : 0.0f;
                v[0][i] = G.alpha * v[0][i] + dg;
                if (CPLX) v[CPLX ? 1 : 0][i] = G.alpha * v[CPLX ? 1 : 0][i];
              }
              if (G.out64) {  // FP64 matrices (FP64 factorisation): the FP32 sums widened exactly
                if (CPLX) {
                  double2* o = reinterpret_cast<double2*>(G.out) + f * G.mat_stride + (long long)P * G.ldm + qb;
                  for (int i = 0; i < 16; ++i)
                    if (full || (qb + i < G.n_aux && qb + i <= P))
                      o[i] = make_double2((double)v[0][i], (double)v[CPLX ? 1 : 0][i]);
                } else {
                  double* o = reinterpret_cast<double*>(G.out) + f * G.mat_stride + (long long)P * G.ldm + qb;
                  for (int i = 0; i < 16; ++i)
                    if (full || (qb + i < G.n_aux && qb + i <= P)) o[i] = (double)v[0][i];
                }
              } else if (CPLX) {
                float2* o = reinterpret_cast<float2*>(G.out) + f * G.mat_stride + (long long)P * G.ldm + qb;
                if (full) {
#pragma unroll
                  for (int i = 0; i < 16; i += 2)
                    *reinterpret_cast<float4*>(o + i) = make_float4(v[0][i], v[CPLX ? 1 : 0][i], v[0][i + 1], v[CPLX ? 1 : 0][i + 1]);
                } else {
                  for (int i = 0; i < 16; ++i)
                    if (qb + i < G.n_aux && qb + i <= P) o[i] = make_float2(v[0][i], v[CPLX ? 1 : 0][i]);
                }
              } else {
                float* o = reinterpret_cast<float*>(G.out) + f * G.mat_stride + (long long)P * G.ldm + qb;
                if (full) {
#pragma unroll
                  for (int i = 0; i < 16; i += 4)
                    *reinterpret_cast<float4*>(o + i) = make_float4(v[0][i], v[0][i + 1], v[0][i + 2], v[0][i + 3]);
                } else {
                  for (int i = 0; i < 16; ++i)
                    if (qb + i < G.n_aux && qb + i <= P) o[i] = v[0][i];
                }
              }
            }
          }
          // the accumulators of this item are read: the next item's first segment may overwrite them
          tc_fence_before();
          for (int part = 0; part < x.n_parts; ++part) {
            mbar_arrive(smem_u32(&fold_done[part]));
            if (part) ++segf1; else ++segf0;
          }
        }
      }
    }
  }
  // drain: every issued MMA completes before TMEM is freed (immediate on the normal path)
  if (warp == 2) {
    if (lane == 0) mbar_drain(smem_u32(mma_done), 0);
    __syncwarp();
  }
  tc_fence_before();
  __syncthreads();
  if (threadIdx.x == 0 && *abort_flag) atomicOr(p.status, kStatTimeout);
  if (warp == 2) {
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, 512;" ::"r"(tmem_base));
  }
}

}  // namespace

namespace {

// Fills one group descriptor; false if the shape or alignment is not supported by the kernel.
bool fill_group(Chi0Group* G, bool split3, const __nv_bfloat16* o_hi, const __nv_bfloat16* o_lo, const float* o_f32,
                int ld_pad, int n_aux, int n_aux_pad, int n_ov_pad, const float* dtab, int ld_dtab, int F, bool complex_out,
                double alpha, double beta, void* out, long long ldm, long long mat_stride, const int* active, bool out64,
                int item0) {
  if (n_aux_pad % BM || n_ov_pad % BK || ld_pad != n_ov_pad || ld_dtab % BK || F < 1) return false;
  // TMA: 16-B aligned bases, row strides multiples of 16 B, x coordinates multiples of 64 / 32
  if ((reinterpret_cast<uintptr_t>(o_hi) & 15) || (reinterpret_cast<uintptr_t>(o_lo) & 15) ||
      (reinterpret_cast<uintptr_t>(o_f32) & 15) || (reinterpret_cast<uintptr_t>(dtab) & 15))
    return false;
  std::memset(static_cast<void*>(G), 0, sizeof(Chi0Group));
  if (!make_map(&G->tm_hi, o_hi, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, n_aux_pad, n_ov_pad, BK, BM) ||
      !make_map(&G->tm_lo, o_lo, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, n_aux_pad, n_ov_pad, BK, BM) ||
      !make_map(&G->tm_raw, o_f32, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 4, n_aux_pad, n_ov_pad, 32, BM))
    return false;
  const int nt = n_aux_pad / BM;
  G->dtab = dtab;
  G->out = out;
  G->active = active;
  G->ldm = ldm;
  G->mat_stride = mat_stride;
  G->ld_dtab = ld_dtab;
  G->n_aux = n_aux;
  G->n_kc = n_ov_pad / BK;
  G->F = F;
  G->ppf = complex_out ? 2 : 1;
  G->fpc = kParts / G->ppf;
  G->n_tiles = nt * (nt + 1) / 2;
  G->item0 = item0;
  G->n_items = G->n_tiles * ((F + G->fpc - 1) / G->fpc);
  G->split3 = split3 ? 1 : 0;
  G->out64 = out64 ? 1 : 0;
  G->alpha = (float)alpha;
  G->beta = (float)beta;
  return true;
}

template <bool CPLX, bool GROUPED>
int launch_kernel(const Chi0Group& own, const TcParams& p, int grid, cudaStream_t s) {
  static bool attr = false;
  if (!attr) {
    if (cudaFuncSetAttribute(chi0_tc_kernel<CPLX, GROUPED>, cudaFuncAttributeMaxDynamicSharedMemorySize, SMEM_BYTES) !=
        cudaSuccess)
      return -1;
    attr = true;
  }
  chi0_tc_kernel<CPLX, GROUPED><<<grid, NTHREADS, SMEM_BYTES, s>>>(own, p);
  return cudaPeekAtLastError() == cudaSuccess ? 1 : -1;
}

}  // namespace

// Returns launches (1), -1 on a launch error, -2 if unsupported (device or shape). persist = 0: one CTA per
// (tile, frequency group) item; > 0: at most that many CTAs, each looping over items.
int launch_chi0_tc(bool split3, const __nv_bfloat16* o_hi, const __nv_bfloat16* o_lo, const float* o_f32, int ld_pad,
                   int n_aux, int n_aux_pad, int n_ov_pad, const float* dtab, int ld_dtab, int F, bool complex_out,
                   double alpha, double beta, void* out, long long ldm, long long mat_stride, const int* active,
                   unsigned* status, unsigned long long wait_ns, bool out64, cudaStream_t s, int persist) {
  if (!tc_supported()) return -2;
  Chi0Group G;
  if (!fill_group(&G, split3, o_hi, o_lo, o_f32, ld_pad, n_aux, n_aux_pad, n_ov_pad, dtab, ld_dtab, F, complex_out, alpha,
                  beta, out, ldm, mat_stride, active, out64, 0))
    return -2;
  TcParams p;
  p.groups = nullptr;
  p.n_groups = 1;
  p.n_items = G.n_items;
  p.status = status;
  p.wait_ns = wait_ns;
  const int grid = persist > 0 ? std::min(persist, G.n_items) : G.n_items;
  return complex_out ? launch_kernel<true, false>(G, p, grid, s) : launch_kernel<false, false>(G, p, grid, s);
}

size_t chi0_group_bytes() { return sizeof(Chi0Group); }

int chi0_group_fill(void* dst, bool split3, const __nv_bfloat16* o_hi, const __nv_bfloat16* o_lo, const float* o_f32,
                    int ld_pad, int n_aux, int n_aux_pad, int n_ov_pad, const float* dtab, int ld_dtab, int F,
                    bool complex_out, double alpha, double beta, void* out, long long ldm, long long mat_stride,
                    const int* active, bool out64, int item0) {
  Chi0Group G;  // aligned for the tensor-map encoder; dst may be any byte buffer
  if (!fill_group(&G, split3, o_hi, o_lo, o_f32, ld_pad, n_aux, n_aux_pad, n_ov_pad, dtab, ld_dtab, F, complex_out, alpha,
                  beta, out, ldm, mat_stride, active, out64, item0))
    return -2;
  std::memcpy(dst, &G, sizeof(G));
  return G.n_items;
}

int launch_chi0_tc_grouped(const void* d_groups, int n_groups, int n_items, bool complex_out, int grid, unsigned* status,
                           unsigned long long wait_ns, cudaStream_t s) {
  if (!tc_supported()) return -2;
  if (n_groups < 1 || n_items < 1 || grid < 1 || (reinterpret_cast<uintptr_t>(d_groups) & 63)) return -1;
  TcParams p;
  p.groups = static_cast<const Chi0Group*>(d_groups);
  p.n_groups = n_groups;
  p.n_items = n_items;
  p.status = status;
  p.wait_ns = wait_ns;
  Chi0Group unused;
  std::memset(static_cast<void*>(&unused), 0, sizeof(unused));
  grid = std::min(grid, n_items);
  return complex_out ? launch_kernel<true, true>(unused, p, grid, s) : launch_kernel<false, true>(unused, p, grid, s);
}

}  // namespace gwc
