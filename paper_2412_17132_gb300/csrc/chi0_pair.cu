// Tensor-core polarizability build on CTA pairs (tcgen05 cta_group::2, sm_103a).
//
//   Pi_PQ(z_f) = sum_k O_Pk D_f(k) O_Qk      (RI polarizability, Sec. "Self-energy evaluation")
//
// The same contraction as chi0_tc.cu, on a 2-CTA cluster that shares one MMA: the pair computes a
// 256 x 128 tile (P rows 256, Q columns 128) of the lower triangle for two frequency parts. Each
// tcgen05.mma (M = 256, N = 128, K = 16, kind::f16) is issued by CTA 0 and reads, in each CTA's own
// shared memory, 128 rows of the A operand and 64 rows of the B operand (read once for both tensor
// cores); each CTA's TMEM receives its 128 rows of the accumulator. Per CTA and chunk the transform
// scales half the rows of the one-CTA kernel, and the MMA reads 144 KB of shared memory instead of 192 KB.
//
//   * A = O[P-rows of this CTA][k] (BF16 hi, lo), static: TMA, SWIZZLE_128B, K-major.
//   * B = O[Q][k] D_p(k) split into BF16 hi and lo, per part: each CTA scales its 64 Q rows (FP32 rows
//     brought by TMA, D slices by bulk copies), four transform threads per row.
//   * CTA 0's warp 1 runs the MMA loop (one elected lane issues) and signals both CTAs through multicast
//     commits (slot release, segment complete, all done). The transform and fold warps of both CTAs
//     arrive on CTA 0's barriers directly (one arrive per warp); CTA 1's warp 1 relays the completion of
//     its A copies. The arrives use CTA-scope release: a cluster-scope release costs about 870 cycles per
//     arrive on a GB300 (measured) and, done per warp and part, halved the transform rate.
//   * Segmented accumulation and the fold/epilogue are those of chi0_tc.cu, per CTA on its own TMEM
//     rows: each part accumulates kSeg chunks in a fresh accumulator, fold warps add it into a running
//     FP32 sum (round to nearest) while the other part's MMAs run, and the last fold writes
//     alpha * Pi + beta * I (lower triangle) to global memory.
//
// Every wait is bounded; a CTA that gives up raises its own and its peer's abort flag, both stop issuing,
// drain their copies and MMAs, meet at a cluster barrier (so that neither leaves while the other may still
// signal it) and free TMEM.
#include <cuda.h>

#include <algorithm>
#include <cstring>

#include "gwc_internal.h"
#include "tc_common.cuh"

namespace gwc {

namespace {

constexpr int BMC = 128;                // P rows per CTA (256 per pair)
constexpr int BNC = 64;                 // Q rows of the B operand per CTA (128 per pair)
constexpr int BNP = 128;                // accumulator columns
constexpr int BK = 64;
constexpr int kParts = 2;
constexpr int kSeg = 8;
constexpr int ATILE = BMC * BK * 2;     // 16 KB: BF16 128 x 64
constexpr int XTILE = BNC * BK * 2;     // 8 KB: BF16 64 x 64
constexpr int RAWP = BNC * BK * 4;      // 16 KB: FP32 64 x 64 as two 128-B swizzled halves
constexpr int DSL = kParts * BK * 4;
constexpr int NTHREADS = 512;           // warp 0 TMA, 1 MMA (CTA 0) / relay (CTA 1), 12-15 fold
constexpr int NXW = 8;                  // transform warps, none on warp 1's scheduler
constexpr int NFW = 4;                  // fold warps
// NS: A / raw / D ring stages; NX: scaled-B slots (one part each). Measured at the pentacene width: (3, 4)
// 11.9 ms per 8 frequencies, (3, 5) 12.4 ms, (2, 8) 14.7 ms.
constexpr int NS = 3, NX = 4;
constexpr int smem_bytes(int ns, int nx) { return 1024 + ns * 2 * ATILE + ns * RAWP + nx * 2 * XTILE + ns * DSL + 512; }

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

struct Chi0PairGroup {
  CUtensorMap tm_hi, tm_lo, tm_raw;  // A operand (BF16 hi, lo; box 64 x 128) and FP32 rows (box 32 x 64)
  const float* dtab;
  void* out;
  const int* active;
  long long ldm, mat_stride;
  int ld_dtab;
  int n_aux;
  int n_kc;
  int F;
  int ppf;
  int fpc;
  int n_pb;       // 256-row P blocks
  int n_qb;       // 128-column Q blocks
  int n_tiles;    // pair tiles of the lower triangle
  int item0;
  int n_items;
  int split3;
  int out64;
  float alpha, beta;
};

struct PairParams {
  const Chi0PairGroup* groups;
  int n_groups;
  int n_items;
  unsigned* status;
  unsigned long long wait_ns;
};

// kind::f16, D = F32, A = B = BF16, K-major, M = 256 (pair), N = 128.
constexpr uint32_t kIdesc2 = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(BNP >> 3) << 17) | ((uint32_t)(256 >> 4) << 24);

__device__ __forceinline__ void mma2_bf16(uint32_t d_tmem, uint64_t a, uint64_t b, uint32_t accum) {
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "setp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::2.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(d_tmem),
      "l"(a), "l"(b), "r"(kIdesc2), "r"(accum));
}

// arrives on the barrier at this offset in both CTAs of the pair once the MMAs issued so far complete
__device__ __forceinline__ void commit_both(uint32_t bar) {
  asm volatile(
      "tcgen05.commit.cta_group::2.mbarrier::arrive::one.shared::cluster.multicast::cluster.b64 [%0], %1;" ::"r"(bar),
      "h"((unsigned short)3)
      : "memory");
}

// true in one lane of the (converged) warp
__device__ __forceinline__ bool elect_one() {
  uint32_t pred;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "elect.sync _|p, 0xffffffff;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(pred));
  return pred != 0;
}

__device__ __forceinline__ uint32_t peer_addr(uint32_t local, uint32_t rank) {
  uint32_t r;
  asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(r) : "r"(local), "r"(rank));
  return r;
}

// Arrive on a barrier of either CTA of the pair (default semantics: release at CTA scope). A release at
// cluster scope costs about 870 cycles per arrive on a GB300 (measured), half the transform warps' time.
__device__ __forceinline__ void remote_arrive(uint32_t cluster_addr) {
  asm volatile("mbarrier.arrive.shared::cluster.b64 _, [%0];" ::"r"(cluster_addr) : "memory");
}

__device__ __forceinline__ void cluster_sync() {
  asm volatile("barrier.cluster.arrive.release.aligned;\n\tbarrier.cluster.wait.acquire.aligned;" ::: "memory");
}

__device__ __forceinline__ uint32_t cta_rank() {
  uint32_t r;
  asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
  return r;
}

// Bounded wait; on expiry both CTAs' abort flags are raised. A bound shorter than the default: each try
// suspends at most a quarter of it and the clock is read after every try.
__device__ __forceinline__ bool pwait(uint32_t bar, uint32_t parity, volatile int* abort_flag, uint32_t peer_abort,
                                      unsigned long long limit_ns) {
  if (mbar_try(bar, parity)) return true;
  const unsigned long long t0 = gtime();
  const bool short_bound = limit_ns < kWaitNs;
  const uint32_t hint = (uint32_t)(limit_ns / 4 + 1);
  for (uint32_t it = 0;; ++it) {
    if (short_bound ? mbar_try_hint(bar, parity, hint) : mbar_try(bar, parity)) return true;
    if (short_bound || (it & 63u) == 63u) {
      if (*abort_flag) return false;
      if (gtime() - t0 > limit_ns) {
        *abort_flag = 1;
        asm volatile("st.shared::cluster.u32 [%0], %1;" ::"r"(peer_abort), "r"(1) : "memory");
        return false;
      }
    }
  }
}

// Exit drain of a copy phase, bounded by 1 ms (copies land within microseconds; on CTA 0 an a_full phase
// also needs CTA 1's relay, which never comes after an abort)
__device__ __forceinline__ void pdrain(uint32_t bar, uint32_t parity) {
  const unsigned long long t0 = gtime();
  for (uint32_t it = 0;; ++it) {
    if (mbar_try(bar, parity)) return;
    if ((it & 63u) == 63u && gtime() - t0 > 1000000ull) return;
  }
}

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

struct Item {
  int g, P0, Q0, f0, nf, n_parts;
};

// pair tile t -> (P block, Q block): P block ip holds Q blocks 0 .. 2 ip + 1 (the last one up to n_qb - 1)
__device__ __forceinline__ void pair_tile(int t, int n_pb, int& ip, int& iq) {
  int a = (int)((sqrt(4.0 * t + 1.0) - 1.0) * 0.5);
  while ((a + 1) * (a + 2) <= t) ++a;
  while (a * (a + 1) > t) --a;
  if (a > n_pb - 1) a = n_pb - 1;
  ip = a;
  iq = t - a * (a + 1);
}

__device__ __forceinline__ bool decode_item(const Chi0PairGroup* gs, int n_groups, int it, int& g, Item& x) {
  while (g + 1 < n_groups && it >= gs[g + 1].item0) ++g;
  const Chi0PairGroup& G = gs[g];
  const int local = it - G.item0;
  const int t = local % G.n_tiles, fgi = local / G.n_tiles;
  int ip, iq;
  pair_tile(t, G.n_pb, ip, iq);
  x.g = g;
  x.P0 = ip * 2 * BMC;
  x.Q0 = iq * BNP;
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

template <bool CPLX, bool GROUPED>
__global__ void __cluster_dims__(2, 1, 1) __launch_bounds__(NTHREADS, 1)
    chi0_pair_kernel(const __grid_constant__ Chi0PairGroup g_own, PairParams p) {
  extern __shared__ uint8_t smem_raw[];
  uint8_t* base = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~(uintptr_t)1023);
  uint8_t* a_ring = base;                           // NS x [hi | lo], 128 rows
  uint8_t* r_ring = a_ring + NS * 2 * ATILE;        // NS x [k 0..31 | k 32..63] FP32, 64 rows
  uint8_t* x_ring = r_ring + NS * RAWP;             // NX x [hi | lo], 64 rows
  float* d_ring = reinterpret_cast<float*>(x_ring + NX * 2 * XTILE);  // NS x [part][64]
  uint64_t* bars = reinterpret_cast<uint64_t*>(d_ring + NS * kParts * BK);
  uint64_t* a_full = bars;
  uint64_t* a_empty = a_full + NS;
  uint64_t* r_full = a_empty + NS;
  uint64_t* r_empty = r_full + NS;
  uint64_t* x_full = r_empty + NS;
  uint64_t* x_empty = x_full + NX;
  uint64_t* seg_full = x_empty + NX;
  uint64_t* fold_done = seg_full + kParts;
  uint64_t* mma_done = fold_done + kParts;
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(mma_done + 1);
  volatile int* abort_flag = reinterpret_cast<volatile int*>(tmem_slot + 1);

  const Chi0PairGroup* gs = GROUPED ? p.groups : &g_own;
  const int n_groups = GROUPED ? p.n_groups : 1;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const uint32_t rank = cta_rank();
  const bool lead = rank == 0;
  const int cid = blockIdx.x >> 1, n_cl = gridDim.x >> 1;
  if (cid >= p.n_items) return;  // uniform across the pair, before any barrier or TMEM use
  const uint32_t peer_abort = peer_addr(smem_u32((const void*)abort_flag), rank ^ 1u);

  if (threadIdx.x == 0) {
    for (int i = 0; i < NS; ++i) {
      mbar_init(smem_u32(&a_full[i]), lead ? 2 : 1);  // own copy (+ CTA 1's relay on CTA 0)
      mbar_init(smem_u32(&a_empty[i]), 1);
      mbar_init(smem_u32(&r_full[i]), 1);
      mbar_init(smem_u32(&r_empty[i]), NXW);
    }
    for (int i = 0; i < NX; ++i) {
      mbar_init(smem_u32(&x_full[i]), 2 * NXW);  // CTA 0: its own and CTA 1's transform warps
      mbar_init(smem_u32(&x_empty[i]), 1);
    }
    for (int i = 0; i < kParts; ++i) {
      mbar_init(smem_u32(&seg_full[i]), 1);
      mbar_init(smem_u32(&fold_done[i]), 2 * NFW);  // CTA 0: its own and CTA 1's fold warps
    }
    mbar_init(smem_u32(mma_done), 1);
    *abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 2) {  // one warp of each CTA allocates the pair's TMEM together
    asm volatile("tcgen05.alloc.cta_group::2.sync.aligned.shared::cta.b32 [%0], 512;" ::"r"(smem_u32(tmem_slot)));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::2.sync.aligned;");
  }
  tc_fence_before();
  cluster_sync();  // both CTAs' barriers are initialised before any remote arrive or multicast commit
  tc_fence_after();
  const uint32_t tmem_base = *tmem_slot;
  const unsigned long long wns = p.wait_ns;

  if (warp == 0) {
    // ---------------- TMA producer (each CTA its own rows) -------------------------------------
    if (lane == 0) {
      long long C = 0, issued = 0;
      bool ok = true;
      int g = 0;
      for (int it = cid; it < p.n_items && ok; it += n_cl) {
        Item x;
        if (!decode_item(gs, n_groups, it, g, x)) continue;
        const Chi0PairGroup& G = gs[x.g];
        const uint32_t a_bytes = G.split3 ? 2 * ATILE : ATILE;
        const int prow = x.P0 + (int)rank * BMC, qrow = x.Q0 + (int)rank * BNC;
        for (int kc = 0; kc < G.n_kc; ++kc, ++C) {
          const int s = (int)(C % NS);
          const uint32_t u = (uint32_t)(C / NS);
          if (!pwait(smem_u32(&a_empty[s]), (u & 1) ^ 1, abort_flag, peer_abort, wns)) {
            ok = false;
            break;
          }
          mbar_expect_tx(smem_u32(&a_full[s]), a_bytes);
          uint8_t* ad = a_ring + s * 2 * ATILE;
          tma_load_2d(smem_u32(ad), &G.tm_hi, kc * BK, prow, smem_u32(&a_full[s]));
          if (G.split3) tma_load_2d(smem_u32(ad + ATILE), &G.tm_lo, kc * BK, prow, smem_u32(&a_full[s]));
          issued = C + 1;
          if (!pwait(smem_u32(&r_empty[s]), (u & 1) ^ 1, abort_flag, peer_abort, wns)) {
            ok = false;
            break;
          }
          mbar_expect_tx(smem_u32(&r_full[s]), RAWP + x.n_parts * BK * 4);
          uint8_t* rd = r_ring + s * RAWP;
          tma_load_2d(smem_u32(rd), &G.tm_raw, kc * BK, qrow, smem_u32(&r_full[s]));
          tma_load_2d(smem_u32(rd + RAWP / 2), &G.tm_raw, kc * BK + 32, qrow, smem_u32(&r_full[s]));
          for (int part = 0; part < x.n_parts; ++part) {
            const int f = x.f0 + part / G.ppf, comp = part % G.ppf;
            bulk_load(smem_u32(d_ring + (s * kParts + part) * BK), G.dtab + ((size_t)f * 2 + comp) * G.ld_dtab + kc * BK,
                      BK * 4, smem_u32(&r_full[s]));
          }
        }
      }
      // no copy may still be writing shared memory when the CTA exits (on CTA 0 an a_full phase also
      // needs CTA 1's relay; after an abort the bounded drain covers a relay that never comes)
      for (long long c = issued > NS ? issued - NS : 0; c < issued; ++c) {
        const uint32_t par = (uint32_t)(c / NS) & 1;
        pdrain(smem_u32(&a_full[c % NS]), par);
        pdrain(smem_u32(&r_full[c % NS]), par);
      }
    }
  } else if (warp == 1) {
    if (lead) {
      // ---------------- MMA issuer (CTA 0) ----------------------------------------------------
      // The whole warp runs the loop (its bookkeeping and descriptors are warp-uniform); one elected
      // lane issues each MMA and commit.
      long long C = 0, a = 0;
      long long segc0 = 0, segc1 = 0;
      bool ok = true;
      int g = 0;
      for (int it = cid; it < p.n_items && ok; it += n_cl) {
        Item x;
        if (!decode_item(gs, n_groups, it, g, x)) continue;
        const Chi0PairGroup& G = gs[x.g];
        const bool split3 = G.split3 != 0;
        for (int kc = 0; kc < G.n_kc && ok; ++kc, ++C) {
          const int s = (int)(C % NS);
          const uint32_t u = (uint32_t)(C / NS);
          ok = __all_sync(0xffffffffu, pwait(smem_u32(&a_full[s]), u & 1, abort_flag, peer_abort, wns));
          if (!ok) break;
          tc_fence_after();
          const uint32_t ah = smem_u32(a_ring + s * 2 * ATILE), al = ah + ATILE;
          const bool seg_start = (kc % kSeg) == 0;
          const bool seg_end = (kc % kSeg) == kSeg - 1 || kc == G.n_kc - 1;
          for (int part = 0; part < x.n_parts; ++part, ++a) {
            const int t = (int)(a % NX);
            const uint32_t ua = (uint32_t)(a / NX);
            if (seg_start) {
              const long long sc = part ? segc1 : segc0;
              if (sc > 0) {
                ok = __all_sync(0xffffffffu, pwait(smem_u32(&fold_done[part]), (uint32_t)(sc - 1) & 1, abort_flag,
                                                   peer_abort, wns));
                if (!ok) break;
              }
              if (part) ++segc1; else ++segc0;
            }
            ok = __all_sync(0xffffffffu, pwait(smem_u32(&x_full[t]), ua & 1, abort_flag, peer_abort, wns));
            if (!ok) break;
            tc_fence_after();
            const uint32_t bh = smem_u32(x_ring + t * 2 * XTILE), bl = bh + XTILE;
            const uint32_t d = tmem_base + (uint32_t)(part * BNP);
            const uint64_t dah = sdesc(ah), dal = sdesc(al), dbh = sdesc(bh), dbl = sdesc(bl);
            if (elect_one()) {
#pragma unroll
              for (int k = 0; k < BK / 16; ++k) {
                const uint64_t o = 2u * k;
                mma2_bf16(d, dah + o, dbh + o, (seg_start && k == 0) ? 0u : 1u);
                if (split3) {
                  mma2_bf16(d, dah + o, dbl + o, 1u);
                  mma2_bf16(d, dal + o, dbh + o, 1u);
                }
              }
              commit_both(smem_u32(&x_empty[t]));
              if (seg_end) commit_both(smem_u32(&seg_full[part]));
            }
            __syncwarp();
          }
          if (!ok) break;
          if (elect_one()) commit_both(smem_u32(&a_empty[s]));
          __syncwarp();
        }
      }
      if (elect_one()) commit_both(smem_u32(mma_done));  // fires in both CTAs when every MMA above completed
      __syncwarp();
    } else if (lane == 0) {
      // ---------------- relay (CTA 1): its A tile of each chunk has landed -> CTA 0 -------------------
      long long C = 0;
      bool ok = true;
      int g = 0;
      for (int it = cid; it < p.n_items && ok; it += n_cl) {
        Item x;
        if (!decode_item(gs, n_groups, it, g, x)) continue;
        const Chi0PairGroup& G = gs[x.g];
        for (int kc = 0; kc < G.n_kc; ++kc, ++C) {
          if (!pwait(smem_u32(&a_full[C % NS]), (uint32_t)(C / NS) & 1, abort_flag, peer_abort, wns)) {
            ok = false;
            break;
          }
          remote_arrive(peer_addr(smem_u32(&a_full[C % NS]), 0));
        }
      }
    }
  } else if (transform_rank(warp) >= 0) {
    // ---------------- transform: B = O[Q][k] D_p(k) for this CTA's 64 Q rows, BF16 hi / lo ---------
    const int tt = 32 * transform_rank(warp) + lane;
    const int r = tt & 63, qt = tt >> 6;  // row of the Q half, quarter of the 64-wide chunk
    const int hh = qt >> 1, cb = 4 * (qt & 1);
    long long C = 0, a = 0;
    bool ok = true;
    int g = 0;
    for (int it = cid; it < p.n_items && ok; it += n_cl) {
      Item x;
      if (!decode_item(gs, n_groups, it, g, x)) continue;
      const Chi0PairGroup& G = gs[x.g];
      for (int kc = 0; kc < G.n_kc; ++kc, ++C) {
        const int s = (int)(C % NS);
        const uint32_t u = (uint32_t)(C / NS);
        ok = __all_sync(0xffffffffu, pwait(smem_u32(&r_full[s]), u & 1, abort_flag, peer_abort, wns));
        if (!ok) break;  // warp-uniform: the arrivals below are per warp
        float raw[16];
        const uint8_t* rrow = r_ring + s * RAWP + hh * (RAWP / 2) + r * 128;
#pragma unroll
        for (int j = 0; j < 4; ++j) {  // 16-byte chunk cb + j of this half, swizzled by row % 8
          const float4 v = *reinterpret_cast<const float4*>(rrow + (((cb + j) ^ (r & 7)) << 4));
          raw[4 * j] = v.x;
          raw[4 * j + 1] = v.y;
          raw[4 * j + 2] = v.z;
          raw[4 * j + 3] = v.w;
        }
        for (int part = 0; part < x.n_parts; ++part, ++a) {
          const int t = (int)(a % NX);
          const uint32_t ua = (uint32_t)(a / NX);
          ok = __all_sync(0xffffffffu, pwait(smem_u32(&x_empty[t]), (ua & 1) ^ 1, abort_flag, peer_abort, wns));
          if (!ok) break;
          const float4* ds = reinterpret_cast<const float4*>(d_ring + (s * kParts + part) * BK + 16 * qt);  // broadcast
          uint8_t* xh = x_ring + t * 2 * XTILE + r * 128;
#pragma unroll
          for (int e = 0; e < 2; ++e) {  // 16-byte chunk 2 qt + e = 8 BF16 values k = 16 qt + 8 e .. + 7
            const float4 d0 = ds[2 * e], d1 = ds[2 * e + 1];
            const float v[8] = {raw[8 * e] * d0.x,     raw[8 * e + 1] * d0.y, raw[8 * e + 2] * d0.z, raw[8 * e + 3] * d0.w,
                                raw[8 * e + 4] * d1.x, raw[8 * e + 5] * d1.y, raw[8 * e + 6] * d1.z, raw[8 * e + 7] * d1.w};
            uint32_t hw[4], lw[4];
#pragma unroll
            for (int q = 0; q < 4; ++q) {
              hw[q] = pack_bf16x2(v[2 * q], v[2 * q + 1]);
              __nv_bfloat162 hb = *reinterpret_cast<__nv_bfloat162*>(&hw[q]);
              float2 hf = __bfloat1622float2(hb);
              lw[q] = pack_bf16x2(v[2 * q] - hf.x, v[2 * q + 1] - hf.y);
            }
            const int chunk = (2 * qt + e) ^ (r & 7);  // SWIZZLE_128B
            *reinterpret_cast<uint4*>(xh + chunk * 16) = make_uint4(hw[0], hw[1], hw[2], hw[3]);
            if (G.split3) *reinterpret_cast<uint4*>(xh + XTILE + chunk * 16) = make_uint4(lw[0], lw[1], lw[2], lw[3]);
          }
          asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
          __syncwarp();
          if (lane == 0) remote_arrive(peer_addr(smem_u32(&x_full[t]), 0));  // CTA 0's barrier (own on CTA 0)
        }
        if (!ok) break;
        __syncwarp();
        if (lane == 0) mbar_arrive(smem_u32(&r_empty[s]));
      }
    }
  } else if (warp >= 12) {
    // ---------------- fold + epilogue on this CTA's 128 TMEM lanes ------------------------------
    const int q = warp & 3;
    const int row = 32 * q + lane;
    const uint32_t lane_base = tmem_base + ((uint32_t)(32 * q) << 16);
    long long segf0 = 0, segf1 = 0;
    bool ok = true;
    int g = 0;
    for (int it = cid; it < p.n_items && ok; it += n_cl) {
      Item x;
      if (!decode_item(gs, n_groups, it, g, x)) continue;
      const Chi0PairGroup& G = gs[x.g];
      const int P = x.P0 + (int)rank * BMC + row;
      const int n_seg = (G.n_kc + kSeg - 1) / kSeg;
      for (int seg = 0; seg < n_seg && ok; ++seg) {
        const bool last = seg == n_seg - 1;
        if (!last) {
          for (int part = 0; part < x.n_parts; ++part) {
            ok = pwait(smem_u32(&seg_full[part]), (uint32_t)(part ? segf1 : segf0) & 1, abort_flag, peer_abort, wns);
            ok = __all_sync(0xffffffffu, ok);
            if (!ok) break;
            tc_fence_after();
            for (int cc = 0; cc < BNP / 16; cc += 2) {
              const uint32_t fa = lane_base + (uint32_t)(part * BNP + cc * 16), ra = fa + (uint32_t)(2 * BNP);
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
            __syncwarp();
            if (lane == 0) remote_arrive(peer_addr(smem_u32(&fold_done[part]), 0));
            if (part) ++segf1; else ++segf0;
          }
        } else {
          for (int part = 0; part < x.n_parts && ok; ++part) {
            ok = pwait(smem_u32(&seg_full[part]), (uint32_t)(part ? segf1 : segf0) & 1, abort_flag, peer_abort, wns);
            ok = __all_sync(0xffffffffu, ok);
          }
          if (!ok) break;
          tc_fence_after();
          const int nfl = x.n_parts / G.ppf;
          for (int fl = 0; fl < nfl; ++fl) {
            const int f = x.f0 + fl;
            const bool write = (!G.active || G.active[f]) && P < G.n_aux;
            for (int cc = 0; cc < BNP / 16; ++cc) {
              float v[CPLX ? 2 : 1][16];
              {
                uint32_t fr[CPLX ? 2 : 1][16];
                const uint32_t fa = lane_base + (uint32_t)(fl * G.ppf * BNP + cc * 16);
#pragma unroll
                for (int comp = 0; comp < (CPLX ? 2 : 1); ++comp) tmem_ld16_async(fa + (uint32_t)(comp * BNP), fr[comp]);
                if (seg > 0) {
                  uint32_t rn[CPLX ? 2 : 1][16];
#pragma unroll
                  for (int comp = 0; comp < (CPLX ? 2 : 1); ++comp)
                    tmem_ld16_async(fa + (uint32_t)((2 + comp) * BNP), rn[comp]);
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
              const bool full = qb + 15 < G.n_aux && qb + 15 <= P;
#pragma unroll
              for (int i = 0; i < 16; ++i) {
                const float dg = (P == qb + i) ? G.beta : 0.0f;
                v[0][i] = G.alpha * v[0][i] + dg;
                if (CPLX) v[CPLX ? 1 : 0][i] = G.alpha * v[CPLX ? 1 : 0][i];
              }
              if (G.out64) {
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
                    *reinterpret_cast<float4*>(o + i) =
                        make_float4(v[0][i], v[CPLX ? 1 : 0][i], v[0][i + 1], v[CPLX ? 1 : 0][i + 1]);
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
          tc_fence_before();
          __syncwarp();
          for (int part = 0; part < x.n_parts; ++part) {
            if (lane == 0) remote_arrive(peer_addr(smem_u32(&fold_done[part]), 0));
            if (part) ++segf1; else ++segf0;
          }
        }
      }
    }
  }
  // drain: every MMA of the pair has completed (CTA 0's final multicast commit) before TMEM is freed
  if (warp == 2) {
    if (lane == 0) mbar_drain(smem_u32(mma_done), 0);
    __syncwarp();
  }
  tc_fence_before();
  __syncthreads();
  cluster_sync();  // neither CTA leaves while the other may still signal its barriers
  if (threadIdx.x == 0 && *abort_flag) atomicOr(p.status, kStatTimeout);
  if (warp == 2) {
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::2.sync.aligned.b32 %0, 512;" ::"r"(tmem_base));
  }
}

bool fill_pair_group(Chi0PairGroup* G, bool split3, const __nv_bfloat16* o_hi, const __nv_bfloat16* o_lo,
                     const float* o_f32, int ld_pad, int n_aux, int n_aux_pad, int n_ov_pad, const float* dtab, int ld_dtab,
                     int F, bool complex_out, double alpha, double beta, void* out, long long ldm, long long mat_stride,
                     const int* active, bool out64, int item0) {
  if (n_aux_pad % BMC || n_ov_pad % BK || ld_pad != n_ov_pad || ld_dtab % BK || F < 1) return false;
  if ((reinterpret_cast<uintptr_t>(o_hi) & 15) || (reinterpret_cast<uintptr_t>(o_lo) & 15) ||
      (reinterpret_cast<uintptr_t>(o_f32) & 15) || (reinterpret_cast<uintptr_t>(dtab) & 15))
    return false;
  std::memset(static_cast<void*>(G), 0, sizeof(Chi0PairGroup));
  if (!make_map(&G->tm_hi, o_hi, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, n_aux_pad, n_ov_pad, BK, BMC) ||
      !make_map(&G->tm_lo, o_lo, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, n_aux_pad, n_ov_pad, BK, BMC) ||
      !make_map(&G->tm_raw, o_f32, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 4, n_aux_pad, n_ov_pad, 32, BNC))
    return false;
  const int n_qb = n_aux_pad / BNP;
  const int n_pb = (n_aux_pad + 2 * BMC - 1) / (2 * BMC);
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
  G->n_pb = n_pb;
  G->n_qb = n_qb;
  G->n_tiles = n_pb * (n_pb - 1) + std::min(2 * n_pb, n_qb);
  G->item0 = item0;
  G->n_items = G->n_tiles * ((F + G->fpc - 1) / G->fpc);
  G->split3 = split3 ? 1 : 0;
  G->out64 = out64 ? 1 : 0;
  G->alpha = (float)alpha;
  G->beta = (float)beta;
  return true;
}

template <bool CPLX, bool GROUPED>
int launch_pair(const Chi0PairGroup& own, const PairParams& p, int clusters, cudaStream_t s) {
  static bool attr = false;
  constexpr int bytes = smem_bytes(NS, NX);
  if (!attr) {
    if (cudaFuncSetAttribute(chi0_pair_kernel<CPLX, GROUPED>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes) !=
        cudaSuccess)
      return -1;
    attr = true;
  }
  chi0_pair_kernel<CPLX, GROUPED><<<2 * clusters, NTHREADS, bytes, s>>>(own, p);
  return cudaPeekAtLastError() == cudaSuccess ? 1 : -1;
}

}  // namespace

int launch_chi0_pair(bool split3, const __nv_bfloat16* o_hi, const __nv_bfloat16* o_lo, const float* o_f32, int ld_pad,
                     int n_aux, int n_aux_pad, int n_ov_pad, const float* dtab, int ld_dtab, int F, bool complex_out,
                     double alpha, double beta, void* out, long long ldm, long long mat_stride, const int* active,
                     unsigned* status, unsigned long long wait_ns, bool out64, cudaStream_t s, int persist) {
  if (!tc_supported()) return -2;
  Chi0PairGroup G;
  if (!fill_pair_group(&G, split3, o_hi, o_lo, o_f32, ld_pad, n_aux, n_aux_pad, n_ov_pad, dtab, ld_dtab, F, complex_out,
                       alpha, beta, out, ldm, mat_stride, active, out64, 0))
    return -2;
  PairParams p;
  p.groups = nullptr;
  p.n_groups = 1;
  p.n_items = G.n_items;
  p.status = status;
  p.wait_ns = wait_ns;
  const int clusters = persist > 0 ? std::max(1, std::min(persist / 2, G.n_items)) : G.n_items;
  return complex_out ? launch_pair<true, false>(G, p, clusters, s) : launch_pair<false, false>(G, p, clusters, s);
}

size_t chi0_pair_group_bytes() { return sizeof(Chi0PairGroup); }

int chi0_pair_group_fill(void* dst, bool split3, const __nv_bfloat16* o_hi, const __nv_bfloat16* o_lo, const float* o_f32,
                         int ld_pad, int n_aux, int n_aux_pad, int n_ov_pad, const float* dtab, int ld_dtab, int F,
                         bool complex_out, double alpha, double beta, void* out, long long ldm, long long mat_stride,
                         const int* active, bool out64, int item0) {
  Chi0PairGroup G;
  if (!fill_pair_group(&G, split3, o_hi, o_lo, o_f32, ld_pad, n_aux, n_aux_pad, n_ov_pad, dtab, ld_dtab, F, complex_out,
                       alpha, beta, out, ldm, mat_stride, active, out64, item0))
    return -2;
  std::memcpy(dst, &G, sizeof(G));
  return G.n_items;
}

int launch_chi0_pair_grouped(const void* d_groups, int n_groups, int n_items, bool complex_out, int grid,
                             unsigned* status, unsigned long long wait_ns, cudaStream_t s) {
  if (!tc_supported()) return -2;
  if (n_groups < 1 || n_items < 1 || grid < 1 || (reinterpret_cast<uintptr_t>(d_groups) & 63)) return -1;
  PairParams p;
  p.groups = static_cast<const Chi0PairGroup*>(d_groups);
  p.n_groups = n_groups;
  p.n_items = n_items;
  p.status = status;
  p.wait_ns = wait_ns;
  Chi0PairGroup unused;
  std::memset(static_cast<void*>(&unused), 0, sizeof(unused));
  const int clusters = std::max(1, std::min(grid / 2, n_items));
  return complex_out ? launch_pair<true, true>(unused, p, clusters, s) : launch_pair<false, true>(unused, p, clusters, s);
}

}  // namespace gwc
