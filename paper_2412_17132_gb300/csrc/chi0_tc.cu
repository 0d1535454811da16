// Tensor-core polarizability build for sm_103a (tcgen05 + TMEM + TMA).
//
//   Pi_PQ(z_f) = sum_k O_Pk D_f(k) O_Qk      (RI polarizability, Sec. "Self-energy evaluation")
//
// One CTA computes a 128 x 128 lower-triangle tile (P-tile >= Q-tile) for up to four
// frequency parts (a complex z has two parts, Re D and Im D; a point on the imaginary axis
// one). The contraction index k = (i, a) runs over the occupied-virtual pairs in chunks of 64.
//
//   * B operand  O[Q-tile][k-chunk] (BF16 hi, and lo in split mode) arrives by TMA
//     (SWIZZLE_128B, K-major) into a 2-stage ring; it is shared by every frequency part.
//   * A operand  O[P-tile][k] * D_f(k) is formed on the fly by 8 transform warps: each
//     thread reads its row's 32 FP32 values once per chunk, scales them by D of each part,
//     splits them into BF16 hi (+ lo = bf16(v - hi)) and writes them in the swizzled K-major
//     layout the MMA reads; the D scaling is thereby fused into the operand load.
//   * One thread issues tcgen05.mma (kind::f16, BF16 x BF16 -> FP32 in TMEM): per part and
//     16-wide k step, hi*hi (+ hi*lo + lo*hi in split mode, Henry, Tang & Heinecke 2019).
//   * Epilogue: the transform warps read the accumulators with tcgen05.ld and write
//     alpha * Pi + beta * I (eps = 1 - Pi with alpha = -1, beta = 1) in FP32.
//
// Every wait on an mbarrier is bounded (about one second); on expiry the CTA records
// kStatTimeout, stops issuing work, waits (bounded) for its issued MMAs and frees TMEM.
#include <cuda.h>

#include <cstdio>
#include <mutex>

#include "gwc_internal.h"

namespace gwc {

namespace {

constexpr int BM = 128, BN = 128, BK = 64;
constexpr int NB_ST = 2;               // B ring stages
constexpr int NA_ST = 4;               // A ring slots (one frequency part each)
constexpr int TILE = BM * BK * 2;      // 16 KB: one BF16 128 x 64 operand tile
constexpr int NTHREADS = 384;          // warps 0-3 control, 4-11 transform + epilogue
constexpr int NXF = 256;               // transform threads
constexpr int SMEM_BYTES = 1024 + NB_ST * 2 * TILE + NA_ST * 2 * TILE + 256;
constexpr unsigned long long kWaitNs = 1000000000ull;  // 1 s bound per wait

struct TcParams {
  const float* o32;
  int ld;                 // leading dim of o32 (= n_ov_pad)
  const float* dtab;
  int ld_dtab;
  int n_aux;
  int n_kc;               // number of 64-wide chunks
  int F;
  int ppf;                // parts per frequency (1 real, 2 complex)
  int fpc;                // frequencies per CTA
  int split3;
  float alpha, beta;
  void* out;
  long long ldm, mat_stride;
  const int* active;
  unsigned* status;
};

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ unsigned long long gtime() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %globaltimer;" : "=l"(t));
  return t;
}

__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count));
}

__device__ __forceinline__ void mbar_arrive(uint32_t bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(bar) : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint32_t bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
}

__device__ __forceinline__ bool mbar_try(uint32_t bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(bar), "r"(parity)
      : "memory");
  return ok != 0;
}

// Bounded wait: returns false (and raises the CTA abort flag) if the phase does not
// complete within kWaitNs or if another role already aborted.
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity, volatile int* abort_flag) {
  if (mbar_try(bar, parity)) return true;
  unsigned long long t0 = gtime();
  for (uint32_t it = 0;; ++it) {
    if (mbar_try(bar, parity)) return true;
    if ((it & 255u) == 255u) {
      if (*abort_flag) return false;
      if (gtime() - t0 > kWaitNs) {
        *abort_flag = 1;
        return false;
      }
    }
  }
}

// Bounded drain wait that ignores the abort flag (for copies already in flight).
__device__ __forceinline__ void mbar_drain(uint32_t bar, uint32_t parity) {
  unsigned long long t0 = gtime();
  for (uint32_t it = 0;; ++it) {
    if (mbar_try(bar, parity)) return;
    if ((it & 255u) == 255u && gtime() - t0 > kWaitNs) return;
  }
}

__device__ __forceinline__ void tma_load_2d(uint32_t dst, const CUtensorMap* tm, int x, int y, uint32_t bar) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];" ::"r"(dst),
      "l"(reinterpret_cast<uint64_t>(tm)), "r"(x), "r"(y), "r"(bar)
      : "memory");
}

// Shared-memory matrix descriptor: K-major, SWIZZLE_128B, 8-row groups 1024 B apart.
__device__ __forceinline__ uint64_t sdesc(uint32_t addr) {
  uint64_t d = 0;
  d |= (uint64_t)((addr >> 4) & 0x3FFFu);
  d |= (uint64_t)1u << 16;             // leading byte offset (unused for swizzled K-major)
  d |= (uint64_t)(1024u >> 4) << 32;    // stride byte offset: 8 rows x 128 B
  d |= (uint64_t)1u << 46;              // descriptor version for sm_100 family
  d |= (uint64_t)2u << 61;              // SWIZZLE_128B
  return d;
}

// Instruction descriptor, kind::f16: D = F32, A = B = BF16, both K-major, M = 128, N = 128.
constexpr uint32_t kIdesc = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(BN >> 3) << 17) | ((uint32_t)(BM >> 4) << 24);

__device__ __forceinline__ void mma_bf16(uint32_t d_tmem, uint64_t a, uint64_t b, uint32_t accum) {
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "setp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(d_tmem),
      "l"(a), "l"(b), "r"(kIdesc), "r"(accum));
}

__device__ __forceinline__ void mma_commit(uint32_t bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar) : "memory");
}

__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float* v) {
  uint32_t r[16];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]),
        "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}

__device__ __forceinline__ void tile_pair(int t, int& ip, int& iq) {
  int a = (int)((sqrt(8.0 * t + 1.0) - 1.0) * 0.5);
  while ((a + 1) * (a + 2) / 2 <= t) ++a;
  while (a * (a + 1) / 2 > t) --a;
  ip = a;
  iq = t - a * (a + 1) / 2;
}

__device__ __forceinline__ uint32_t pack_bf16x2(float a, float b) {
  __nv_bfloat162 h = __floats2bfloat162_rn(a, b);
  return *reinterpret_cast<uint32_t*>(&h);
}

template <bool CPLX>
__global__ void __launch_bounds__(NTHREADS, 1)
    chi0_tc_kernel(const __grid_constant__ CUtensorMap tm_hi, const __grid_constant__ CUtensorMap tm_lo, TcParams p) {
  extern __shared__ uint8_t smem_raw[];
  uint8_t* base = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~(uintptr_t)1023);
  uint8_t* b_ring = base;                          // NB_ST x [hi | lo]
  uint8_t* a_ring = base + NB_ST * 2 * TILE;       // NA_ST x [hi | lo]
  uint64_t* bars = reinterpret_cast<uint64_t*>(a_ring + NA_ST * 2 * TILE);
  uint64_t* b_full = bars;
  uint64_t* b_empty = bars + NB_ST;
  uint64_t* a_full = bars + 2 * NB_ST;
  uint64_t* a_empty = bars + 2 * NB_ST + NA_ST;
  uint64_t* acc_done = bars + 2 * NB_ST + 2 * NA_ST;
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(acc_done + 1);
  volatile int* abort_flag = reinterpret_cast<volatile int*>(tmem_slot + 1);

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  int ip, iq;
  tile_pair(blockIdx.x, ip, iq);
  const int P0 = ip * BM, Q0 = iq * BN;
  const int f0 = blockIdx.y * p.fpc;
  const int nf = min(p.fpc, p.F - f0);
  if (p.active) {
    int any = 0;
    for (int u = 0; u < nf; ++u) any |= p.active[f0 + u];
    if (!any) return;  // uniform across the CTA, before any barrier or TMEM use
  }
  const int n_parts = nf * p.ppf;

  if (threadIdx.x == 0) {
    for (int i = 0; i < NB_ST; ++i) {
      mbar_init(smem_u32(&b_full[i]), 1);
      mbar_init(smem_u32(&b_empty[i]), 1);
    }
    for (int i = 0; i < NA_ST; ++i) {
      mbar_init(smem_u32(&a_full[i]), NXF);
      mbar_init(smem_u32(&a_empty[i]), 1);
    }
    mbar_init(smem_u32(acc_done), 1);
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
  const uint32_t b_bytes = p.split3 ? 2 * TILE : TILE;

  if (warp == 0) {
    if (lane == 0) {
      int issued = 0;
      for (int kc = 0; kc < p.n_kc; ++kc) {
        const int s = kc % NB_ST, u = kc / NB_ST;
        if (!mbar_wait(smem_u32(&b_empty[s]), (u & 1) ^ 1, abort_flag)) break;
        mbar_expect_tx(smem_u32(&b_full[s]), b_bytes);
        uint8_t* dst = b_ring + s * 2 * TILE;
        tma_load_2d(smem_u32(dst), &tm_hi, kc * BK, Q0, smem_u32(&b_full[s]));
        if (p.split3) tma_load_2d(smem_u32(dst + TILE), &tm_lo, kc * BK, Q0, smem_u32(&b_full[s]));
        issued = kc + 1;
      }
      // no copy may still be writing shared memory when the CTA exits
      for (int kc = issued > NB_ST ? issued - NB_ST : 0; kc < issued; ++kc)
        mbar_drain(smem_u32(&b_full[kc % NB_ST]), (kc / NB_ST) & 1);
    }
  } else if (warp == 1) {
    if (lane == 0) {
      int a = 0;
      bool ok = true;
      for (int kc = 0; kc < p.n_kc && ok; ++kc) {
        const int s = kc % NB_ST, u = kc / NB_ST;
        if (!mbar_wait(smem_u32(&b_full[s]), u & 1, abort_flag)) {
          ok = false;
          break;
        }
        tc_fence_after();
        const uint32_t bh = smem_u32(b_ring + s * 2 * TILE), bl = bh + TILE;
        for (int part = 0; part < n_parts; ++part, ++a) {
          const int t = a % NA_ST, ua = a / NA_ST;
          if (!mbar_wait(smem_u32(&a_full[t]), ua & 1, abort_flag)) {
            ok = false;
            break;
          }
          tc_fence_after();
          const uint32_t ah = smem_u32(a_ring + t * 2 * TILE), al = ah + TILE;
          const uint32_t d = tmem_base + (uint32_t)(part * BN);
#pragma unroll
          for (int k = 0; k < BK / 16; ++k) {
            const uint32_t off = k * 32;  // 16 BF16 = 32 bytes along K inside the 128-B row
            const uint32_t acc = (kc > 0 || k > 0) ? 1u : 0u;
            mma_bf16(d, sdesc(ah + off), sdesc(bh + off), acc);
            if (p.split3) {
              mma_bf16(d, sdesc(ah + off), sdesc(bl + off), 1u);
              mma_bf16(d, sdesc(al + off), sdesc(bh + off), 1u);
            }
          }
          mma_commit(smem_u32(&a_empty[t]));
        }
        if (!ok) break;
        mma_commit(smem_u32(&b_empty[s]));
      }
      // acc_done fires when every MMA issued so far has completed (also after an abort)
      mma_commit(smem_u32(acc_done));
    }
  } else if (warp >= 4) {
    const int tt = threadIdx.x - 128;
    const int r = tt & 127, h = tt >> 7;
    const float* orow = p.o32 + (size_t)(P0 + r) * p.ld + 32 * h;
    int a = 0;
    bool ok = true;
    for (int kc = 0; kc < p.n_kc && ok; ++kc) {
      float raw[32];
      const float4* src = reinterpret_cast<const float4*>(orow + kc * BK);
#pragma unroll
      for (int u = 0; u < 8; ++u) {
        float4 v = __ldg(src + u);
        raw[4 * u] = v.x;
        raw[4 * u + 1] = v.y;
        raw[4 * u + 2] = v.z;
        raw[4 * u + 3] = v.w;
      }
      for (int part = 0; part < n_parts; ++part, ++a) {
        const int t = a % NA_ST, ua = a / NA_ST;
        if (!mbar_wait(smem_u32(&a_empty[t]), (ua & 1) ^ 1, abort_flag)) {
          ok = false;
          break;
        }
        const int f = f0 + part / p.ppf, comp = part % p.ppf;
        const float4* dsrc = reinterpret_cast<const float4*>(p.dtab + ((size_t)f * 2 + comp) * p.ld_dtab + kc * BK + 32 * h);
        uint8_t* ah = a_ring + t * 2 * TILE + r * 128;
        uint8_t* al = ah + TILE;
#pragma unroll
        for (int c = 0; c < 4; ++c) {  // 16-byte chunk c (8 values) of this thread's 32
          float4 d0 = __ldg(dsrc + 2 * c), d1 = __ldg(dsrc + 2 * c + 1);
          float v[8] = {raw[8 * c] * d0.x, raw[8 * c + 1] * d0.y, raw[8 * c + 2] * d0.z, raw[8 * c + 3] * d0.w,
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
          if (p.split3) *reinterpret_cast<uint4*>(al + chunk * 16) = make_uint4(lw[0], lw[1], lw[2], lw[3]);
        }
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        mbar_arrive(smem_u32(&a_full[t]));
      }
    }
    // ---- epilogue -----------------------------------------------------------------------
    bool done = mbar_wait(smem_u32(acc_done), 0, abort_flag) && ok;
    if (!done) mbar_drain(smem_u32(acc_done), 0);  // issued MMAs must finish before TMEM is freed
    done = __all_sync(0xffffffffu, done && !*abort_flag);
    tc_fence_after();
    if (done) {
      const int q = warp & 3, chalf = (warp - 4) >> 2;
      const int row = 32 * q + lane;
      const int P = P0 + row;
      const uint32_t lane_base = tmem_base + ((uint32_t)(32 * q) << 16);
      for (int fl = 0; fl < nf; ++fl) {
        const int f = f0 + fl;
        if (p.active && !p.active[f]) continue;
        for (int cc = 0; cc < 4; ++cc) {
          const int col = chalf * 64 + cc * 16;
          float re[16], im[16];
          tmem_ld16(lane_base + (uint32_t)((fl * p.ppf) * BN + col), re);
          if (CPLX) tmem_ld16(lane_base + (uint32_t)((fl * p.ppf + 1) * BN + col), im);
          if (P >= p.n_aux) continue;
#pragma unroll
          for (int i = 0; i < 16; ++i) {
            const int Q = Q0 + col + i;
            if (Q >= p.n_aux || Q > P) continue;
            const float dg = (P == Q) ? p.beta : 0.0f;
            if (CPLX) {
              float2* o = reinterpret_cast<float2*>(p.out) + f * p.mat_stride + (long long)P * p.ldm + Q;
              *o = make_float2(p.alpha * re[i] + dg, p.alpha * im[i]);
            } else {
              float* o = reinterpret_cast<float*>(p.out) + f * p.mat_stride + (long long)P * p.ldm + Q;
              *o = p.alpha * re[i] + dg;
            }
          }
        }
      }
    }
  }
  tc_fence_before();
  __syncthreads();
  if (threadIdx.x == 0 && *abort_flag) atomicOr(p.status, kStatTimeout);
  if (warp == 2) {
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, 512;" ::"r"(tmem_base));
  }
}

typedef CUresult (*EncodeTiledFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*, const cuuint64_t*,
                                  const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave, CUtensorMapSwizzle,
                                  CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeTiledFn encoder() {
  static EncodeTiledFn fn = nullptr;
  static std::once_flag once;
  std::call_once(once, [] {
    void* f = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &f, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<EncodeTiledFn>(f);
  });
  return fn;
}

bool make_map(CUtensorMap* tm, const __nv_bfloat16* ptr, int rows, int cols) {
  EncodeTiledFn enc = encoder();
  if (!enc) return false;
  cuuint64_t dims[2] = {(cuuint64_t)cols, (cuuint64_t)rows};
  cuuint64_t strides[1] = {(cuuint64_t)cols * 2};
  cuuint32_t box[2] = {BK, BN};
  cuuint32_t es[2] = {1, 1};
  CUresult r = enc(tm, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, (void*)ptr, dims, strides, box, es, CU_TENSOR_MAP_INTERLEAVE_NONE,
                   CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS;
}

bool tc_supported() {
  static int ok = -1;
  if (ok < 0) {
    int dev = 0, major = 0, minor = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&major, cudaDevAttrComputeCapabilityMajor, dev);
    cudaDeviceGetAttribute(&minor, cudaDevAttrComputeCapabilityMinor, dev);
    ok = (major == 10 && minor == 3) ? 1 : 0;
  }
  return ok == 1;
}

}  // namespace

// Returns launches (1), -1 on a launch error, -2 if unsupported (device or shape).
int launch_chi0_tc(bool split3, const __nv_bfloat16* o_hi, const __nv_bfloat16* o_lo, const float* o_f32, int ld_pad,
                   int n_aux, int n_aux_pad, int n_ov_pad, const float* dtab, int ld_dtab, int F, bool complex_out,
                   double alpha, double beta, void* out, long long ldm, long long mat_stride, const int* active,
                   unsigned* status, cudaStream_t s) {
  if (!tc_supported()) return -2;
  if (n_aux_pad % BM || n_ov_pad % BK || ld_pad != n_ov_pad) return -2;
  // TMA: base 16-B aligned and row stride a multiple of 16 B (n_ov_pad is a multiple of 64)
  if ((reinterpret_cast<uintptr_t>(o_hi) & 15) || (reinterpret_cast<uintptr_t>(o_lo) & 15)) return -2;
  CUtensorMap tm_hi, tm_lo;
  if (!make_map(&tm_hi, o_hi, n_aux_pad, n_ov_pad) || !make_map(&tm_lo, o_lo, n_aux_pad, n_ov_pad)) return -2;
  TcParams p;
  p.o32 = o_f32;
  p.ld = ld_pad;
  p.dtab = dtab;
  p.ld_dtab = ld_dtab;
  p.n_aux = n_aux;
  p.n_kc = n_ov_pad / BK;
  p.F = F;
  p.ppf = complex_out ? 2 : 1;
  p.fpc = complex_out ? 2 : 4;
  p.split3 = split3 ? 1 : 0;
  p.alpha = (float)alpha;
  p.beta = (float)beta;
  p.out = out;
  p.ldm = ldm;
  p.mat_stride = mat_stride;
  p.active = active;
  p.status = status;
  const int nt = n_aux_pad / BM;
  dim3 grid(nt * (nt + 1) / 2, (F + p.fpc - 1) / p.fpc);
  static bool attr_c = false, attr_r = false;
  if (complex_out) {
    if (!attr_c) {
      if (cudaFuncSetAttribute(chi0_tc_kernel<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, SMEM_BYTES) != cudaSuccess)
        return -1;
      attr_c = true;
    }
    chi0_tc_kernel<true><<<grid, NTHREADS, SMEM_BYTES, s>>>(tm_hi, tm_lo, p);
  } else {
    if (!attr_r) {
      if (cudaFuncSetAttribute(chi0_tc_kernel<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, SMEM_BYTES) != cudaSuccess)
        return -1;
      attr_r = true;
    }
    chi0_tc_kernel<false><<<grid, NTHREADS, SMEM_BYTES, s>>>(tm_hi, tm_lo, p);
  }
  return cudaPeekAtLastError() == cudaSuccess ? 1 : -1;
}

}  // namespace gwc
