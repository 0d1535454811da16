// Tensor-core LDL^T of complex-symmetric FP32 dielectric matrices (sm_103a: tcgen05 + TMEM).
//
// Same factorisation, storage and panel order as the SIMT kernel (eps = L D L^T without pivoting;
// W = L D below the diagonal, d on it, L^T above it; appended rows n..nrow-1 become L^-1 b), with
// the rank-64 trailing update of every panel moved to the tensor cores:
//
//   C[i][j] -= sum_l W[i][l] L[j][l],   l in the panel, i >= j beyond the panel.
//
// Complex products as real GEMMs over split planes. With A = W rows (Ar, Ai) and B = L rows
// (Lr, Li), one accumulator of N = 128 columns holds Re (columns 0-63) and Im (64-127) of a
// 128 x 64 complex tile:
//     D += Ar [Lr ; Li]^T + Ai [-Li ; Lr]^T,
// so each shared-memory stage keeps the planes -Li, Lr, Li back to back and the two B operands
// are the 128-row windows starting at Lr and at -Li.
//
// FP32 accuracy from TF32 operands (kind::tf32): every value v is split into hi = tf32(v) and
// lo = tf32(v - hi) (3xTF32; Henry, Tang & Heinecke 2019 for the BF16 analogue), and the tile is
// D1 = hi*hi (one accumulator) plus D2 = hi*lo + lo*hi (a second one), so the truncating
// accumulator of the tensor core adds only 16 large partial products into D1 per panel; the
// epilogue forms C - D1 - D2 in round-to-nearest FP32.
//
// Roles (288 threads, one CTA per matrix):
//   warps 0-7   panel factorisation (the shared SIMT routines, named barrier 1)
//   warps 4-7   operand transform: W rows and L^T rows from global memory (L2) -> hi/lo planes
//               in the 128-byte-swizzled K-major layout, one 32-column half of the panel per stage
//   warp 8      TMEM allocation (512 columns: two tiles in flight x {D1, D2}) and the MMA issuer
//   warps 0-3   epilogue: TMEM -> registers, read-modify-write of the target tile in global memory
// The panel scratch of the SIMT routines aliases the two operand stages (the phases alternate).
// Every mbarrier wait is bounded (one second); on expiry the CTA records kStatTimeout, stops,
// drains the MMAs it issued and frees TMEM.
#include "gwc_internal.h"
#include "ldlt_simt.cuh"
#include "tc_common.cuh"

namespace gwc {

namespace {

constexpr int TM = 128;                                  // rows per trailing tile (MMA M)
constexpr int TN = 64;                                   // complex columns per tile (MMA N = 2 TN)
constexpr int KH = 32;                                   // panel columns per stage (128-byte plane rows)
constexpr int A_PLANE = TM * 128;                        // 16 KB: Ar, Ai, Ar_lo, Ai_lo
constexpr int B_PLANE = TN * 128;                        // 8 KB: -Li, Lr, Li, -Li_lo, Lr_lo, Li_lo
constexpr int STAGE_BYTES = 4 * A_PLANE + 6 * B_PLANE;   // 112 KB
constexpr int NSTAGE = 2;
constexpr int NT_TC = 288;
constexpr int META_BYTES = 128;
constexpr int SMEM_TC = 1024 + NSTAGE * STAGE_BYTES + META_BYTES;
static_assert(PW == 2 * KH, "one panel is two stages");
static_assert(FactorSmem<float2>::bytes() <= (size_t)NSTAGE * STAGE_BYTES, "panel scratch fits in the stages");

// kind::tf32 instruction descriptor: D = F32, A = B = TF32, both K-major, N = 2 TN, M = TM.
constexpr uint32_t kIdescTf32 =
    (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(2 * TN >> 3) << 17) | ((uint32_t)(TM >> 4) << 24);

__device__ __forceinline__ void mma_tf32(uint32_t d_tmem, uint64_t a, uint64_t b, uint32_t accum) {
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "setp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}" ::"r"(d_tmem),
      "l"(a), "l"(b), "r"(kIdescTf32), "r"(accum));
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
  uint8_t* base;
  uint64_t *full, *empty, *tfull, *tempty, *mma_done;
  uint32_t* tmem_slot;
  volatile int* abort_flag;
  int* sing;
};

// ---- operand transform (warps 4-7): one stage = one 32-column half of the panel for one tile ----
// (A is written by this kernel: plain coherent loads, no read-only path)
__device__ void transform_role(const TcSmem& sm, const float2* A, int n, int nrow, long long ldm, int k0,
                               int R0, int n_ti, int seq) {
  const int tt = threadIdx.x - 128;  // 0..127
  bool ok = true;
  for (int tI = 0; tI < n_ti && ok; ++tI) {
    const int i0 = R0 + TM * tI;
    const int nc = tile_cols(R0, n, tI);
    for (int tJ = 0; tJ < nc && ok; ++tJ) {
      const int j0 = R0 + TN * tJ;
      for (int h = 0; h < 2; ++h, ++seq) {
        const int s = seq & 1, us = seq >> 1;
        if (!mbar_wait(smem_u32(&sm.empty[s]), (us & 1) ^ 1, sm.abort_flag)) {
          ok = false;
          break;
        }
        uint8_t* st = sm.base + s * STAGE_BYTES;
        // A planes: row tt of the tile = W[i0 + tt][k0 + KH h .. + KH)
        {
          const int r = tt, i = i0 + r, sw = r & 7;
          uint8_t* rowp = st + r * 128;
          if (i < nrow) {
            const float4* src = reinterpret_cast<const float4*>(A + (long long)i * ldm + k0 + KH * h);
#pragma unroll 2
            for (int c = 0; c < 8; ++c) {  // chunk c: complex l = 4c .. 4c+3
              const float4 v0 = src[2 * c], v1 = src[2 * c + 1];
              const float re[4] = {v0.x, v0.z, v1.x, v1.z};
              const float im[4] = {v0.y, v0.w, v1.y, v1.w};
              float4 rh, rl, ih, il;
              split4(re, rh, rl);
              split4(im, ih, il);
              const int off = (c ^ sw) << 4;
              *reinterpret_cast<float4*>(rowp + off) = rh;
              *reinterpret_cast<float4*>(rowp + A_PLANE + off) = ih;
              *reinterpret_cast<float4*>(rowp + 2 * A_PLANE + off) = rl;
              *reinterpret_cast<float4*>(rowp + 3 * A_PLANE + off) = il;
            }
          } else {
            const float4 z = make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
            for (int c = 0; c < 8; ++c)
#pragma unroll
              for (int pl = 0; pl < 4; ++pl) *reinterpret_cast<float4*>(rowp + pl * A_PLANE + (c << 4)) = z;
          }
        }
        // B planes: row jj of the tile = L[j0 + jj][l] = L^T[l][j0 + jj], 16 of the 32 columns l
        {
          const int jj = tt & 63, lh = tt >> 6, j = j0 + jj, sw = jj & 7;
          uint8_t* rowp = st + 4 * A_PLANE + jj * 128;
          const bool jv = j < n;
          const float2* colp = A + (long long)(k0 + KH * h + 16 * lh) * ldm + j;
#pragma unroll
          for (int c = 0; c < 4; ++c) {
            float lr[4], li[4], nli[4];
#pragma unroll
            for (int e = 0; e < 4; ++e) {
              const float2 v = jv ? colp[(long long)(4 * c + e) * ldm] : make_float2(0.f, 0.f);
              lr[e] = v.x;
              li[e] = v.y;
              nli[e] = -v.y;
            }
            float4 rh, rl, ih, il, nh, nl;
            split4(lr, rh, rl);
            split4(li, ih, il);
            split4(nli, nh, nl);
            const int off = ((4 * lh + c) ^ sw) << 4;
            *reinterpret_cast<float4*>(rowp + off) = nh;
            *reinterpret_cast<float4*>(rowp + B_PLANE + off) = rh;
            *reinterpret_cast<float4*>(rowp + 2 * B_PLANE + off) = ih;
            *reinterpret_cast<float4*>(rowp + 3 * B_PLANE + off) = nl;
            *reinterpret_cast<float4*>(rowp + 4 * B_PLANE + off) = rl;
            *reinterpret_cast<float4*>(rowp + 5 * B_PLANE + off) = il;
          }
        }
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        mbar_arrive(smem_u32(&sm.full[s]));
      }
    }
  }
}

// ---- MMA issuer (one thread of warp 8) ----------------------------------------------------------
__device__ void mma_role(const TcSmem& sm, uint32_t tmem_base, int n, int R0, int n_ti, int seq, int tcount) {
  bool ok = true;
  for (int tI = 0; tI < n_ti && ok; ++tI) {
    const int nc = tile_cols(R0, n, tI);
    for (int tJ = 0; tJ < nc && ok; ++tJ, ++tcount) {
      const int b = tcount & 1, ub = tcount >> 1;
      if (!mbar_wait(smem_u32(&sm.tempty[b]), (ub & 1) ^ 1, sm.abort_flag)) {
        ok = false;
        break;
      }
      tc_fence_after();
      const uint32_t d1 = tmem_base + (uint32_t)(b * 256), d2 = d1 + 128;
      for (int h = 0; h < 2; ++h, ++seq) {
        const int s = seq & 1, us = seq >> 1;
        if (!mbar_wait(smem_u32(&sm.full[s]), us & 1, sm.abort_flag)) {
          ok = false;
          break;
        }
        tc_fence_after();
        const uint32_t st = smem_u32(sm.base + s * STAGE_BYTES);
        const uint32_t ar = st, ai = st + A_PLANE, arl = st + 2 * A_PLANE, ail = st + 3 * A_PLANE;
        const uint32_t bb = st + 4 * A_PLANE;
        const uint32_t b2 = bb, b1 = bb + B_PLANE;                  // [-Li ; Lr], [Lr ; Li]
        const uint32_t b2l = bb + 3 * B_PLANE, b1l = bb + 4 * B_PLANE;
#pragma unroll
        for (int k = 0; k < KH / 8; ++k) {
          const uint32_t off = k * 32;  // 8 TF32 values = 32 bytes along K inside the 128-B row
          const uint32_t acc = (h == 0 && k == 0) ? 0u : 1u;
          mma_tf32(d1, sdesc(ar + off), sdesc(b1 + off), acc);
          mma_tf32(d1, sdesc(ai + off), sdesc(b2 + off), 1u);
          mma_tf32(d2, sdesc(ar + off), sdesc(b1l + off), acc);
          mma_tf32(d2, sdesc(arl + off), sdesc(b1 + off), 1u);
          mma_tf32(d2, sdesc(ai + off), sdesc(b2l + off), 1u);
          mma_tf32(d2, sdesc(ail + off), sdesc(b2 + off), 1u);
        }
        mma_commit(smem_u32(&sm.empty[s]));
      }
      if (!ok) break;
      mma_commit(smem_u32(&sm.tfull[b]));
    }
  }
}

// ---- epilogue (warps 0-3): C -= D1 + D2 for rows i0 + 32 q + lane --------------------------------
__device__ void epilogue_role(const TcSmem& sm, uint32_t tmem_base, float2* __restrict__ A, int n, int nrow,
                              long long ldm, int R0, int n_ti, int tcount) {
  const int q = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const uint32_t lane_base = tmem_base + ((uint32_t)(32 * q) << 16);
  bool ok = true;
  for (int tI = 0; tI < n_ti && ok; ++tI) {
    const int i0 = R0 + TM * tI;
    const int nc = tile_cols(R0, n, tI);
    const int i = i0 + 32 * q + lane;
    // columns j < jlim of row i are updated: j <= i inside the factored block, all j < n below it
    const int jlim = i < nrow ? (i < n ? min(n, i + 1) : n) : 0;
    for (int tJ = 0; tJ < nc; ++tJ, ++tcount) {
      const int j0 = R0 + TN * tJ;
      const int b = tcount & 1, ub = tcount >> 1;
      ok = mbar_wait(smem_u32(&sm.tfull[b]), ub & 1, sm.abort_flag);
      ok = __all_sync(0xffffffffu, ok);
      if (!ok) break;
      tc_fence_after();
#pragma unroll 1
      for (int cc = 0; cc < TN / 16; ++cc) {
        float d1r[16], d1i[16], d2r[16], d2i[16];
        const uint32_t col = lane_base + (uint32_t)(b * 256 + 16 * cc);
        tmem_ld16(col, d1r);
        tmem_ld16(col + 64, d1i);
        tmem_ld16(col + 128, d2r);
        tmem_ld16(col + 192, d2i);
        const int jb = j0 + 16 * cc;
        if (jb >= jlim) continue;
        float2* p = A + (long long)i * ldm + jb;
        if (jb + 16 <= jlim) {
#pragma unroll
          for (int e = 0; e < 16; e += 2) {
            float4 c = *reinterpret_cast<const float4*>(p + e);
            c.x = c.x - d1r[e] - d2r[e];
            c.y = c.y - d1i[e] - d2i[e];
            c.z = c.z - d1r[e + 1] - d2r[e + 1];
            c.w = c.w - d1i[e + 1] - d2i[e + 1];
            *reinterpret_cast<float4*>(p + e) = c;
          }
        } else {
#pragma unroll
          for (int e = 0; e < 16; ++e)
            if (jb + e < jlim) {
              float2 c = p[e];
              c.x = c.x - d1r[e] - d2r[e];
              c.y = c.y - d1i[e] - d2i[e];
              p[e] = c;
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
  uint64_t* bars = reinterpret_cast<uint64_t*>(sm.base + NSTAGE * STAGE_BYTES);
  sm.full = bars;
  sm.empty = bars + 2;
  sm.tfull = bars + 4;
  sm.tempty = bars + 6;
  sm.mma_done = bars + 8;
  sm.tmem_slot = reinterpret_cast<uint32_t*>(bars + 9);
  sm.abort_flag = reinterpret_cast<volatile int*>(sm.tmem_slot + 1);
  sm.sing = reinterpret_cast<int*>(sm.tmem_slot + 2);
  using FS = FactorSmem<float2>;
  float2(*lkk)[NB + 1] = reinterpret_cast<float2(*)[NB + 1]>(sm.base);
  float2* dinv = reinterpret_cast<float2*>(sm.base + sizeof(float2) * NB * (NB + 1));
  float2* stages = reinterpret_cast<float2*>(sm.base + FS::LKK_BYTES);

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (threadIdx.x == 0) {
    for (int i = 0; i < 2; ++i) {
      mbar_init(smem_u32(&sm.full[i]), 128);
      mbar_init(smem_u32(&sm.empty[i]), 1);
      mbar_init(smem_u32(&sm.tfull[i]), 1);
      mbar_init(smem_u32(&sm.tempty[i]), 128);
    }
    mbar_init(smem_u32(sm.mma_done), 1);
    *sm.abort_flag = 0;
    *sm.sing = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 8) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], 512;" ::"r"(smem_u32(sm.tmem_slot)));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem_base = *sm.tmem_slot;

  int seq = 0, tcount = 0;  // stages and tiles issued so far; every role advances them alike
  for (int k0 = 0; k0 < n; k0 += PW) {
    const int kb = min(PW, n - k0);
    if (warp < 8) {
      factor_subpanel(A, n, nrow, ldm, k0, lkk, dinv, *sm.sing);
      if (kb > NB) {
        update_region(A, nrow, ldm, k0 + NB, k0 + NB, k0 + kb, k0, NB, stages);
        factor_subpanel(A, n, nrow, ldm, k0 + NB, lkk, dinv, *sm.sing);
      }
    }
    __syncthreads();  // panel W / L^T in global memory; the panel scratch is free
    const int R0 = k0 + kb;
    if (R0 < n) {
      const int n_ti = (nrow - R0 + TM - 1) / TM;
      if (warp == 8) {
        if (lane == 0) mma_role(sm, tmem_base, n, R0, n_ti, seq, tcount);
        __syncwarp();
      } else if (warp >= 4) {
        transform_role(sm, A, n, nrow, ldm, k0, R0, n_ti, seq);
      } else {
        epilogue_role(sm, tmem_base, A, n, nrow, ldm, R0, n_ti, tcount);
      }
      int nt = 0;
      for (int tI = 0; tI < n_ti; ++tI) nt += tile_cols(R0, n, tI);
      seq += 2 * nt;
      tcount += nt;
    }
    tc_fence_before();
    __syncthreads();  // every tile of the panel is written back; the stages are free
    tc_fence_after();
    if (*sm.abort_flag) break;
  }
  // every MMA issued has completed before TMEM is freed (immediate unless a wait gave up)
  if (warp == 8) {
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
  if (warp == 8) {
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
