// Imaginary-axis W table on the tensor cores (sm_103a: tcgen05 kind::tf32 + TMEM + TMA).
//
//   W^c_mn(i xi) = b^T (eps^-1 - 1) b = sum_p y_p^2 / d_p - b^T b,   y = L^-1 b,   b = O^P_mn
//   (Sec. Self-energy evaluation, eqs cd_imaginary and the screened interaction), for the N_states x N_core
//   right-hand sides of every imaginary node, eps = L D L^T factored in FP32 (real SPD on the imaginary axis).
//
// The forward substitution is blocked right-looking over 128-row blocks of L, as two GEMMs per block on the
// tensor cores in 3xTF32 (every operand split into TF32 hi and lo = tf32(v - hi); hi*hi + hi*lo + lo*hi):
//   DIAG   y_i = Linv_ii c_i         (Linv_ii: inverse of the unit lower diagonal block, formed once per node)
//          table += sum_p y_p^2 / d_p, and z_i = y_i / d_i kept as TF32 planes;
//   UPDATE c_P -= sum_{q in block i} W_Pq z_q   for the rows P below the block (W = L D, the factored matrix).
// The right-hand sides are stored one per row ([col][P], P contiguous), which is the K-major layout of the
// B operand; the A operands (Linv, W) are K-major by rows. A CTA computes a 128 x 256 tile (rows x columns)
// over K = 128 in four 32-wide chunks (two TMA stages); the epilogue either reduces the norm and writes z
// (DIAG) or read-modify-writes the right-hand sides (UPDATE). The right-hand sides stream through HBM once
// per block; the GEMM work is N^2 R / 2 multiply-adds per node, three TF32 products each.
//
// Every mbarrier wait is bounded (the context's bound); on expiry the CTA records kStatTimeout, drains its
// copies and MMAs and frees TMEM.
#include <cuda.h>

#include <algorithm>
#include <cstring>

#include "gwc_internal.h"
#include "tc_common.cuh"

namespace gwc {

namespace {

constexpr int TB = 128;          // rows per block of L (K of both GEMMs) and per tile
constexpr int TNC = 256;         // right-hand-side columns per tile (MMA N)
constexpr int KC = 32;           // K per TMA chunk (128-byte rows of FP32)
constexpr int NCH = TB / KC;     // chunks per tile
constexpr int NST = 2;           // stages
constexpr int A_TILE = TB * KC * 4;    // 16 KB
constexpr int B_TILE = TNC * KC * 4;   // 32 KB
constexpr int STAGE = 2 * A_TILE + 2 * B_TILE;  // hi and lo of both operands: 96 KB
constexpr int NTHR = 256;        // warp 0 TMA, 1 MMA, 2 TMEM, 4-7 epilogue
constexpr int SMEM = 1024 + NST * STAGE + 256 + 4 * TNC * 8;
static_assert(TB * TNC * 4 <= NST * STAGE, "the C tile of an UPDATE fits in the stage buffers");

// kind::tf32: D = F32, A = B = TF32, K-major, M = 128, N = 256
constexpr uint32_t kIdesc = (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(TNC >> 3) << 17) | ((uint32_t)(TB >> 4) << 24);

__device__ __forceinline__ void mma_tf32(uint32_t d, uint64_t a, uint64_t b, uint32_t acc) {
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "setp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}" ::"r"(d),
      "l"(a), "l"(b), "r"(kIdesc), "r"(acc));
}

__device__ __forceinline__ float tf32_rn(float x) {
  uint32_t r;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
  return __uint_as_float(r);
}

struct WtParams {
  CUtensorMap a_hi, a_lo, b_hi, b_lo;  // A: Linv blocks (DIAG) or W planes (UPDATE); B: c blocks or z blocks
  CUtensorMap c_map;                   // the right-hand sides as (P, col, node), box 128 x 256 x 1 (UPDATE)
  int mode;                            // 0 DIAG, 1 UPDATE
  int blk;                             // block index i
  int n;                               // N_aux
  int r;                               // right-hand sides per node
  int ng;                              // nodes in the launch
  int a_rows;                          // rows of one node's A slab in the A map
  int b_rows;                          // rows of one node's B slab in the B map (R rounded up to 256)
  int n_rt, n_ct;                      // row tiles, column tiles per node
  float* c;                            // right-hand sides [node][col][ldc]
  long long ldc, c_node;
  const float* mats;                   // factored matrices (d on the diagonal): element (P, Q) of node u at
  long long ldm, m_node;               // mats[u m_node + (P ldm + Q) es], es = 2 for the real parts of complex storage
  int es;
  float* z_hi;                         // z planes [node][b_rows][TB]
  float* z_lo;
  double* table;                       // [node][r] (node stride r)
  unsigned* status;
  unsigned long long wait_ns;
};

__device__ __forceinline__ void tma_load_3d(uint32_t dst, const CUtensorMap* tm, int x, int y, int z, uint32_t bar) {
  asm volatile(
      "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], [%5];" ::"r"(dst),
      "l"(reinterpret_cast<uint64_t>(tm)), "r"(x), "r"(y), "r"(z), "r"(bar)
      : "memory");
}

// shared -> global tile store; elements outside the map (P >= n, col >= r) are not written
__device__ __forceinline__ void tma_store_3d(const CUtensorMap* tm, int x, int y, int z, uint32_t src) {
  asm volatile("cp.async.bulk.tensor.3d.global.shared::cta.bulk_group [%0, {%1, %2, %3}], [%4];" ::"l"(
                   reinterpret_cast<uint64_t>(tm)),
               "r"(x), "r"(y), "r"(z), "r"(src)
               : "memory");
  asm volatile("cp.async.bulk.commit_group;" ::: "memory");
}

__device__ __forceinline__ void tma_store_wait_read() { asm volatile("cp.async.bulk.wait_group.read 0;" ::: "memory"); }

__global__ void __launch_bounds__(NTHR, 1) wtable_gemm_kernel(const __grid_constant__ WtParams p) {
  extern __shared__ uint8_t smem_raw[];
  uint8_t* base = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~(uintptr_t)1023);
  uint64_t* full = reinterpret_cast<uint64_t*>(base + NST * STAGE);
  uint64_t* empty = full + NST;
  uint64_t* done = empty + NST;
  uint64_t* c_full = done + 1;  // the C tile of an UPDATE has landed in the (then idle) stage buffers
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(c_full + 1);
  volatile int* abort_flag = reinterpret_cast<volatile int*>(tmem_slot + 1);
  double* red = reinterpret_cast<double*>(base + NST * STAGE + 256);  // [4 warps][TNC] norm partials

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int t = blockIdx.x;
  const int ct = t % p.n_ct, rt = (t / p.n_ct) % p.n_rt, u = t / (p.n_ct * p.n_rt);
  if (u >= p.ng) return;
  const int row0 = p.mode == 0 ? p.blk * TB : (p.blk + 1) * TB + rt * TB;  // first row of the tile
  const int col0 = ct * TNC;

  if (threadIdx.x == 0) {
    for (int s = 0; s < NST; ++s) {
      mbar_init(smem_u32(&full[s]), 1);
      mbar_init(smem_u32(&empty[s]), 1);
    }
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
      // A rows of this tile in the A map: DIAG -> block i of node u's Linv slab; UPDATE -> rows row0.. of W
      const int ay = u * p.a_rows + (p.mode == 0 ? p.blk * TB : row0);
      const int ax0 = p.mode == 0 ? 0 : p.blk * TB;  // K columns of A
      const int by = u * p.b_rows + col0;
      int issued = 0;
      for (int kc = 0; kc < NCH; ++kc) {
        const int s = kc % NST;
        const uint32_t ph = (uint32_t)(kc / NST);
        if (!mbar_wait(smem_u32(&empty[s]), (ph & 1) ^ 1, abort_flag, p.wait_ns)) break;
        uint8_t* st = base + s * STAGE;
        mbar_expect_tx(smem_u32(&full[s]), STAGE);
        tma_load_2d(smem_u32(st), &p.a_hi, ax0 + kc * KC, ay, smem_u32(&full[s]));
        tma_load_2d(smem_u32(st + A_TILE), &p.a_lo, ax0 + kc * KC, ay, smem_u32(&full[s]));
        tma_load_2d(smem_u32(st + 2 * A_TILE), &p.b_hi, kc * KC, by, smem_u32(&full[s]));
        tma_load_2d(smem_u32(st + 2 * A_TILE + B_TILE), &p.b_lo, kc * KC, by, smem_u32(&full[s]));
        issued = kc + 1;
      }
      for (int kc = issued > NST ? issued - NST : 0; kc < issued; ++kc)
        mbar_drain(smem_u32(&full[kc % NST]), (uint32_t)(kc / NST) & 1);
    }
  } else if (warp == 1) {
    if (lane == 0) {
      for (int kc = 0; kc < NCH; ++kc) {
        const int s = kc % NST;
        if (!mbar_wait(smem_u32(&full[s]), (uint32_t)(kc / NST) & 1, abort_flag, p.wait_ns)) break;
        tc_fence_after();
        const uint32_t st = smem_u32(base + s * STAGE);
        const uint64_t ah = sdesc(st), al = sdesc(st + A_TILE), bh = sdesc(st + 2 * A_TILE),
                       bl = sdesc(st + 2 * A_TILE + B_TILE);
#pragma unroll
        for (int k = 0; k < KC / 8; ++k) {
          const uint64_t o = 2u * k;  // 8 TF32 = 32 bytes along K
          mma_tf32(tmem, ah + o, bh + o, (kc == 0 && k == 0) ? 0u : 1u);
          mma_tf32(tmem, ah + o, bl + o, 1u);
          mma_tf32(tmem, al + o, bh + o, 1u);
        }
        mma_commit(smem_u32(&empty[s]));
      }
      mma_commit(smem_u32(done));
    }
  } else if (warp >= 4) {
    // ---------------- epilogue: one TMEM lane (tile row) per thread -------------------------------
    const int q = warp & 3;
    const int rrow = 32 * q + lane;
    const int P = row0 + rrow;
    const bool ok = __all_sync(0xffffffffu, mbar_wait(smem_u32(done), 0, abort_flag, p.wait_ns));
    tc_fence_after();
    const uint32_t lb = tmem + ((uint32_t)(32 * q) << 16);
    if (p.mode == 1) {
      // C tile [256 cols][128 rows] through shared memory: TMA load (zero beyond n and r), subtract, TMA store
      float* ct = reinterpret_cast<float*>(base);
      bool landed = false;
      if (ok && !*abort_flag) {  // no operand copy can still be landing in the stage buffers
        if (threadIdx.x == 128) {
          mbar_expect_tx(smem_u32(c_full), TB * TNC * 4);
          tma_load_3d(smem_u32(base), &p.c_map, row0, col0, u, smem_u32(c_full));
        }
        landed = __all_sync(0xffffffffu, mbar_wait(smem_u32(c_full), 0, abort_flag, p.wait_ns));
        if (landed) {
          for (int cc = 0; cc < TNC / 16; ++cc) {
            float v[16];
            tmem_ld16(lb + cc * 16, v);
#pragma unroll
            for (int j = 0; j < 16; ++j) ct[(cc * 16 + j) * TB + rrow] -= v[j];
          }
        }
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      }
      asm volatile("bar.sync 1, 128;" ::: "memory");  // every epilogue warp, whatever its waits gave
      if (threadIdx.x == 128) {
        if (landed && !*abort_flag) {
          tma_store_3d(&p.c_map, row0, col0, u, smem_u32(base));
          tma_store_wait_read();  // the tile is read out of shared memory before the CTA leaves
        } else if (ok) {
          mbar_drain(smem_u32(c_full), 0);  // a load issued above lands before the CTA leaves
        }
      }
    } else {
      {
        const bool valid = P < p.n;
        const float dinv = valid ? 1.0f / p.mats[(long long)u * p.m_node + ((long long)P * p.ldm + P) * p.es] : 0.0f;
        float* zh = p.z_hi + ((long long)u * p.b_rows + col0) * TB + rrow;
        float* zl = p.z_lo + ((long long)u * p.b_rows + col0) * TB + rrow;
        for (int cc = 0; cc < TNC / 16 && ok; ++cc) {
          float v[16];
          tmem_ld16(lb + cc * 16, v);
#pragma unroll
          for (int j = 0; j < 16; ++j) {
            const float y = valid ? v[j] : 0.0f;
            const float zz = y * dinv;
            const float h = tf32_rn(zz);
            zh[(long long)(cc * 16 + j) * TB] = h;
            zl[(long long)(cc * 16 + j) * TB] = tf32_rn(zz - h);
            double w = (double)y * (double)y * (double)dinv;
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) w += __shfl_xor_sync(0xffffffffu, w, o);
            if (lane == 0) red[q * TNC + cc * 16 + j] = w;
          }
        }
        // the four epilogue warps meet whatever their wait gave (no warp may skip the barrier)
        asm volatile("bar.sync 1, 128;" ::: "memory");
        const bool all_ok = !*abort_flag;
        const int tid = threadIdx.x - 128;
        for (int cidx = tid; cidx < TNC && all_ok; cidx += 128) {
          const int col = col0 + cidx;
          if (col < p.r) {
            const double w = red[cidx] + red[TNC + cidx] + red[2 * TNC + cidx] + red[3 * TNC + cidx];
            atomicAdd(p.table + (long long)u * p.r + col, w);
          }
        }
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

// W planes: hi / lo TF32 of the strictly lower part of each factored matrix (rows and columns >= n zero).
__global__ void wt_split_w_kernel(const float* __restrict__ mats, long long ldm, long long m_node, int es, int n, int n_pad,
                                  float* __restrict__ w_hi, float* __restrict__ w_lo, int ng) {
  const long long per = (long long)n_pad * n_pad;
  for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < per * ng; e += (long long)gridDim.x * blockDim.x) {
    const int u = (int)(e / per);
    const long long f = e - (long long)u * per;
    const int row = (int)(f / n_pad), col = (int)(f - (long long)row * n_pad);
    float v = 0.0f;
    if (row < n && col < row) v = mats[(long long)u * m_node + ((long long)row * ldm + col) * es];
    const float h = tf32_rn(v);
    w_hi[e] = h;
    w_lo[e] = tf32_rn(v - h);
  }
}

// Linv planes: inverse of each unit lower 128 x 128 diagonal block, L_pq = W_pq / d_q (identity beyond n).
// One CTA per (node, block); thread c forms column c of X = L^-1 (X_pc = -sum_{c <= q < p} L_pq X_qc).
constexpr int LINV_SMEM = 2 * TB * (TB + 1) * 4;

__global__ void __launch_bounds__(TB) wt_linv_kernel(const float* __restrict__ mats, long long ldm, long long m_node, int es,
                                                     int n, int n_blk, float* __restrict__ l_hi, float* __restrict__ l_lo) {
  extern __shared__ float lsm[];
  float (*L)[TB + 1] = reinterpret_cast<float (*)[TB + 1]>(lsm);
  float (*X)[TB + 1] = reinterpret_cast<float (*)[TB + 1]>(lsm + TB * (TB + 1));
  const int blk = blockIdx.x % n_blk, u = blockIdx.x / n_blk;
  const int k0 = blk * TB;
  const float* m = mats + (long long)u * m_node;
  const int c = threadIdx.x;
  for (int p = 0; p < TB; ++p) {
    const int gp = k0 + p, gc = k0 + c;
    float v = 0.0f;
    if (c < p && gp < n && gc < n) v = m[((long long)gp * ldm + gc) * es] / m[((long long)gc * ldm + gc) * es];
    L[p][c] = v;
  }
  __syncthreads();
  for (int p = 0; p < TB; ++p) {
    float x = 0.0f;
    if (p == c) {
      x = 1.0f;
    } else if (p > c) {
      for (int q = c; q < p; ++q) x -= L[p][q] * X[q][c];
    }
    X[p][c] = x;
  }
  __syncthreads();
  float* hi = l_hi + ((long long)u * n_blk + blk) * TB * TB;
  float* lo = l_lo + ((long long)u * n_blk + blk) * TB * TB;
  for (int p = 0; p < TB; ++p) {
    const float v = X[p][c];
    const float h = tf32_rn(v);
    hi[p * TB + c] = h;
    lo[p * TB + c] = tf32_rn(v - h);
  }
}

// c planes of block i: hi / lo TF32 of the right-hand sides' rows k0 .. k0 + 127 (zero beyond n and r).
__global__ void wt_split_c_kernel(const float* __restrict__ c, long long ldc, long long c_node, int n, int r, int b_rows,
                                  int k0, int ng, float* __restrict__ c_hi, float* __restrict__ c_lo) {
  const long long per = (long long)b_rows * TB;
  for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < per * ng; e += (long long)gridDim.x * blockDim.x) {
    const int u = (int)(e / per);
    const long long f = e - (long long)u * per;
    const int col = (int)(f / TB), k = (int)(f - (long long)col * TB);
    float v = 0.0f;
    if (col < r && k0 + k < n) v = c[(long long)u * c_node + (long long)col * ldc + k0 + k];
    const float h = tf32_rn(v);
    c_hi[e] = h;
    c_lo[e] = tf32_rn(v - h);
  }
}

// table[u][col] = -b^T b (the sum over y_p^2 / d_p is added block by block)
__global__ void wt_init_kernel(const double* __restrict__ bnorm, int r, int ng, double* __restrict__ table, long long t_node) {
  for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < (long long)r * ng; e += (long long)gridDim.x * blockDim.x) {
    const int u = (int)(e / r), col = (int)(e - (long long)u * r);
    table[(long long)u * t_node + col] = -bnorm[e];
  }
}

int grid_for(long long n) { return (int)std::min<long long>((n + 255) / 256, 152LL * 16); }

// complex storage (v, 0) of real matrices: dst[u][e] = (src[u][e], 0) for e < per
__global__ void widen_kernel(const float* __restrict__ src, long long src_node, float2* __restrict__ dst, long long dst_node,
                             long long per, int nb) {
  for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < per * nb; e += (long long)gridDim.x * blockDim.x) {
    const int u = (int)(e / per);
    const long long k = e - (long long)u * per;
    dst[(long long)u * dst_node + k] = make_float2(src[(long long)u * src_node + k], 0.0f);
  }
}

// (P, col, node) view of the right-hand sides [node][col][ldc]: extents n, r, ng; box 128 x 256 x 1, no swizzle
bool make_c_map(CUtensorMap* tm, float* c, int n, int r, int ng, long long ldc, long long c_node) {
  EncodeTiledFn enc = encoder();
  if (!enc) return false;
  cuuint64_t dims[3] = {(cuuint64_t)n, (cuuint64_t)r, (cuuint64_t)ng};
  cuuint64_t strides[2] = {(cuuint64_t)ldc * 4, (cuuint64_t)c_node * 4};
  cuuint32_t box[3] = {(cuuint32_t)TB, (cuuint32_t)TNC, 1};
  cuuint32_t es[3] = {1, 1, 1};
  return enc(tm, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, c, dims, strides, box, es, CU_TENSOR_MAP_INTERLEAVE_NONE,
             CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) ==
         CUDA_SUCCESS;
}

}  // namespace

size_t wtable_tc_bytes(int n_aux, int r, int ng) {
  const size_t n_pad = ((size_t)n_aux + TB - 1) / TB * TB;
  const size_t r_pad = ((size_t)r + TNC - 1) / TNC * TNC;
  const size_t per = 4 * (2 * n_pad * n_pad + 2 * n_pad * TB + 4 * r_pad * TB);
  return per * (size_t)ng + 4096;
}

int launch_wtable_tc(const float* mats, int es, int n, long long ldm, long long m_node, float* rhs, long long ldc, long long c_node,
                     int r, int ng, const double* bnorm, double* table, long long t_node, void* work, size_t work_bytes,
                     unsigned* status, unsigned long long wait_ns, cudaStream_t s) {
  if (!tc_supported()) return -2;
  if (t_node != r || (es != 1 && es != 2)) return -2;  // the GEMM epilogue addresses the table as [node][r]
  if (wtable_tc_bytes(n, r, ng) > work_bytes || (reinterpret_cast<uintptr_t>(work) & 15)) return -2;
  if ((ldc * 4) % 16 || (reinterpret_cast<uintptr_t>(rhs) & 15)) return -2;
  const int n_pad = (n + TB - 1) / TB * TB;
  const int n_blk = n_pad / TB;
  const int r_pad = (r + TNC - 1) / TNC * TNC;
  float* w_hi = static_cast<float*>(work);
  float* w_lo = w_hi + (size_t)ng * n_pad * n_pad;
  float* l_hi = w_lo + (size_t)ng * n_pad * n_pad;
  float* l_lo = l_hi + (size_t)ng * n_pad * TB;
  float* c_hi = l_lo + (size_t)ng * n_pad * TB;
  float* c_lo = c_hi + (size_t)ng * r_pad * TB;
  float* z_hi = c_lo + (size_t)ng * r_pad * TB;
  float* z_lo = z_hi + (size_t)ng * r_pad * TB;
  static bool attr = false;
  if (!attr) {
    if (cudaFuncSetAttribute(wtable_gemm_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, SMEM) != cudaSuccess ||
        cudaFuncSetAttribute(wt_linv_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, LINV_SMEM) != cudaSuccess)
      return -1;
    attr = true;
  }
  // tensor maps: A slabs [ng * rows][cols], B slabs [ng * r_pad][TB]; boxes 32 x 128 (A), 32 x 256 (B)
  WtParams p;
  std::memset(static_cast<void*>(&p), 0, sizeof(p));
  CUtensorMap w_hi_m, w_lo_m, l_hi_m, l_lo_m, c_hi_m, c_lo_m, z_hi_m, z_lo_m;
  if (!make_map(&w_hi_m, w_hi, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 4, ng * n_pad, n_pad, KC, TB) ||
      !make_map(&w_lo_m, w_lo, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 4, ng * n_pad, n_pad, KC, TB) ||
      !make_map(&l_hi_m, l_hi, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 4, ng * n_pad, TB, KC, TB) ||
      !make_map(&l_lo_m, l_lo, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 4, ng * n_pad, TB, KC, TB) ||
      !make_map(&c_hi_m, c_hi, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 4, ng * r_pad, TB, KC, TNC) ||
      !make_map(&c_lo_m, c_lo, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 4, ng * r_pad, TB, KC, TNC) ||
      !make_map(&z_hi_m, z_hi, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 4, ng * r_pad, TB, KC, TNC) ||
      !make_map(&z_lo_m, z_lo, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 4, ng * r_pad, TB, KC, TNC) ||
      !make_c_map(&p.c_map, rhs, n, r, ng, ldc, c_node))
    return -2;
  p.n = n;
  p.r = r;
  p.ng = ng;
  p.b_rows = r_pad;
  p.n_ct = r_pad / TNC;
  p.c = rhs;
  p.ldc = ldc;
  p.c_node = c_node;
  p.mats = mats;
  p.ldm = ldm;
  p.m_node = m_node;
  p.es = es;
  p.z_hi = z_hi;
  p.z_lo = z_lo;
  p.table = table;
  p.status = status;
  p.wait_ns = wait_ns;

  wt_init_kernel<<<grid_for((long long)r * ng), 256, 0, s>>>(bnorm, r, ng, table, t_node);
  wt_split_w_kernel<<<grid_for((long long)n_pad * n_pad * ng), 256, 0, s>>>(mats, ldm, m_node, es, n, n_pad, w_hi, w_lo, ng);
  wt_linv_kernel<<<n_blk * ng, TB, LINV_SMEM, s>>>(mats, ldm, m_node, es, n, n_blk, l_hi, l_lo);
  if (cudaPeekAtLastError() != cudaSuccess) return -1;
  int launches = 3;
  for (int i = 0; i < n_blk; ++i) {
    wt_split_c_kernel<<<grid_for((long long)r_pad * TB * ng), 256, 0, s>>>(rhs, ldc, c_node, n, r, r_pad, i * TB, ng, c_hi,
                                                                            c_lo);
    p.mode = 0;
    p.blk = i;
    p.a_hi = l_hi_m;
    p.a_lo = l_lo_m;
    p.a_rows = n_pad;  // one node's Linv slab: n_blk blocks of 128 rows
    p.b_hi = c_hi_m;
    p.b_lo = c_lo_m;
    p.n_rt = 1;
    wtable_gemm_kernel<<<p.n_ct * ng, NTHR, SMEM, s>>>(p);
    launches += 2;
    const int rows_below = n - (i + 1) * TB;
    if (rows_below > 0) {
      p.mode = 1;
      p.a_hi = w_hi_m;
      p.a_lo = w_lo_m;
      p.a_rows = n_pad;
      p.b_hi = z_hi_m;
      p.b_lo = z_lo_m;
      p.n_rt = (rows_below + TB - 1) / TB;
      wtable_gemm_kernel<<<p.n_rt * p.n_ct * ng, NTHR, SMEM, s>>>(p);
      ++launches;
    }
    if (cudaPeekAtLastError() != cudaSuccess) return -1;
  }
  return launches;
}

int launch_widen_real(const float* src, long long src_node, void* dst, long long dst_node, long long per, int nb,
                      cudaStream_t s) {
  widen_kernel<<<grid_for(per * nb), 256, 0, s>>>(src, src_node, static_cast<float2*>(dst), dst_node, per, nb);
  return cudaPeekAtLastError() == cudaSuccess ? 1 : -1;
}

}  // namespace gwc
