// Internal declarations of libgwc (not part of the ABI).
#pragma once

#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <cstdint>
#include <string>
#include <vector>

#include "../../include/gwc.h"

namespace gwc {

// ------------------------------------------------------------------------------------------
// Scalar traits for the dielectric matrices: real/complex, float/double.
// Complex matrices are complex SYMMETRIC (eps(z)^T = eps(z)); no conjugation anywhere.
// ------------------------------------------------------------------------------------------
template <typename S> struct ST;
template <> struct ST<float> { using R = float; static constexpr bool kComplex = false; };
template <> struct ST<double> { using R = double; static constexpr bool kComplex = false; };
template <> struct ST<float2> { using R = float; static constexpr bool kComplex = true; };
template <> struct ST<double2> { using R = double; static constexpr bool kComplex = true; };

__host__ __device__ inline float sadd(float a, float b) { return a + b; }
__host__ __device__ inline double sadd(double a, double b) { return a + b; }
__host__ __device__ inline float2 sadd(float2 a, float2 b) { return make_float2(a.x + b.x, a.y + b.y); }
__host__ __device__ inline double2 sadd(double2 a, double2 b) { return make_double2(a.x + b.x, a.y + b.y); }
__host__ __device__ inline float ssub(float a, float b) { return a - b; }
__host__ __device__ inline double ssub(double a, double b) { return a - b; }
__host__ __device__ inline float2 ssub(float2 a, float2 b) { return make_float2(a.x - b.x, a.y - b.y); }
__host__ __device__ inline double2 ssub(double2 a, double2 b) { return make_double2(a.x - b.x, a.y - b.y); }
__host__ __device__ inline float smul(float a, float b) { return a * b; }
__host__ __device__ inline double smul(double a, double b) { return a * b; }
__host__ __device__ inline float2 smul(float2 a, float2 b) {
  return make_float2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
__host__ __device__ inline double2 smul(double2 a, double2 b) {
  return make_double2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
// c - a*b
__host__ __device__ inline float sfnms(float a, float b, float c) { return fmaf(-a, b, c); }
__host__ __device__ inline double sfnms(double a, double b, double c) { return fma(-a, b, c); }
__host__ __device__ inline float2 sfnms(float2 a, float2 b, float2 c) {
  return make_float2(fmaf(-a.x, b.x, fmaf(a.y, b.y, c.x)), fmaf(-a.x, b.y, fmaf(-a.y, b.x, c.y)));
}
__host__ __device__ inline double2 sfnms(double2 a, double2 b, double2 c) {
  return make_double2(fma(-a.x, b.x, fma(a.y, b.y, c.x)), fma(-a.x, b.y, fma(-a.y, b.x, c.y)));
}
__host__ __device__ inline float sinv(float a) { return 1.0f / a; }
__host__ __device__ inline double sinv(double a) { return 1.0 / a; }
__host__ __device__ inline float2 sinv(float2 a) {
  float d = a.x * a.x + a.y * a.y;
  return make_float2(a.x / d, -a.y / d);
}
__host__ __device__ inline double2 sinv(double2 a) {
  double d = a.x * a.x + a.y * a.y;
  return make_double2(a.x / d, -a.y / d);
}
__host__ __device__ inline double sabs2(float a) { return (double)a * a; }
__host__ __device__ inline double sabs2(double a) { return a * a; }
__host__ __device__ inline double sabs2(float2 a) { return (double)a.x * a.x + (double)a.y * a.y; }
__host__ __device__ inline double sabs2(double2 a) { return a.x * a.x + a.y * a.y; }
template <typename S> __host__ __device__ inline S szero();
template <> __host__ __device__ inline float szero<float>() { return 0.f; }
template <> __host__ __device__ inline double szero<double>() { return 0.0; }
template <> __host__ __device__ inline float2 szero<float2>() { return make_float2(0.f, 0.f); }
template <> __host__ __device__ inline double2 szero<double2>() { return make_double2(0.0, 0.0); }
template <typename S> __host__ __device__ inline S sfrom(double re, double im);
template <> __host__ __device__ inline float sfrom<float>(double re, double) { return (float)re; }
template <> __host__ __device__ inline double sfrom<double>(double re, double) { return re; }
template <> __host__ __device__ inline float2 sfrom<float2>(double re, double im) { return make_float2((float)re, (float)im); }
template <> __host__ __device__ inline double2 sfrom<double2>(double re, double im) { return make_double2(re, im); }
__host__ __device__ inline double sre(float a) { return a; }
__host__ __device__ inline double sre(double a) { return a; }
__host__ __device__ inline double sre(float2 a) { return a.x; }
__host__ __device__ inline double sre(double2 a) { return a.x; }
__host__ __device__ inline double sim(float) { return 0.0; }
__host__ __device__ inline double sim(double) { return 0.0; }
__host__ __device__ inline double sim(float2 a) { return a.y; }
__host__ __device__ inline double sim(double2 a) { return a.y; }

#ifdef __CUDACC__
// Butterfly exchange within a warp (all 32 lanes take part) of a scalar of each kind.
__device__ inline float shfl_xor_s(float v, int m) { return __shfl_xor_sync(0xffffffffu, v, m); }
__device__ inline double shfl_xor_s(double v, int m) { return __shfl_xor_sync(0xffffffffu, v, m); }
__device__ inline float2 shfl_xor_s(float2 v, int m) {
  return make_float2(__shfl_xor_sync(0xffffffffu, v.x, m), __shfl_xor_sync(0xffffffffu, v.y, m));
}
__device__ inline double2 shfl_xor_s(double2 v, int m) {
  return make_double2(__shfl_xor_sync(0xffffffffu, v.x, m), __shfl_xor_sync(0xffffffffu, v.y, m));
}
#endif

// Device status bits (ORed into ctx->d_status[0]).
enum : unsigned { kStatSingular = 1u, kStatNotConverged = 2u, kStatTimeout = 4u, kStatBadIndex = 8u };

// Which arithmetic a batch of dielectric matrices lives in.
enum class MatKind { RealF32, CplxF32, RealF64, CplxF64 };

inline size_t mat_elem_bytes(MatKind k) {
  switch (k) {
    case MatKind::RealF32: return 4;
    case MatKind::CplxF32: return 8;
    case MatKind::RealF64: return 8;
    default: return 16;
  }
}

// ------------------------------------------------------------------------------------------
// Kernel launchers (each returns the number of kernels it launched, or -1 on a launch error)
// ------------------------------------------------------------------------------------------

// D table: D_f(k) = 4 Delta_k / (z_f^2 - Delta_k^2) for the batch, FP64 (dre,dim) or FP32.
// Layout: [F][2][ld] with ld >= n_ov; entries k >= n_ov are 0.
int launch_dtable(const double* z, int F, const double* delta, int n_ov, int ld, bool fp32, void* out,
                  cudaStream_t s);

// SIMT chi0: out[f] (type per kind, leading dim ldm) = alpha*Pi(z_f) + beta*I, lower triangle
// (and the full square if full != 0). dtab from launch_dtable (same precision as the kernel).
int launch_chi0_simt(MatKind kind, const void* o_ov /*double or float [n_aux][ldo]*/, int ldo, int n_aux, int n_ov,
                     const void* dtab, int ld_dtab, int F, double alpha, double beta, void* out, long long ldm,
                     long long mat_stride, int full, const int* active, cudaStream_t s);

// tcgen05 chi0 (BF16 or split BF16): same output contract as launch_chi0_simt for complex
// kinds (CplxF32) and real (RealF32). Returns -1 if unavailable.
int launch_chi0_tc(bool split3, const __nv_bfloat16* o_hi, const __nv_bfloat16* o_lo, const float* o_f32, int ld_pad,
                   int n_aux, int n_aux_pad, int n_ov_pad, const float* dtab, int ld_dtab, int F, bool complex_out,
                   double alpha, double beta, void* out, long long ldm, long long mat_stride, const int* active,
                   unsigned* status, unsigned long long wait_ns, bool out64 /*FP64 matrices*/, cudaStream_t s,
                   int persist = 0 /*0: one CTA per item; > 0: at most that many CTAs looping over items*/);
// Grouped chi0: several molecules' frequency batches in one launch. chi0_group_fill writes one descriptor
// (chi0_group_bytes() bytes, 64-byte aligned in device memory) whose items are numbered from item0 and
// returns its item count (or -2 if unsupported); launch_chi0_tc_grouped runs n_items items of the
// n_groups descriptors (ascending item0) on `grid` CTAs, each looping over items.
size_t chi0_group_bytes();
int chi0_group_fill(void* dst, bool split3, const __nv_bfloat16* o_hi, const __nv_bfloat16* o_lo, const float* o_f32,
                    int ld_pad, int n_aux, int n_aux_pad, int n_ov_pad, const float* dtab, int ld_dtab, int F,
                    bool complex_out, double alpha, double beta, void* out, long long ldm, long long mat_stride,
                    const int* active, bool out64, int item0);
int launch_chi0_tc_grouped(const void* d_groups, int n_groups, int n_items, bool complex_out, int grid, unsigned* status,
                           unsigned long long wait_ns, cudaStream_t s);
// Split factorisation of F complex FP32 matrices (same layout and result as launch_ldlt_tc): per 64-column
// panel one panel launch (one CTA per matrix) and one batched tensor-core trailing update over all matrices.
// `work` holds ldlt_split_bytes(n, nrow, F) bytes. Returns the launches, -1 on a launch error or bad layout,
// -2 if unsupported.
size_t ldlt_split_bytes(int n, int nrow, int F);
int launch_ldlt_split(void* mats, int n, int nrow, long long ldm, long long stride, int F, const int* active,
                      unsigned* status, unsigned long long wait_ns, void* work, size_t work_bytes, cudaStream_t s);

// Imaginary-axis W table on the tensor cores: for ng factored real matrices (eps = L D L^T; element (P, Q) of node
// u at mats[u m_node + (P ldm + Q) es] in floats, es = 2 for the real parts of complex FP32 storage) and their
// right-hand sides ([node][r][ldc] FP32, rewritten), table[node][col] = sum_p y_p^2 / d_p - bnorm[node][col] with
// y = L^-1 b (table node stride t_node = r). `work` holds wtable_tc_bytes(n, r, ng) bytes (16-byte aligned).
// Returns the launches, -1 on a launch error, -2 if unsupported.
size_t wtable_tc_bytes(int n_aux, int r, int ng);
// dst[u][e] = (src[u][e], 0), e < per, u < nb (real matrices into complex FP32 storage)
int launch_widen_real(const float* src, long long src_node, void* dst, long long dst_node, long long per, int nb,
                      cudaStream_t s);
int launch_wtable_tc(const float* mats, int es, int n, long long ldm, long long m_node, float* rhs, long long ldc, long long c_node,
                     int r, int ng, const double* bnorm, double* table, long long t_node, void* work, size_t work_bytes,
                     unsigned* status, unsigned long long wait_ns, cudaStream_t s);

// The same three entry points for the CTA-pair kernel (256 x 128 pair tiles, tcgen05 cta_group::2): same
// arguments and output contract; `persist` / `grid` count CTAs (two per cluster).
int launch_chi0_pair(bool split3, const __nv_bfloat16* o_hi, const __nv_bfloat16* o_lo, const float* o_f32, int ld_pad,
                     int n_aux, int n_aux_pad, int n_ov_pad, const float* dtab, int ld_dtab, int F, bool complex_out,
                     double alpha, double beta, void* out, long long ldm, long long mat_stride, const int* active,
                     unsigned* status, unsigned long long wait_ns, bool out64, cudaStream_t s, int persist);
size_t chi0_pair_group_bytes();
int chi0_pair_group_fill(void* dst, bool split3, const __nv_bfloat16* o_hi, const __nv_bfloat16* o_lo, const float* o_f32,
                         int ld_pad, int n_aux, int n_aux_pad, int n_ov_pad, const float* dtab, int ld_dtab, int F,
                         bool complex_out, double alpha, double beta, void* out, long long ldm, long long mat_stride,
                         const int* active, bool out64, int item0);
int launch_chi0_pair_grouped(const void* d_groups, int n_groups, int n_items, bool complex_out, int grid,
                             unsigned* status, unsigned long long wait_ns, cudaStream_t s);

// Batched in-place LDL^T of F matrices [nrow][ldm]: the first n columns are factored (W = L D below
// the diagonal, d on it, L^T above it); rows n..nrow-1 are appended right-hand sides that the row
// solves turn into y = L^-1 b. Zero pivot -> status |= kStatSingular.
int launch_ldlt(MatKind kind, void* mats, int n, int nrow, long long ldm, long long mat_stride, int F, const int* active,
                unsigned* status, cudaStream_t s);
// Same contract for complex FP32 matrices, trailing updates on the tensor cores (3xTF32).
// Returns -2 if the device has no tcgen05.
int launch_ldlt_tc(void* mats, int n, int nrow, long long ldm, long long mat_stride, int F, const int* active,
                   unsigned* status, unsigned long long wait_ns, cudaStream_t s);
// Grouped tensor-core factorisation: several batches of complex FP32 matrices (of different sizes) in one
// launch, one CTA per matrix; group g owns CTAs cta0 .. cta0 + F - 1 (groups ascending in cta0). The
// layout rules of launch_ldlt_tc hold per group (ldm, stride multiples of 4, 16-byte aligned mats).
struct LdltGroup {
  float2* mats;
  long long ldm, stride;
  const int* active;  // per matrix, or null
  int n, nrow, F, cta0;
};
int launch_ldlt_tc_grouped(const LdltGroup* d_groups, int n_groups, int n_ctas, unsigned* status,
                           unsigned long long wait_ns, cudaStream_t s);
// Appended rows: row n+q of matrix f = o_core row row_of[f*r+q]; bnorm2 = |b|^2.
int launch_border_rows(MatKind kind, void* mats, int n, long long ldm, long long stride, const double* src,
                       long long src_row_stride, const int* row_of, int F, int r, double* bnorm2, cudaStream_t s);
// w[f][q] = sum_k y_k^2 / d_k - bnorm2[f][q] from the factored appended rows (FP64 accumulation).
int launch_border_w(MatKind kind, const void* mats, int n, long long ldm, long long stride, int F, int r,
                    const double* bnorm2, double* w, long long w_stride, const int* active, cudaStream_t s);

// Right-hand sides: rhs (S type) [F][r][ldr] overwritten by y = L^{-1} b; then
// w[f][q] = sum_k y_k^2 / d_k - bnorm2[f][q] (FP64 complex out, interleaved).
int launch_ldlt_solve_w(MatKind kind, const void* mats, int n, long long ldm, long long mat_stride, void* rhs, int r,
                        long long ldr, long long rhs_stride, const double* bnorm2, int F, double* w,
                        long long w_stride, const int* active, cudaStream_t s);

// Convert FP64 right-hand sides to the matrix kind: src rows given by an index map.
// dst[f][q][p] = src[row(f,q)][p]; bnorm2[f][q] = sum_p src^2 (FP64).
int launch_rhs_gather(MatKind kind, const double* src, long long src_row_stride, const int* row_of /*[F*r]*/, int F,
                      int r, int n_aux, void* dst, long long ldr, long long rhs_stride, double* bnorm2,
                      cudaStream_t s);

// Residue batch helpers ------------------------------------------------------------------
int launch_fill_z_pairs(const double* eps, const int* pair_m, const double* pair_w, int n_pairs, double eta, double* z,
                        cudaStream_t s);

// Self-energy assembly on a grid: see sigma.cu
// sigma [n_core][2] = Sigma^c_j(omega_j) of core j at its own frequency; wres1 [pair][2] (one RHS per pair)
int launch_sigma_diag(const double* eps, int n_states, int n_core, const double* omega, double eps_f, const double* xi,
                      const double* wxi, int n_im, const double* wim, const int* pidx, const double* wres1, double* sigma,
                      cudaStream_t s);
// e[k] = eps_k + sx_k - vxc_k + Re sigma[k] (sigma [n][2]); diff_bits = max |change| as double bits
int launch_evgw0_update(const double* eps, const double* sx, const double* vxc, const double* sigma, int n, double* e,
                        unsigned long long* diff_bits, cudaStream_t s);
int launch_sigma_grid(const double* eps, int n_states, int n_core, const int* core_idx, const double* omega, int n_w,
                      double eps_f, const double* xi, const double* wxi, int n_im, const double* wim,
                      const int* pidx /*[n_w][n_states] -> pair or -1*/, const double* wres /*[pair][n_core][2]*/,
                      int dec_mode, const int* group_of_core, double* sigma /*[n_core][n_w][2]*/,
                      double* im_dec /*[n_core][n_w] or null*/, cudaStream_t s);

int launch_sigma_x(const double* o_core, int n_occ, int n_core, int n_aux, double* sx, cudaStream_t s);

// QP (device-side secant state machine); see qp.cu
struct QpState {
  double x0, g0, x1, g1, dh, w_eval;
  int phase, it, done, pad;
};
// mask [n_core] (or null: every core): cores with mask 0 are not solved (NaN results, 0 iterations)
int launch_qp_init(const double* eps, const int* core_idx, int n_core, const int* mask, QpState* st, cudaStream_t s);
int launch_qp_pairs(const double* eps, const int* core_idx, int n_core, int n_occ, double eps_f, double eta,
                    const QpState* st, double* z, int* active, double* fac, int* all_done,
                    unsigned long long* active_count /*+= active pairs, or null*/, cudaStream_t s);
int launch_qp_assemble_update(const double* eps, int n_states, int n_occ, int n_core, const int* core_idx,
                              double eps_f, const double* xi, const double* wxi, int n_im, const double* wim,
                              const double* wpair /*[n_core*n_occ][2]*/, const double* fac, const double* sx,
                              const double* vxc, double tol, int max_iter, int g0w0, QpState* st, int* all_done,
                              cudaStream_t s);
// Graphical solutions of the plain G0W0 QP equation on a grid: roots [n_core][max_roots][2] = (w, Z),
// n_roots [n_core] = number found (may exceed max_roots; only the first max_roots stored).
int launch_g0w0_scan(const double* omega, int n_w, const double* sigma, const double* eps, const int* core_idx,
                     const double* sx, const double* vxc, int n_core, int max_roots, double* roots, int* n_roots,
                     cudaStream_t s);
int launch_qp_finish(const QpState* st, int n_core, double* eps_qp, double* dh, int* iters, unsigned* status,
                     cudaStream_t s);
// eps_qp = eps_n + dH_n after the phase-0 round (closed form of the G_dH W0 QP equation)
int launch_qp_finish_hedin(const QpState* st, const double* eps, const int* core_idx, int n_core, double* eps_qp,
                           double* dh, int* iters, cudaStream_t s);

// CD-WAC: continued-fraction coefficients per (occupied m, core c) and the self-energy from them
int launch_thiele_fit(const double* wim, int n_states, int n_core, int n_im, const double* wref, int n_ref, int n_pairs,
                      const double* zref, double* coef, cudaStream_t s);
int launch_sigma_grid_wac(const double* eps, int n_states, int n_occ, int n_core, const int* core_idx, const double* omega,
                          int n_w, double eps_f, double eta, const double* xi, const double* wxi, int n_im,
                          const double* wim, const double* coef, const double* zref, int n_pts, double* sigma,
                          double* im_dec, unsigned* status, cudaStream_t s);

int launch_gdh_spectrum(const double* eps, const int* core_idx, int n_core, const double* omega, int n_w,
                        const double* sigma, const double* dh, const double* sx, const double* vxc, double* a,
                        double* w_out, cudaStream_t s);

// Request mode: im[c][j] = f_c(eps_c + w_j) Im W[pair_of[j]][c] (0 when pair_of[j] < 0).
int launch_request_dec(const double* eps, const int* core_idx, int n_core, double eps_f, const double* omega_rel, int n_w,
                       const int* pair_of, const double* wpair, double* im, cudaStream_t s);

// Cumulant + FFT; see cumulant.cu
int launch_cumulant_spectrum(const double* omega_rel, int n_w, const double* im_sigma, int n_core, int n_t,
                             double t_max, double eta, double* work_a /*[n_core][n_t][2]*/,
                             double* work_b /*[n_core][n_t][2]*/, double* coef /*[n_core][n_w]*/,
                             double* twiddle /*[n_t/2][2]*/, double* a_out, double* nu_out, cudaStream_t s);

// Sets the message returned by gwc_last_error(NULL) (calls without a context).
void set_noctx_error(const char* msg);

// Precision copies of O_ov: hi/lo BF16 and FP32, padded [n_aux_pad][n_ov_pad], zero padding.
int launch_split_o(const double* o_ov, int n_aux, int n_ov, int n_aux_pad, int n_ov_pad, __nv_bfloat16* hi,
                   __nv_bfloat16* lo, float* f32, cudaStream_t s);

int launch_delta(const double* eps, int n_occ, int n_virt, double* delta, cudaStream_t s);

// Chi0 output conversion for the public gwc_build_chi0 (any kind -> FP64 complex full).
int launch_mat_to_c128(MatKind kind, const void* mats, int n, long long ldm, long long mat_stride, int F, double* out,
                       cudaStream_t s);

}  // namespace gwc

// ------------------------------------------------------------------------------------------
// Context
// ------------------------------------------------------------------------------------------
struct gwc_ctx {
  int device = 0;
  int n_states = 0, n_occ = 0, n_virt = 0, n_aux = 0, n_core = 0, n_ov = 0;
  int n_aux_pad = 0, n_ov_pad = 0;
  gwc_options opt{};
  bool loaded = false;  // a system's arrays are resident (gwc_create with arrays, or gwc_load)
  unsigned long long wait_ns = 1000000000ull;  // bound of the tensor-core kernels' device waits
  double eps_f = 0.0;
  bool vxc_given = false;
  std::vector<double> h_eps;
  std::vector<int> h_core, h_group;

  double *d_eps = nullptr, *d_o_ov = nullptr, *d_o_core = nullptr, *d_vxc = nullptr, *d_delta = nullptr;
  int* d_core_idx = nullptr;
  int* d_group = nullptr;
  double *d_xi = nullptr, *d_wxi = nullptr;
  double* d_wim = nullptr;  // [n_im + 1][n_states][n_core]; node n_im is xi = 0
  bool wim_valid = false;
  double* d_sx = nullptr;   // [n_core]
  double* d_vxc_eff = nullptr;  // [n_core] v^xc actually used

  __nv_bfloat16 *d_o_hi = nullptr, *d_o_lo = nullptr;
  float* d_o_f32 = nullptr;
  float* d_o_f32_unpadded = nullptr;  // not used

  // workspace
  int batch = 0;            // matrices per batch
  void* d_mats = nullptr;   // batch * n_aux * ldm elements of the widest kind
  long long ldm = 0;        // leading dimension of matrices
  int n_sm = 1;             // streaming multiprocessors of the device
  int wim_group = 1;        // imaginary-axis nodes whose solves share one launch
  bool factor_tc = true;    // complex FP32 factorisations on the tensor cores (mixed-precision modes)
  bool chi0_pair = false;   // tensor-core chi0 on CTA pairs (cta_group::2) instead of one CTA per tile
  bool wtable_tc = false;   // imaginary-axis W-table solves on the tensor cores (else the SIMT forward substitution)
  bool factor_split = false;  // complex FP32 factorisations as panel launches + batched tensor-core updates
  void* d_lp = nullptr;     // their TF32 planes, lp_bytes bytes
  size_t lp_bytes = 0;
  void* d_wt = nullptr;     // their workspace (TF32 planes), wt_bytes bytes
  size_t wt_bytes = 0;
  int border_max = 0;       // right-hand sides that may be appended as rows (matrix rows n_aux + border_max)
  size_t mats_bytes = 0;
  void* d_dtab = nullptr;   // [batch][2][ld_dtab] FP64-sized
  int ld_dtab = 0;
  double* d_z = nullptr;    // [batch][2]
  int* d_active = nullptr;  // [batch]
  void* d_rhs = nullptr;    // residue RHS [batch][n_core][n_aux] widest kind
  size_t rhs_bytes = 0;
  double* d_bnorm = nullptr;  // [max(batch*n_core, rhs_im)]
  int* d_rowmap = nullptr;    // [batch * n_core]
  double* d_wtmp = nullptr;   // [max(batch*n_core, wim_group*n_states*n_core)][2]
  void* d_rhs_im = nullptr;   // imaginary-axis RHS [wim_group][n_states*n_core][ldm] (widest real kind)
  unsigned* d_status = nullptr;

  // residue grid plan
  int plan_cap = 0;
  int* d_pidx = nullptr;      // [n_w][n_states]
  double* d_wres = nullptr;   // [n_pairs][n_core][2]
  int* d_pair_m = nullptr;
  double* d_pair_w = nullptr;
  double* d_pair_z = nullptr;   // [n_pairs][2]
  int* d_pair_rows = nullptr;   // [n_pairs][n_core]
  double* d_grid_w = nullptr;
  int pidx_cap = 0, wres_cap = 0, grid_cap = 0;

  // QP
  gwc::QpState* d_qp = nullptr;
  double* d_qp_z = nullptr;     // [n_core*n_occ][2]
  int* d_qp_active = nullptr;   // [n_core*n_occ]
  double* d_qp_fac = nullptr;   // [n_core*n_occ]
  double* d_qp_w = nullptr;     // [n_core*n_occ][2]
  int* d_qp_rowmap = nullptr;   // [n_core*n_occ]
  int* d_all_done = nullptr;
  int* d_qp_mask = nullptr;     // [n_core] cores whose QP energies are computed (gwc_set_qp_cores)
  bool qp_mask_set = false;
  // builds of masked launches (QP rounds) that are not skipped: counted on the device, folded into
  // the stats by gwc_get_stats / gwc_reset_stats
  unsigned long long* d_active_builds = nullptr;
  unsigned long long active_folded = 0;

  // cumulant
  double *d_cw_a = nullptr, *d_cw_b = nullptr, *d_coef = nullptr, *d_tw = nullptr;
  size_t cw_cap = 0, coef_cap = 0;

  // imaginary-axis frequencies (0, xi_k) and (0, 0), uploaded at creation
  double* d_zim = nullptr;  // [n_im + 1][2]
  int batch_cap = 0;        // batch the workspace was sized for (gwc_autotune may lower batch)

  // request mode
  int req_n_omega = 0, req_n_pairs = 0;
  double* d_req_wrel = nullptr;    // [n_core][n_omega] relative grid (same row for every core)
  double* d_req_z = nullptr;       // [n_pairs][2]
  int* d_req_rows = nullptr;       // [n_pairs][n_core]
  int* d_req_pair_of = nullptr;    // [n_omega] -> pair or -1
  double* d_req_w = nullptr;       // [n_pairs][n_core][2]
  double* d_req_im = nullptr;      // [n_core][n_omega]
  double *d_req_a = nullptr, *d_req_nu = nullptr;
  double *d_req_eqp = nullptr, *d_req_dh = nullptr;
  int* d_req_it = nullptr;

  // orbital energies in G (gwc_set_g_energies): the input energies unless set; W always uses d_eps
  bool g_set = false;
  std::vector<double> h_eps_g;
  double* d_eps_g = nullptr;
  double eps_f_g = 0.0;
  bool cores_occupied = true;   // every core_idx < n_occ (needed by the QP, request and CD-WAC paths)
  double* d_ev_sig = nullptr;   // evGW0: [n_states][2] Sigma^c_j(eps_j) at the current energies
  unsigned long long* d_ev_diff = nullptr;  // evGW0: max |eps_new - eps| as the bits of a double
  // evGW0 diagonal residue plan: pair (j, m) with one right-hand side o_mj
  int* d_ev_pidx = nullptr;      // [n_states][n_states] -> pair or -1
  int* d_ev_pm = nullptr;        // [pairs] residue state m
  double* d_ev_pw = nullptr;     // [pairs] frequency e_j
  double* d_ev_z = nullptr;      // [pairs][2]
  int* d_ev_rows = nullptr;      // [pairs] o_core row m * n_core + j
  double* d_ev_wres = nullptr;   // [pairs][2]
  double* d_ev_w = nullptr;      // [n_states] current energies
  size_t ev_pair_cap = 0;

  // element counts (bytes where named so) the shape-sized buffers were allocated with, at creation; a
  // smaller system may be loaded into the context as long as every count fits (gwc_load)
  struct Caps {
    size_t n_states = 0, n_core = 0, n_ov = 0, o_ov = 0, o_core = 0, o_pad = 0, plane = 0, qp_np = 0;
    size_t mats_bytes = 0, dtab = 0, rhs_bytes = 0, rhs_im_bytes = 0, bnorm = 0;
    int batch = 0;
  } cap;
  // grow-only request-mode buffers: element counts allocated
  size_t req_cap_wrel = 0, req_cap_z = 0, req_cap_rows = 0, req_cap_pair = 0, req_cap_w = 0, req_cap_im = 0,
         req_cap_a = 0, req_cap_nu = 0, req_cap_core = 0;

  // host staging
  int* h_pin_i = nullptr;
  size_t h_pin_i_cap = 0;
  double* h_pin_d = nullptr;
  size_t h_pin_d_cap = 0;

  gwc_stats stats{};
  std::string last_error;

  // profile mode: (class, start, stop) events pending resolution
  struct EvRec {
    int cls;
    cudaEvent_t a, b;
  };
  std::vector<EvRec> ev_pending;
  std::vector<cudaEvent_t> ev_pool;
};
