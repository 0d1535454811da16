// C ABI of libgwc: context, residency, batching of frequencies, and the host-side
// control of the self-energy, QP and cumulant steps. Every arithmetic step of the
// path runs in the kernels of this library; the host only plans and launches.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <limits>
#include <map>
#include <mutex>
#include <tuple>
#include <string>
#include <vector>

#include "gwc_internal.h"

using namespace gwc;

namespace {

thread_local std::string g_create_error;

const double kPi = 3.14159265358979323846;

gwc_status fail(gwc_ctx* ctx, gwc_status st, const std::string& msg) {
  if (ctx)
    ctx->last_error = msg;
  else
    g_create_error = msg;
  return st;
}

#define CU(call)                                                                                   \
  do {                                                                                             \
    cudaError_t e_ = (call);                                                                       \
    if (e_ != cudaSuccess)                                                                         \
      return fail(ctx, e_ == cudaErrorMemoryAllocation ? GWC_ERR_OOM : GWC_ERR_CUDA,               \
                  std::string(#call) + ": " + cudaGetErrorString(e_));                            \
  } while (0)

#define LAUNCH(expr)                                                                               \
  do {                                                                                             \
    int n_ = (expr);                                                                               \
    if (n_ < 0) {                                                                                  \
      cudaError_t e_ = cudaGetLastError();                                                         \
      return fail(ctx, GWC_ERR_CUDA, std::string("launch failed: ") + #expr + ": " + cudaGetErrorString(e_)); \
    }                                                                                              \
    ctx->stats.kernel_launches += n_;                                                              \
  } while (0)

inline long long round_up(long long x, long long m) { return (x + m - 1) / m * m; }

// ---- profile mode: CUDA events around the timed kernel classes ------------------------------
enum { kClsChi0 = 0, kClsFactor = 1, kClsSolve = 2 };

cudaEvent_t ev_get(gwc_ctx* ctx) {
  if (!ctx->ev_pool.empty()) {
    cudaEvent_t e = ctx->ev_pool.back();
    ctx->ev_pool.pop_back();
    return e;
  }
  cudaEvent_t e = nullptr;
  cudaEventCreate(&e);
  return e;
}

cudaEvent_t ev_begin(gwc_ctx* ctx, cudaStream_t st) {
  if (!ctx->opt.profile) return nullptr;
  cudaEvent_t a = ev_get(ctx);
  cudaEventRecord(a, st);
  return a;
}

void ev_end(gwc_ctx* ctx, int cls, cudaEvent_t a, cudaStream_t st) {
  if (!ctx->opt.profile || !a) return;
  cudaEvent_t b = ev_get(ctx);
  cudaEventRecord(b, st);
  ctx->ev_pending.push_back({cls, a, b});
}

// Folds the elapsed times of completed records into the stats (synchronises on the last one).
void ev_flush(gwc_ctx* ctx) {
  if (ctx->ev_pending.empty()) return;
  cudaEventSynchronize(ctx->ev_pending.back().b);
  for (auto& r : ctx->ev_pending) {
    float ms = 0.f;
    if (cudaEventElapsedTime(&ms, r.a, r.b) == cudaSuccess) {
      if (r.cls == kClsChi0) {
        ctx->stats.chi0_ms += ms;
        ctx->stats.chi0_launches += 1;
      } else if (r.cls == kClsFactor) {
        ctx->stats.factor_ms += ms;
        ctx->stats.factor_launches += 1;
      } else {
        ctx->stats.solve_ms += ms;
        ctx->stats.solve_launches += 1;
      }
    }
    ctx->ev_pool.push_back(r.a);
    ctx->ev_pool.push_back(r.b);
  }
  ctx->ev_pending.clear();
}

// Gauss-Legendre nodes and weights on (-1, 1), ascending, by Newton iteration on P_n
// (three-term recurrence; initial guesses cos(pi (i - 1/4)/(n + 1/2))).
void gauss_legendre(int n, std::vector<double>& x, std::vector<double>& w) {
  x.assign(n, 0.0);
  w.assign(n, 0.0);
  for (int i = 0; i < (n + 1) / 2; ++i) {
    double z = std::cos(kPi * (i + 0.75) / (n + 0.5));
    double dp = 1.0;
    for (int it = 0; it < 100; ++it) {
      double p0 = 1.0, p1 = z;
      for (int k = 2; k <= n; ++k) {
        double p2 = ((2.0 * k - 1.0) * z * p1 - (k - 1.0) * p0) / k;
        p0 = p1;
        p1 = p2;
      }
      if (n == 1) {
        p1 = z;
        p0 = 1.0;
      }
      dp = n * (z * p1 - p0) / (z * z - 1.0);
      double dz = p1 / dp;
      z -= dz;
      if (std::fabs(dz) < 1e-16) break;
    }
    // recompute derivative at the converged node
    double p0 = 1.0, p1 = z;
    for (int k = 2; k <= n; ++k) {
      double p2 = ((2.0 * k - 1.0) * z * p1 - (k - 1.0) * p0) / k;
      p0 = p1;
      p1 = p2;
    }
    dp = n == 1 ? 1.0 : n * (z * p1 - p0) / (z * z - 1.0);
    double wt = 2.0 / ((1.0 - z * z) * dp * dp);
    x[i] = -z;
    x[n - 1 - i] = z;
    w[i] = wt;
    w[n - 1 - i] = wt;
  }
  if (n % 2 == 1) x[n / 2] = 0.0;
}

// Modes whose dielectric matrices (factorisation, solves, residue contractions) are FP64.
bool factor64(int prec) { return prec == GWC_PREC_FP64 || prec == GWC_PREC_BF16X3_F64; }
MatKind real_kind(const gwc_ctx* c) { return factor64(c->opt.prec) ? MatKind::RealF64 : MatKind::RealF32; }
MatKind cplx_kind(const gwc_ctx* c) { return factor64(c->opt.prec) ? MatKind::CplxF64 : MatKind::CplxF32; }

template <typename T>
gwc_status dalloc(gwc_ctx* ctx, T** p, size_t count) {
  if (*p) {
    cudaFree(*p);
    *p = nullptr;
  }
  if (count == 0) count = 1;
  cudaError_t e = cudaMalloc((void**)p, count * sizeof(T));
  if (e != cudaSuccess) {
    *p = nullptr;
    return fail(ctx, GWC_ERR_OOM, std::string("cudaMalloc(") + std::to_string(count * sizeof(T)) + "): " + cudaGetErrorString(e));
  }
  return GWC_OK;
}

// (Re)allocates *p only when `count` exceeds the capacity *cap (grow-only buffers).
template <typename T>
gwc_status grow(gwc_ctx* ctx, T** p, size_t* cap, size_t count) {
  if (*p && count <= *cap) return GWC_OK;
  gwc_status r = dalloc(ctx, p, count);
  *cap = r == GWC_OK ? std::max<size_t>(count, 1) : 0;
  return r;
}

#define TRY(x)                     \
  do {                             \
    gwc_status s_ = (x);           \
    if (s_ != GWC_OK) return s_;   \
  } while (0)

gwc_status validate_system(const gwc_system* s) {
  if (!s) return fail(nullptr, GWC_ERR_INVALID_ARG, "system is NULL");
  if (s->n_states < 2 || s->n_occ < 1 || s->n_occ >= s->n_states || s->n_aux < 1 || s->n_core < 1 ||
      s->n_core > s->n_states)
    return fail(nullptr, GWC_ERR_INVALID_ARG,
                "invalid sizes (need n_states>=2, 1<=n_occ<n_states, n_aux>=1, 1<=n_core<=n_states)");
  if (s->n_aux > 65536 || s->n_states > 65536) return fail(nullptr, GWC_ERR_INVALID_ARG, "n_aux and n_states must be <= 65536");
  if ((long long)s->n_occ * (s->n_states - s->n_occ) > (1LL << 31) - 1)
    return fail(nullptr, GWC_ERR_INVALID_ARG, "n_occ * n_virt too large");
  if (!s->core_idx && !s->eps && !s->o_ov && !s->o_core) return GWC_OK;  // sizes only (a capacity for gwc_create)
  if (!s->core_idx || !s->eps || !s->o_ov || !s->o_core) return fail(nullptr, GWC_ERR_INVALID_ARG, "NULL input pointer");
  for (int c = 0; c < s->n_core; ++c)
    if (s->core_idx[c] < 0 || s->core_idx[c] >= s->n_states)
      return fail(nullptr, GWC_ERR_INVALID_ARG, "core_idx must index states 0..n_states-1");
  if (s->memory != GWC_MEM_DEVICE && s->memory != GWC_MEM_HOST) return fail(nullptr, GWC_ERR_INVALID_ARG, "bad memory kind");
  return GWC_OK;
}

gwc_status validate_options(const gwc_options* o, int n_core) {
  if (!o) return fail(nullptr, GWC_ERR_INVALID_ARG, "options is NULL");
  if (!(o->eta > 0.0) || !std::isfinite(o->eta)) return fail(nullptr, GWC_ERR_INVALID_ARG, "eta must be > 0");
  if (o->n_im < 1 || o->n_im > 1024) return fail(nullptr, GWC_ERR_INVALID_ARG, "n_im must be in 1..1024");
  if (!(o->xi0 > 0.0)) return fail(nullptr, GWC_ERR_INVALID_ARG, "xi0 must be > 0");
  if (o->prec < 0 || o->prec > 4) return fail(nullptr, GWC_ERR_INVALID_ARG, "bad precision");
  if (o->dec < 0 || o->dec > 2) return fail(nullptr, GWC_ERR_INVALID_ARG, "bad decoupling mode");
  if (o->n_t < 16 || o->n_t > (1 << 22) || (o->n_t & (o->n_t - 1)))
    return fail(nullptr, GWC_ERR_INVALID_ARG, "n_t must be a power of two in 16..2^22");
  if (!(o->t_max > 0.0)) return fail(nullptr, GWC_ERR_INVALID_ARG, "t_max must be > 0");
  if (o->max_qp_iter < 2 || o->max_qp_iter > 200) return fail(nullptr, GWC_ERR_INVALID_ARG, "max_qp_iter must be in 2..200");
  if (!(o->qp_tol > 0.0)) return fail(nullptr, GWC_ERR_INVALID_ARG, "qp_tol must be > 0");
  if (o->batch < 0 || o->batch > 4096) return fail(nullptr, GWC_ERR_INVALID_ARG, "batch must be in 0..4096");
  if (o->qp_mode < 0 || o->qp_mode > 2) return fail(nullptr, GWC_ERR_INVALID_ARG, "bad qp_mode");
  if (o->wait_us < 0 || o->wait_us > 60000000) return fail(nullptr, GWC_ERR_INVALID_ARG, "wait_us must be in 0..6e7");
  if (o->chi0_ctas < 0) return fail(nullptr, GWC_ERR_INVALID_ARG, "chi0_ctas must be >= 0");
  if (o->chi0_tile < 0 || o->chi0_tile > 1) return fail(nullptr, GWC_ERR_INVALID_ARG, "chi0_tile must be 0 or 1");
  (void)n_core;
  return GWC_OK;
}

// Orbital energies in G (the poles of the Green's function) and the Fermi level of the residue
// prefactors: the input energies unless gwc_set_g_energies replaced them. W always uses d_eps.
const double* g_eps_dev(const gwc_ctx* c) { return c->g_set ? c->d_eps_g : c->d_eps; }
const std::vector<double>& g_eps_host(const gwc_ctx* c) { return c->g_set ? c->h_eps_g : c->h_eps; }
double g_eps_f(const gwc_ctx* c) { return c->g_set ? c->eps_f_g : c->eps_f; }

gwc_status need_occupied_cores(gwc_ctx* ctx, const char* what) {
  if (ctx->cores_occupied) return GWC_OK;
  return fail(ctx, GWC_ERR_INVALID_ARG, std::string(what) + " needs every core_idx to be an occupied state");
}

struct Sizes {
  int n_aux_pad, n_ov_pad, ld_dtab;
  long long ldm;
  size_t elem_c, elem_r;
};

Sizes sizes_of(const gwc_system* s, const gwc_options* o) {
  Sizes z{};
  int n_ov = s->n_occ * (s->n_states - s->n_occ);
  z.n_aux_pad = (int)round_up(s->n_aux, 128);
  z.n_ov_pad = (int)round_up(n_ov, 64);
  z.ld_dtab = z.n_ov_pad;
  z.ldm = round_up(s->n_aux, 4);
  z.elem_c = factor64(o->prec) ? 16 : 8;
  z.elem_r = factor64(o->prec) ? 8 : 4;
  return z;
}

size_t per_matrix_bytes(const gwc_system* s, const Sizes& z) {
  return (size_t)s->n_aux * z.ldm * z.elem_c + (size_t)s->n_core * z.ldm * z.elem_c + 2 * (size_t)z.ld_dtab * 8 + 256;
}

size_t resident_bytes(const gwc_system* s, const gwc_options* o, const Sizes& z) {
  size_t n_ov = (size_t)s->n_occ * (s->n_states - s->n_occ);
  size_t b = 0;
  b += (size_t)s->n_states * 8 + n_ov * 8;                         // eps, delta
  b += (size_t)s->n_aux * n_ov * 8;                                 // o_ov
  b += (size_t)s->n_states * s->n_core * s->n_aux * 8;              // o_core
  b += (size_t)(o->n_im + 1) * s->n_states * s->n_core * 8;         // W(i xi) table
  b += (size_t)s->n_states * s->n_core * z.ldm * z.elem_r;          // imaginary-axis RHS
  b += (size_t)s->n_states * s->n_core * (8 + 16 + 4);              // bnorm, w tmp, rowmap
  if (o->prec != GWC_PREC_FP64) b += (size_t)z.n_aux_pad * z.n_ov_pad * (2 + 2 + 4);
  return b;
}

// Matrices per residue batch. One factorisation occupies one SM, so a batch is a whole number of
// SM-waves (a ragged last wave idles SMs for a full factorisation time).
int choose_batch(const gwc_system* s, const gwc_options* o, const Sizes& z, int n_sm) {
  if (o->batch > 0) return o->batch;
  size_t freeb = 0, totalb = 0;
  size_t budget = (size_t)8 << 30;
  if (cudaMemGetInfo(&freeb, &totalb) == cudaSuccess) budget = std::min<size_t>((size_t)(0.35 * freeb), (size_t)24 << 30);
  size_t per = per_matrix_bytes(s, z);
  long long f = (long long)(budget / per);
  f = std::max(1LL, std::min(std::max(512LL, 4LL * n_sm), f));
  if (f >= n_sm) f -= f % n_sm;
  return (int)f;
}

gwc_status upload(gwc_ctx* ctx, void* dst, const void* src, size_t bytes, int memory, cudaStream_t st) {
  CU(cudaMemcpyAsync(dst, src, bytes, memory == GWC_MEM_HOST ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToDevice, st));
  return GWC_OK;
}

// Loads eps / O / vxc into the context and derives everything that depends only on them.
gwc_status load_system(gwc_ctx* ctx, const gwc_system* s, cudaStream_t st) {
  const size_t n_ov = (size_t)ctx->n_ov;
  ctx->h_eps.resize(s->n_states);
  if (s->memory == GWC_MEM_HOST) {
    std::memcpy(ctx->h_eps.data(), s->eps, sizeof(double) * s->n_states);
  } else {
    CU(cudaMemcpyAsync(ctx->h_eps.data(), s->eps, sizeof(double) * s->n_states, cudaMemcpyDeviceToHost, st));
    CU(cudaStreamSynchronize(st));
  }
  for (int i = 1; i < s->n_states; ++i)
    if (!(ctx->h_eps[i] >= ctx->h_eps[i - 1])) return fail(ctx, GWC_ERR_INVALID_ARG, "eps must be ascending and finite");
  ctx->eps_f = std::isnan(s->eps_f) ? 0.5 * (ctx->h_eps[s->n_occ - 1] + ctx->h_eps[s->n_occ]) : s->eps_f;
  ctx->h_core.assign(s->core_idx, s->core_idx + s->n_core);
  ctx->cores_occupied = true;
  for (int c : ctx->h_core) ctx->cores_occupied = ctx->cores_occupied && c < s->n_occ;
  ctx->g_set = false;  // G takes the (new) input energies
  TRY(upload(ctx, ctx->d_eps, s->eps, sizeof(double) * s->n_states, s->memory, st));
  TRY(upload(ctx, ctx->d_o_ov, s->o_ov, sizeof(double) * s->n_aux * n_ov, s->memory, st));
  TRY(upload(ctx, ctx->d_o_core, s->o_core, sizeof(double) * s->n_states * s->n_core * s->n_aux, s->memory, st));
  CU(cudaMemcpyAsync(ctx->d_core_idx, ctx->h_core.data(), sizeof(int) * s->n_core, cudaMemcpyHostToDevice, st));
  LAUNCH(launch_delta(ctx->d_eps, ctx->n_occ, ctx->n_virt, ctx->d_delta, st));
  if (ctx->opt.prec != GWC_PREC_FP64)
    LAUNCH(launch_split_o(ctx->d_o_ov, ctx->n_aux, ctx->n_ov, ctx->n_aux_pad, ctx->n_ov_pad, ctx->d_o_hi, ctx->d_o_lo,
                          ctx->d_o_f32, st));
  LAUNCH(launch_sigma_x(ctx->d_o_core, ctx->n_occ, ctx->n_core, ctx->n_aux, ctx->d_sx, st));
  ctx->vxc_given = s->vxc != nullptr;
  if (s->vxc)
    TRY(upload(ctx, ctx->d_vxc_eff, s->vxc, sizeof(double) * s->n_core, s->memory, st));
  else
    CU(cudaMemcpyAsync(ctx->d_vxc_eff, ctx->d_sx, sizeof(double) * s->n_core, cudaMemcpyDeviceToDevice, st));
  ctx->wim_valid = false;
  CU(cudaStreamSynchronize(st));
  return GWC_OK;
}

// ---- chi0 dispatch ------------------------------------------------------------------------------
gwc_status run_chi0_any(gwc_ctx* ctx, bool complex_z, int F, const double* d_z, const int* active, void* out,
                        double alpha, double beta, int full, long long stride, cudaStream_t st) {
  const int prec = ctx->opt.prec;
  const bool fp64 = prec == GWC_PREC_FP64;
  LAUNCH(launch_dtable(d_z, F, ctx->d_delta, ctx->n_ov, ctx->ld_dtab, !fp64, ctx->d_dtab, st));
  MatKind kind = complex_z ? cplx_kind(ctx) : real_kind(ctx);
  cudaEvent_t ev = ev_begin(ctx, st);
  if (prec == GWC_PREC_FP64) {
    LAUNCH(launch_chi0_simt(kind, ctx->d_o_ov, ctx->n_ov, ctx->n_aux, ctx->n_ov, ctx->d_dtab, ctx->ld_dtab, F, alpha, beta,
                            out, ctx->ldm, stride, full, active, st));
  } else if (prec == GWC_PREC_FP32) {
    LAUNCH(launch_chi0_simt(kind, ctx->d_o_f32, ctx->n_ov_pad, ctx->n_aux, ctx->n_ov_pad, ctx->d_dtab, ctx->ld_dtab, F,
                            alpha, beta, out, ctx->ldm, stride, full, active, st));
  } else {
    int n = (ctx->chi0_pair ? launch_chi0_pair : launch_chi0_tc)(
        prec != GWC_PREC_BF16, ctx->d_o_hi, ctx->d_o_lo, ctx->d_o_f32, ctx->n_ov_pad, ctx->n_aux, ctx->n_aux_pad,
        ctx->n_ov_pad, (const float*)ctx->d_dtab, ctx->ld_dtab, F, complex_z, alpha, beta, out, ctx->ldm, stride, active,
        ctx->d_status, ctx->wait_ns, factor64(prec), st, ctx->opt.chi0_ctas);
    if (n == -2) return fail(ctx, GWC_ERR_UNSUPPORTED, "tensor-core chi0 not available for this shape/device");
    LAUNCH(n);
    if (full) {
      // the tensor-core kernel writes the lower triangle; mirror for a full matrix
      return fail(ctx, GWC_ERR_UNSUPPORTED, "full-matrix output not supported by the tensor-core path");
    }
  }
  ev_end(ctx, kClsChi0, ev, st);
  if (!active) {  // masked launches (QP rounds) are counted on the device: only the builds they do
    ctx->stats.chi0_builds += F;
    ctx->stats.chi0_flop += (double)F * (complex_z ? 2.0 : 1.0) * (double)ctx->n_aux * (ctx->n_aux + 1.0) * (double)ctx->n_ov;
  }
  return GWC_OK;
}

// Complex factorisations: the tensor-core kernel in the mixed-precision modes, else the SIMT one.
int launch_factor(gwc_ctx* ctx, MatKind kind, void* mats, int n, int nrow, long long stride, int F, const int* act,
                  cudaStream_t st) {
  const bool mixed = ctx->opt.prec == GWC_PREC_BF16 || ctx->opt.prec == GWC_PREC_BF16X3;
  if (kind == MatKind::CplxF32 && mixed && ctx->factor_tc) {
    if (ctx->factor_split && ldlt_split_bytes(n, nrow, F) <= ctx->lp_bytes) {
      const int r = launch_ldlt_split(mats, n, nrow, ctx->ldm, stride, F, act, ctx->d_status, ctx->wait_ns, ctx->d_lp,
                                      ctx->lp_bytes, st);
      if (r != -2) return r;
    }
    const int r = launch_ldlt_tc(mats, n, nrow, ctx->ldm, stride, F, act, ctx->d_status, ctx->wait_ns, st);
    if (r != -2) return r;
  }
  return launch_ldlt(kind, mats, n, nrow, ctx->ldm, stride, F, act, ctx->d_status, st);
}

double factor_flop(int n, bool cplx, int F) {
  return (double)F * (cplx ? 8.0 : 2.0) * (double)n * n * n / 3.0;
}

gwc_status run_chi0(gwc_ctx* ctx, bool complex_z, int F, const double* d_z, const int* active, void* out, double alpha,
                    double beta, int full, cudaStream_t st) {
  return run_chi0_any(ctx, complex_z, F, d_z, active, out, alpha, beta, full, (long long)ctx->n_aux * ctx->ldm, st);
}

// eps = 1 - Pi into matrices of `stride` elements (room for appended rows)
gwc_status run_chi0_stride(gwc_ctx* ctx, bool complex_z, int F, const double* d_z, const int* active, void* out,
                           long long stride, cudaStream_t st) {
  return run_chi0_any(ctx, complex_z, F, d_z, active, out, -1.0, 1.0, 0, stride, st);
}

// ---- imaginary-axis W table --------------------------------------------------------------------
// Enqueues W^c_mn(i xi_k) for all states m and cores n, k = 0..n_im (node n_im is xi = 0), without
// host synchronisation or allocation (the frequencies were uploaded at creation).
// Imaginary-axis nodes per table batch (all n_im + 1 in one batch when the workspace holds them).
int wim_batch(const gwc_ctx* ctx) {
  // the tensor-core table factors the real eps(i xi) in complex storage (zero imaginary parts), built real
  // behind the complex matrices and widened: 8 + 4 bytes per element
  const size_t per_real = (size_t)ctx->n_aux * ctx->ldm * (ctx->wtable_tc ? 12 : mat_elem_bytes(real_kind(ctx)));
  const int fb = (int)std::max<size_t>(1, std::min<size_t>(ctx->mats_bytes / per_real, (size_t)ctx->batch));
  return std::min(fb, ctx->opt.n_im + 1);
}

gwc_status enqueue_wim_tail(gwc_ctx* ctx, int k0, int nb, cudaStream_t st);

gwc_status enqueue_wim(gwc_ctx* ctx, cudaStream_t st) {
  const int nodes = ctx->opt.n_im + 1;
  const int fb = wim_batch(ctx);
  for (int k0 = 0; k0 < nodes; k0 += fb) {
    const int nb = std::min(fb, nodes - k0);
    if (ctx->wtable_tc) {
      // real builds behind the nb complex matrices, widened into them (Im = 0) for the tensor-core LDL^T
      const long long per = (long long)ctx->n_aux * ctx->ldm;
      float* real = reinterpret_cast<float*>(static_cast<char*>(ctx->d_mats) + (size_t)nb * per * 8);
      TRY(run_chi0(ctx, false, nb, ctx->d_zim + 2 * k0, nullptr, real, -1.0, 1.0, 0, st));
      LAUNCH(launch_widen_real(real, per, ctx->d_mats, per, per, nb, st));
    } else {
      TRY(run_chi0(ctx, false, nb, ctx->d_zim + 2 * k0, nullptr, ctx->d_mats, -1.0, 1.0, 0, st));
    }
    TRY(enqueue_wim_tail(ctx, k0, nb, st));
  }
  return GWC_OK;
}

// Nodes k0 .. k0+nb-1 of the W table once their eps = 1 - Pi(i xi) are in the workspace: factorisations,
// right-hand sides, solves and the copy into the table.
gwc_status enqueue_wim_tail(gwc_ctx* ctx, int k0, int nb, cudaStream_t st) {
  MatKind rk = real_kind(ctx);
  const int r = ctx->n_states * ctx->n_core;
  const size_t plane = (size_t)ctx->n_states * ctx->n_core;
  const long long stride = (long long)ctx->n_aux * ctx->ldm;
  const bool tc = ctx->wtable_tc && rk == MatKind::RealF32;
  {
    cudaEvent_t ev = ev_begin(ctx, st);
    if (tc)  // complex storage with zero imaginary parts: the tensor-core LDL^T (they stay exactly zero)
      LAUNCH(launch_factor(ctx, cplx_kind(ctx), ctx->d_mats, ctx->n_aux, ctx->n_aux, stride, nb, nullptr, st));
    else
      LAUNCH(launch_ldlt(rk, ctx->d_mats, ctx->n_aux, ctx->n_aux, ctx->ldm, stride, nb, nullptr, ctx->d_status, st));
    ev_end(ctx, kClsFactor, ev, st);
    ctx->stats.factor_flop += factor_flop(ctx->n_aux, tc, nb);
    ctx->stats.factorizations += nb;
    // W^c for ng nodes per solve launch (one RHS buffer per node)
    const size_t ebytes = mat_elem_bytes(rk);
    for (int u0 = 0; u0 < nb; u0 += ctx->wim_group) {
      const int ng = std::min(ctx->wim_group, nb - u0);
      for (int u = 0; u < ng; ++u)
        LAUNCH(launch_rhs_gather(rk, ctx->d_o_core, ctx->n_aux, ctx->d_rowmap, 1, r, ctx->n_aux,
                                 (char*)ctx->d_rhs_im + (size_t)u * plane * ctx->ldm * ebytes, ctx->ldm, 0,
                                 ctx->d_bnorm + (size_t)u * plane, st));
      cudaEvent_t evs = ev_begin(ctx, st);
      if (tc) {
        // blocked forward substitution on the tensor cores (real parts of the complex factors), straight into
        // the table planes
        const float* mat = (const float*)ctx->d_mats + (size_t)u0 * stride * 2;
        const int n = launch_wtable_tc(mat, 2, ctx->n_aux, ctx->ldm, 2 * stride, (float*)ctx->d_rhs_im, ctx->ldm,
                                       (long long)plane * ctx->ldm, r, ng, ctx->d_bnorm, ctx->d_wim + (size_t)(k0 + u0) * plane,
                                       (long long)plane, ctx->d_wt, ctx->wt_bytes, ctx->d_status, ctx->wait_ns, st);
        if (n == -2) return fail(ctx, GWC_ERR_UNSUPPORTED, "tensor-core W-table solve not available for this shape");
        LAUNCH(n);
        ev_end(ctx, kClsSolve, evs, st);
      } else {
        char* mat = (char*)ctx->d_mats + (size_t)u0 * stride * ebytes;
        LAUNCH(launch_ldlt_solve_w(rk, mat, ctx->n_aux, ctx->ldm, stride, ctx->d_rhs_im, r, ctx->ldm,
                                   (long long)plane * ctx->ldm, ctx->d_bnorm, ng, ctx->d_wtmp, (long long)plane * 2,
                                   nullptr, st));
        ev_end(ctx, kClsSolve, evs, st);
        // real parts of w -> W table planes k0+u0 .. k0+u0+ng-1
        CU(cudaMemcpy2DAsync(ctx->d_wim + (size_t)(k0 + u0) * plane, sizeof(double), ctx->d_wtmp, 2 * sizeof(double),
                             sizeof(double), (size_t)ng * plane, cudaMemcpyDeviceToDevice, st));
      }
    }
  }
  return GWC_OK;
}

gwc_status compute_wim(gwc_ctx* ctx, cudaStream_t st) {
  if (ctx->wim_valid) return GWC_OK;
  TRY(enqueue_wim(ctx, st));
  ctx->wim_valid = true;
  return GWC_OK;
}

// ---- residue W for a list of (frequency, state m) pairs ---------------------------------------------
// z_dev [n_pairs][2], rows_dev [n_pairs * r] (rows of o_core flattened [m][c]), output w [n_pairs][r][2].
// rhs/bnorm: right-hand-side staging for `chunk` frequencies of r vectors each.
gwc_status residue_batches_buf(gwc_ctx* ctx, int n_pairs, const double* z_dev, const int* rows_dev, int r, double* w_out,
                               const int* active, void* rhs, double* bnorm, int chunk, cudaStream_t st) {
  MatKind ck = cplx_kind(ctx);
  const bool border = r <= ctx->border_max;  // right-hand sides appended as rows of the factored matrix
  const long long stride = (long long)(ctx->n_aux + (border ? r : 0)) * ctx->ldm;
  const long long rstride = (long long)r * ctx->ldm;
  chunk = std::max(1, std::min(chunk, ctx->batch));
  if (chunk >= ctx->n_sm) chunk -= chunk % ctx->n_sm;  // whole SM-waves; only the last batch is ragged
  for (int p0 = 0; p0 < n_pairs; p0 += chunk) {
    const int nb = std::min(chunk, n_pairs - p0);
    const int* act = active ? active + p0 : nullptr;
    const int* rows = rows_dev + (size_t)p0 * r;
    double* wout = w_out + (size_t)p0 * r * 2;
    if (border) {
      // chi0 writes eps into rows 0..n-1 of each [n+r][ldm] matrix
      TRY(run_chi0_stride(ctx, true, nb, z_dev + 2 * (size_t)p0, act, ctx->d_mats, stride, st));
      LAUNCH(launch_border_rows(ck, ctx->d_mats, ctx->n_aux, ctx->ldm, stride, ctx->d_o_core, ctx->n_aux, rows, nb, r,
                                ctx->d_bnorm, st));
      cudaEvent_t ev = ev_begin(ctx, st);
      LAUNCH(launch_factor(ctx, ck, ctx->d_mats, ctx->n_aux, ctx->n_aux + r, stride, nb, act, st));
      ev_end(ctx, kClsFactor, ev, st);
      LAUNCH(launch_border_w(ck, ctx->d_mats, ctx->n_aux, ctx->ldm, stride, nb, r, ctx->d_bnorm, wout, (long long)r * 2,
                             act, st));
    } else {
      TRY(run_chi0(ctx, true, nb, z_dev + 2 * (size_t)p0, act, ctx->d_mats, -1.0, 1.0, 0, st));
      cudaEvent_t ev = ev_begin(ctx, st);
      LAUNCH(launch_factor(ctx, ck, ctx->d_mats, ctx->n_aux, ctx->n_aux, stride, nb, act, st));
      ev_end(ctx, kClsFactor, ev, st);
      LAUNCH(launch_rhs_gather(ck, ctx->d_o_core, ctx->n_aux, rows, nb, r, ctx->n_aux, rhs, ctx->ldm, rstride, bnorm, st));
      cudaEvent_t evs = ev_begin(ctx, st);
      LAUNCH(launch_ldlt_solve_w(ck, ctx->d_mats, ctx->n_aux, ctx->ldm, stride, rhs, r, ctx->ldm, rstride, bnorm, nb, wout,
                                 (long long)r * 2, act, st));
      ev_end(ctx, kClsSolve, evs, st);
    }
    if (!act) {
      ctx->stats.factorizations += nb;
      ctx->stats.factor_flop += factor_flop(ctx->n_aux, true, nb);
    }
  }
  return GWC_OK;
}

// Folds the builds that masked launches really did (counted by the QP pair kernel) into the stats.
void fold_active_builds(gwc_ctx* ctx) {
  if (!ctx->d_active_builds) return;
  unsigned long long n = 0;
  if (cudaMemcpy(&n, ctx->d_active_builds, sizeof(n), cudaMemcpyDeviceToHost) != cudaSuccess) return;
  const unsigned long long add = n - ctx->active_folded;
  ctx->active_folded = n;
  ctx->stats.chi0_builds += (long long)add;
  ctx->stats.chi0_flop += (double)add * 2.0 * (double)ctx->n_aux * (ctx->n_aux + 1.0) * (double)ctx->n_ov;
  ctx->stats.factorizations += (long long)add;
  ctx->stats.factor_flop += (double)add * factor_flop(ctx->n_aux, true, 1);
}

gwc_status residue_batches(gwc_ctx* ctx, int n_pairs, const double* z_dev, const int* rows_dev, int r, double* w_out,
                           const int* active, cudaStream_t st) {
  return residue_batches_buf(ctx, n_pairs, z_dev, rows_dev, r, w_out, active, ctx->d_rhs, ctx->d_bnorm, ctx->batch, st);
}

// QP rounds on the device (eqs hedin_shift, quasiparticle_equation, hedin_sigma_spectral, QPGWC).
// With poll, the host reads the 4-byte "all converged" flag every 4 rounds and stops early;
// without, all rounds are enqueued and finished cores cost only empty launches (capturable).
gwc_status enqueue_qp(gwc_ctx* ctx, double* eps_qp, double* dh, int* iters, bool poll, cudaStream_t st) {
  const int nc = ctx->n_core, no = ctx->n_occ;
  const int np = nc * no;
  const bool hedin = ctx->opt.qp_mode == GWC_QP_HEDIN;
  LAUNCH(launch_qp_init(ctx->d_eps, ctx->d_core_idx, nc, ctx->qp_mask_set ? ctx->d_qp_mask : nullptr, ctx->d_qp, st));
  const int rounds = hedin ? 1 : ctx->opt.max_qp_iter + 2;
  for (int r = 0; r < rounds; ++r) {
    LAUNCH(launch_qp_pairs(ctx->d_eps, ctx->d_core_idx, nc, no, ctx->eps_f, ctx->opt.eta, ctx->d_qp, ctx->d_qp_z,
                           ctx->d_qp_active, ctx->d_qp_fac, ctx->d_all_done, ctx->d_active_builds, st));
    TRY(residue_batches(ctx, np, ctx->d_qp_z, ctx->d_qp_rowmap, 1, ctx->d_qp_w, ctx->d_qp_active, st));
    LAUNCH(launch_qp_assemble_update(ctx->d_eps, ctx->n_states, no, nc, ctx->d_core_idx, ctx->eps_f, ctx->d_xi,
                                     ctx->d_wxi, ctx->opt.n_im, ctx->d_wim, ctx->d_qp_w, ctx->d_qp_fac, ctx->d_sx,
                                     ctx->d_vxc_eff, ctx->opt.qp_tol, ctx->opt.max_qp_iter,
                                     ctx->opt.qp_mode == GWC_QP_G0W0 ? 1 : 0, ctx->d_qp, ctx->d_all_done, st));
    if (poll && (r & 3) == 3) {
      int done = 0;
      CU(cudaMemcpyAsync(&done, ctx->d_all_done, sizeof(int), cudaMemcpyDeviceToHost, st));
      CU(cudaStreamSynchronize(st));
      if (done) break;
    }
  }
  if (hedin)
    LAUNCH(launch_qp_finish_hedin(ctx->d_qp, ctx->d_eps, ctx->d_core_idx, nc, eps_qp, dh, iters, st));
  else
    LAUNCH(launch_qp_finish(ctx->d_qp, nc, eps_qp, dh, iters, ctx->d_status, st));
  return GWC_OK;
}

gwc_status check_stream_error(gwc_ctx* ctx) {
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return fail(ctx, GWC_ERR_CUDA, cudaGetErrorString(e));
  return GWC_OK;
}

}  // namespace

namespace gwc {
void set_noctx_error(const char* msg) { g_create_error = msg ? msg : ""; }
}  // namespace gwc

// =====================================================================================================
extern "C" {

int gwc_abi_version(void) { return GWC_ABI_VERSION; }

const char* gwc_status_string(gwc_status s) {
  switch (s) {
    case GWC_OK: return "ok";
    case GWC_ERR_INVALID_ARG: return "invalid argument";
    case GWC_ERR_OOM: return "out of memory";
    case GWC_ERR_CUDA: return "CUDA error";
    case GWC_ERR_SINGULAR: return "singular dielectric matrix";
    case GWC_ERR_NOT_CONVERGED: return "QP iteration not converged";
    case GWC_ERR_TIMEOUT: return "device wait timed out";
    case GWC_ERR_UNSUPPORTED: return "unsupported";
  }
  return "unknown status";
}

const char* gwc_last_error(const gwc_ctx* ctx) { return ctx ? ctx->last_error.c_str() : g_create_error.c_str(); }

gwc_status gwc_default_options(gwc_options* o) {
  if (!o) return GWC_ERR_INVALID_ARG;
  o->eta = 1e-3;
  o->n_im = 32;
  o->xi0 = 1.0;
  o->prec = GWC_PREC_BF16X3;
  o->dec = GWC_DECOUPLE_DIAG;
  o->group_of_core = nullptr;
  o->n_t = 1 << 16;
  o->t_max = 2000.0;
  o->max_qp_iter = 50;
  o->qp_tol = 1e-7;
  o->batch = 0;
  o->profile = 0;
  o->qp_mode = GWC_QP_SECANT;
  o->wait_us = 0;
  o->chi0_ctas = 0;
  o->chi0_tile = 0;
  return GWC_OK;
}

gwc_status gwc_workspace_bytes(const gwc_system* sys, const gwc_options* opt, int n_omega, size_t* bytes) {
  TRY(validate_system(sys));
  TRY(validate_options(opt, sys->n_core));
  if (!bytes || n_omega < 0) return fail(nullptr, GWC_ERR_INVALID_ARG, "bytes NULL or n_omega < 0");
  Sizes z = sizes_of(sys, opt);
  int batch = opt->batch > 0 ? opt->batch : 64;
  size_t b = resident_bytes(sys, opt, z) + (size_t)batch * per_matrix_bytes(sys, z);
  b += (size_t)n_omega * sys->n_states * (4 + 4 + 8 + 16 + 8 + 4 * sys->n_core) + (size_t)n_omega * sys->n_occ * sys->n_core * 16;
  b += (size_t)sys->n_core * opt->n_t * 32 + (size_t)opt->n_t * 8;
  *bytes = b;
  return GWC_OK;
}

gwc_status gwc_create(gwc_ctx** out, const gwc_system* s, const gwc_options* o, void* stream) {
  if (!out) return fail(nullptr, GWC_ERR_INVALID_ARG, "ctx out pointer is NULL");
  *out = nullptr;
  TRY(validate_system(s));
  TRY(validate_options(o, s->n_core));
  cudaStream_t st = (cudaStream_t)stream;
  gwc_ctx* ctx = new gwc_ctx();
  cudaGetDevice(&ctx->device);
  if (cudaDeviceGetAttribute(&ctx->n_sm, cudaDevAttrMultiProcessorCount, ctx->device) != cudaSuccess || ctx->n_sm < 1)
    ctx->n_sm = 1;
  {
    // complex factorisations of the mixed modes run on the tensor cores, as panel launches + batched updates
    // (split); GWC_FACTOR=tc keeps the one-CTA-per-matrix tensor-core kernel, =simt the SIMT kernel (A/B
    // measurements)
    const char* fe = std::getenv("GWC_FACTOR");
    ctx->factor_tc = !(fe && std::strcmp(fe, "simt") == 0);
    ctx->factor_split = ctx->factor_tc && !(fe && std::strcmp(fe, "tc") == 0);
  }
  ctx->n_states = s->n_states;
  ctx->n_occ = s->n_occ;
  ctx->n_virt = s->n_states - s->n_occ;
  ctx->n_aux = s->n_aux;
  ctx->n_core = s->n_core;
  ctx->n_ov = s->n_occ * ctx->n_virt;
  ctx->opt = *o;
  {
    // GWC_CHI0_KERNEL=single keeps the one-CTA 128 x 128 chi0 kernel whatever the options say (A/B measurements)
    const char* ck = std::getenv("GWC_CHI0_KERNEL");
    if (ck && std::strcmp(ck, "single") == 0) ctx->opt.chi0_tile = 1;
    ctx->chi0_pair = ctx->opt.chi0_tile == 0;
  }
  ctx->wait_ns = o->wait_us > 0 ? 1000ull * (unsigned long long)o->wait_us : 1000000000ull;
  if (o->group_of_core) ctx->h_group.assign(o->group_of_core, o->group_of_core + s->n_core);
  ctx->opt.group_of_core = nullptr;
  Sizes z = sizes_of(s, o);
  ctx->n_aux_pad = z.n_aux_pad;
  ctx->n_ov_pad = z.n_ov_pad;
  ctx->ld_dtab = z.ld_dtab;
  ctx->ldm = z.ldm;
  auto bail = [&](gwc_status stt) {
    std::string msg = ctx->last_error;
    gwc_destroy(ctx);
    g_create_error = msg;
    return stt;
  };
#define CTRY(x)                        \
  do {                                 \
    gwc_status s_ = (x);               \
    if (s_ != GWC_OK) return bail(s_); \
  } while (0)
  const size_t n_ov = ctx->n_ov;
  CTRY(dalloc(ctx, &ctx->d_eps, s->n_states));
  CTRY(dalloc(ctx, &ctx->d_delta, n_ov));
  CTRY(dalloc(ctx, &ctx->d_o_ov, (size_t)s->n_aux * n_ov));
  CTRY(dalloc(ctx, &ctx->d_o_core, (size_t)s->n_states * s->n_core * s->n_aux));
  CTRY(dalloc(ctx, &ctx->d_core_idx, s->n_core));
  CTRY(dalloc(ctx, &ctx->d_sx, s->n_core));
  CTRY(dalloc(ctx, &ctx->d_vxc_eff, s->n_core));
  CTRY(dalloc(ctx, &ctx->d_status, 4));
  CTRY(dalloc(ctx, &ctx->d_all_done, 1));
  CTRY(dalloc(ctx, &ctx->d_active_builds, 1));
  if (cudaMemset(ctx->d_active_builds, 0, sizeof(unsigned long long)) != cudaSuccess)
    return bail(fail(ctx, GWC_ERR_CUDA, "counter reset failed"));
  if (!ctx->h_group.empty()) {
    CTRY(dalloc(ctx, &ctx->d_group, s->n_core));
    if (cudaMemcpy(ctx->d_group, ctx->h_group.data(), sizeof(int) * s->n_core, cudaMemcpyHostToDevice) != cudaSuccess)
      return bail(fail(ctx, GWC_ERR_CUDA, "group upload failed"));
  }
  cudaMemsetAsync(ctx->d_status, 0, 4 * sizeof(unsigned), st);
  if (o->prec != GWC_PREC_FP64) {
    size_t np = (size_t)z.n_aux_pad * z.n_ov_pad;
    CTRY(dalloc(ctx, &ctx->d_o_hi, np));
    CTRY(dalloc(ctx, &ctx->d_o_lo, np));
    CTRY(dalloc(ctx, &ctx->d_o_f32, np));
  }
  // imaginary grid
  {
    std::vector<double> x, w;
    gauss_legendre(o->n_im, x, w);
    std::vector<double> xi(o->n_im), wx(o->n_im);
    for (int k = 0; k < o->n_im; ++k) {
      xi[k] = o->xi0 * (1.0 + x[k]) / (1.0 - x[k]);
      wx[k] = 2.0 * o->xi0 * w[k] / ((1.0 - x[k]) * (1.0 - x[k]));
    }
    CTRY(dalloc(ctx, &ctx->d_xi, o->n_im));
    CTRY(dalloc(ctx, &ctx->d_wxi, o->n_im));
    std::vector<double> zim(2 * (o->n_im + 1), 0.0);
    for (int k = 0; k < o->n_im; ++k) zim[2 * k + 1] = xi[k];
    CTRY(dalloc(ctx, &ctx->d_zim, zim.size()));
    if (cudaMemcpy(ctx->d_zim, zim.data(), sizeof(double) * zim.size(), cudaMemcpyHostToDevice) != cudaSuccess)
      return bail(fail(ctx, GWC_ERR_CUDA, "grid upload failed"));
    if (cudaMemcpy(ctx->d_xi, xi.data(), sizeof(double) * o->n_im, cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemcpy(ctx->d_wxi, wx.data(), sizeof(double) * o->n_im, cudaMemcpyHostToDevice) != cudaSuccess)
      return bail(fail(ctx, GWC_ERR_CUDA, "grid upload failed"));
  }
  const size_t plane = (size_t)s->n_states * s->n_core;
  CTRY(dalloc(ctx, &ctx->d_wim, (size_t)(o->n_im + 1) * plane));
  // workspace
  ctx->batch = choose_batch(s, o, z, ctx->n_sm);
  ctx->batch_cap = ctx->batch;
  ctx->border_max = std::min(s->n_core, 64);
  ctx->mats_bytes = (size_t)ctx->batch * (s->n_aux + ctx->border_max) * z.ldm * z.elem_c;
  {
    char* p = nullptr;
    CTRY(dalloc(ctx, &p, ctx->mats_bytes));
    ctx->d_mats = p;
    char* q = nullptr;
    CTRY(dalloc(ctx, &q, (size_t)ctx->batch * 2 * z.ld_dtab * 8));
    ctx->d_dtab = q;
    ctx->rhs_bytes = (size_t)ctx->batch * s->n_core * z.ldm * z.elem_c;
    char* r = nullptr;
    CTRY(dalloc(ctx, &r, ctx->rhs_bytes));
    ctx->d_rhs = r;
    // imaginary-axis solves: one right-hand-side buffer per node solved in the same launch (<= 1 GiB)
    const size_t per_node = plane * z.ldm * z.elem_r;
    ctx->wim_group = (int)std::max<size_t>(1, std::min<size_t>(((size_t)1 << 30) / per_node,
                                                               (size_t)std::min(ctx->batch, o->n_im + 1)));
    char* ri = nullptr;
    CTRY(dalloc(ctx, &ri, (size_t)ctx->wim_group * per_node));
    ctx->d_rhs_im = ri;
    // W-table solves on the tensor cores (mixed modes: real FP32 factors); GWC_WTABLE=simt keeps the SIMT
    // forward substitution (A/B measurements)
    const char* wt = std::getenv("GWC_WTABLE");
    if ((o->prec == GWC_PREC_BF16X3 || o->prec == GWC_PREC_BF16) && ctx->factor_split) {
      ctx->lp_bytes = ldlt_split_bytes(s->n_aux, s->n_aux + ctx->border_max, ctx->batch);
      char* lp = nullptr;
      CTRY(dalloc(ctx, &lp, ctx->lp_bytes));
      ctx->d_lp = lp;
    }
    if ((o->prec == GWC_PREC_BF16X3 || o->prec == GWC_PREC_BF16) && !(wt && std::strcmp(wt, "simt") == 0)) {
      ctx->wt_bytes = wtable_tc_bytes(s->n_aux, (int)plane, ctx->wim_group);
      char* w = nullptr;
      CTRY(dalloc(ctx, &w, ctx->wt_bytes));
      ctx->d_wt = w;
      ctx->wtable_tc = true;
    }
  }
  const size_t wim_rows = (size_t)ctx->wim_group * plane;
  CTRY(dalloc(ctx, &ctx->d_z, 2 * (size_t)ctx->batch));
  CTRY(dalloc(ctx, &ctx->d_active, ctx->batch));
  CTRY(dalloc(ctx, &ctx->d_bnorm, std::max(wim_rows, (size_t)ctx->batch * s->n_core)));
  CTRY(dalloc(ctx, &ctx->d_wtmp, 2 * std::max(wim_rows, (size_t)ctx->batch * s->n_core)));
  CTRY(dalloc(ctx, &ctx->d_rowmap, plane));
  {
    std::vector<int> ident(plane);
    for (size_t i = 0; i < plane; ++i) ident[i] = (int)i;
    if (cudaMemcpy(ctx->d_rowmap, ident.data(), sizeof(int) * plane, cudaMemcpyHostToDevice) != cudaSuccess)
      return bail(fail(ctx, GWC_ERR_CUDA, "rowmap upload failed"));
  }
  // QP buffers
  {
    const size_t np = (size_t)s->n_core * s->n_occ;
    CTRY(dalloc(ctx, &ctx->d_qp, s->n_core));
    CTRY(dalloc(ctx, &ctx->d_qp_z, 2 * np));
    CTRY(dalloc(ctx, &ctx->d_qp_active, np));
    CTRY(dalloc(ctx, &ctx->d_qp_fac, np));
    CTRY(dalloc(ctx, &ctx->d_qp_w, 2 * np));
    CTRY(dalloc(ctx, &ctx->d_qp_rowmap, np));
    std::vector<int> rows(np);
    for (int c = 0; c < s->n_core; ++c)
      for (int m = 0; m < s->n_occ; ++m) rows[(size_t)c * s->n_occ + m] = m * s->n_core + c;
    if (cudaMemcpy(ctx->d_qp_rowmap, rows.data(), sizeof(int) * np, cudaMemcpyHostToDevice) != cudaSuccess)
      return bail(fail(ctx, GWC_ERR_CUDA, "qp rowmap upload failed"));
  }
  {
    gwc_ctx::Caps& c = ctx->cap;
    c.n_states = s->n_states;
    c.n_core = s->n_core;
    c.n_ov = n_ov;
    c.o_ov = (size_t)s->n_aux * n_ov;
    c.o_core = (size_t)s->n_states * s->n_core * s->n_aux;
    c.o_pad = o->prec != GWC_PREC_FP64 ? (size_t)z.n_aux_pad * z.n_ov_pad : 0;
    c.plane = plane;
    c.qp_np = (size_t)s->n_core * s->n_occ;
    c.mats_bytes = ctx->mats_bytes;
    c.dtab = (size_t)ctx->batch * 2 * z.ld_dtab;
    c.rhs_bytes = ctx->rhs_bytes;
    c.rhs_im_bytes = (size_t)ctx->wim_group * plane * z.ldm * z.elem_r;
    c.bnorm = std::max(wim_rows, (size_t)ctx->batch * s->n_core);
    c.batch = ctx->batch;
  }
  if (s->eps) {
    CTRY(load_system(ctx, s, st));
    ctx->loaded = true;
  }
#undef CTRY
  *out = ctx;
  return GWC_OK;
}

// Sets the context's sizes to those of `s` inside the capacity it was created with: no allocation.
gwc_status reshape(gwc_ctx* ctx, const gwc_system* s) {
  const gwc_ctx::Caps& c = ctx->cap;
  if (!ctx->h_group.empty() && s->n_core != ctx->n_core)
    return fail(ctx, GWC_ERR_INVALID_ARG, "a context with core groups keeps its number of cores");
  const Sizes z = sizes_of(s, &ctx->opt);
  const size_t n_ov = (size_t)s->n_occ * (s->n_states - s->n_occ);
  const size_t plane = (size_t)s->n_states * s->n_core;
  const bool fits = (size_t)s->n_states <= c.n_states && (size_t)s->n_core <= c.n_core && n_ov <= c.n_ov &&
                    (size_t)s->n_aux * n_ov <= c.o_ov && plane * s->n_aux <= c.o_core &&
                    (ctx->opt.prec == GWC_PREC_FP64 || (size_t)z.n_aux_pad * z.n_ov_pad <= c.o_pad) && plane <= c.plane &&
                    (size_t)s->n_core * s->n_occ <= c.qp_np;
  if (!fits) return fail(ctx, GWC_ERR_INVALID_ARG, "system larger than the capacity of this context (create a larger one)");
  const int border = std::min(s->n_core, 64);
  const size_t per_mat = (size_t)(s->n_aux + border) * z.ldm * z.elem_c;
  long long b = std::min<long long>(c.batch, (long long)(c.mats_bytes / per_mat));
  b = std::min<long long>(b, (long long)(c.dtab / (2 * (size_t)z.ld_dtab)));
  b = std::min<long long>(b, (long long)(c.rhs_bytes / ((size_t)s->n_core * z.ldm * z.elem_c)));
  b = std::min<long long>(b, (long long)(c.bnorm / s->n_core));
  if (b >= ctx->n_sm) b -= b % ctx->n_sm;
  const size_t per_node = plane * z.ldm * z.elem_r;
  const long long wg = std::min<long long>({(long long)(c.rhs_im_bytes / per_node), b, (long long)ctx->opt.n_im + 1,
                                            (long long)(c.bnorm / plane)});
  if (b < 1 || wg < 1) return fail(ctx, GWC_ERR_INVALID_ARG, "system does not fit the context's workspace");
  std::vector<int> ident(plane);
  for (size_t i = 0; i < plane; ++i) ident[i] = (int)i;
  CU(cudaMemcpy(ctx->d_rowmap, ident.data(), sizeof(int) * plane, cudaMemcpyHostToDevice));
  std::vector<int> rows((size_t)s->n_core * s->n_occ);
  for (int cc = 0; cc < s->n_core; ++cc)
    for (int m = 0; m < s->n_occ; ++m) rows[(size_t)cc * s->n_occ + m] = m * s->n_core + cc;
  CU(cudaMemcpy(ctx->d_qp_rowmap, rows.data(), sizeof(int) * rows.size(), cudaMemcpyHostToDevice));
  ctx->n_states = s->n_states;
  ctx->n_occ = s->n_occ;
  ctx->n_virt = s->n_states - s->n_occ;
  ctx->n_aux = s->n_aux;
  ctx->n_core = s->n_core;
  ctx->n_ov = (int)n_ov;
  ctx->n_aux_pad = z.n_aux_pad;
  ctx->n_ov_pad = z.n_ov_pad;
  ctx->ld_dtab = z.ld_dtab;
  ctx->ldm = z.ldm;
  ctx->batch = (int)b;
  ctx->border_max = border;
  ctx->wim_group = (int)wg;
  ctx->wtable_tc = ctx->d_wt && wtable_tc_bytes(s->n_aux, (int)plane, (int)wg) <= ctx->wt_bytes;
  ctx->req_n_omega = 0;       // a request plan belongs to the previous system
  ctx->req_n_pairs = 0;
  ctx->qp_mask_set = false;   // so does a QP core selection
  return GWC_OK;
}

gwc_status gwc_load(gwc_ctx* ctx, const gwc_system* s, void* stream) {
  if (!ctx) return fail(nullptr, GWC_ERR_INVALID_ARG, "ctx is NULL");
  if (validate_system(s) != GWC_OK) return fail(ctx, GWC_ERR_INVALID_ARG, g_create_error);
  if (!s->eps) return fail(ctx, GWC_ERR_INVALID_ARG, "gwc_load needs the system's arrays");
  if (s->n_states != ctx->n_states || s->n_occ != ctx->n_occ || s->n_aux != ctx->n_aux || s->n_core != ctx->n_core)
    TRY(reshape(ctx, s));
  ctx->loaded = false;
  TRY(load_system(ctx, s, (cudaStream_t)stream));
  ctx->loaded = true;
  return GWC_OK;
}

void gwc_destroy(gwc_ctx* ctx) {
  if (!ctx) return;
  void* ptrs[] = {ctx->d_eps, ctx->d_o_ov, ctx->d_o_core, ctx->d_vxc, ctx->d_delta, ctx->d_core_idx, ctx->d_group,
                  ctx->d_xi, ctx->d_wxi, ctx->d_wim, ctx->d_sx, ctx->d_vxc_eff, ctx->d_o_hi, ctx->d_o_lo, ctx->d_o_f32,
                  ctx->d_mats, ctx->d_dtab, ctx->d_z, ctx->d_active, ctx->d_rhs, ctx->d_bnorm, ctx->d_rowmap,
                  ctx->d_wtmp, ctx->d_rhs_im, ctx->d_status, ctx->d_pidx, ctx->d_wres, ctx->d_pair_m, ctx->d_pair_w,
                  ctx->d_grid_w, ctx->d_qp, ctx->d_qp_z, ctx->d_qp_active, ctx->d_qp_fac, ctx->d_qp_w,
                  ctx->d_qp_rowmap, ctx->d_all_done, ctx->d_cw_a, ctx->d_cw_b, ctx->d_coef, ctx->d_tw,
                  ctx->d_pair_z, ctx->d_pair_rows, ctx->d_zim, ctx->d_req_wrel, ctx->d_req_z, ctx->d_req_rows,
                  ctx->d_req_pair_of, ctx->d_req_w, ctx->d_req_im, ctx->d_req_a, ctx->d_req_nu, ctx->d_req_eqp,
                  ctx->d_req_dh, ctx->d_req_it, ctx->d_eps_g, ctx->d_ev_sig, ctx->d_ev_diff, ctx->d_active_builds,
                  ctx->d_ev_pidx, ctx->d_ev_pm, ctx->d_ev_pw, ctx->d_ev_z, ctx->d_ev_rows, ctx->d_ev_wres, ctx->d_ev_w,
                  ctx->d_qp_mask, ctx->d_wt, ctx->d_lp};
  for (void* p : ptrs)
    if (p) cudaFree(p);
  for (auto& r : ctx->ev_pending) {
    cudaEventDestroy(r.a);
    cudaEventDestroy(r.b);
  }
  for (cudaEvent_t e : ctx->ev_pool) cudaEventDestroy(e);
  if (ctx->h_pin_i) cudaFreeHost(ctx->h_pin_i);
  if (ctx->h_pin_d) cudaFreeHost(ctx->h_pin_d);
  delete ctx;
}

gwc_status gwc_build_chi0(gwc_ctx* ctx, const double* z, int F, double* chi0, void* stream) {
  if (!ctx) return fail(nullptr, GWC_ERR_INVALID_ARG, "ctx is NULL");
  if (!ctx->loaded) return fail(ctx, GWC_ERR_INVALID_ARG, "no system loaded (gwc_load)");
  if (!z || !chi0 || F < 1 || F > 4096) return fail(ctx, GWC_ERR_INVALID_ARG, "need z, chi0 and 1 <= F <= 4096");
  cudaStream_t st = (cudaStream_t)stream;
  MatKind ck = cplx_kind(ctx);
  const long long stride = (long long)ctx->n_aux * ctx->ldm;
  for (int f0 = 0; f0 < F; f0 += ctx->batch) {
    int nb = std::min(ctx->batch, F - f0);
    TRY(run_chi0(ctx, true, nb, z + 2 * (size_t)f0, nullptr, ctx->d_mats, 1.0, 0.0, 0, st));
    LAUNCH(launch_mat_to_c128(ck, ctx->d_mats, ctx->n_aux, ctx->ldm, stride, nb,
                              chi0 + (size_t)f0 * ctx->n_aux * ctx->n_aux * 2, st));
  }
  return check_stream_error(ctx);
}

gwc_status gwc_screen(gwc_ctx* ctx, const double* z, int F, const double* rhs, int n_rhs, double* w, void* stream) {
  if (!ctx) return fail(nullptr, GWC_ERR_INVALID_ARG, "ctx is NULL");
  if (!ctx->loaded) return fail(ctx, GWC_ERR_INVALID_ARG, "no system loaded (gwc_load)");
  if (!z || !rhs || !w || F < 1 || F > 4096 || n_rhs < 1 || n_rhs > (1 << 20))
    return fail(ctx, GWC_ERR_INVALID_ARG, "need z, rhs, w, 1 <= F <= 4096, 1 <= n_rhs <= 2^20");
  cudaStream_t st = (cudaStream_t)stream;
  MatKind ck = cplx_kind(ctx);
  const size_t es = mat_elem_bytes(ck);
  // per-call scratch for the right-hand sides of one frequency chunk
  int chunk = std::max(1, std::min(ctx->batch, (int)std::max<size_t>(1, ((size_t)1 << 30) / ((size_t)n_rhs * ctx->ldm * es))));
  void* d_r = nullptr;
  double* d_bn = nullptr;
  int* d_rows = nullptr;
  size_t nrow = (size_t)chunk * n_rhs;
  if (cudaMalloc(&d_r, nrow * ctx->ldm * es) != cudaSuccess || cudaMalloc((void**)&d_bn, nrow * sizeof(double)) != cudaSuccess ||
      cudaMalloc((void**)&d_rows, nrow * sizeof(int)) != cudaSuccess) {
    cudaFree(d_r);
    cudaFree(d_bn);
    cudaFree(d_rows);
    return fail(ctx, GWC_ERR_OOM, "gwc_screen scratch allocation failed");
  }
  std::vector<int> rows(nrow);
  gwc_status res = GWC_OK;
  const long long stride = (long long)ctx->n_aux * ctx->ldm;
  for (int f0 = 0; f0 < F && res == GWC_OK; f0 += chunk) {
    int nb = std::min(chunk, F - f0);
    for (size_t i = 0; i < (size_t)nb * n_rhs; ++i) rows[i] = (int)((size_t)f0 * n_rhs + i);
    if (cudaMemcpyAsync(d_rows, rows.data(), sizeof(int) * nb * n_rhs, cudaMemcpyHostToDevice, st) != cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess) {
      res = fail(ctx, GWC_ERR_CUDA, "row map upload failed");
      break;
    }
    res = run_chi0(ctx, true, nb, z + 2 * (size_t)f0, nullptr, ctx->d_mats, -1.0, 1.0, 0, st);
    if (res != GWC_OK) break;
    cudaEvent_t evf = ev_begin(ctx, st);
    int n1 = launch_factor(ctx, ck, ctx->d_mats, ctx->n_aux, ctx->n_aux, stride, nb, nullptr, st);
    ev_end(ctx, kClsFactor, evf, st);
    int n2 = launch_rhs_gather(ck, rhs, ctx->n_aux, d_rows, nb, n_rhs, ctx->n_aux, d_r, ctx->ldm,
                               (long long)n_rhs * ctx->ldm, d_bn, st);
    cudaEvent_t evs = ev_begin(ctx, st);
    int n3 = launch_ldlt_solve_w(ck, ctx->d_mats, ctx->n_aux, ctx->ldm, stride, d_r, n_rhs, ctx->ldm,
                                 (long long)n_rhs * ctx->ldm, d_bn, nb, w + (size_t)f0 * n_rhs * 2, (long long)n_rhs * 2,
                                 nullptr, st);
    ev_end(ctx, kClsSolve, evs, st);
    if (n1 < 0 || n2 < 0 || n3 < 0) res = fail(ctx, GWC_ERR_CUDA, "screen launch failed");
    ctx->stats.kernel_launches += std::max(n1, 0) + std::max(n2, 0) + std::max(n3, 0);
    ctx->stats.factorizations += nb;
    ctx->stats.factor_flop += factor_flop(ctx->n_aux, true, nb);
  }
  cudaStreamSynchronize(st);
  cudaFree(d_r);
  cudaFree(d_bn);
  cudaFree(d_rows);
  if (res != GWC_OK) return res;
  return check_stream_error(ctx);
}

gwc_status gwc_sigma_core(gwc_ctx* ctx, const double* omega, int n_omega, double* sigma_c, double* im_sigma_dec,
                          double* sigma_x, void* stream) {
  if (!ctx) return fail(nullptr, GWC_ERR_INVALID_ARG, "ctx is NULL");
  if (!ctx->loaded) return fail(ctx, GWC_ERR_INVALID_ARG, "no system loaded (gwc_load)");
  if (!omega || !sigma_c || n_omega < 1 || n_omega > (1 << 20))
    return fail(ctx, GWC_ERR_INVALID_ARG, "need omega, sigma_c and 1 <= n_omega <= 2^20");
  for (int j = 0; j < n_omega; ++j)
    if (!std::isfinite(omega[j])) return fail(ctx, GWC_ERR_INVALID_ARG, "omega must be finite");
  cudaStream_t st = (cudaStream_t)stream;
  TRY(compute_wim(ctx, st));
  const int ns = ctx->n_states, nc = ctx->n_core;
  // plan: one residue pair per (w_j, m) with f_m(w_j) != 0 (Eq. cd_prefactors)
  auto th = [](double x) { return x > 0.0 ? 1.0 : (x < 0.0 ? 0.0 : 0.5); };
  const std::vector<double>& eg = g_eps_host(ctx);  // poles of G
  const double ef = g_eps_f(ctx);
  std::vector<int> pidx((size_t)n_omega * ns, -1);
  std::vector<int> pm;
  std::vector<double> pw;
  for (int j = 0; j < n_omega; ++j)
    for (int m = 0; m < ns; ++m) {
      double em = eg[m], w = omega[j];
      double f = -th(ef - em) * th(em - w) + th(em - ef) * th(w - em);
      if (f != 0.0) {
        pidx[(size_t)j * ns + m] = (int)pm.size();
        pm.push_back(m);
        pw.push_back(w);
      }
    }
  const int n_pairs = (int)pm.size();
  if ((size_t)n_omega * ns > (size_t)ctx->pidx_cap) {
    TRY(dalloc(ctx, &ctx->d_pidx, (size_t)n_omega * ns));
    ctx->pidx_cap = n_omega * ns;
  }
  if ((size_t)std::max(1, n_pairs) > (size_t)ctx->wres_cap) {
    size_t cap = std::max(1, n_pairs);
    TRY(dalloc(ctx, &ctx->d_wres, cap * nc * 2));
    TRY(dalloc(ctx, &ctx->d_pair_m, cap));
    TRY(dalloc(ctx, &ctx->d_pair_w, cap));
    TRY(dalloc(ctx, &ctx->d_pair_z, cap * 2));
    TRY(dalloc(ctx, &ctx->d_pair_rows, cap * nc));
    ctx->wres_cap = (int)cap;
  }
  if (n_omega > ctx->grid_cap) {
    TRY(dalloc(ctx, &ctx->d_grid_w, n_omega));
    ctx->grid_cap = n_omega;
  }
  std::vector<int> rows((size_t)n_pairs * nc);
  for (int p = 0; p < n_pairs; ++p)
    for (int c = 0; c < nc; ++c) rows[(size_t)p * nc + c] = pm[p] * nc + c;
  CU(cudaMemcpyAsync(ctx->d_pidx, pidx.data(), sizeof(int) * pidx.size(), cudaMemcpyHostToDevice, st));
  CU(cudaMemcpyAsync(ctx->d_grid_w, omega, sizeof(double) * n_omega, cudaMemcpyHostToDevice, st));
  if (n_pairs > 0) {
    CU(cudaMemcpyAsync(ctx->d_pair_m, pm.data(), sizeof(int) * n_pairs, cudaMemcpyHostToDevice, st));
    CU(cudaMemcpyAsync(ctx->d_pair_w, pw.data(), sizeof(double) * n_pairs, cudaMemcpyHostToDevice, st));
    CU(cudaMemcpyAsync(ctx->d_pair_rows, rows.data(), sizeof(int) * rows.size(), cudaMemcpyHostToDevice, st));
    LAUNCH(launch_fill_z_pairs(g_eps_dev(ctx), ctx->d_pair_m, ctx->d_pair_w, n_pairs, ctx->opt.eta, ctx->d_pair_z, st));
    TRY(residue_batches(ctx, n_pairs, ctx->d_pair_z, ctx->d_pair_rows, nc, ctx->d_wres, nullptr, st));
  }
  LAUNCH(launch_sigma_grid(g_eps_dev(ctx), ns, nc, ctx->d_core_idx, ctx->d_grid_w, n_omega, ef, ctx->d_xi, ctx->d_wxi,
                           ctx->opt.n_im, ctx->d_wim, ctx->d_pidx, ctx->d_wres, ctx->opt.dec, ctx->d_group, sigma_c,
                           im_sigma_dec, st));
  if (sigma_x) CU(cudaMemcpyAsync(sigma_x, ctx->d_sx, sizeof(double) * nc, cudaMemcpyDeviceToDevice, st));
  // the host vectors above are read by the async copies: wait before they go out of scope
  CU(cudaStreamSynchronize(st));
  return check_stream_error(ctx);
}

gwc_status gwc_set_g_energies(gwc_ctx* ctx, const double* eps_g, double eps_f, void* stream) {
  if (!ctx) return fail(nullptr, GWC_ERR_INVALID_ARG, "ctx is NULL");
  if (!eps_g) {
    ctx->g_set = false;
    return GWC_OK;
  }
  const int n = ctx->n_states;
  for (int m = 0; m < n; ++m)
    if (!std::isfinite(eps_g[m])) return fail(ctx, GWC_ERR_INVALID_ARG, "eps_g must be finite");
  const double ef = std::isnan(eps_f) ? 0.5 * (eps_g[ctx->n_occ - 1] + eps_g[ctx->n_occ]) : eps_f;
  for (int m = 0; m < n; ++m)
    if ((m < ctx->n_occ) != (eps_g[m] < ef))
      return fail(ctx, GWC_ERR_INVALID_ARG, "eps_g must keep the occupied states below eps_f and the virtual ones above");
  cudaStream_t st = (cudaStream_t)stream;
  if (!ctx->d_eps_g) TRY(dalloc(ctx, &ctx->d_eps_g, ctx->cap.n_states));
  ctx->h_eps_g.assign(eps_g, eps_g + n);
  CU(cudaMemcpyAsync(ctx->d_eps_g, ctx->h_eps_g.data(), sizeof(double) * n, cudaMemcpyHostToDevice, st));
  CU(cudaStreamSynchronize(st));  // the host vector may change on the next call
  ctx->eps_f_g = ef;
  ctx->g_set = true;
  return GWC_OK;
}

// Sigma^c_j(e_j) of every state j at its own current energy e_j, the only values evGW0 uses: one residue
// pair per (j, m) with f_m(e_j) != 0, each with the single right-hand side o_mj (not all n cores), then
// the diagonal assembly. Uses the G energies set by gwc_set_g_energies; synchronises `st`.
static gwc_status evgw0_sigma_diag(gwc_ctx* ctx, const std::vector<double>& e, cudaStream_t st) {
  const int n = ctx->n_states;
  auto th = [](double x) { return x > 0.0 ? 1.0 : (x < 0.0 ? 0.0 : 0.5); };
  const std::vector<double>& eg = g_eps_host(ctx);
  const double ef = g_eps_f(ctx);
  std::vector<int> pidx((size_t)n * n, -1), rows, pm;
  std::vector<double> pw;
  for (int j = 0; j < n; ++j)
    for (int m = 0; m < n; ++m) {
      const double f = -th(ef - eg[m]) * th(eg[m] - e[j]) + th(eg[m] - ef) * th(e[j] - eg[m]);
      if (f == 0.0) continue;
      if (pm.size() >= (size_t)std::numeric_limits<int>::max())
        return fail(ctx, GWC_ERR_INVALID_ARG, "evGW0: too many residue pairs");
      pidx[(size_t)j * n + m] = (int)pm.size();
      pm.push_back(m);
      pw.push_back(e[j]);
      rows.push_back(m * n + j);  // o_core row (m, core j) = O^.(m, j)
    }
  const size_t np = pm.size();
  if (np > ctx->ev_pair_cap) {
    TRY(dalloc(ctx, &ctx->d_ev_pm, np));
    TRY(dalloc(ctx, &ctx->d_ev_pw, np));
    TRY(dalloc(ctx, &ctx->d_ev_z, 2 * np));
    TRY(dalloc(ctx, &ctx->d_ev_rows, np));
    TRY(dalloc(ctx, &ctx->d_ev_wres, 2 * np));
    ctx->ev_pair_cap = np;
  }
  if (!ctx->d_ev_pidx) TRY(dalloc(ctx, &ctx->d_ev_pidx, ctx->cap.n_states * ctx->cap.n_states));
  if (!ctx->d_ev_w) TRY(dalloc(ctx, &ctx->d_ev_w, ctx->cap.n_states));
  CU(cudaMemcpyAsync(ctx->d_ev_pidx, pidx.data(), sizeof(int) * pidx.size(), cudaMemcpyHostToDevice, st));
  CU(cudaMemcpyAsync(ctx->d_ev_w, e.data(), sizeof(double) * n, cudaMemcpyHostToDevice, st));
  if (np > 0) {
    CU(cudaMemcpyAsync(ctx->d_ev_pm, pm.data(), sizeof(int) * np, cudaMemcpyHostToDevice, st));
    CU(cudaMemcpyAsync(ctx->d_ev_pw, pw.data(), sizeof(double) * np, cudaMemcpyHostToDevice, st));
    CU(cudaMemcpyAsync(ctx->d_ev_rows, rows.data(), sizeof(int) * np, cudaMemcpyHostToDevice, st));
    LAUNCH(launch_fill_z_pairs(g_eps_dev(ctx), ctx->d_ev_pm, ctx->d_ev_pw, (int)np, ctx->opt.eta, ctx->d_ev_z, st));
    TRY(residue_batches(ctx, (int)np, ctx->d_ev_z, ctx->d_ev_rows, 1, ctx->d_ev_wres, nullptr, st));
  }
  LAUNCH(launch_sigma_diag(g_eps_dev(ctx), n, n, ctx->d_ev_w, ef, ctx->d_xi, ctx->d_wxi, ctx->opt.n_im, ctx->d_wim,
                           ctx->d_ev_pidx, ctx->d_ev_wres, ctx->d_ev_sig, st));
  CU(cudaStreamSynchronize(st));  // the host vectors above are read by the async copies
  return GWC_OK;
}

gwc_status gwc_evgw0(gwc_ctx* ctx, double tol, int max_iter, double* eps_qp, int* iters, void* stream) {
  if (!ctx) return fail(nullptr, GWC_ERR_INVALID_ARG, "ctx is NULL");
  if (!ctx->loaded) return fail(ctx, GWC_ERR_INVALID_ARG, "no system loaded (gwc_load)");
  if (!eps_qp || !iters || !(tol > 0.0) || max_iter < 1 || max_iter > 1000)
    return fail(ctx, GWC_ERR_INVALID_ARG, "need eps_qp, iters, tol > 0 and 1 <= max_iter <= 1000");
  const int n = ctx->n_states;
  if (ctx->n_core != n) return fail(ctx, GWC_ERR_INVALID_ARG, "evGW0 needs every state as a core (n_core = n_states)");
  for (int c = 0; c < n; ++c)
    if (ctx->h_core[c] != c) return fail(ctx, GWC_ERR_INVALID_ARG, "evGW0 needs core_idx = 0..n_states-1");
  cudaStream_t st = (cudaStream_t)stream;
  if (!ctx->d_ev_sig) TRY(dalloc(ctx, &ctx->d_ev_sig, ctx->cap.n_states * 2));
  if (!ctx->d_ev_diff) TRY(dalloc(ctx, &ctx->d_ev_diff, 1));
  struct GReset {  // later calls see the input energies in G again, on every return path
    gwc_ctx* c;
    ~GReset() { c->g_set = false; }
  } g_reset{ctx};
  TRY(compute_wim(ctx, st));
  std::vector<double> e(ctx->h_eps);
  CU(cudaMemcpyAsync(eps_qp, ctx->d_eps, sizeof(double) * n, cudaMemcpyDeviceToDevice, st));
  gwc_status res = GWC_ERR_NOT_CONVERGED;
  std::string why = "evGW0 did not converge within max_iter";
  int it = 0;
  while (it < max_iter) {
    ++it;
    if (gwc_set_g_energies(ctx, e.data(), NAN, stream) != GWC_OK) {
      // an iterate moved a QP energy across the Fermi level: the occupations of G are no longer
      // those of the input, and the scheme stops there
      why = "evGW0: QP energies crossed eps_F at iteration " + std::to_string(it);
      --it;
      break;
    }
    TRY(evgw0_sigma_diag(ctx, e, st));
    unsigned long long bits = 0;
    CU(cudaMemsetAsync(ctx->d_ev_diff, 0, sizeof(unsigned long long), st));
    LAUNCH(launch_evgw0_update(ctx->d_eps, ctx->d_sx, ctx->d_vxc_eff, ctx->d_ev_sig, n, eps_qp, ctx->d_ev_diff, st));
    CU(cudaMemcpyAsync(e.data(), eps_qp, sizeof(double) * n, cudaMemcpyDeviceToHost, st));
    CU(cudaMemcpyAsync(&bits, ctx->d_ev_diff, sizeof(bits), cudaMemcpyDeviceToHost, st));
    CU(cudaStreamSynchronize(st));
    double diff;
    std::memcpy(&diff, &bits, sizeof(diff));
    if (diff < tol) {
      res = GWC_OK;
      break;
    }
  }
  *iters = it;
  if (res == GWC_ERR_NOT_CONVERGED) return fail(ctx, res, why);
  return check_stream_error(ctx);
}

gwc_status gwc_qp_solve(gwc_ctx* ctx, double* eps_qp, double* dh, int* iters, void* stream) {
  if (!ctx) return fail(nullptr, GWC_ERR_INVALID_ARG, "ctx is NULL");
  if (!ctx->loaded) return fail(ctx, GWC_ERR_INVALID_ARG, "no system loaded (gwc_load)");
  if (!eps_qp || !dh || !iters) return fail(ctx, GWC_ERR_INVALID_ARG, "need eps_qp, dh, iters");
  TRY(need_occupied_cores(ctx, "gwc_qp_solve"));
  cudaStream_t st = (cudaStream_t)stream;
  TRY(compute_wim(ctx, st));
  TRY(enqueue_qp(ctx, eps_qp, dh, iters, true, st));
  return check_stream_error(ctx);
}

gwc_status gwc_set_qp_cores(gwc_ctx* ctx, const int* cores, int n, void* stream) {
  if (!ctx) return fail(nullptr, GWC_ERR_INVALID_ARG, "ctx is NULL");
  if (n < 0 || (n > 0 && !cores)) return fail(ctx, GWC_ERR_INVALID_ARG, "need cores for n > 0");
  if (!cores) {
    ctx->qp_mask_set = false;
    return GWC_OK;
  }
  std::vector<int> mask(ctx->n_core, 0);
  for (int k = 0; k < n; ++k) {
    if (cores[k] < 0 || cores[k] >= ctx->n_core) return fail(ctx, GWC_ERR_INVALID_ARG, "core index out of range");
    mask[cores[k]] = 1;
  }
  cudaStream_t st = (cudaStream_t)stream;
  if (!ctx->d_qp_mask) TRY(dalloc(ctx, &ctx->d_qp_mask, ctx->cap.n_core));
  CU(cudaMemcpyAsync(ctx->d_qp_mask, mask.data(), sizeof(int) * ctx->n_core, cudaMemcpyHostToDevice, st));
  CU(cudaStreamSynchronize(st));  // the host vector goes out of scope
  ctx->qp_mask_set = true;
  return GWC_OK;
}

gwc_status gwc_copy_out(gwc_ctx* ctx, void* dst, const void* src, size_t bytes, void* stream) {
  if (!ctx) return fail(nullptr, GWC_ERR_INVALID_ARG, "ctx is NULL");
  if (!dst || !src) return fail(ctx, GWC_ERR_INVALID_ARG, "need dst and src");
  CU(cudaMemcpyAsync(dst, src, bytes, cudaMemcpyDefault, (cudaStream_t)stream));
  return GWC_OK;
}

gwc_status gwc_cumulant_spectrum(gwc_ctx* ctx, const double* omega_rel, int n_omega, const double* im_sigma,
                                 double* a_out, double* nu_out, void* stream) {
  if (!ctx) return fail(nullptr, GWC_ERR_INVALID_ARG, "ctx is NULL");
  if (!ctx->loaded) return fail(ctx, GWC_ERR_INVALID_ARG, "no system loaded (gwc_load)");
  if (!omega_rel || !im_sigma || !a_out || n_omega < 1 || n_omega > 8192)
    return fail(ctx, GWC_ERR_INVALID_ARG, "need omega_rel, im_sigma, a_out and 1 <= n_omega <= 8192");
  cudaStream_t st = (cudaStream_t)stream;
  const size_t nt = ctx->opt.n_t, nc = ctx->n_core;
  if (nc * nt * 2 > ctx->cw_cap) {
    TRY(dalloc(ctx, &ctx->d_cw_a, nc * nt * 2));
    TRY(dalloc(ctx, &ctx->d_cw_b, nc * nt * 2));
    TRY(dalloc(ctx, &ctx->d_tw, nt));
    ctx->cw_cap = nc * nt * 2;
  }
  if (nc * (size_t)n_omega > ctx->coef_cap) {
    TRY(dalloc(ctx, &ctx->d_coef, nc * (size_t)n_omega));
    ctx->coef_cap = nc * (size_t)n_omega;
  }
  LAUNCH(launch_cumulant_spectrum(omega_rel, n_omega, im_sigma, (int)nc, (int)nt, ctx->opt.t_max, ctx->opt.eta,
                                  ctx->d_cw_a, ctx->d_cw_b, ctx->d_coef, ctx->d_tw, a_out, nu_out, st));
  return check_stream_error(ctx);
}

gwc_status gwc_sigma_core_wac(gwc_ctx* ctx, const double* omega, int n_omega, int n_core_ref, int n_val_ref,
                              double* sigma_c, double* im_sigma_dec, void* stream) {
  if (!ctx) return fail(nullptr, GWC_ERR_INVALID_ARG, "ctx is NULL");
  if (!ctx->loaded) return fail(ctx, GWC_ERR_INVALID_ARG, "no system loaded (gwc_load)");
  TRY(need_occupied_cores(ctx, "gwc_sigma_core_wac"));
  if (!omega || !sigma_c || n_omega < 1 || n_omega > (1 << 20) || n_core_ref < 0 || n_val_ref < 0 ||
      n_core_ref + n_val_ref > 4096)
    return fail(ctx, GWC_ERR_INVALID_ARG, "need omega, sigma_c, 1 <= n_omega <= 2^20, reference counts in 0..4096");
  if (n_core_ref == 0 && n_val_ref == 0) n_core_ref = n_val_ref = 100;
  cudaStream_t st = (cudaStream_t)stream;
  TRY(compute_wim(ctx, st));
  auto th = [](double x) { return x > 0.0 ? 1.0 : (x < 0.0 ? 0.0 : 0.5); };
  // real reference points (reading of the paper's N_C, N_V, w_C^max = 40 eV, Delta_lower/upper = 8 %/1 %)
  std::vector<double> xref;
  for (int l = 0; l < n_core_ref; ++l)
    xref.push_back(n_core_ref > 1 ? (40.0 / 27.211386245988) * l / (n_core_ref - 1) : 0.0);
  double lo = 1e300, hi = -1e300;
  for (int j = 0; j < n_omega; ++j)
    for (int m = 0; m < ctx->n_occ; ++m) {
      if (std::find(ctx->h_core.begin(), ctx->h_core.end(), m) != ctx->h_core.end()) continue;
      const double em = ctx->h_eps[m], w = omega[j];
      const double f = -th(ctx->eps_f - em) * th(em - w) + th(em - ctx->eps_f) * th(w - em);
      if (f == 0.0) continue;
      lo = std::min(lo, std::fabs(em - w));
      hi = std::max(hi, std::fabs(em - w));
    }
  if (hi >= lo && n_val_ref > 0) {
    lo *= 1.0 - 0.08;
    hi *= 1.0 + 0.01;
    for (int l = 0; l < n_val_ref; ++l) xref.push_back(n_val_ref > 1 ? lo + (hi - lo) * l / (n_val_ref - 1) : lo);
  }
  const int n_ref = (int)xref.size(), n_im = ctx->opt.n_im, n_pts = n_im + 1 + n_ref;
  const int pairs = ctx->n_occ * ctx->n_core;
  if (n_ref == 0) return fail(ctx, GWC_ERR_INVALID_ARG, "no real reference points");
  std::vector<double> zall(2 * (size_t)n_pts), zreal(2 * (size_t)n_ref);
  std::vector<double> xi(n_im);
  CU(cudaMemcpyAsync(xi.data(), ctx->d_xi, sizeof(double) * n_im, cudaMemcpyDeviceToHost, st));
  CU(cudaStreamSynchronize(st));
  for (int k = 0; k < n_im; ++k) zall[2 * k + 1] = xi[k];
  for (int l = 0; l < n_ref; ++l) {
    zall[2 * (n_im + 1 + l)] = zreal[2 * l] = xref[l];
    zall[2 * (n_im + 1 + l) + 1] = zreal[2 * l + 1] = ctx->opt.eta;
  }
  std::vector<int> rows((size_t)n_ref * pairs);
  for (int l = 0; l < n_ref; ++l)
    for (int p = 0; p < pairs; ++p) rows[(size_t)l * pairs + p] = p;  // o_core row (m, c) = m n_core + c, m < n_occ
  const size_t es = mat_elem_bytes(cplx_kind(ctx));
  int chunk = (int)std::max<size_t>(1, std::min<size_t>((size_t)ctx->batch, ((size_t)1 << 31) / ((size_t)pairs * ctx->ldm * es)));
  chunk = std::min(chunk, n_ref);
  double *d_zall = nullptr, *d_zreal = nullptr, *d_wref = nullptr, *d_coef = nullptr, *d_om = nullptr, *d_bn = nullptr;
  int* d_rows = nullptr;
  void* d_rhs = nullptr;
  auto release = [&]() {
    cudaFree(d_zall);
    cudaFree(d_zreal);
    cudaFree(d_wref);
    cudaFree(d_coef);
    cudaFree(d_om);
    cudaFree(d_bn);
    cudaFree(d_rows);
    cudaFree(d_rhs);
  };
  if (cudaMalloc(&d_zall, sizeof(double) * zall.size()) != cudaSuccess ||
      cudaMalloc(&d_zreal, sizeof(double) * zreal.size()) != cudaSuccess ||
      cudaMalloc(&d_wref, sizeof(double) * 2 * (size_t)n_ref * pairs) != cudaSuccess ||
      cudaMalloc(&d_coef, sizeof(double) * 2 * (size_t)pairs * n_pts) != cudaSuccess ||
      cudaMalloc(&d_om, sizeof(double) * n_omega) != cudaSuccess ||
      cudaMalloc(&d_bn, sizeof(double) * (size_t)chunk * pairs) != cudaSuccess ||
      cudaMalloc(&d_rows, sizeof(int) * rows.size()) != cudaSuccess ||
      cudaMalloc(&d_rhs, (size_t)chunk * pairs * ctx->ldm * es) != cudaSuccess) {
    release();
    return fail(ctx, GWC_ERR_OOM, "CD-WAC scratch allocation failed");
  }
  gwc_status res = GWC_OK;
  if (cudaMemcpyAsync(d_zall, zall.data(), sizeof(double) * zall.size(), cudaMemcpyHostToDevice, st) != cudaSuccess ||
      cudaMemcpyAsync(d_zreal, zreal.data(), sizeof(double) * zreal.size(), cudaMemcpyHostToDevice, st) != cudaSuccess ||
      cudaMemcpyAsync(d_rows, rows.data(), sizeof(int) * rows.size(), cudaMemcpyHostToDevice, st) != cudaSuccess ||
      cudaMemcpyAsync(d_om, omega, sizeof(double) * n_omega, cudaMemcpyHostToDevice, st) != cudaSuccess)
    res = fail(ctx, GWC_ERR_CUDA, "CD-WAC upload failed");
  if (res == GWC_OK) res = residue_batches_buf(ctx, n_ref, d_zreal, d_rows, pairs, d_wref, nullptr, d_rhs, d_bn, chunk, st);
  if (res == GWC_OK) {
    int n1 = launch_thiele_fit(ctx->d_wim, ctx->n_states, ctx->n_core, n_im, d_wref, n_ref, pairs, d_zall, d_coef, st);
    int n2 = launch_sigma_grid_wac(ctx->d_eps, ctx->n_states, ctx->n_occ, ctx->n_core, ctx->d_core_idx, d_om, n_omega,
                                   ctx->eps_f, ctx->opt.eta, ctx->d_xi, ctx->d_wxi, n_im, ctx->d_wim, d_coef, d_zall, n_pts,
                                   sigma_c, im_sigma_dec, ctx->d_status, st);
    if (n1 < 0 || n2 < 0) res = fail(ctx, GWC_ERR_CUDA, "CD-WAC launch failed");
    ctx->stats.kernel_launches += std::max(0, n1) + std::max(0, n2);
  }
  cudaStreamSynchronize(st);
  release();
  if (res != GWC_OK) return res;
  return check_stream_error(ctx);
}

gwc_status gwc_g0w0_solutions(gwc_ctx* ctx, const double* omega, int n_omega, const double* sigma_c, int max_roots,
                              double* roots, int* n_roots, void* stream) {
  if (!ctx) return GWC_ERR_INVALID_ARG;
  if (!omega || !sigma_c || !roots || !n_roots || n_omega < 2 || max_roots < 1)
    return fail(ctx, GWC_ERR_INVALID_ARG, "g0w0_solutions: null pointer, n_omega < 2 or max_roots < 1");
  cudaStream_t st = (cudaStream_t)stream;
  LAUNCH(launch_g0w0_scan(omega, n_omega, sigma_c, ctx->d_eps, ctx->d_core_idx, ctx->d_sx, ctx->d_vxc_eff, ctx->n_core,
                          max_roots, roots, n_roots, st));
  return GWC_OK;
}

gwc_status gwc_gdh_spectrum(gwc_ctx* ctx, const double* omega, int n_omega, const double* sigma_c, const double* dh,
                            double* a_out, double* omega_out, void* stream) {
  if (!ctx) return fail(nullptr, GWC_ERR_INVALID_ARG, "ctx is NULL");
  if (!ctx->loaded) return fail(ctx, GWC_ERR_INVALID_ARG, "no system loaded (gwc_load)");
  if (!omega || !sigma_c || !dh || !a_out || n_omega < 1)
    return fail(ctx, GWC_ERR_INVALID_ARG, "need omega, sigma_c, dh, a_out and n_omega >= 1");
  LAUNCH(launch_gdh_spectrum(ctx->d_eps, ctx->d_core_idx, ctx->n_core, omega, n_omega, sigma_c, dh, ctx->d_sx,
                             ctx->d_vxc_eff, a_out, omega_out, (cudaStream_t)stream));
  return check_stream_error(ctx);
}

// ---- request mode ----------------------------------------------------------------------------------
gwc_status gwc_request_plan(gwc_ctx* ctx, const double* omega_rel, int n_omega, void* stream) {
  if (ctx) TRY(need_occupied_cores(ctx, "gwc_request_plan"));
  if (!ctx) return fail(nullptr, GWC_ERR_INVALID_ARG, "ctx is NULL");
  if (!ctx->loaded) return fail(ctx, GWC_ERR_INVALID_ARG, "no system loaded (gwc_load)");
  if (!omega_rel || n_omega < 1 || n_omega > 8192)
    return fail(ctx, GWC_ERR_INVALID_ARG, "need omega_rel and 1 <= n_omega <= 8192");
  if (ctx->opt.dec != GWC_DECOUPLE_DIAG)
    return fail(ctx, GWC_ERR_UNSUPPORTED, "request mode computes the DIAG decoupled Im Sigma only");
  for (int j = 0; j < n_omega; ++j) {
    if (!std::isfinite(omega_rel[j])) return fail(ctx, GWC_ERR_INVALID_ARG, "omega_rel must be finite");
    if (j > 0 && !(omega_rel[j] > omega_rel[j - 1])) return fail(ctx, GWC_ERR_INVALID_ARG, "omega_rel must ascend");
  }
  cudaStream_t st = (cudaStream_t)stream;
  const int nc = ctx->n_core;
  // one residue pair per grid point with f != 0 for the (occupied) cores: w_rel <= 0 (eq cd_prefactors)
  auto th = [](double x) { return x > 0.0 ? 1.0 : (x < 0.0 ? 0.0 : 0.5); };
  std::vector<int> pair_of(n_omega, -1), rows;
  std::vector<double> z;
  for (int j = 0; j < n_omega; ++j) {
    bool any = false;
    for (int c = 0; c < nc; ++c) {
      const double ec = ctx->h_eps[ctx->h_core[c]], w = ec + omega_rel[j];
      const double f = -th(ctx->eps_f - ec) * th(ec - w) + th(ec - ctx->eps_f) * th(w - ec);
      any = any || f != 0.0;
    }
    if (!any) continue;
    pair_of[j] = (int)(z.size() / 2);
    z.push_back(std::fabs(omega_rel[j]));
    z.push_back(ctx->opt.eta);
    for (int c = 0; c < nc; ++c) rows.push_back(ctx->h_core[c] * nc + c);  // o_core[core c][c]: O^P_cc
  }
  const int np = (int)(z.size() / 2);
  std::vector<double> wrel((size_t)nc * n_omega);
  for (int c = 0; c < nc; ++c)
    for (int j = 0; j < n_omega; ++j) wrel[(size_t)c * n_omega + j] = omega_rel[j];
  const size_t nt = ctx->opt.n_t;
  // grow-only: a context reused for requests of other sizes (serving) allocates only to grow
  TRY(grow(ctx, &ctx->d_req_wrel, &ctx->req_cap_wrel, wrel.size()));
  TRY(grow(ctx, &ctx->d_req_z, &ctx->req_cap_z, std::max<size_t>(2, z.size())));
  TRY(grow(ctx, &ctx->d_req_rows, &ctx->req_cap_rows, std::max<size_t>(1, rows.size())));
  TRY(grow(ctx, &ctx->d_req_pair_of, &ctx->req_cap_pair, n_omega));
  TRY(grow(ctx, &ctx->d_req_w, &ctx->req_cap_w, std::max<size_t>(1, (size_t)np) * nc * 2));
  TRY(grow(ctx, &ctx->d_req_im, &ctx->req_cap_im, (size_t)nc * n_omega));
  TRY(grow(ctx, &ctx->d_req_a, &ctx->req_cap_a, (size_t)nc * nt));
  TRY(grow(ctx, &ctx->d_req_nu, &ctx->req_cap_nu, nt));
  size_t cap_core = ctx->req_cap_core;
  TRY(grow(ctx, &ctx->d_req_eqp, &cap_core, nc));
  cap_core = ctx->req_cap_core;
  TRY(grow(ctx, &ctx->d_req_dh, &cap_core, nc));
  cap_core = ctx->req_cap_core;
  TRY(grow(ctx, &ctx->d_req_it, &cap_core, nc));
  ctx->req_cap_core = cap_core;
  if (nc * nt * 2 > ctx->cw_cap) {
    TRY(dalloc(ctx, &ctx->d_cw_a, nc * nt * 2));
    TRY(dalloc(ctx, &ctx->d_cw_b, nc * nt * 2));
    TRY(dalloc(ctx, &ctx->d_tw, nt));
    ctx->cw_cap = nc * nt * 2;
  }
  if ((size_t)nc * n_omega > ctx->coef_cap) {
    TRY(dalloc(ctx, &ctx->d_coef, (size_t)nc * n_omega));
    ctx->coef_cap = (size_t)nc * n_omega;
  }
  CU(cudaMemcpyAsync(ctx->d_req_wrel, wrel.data(), sizeof(double) * wrel.size(), cudaMemcpyHostToDevice, st));
  if (np > 0) {
    CU(cudaMemcpyAsync(ctx->d_req_z, z.data(), sizeof(double) * z.size(), cudaMemcpyHostToDevice, st));
    CU(cudaMemcpyAsync(ctx->d_req_rows, rows.data(), sizeof(int) * rows.size(), cudaMemcpyHostToDevice, st));
  }
  CU(cudaMemcpyAsync(ctx->d_req_pair_of, pair_of.data(), sizeof(int) * n_omega, cudaMemcpyHostToDevice, st));
  CU(cudaStreamSynchronize(st));
  ctx->req_n_omega = n_omega;
  ctx->req_n_pairs = np;
  return check_stream_error(ctx);
}

gwc_status gwc_request_step(gwc_ctx* ctx, void* stream) {
  if (!ctx) return fail(nullptr, GWC_ERR_INVALID_ARG, "ctx is NULL");
  if (!ctx->loaded) return fail(ctx, GWC_ERR_INVALID_ARG, "no system loaded (gwc_load)");
  if (ctx->req_n_omega <= 0) return fail(ctx, GWC_ERR_INVALID_ARG, "no request plan (call gwc_request_plan first)");
  cudaStream_t st = (cudaStream_t)stream;
  const int nc = ctx->n_core;
  TRY(enqueue_wim(ctx, st));
  ctx->wim_valid = true;
  TRY(enqueue_qp(ctx, ctx->d_req_eqp, ctx->d_req_dh, ctx->d_req_it, false, st));
  if (ctx->req_n_pairs > 0)
    TRY(residue_batches(ctx, ctx->req_n_pairs, ctx->d_req_z, ctx->d_req_rows, nc, ctx->d_req_w, nullptr, st));
  LAUNCH(launch_request_dec(ctx->d_eps, ctx->d_core_idx, nc, ctx->eps_f, ctx->d_req_wrel, ctx->req_n_omega,
                            ctx->d_req_pair_of, ctx->d_req_w, ctx->d_req_im, st));
  LAUNCH(launch_cumulant_spectrum(ctx->d_req_wrel, ctx->req_n_omega, ctx->d_req_im, nc, ctx->opt.n_t, ctx->opt.t_max,
                                  ctx->opt.eta, ctx->d_cw_a, ctx->d_cw_b, ctx->d_coef, ctx->d_tw, ctx->d_req_a,
                                  ctx->d_req_nu, st));
  return check_stream_error(ctx);
}

gwc_status gwc_request_results_get(const gwc_ctx* ctx, gwc_request_results* out) {
  if (!ctx || !out) return GWC_ERR_INVALID_ARG;
  if (ctx->req_n_omega <= 0) return GWC_ERR_INVALID_ARG;
  out->eps_qp = ctx->d_req_eqp;
  out->dh = ctx->d_req_dh;
  out->iters = ctx->d_req_it;
  out->im_sigma = ctx->d_req_im;
  out->a = ctx->d_req_a;
  out->nu = ctx->d_req_nu;
  out->n_core = ctx->n_core;
  out->n_omega = ctx->req_n_omega;
  out->n_t = ctx->opt.n_t;
  return GWC_OK;
}

gwc_status gwc_request_copy_results(const gwc_ctx* ctx, double* eps_qp, double* dh, int* iters, double* im_sigma,
                                    double* a, double* nu, void* stream) {
  if (!ctx || ctx->req_n_omega <= 0) return GWC_ERR_INVALID_ARG;
  cudaStream_t st = (cudaStream_t)stream;
  const size_t nc = ctx->n_core, nw = ctx->req_n_omega, nt = ctx->opt.n_t;
  struct Cp {
    void* dst;
    const void* src;
    size_t bytes;
  } cps[] = {{eps_qp, ctx->d_req_eqp, nc * 8}, {dh, ctx->d_req_dh, nc * 8}, {iters, ctx->d_req_it, nc * 4},
             {im_sigma, ctx->d_req_im, nc * nw * 8}, {a, ctx->d_req_a, nc * nt * 8}, {nu, ctx->d_req_nu, nt * 8}};
  for (auto& c : cps)
    if (c.dst && cudaMemcpyAsync(c.dst, c.src, c.bytes, cudaMemcpyDefault, st) != cudaSuccess) return GWC_ERR_CUDA;
  return GWC_OK;
}

// ---- autotuner: frequencies per batch and chi0 tile/launch shapes, timed on residue batches, cached per shape bucket
namespace {
std::mutex g_tune_mutex;
struct TuneChoice {
  int batch;      // frequencies per batch
  int chi0_ctas;  // 0: one CTA (pair) per chi0 item, else persistent
  int chi0_tile;  // 0: 256 x 128 pair tiles, 1: 128 x 128 one-CTA tiles
};
// (n_aux/128, n_ov/4096, n_core, prec, tile shapes allowed) -> choice
std::map<std::tuple<int, int, int, int, int>, TuneChoice> g_tune_cache;
}  // namespace

gwc_status gwc_autotune(gwc_ctx* ctx, void* stream, int* chosen) {
  if (!ctx) return fail(nullptr, GWC_ERR_INVALID_ARG, "ctx is NULL");
  if (ctx->req_n_omega <= 0) return fail(ctx, GWC_ERR_INVALID_ARG, "no request plan (call gwc_request_plan first)");
  cudaStream_t st = (cudaStream_t)stream;
  const bool tc = ctx->opt.prec == GWC_PREC_BF16 || ctx->opt.prec == GWC_PREC_BF16X3 || ctx->opt.prec == GWC_PREC_BF16X3_F64;
  // both tile shapes are candidates unless GWC_CHI0_KERNEL=single pinned the one-CTA kernel
  const char* ck = std::getenv("GWC_CHI0_KERNEL");
  const bool both_tiles = tc && !(ck && std::strcmp(ck, "single") == 0);
  const auto key = std::make_tuple((ctx->n_aux + 127) / 128, (ctx->n_ov + 4095) / 4096, ctx->n_core, ctx->opt.prec,
                                   both_tiles ? 2 : 1);
  {
    std::lock_guard<std::mutex> lock(g_tune_mutex);
    auto it = g_tune_cache.find(key);
    if (it != g_tune_cache.end()) {
      ctx->batch = std::min(it->second.batch, ctx->batch_cap);
      ctx->opt.chi0_ctas = it->second.chi0_ctas;
      ctx->opt.chi0_tile = it->second.chi0_tile;
      ctx->chi0_pair = ctx->opt.chi0_tile == 0;
      if (chosen) *chosen = ctx->batch;
      return GWC_OK;
    }
  }
  const int saved_profile = ctx->opt.profile;
  ctx->opt.profile = 0;
  int best = ctx->batch_cap;
  double best_per = 1e300;
  cudaEvent_t e0, e1;
  CU(cudaEventCreate(&e0));
  CU(cudaEventCreate(&e1));
  gwc_status res = GWC_OK;
  // candidates 16, 32, ... below one SM-wave, whole SM-waves, and the capacity; each timed on ONE
  // residue batch of that size (its per-build time), after one warm-up launch, so tuning costs a
  // few batches, not whole steps
  std::vector<int> cands;
  for (int f = 16; f < std::min(ctx->batch_cap, ctx->n_sm); f *= 2) cands.push_back(f);
  for (int f = ctx->n_sm; f < ctx->batch_cap; f += ctx->n_sm) cands.push_back(f);
  cands.push_back(ctx->batch_cap);
  const int np = ctx->req_n_pairs;
  const int saved_ctas = ctx->opt.chi0_ctas, saved_tile = ctx->opt.chi0_tile;
  int best_ctas = saved_ctas, best_tile = saved_tile;
  for (int f : cands) {
    if (res != GWC_OK || np <= 0) break;
    const int nb = std::min(f, np);
    ctx->batch = nb;
    for (int cand = 0; cand < (tc ? (both_tiles ? 4 : 2) : 1) && res == GWC_OK; ++cand) {
      const int shape = cand & 1;
      ctx->opt.chi0_ctas = tc ? (shape == 0 ? 0 : ctx->n_sm) : saved_ctas;
      ctx->opt.chi0_tile = both_tiles ? (cand >> 1) : saved_tile;
      ctx->chi0_pair = ctx->opt.chi0_tile == 0;
      res = residue_batches(ctx, nb, ctx->d_req_z, ctx->d_req_rows, ctx->n_core, ctx->d_req_w, nullptr, st);
      if (res != GWC_OK) break;
      cudaEventRecord(e0, st);
      res = residue_batches(ctx, nb, ctx->d_req_z, ctx->d_req_rows, ctx->n_core, ctx->d_req_w, nullptr, st);
      cudaEventRecord(e1, st);
      if (cudaEventSynchronize(e1) != cudaSuccess) res = fail(ctx, GWC_ERR_CUDA, "autotune sync failed");
      float ms = 0.f;
      cudaEventElapsedTime(&ms, e0, e1);
      const double per = ms / nb;
      if (res == GWC_OK && per < best_per) {
        best_per = per;
        best = f;
        best_ctas = ctx->opt.chi0_ctas;
        best_tile = ctx->opt.chi0_tile;
      }
    }
    if (nb < f) break;  // fewer pairs than the candidate: larger batches change nothing
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  ctx->opt.profile = saved_profile;
  ctx->batch = best;
  ctx->opt.chi0_ctas = best_ctas;
  ctx->opt.chi0_tile = best_tile;
  ctx->chi0_pair = best_tile == 0;
  if (res != GWC_OK) return res;
  {
    std::lock_guard<std::mutex> lock(g_tune_mutex);
    g_tune_cache[key] = TuneChoice{best, best_ctas, best_tile};
  }
  if (chosen) *chosen = best;
  return GWC_OK;
}

// ---- batched form: one CUDA graph over many contexts ----------------------------------------------------
// Grouped form (all contexts in a tensor-core mode, Hedin QP, DIAG decoupling): every polarizability build of
// a phase, over all molecules, goes through ONE persistent grouped chi0 launch (n_SM CTAs looping over the
// (molecule, frequency batch, tile) items) and every complex factorisation through ONE grouped LDL^T launch;
// the small per-molecule kernels (D tables, appended rows, contractions, QP update, spectra) sit between
// them. The whole sequence is captured into one CUDA graph.
namespace {

struct GroupedLaunch {
  bool complex_z = false;
  std::vector<int> ctx_of;      // context of each chi0 group / factor group
  std::vector<int> p0, nb;      // pair range of each context in this launch
  std::vector<int> half;        // first matrix of the workspace half each context's chunk uses
  size_t chi0_off = 0;          // byte offset of the chi0 descriptors in the batch's device buffer
  int chi0_groups = 0, chi0_items = 0;
  size_t fac_off = 0;           // byte offset of the factor descriptors (complex launches)
  int fac_groups = 0, fac_ctas = 0;
};

struct GroupedPlan {
  bool pipelined = false;  // residue chunks in workspace halves, builds of chunk k+1 beside factorisations of k
  bool chi0_pair = false;  // descriptors of the CTA-pair chi0 kernel
  std::vector<GroupedLaunch> table, qp, spec;  // one per chunk of imaginary nodes / pairs
  void* d_desc = nullptr;
  size_t desc_bytes = 0;
  int chi0_ctas = 0;
};

bool grouped_eligible(gwc_ctx* const* ctxs, int n) {
  for (int i = 0; i < n; ++i) {
    const gwc_ctx* c = ctxs[i];
    if (c->chi0_pair != ctxs[0]->chi0_pair) return false;  // one chi0 kernel per grouped launch
    if (c->wtable_tc != ctxs[0]->wtable_tc) return false;  // one storage of the table builds
    if (!(c->opt.prec == GWC_PREC_BF16 || c->opt.prec == GWC_PREC_BF16X3) || !c->factor_tc) return false;
    if (c->opt.qp_mode != GWC_QP_HEDIN || c->opt.dec != GWC_DECOUPLE_DIAG || c->req_n_omega <= 0) return false;
    if (c->n_core > c->border_max) return false;
  }
  return true;
}

// Residue chunk of one context in the grouped form: its whole workspace, or half of it when two chunks are
// in flight (pipelined).
int grouped_chunk(const gwc_ctx* c, bool pipelined) { return std::max(1, pipelined ? c->batch / 2 : c->batch); }

// Appends the descriptors of one grouped launch: a chi0 group and (complex) a factor group per context
// chunk. kind 0: table, 1: QP pairs, 2: spectrum pairs; k: chunk index.
gwc_status plan_launch(gwc_ctx* const* ctxs, int n, int kind, int k, bool pipelined, std::vector<uint8_t>& host,
                       GroupedLaunch& L) {
  const bool pair = ctxs[0]->chi0_pair;
  const size_t gb = pair ? chi0_pair_group_bytes() : chi0_group_bytes();
  L.complex_z = kind != 0 || ctxs[0]->wtable_tc;  // the tensor-core table builds in complex storage
  std::vector<uint8_t> chi0((size_t)n * gb);
  std::vector<LdltGroup> fac;
  int items = 0, ctas = 0, groups = 0;
  // largest contraction first: with the items dealt round-robin to the persistent CTAs, the long items are
  // spread over all CTAs and the short ones fill in behind them
  std::vector<int> order(n);
  for (int i = 0; i < n; ++i) order[i] = i;
  std::stable_sort(order.begin(), order.end(), [&](int a, int b) {
    return (long long)ctxs[a]->n_ov_pad * ctxs[a]->n_aux_pad > (long long)ctxs[b]->n_ov_pad * ctxs[b]->n_aux_pad;
  });
  for (int i : order) {
    gwc_ctx* c = ctxs[i];
    int F, p0 = 0;
    const int* act = nullptr;
    long long stride;
    int r = 0;
    if (kind == 0) {
      const int fb = wim_batch(c);
      p0 = k * fb;
      if (p0 >= c->opt.n_im + 1) continue;
      F = std::min(fb, c->opt.n_im + 1 - p0);
      stride = (long long)c->n_aux * c->ldm;
    } else {
      const int np = kind == 1 ? c->n_core * c->n_occ : c->req_n_pairs;
      const int chunk = grouped_chunk(c, pipelined);
      p0 = k * chunk;
      if (p0 >= np) continue;
      F = std::min(chunk, np - p0);
      r = kind == 1 ? 1 : c->n_core;
      stride = (long long)(c->n_aux + r) * c->ldm;
      if (kind == 1) act = c->d_qp_active + p0;
    }
    // residue chunks alternate between the two halves of the workspace (the build of chunk k + 1 overlaps
    // the factorisation of chunk k); the table uses the whole workspace
    const int half = (kind == 0 || !pipelined) ? 0 : (k & 1) * grouped_chunk(c, true);
    float* dtab = reinterpret_cast<float*>(c->d_dtab) + (size_t)half * 2 * c->ld_dtab;
    float2* mats = static_cast<float2*>(c->d_mats) + (size_t)half * stride;
    const int got = (pair ? chi0_pair_group_fill : chi0_group_fill)(
        chi0.data() + (size_t)groups * gb, c->opt.prec != GWC_PREC_BF16, c->d_o_hi, c->d_o_lo, c->d_o_f32, c->n_ov_pad,
        c->n_aux, c->n_aux_pad, c->n_ov_pad, dtab, c->ld_dtab, F, L.complex_z, -1.0, 1.0, mats, c->ldm, stride, act, false,
        items);
    if (got < 0) return fail(nullptr, GWC_ERR_UNSUPPORTED, "tensor-core chi0 not available for a batch member");
    items += got;
    if (kind != 0) {
      LdltGroup G;
      G.mats = mats;
      G.ldm = c->ldm;
      G.stride = stride;
      G.active = act;
      G.n = c->n_aux;
      G.nrow = c->n_aux + r;
      G.F = F;
      G.cta0 = ctas;
      ctas += F;
      fac.push_back(G);
    }
    L.ctx_of.push_back(i);
    L.p0.push_back(p0);
    L.nb.push_back(F);
    L.half.push_back(half);
    ++groups;
  }
  L.chi0_groups = groups;
  L.chi0_items = items;
  if (groups == 0) return GWC_OK;
  // descriptors, 64-byte aligned pieces of one buffer
  auto align = [](size_t x) { return (x + 255) / 256 * 256; };
  L.chi0_off = align(host.size());
  host.resize(L.chi0_off + (size_t)groups * gb);
  std::memcpy(host.data() + L.chi0_off, chi0.data(), (size_t)groups * gb);
  if (!fac.empty()) {
    L.fac_off = align(host.size());
    host.resize(L.fac_off + fac.size() * sizeof(LdltGroup));
    std::memcpy(host.data() + L.fac_off, fac.data(), fac.size() * sizeof(LdltGroup));
    L.fac_groups = (int)fac.size();
    L.fac_ctas = ctas;
  }
  return GWC_OK;
}

gwc_status build_plan(gwc_ctx* const* ctxs, int n, GroupedPlan& P) {
  const bool pl = P.pipelined;
  P.chi0_pair = ctxs[0]->chi0_pair;
  std::vector<uint8_t> host;
  for (int k = 0;; ++k) {
    GroupedLaunch L;
    TRY(plan_launch(ctxs, n, 0, k, pl, host, L));
    if (L.chi0_groups == 0) break;
    P.table.push_back(L);
  }
  for (int k = 0;; ++k) {
    GroupedLaunch L;
    TRY(plan_launch(ctxs, n, 1, k, pl, host, L));
    if (L.chi0_groups == 0) break;
    P.qp.push_back(L);
  }
  for (int k = 0;; ++k) {
    GroupedLaunch L;
    TRY(plan_launch(ctxs, n, 2, k, pl, host, L));
    if (L.chi0_groups == 0) break;
    P.spec.push_back(L);
  }
  P.desc_bytes = host.size();
  if (cudaMalloc(&P.d_desc, std::max<size_t>(host.size(), 256)) != cudaSuccess)
    return fail(nullptr, GWC_ERR_OOM, "batch descriptor allocation failed");
  if (cudaMemcpy(P.d_desc, host.data(), host.size(), cudaMemcpyHostToDevice) != cudaSuccess)
    return fail(nullptr, GWC_ERR_CUDA, "batch descriptor upload failed");
  return GWC_OK;
}

#define BCU(call)                                                                                              \
  do {                                                                                                         \
    if ((call) < 0) return fail(nullptr, GWC_ERR_CUDA, std::string("batch launch failed: ") + #call);        \
  } while (0)

// One grouped launch of residue builds, in two parts: (a) the D tables of every member and one chi0 launch,
// (b) the appended rows, one factorisation launch and the contractions. Part (a) of the next chunk runs
// on its own stream beside part (b) of this one (they use the two halves of each workspace).
gwc_status enqueue_grouped_build(gwc_ctx* const* ctxs, const GroupedPlan& P, const GroupedLaunch& L, int kind,
                                 cudaStream_t st) {
  const char* base = static_cast<const char*>(P.d_desc);
  for (size_t j = 0; j < L.ctx_of.size(); ++j) {
    gwc_ctx* c = ctxs[L.ctx_of[j]];
    const double* z = (kind == 1 ? c->d_qp_z : c->d_req_z) + 2 * (size_t)L.p0[j];
    float* dtab = reinterpret_cast<float*>(c->d_dtab) + (size_t)L.half[j] * 2 * c->ld_dtab;
    BCU(launch_dtable(z, L.nb[j], c->d_delta, c->n_ov, c->ld_dtab, true, dtab, st));
  }
  BCU((P.chi0_pair ? launch_chi0_pair_grouped : launch_chi0_tc_grouped)(base + L.chi0_off, L.chi0_groups, L.chi0_items, true, P.chi0_ctas,
                             ctxs[L.ctx_of[0]]->d_status, ctxs[L.ctx_of[0]]->wait_ns, st));
  return GWC_OK;
}

gwc_status enqueue_grouped_factor(gwc_ctx* const* ctxs, const GroupedPlan& P, const GroupedLaunch& L, int kind,
                                  cudaStream_t st) {
  const char* base = static_cast<const char*>(P.d_desc);
  for (size_t j = 0; j < L.ctx_of.size(); ++j) {
    gwc_ctx* c = ctxs[L.ctx_of[j]];
    const int r = kind == 1 ? 1 : c->n_core;
    const long long stride = (long long)(c->n_aux + r) * c->ldm;
    const int* rows = (kind == 1 ? c->d_qp_rowmap : c->d_req_rows) + (size_t)L.p0[j] * r;
    float2* mats = static_cast<float2*>(c->d_mats) + (size_t)L.half[j] * stride;
    BCU(launch_border_rows(MatKind::CplxF32, mats, c->n_aux, c->ldm, stride, c->d_o_core, c->n_aux, rows, L.nb[j], r,
                           c->d_bnorm + (size_t)L.half[j] * r, st));
  }
  BCU(launch_ldlt_tc_grouped(reinterpret_cast<const LdltGroup*>(base + L.fac_off), L.fac_groups, L.fac_ctas,
                             ctxs[L.ctx_of[0]]->d_status, ctxs[L.ctx_of[0]]->wait_ns, st));
  for (size_t j = 0; j < L.ctx_of.size(); ++j) {
    gwc_ctx* c = ctxs[L.ctx_of[j]];
    const int r = kind == 1 ? 1 : c->n_core;
    const long long stride = (long long)(c->n_aux + r) * c->ldm;
    double* w = (kind == 1 ? c->d_qp_w : c->d_req_w) + (size_t)L.p0[j] * r * 2;
    const int* act = kind == 1 ? c->d_qp_active + L.p0[j] : nullptr;
    float2* mats = static_cast<float2*>(c->d_mats) + (size_t)L.half[j] * stride;
    BCU(launch_border_w(MatKind::CplxF32, mats, c->n_aux, c->ldm, stride, L.nb[j], r, c->d_bnorm + (size_t)L.half[j] * r,
                        w, (long long)r * 2, act, st));
  }
  return GWC_OK;
}

// The chunks of one residue phase: builds on `st`, factorisations on `side`, two chunks in flight.
gwc_status enqueue_grouped_phase(gwc_ctx* const* ctxs, const GroupedPlan& P, const std::vector<GroupedLaunch>& Ls,
                                 int kind, cudaStream_t st, cudaStream_t side, const std::vector<cudaEvent_t>& ev) {
  const size_t n = Ls.size();
  if (n == 0) return GWC_OK;
  if (ev.size() < 2 * n) return fail(nullptr, GWC_ERR_INVALID_ARG, "batch event pool too small");
  if (!P.pipelined) {  // one stream, chunk after chunk
    for (size_t k = 0; k < n; ++k) {
      TRY(enqueue_grouped_build(ctxs, P, Ls[k], kind, st));
      TRY(enqueue_grouped_factor(ctxs, P, Ls[k], kind, st));
    }
    return GWC_OK;
  }
  const cudaEvent_t* ev_a = ev.data();      // build of chunk k done
  const cudaEvent_t* ev_b = ev.data() + n;  // factorisation of chunk k done: its workspace half is free
  for (size_t k = 0; k < n; ++k) {
    if (k >= 2 && cudaStreamWaitEvent(st, ev_b[k - 2], 0) != cudaSuccess) return fail(nullptr, GWC_ERR_CUDA, "wait");
    TRY(enqueue_grouped_build(ctxs, P, Ls[k], kind, st));
    if (cudaEventRecord(ev_a[k], st) != cudaSuccess || cudaStreamWaitEvent(side, ev_a[k], 0) != cudaSuccess)
      return fail(nullptr, GWC_ERR_CUDA, "batch event record failed");
    TRY(enqueue_grouped_factor(ctxs, P, Ls[k], kind, side));
    if (cudaEventRecord(ev_b[k], side) != cudaSuccess) return fail(nullptr, GWC_ERR_CUDA, "batch event record failed");
  }
  if (cudaStreamWaitEvent(st, ev_b[n - 1], 0) != cudaSuccess) return fail(nullptr, GWC_ERR_CUDA, "batch join failed");
  return GWC_OK;
}

// The request step of every context as grouped launches, enqueued on `st` (capturable: no host sync).
gwc_status enqueue_grouped_step(gwc_ctx* const* ctxs, int n, const GroupedPlan& P, cudaStream_t st, cudaStream_t side,
                                const std::vector<cudaEvent_t>& ev) {
  const char* base = static_cast<const char*>(P.d_desc);
  // imaginary-axis W tables: one grouped chi0 launch over all molecules' nodes (per chunk of nodes)
  for (const GroupedLaunch& L : P.table) {
    for (size_t j = 0; j < L.ctx_of.size(); ++j) {
      gwc_ctx* c = ctxs[L.ctx_of[j]];
      BCU(launch_dtable(c->d_zim + 2 * (size_t)L.p0[j], L.nb[j], c->d_delta, c->n_ov, c->ld_dtab, true, c->d_dtab, st));
    }
    BCU((P.chi0_pair ? launch_chi0_pair_grouped : launch_chi0_tc_grouped)(base + L.chi0_off, L.chi0_groups, L.chi0_items, L.complex_z, P.chi0_ctas,
                               ctxs[L.ctx_of[0]]->d_status, ctxs[L.ctx_of[0]]->wait_ns, st));
    for (size_t j = 0; j < L.ctx_of.size(); ++j) TRY(enqueue_wim_tail(ctxs[L.ctx_of[j]], L.p0[j], L.nb[j], st));
  }
  for (int i = 0; i < n; ++i) ctxs[i]->wim_valid = true;
  // QP: the Hedin shift of every core (eq QPGWC), its residue pairs in grouped launches
  for (int i = 0; i < n; ++i) {
    gwc_ctx* c = ctxs[i];
    BCU(launch_qp_init(c->d_eps, c->d_core_idx, c->n_core, c->qp_mask_set ? c->d_qp_mask : nullptr, c->d_qp, st));
    BCU(launch_qp_pairs(c->d_eps, c->d_core_idx, c->n_core, c->n_occ, c->eps_f, c->opt.eta, c->d_qp, c->d_qp_z,
                        c->d_qp_active, c->d_qp_fac, c->d_all_done, c->d_active_builds, st));
  }
  TRY(enqueue_grouped_phase(ctxs, P, P.qp, 1, st, side, ev));
  for (int i = 0; i < n; ++i) {
    gwc_ctx* c = ctxs[i];
    BCU(launch_qp_assemble_update(c->d_eps, c->n_states, c->n_occ, c->n_core, c->d_core_idx, c->eps_f, c->d_xi, c->d_wxi,
                                  c->opt.n_im, c->d_wim, c->d_qp_w, c->d_qp_fac, c->d_sx, c->d_vxc_eff, c->opt.qp_tol,
                                  c->opt.max_qp_iter, 0, c->d_qp, c->d_all_done, st));
    BCU(launch_qp_finish_hedin(c->d_qp, c->d_eps, c->d_core_idx, c->n_core, c->d_req_eqp, c->d_req_dh, c->d_req_it, st));
  }
  // decoupled Im Sigma on the relative grid and the spectra
  TRY(enqueue_grouped_phase(ctxs, P, P.spec, 2, st, side, ev));
  for (int i = 0; i < n; ++i) {
    gwc_ctx* c = ctxs[i];
    BCU(launch_request_dec(c->d_eps, c->d_core_idx, c->n_core, c->eps_f, c->d_req_wrel, c->req_n_omega, c->d_req_pair_of,
                           c->d_req_w, c->d_req_im, st));
    BCU(launch_cumulant_spectrum(c->d_req_wrel, c->req_n_omega, c->d_req_im, c->n_core, c->opt.n_t, c->opt.t_max,
                                 c->opt.eta, c->d_cw_a, c->d_cw_b, c->d_coef, c->d_tw, c->d_req_a, c->d_req_nu, st));
  }
  return GWC_OK;
}
#undef BCU

}  // namespace

struct gwc_batch {
  cudaStream_t cap = nullptr;  // internal capture origin (the caller's stream may be the legacy one)
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  std::vector<cudaStream_t> streams;
  std::vector<cudaEvent_t> events;
  std::vector<gwc_ctx*> ctxs;
  bool grouped = false;
  GroupedPlan plan;   // the grouped plan in use (after creation: the chosen one)
  GroupedPlan plan2;  // the other grouped candidate
  cudaStream_t side = nullptr;          // grouped form: the factorisation stream
  std::vector<cudaEvent_t> gev;         // grouped form: events of the two-chunk pipeline
  float t_candidates[3] = {-1.f, -1.f, -1.f};  // timed plans (ms): per-molecule, grouped persistent, grouped
                                               // pipelined with one chi0 CTA per item
};

void gwc_batch_destroy(gwc_batch* b) {
  if (!b) return;
  if (b->exec) cudaGraphExecDestroy(b->exec);
  if (b->graph) cudaGraphDestroy(b->graph);
  for (auto e : b->events) cudaEventDestroy(e);
  for (auto s : b->streams) cudaStreamDestroy(s);
  if (b->cap) cudaStreamDestroy(b->cap);
  if (b->side) cudaStreamDestroy(b->side);
  for (auto e : b->gev) cudaEventDestroy(e);
  if (b->plan.d_desc) cudaFree(b->plan.d_desc);
  if (b->plan2.d_desc) cudaFree(b->plan2.d_desc);
  delete b;
}

int gwc_batch_is_grouped(const gwc_batch* b) { return b && b->grouped ? (b->plan.chi0_ctas < (1 << 30) ? 2 : 1) : 0; }

gwc_status gwc_batch_timings(const gwc_batch* b, float* ms3) {
  if (!b || !ms3) return GWC_ERR_INVALID_ARG;
  for (int k = 0; k < 3; ++k) ms3[k] = b->t_candidates[k];
  return GWC_OK;
}

gwc_status gwc_batch_create(gwc_batch** out, gwc_ctx* const* ctxs, int n, void* stream) {
  // errors of this function go to gwc_last_error(NULL)
  if (!out || !ctxs || n < 1) return fail(nullptr, GWC_ERR_INVALID_ARG, "need out, ctxs and n >= 1");
  *out = nullptr;
  for (int i = 0; i < n; ++i)
    if (!ctxs[i] || ctxs[i]->req_n_omega <= 0)
      return fail(nullptr, GWC_ERR_INVALID_ARG, "every context needs a request plan");
  gwc_batch* b = new gwc_batch();
  b->ctxs.assign(ctxs, ctxs + n);
  auto bail = [&](gwc_status s, const std::string& m) {
    gwc_batch_destroy(b);
    return fail(nullptr, s, m);
  };
  if (cudaStreamSynchronize((cudaStream_t)stream) != cudaSuccess ||
      cudaStreamCreateWithFlags(&b->cap, cudaStreamNonBlocking) != cudaSuccess)
    return bail(GWC_ERR_CUDA, "capture stream creation failed");
  cudaStream_t st = b->cap;
  std::vector<int> saved(n);
  for (int i = 0; i < n; ++i) {
    saved[i] = ctxs[i]->opt.profile;
    ctxs[i]->opt.profile = 0;
  }
  auto restore = [&]() {
    for (int i = 0; i < n; ++i) ctxs[i]->opt.profile = saved[i];
  };
  // The launch plan is chosen by timing one uncaptured run of each candidate (they also set function
  // attributes and first-use state): the per-molecule steps on forked streams, and, where every molecule
  // allows it, the grouped form with the persistent chi0 launch and with one CTA per chi0 item. The
  // fastest is captured. GWC_BATCH=per-molecule or =grouped restricts the choice.
  const char* force = std::getenv("GWC_BATCH");
  const bool allow_grouped = grouped_eligible(ctxs, n) && !(force && std::strcmp(force, "grouped") != 0);
  const bool allow_pm = !(force && std::strcmp(force, "grouped") == 0 && allow_grouped);
  b->streams.resize(n);
  b->events.resize(n + 1);
  for (int i = 0; i < n; ++i)
    if (cudaStreamCreateWithFlags(&b->streams[i], cudaStreamNonBlocking) != cudaSuccess) {
      restore();
      return bail(GWC_ERR_CUDA, "stream creation failed");
    }
  for (int i = 0; i <= n; ++i)
    if (cudaEventCreateWithFlags(&b->events[i], cudaEventDisableTiming) != cudaSuccess) {
      restore();
      return bail(GWC_ERR_CUDA, "event creation failed");
    }
  cudaEvent_t t0 = nullptr, t1 = nullptr;
  cudaEventCreate(&t0);
  cudaEventCreate(&t1);
  auto elapsed = [&]() {
    float ms = 0.f;
    return cudaEventSynchronize(t1) == cudaSuccess && cudaEventElapsedTime(&ms, t0, t1) == cudaSuccess ? ms : -1.f;
  };
  // the per-molecule steps, forked from and joined into `st`
  auto enqueue_pm = [&]() -> gwc_status {
    cudaEventRecord(b->events[n], st);
    for (int i = 0; i < n; ++i) {
      cudaStreamWaitEvent(b->streams[i], b->events[n], 0);
      if (gwc_request_step(ctxs[i], b->streams[i]) != GWC_OK)
        return fail(nullptr, GWC_ERR_CUDA, std::string("step failed: ") + ctxs[i]->last_error);
      cudaEventRecord(b->events[i], b->streams[i]);
      cudaStreamWaitEvent(st, b->events[i], 0);
    }
    return GWC_OK;
  };
  float t_pm = -1.f, t_gp = -1.f, t_gi = -1.f;
  if (allow_pm) {
    cudaEventRecord(t0, st);
    if (enqueue_pm() != GWC_OK) {
      cudaStreamSynchronize(st);
      restore();
      return bail(GWC_ERR_CUDA, std::string("warm-up: ") + g_create_error);
    }
    cudaEventRecord(t1, st);
    t_pm = elapsed();
  }
  if (allow_grouped) {
    // candidate 1: whole-workspace chunks one after another, persistent chi0 grid (one CTA per SM);
    // candidate 2: half-workspace chunks with builds beside factorisations, one chi0 CTA per item
    b->plan.pipelined = false;
    b->plan2.pipelined = true;
    if (build_plan(ctxs, n, b->plan) != GWC_OK || build_plan(ctxs, n, b->plan2) != GWC_OK) {
      restore();
      return bail(GWC_ERR_CUDA, std::string("grouped plan: ") + g_create_error);
    }
    b->plan.chi0_ctas = ctxs[0]->n_sm;
    b->plan2.chi0_ctas = 1 << 30;
    const size_t n_ev = 2 * std::max(b->plan2.qp.size(), b->plan2.spec.size());
    b->gev.resize(n_ev, nullptr);
    bool ok_ev = cudaStreamCreateWithFlags(&b->side, cudaStreamNonBlocking) == cudaSuccess;
    for (auto& e : b->gev) ok_ev = ok_ev && cudaEventCreateWithFlags(&e, cudaEventDisableTiming) == cudaSuccess;
    if (!ok_ev) {
      restore();
      return bail(GWC_ERR_CUDA, "batch stream/event creation failed");
    }
    for (int k = 0; k < 2; ++k) {
      cudaEventRecord(t0, st);
      const bool ok = enqueue_grouped_step(ctxs, n, k == 0 ? b->plan : b->plan2, st, b->side, b->gev) == GWC_OK;
      cudaEventRecord(t1, st);
      const float ms = elapsed();
      if (!ok || ms < 0.f) {
        cudaStreamSynchronize(st);
        restore();
        return bail(GWC_ERR_CUDA, std::string("grouped warm-up step failed: ") + g_create_error);
      }
      (k == 0 ? t_gp : t_gi) = ms;
    }
  }
  cudaEventDestroy(t0);
  cudaEventDestroy(t1);
  // the fastest candidate
  float best = 1e30f;
  int pick = -1;  // 0 per-molecule, 1 grouped persistent, 2 grouped one CTA per item
  const float cand[3] = {t_pm, t_gp, t_gi};
  for (int k = 0; k < 3; ++k)
    if (cand[k] >= 0.f && cand[k] < best) {
      best = cand[k];
      pick = k;
    }
  b->t_candidates[0] = t_pm;
  b->t_candidates[1] = t_gp;
  b->t_candidates[2] = t_gi;
  b->grouped = pick >= 1;
  if (pick == 2) std::swap(b->plan, b->plan2);
  gwc_status res = GWC_OK;
  std::string msg;
  if (cudaStreamBeginCapture(st, cudaStreamCaptureModeRelaxed) != cudaSuccess) {
    res = GWC_ERR_CUDA;
    msg = "cudaStreamBeginCapture failed";
  } else {
    const gwc_status r = b->grouped ? enqueue_grouped_step(ctxs, n, b->plan, st, b->side, b->gev) : enqueue_pm();
    if (r != GWC_OK) {
      res = GWC_ERR_CUDA;
      msg = std::string("capture failed: ") + g_create_error;
    }
    cudaError_t e = cudaStreamEndCapture(st, &b->graph);
    if (res == GWC_OK && e != cudaSuccess) {
      res = GWC_ERR_CUDA;
      msg = std::string("cudaStreamEndCapture: ") + cudaGetErrorString(e);
    }
  }
  restore();
  if (res != GWC_OK) return bail(res, msg);
  cudaError_t e = cudaGraphInstantiate(&b->exec, b->graph, 0);
  if (e != cudaSuccess) return bail(GWC_ERR_CUDA, std::string("cudaGraphInstantiate: ") + cudaGetErrorString(e));
  *out = b;
  return GWC_OK;
}

gwc_status gwc_batch_launch(gwc_batch* b, void* stream) {
  if (!b || !b->exec) return fail(nullptr, GWC_ERR_INVALID_ARG, "batch is NULL");
  cudaError_t e = cudaGraphLaunch(b->exec, (cudaStream_t)stream);
  if (e != cudaSuccess) return fail(nullptr, GWC_ERR_CUDA, std::string("cudaGraphLaunch: ") + cudaGetErrorString(e));
  return GWC_OK;
}

gwc_status gwc_sync(gwc_ctx* ctx, void* stream) {
  if (!ctx) return fail(nullptr, GWC_ERR_INVALID_ARG, "ctx is NULL");
  cudaStream_t st = (cudaStream_t)stream;
  unsigned flags = 0;
  CU(cudaMemcpyAsync(&flags, ctx->d_status, sizeof(unsigned), cudaMemcpyDeviceToHost, st));
  CU(cudaStreamSynchronize(st));
  ev_flush(ctx);
  CU(cudaMemsetAsync(ctx->d_status, 0, sizeof(unsigned), st));
  CU(cudaStreamSynchronize(st));
  if (flags & kStatTimeout) return fail(ctx, GWC_ERR_TIMEOUT, "a bounded device wait gave up");
  if (flags & kStatSingular) return fail(ctx, GWC_ERR_SINGULAR, "zero pivot in a dielectric factorisation");
  if (flags & kStatNotConverged) return fail(ctx, GWC_ERR_NOT_CONVERGED, "QP secant iteration hit max_qp_iter");
  if (flags & kStatBadIndex) return fail(ctx, GWC_ERR_INVALID_ARG, "device-side index check failed");
  return GWC_OK;
}

gwc_status gwc_get_options(const gwc_ctx* ctx, gwc_options* out) {
  if (!ctx || !out) return GWC_ERR_INVALID_ARG;
  *out = ctx->opt;
  return GWC_OK;
}

gwc_status gwc_get_stats(gwc_ctx* ctx, gwc_stats* out) {
  if (!ctx || !out) return GWC_ERR_INVALID_ARG;
  ev_flush(ctx);
  fold_active_builds(ctx);
  *out = ctx->stats;
  return GWC_OK;
}

gwc_status gwc_reset_stats(gwc_ctx* ctx) {
  if (!ctx) return GWC_ERR_INVALID_ARG;
  ev_flush(ctx);
  fold_active_builds(ctx);
  ctx->stats = gwc_stats{};
  return GWC_OK;
}

}  // extern "C"
