// Self-energy assembly by contour deformation and the device-side QP secant iteration.
//
// Sigma^c_n(w) = -I_n(w) + R_n(w)                                        (Eq. cd_terms)
// I_n(w) = (1/pi) sum_m int_0^inf dxi a_m/(a_m^2 + xi^2) W^c_mn(i xi),    a_m = w - eps_m
//          evaluated as sum_k q_k a/(a^2+xi_k^2)/pi [W(i xi_k) - W(i0)] + sgn(a) W(i0)/2
//          (Eq. cd_imaginary; the odd part of the integrand cancels because W^c(i xi) is
//          even and real; W(i0) is subtracted and integrated exactly; 0 at a = 0)
// R_n(w) = sum_m f_m W^c_mn(|eps_m - w| + i eta)                          (Eq. cd_residue)
// f_m = -Theta(eps_F - eps_m) Theta(eps_m - w) + Theta(eps_m - eps_F) Theta(w - eps_m),
//       Theta(0) = 1/2                                                    (Eq. cd_prefactors)
// All arithmetic here is FP64; one warp reduces over the states m for one (core, w).
#include "gwc_internal.h"

namespace gwc {

namespace {

__device__ __forceinline__ double theta(double x) { return x > 0.0 ? 1.0 : (x < 0.0 ? 0.0 : 0.5); }

__device__ __forceinline__ double prefactor(double eps_m, double w, double eps_f) {
  return -theta(eps_f - eps_m) * theta(eps_m - w) + theta(eps_m - eps_f) * theta(w - eps_m);
}

// Imaginary-axis contribution of state m to I_n(w) for core c.
__device__ __forceinline__ double imag_term(double a, int m, int c, int n_states, int n_core, const double* __restrict__ xi,
                                            const double* __restrict__ wxi, int n_im, const double* __restrict__ wim) {
  if (a == 0.0) return 0.0;
  const size_t plane = (size_t)n_states * n_core;
  const size_t off = (size_t)m * n_core + c;
  const double w0 = wim[(size_t)n_im * plane + off];
  double s = 0.0;
  for (int k = 0; k < n_im; ++k) {
    double x = xi[k];
    s += wxi[k] * a / (a * a + x * x) * (wim[k * plane + off] - w0);
  }
  return s * (1.0 / 3.14159265358979323846) + 0.5 * copysign(1.0, a) * w0;
}

__global__ void sigma_grid_kernel(const double* __restrict__ eps, int n_states, int n_core, const int* __restrict__ core_idx,
                                  const double* __restrict__ omega, int n_w, double eps_f, const double* __restrict__ xi,
                                  const double* __restrict__ wxi, int n_im, const double* __restrict__ wim,
                                  const int* __restrict__ pidx, const double* __restrict__ wres, int dec_mode,
                                  const int* __restrict__ group_of_core, double* __restrict__ sigma,
                                  double* __restrict__ im_dec) {
  const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (warp >= n_core * n_w) return;
  const int c = warp / n_w, j = warp % n_w;
  const double w = omega[j];
  const int n = core_idx[c];
  const int gc = group_of_core ? group_of_core[c] : c;
  double si = 0.0, rr = 0.0, ri = 0.0, dec = 0.0;
  for (int m = lane; m < n_states; m += 32) {
    const double em = eps[m];
    si += imag_term(w - em, m, c, n_states, n_core, xi, wxi, n_im, wim);
    const double f = prefactor(em, w, eps_f);
    if (f != 0.0) {
      const int p = pidx[(size_t)j * n_states + m];
      const double* wv = wres + ((size_t)p * n_core + c) * 2;
      rr += f * wv[0];
      ri += f * wv[1];
      if (dec_mode == GWC_DECOUPLE_DIAG && m == n) dec += f * wv[1];
      if (dec_mode == GWC_DECOUPLE_GROUP) {
        // m belongs to the group of core c if m is a core with the same group label
        for (int c2 = 0; c2 < n_core; ++c2)
          if (core_idx[c2] == m && (group_of_core ? group_of_core[c2] : c2) == gc) dec += f * wv[1];
      }
    }
  }
  for (int o = 16; o > 0; o >>= 1) {
    si += __shfl_down_sync(0xffffffffu, si, o);
    rr += __shfl_down_sync(0xffffffffu, rr, o);
    ri += __shfl_down_sync(0xffffffffu, ri, o);
    dec += __shfl_down_sync(0xffffffffu, dec, o);
  }
  if (lane == 0) {
    double* o = sigma + ((size_t)c * n_w + j) * 2;
    o[0] = -si + rr;
    o[1] = ri;
    if (im_dec) im_dec[(size_t)c * n_w + j] = dec_mode == GWC_DECOUPLE_NONE ? ri : dec;
  }
}

// ---------------------------------------------------------------------------------------------
// QP: dH_n = Re Sigma^c_n(eps_n) + Sigma^x_n - v^xc_n (Eq. hedin_shift), then the G_dH W0 QP
// equation eps = eps_n + Sigma^x_n - v^xc_n + Re Sigma^c_n(eps - dH_n) (Eqs. quasiparticle_equation,
// hedin_sigma_spectral) by the secant method from eps_n. Phases of the per-core state machine:
//   0: evaluate Sigma at eps_n -> dH;  1: g(x0), x1 = x0 + g0;  2: g(x1), secant step;
//   3: final g(x1) after a step below tolerance;  done.
// With g0w0 set, the plain G0W0 equation (Eq. quasiparticle_equation, Sigma^c at eps itself): the
// phase-0 evaluation at eps_n already is g(x0) = dH_n, so phase 1 is skipped.
// ---------------------------------------------------------------------------------------------

// done: 0 iterating, 1 converged, 2 stopped at max_iter, 3 not requested (mask[c] == 0)
__global__ void qp_init_kernel(const double* __restrict__ eps, const int* __restrict__ core_idx, int n_core,
                               const int* __restrict__ mask, QpState* __restrict__ st) {
  int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= n_core) return;
  QpState s{};
  s.w_eval = eps[core_idx[c]];
  s.phase = 0;
  s.it = 0;
  s.done = (mask && !mask[c]) ? 3 : 0;
  st[c] = s;
}

__global__ void qp_pairs_kernel(const double* __restrict__ eps, const int* __restrict__ core_idx, int n_core, int n_occ,
                                double eps_f, double eta, const QpState* __restrict__ st, double* __restrict__ z,
                                int* __restrict__ active, double* __restrict__ fac, int* __restrict__ all_done,
                                unsigned long long* __restrict__ active_count) {
  int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t == 0) {
    int d = 1;
    for (int c = 0; c < n_core; ++c) d &= st[c].done != 0;
    *all_done = d;
  }
  if (t >= n_core * n_occ) return;
  int c = t / n_occ, m = t % n_occ;
  double w = st[c].w_eval;
  double f = st[c].done ? 0.0 : prefactor(eps[m], w, eps_f);
  fac[t] = f;
  active[t] = f != 0.0;
  if (f != 0.0 && active_count) atomicAdd(active_count, 1ull);  // builds this round really does
  z[2 * t] = fabs(eps[m] - w);
  z[2 * t + 1] = eta;
}

__global__ void qp_update_kernel(const double* __restrict__ eps, int n_states, int n_occ, int n_core,
                                 const int* __restrict__ core_idx, double eps_f, const double* __restrict__ xi,
                                 const double* __restrict__ wxi, int n_im, const double* __restrict__ wim,
                                 const double* __restrict__ wpair, const double* __restrict__ fac,
                                 const double* __restrict__ sx, const double* __restrict__ vxc, double tol, int max_iter,
                                 int g0w0, QpState* __restrict__ st, const int* __restrict__ all_done) {
  if (*all_done) return;
  const int c = blockIdx.x;
  const int lane = threadIdx.x;
  QpState s = st[c];
  if (s.done) return;
  const double w = s.w_eval;
  double si = 0.0, rr = 0.0;
  for (int m = lane; m < n_states; m += 32) {
    si += imag_term(w - eps[m], m, c, n_states, n_core, xi, wxi, n_im, wim);
    if (m < n_occ) {
      double f = fac[c * n_occ + m];
      if (f != 0.0) rr += f * wpair[(size_t)(c * n_occ + m) * 2];
    }
  }
  // virtual states with f != 0 (w above eps_m > eps_F) do not occur for a core-level w;
  // they would need residue pairs beyond n_occ and are excluded by construction.
  for (int o = 16; o > 0; o >>= 1) {
    si += __shfl_down_sync(0xffffffffu, si, o);
    rr += __shfl_down_sync(0xffffffffu, rr, o);
  }
  if (lane != 0) return;
  const double re_sigma = -si + rr;
  const double e_n = eps[core_idx[c]];
  const double stat = sx[c] - vxc[c];
  switch (s.phase) {
    case 0: {
      s.dh = re_sigma + stat;
      s.x0 = e_n;
      if (g0w0) {
        s.g0 = s.dh;  // e_n + stat + Re Sigma(e_n) - e_n
        s.x1 = s.x0 + s.g0;
        s.it = 1;
        s.w_eval = s.x1;
        s.phase = 2;
      } else {
        s.w_eval = s.x0 - s.dh;
        s.phase = 1;
      }
      break;
    }
    case 1: {
      s.g0 = e_n + stat + re_sigma - s.x0;
      s.x1 = s.x0 + s.g0;
      s.it = 1;
      s.w_eval = s.x1 - s.dh;
      s.phase = 2;
      break;
    }
    case 2: {
      s.g1 = e_n + stat + re_sigma - s.x1;
      s.it += 1;
      if (fabs(s.g1) < tol || s.it >= max_iter) {
        s.done = (fabs(s.g1) < tol) ? 1 : 2;
        break;
      }
      double denom = s.g1 - s.g0;
      double x2 = denom == 0.0 ? s.x1 + s.g1 : s.x1 - s.g1 * (s.x1 - s.x0) / denom;
      s.x0 = s.x1;
      s.g0 = s.g1;
      s.x1 = x2;
      s.w_eval = g0w0 ? s.x1 : s.x1 - s.dh;
      if (fabs(s.x1 - s.x0) < tol) s.phase = 3;
      break;
    }
    default: {
      s.g1 = e_n + stat + re_sigma - s.x1;
      s.it += 1;
      s.done = 1;
      break;
    }
  }
  st[c] = s;
}

__global__ void qp_finish_kernel(const QpState* __restrict__ st, int n_core, double* __restrict__ eps_qp,
                                 double* __restrict__ dh, int* __restrict__ iters, unsigned* __restrict__ status) {
  int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= n_core) return;
  QpState s = st[c];
  if (s.done == 3) {  // not requested
    eps_qp[c] = dh[c] = __longlong_as_double(0x7ff8000000000000ll);
    iters[c] = 0;
    return;
  }
  eps_qp[c] = s.x1;
  dh[c] = s.dh;
  iters[c] = s.it;
  if (s.done != 1) atomicOr(status, kStatNotConverged);
}

// Closed form of the G_dH W0 QP equation (eq QPGWC): eps^QP_n = eps_n + dH_n, after the phase-0
// round computed dH_n.
__global__ void qp_finish_hedin_kernel(const QpState* __restrict__ st, const double* __restrict__ eps,
                                       const int* __restrict__ core_idx, int n_core, double* __restrict__ eps_qp,
                                       double* __restrict__ dh, int* __restrict__ iters) {
  int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= n_core) return;
  const QpState s = st[c];
  if (s.done == 3) {  // not requested
    eps_qp[c] = dh[c] = __longlong_as_double(0x7ff8000000000000ll);
    iters[c] = 0;
    return;
  }
  eps_qp[c] = eps[core_idx[c]] + s.dh;
  dh[c] = s.dh;
  iters[c] = 1;
}

// Decoupled Im Sigma on a relative grid shared by all cores (eq cd_sigma_imaginary_decoupled):
// Im Sigma_c(eps_c + w_j) = f_c(eps_c + w_j) Im W^c_cc(|w_j| + i eta).
__global__ void request_dec_kernel(const double* __restrict__ eps, const int* __restrict__ core_idx, int n_core,
                                   double eps_f, const double* __restrict__ omega_rel, int n_w,
                                   const int* __restrict__ pair_of, const double* __restrict__ wpair,
                                   double* __restrict__ im) {
  int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= n_core * n_w) return;
  const int c = t / n_w, j = t % n_w;
  const int p = pair_of[j];
  const double ec = eps[core_idx[c]];
  const double f = prefactor(ec, ec + omega_rel[j], eps_f);
  im[t] = (p < 0 || f == 0.0) ? 0.0 : f * wpair[((size_t)p * n_core + c) * 2 + 1];
}

// G_dH W0 spectral function (eqs gw_full_propagator, A_explicit_real_imaginary with the shifted
// self-energy of eq hedin_sigma_spectral): on w = w' + dH_n,
//   A_n(w) = (1/pi) |Im S| / ([w - eps_n + v^xc_n - Sigma^x_n - Re S]^2 + [Im S]^2),  S = Sigma^c_n(w').
__global__ void gdh_spectrum_kernel(const double* __restrict__ eps, const int* __restrict__ core_idx, int n_core,
                                    const double* __restrict__ omega, int n_w, const double* __restrict__ sigma,
                                    const double* __restrict__ dh, const double* __restrict__ sx,
                                    const double* __restrict__ vxc, double* __restrict__ a, double* __restrict__ w_out) {
  int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= n_core * n_w) return;
  const int c = t / n_w, j = t % n_w;
  const double w = omega[j] + dh[c];
  const double re = w - eps[core_idx[c]] + vxc[c] - sx[c] - sigma[2 * (size_t)t];
  const double im = sigma[2 * (size_t)t + 1];
  a[t] = fabs(im) / (re * re + im * im) * (1.0 / 3.14159265358979323846);
  if (w_out) w_out[t] = w;
}

// ---- CD-WAC (Eq. pade_approximation) ------------------------------------------------------------
// Continued-fraction coefficients through (z_i, u_i), one thread per (occupied m, core c) pair:
// g_0(z_i) = u_i, g_p(z_i) = [g_{p-1}(z_{p-1}) - g_{p-1}(z_i)] / [(z_i - z_{p-1}) g_{p-1}(z_i)], a_p = g_p(z_p).
// u: W^c(i xi_k) (k < n_im), W^c(i0), then W^c(x_l + i eta) (l < n_ref). In place in a[pair][n_pts].
__device__ __forceinline__ double2 cmul(double2 a, double2 b) { return make_double2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x); }
__device__ __forceinline__ double2 cdiv(double2 a, double2 b) {
  const double d = b.x * b.x + b.y * b.y;
  return make_double2((a.x * b.x + a.y * b.y) / d, (a.y * b.x - a.x * b.y) / d);
}

__global__ void thiele_fit_kernel(const double* __restrict__ wim, int n_states, int n_core, int n_im,
                                  const double* __restrict__ wref /*[n_ref][n_pairs][2]*/, int n_ref, int n_pairs,
                                  const double2* __restrict__ zref, double2* __restrict__ a) {
  const int pr = blockIdx.x * blockDim.x + threadIdx.x;
  if (pr >= n_pairs) return;
  const int m = pr / n_core, c = pr % n_core;
  const int n_pts = n_im + 1 + n_ref;
  double2* g = a + (size_t)pr * n_pts;
  const size_t plane = (size_t)n_states * n_core;
  for (int k = 0; k <= n_im; ++k) g[k] = make_double2(wim[(size_t)k * plane + (size_t)m * n_core + c], 0.0);
  for (int l = 0; l < n_ref; ++l) {
    const double* w = wref + ((size_t)l * n_pairs + pr) * 2;
    g[n_im + 1 + l] = make_double2(w[0], w[1]);
  }
  for (int p = 1; p < n_pts; ++p) {
    const double2 gp = g[p - 1], zp = zref[p - 1];
    for (int i = p; i < n_pts; ++i) {
      const double2 gi = g[i];
      const double2 dz = make_double2(zref[i].x - zp.x, zref[i].y - zp.y);
      g[i] = cdiv(make_double2(gp.x - gi.x, gp.y - gi.y), cmul(dz, gi));
    }
  }
}

__device__ __forceinline__ double2 thiele_eval(const double2* __restrict__ a, const double2* __restrict__ zref, int n,
                                               double2 z) {
  double2 t = make_double2(1.0, 0.0);
  for (int p = n - 1; p > 0; --p) {
    const double2 dz = make_double2(z.x - zref[p - 1].x, z.y - zref[p - 1].y);
    const double2 q = cdiv(cmul(a[p], dz), t);
    t = make_double2(1.0 + q.x, q.y);
  }
  return cdiv(a[0], t);
}

// Sigma^c by CD-WAC: the imaginary-axis term as in CD, the residue term from the continued fraction.
__global__ void sigma_grid_wac_kernel(const double* __restrict__ eps, int n_states, int n_occ, int n_core,
                                      const int* __restrict__ core_idx, const double* __restrict__ omega, int n_w,
                                      double eps_f, double eta, const double* __restrict__ xi,
                                      const double* __restrict__ wxi, int n_im, const double* __restrict__ wim,
                                      const double2* __restrict__ coef, const double2* __restrict__ zref, int n_pts,
                                      double* __restrict__ sigma, double* __restrict__ im_dec,
                                      unsigned* __restrict__ status) {
  const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (warp >= n_core * n_w) return;
  const int c = warp / n_w, j = warp % n_w;
  const double w = omega[j];
  const int n = core_idx[c];
  double si = 0.0, rr = 0.0, ri = 0.0, dec = 0.0;
  for (int m = lane; m < n_states; m += 32) {
    const double em = eps[m];
    si += imag_term(w - em, m, c, n_states, n_core, xi, wxi, n_im, wim);
    const double f = prefactor(em, w, eps_f);
    if (f == 0.0) continue;
    if (m >= n_occ) {  // a virtual residue (w above the LUMO) has no fit: flag it
      atomicOr(status, kStatBadIndex);
      continue;
    }
    const double2 wv = thiele_eval(coef + (size_t)(m * n_core + c) * n_pts, zref, n_pts, make_double2(fabs(em - w), eta));
    rr += f * wv.x;
    ri += f * wv.y;
    if (m == n) dec += f * wv.y;
  }
  for (int o = 16; o > 0; o >>= 1) {
    si += __shfl_down_sync(0xffffffffu, si, o);
    rr += __shfl_down_sync(0xffffffffu, rr, o);
    ri += __shfl_down_sync(0xffffffffu, ri, o);
    dec += __shfl_down_sync(0xffffffffu, dec, o);
  }
  if (lane == 0) {
    double* o = sigma + ((size_t)c * n_w + j) * 2;
    o[0] = -si + rr;
    o[1] = ri;
    if (im_dec) im_dec[(size_t)c * n_w + j] = dec;
  }
}

// ---- evGW0 update (Sec. "GW for core-levels: beyond G0W0") --------------------------------------
// Every state at once: e_n <- eps_n + Sigma^x_n - v^xc_n + Re Sigma^c_n[G(e)](e_n), with
// sigma [n][n][2] the self-energies of all states on the grid of the current energies (so the
// diagonal holds Sigma^c_n(e_n)). The largest change |e_new - e| goes to *diff_bits as the bit
// pattern of a non-negative double (ordered like the value, so atomicMax is the maximum).
// Sigma^c_j(w_j) of core j at its own frequency w_j only (evGW0: every state is a core, evaluated at
// its own current energy). The residue pairs (w_j, m) carry the one right-hand side o_mj each, so
// wres1 is [pair][2]; otherwise the terms of sigma_grid_kernel.
__global__ void sigma_diag_kernel(const double* __restrict__ eps, int n_states, int n_core, const double* __restrict__ omega,
                                  double eps_f, const double* __restrict__ xi, const double* __restrict__ wxi, int n_im,
                                  const double* __restrict__ wim, const int* __restrict__ pidx,
                                  const double* __restrict__ wres1, double* __restrict__ sigma) {
  const int j = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (j >= n_core) return;
  const double w = omega[j];
  double si = 0.0, rr = 0.0, ri = 0.0;
  for (int m = lane; m < n_states; m += 32) {
    const double em = eps[m];
    si += imag_term(w - em, m, j, n_states, n_core, xi, wxi, n_im, wim);
    const double f = prefactor(em, w, eps_f);
    if (f != 0.0) {
      const int p = pidx[(size_t)j * n_states + m];
      rr += f * wres1[2 * (size_t)p];
      ri += f * wres1[2 * (size_t)p + 1];
    }
  }
  for (int o = 16; o > 0; o >>= 1) {
    si += __shfl_down_sync(0xffffffffu, si, o);
    rr += __shfl_down_sync(0xffffffffu, rr, o);
    ri += __shfl_down_sync(0xffffffffu, ri, o);
  }
  if (lane == 0) {
    sigma[2 * (size_t)j] = -si + rr;
    sigma[2 * (size_t)j + 1] = ri;
  }
}

__global__ void evgw0_update_kernel(const double* __restrict__ eps, const double* __restrict__ sx,
                                    const double* __restrict__ vxc, const double* __restrict__ sigma, int n,
                                    double* __restrict__ e, unsigned long long* __restrict__ diff_bits) {
  for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < n; k += gridDim.x * blockDim.x) {
    const double e_new = eps[k] + sx[k] - vxc[k] + sigma[2 * (size_t)k];
    const double d = fabs(e_new - e[k]);
    e[k] = e_new;
    atomicMax(diff_bits, (unsigned long long)__double_as_longlong(d));
  }
}

}  // namespace

int launch_sigma_diag(const double* eps, int n_states, int n_core, const double* omega, double eps_f, const double* xi,
                      const double* wxi, int n_im, const double* wim, const int* pidx, const double* wres1, double* sigma,
                      cudaStream_t s) {
  const long long threads = 32LL * n_core;
  sigma_diag_kernel<<<(int)((threads + 255) / 256), 256, 0, s>>>(eps, n_states, n_core, omega, eps_f, xi, wxi, n_im, wim,
                                                                  pidx, wres1, sigma);
  return cudaPeekAtLastError() == cudaSuccess ? 1 : -1;
}

int launch_evgw0_update(const double* eps, const double* sx, const double* vxc, const double* sigma, int n, double* e,
                        unsigned long long* diff_bits, cudaStream_t s) {
  evgw0_update_kernel<<<(n + 255) / 256, 256, 0, s>>>(eps, sx, vxc, sigma, n, e, diff_bits);
  return cudaPeekAtLastError() == cudaSuccess ? 1 : -1;
}

int launch_thiele_fit(const double* wim, int n_states, int n_core, int n_im, const double* wref, int n_ref, int n_pairs,
                      const double* zref, double* coef, cudaStream_t s) {
  thiele_fit_kernel<<<(n_pairs + 63) / 64, 64, 0, s>>>(wim, n_states, n_core, n_im, wref, n_ref, n_pairs,
                                                       (const double2*)zref, (double2*)coef);
  return cudaPeekAtLastError() == cudaSuccess ? 1 : -1;
}

int launch_sigma_grid_wac(const double* eps, int n_states, int n_occ, int n_core, const int* core_idx, const double* omega,
                          int n_w, double eps_f, double eta, const double* xi, const double* wxi, int n_im,
                          const double* wim, const double* coef, const double* zref, int n_pts, double* sigma,
                          double* im_dec, unsigned* status, cudaStream_t s) {
  long long warps = (long long)n_core * n_w;
  int blocks = (int)((warps * 32 + 255) / 256);
  sigma_grid_wac_kernel<<<blocks, 256, 0, s>>>(eps, n_states, n_occ, n_core, core_idx, omega, n_w, eps_f, eta, xi, wxi,
                                               n_im, wim, (const double2*)coef, (const double2*)zref, n_pts, sigma,
                                               im_dec, status);
  return cudaPeekAtLastError() == cudaSuccess ? 1 : -1;
}

int launch_gdh_spectrum(const double* eps, const int* core_idx, int n_core, const double* omega, int n_w,
                        const double* sigma, const double* dh, const double* sx, const double* vxc, double* a,
                        double* w_out, cudaStream_t s) {
  int n = n_core * n_w;
  gdh_spectrum_kernel<<<(n + 255) / 256, 256, 0, s>>>(eps, core_idx, n_core, omega, n_w, sigma, dh, sx, vxc, a, w_out);
  return cudaPeekAtLastError() == cudaSuccess ? 1 : -1;
}

// Graphical solutions of the plain G0W0 QP equation (Eq. quasiparticle_equation) on a grid:
// f(w) = eps_n + Sigma^x_n - v^xc_n + Re Sigma^c_n(w) - w; a grid point with f = 0 is a root; a sign
// change between j and j+1 gives the linear interpolant w* = w_j - f_j (w_{j+1} - w_j)/(f_{j+1} - f_j)
// with Z = 1/(1 - dRe Sigma/dw) from the slope over that interval. One block per core; lane 0 scans
// the grid in order so the roots come out ascending. n_roots = all roots found (only the first
// max_roots are stored).
__global__ void g0w0_scan_kernel(const double* __restrict__ omega, int n_w, const double* __restrict__ sigma,
                                 const double* __restrict__ eps, const int* __restrict__ core_idx,
                                 const double* __restrict__ sx, const double* __restrict__ vxc, int max_roots,
                                 double* __restrict__ roots, int* __restrict__ n_roots) {
  const int c = blockIdx.x;
  if (threadIdx.x != 0) return;
  const double* sg = sigma + (size_t)c * n_w * 2;
  const double base = eps[core_idx[c]] + sx[c] - vxc[c];
  double* out = roots + (size_t)c * max_roots * 2;
  int k = 0;
  for (int j = 0; j < n_w; ++j) {
    const double fj = base + sg[2 * j] - omega[j];
    double ws = 0.0, slope = 0.0;
    bool root = false;
    if (fj == 0.0) {
      const int a = j + 1 < n_w ? j : j - 1;
      slope = (sg[2 * (a + 1)] - sg[2 * a]) / (omega[a + 1] - omega[a]);
      ws = omega[j];
      root = n_w > 1;
    } else if (j + 1 < n_w) {
      const double fk = base + sg[2 * (j + 1)] - omega[j + 1];
      if (fj * fk < 0.0) {
        ws = omega[j] - fj * (omega[j + 1] - omega[j]) / (fk - fj);
        slope = (sg[2 * (j + 1)] - sg[2 * j]) / (omega[j + 1] - omega[j]);
        root = true;
      }
    }
    if (root) {
      if (k < max_roots) {
        out[2 * k] = ws;
        out[2 * k + 1] = 1.0 / (1.0 - slope);
      }
      ++k;
    }
  }
  n_roots[c] = k;
}

int launch_g0w0_scan(const double* omega, int n_w, const double* sigma, const double* eps, const int* core_idx,
                     const double* sx, const double* vxc, int n_core, int max_roots, double* roots, int* n_roots,
                     cudaStream_t s) {
  g0w0_scan_kernel<<<n_core, 32, 0, s>>>(omega, n_w, sigma, eps, core_idx, sx, vxc, max_roots, roots, n_roots);
  return cudaPeekAtLastError() == cudaSuccess ? 1 : -1;
}

int launch_qp_finish_hedin(const QpState* st, const double* eps, const int* core_idx, int n_core, double* eps_qp,
                           double* dh, int* iters, cudaStream_t s) {
  qp_finish_hedin_kernel<<<(n_core + 63) / 64, 64, 0, s>>>(st, eps, core_idx, n_core, eps_qp, dh, iters);
  return cudaPeekAtLastError() == cudaSuccess ? 1 : -1;
}

int launch_request_dec(const double* eps, const int* core_idx, int n_core, double eps_f, const double* omega_rel, int n_w,
                       const int* pair_of, const double* wpair, double* im, cudaStream_t s) {
  int n = n_core * n_w;
  request_dec_kernel<<<(n + 255) / 256, 256, 0, s>>>(eps, core_idx, n_core, eps_f, omega_rel, n_w, pair_of, wpair, im);
  return cudaPeekAtLastError() == cudaSuccess ? 1 : -1;
}

int launch_sigma_grid(const double* eps, int n_states, int n_core, const int* core_idx, const double* omega, int n_w,
                      double eps_f, const double* xi, const double* wxi, int n_im, const double* wim, const int* pidx,
                      const double* wres, int dec_mode, const int* group_of_core, double* sigma, double* im_dec,
                      cudaStream_t s) {
  long long warps = (long long)n_core * n_w;
  int blocks = (int)((warps * 32 + 255) / 256);
  sigma_grid_kernel<<<blocks, 256, 0, s>>>(eps, n_states, n_core, core_idx, omega, n_w, eps_f, xi, wxi, n_im, wim, pidx,
                                           wres, dec_mode, group_of_core, sigma, im_dec);
  return cudaPeekAtLastError() == cudaSuccess ? 1 : -1;
}

int launch_qp_init(const double* eps, const int* core_idx, int n_core, const int* mask, QpState* st, cudaStream_t s) {
  qp_init_kernel<<<(n_core + 63) / 64, 64, 0, s>>>(eps, core_idx, n_core, mask, st);
  return cudaPeekAtLastError() == cudaSuccess ? 1 : -1;
}

int launch_qp_pairs(const double* eps, const int* core_idx, int n_core, int n_occ, double eps_f, double eta,
                    const QpState* st, double* z, int* active, double* fac, int* all_done,
                    unsigned long long* active_count, cudaStream_t s) {
  int n = n_core * n_occ;
  qp_pairs_kernel<<<(n + 127) / 128, 128, 0, s>>>(eps, core_idx, n_core, n_occ, eps_f, eta, st, z, active, fac, all_done,
                                                  active_count);
  return cudaPeekAtLastError() == cudaSuccess ? 1 : -1;
}

int launch_qp_assemble_update(const double* eps, int n_states, int n_occ, int n_core, const int* core_idx, double eps_f,
                              const double* xi, const double* wxi, int n_im, const double* wim, const double* wpair,
                              const double* fac, const double* sx, const double* vxc, double tol, int max_iter,
                              int g0w0, QpState* st, int* all_done, cudaStream_t s) {
  qp_update_kernel<<<n_core, 32, 0, s>>>(eps, n_states, n_occ, n_core, core_idx, eps_f, xi, wxi, n_im, wim, wpair, fac,
                                         sx, vxc, tol, max_iter, g0w0, st, all_done);
  return cudaPeekAtLastError() == cudaSuccess ? 1 : -1;
}

int launch_qp_finish(const QpState* st, int n_core, double* eps_qp, double* dh, int* iters, unsigned* status,
                     cudaStream_t s) {
  qp_finish_kernel<<<(n_core + 63) / 64, 64, 0, s>>>(st, n_core, eps_qp, dh, iters, status);
  return cudaPeekAtLastError() == cudaSuccess ? 1 : -1;
}

}  // namespace gwc
