/*
 * gwc.h -- C ABI of libgwc: the real-frequency correlation self-energy of molecular
 * 1s core states by contour deformation on an RI basis, the quasiparticle fixed point
 * and the retarded-cumulant spectral function (GW+C), on one NVIDIA GB300 (sm_103a).
 *
 * Method: arXiv 2412.17132, "GW plus cumulant approach for predicting core-level
 * shake-up satellites in large molecules". Equation labels below are the paper's
 * LaTeX labels (the paper does not number its equations).
 *
 * Conventions for every entry point
 *   - Units: Hartree atomic units (energies in Ha, times in hbar/Ha).
 *   - Arrays are row-major, float64 unless stated. "DEVICE" pointers are CUDA device
 *     memory of the current device; "HOST" pointers are host memory (pinned or pageable).
 *   - Ownership: the library never frees caller memory. A gwc_ctx copies what it keeps
 *     resident (orbital energies, RI coefficients and their precision-split copies) and
 *     owns its workspace; gwc_destroy releases both.
 *   - Streams: `stream` is a cudaStream_t passed as void* (NULL = legacy default stream).
 *     Calls enqueue work on that stream and return without synchronising, except where a
 *     function says it synchronises.
 *   - Errors: every function returns a gwc_status; no exception or abort crosses the ABI.
 *     Invalid sizes and NULL pointers are rejected before any launch (GWC_ERR_INVALID_ARG).
 *     Device-side conditions (a zero pivot, an exhausted bounded wait, a QP that did not
 *     converge) are recorded in a device status word and reported by gwc_sync.
 *     gwc_last_error returns a message for the last failing call on that context.
 *   - Threading: a gwc_ctx is used by one host thread at a time.
 */
#ifndef GWC_H
#define GWC_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

#define GWC_ABI_VERSION 3

typedef enum {
  GWC_OK = 0,
  GWC_ERR_INVALID_ARG = 1,   /* bad size, NULL pointer, inconsistent options          */
  GWC_ERR_OOM = 2,           /* device or pinned host allocation failed               */
  GWC_ERR_CUDA = 3,          /* a CUDA runtime call or kernel launch failed           */
  GWC_ERR_SINGULAR = 4,      /* zero pivot in the dielectric factorisation            */
  GWC_ERR_NOT_CONVERGED = 5, /* QP secant iteration hit max_qp_iter                   */
  GWC_ERR_TIMEOUT = 6,       /* a bounded device-side wait gave up                    */
  GWC_ERR_UNSUPPORTED = 7    /* precision/feature not available on this device        */
} gwc_status;

/* Arithmetic of the polarizability build chi0 and of the dielectric factorisation.
 * All modes keep the self-energy assembly, the QP iteration and the cumulant in FP64.
 *   FP64       : chi0 FP64 (SIMT), factorisation and solves FP64        (plain FP64 path)
 *   FP32       : chi0 FP32 (SIMT), factorisation and solves FP32
 *   BF16       : chi0 on tcgen05 tensor cores, BF16 operands, FP32 accumulate; factor FP32
 *   BF16X3     : chi0 on tcgen05, split-BF16 operands (hi*hi + hi*lo + lo*hi), FP32
 *                accumulate; factor FP32-accurate (3xTF32 tensor-core updates)  (mixed path)
 *   BF16X3_F64 : chi0 as BF16X3, widened to FP64; factorisation of eps, the imaginary-axis solves
 *                and the residue contractions y_k^2/d_k in FP64 (SIMT)                           */
typedef enum {
  GWC_PREC_FP64 = 0,
  GWC_PREC_BF16 = 1,
  GWC_PREC_BF16X3 = 2,
  GWC_PREC_FP32 = 3,
  GWC_PREC_BF16X3_F64 = 4
} gwc_precision;

/* Form of Im Sigma handed to the cumulant (Sec. "Core-valence decoupling", Eqs.
 * sigma_spectral_decoupled, sigma_spectral_decoupled_symmetric, cd_sigma_imaginary_decoupled):
 *   NONE : full Im Sigma^c (all residue states m)
 *   DIAG : f_n Im W^c_nn(|eps_n - w| + i eta)
 *   GROUP: sum over the symmetry group of n of f_i Im W^c_ni(|eps_i - w| + i eta)          */
typedef enum { GWC_DECOUPLE_NONE = 0, GWC_DECOUPLE_DIAG = 1, GWC_DECOUPLE_GROUP = 2 } gwc_decouple;

typedef enum { GWC_MEM_DEVICE = 0, GWC_MEM_HOST = 1 } gwc_memory;

/* One molecule. Sizes: n_virt = n_states - n_occ, n_ov = n_occ * n_virt.
 * The RI coefficients are the symmetrised three-centre integrals O^P_mn (the Coulomb
 * metric already applied), so that (mn|kl) = sum_P O^P_mn O^P_kl.                          */
typedef struct {
  int n_states;          /* number of orbitals, >= 2                                          */
  int n_occ;             /* occupied orbitals are 0..n_occ-1, 1 <= n_occ < n_states            */
  int n_aux;             /* auxiliary (RI) basis size, >= 1                                    */
  int n_core;            /* number of core states whose self-energy is computed, >= 1          */
  const int* core_idx;   /* HOST [n_core]: orbital index of each state whose self-energy is
                            computed, each < n_states. gwc_qp_solve, gwc_sigma_core_wac and the
                            request mode need occupied (core) states, < n_occ; gwc_evgw0 needs
                            every state, core_idx = 0..n_states-1                              */
  const double* eps;     /* [n_states] orbital energies, ascending                            */
  const double* o_ov;    /* [n_aux][n_ov]: O^P_ia, column (i, a) = i * n_virt + (a - n_occ)    */
  const double* o_core;  /* [n_states][n_core][n_aux]: O^P_{m, core_idx[c]} for every m       */
  const double* vxc;     /* [n_core] <psi_n|v^xc|psi_n>, or NULL: v^xc_n := Sigma^x_n          */
  double eps_f;          /* Fermi level; NaN: midpoint of HOMO and LUMO                        */
  int memory;            /* gwc_memory: where eps, o_ov, o_core and vxc live                  */
} gwc_system;

typedef struct {
  double eta;            /* broadening (Ha) of residues and of the spectrum damping, > 0      */
  int n_im;              /* imaginary-axis Gauss-Legendre nodes, 1..1024                       */
  double xi0;            /* scale of the map xi = xi0 (1+x)/(1-x), > 0                         */
  int prec;              /* gwc_precision                                                      */
  int dec;               /* gwc_decouple, form of im_sigma_dec in gwc_sigma_core               */
  const int* group_of_core; /* HOST [n_core] group label per core (GROUP mode), or NULL       */
  int n_t;               /* cumulant time points, a power of two, 16..2^22                    */
  double t_max;          /* cumulant time window, > 0                                          */
  int max_qp_iter;       /* secant iterations, 2..200                                          */
  double qp_tol;         /* secant tolerance on the QP residual (Ha), > 0                     */
  int batch;             /* frequencies per internal batch (0: chosen from free memory)       */
  int profile;           /* nonzero: time the chi0, factorisation and solve kernels with CUDA
                            events on the launching stream (accumulated in gwc_stats)          */
  int qp_mode;           /* gwc_qp_mode: how gwc_qp_solve and the request step get eps^QP     */
  int wait_us;           /* bound of every device-side wait of the tensor-core kernels, in
                            microseconds (0: one second). A wait that runs out stops its
                            kernel's work on that tile or matrix, which drains the copies and
                            MMAs it issued, frees its tensor memory and records
                            GWC_ERR_TIMEOUT (reported by gwc_sync); the results of that call
                            are undefined, and the context stays usable. 0..60000000          */
  int chi0_ctas;         /* launch shape of the tensor-core polarizability build: 0 one CTA (or
                            CTA pair) per (tile, frequency group) item; > 0 at most that many
                            CTAs, each looping over the items (persistent). gwc_autotune may
                            change it */
  int chi0_tile;         /* tile shape of the tensor-core polarizability build: 0 256 x 128 tiles
                            on CTA pairs (tcgen05 cta_group::2), 1 128 x 128 tiles on one CTA
                            each (less padding of the triangle at small N_aux, a lower MMA rate
                            per SM). gwc_autotune may change it                                */
} gwc_options;

/* GWC_QP_SECANT: iterate the G_dH W0 QP equation (eq quasiparticle_equation with the shifted
 *   self-energy of eq hedin_sigma_spectral) by the secant method from eps_n;
 * GWC_QP_HEDIN: the GW+C QP energy of eq QPGWC, eps_n + dH_n, which is the exact fixed point of
 *   that equation (one self-energy evaluation per core instead of one per iterate);
 * GWC_QP_G0W0: the plain G0W0 QP equation (eq quasiparticle_equation, Sigma^c at eps itself), by
 *   the same secant from eps_n; for core levels it has several solutions (Sec. "Satellites in the
 *   G0W0 approximation") and the secant returns the one it reaches — gwc_g0w0_solutions lists all
 *   of them on a grid. dH is still returned. */
typedef enum { GWC_QP_SECANT = 0, GWC_QP_HEDIN = 1, GWC_QP_G0W0 = 2 } gwc_qp_mode;

typedef struct {
  long long chi0_builds;     /* polarizability builds launched (one per frequency)            */
  double chi0_flop;          /* algorithmic chi0 flop: lower triangle, N_aux(N_aux+1) N_ov per part */
  long long kernel_launches; /* library kernels launched since gwc_create / gwc_reset_stats     */
  long long factorizations;  /* dielectric factorisations launched                              */
  long long chi0_launches;   /* chi0 kernel launches (profile mode)                               */
  double chi0_ms;            /* summed device time of the chi0 kernels (profile mode)             */
  long long factor_launches; /* factorisation kernel launches (profile mode)                      */
  double factor_ms;          /* summed device time of the factorisation kernels (profile mode)    */
  double factor_flop;        /* algorithmic factorisation flop: n^3/3 multiply-adds x 2 (x4 complex) */
  long long solve_launches;  /* contraction (forward substitution) launches (profile mode)        */
  double solve_ms;           /* summed device time of the contraction kernels (profile mode)      */
} gwc_stats;

typedef struct gwc_ctx gwc_ctx;

/* Fills o with the defaults: eta 1e-3, n_im 32, xi0 1, BF16X3, DIAG, n_t 2^16, t_max 2000,
 * max_qp_iter 50, qp_tol 1e-7, batch 0, profile 0, qp_mode SECANT, wait_us 0 (one second), chi0_ctas 0. */
gwc_status gwc_default_options(gwc_options* o);

/* Device bytes a context of this shape allocates (resident copies + workspace + the
 * per-grid tables for n_omega real frequencies). Host-only; launches nothing. */
gwc_status gwc_workspace_bytes(const gwc_system* sys, const gwc_options* opt, int n_omega, size_t* bytes);

/* Creates a context on the current device: validates, allocates, copies the system
 * (host->device if memory == GWC_MEM_HOST), builds the resident precision copies of
 * O_ov (BF16 hi/lo and FP32), and computes the imaginary-axis grid. Enqueued on
 * `stream`; gwc_create synchronises that stream once before returning.
 * With core_idx, eps, o_ov and o_core all NULL the system gives sizes only: the context is
 * allocated with that capacity and holds no system until gwc_load (serving slots sized for the
 * largest request of a class); the other entry points return GWC_ERR_INVALID_ARG until then.
 * Kernel choice of the BF16 and BF16X3 modes (defaults, and the environment variables, read here,
 * that keep an earlier kernel for A/B comparisons):
 *   - chi0 on CTA pairs (tcgen05 cta_group::2, 256 x 128 tiles) unless gwc_options.chi0_tile = 1;
 *     GWC_CHI0_KERNEL=single sets chi0_tile = 1 (the one-CTA 128 x 128 kernel).
 *   - complex dielectric matrices factored per 64-column panel: one panel launch (one CTA per
 *     matrix) and one batched tcgen05 trailing update over all matrices (3xTF32, FP32-accurate),
 *     panels in pairs with a one-panel lookahead; GWC_FACTOR=tc keeps the one-CTA-per-matrix
 *     tensor-core kernel, GWC_FACTOR=simt the FP32 SIMT kernel.
 *   - imaginary-axis W table: real chi0 builds widened into complex storage, the same split
 *     factorisation, and the forward substitution of the 33-node table as tcgen05 3xTF32 GEMMs
 *     (explicit inverse of each 128-row diagonal block); GWC_WTABLE=simt keeps the SIMT solve. */
gwc_status gwc_create(gwc_ctx** ctx, const gwc_system* sys, const gwc_options* opt, void* stream);

/* Replaces the system of an existing context (serving slots): no device allocation. The new system
 * may be smaller than the one the context was created with, as long as every buffer sized by the
 * system fits the allocation made at creation (orbitals, cores, occupied-virtual pairs, RI sizes and
 * their products, the dielectric workspace); otherwise GWC_ERR_INVALID_ARG and the context keeps its
 * system. A change of sizes drops the request plan and the QP core selection. Synchronises `stream`. */
gwc_status gwc_load(gwc_ctx* ctx, const gwc_system* sys, void* stream);

/* RI polarizability (Sec. "Self-energy evaluation"; RI form of Ren et al. 2012, which the
 * paper's CD uses): Pi_PQ(z_f) = sum_ia O^P_ia D_ia(z_f) O^Q_ia,
 * D_ia(z) = 2[1/(z - Delta_ia) - 1/(z + Delta_ia)], Delta_ia = eps_a - eps_i.
 *   z   : DEVICE [F][2] (Re z, Im z); any complex z (Im z = 0 and Re z = Delta is a pole)
 *   chi0: DEVICE [F][n_aux][n_aux][2] (Re, Im), full symmetric matrix written
 * Computed with the context's precision (gwc_options.prec). 1 <= F <= 4096. */
gwc_status gwc_build_chi0(gwc_ctx* ctx, const double* z, int F, double* chi0, void* stream);

/* Screened interaction contractions W^c(z) = b^T (eps(z)^-1 - 1) b, eps = 1 - Pi(z), for
 * n_rhs vectors b per frequency (Eqs. cd_imaginary, cd_residue with W^c = W - v):
 *   z  : DEVICE [F][2]
 *   rhs: DEVICE [F][n_rhs][n_aux] real vectors b
 *   w  : DEVICE [F][n_rhs][2] (Re, Im)
 * eps(z) is factored without pivoting (LDL^T, complex symmetric); a zero pivot sets
 * GWC_ERR_SINGULAR (reported by gwc_sync) and leaves w undefined for that frequency.
 * 1 <= F <= 4096, 1 <= n_rhs <= 1<<20. */
gwc_status gwc_screen(gwc_ctx* ctx, const double* z, int F, const double* rhs, int n_rhs, double* w, void* stream);

/* G0W0 correlation self-energy of every core by contour deformation (Eq. cd_terms:
 * Sigma^c_n(w) = -I_n(w) + R_n(w); Eqs. cd_imaginary, cd_residue, cd_prefactors) on an
 * absolute real-frequency grid shared by all cores, plus the exchange Sigma^x_n (Eq. sigma_x,
 * occupied states) and, if requested, the decoupled Im Sigma (Eq. cd_sigma_imaginary_decoupled).
 *   omega       : HOST [n_omega] real frequencies (Ha), any order
 *   sigma_c     : DEVICE [n_core][n_omega][2] (Re, Im) of Sigma^c_n(omega_j)
 *   im_sigma_dec: DEVICE [n_core][n_omega] Im Sigma in the options' decoupling form, or NULL
 *   sigma_x     : DEVICE [n_core], or NULL
 * The G_dH W0 self-energy of Eq. hedin_sigma_spectral is Sigma^c_n(w - dH_n). */
gwc_status gwc_sigma_core(gwc_ctx* ctx, const double* omega, int n_omega, double* sigma_c, double* im_sigma_dec,
                          double* sigma_x, void* stream);

/* Orbital energies in G (the poles of the Green's function) for gwc_sigma_core: Eq. ev_sigma_spectral
 * (Sec. "GW for core-levels: beyond G0W0") replaces them by QP energies while W keeps the RPA
 * excitations of the input energies. The residue positions |eps~_m - w| + i eta, the occupations f_m
 * of Eq. cd_prefactors and the imaginary-axis kernel a_m = w - eps~_m use eps~; chi0 and W use the
 * input energies. Only gwc_sigma_core (and gwc_evgw0) see the replacement.
 *   eps_g: HOST [n_states], or NULL to return to the input energies
 *   eps_f: Fermi level of the replacement; NaN: midpoint of eps_g[n_occ-1] and eps_g[n_occ]
 * Occupied states must stay below eps_f and virtual ones above (GWC_ERR_INVALID_ARG otherwise).
 * Copies eps_g; synchronises `stream`. */
gwc_status gwc_set_g_energies(gwc_ctx* ctx, const double* eps_g, double eps_f, void* stream);

/* Eigenvalue-self-consistent evGW0 (Sec. "GW for core-levels: beyond G0W0", Eq. ev_sigma_spectral):
 * every state's QP energy is fed back into G while W keeps the RPA excitations of the input energies.
 * Needs every state as a core (n_core = n_states, core_idx = 0..n_states-1, o_core = O^P_mn for all
 * m, n). Iteration, all states at once from eps^(0) = eps:
 *   eps^(k+1)_n = eps_n + Sigma^x_n - v^xc_n + Re Sigma^c_n[G(eps^(k))](eps^(k)_n),
 * so the first step gives eps_n + dH_n (Eq. hedin_shift), with eps_F the midpoint of the current QP
 * HOMO and LUMO, until max_n |eps^(k+1)_n - eps^(k)_n| < tol (Ha). Each step is one gwc_sigma_core on
 * the grid of the current energies and one update kernel on the device.
 *   eps_qp: DEVICE [n_states] result; iters: HOST, steps taken
 * GWC_ERR_NOT_CONVERGED if max_iter (1..1000) steps do not reach tol; synchronises `stream`. */
gwc_status gwc_evgw0(gwc_ctx* ctx, double tol, int max_iter, double* eps_qp, int* iters, void* stream);

/* Hedin shift and G_dH W0 quasiparticle energies (Eqs. hedin_shift, quasiparticle_equation,
 * hedin_sigma_spectral, QPGWC): dH_n = Re Sigma^c_n(eps_n) + Sigma^x_n - v^xc_n, then
 * eps = eps_n + Sigma^x_n - v^xc_n + Re Sigma^c_n(eps - dH_n) solved by the secant method
 * from eps_n on the device (no host synchronisation inside).
 *   eps_qp, dh: DEVICE [n_core]; iters: DEVICE int [n_core] (Sigma evaluations used)
 * A core that does not converge in max_qp_iter keeps its last iterate and sets
 * GWC_ERR_NOT_CONVERGED (reported by gwc_sync). */
gwc_status gwc_qp_solve(gwc_ctx* ctx, double* eps_qp, double* dh, int* iters, void* stream);

/* Cores whose QP energies gwc_qp_solve and the request step compute: cores = HOST list of core indices
 * (0..n_core-1), n of them; NULL restores the default (every core). The other cores cost no dielectric
 * build and get NaN in eps_qp and dh and 0 iterations. Synchronises `stream`. */
gwc_status gwc_set_qp_cores(gwc_ctx* ctx, const int* cores, int n, void* stream);

/* Copies `bytes` of a result from device memory (src) to dst (host, pinned or pageable, or device),
 * enqueued on `stream` (an asynchronous copy for pinned host memory): the library's output path for
 * callers that hold results in device buffers and want them on the host through this interface. */
gwc_status gwc_copy_out(gwc_ctx* ctx, void* dst, const void* src, size_t bytes, void* stream);

/* Sigma^c of every core on an absolute grid by CD-WAC (Sec. "Self-energy evaluation", eq
 * pade_approximation): the imaginary-axis term as in gwc_sigma_core; W^c_mn for each occupied residue
 * state m and core n is a continued fraction (Thiele interpolation) through its values at the
 * imaginary-axis nodes, at i0 and at real reference points x_l + i eta: n_core_ref points uniform on
 * [0, 40 eV] and n_val_ref points uniform on [0.92 x_lo, 1.01 x_hi], x_lo/x_hi bounding |eps_m - w| over
 * the non-core occupied states with a residue on the grid (0/0: 100/100). One dielectric build per real
 * reference point replaces one per (w_j, m). Frequencies must lie below the LUMO (occupied residues).
 *   omega: HOST [n_omega]; sigma_c: DEVICE [n_core][n_omega][2]; im_sigma_dec: DEVICE [n_core][n_omega]
 *   (DIAG decoupled Im Sigma from the fitted W^c_nn) or NULL. Allocates scratch; synchronises `stream`. */
gwc_status gwc_sigma_core_wac(gwc_ctx* ctx, const double* omega, int n_omega, int n_core_ref, int n_val_ref,
                              double* sigma_c, double* im_sigma_dec, void* stream);


/* Graphical solutions of the plain G0W0 QP equation (eq quasiparticle_equation; Sec. "Satellites
 * in the G0W0 approximation": for 1s levels the equation has several solutions). On the ascending
 * grid omega, f(w) = eps_n + Sigma^x_n - v^xc_n + Re Sigma^c_n(w) - w; a grid point with f = 0 is a
 * root; where f changes sign between w_j and w_{j+1} the root is the linear interpolant, and each
 * root carries Z = 1/(1 - dRe Sigma^c/dw) from the slope over that interval. A crossing of a pole
 * of Re Sigma^c appears with Z < 0; the quasiparticle-like solutions have 0 < Z < 1.
 *   omega  : DEVICE [n_omega] ascending absolute frequencies (Ha)
 *   sigma_c: DEVICE [n_core][n_omega][2] (as gwc_sigma_core returns it on that grid)
 *   roots  : DEVICE [n_core][max_roots][2] = (w*, Z), ascending in w*
 *   n_roots: DEVICE [n_core] number of roots found (only the first max_roots are stored)
 * Asynchronous on `stream`; INVALID_ARG for n_omega < 2 or max_roots < 1. */
gwc_status gwc_g0w0_solutions(gwc_ctx* ctx, const double* omega, int n_omega, const double* sigma_c, int max_roots,
                              double* roots, int* n_roots, void* stream);

/* G_dH W0 spectral function beside GW+C (Sec. "G0W0 approximation": eqs gw_full_propagator,
 * A_definition, A_explicit_real_imaginary, with the shifted self-energy of eq hedin_sigma_spectral):
 * from Sigma^c_n(w') on a common grid w' (as gwc_sigma_core returns it) and the Hedin shifts,
 *   A_n(w) = (1/pi) |Im S| / ([w - eps_n + v^xc_n - Sigma^x_n - Re S]^2 + [Im S]^2),
 *   S = Sigma^c_n(w'), on the shifted grid w = w' + dH_n.
 *   omega  : DEVICE [n_omega] the common grid w'
 *   sigma_c: DEVICE [n_core][n_omega][2]; dh: DEVICE [n_core] (from gwc_qp_solve)
 *   a_out  : DEVICE [n_core][n_omega]; omega_out: DEVICE [n_core][n_omega] (w' + dH_n) or NULL */
gwc_status gwc_gdh_spectrum(gwc_ctx* ctx, const double* omega, int n_omega, const double* sigma_c, const double* dh,
                            double* a_out, double* omega_out, void* stream);

/* Retarded-cumulant spectral function (Sec. "Numerical GW+C scheme": Eqs.
 * landau_cumulant_truncated, cumulant_propagator_numerical_time,
 * cumulant_propagator_fourier, cumulant_propagator_convolution, eq:AGWC):
 *   beta_j = |Im Sigma_n(eps_n + w_j)| / pi,
 *   C~(t) = sum_j q_j beta_j / w_j^2 (e^{-i w_j t} - 1)   (trapezoid weights q_j; w_j = 0 skipped),
 *   A(eps^QP + nu) = (1/pi) Re int_0^{t_max} e^{i nu t - eta t} e^{C~(t)} dt,
 * discretised with t_k = k t_max/n_t (weight 1/2 at k = 0) and a batched FP64 FFT.
 *   omega_rel: DEVICE [n_core][n_omega] relative frequencies w_j = omega - eps_n, ascending
 *   im_sigma : DEVICE [n_core][n_omega] Im Sigma at those frequencies
 *   a_out    : DEVICE [n_core][n_t] A on the bins nu_j, ascending
 *   nu_out   : DEVICE [n_t] the bins nu_j = 2 pi j / t_max, j = -n_t/2 .. n_t/2-1, or NULL
 * The absolute frequency of bin j of core n is eps^QP_n + nu_j. */
gwc_status gwc_cumulant_spectrum(gwc_ctx* ctx, const double* omega_rel, int n_omega, const double* im_sigma,
                                 double* a_out, double* nu_out, void* stream);

/* Cumulant spectral function that allocates nothing (the paper has no counterpart: this is
 * a deployment variant of gwc_cumulant_spectrum with the same arithmetic and output layout).
 * For callers that cannot call cudaMalloc: a serving thread that shares the GPU with another
 * framework's caching allocator or works under a fixed device-memory budget, where an
 * allocation or free can synchronise the device or exceed the budget, or a caller without a
 * gwc_ctx. It needs no context; all sizes are arguments.
 *   omega_rel, im_sigma: DEVICE [n_core][n_omega]; a_out: DEVICE [n_core][n_t]; nu_out: DEVICE [n_t] or NULL
 * Scratch lives in one static device array of the library (about 10.5 MB, held on every GPU
 * that loads libgwc until the process exits); limits: n_core*n_t <= GWC_NOALLOC_MAX_WORK,
 * n_core*n_omega <= GWC_NOALLOC_MAX_COEF, n_t a power of two in 16..2^18, n_omega <= 8192.
 * Larger sizes return GWC_ERR_INVALID_ARG (message in gwc_last_error(NULL)) before any launch.
 * Set-up: the first call in a device's context looks up the array's device address
 * (cudaGetSymbolAddress) and keeps it for that context (a context created after a device reset
 * is looked up anew). With CUDA's lazy module loading that first call also loads the library's
 * module on the device, which is when the array takes its device memory, and a call with
 * n_omega > 3072 sets the cumulant kernel's shared-memory attribute. So make one warm-up call per
 * device, with the largest n_omega you will use, before any stream capture and before a memory
 * budget applies; later calls then allocate nothing. All calls share the array: calls that
 * overlap on the GPU (other streams, unsynchronised threads) race and must be serialised.
 * Every scratch element a call reads is written earlier in the same call, so stale contents
 * of a previous call never reach the output. */
#define GWC_NOALLOC_MAX_WORK (1 << 18)
#define GWC_NOALLOC_MAX_COEF (1 << 16)
gwc_status gwc_cumulant_spectrum_noalloc(const double* omega_rel, int n_omega, const double* im_sigma, int n_core,
                                         int n_t, double t_max, double eta, double* a_out, double* nu_out,
                                         void* stream);

/* ---- Request mode: one molecule's spectra + QP as one capturable step --------------------------
 * A "request" is the work a user of the serving and batched forms asks for: the decoupled Im Sigma
 * of every core on a relative grid omega_rel (eq cd_sigma_imaginary_decoupled; all cores share the
 * residue frequencies |omega_rel| + i eta, so one dielectric build serves every core), the QP energies
 * (Hedin shift and, with GWC_QP_SECANT, the secant iteration) and one cumulant spectrum per core.
 *
 * gwc_request_plan: HOST omega_rel [n_omega] (relative to each core's eps_n, ascending); builds the
 *   residue plan on the device and sizes the result buffers. Synchronises `stream`. Needs the DIAG
 *   decoupling mode.
 * gwc_request_step: enqueues the whole request (imaginary-axis W table, QP, residues, decoupled
 *   Im Sigma, spectra) on `stream` with no host synchronisation and no allocation; after one call
 *   outside stream capture it may be captured into a CUDA graph (gwc_batch_create does so).
 * gwc_request_results: device pointers to the context-owned results of the last step:
 *   eps_qp, dh [n_core], iters [n_core] (int), im_sigma [n_core][n_omega], a [n_core][n_t], nu [n_t]. */
typedef struct {
  const double* eps_qp;
  const double* dh;
  const int* iters;
  const double* im_sigma;
  const double* a;
  const double* nu;
  int n_core, n_omega, n_t;
} gwc_request_results;

gwc_status gwc_request_plan(gwc_ctx* ctx, const double* omega_rel, int n_omega, void* stream);
gwc_status gwc_request_step(gwc_ctx* ctx, void* stream);
gwc_status gwc_request_results_get(const gwc_ctx* ctx, gwc_request_results* out);
/* Copies the results of the last step into caller buffers (host or device; any may be NULL),
 * enqueued on `stream`: eps_qp, dh [n_core], iters [n_core] int, im_sigma [n_core][n_omega],
 * a [n_core][n_t], nu [n_t]. */
gwc_status gwc_request_copy_results(const gwc_ctx* ctx, double* eps_qp, double* dh, int* iters, double* im_sigma,
                                    double* a, double* nu, void* stream);

/* Launch and tile shapes chosen by timing one residue batch (chi0 build, factorisation and contraction of
 * that many frequencies) per candidate: frequencies per batch 16, 32, ... up to one SM wave, whole SM waves
 * and the capacity the context was created with; in the tensor-core modes each with both chi0 tile shapes
 * (256 x 128 on CTA pairs, 128 x 128 on one CTA) and both launch shapes (one CTA or pair per tile item, a
 * persistent launch of one per SM); the lowest time per frequency wins (cached per shape bucket and
 * precision for the process). Needs a request plan; synchronises `stream`; *chosen receives the batch now
 * used (the chi0 shapes are in the context's options, gwc_options.chi0_ctas and chi0_tile). */
gwc_status gwc_autotune(gwc_ctx* ctx, void* stream, int* chosen);

/* ---- Batched form: many molecules of uneven size in one CUDA-graph launch ----------------------
 * gwc_batch_create captures the request steps of the contexts (each with a request plan) into one CUDA
 * graph. Grouped form (every context in a tensor-core precision mode with the default factorisation,
 * GWC_QP_HEDIN, DIAG decoupling): the polarizability builds of each phase (W tables, QP residues, spectrum
 * residues, chunk by chunk) of ALL molecules go through one grouped chi0 launch and the complex
 * factorisations through one grouped LDL^T launch, with the small per-molecule kernels in between; two
 * grouped plans are candidates: whole-workspace chunks one after another with the persistent chi0 launch
 * (one CTA per SM, each looping over the (molecule, frequency batch, 128 x 128 tile) items), and
 * half-workspace chunks whose builds overlap the previous chunk's factorisations with one chi0 CTA per
 * item. Per-molecule
 * form: each context's step on its own forked stream. gwc_batch_create runs every candidate plan once
 * outside capture, timed (GWC_BATCH=per-molecule or =grouped in the environment restricts the choice),
 * captures the fastest on a private stream, and synchronises `stream` first. The contexts must outlive the batch and must not be used concurrently with a
 * launch of it. gwc_batch_launch replays the whole graph on `stream` (results in each context, see
 * gwc_request_results_get). */
typedef struct gwc_batch gwc_batch;
gwc_status gwc_batch_create(gwc_batch** out, gwc_ctx* const* ctxs, int n, void* stream);
gwc_status gwc_batch_launch(gwc_batch* batch, void* stream);
void gwc_batch_destroy(gwc_batch* batch);
/* 0: the batch is the graph of per-molecule steps; 1: grouped form, pipelined chunks with one CTA per chi0 work
 * item; 2: grouped form, chunks in sequence with the persistent chi0 launch (one CTA per SM looping over the
 * items). */
int gwc_batch_is_grouped(const gwc_batch* batch);
/* The times (ms) of the uncaptured runs gwc_batch_create chose from: [0] per-molecule steps, [1] grouped with
 * the persistent chi0 launch, [2] grouped pipelined with one CTA per chi0 item; -1 for a plan not tried. */
gwc_status gwc_batch_timings(const gwc_batch* batch, float* ms3);

/* The options the context runs with (as created, with what gwc_autotune chose; chi0_tile reads 1 when the
 * environment variable GWC_CHI0_KERNEL=single was set at creation). */
gwc_status gwc_get_options(const gwc_ctx* ctx, gwc_options* out);

/* Synchronises `stream` and reports the first device-side status raised since the
 * previous gwc_sync (then clears it). */
gwc_status gwc_sync(gwc_ctx* ctx, void* stream);

/* Counters since creation or the last reset. In profile mode the kernel times of work still in
 * flight are folded in by gwc_sync / gwc_get_stats (which then synchronise the device). */
gwc_status gwc_get_stats(gwc_ctx* ctx, gwc_stats* out);
gwc_status gwc_reset_stats(gwc_ctx* ctx);

/* Message of the last failing call on ctx (or of the last failing gwc_create when ctx is
 * NULL); valid until the next call on the same context from the same thread. */
const char* gwc_last_error(const gwc_ctx* ctx);
const char* gwc_status_string(gwc_status s);
int gwc_abi_version(void);

void gwc_destroy(gwc_ctx* ctx);

#ifdef __cplusplus
}
#endif

#endif /* GWC_H */
