// Cumulant spectral function for callers that cannot allocate device memory.
//
// gwc_cumulant_spectrum needs a gwc_ctx, and creating one calls cudaMalloc. Some callers
// must not allocate at all: a serving thread that shares the GPU with another framework's
// caching allocator or runs under a fixed device-memory budget (a cudaMalloc/cudaFree there
// can synchronise the whole device, stalling other streams, or push the process over its
// budget), or a caller that holds no context and only has Im Sigma in hand. This file gives
// them one entry point that runs the same kernels with their scratch (the two FFT ping-pong
// buffers, the twiddle table and the cumulant coefficients) in one file-scope device array.
//
// The array is a static __device__ object: every GPU that loads this library holds it (about
// 10.5 MB) until the process exits. All calls share it and it keeps the last call's contents;
// every element a call reads is first written by that same call, so nothing is cleared. Calls
// that overlap on the GPU (different streams, or threads that do not serialise) race on it.
#include <cuda.h>

#include <mutex>
#include <utility>
#include <vector>

#include "gwc_internal.h"

namespace {

constexpr int kMaxWork = 1 << 18;     // n_core * n_t (complex entries per ping-pong buffer)
constexpr int kMaxTwiddle = 1 << 17;  // n_t / 2 (n_t <= 2^18)
constexpr int kMaxCoef = 1 << 16;     // n_core * n_omega (doubles)
constexpr int kScratch2 = 2 * kMaxWork + kMaxTwiddle + kMaxCoef / 2;  // in double2 units

static_assert(GWC_NOALLOC_MAX_WORK == kMaxWork, "header limit");
static_assert(GWC_NOALLOC_MAX_COEF == kMaxCoef, "header limit");

__device__ __align__(256) double2 g_noalloc_scratch[kScratch2];

typedef CUresult (*CtxGetCurrentFn)(CUcontext*);
typedef CUresult (*CtxGetIdFn)(CUcontext, unsigned long long*);

// Unique id of the context current on this thread (cuCtxGetId: never reused within the process, so
// a context created after a device reset gets a new id); false if the driver gives none.
bool current_context_id(unsigned long long* id) {
  static CtxGetCurrentFn get_current = nullptr;
  static CtxGetIdFn get_id = nullptr;
  static std::once_flag once;
  std::call_once(once, [] {
    void* f = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      get_current = reinterpret_cast<CtxGetCurrentFn>(f);
    f = nullptr;
    if (cudaGetDriverEntryPointByVersion("cuCtxGetId", &f, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      get_id = reinterpret_cast<CtxGetIdFn>(f);
  });
  CUcontext c = nullptr;
  if (!get_current || !get_id || get_current(&c) != CUDA_SUCCESS || !c) return false;
  return get_id(c, id) == CUDA_SUCCESS;
}

std::mutex g_addr_mutex;
std::vector<std::pair<unsigned long long, double2*>> g_addr;  // (context id, device address)

// Device address of the scratch array in the current device's context, looked up once per context
// (in host code the symbol itself is only a host-side stand-in, not a device address). Without a
// context id from the driver the address is looked up on every call.
gwc_status scratch_address(double2** out) {
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0) return GWC_ERR_CUDA;
  std::lock_guard<std::mutex> lock(g_addr_mutex);
  unsigned long long id = 0;
  bool have_id = current_context_id(&id);
  if (have_id)
    for (const auto& e : g_addr)
      if (e.first == id) {
        *out = e.second;
        return GWC_OK;
      }
  void* p = nullptr;
  if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || !p) return GWC_ERR_CUDA;
  if (!have_id) have_id = current_context_id(&id);  // the lookup made the primary context current
  if (have_id) g_addr.emplace_back(id, static_cast<double2*>(p));
  *out = static_cast<double2*>(p);
  return GWC_OK;
}

}  // namespace

extern "C" gwc_status gwc_cumulant_spectrum_noalloc(const double* omega_rel, int n_omega, const double* im_sigma,
                                                    int n_core, int n_t, double t_max, double eta, double* a_out,
                                                    double* nu_out, void* stream) {
  if (!omega_rel || !im_sigma || !a_out) {
    gwc::set_noctx_error("gwc_cumulant_spectrum_noalloc: omega_rel, im_sigma and a_out must be non-NULL");
    return GWC_ERR_INVALID_ARG;
  }
  if (n_core < 1 || n_omega < 1 || n_omega > 8192 || n_t < 16 || (n_t & (n_t - 1)) || !(t_max > 0.0) || !(eta > 0.0)) {
    gwc::set_noctx_error("gwc_cumulant_spectrum_noalloc: need n_core >= 1, 1 <= n_omega <= 8192, n_t a power of two >= 16, "
                         "t_max > 0, eta > 0");
    return GWC_ERR_INVALID_ARG;
  }
  if ((long long)n_core * n_t > kMaxWork || n_t / 2 > kMaxTwiddle || (long long)n_core * n_omega > kMaxCoef) {
    gwc::set_noctx_error("gwc_cumulant_spectrum_noalloc: size beyond the static scratch (n_core*n_t <= 2^18, "
                         "n_core*n_omega <= 2^16); use gwc_cumulant_spectrum with a context instead");
    return GWC_ERR_INVALID_ARG;
  }
  double2* base = nullptr;
  if (scratch_address(&base) != GWC_OK) {
    gwc::set_noctx_error("gwc_cumulant_spectrum_noalloc: cudaGetSymbolAddress of the scratch array failed");
    return GWC_ERR_CUDA;
  }
  double* work_a = reinterpret_cast<double*>(base);
  double* work_b = reinterpret_cast<double*>(base + kMaxWork);
  double* twiddle = reinterpret_cast<double*>(base + 2 * kMaxWork);
  double* coef = reinterpret_cast<double*>(base + 2 * kMaxWork + kMaxTwiddle);
  int n = gwc::launch_cumulant_spectrum(omega_rel, n_omega, im_sigma, n_core, n_t, t_max, eta, work_a, work_b, coef,
                                        twiddle, a_out, nu_out, static_cast<cudaStream_t>(stream));
  if (n < 0) {
    gwc::set_noctx_error(cudaGetErrorString(cudaGetLastError()));
    return GWC_ERR_CUDA;
  }
  return GWC_OK;
}
