// chebmg_fd_smooth_noalloc: a Chebyshev smoother on the 2-D five-point operator that
// needs no context and allocates no device memory.
//
// Who needs this: a caller that cannot call cudaMalloc at the point where it smooths --
// for example code embedded in a host application whose device memory is entirely owned
// by that application's own pool (extra allocations are forbidden or fail), or a
// latency-critical loop where cudaMalloc/cudaFree are not allowed because they can
// synchronise the whole device.  Such a caller passes only its own b and x.
//
// The smoother's work vectors (residual r, direction d, operator output y and the Jacobi
// scaling S) live in the file-scope device array below.  It is reserved once on every
// device that loads the library and held until the process exits.  Limits and sharing
// rules are stated next to the declaration in include/chebmg.h.
#include <cuda.h>
#include <cuda_runtime.h>

#include <mutex>

#include "../../include/chebmg.h"
#include "common.cuh"

namespace {

constexpr int64_t kNoAllocMaxN = int64_t(1) << 18;   // 262,144 unknowns, e.g. a 512 x 512 grid
constexpr int kNoAllocMaxDevices = 128;

// r | d | y | S, 4 x 262,144 doubles = 8 MiB on every device that loads the library.
static __device__ __align__(256) double g_noalloc_scratch[4 * kNoAllocMaxN];

// Device address of the array per device, with the id of the CUDA context it was looked up
// in.  A context id is unique for the life of the process, so after a device reset (which
// destroys the context and unloads this module) the next call sees a new id and looks the
// address up again instead of using a stale one.
struct ScratchSlot {
  unsigned long long ctx_id = 0;
  double* ptr = nullptr;
};
std::mutex g_noalloc_mu;
ScratchSlot g_noalloc_slot[kNoAllocMaxDevices];

using CtxGetCurrentFn = CUresult (*)(CUcontext*);
using CtxGetIdFn = CUresult (*)(CUcontext, unsigned long long*);

// Id of the current context through the driver entry points the runtime hands out (no link
// against the driver library needed); 0 if it cannot be had, which forces a fresh look-up.
unsigned long long current_context_id() {
  static CtxGetCurrentFn get_current = nullptr;
  static CtxGetIdFn get_id = nullptr;
  static bool resolved = false;
  if (!resolved) {
    void* f1 = nullptr;
    void* f2 = nullptr;
    cudaDriverEntryPointQueryResult q1, q2;
    if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f1, 12000, cudaEnableDefault, &q1) == cudaSuccess &&
        q1 == cudaDriverEntryPointSuccess &&
        cudaGetDriverEntryPointByVersion("cuCtxGetId", &f2, 12000, cudaEnableDefault, &q2) == cudaSuccess &&
        q2 == cudaDriverEntryPointSuccess) {
      get_current = reinterpret_cast<CtxGetCurrentFn>(f1);
      get_id = reinterpret_cast<CtxGetIdFn>(f2);
    }
    resolved = true;
  }
  if (!get_current || !get_id) return 0;
  CUcontext ctx = nullptr;
  unsigned long long id = 0;
  if (get_current(&ctx) != CUDA_SUCCESS || !ctx || get_id(ctx, &id) != CUDA_SUCCESS) return 0;
  return id;
}

// Device address of the scratch array on the current device: set up (cudaGetSymbolAddress,
// with the device current) on the first call per device and again whenever the device's
// context has changed since.  In host code the name g_noalloc_scratch is only a host-side
// stand-in: it is never passed to a kernel, only the address returned here is.
cudaError_t scratch_on_current_device(double** out) {
  int dev = -1;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= kNoAllocMaxDevices) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lock(g_noalloc_mu);
  ScratchSlot& slot = g_noalloc_slot[dev];
  const unsigned long long id = current_context_id();   // 0 while no context is current
  if (!slot.ptr || id == 0 || slot.ctx_id != id) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_noalloc_scratch);      // makes the device's context current
    if (e != cudaSuccess) return e;
    slot.ptr = static_cast<double*>(p);
    slot.ctx_id = current_context_id();
  }
  *out = slot.ptr;
  return cudaSuccess;
}

__global__ void k_fill(int64_t n, double v, double* __restrict__ out) {
  for (int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; g < n; g += (int64_t)gridDim.x * blockDim.x)
    out[g] = v;
}

int fail(int code, const char* msg) {
  chebmg::set_last_error(msg);
  return code;
}

}  // namespace

extern "C" int chebmg_fd_smooth_noalloc(int m, double Lx, double Ly, int kind, int order, double lmax,
                                        double lmin_ratio, const double* b, double* x, int x_is_zero,
                                        void* stream) {
  using namespace chebmg;
  if (m < 1 || !(Lx > 0.0) || !(Ly > 0.0)) return fail(CHEBMG_EINVAL, "fd_smooth_noalloc: bad grid");
  const int64_t n = (int64_t)m * m;
  if (n > kNoAllocMaxN)
    return fail(CHEBMG_EINVAL, "fd_smooth_noalloc: m*m exceeds the scratch limit of 262144 unknowns");
  if (kind != CHEBMG_CHEB_1ST && kind != CHEBMG_CHEB_4TH && kind != CHEBMG_CHEB_4TH_OPT)
    return fail(CHEBMG_EINVAL, "fd_smooth_noalloc: unknown smoother kind");
  if (order < 1 || (kind == CHEBMG_CHEB_4TH_OPT && order > 16))
    return fail(CHEBMG_EINVAL, "fd_smooth_noalloc: bad order");
  if (!(lmax > 0.0) || (kind == CHEBMG_CHEB_1ST && !(lmin_ratio > 0.0 && lmin_ratio < 1.0)))
    return fail(CHEBMG_EINVAL, "fd_smooth_noalloc: bad spectrum bounds");
  if (!b || !x) return fail(CHEBMG_EINVAL, "fd_smooth_noalloc: NULL vector");

  double* scratch = nullptr;
  cudaError_t e = scratch_on_current_device(&scratch);
  if (e != cudaSuccess) return fail(CHEBMG_ECUDA, cudaGetErrorString(e));
  double* r = scratch;
  double* d = scratch + kNoAllocMaxN;
  double* y = scratch + 2 * kNoAllocMaxN;
  double* S = scratch + 3 * kNoAllocMaxN;
  cudaStream_t s = static_cast<cudaStream_t>(stream);

  double st[9];
  fd_fine_stencil(Lx / (m + 1), Ly / (m + 1), st);
  Stencil9<double> A;
  for (int q = 0; q < 9; ++q) A.c[q] = st[q];

  // Every scratch entry that is read below is written first in this call (S here, y by the
  // operator, r and d by the init kernel), so the previous call's contents cannot leak in.
  k_fill<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(n, 1.0 / st[4], S);
  g_launches.fetch_add(1, std::memory_order_relaxed);
  if (!x_is_zero) fd_apply<double>(m, m, A, x, y, s);

  // The same smoother arithmetic as chebmg_smooth on level 0 of an FD context.
  if (kind == CHEBMG_CHEB_1ST) {
    const double lmin = lmin_ratio * lmax;
    const double theta = 0.5 * (lmax + lmin), delta = 0.5 * (lmax - lmin), sigma = theta / delta;
    double rho = 1.0 / sigma;
    cheb1_init<double>(n, b, x, r, d, y, S, 1.0 / theta, x_is_zero ? 1 : 0, s);
    for (int i = 1; i < order; ++i) {
      fd_apply<double>(m, m, A, d, y, s);
      const double rho_new = 1.0 / (2.0 * sigma - rho);
      cheb1_step<double>(n, x, r, d, y, S, rho_new * rho, 2.0 * rho_new / delta, s);
      rho = rho_new;
    }
    axpy<double>(n, 1.0, d, x, s);
  } else {
    const double* beta = kind == CHEBMG_CHEB_4TH_OPT ? beta_row(order) : nullptr;
    cheb4_init<double>(n, b, x, r, d, y, S, 4.0 / (3.0 * lmax), x_is_zero ? 1 : 0, s);
    for (int i = 1; i < order; ++i) {
      fd_apply<double>(m, m, A, d, y, s);
      cheb4_step<double>(n, x, r, d, y, S, beta ? beta[i - 1] : 1.0, (2.0 * i - 1.0) / (2.0 * i + 3.0),
                         (8.0 * i + 4.0) / ((2.0 * i + 3.0) * lmax), s);
    }
    axpy<double>(n, beta ? beta[order - 1] : 1.0, d, x, s);
  }
  e = cudaGetLastError();
  if (e != cudaSuccess) return fail(CHEBMG_ECUDA, cudaGetErrorString(e));
  return CHEBMG_OK;
}
