// Kernels of restarted flexible GMRES (right preconditioned, classical Gram-Schmidt), FP64.
//
// The Krylov basis V is one allocation [m+1][ld]; step j orthogonalises w = A M v_j against
// v_0..v_j in two passes over HBM: one multi-dot pass (every block reads its rows of w and of
// all v_i once and produces j+1 partial sums), then one multi-AXPY pass that also forms the
// partial sums of ||w||^2.  The Hessenberg entries stay on the device until the host reads the
// finished column for its Givens rotation.
#include <cuda_runtime.h>

#include "common.cuh"

namespace chebmg {

namespace {

constexpr int kThreads = 256;
constexpr int kMaxV = 65;   // restart length + 1 supported by the register tiles below

__device__ __forceinline__ double wsum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  return v;
}

// part[i * nblk + blockIdx.x] = partial <V_i, w>, i = 0..nv-1
__global__ void __launch_bounds__(kThreads)
k_mdot_partial(int64_t n, int64_t ld, int nv, int nblk, const double* __restrict__ V, const double* __restrict__ w,
               double* __restrict__ part) {
  __shared__ double sh[kThreads / 32];
  for (int i = 0; i < nv; ++i) {
    const double* v = V + (int64_t)i * ld;
    double s = 0.0;
    for (int64_t g = blockIdx.x * (int64_t)kThreads + threadIdx.x; g < n; g += (int64_t)nblk * kThreads)
      s += v[g] * w[g];
    s = wsum(s);
    if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x < 32) {
      double t = threadIdx.x < kThreads / 32 ? sh[threadIdx.x] : 0.0;
      t = wsum(t);
      if (threadIdx.x == 0) part[(int64_t)i * nblk + blockIdx.x] = t;
    }
    __syncthreads();
  }
}

// h[i] = sum of part[i][*] (fixed order), one block per i
__global__ void __launch_bounds__(kThreads)
k_mdot_finish(int nblk, const double* __restrict__ part, double* __restrict__ h) {
  __shared__ double sh[kThreads / 32];
  double s = 0.0;
  for (int k = threadIdx.x; k < nblk; k += kThreads) s += part[(int64_t)blockIdx.x * nblk + k];
  s = wsum(s);
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x < 32) {
    double t = threadIdx.x < kThreads / 32 ? sh[threadIdx.x] : 0.0;
    t = wsum(t);
    if (threadIdx.x == 0) h[blockIdx.x] = t;
  }
}

// w -= sum_i h[i] V_i (sign = -1) or x += sum_i h[i] V_i (sign = +1); partial ||w||^2
__global__ void __launch_bounds__(kThreads)
k_maxpy(int64_t n, int64_t ld, int nv, int nblk, const double* __restrict__ V, const double* __restrict__ h,
        double sign, double* __restrict__ w, double* __restrict__ part) {
  __shared__ double sh_h[kMaxV];
  __shared__ double sh[kThreads / 32];
  for (int i = threadIdx.x; i < nv; i += kThreads) sh_h[i] = sign * h[i];
  __syncthreads();
  double s = 0.0;
  for (int64_t g = blockIdx.x * (int64_t)kThreads + threadIdx.x; g < n; g += (int64_t)nblk * kThreads) {
    double acc = w[g];
    for (int i = 0; i < nv; ++i) acc += sh_h[i] * V[(int64_t)i * ld + g];
    w[g] = acc;
    s += acc * acc;
  }
  if (part) {
    s = wsum(s);
    if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x < 32) {
      double t = threadIdx.x < kThreads / 32 ? sh[threadIdx.x] : 0.0;
      t = wsum(t);
      if (threadIdx.x == 0) part[blockIdx.x] = t;
    }
  }
}

// hn = sqrt(sum part); out = w / hn (0 if hn == 0)
__global__ void __launch_bounds__(kThreads)
k_norm_finish(int nblk, const double* __restrict__ part, double* __restrict__ hn) {
  __shared__ double sh[kThreads / 32];
  double s = 0.0;
  for (int k = threadIdx.x; k < nblk; k += kThreads) s += part[k];
  s = wsum(s);
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x < 32) {
    double t = threadIdx.x < kThreads / 32 ? sh[threadIdx.x] : 0.0;
    t = wsum(t);
    if (threadIdx.x == 0) *hn = sqrt(t);
  }
}

__global__ void __launch_bounds__(kThreads)
k_scale_by(int64_t n, const double* __restrict__ w, const double* __restrict__ hn, double* __restrict__ out) {
  const double d = *hn;
  const double inv = d > 0.0 ? 1.0 / d : 0.0;
  for (int64_t g = blockIdx.x * (int64_t)kThreads + threadIdx.x; g < n; g += (int64_t)gridDim.x * kThreads)
    out[g] = w[g] * inv;
}

int blocks(int64_t n) {
  int64_t b = (n + 4 * kThreads - 1) / (4 * kThreads);
  if (b < 1) b = 1;
  if (b > 1184) b = 1184;   // 152 SMs x 8
  return (int)b;
}

}  // namespace

int gmres_max_basis() { return kMaxV; }
int gmres_part_size(int64_t n) { return kMaxV * blocks(n); }

void gmres_mdot(int64_t n, int64_t ld, int nv, const double* V, const double* w, double* part, double* h,
                cudaStream_t s) {
  const int nb = blocks(n);
  k_mdot_partial<<<nb, kThreads, 0, s>>>(n, ld, nv, nb, V, w, part);
  k_mdot_finish<<<nv, kThreads, 0, s>>>(nb, part, h);
  g_launches.fetch_add(2, std::memory_order_relaxed);
}

void gmres_maxpy_norm(int64_t n, int64_t ld, int nv, const double* V, const double* h, double sign, double* w,
                      double* part, double* hn, double* wn, cudaStream_t s) {
  const int nb = blocks(n);
  k_maxpy<<<nb, kThreads, 0, s>>>(n, ld, nv, nb, V, h, sign, w, hn ? part : nullptr);
  g_launches.fetch_add(1, std::memory_order_relaxed);
  if (hn) {
    k_norm_finish<<<1, kThreads, 0, s>>>(nb, part, hn);
    g_launches.fetch_add(1, std::memory_order_relaxed);
    if (wn) {
      k_scale_by<<<nb, kThreads, 0, s>>>(n, w, hn, wn);
      g_launches.fetch_add(1, std::memory_order_relaxed);
    }
  }
}

void gmres_norm_scale(int64_t n, const double* w, double* part, double* hn, double* wn, cudaStream_t s) {
  // ||w|| and wn = w / ||w||: an AXPY with no vectors
  gmres_maxpy_norm(n, 0, 0, nullptr, nullptr, 0.0, const_cast<double*>(w), part, hn, wn, s);
}

}  // namespace chebmg
