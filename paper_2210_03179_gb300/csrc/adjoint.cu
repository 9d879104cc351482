// Kernels of the adjoint (transposed) smoothed V-cycle, FP64, batched (vector q at q * ld).
//
// Reverse mode through Algorithm 2 with weights beta_i and lambda = s * lambda_max:
//   forward  d_0 = (4 / (3 lambda)) S r_0,  x_i = x_{i-1} + beta_i d_{i-1},
//            r_i = r_{i-1} - A d_{i-1},      d_i = c1_i d_{i-1} + (c2_i / lambda) S r_i,
//   backward (xbar = adjoint of the smoother's output; delta = adjoint of d, rho of r)
//            beta_i-bar = <xbar, d_{i-1}>,  delta = beta_k xbar,
//            for i = k-1 .. 1:  rho += (c2_i / lambda) S delta,
//                               lambda-bar -= (c2_i / lambda^2) <delta, S r_i>,
//                               delta = beta_i xbar + c1_i delta - A rho,
//            rho += (4 / (3 lambda)) S delta,  lambda-bar -= (4 / (3 lambda^2)) <delta, S r_0>,
//            b-bar += rho,  x0-bar = xbar - A rho.
// A and S are symmetric, so the transposed products are A and S again.  The forward d_i and
// S r_i are recomputed per smoother call (not stored for the whole cycle).
#include <cuda_runtime.h>

#include "common.cuh"

namespace chebmg {

namespace {

constexpr int kThreads = 256;

inline unsigned blocks_for(int64_t n) {
  int64_t g = (n + kThreads - 1) / kThreads;
  if (g > 2048) g = 2048;
  return (unsigned)(g < 1 ? 1 : g);
}

#define ROWS_LOOP(n)                                                                                 \
  for (int64_t g = blockIdx.x * (int64_t)kThreads + threadIdx.x; g < (n); g += (int64_t)gridDim.x * kThreads)

// Dout = d, SRout = S r  (records one step of the forward recurrence)
__global__ void __launch_bounds__(kThreads)
k_record(int64_t n, int64_t ld, const double* __restrict__ d, const double* __restrict__ r,
         const double* __restrict__ S, double* __restrict__ Dout, double* __restrict__ SRout) {
  const int64_t o = (int64_t)blockIdx.y * ld;
  ROWS_LOOP(n) {
    Dout[o + g] = d[o + g];
    SRout[o + g] = S[g] * r[o + g];
  }
}

// rho += a S delta
__global__ void __launch_bounds__(kThreads)
k_adj_rho(int64_t n, int64_t ld, double a, const double* __restrict__ S, const double* __restrict__ delta,
          double* __restrict__ rho) {
  const int64_t o = (int64_t)blockIdx.y * ld;
  ROWS_LOOP(n) rho[o + g] += a * S[g] * delta[o + g];
}

// delta = beta xbar + c1 delta - y; y = 0
__global__ void __launch_bounds__(kThreads)
k_adj_delta(int64_t n, int64_t ld, double beta, double c1, const double* __restrict__ xbar,
            double* __restrict__ delta, double* __restrict__ y) {
  const int64_t o = (int64_t)blockIdx.y * ld;
  ROWS_LOOP(n) {
    delta[o + g] = beta * xbar[o + g] + c1 * delta[o + g] - y[o + g];
    y[o + g] = 0.0;
  }
}

// out = a x + b y  (out may alias x or y)
__global__ void __launch_bounds__(kThreads)
k_lincomb(int64_t n, int64_t ld, double a, const double* x, double b, const double* y, double* out) {
  const int64_t o = (int64_t)blockIdx.y * ld;
  ROWS_LOOP(n) out[o + g] = a * x[o + g] + (y ? b * y[o + g] : 0.0);
}

// out_q = coef[q] x_q
__global__ void __launch_bounds__(kThreads)
k_scale_rows(int64_t n, int64_t ld, const double* __restrict__ coef, const double* x, double* out) {
  const int64_t o = (int64_t)blockIdx.y * ld;
  const double c = coef[blockIdx.y];
  ROWS_LOOP(n) out[o + g] = c * x[o + g];
}

__device__ __forceinline__ double wsum(double v) {
#pragma unroll
  for (int s = 16; s > 0; s >>= 1) v += __shfl_down_sync(0xffffffffu, v, s);
  return v;
}

__device__ __forceinline__ double block_sum(double v) {
  __shared__ double sh[kThreads / 32];
  v = wsum(v);
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  if (l == 0) sh[w] = v;
  __syncthreads();
  double t = 0.0;
  if (w == 0) {
    t = l < kThreads / 32 ? sh[l] : 0.0;
    t = wsum(t);
  }
  return t;
}

// part[q * nblk + blockIdx.x] = partial sum of <a_q, b_q>
__global__ void __launch_bounds__(kThreads)
k_dot_partial(int64_t n, int64_t ld, int nblk, const double* __restrict__ a, const double* __restrict__ b,
              double* __restrict__ part) {
  const int64_t o = (int64_t)blockIdx.y * ld;
  double s = 0.0;
  for (int64_t g = blockIdx.x * (int64_t)kThreads + threadIdx.x; g < n; g += (int64_t)nblk * kThreads)
    s += a[o + g] * b[o + g];
  s = block_sum(s);
  if (threadIdx.x == 0) part[(int64_t)blockIdx.y * nblk + blockIdx.x] = s;
}

// acc[slot] += coef * (sum of all partials), fixed order
__global__ void __launch_bounds__(kThreads)
k_dot_accumulate(int64_t count, const double* __restrict__ part, double coef, double* __restrict__ acc, int slot) {
  double s = 0.0;
  for (int64_t k = threadIdx.x; k < count; k += kThreads) s += part[k];
  s = block_sum(s);
  if (threadIdx.x == 0) acc[slot] += coef * s;
}

// out[q] = sum of the partials of right-hand side q
__global__ void __launch_bounds__(kThreads)
k_dot_rows(int nblk, const double* __restrict__ part, double* __restrict__ out) {
  double s = 0.0;
  for (int k = threadIdx.x; k < nblk; k += kThreads) s += part[(int64_t)blockIdx.x * nblk + k];
  s = block_sum(s);
  if (threadIdx.x == 0) out[blockIdx.x] = s;
}

int dot_blocks(int64_t n) {
  int64_t b = (n + 4095) / 4096;
  if (b < 1) b = 1;
  if (b > 128) b = 128;
  return (int)b;
}

}  // namespace

void adj_record(int64_t n, int64_t ld, int nb, const double* d, const double* r, const double* S, double* Dout,
                double* SRout, cudaStream_t s) {
  k_record<<<dim3(blocks_for(n), nb), kThreads, 0, s>>>(n, ld, d, r, S, Dout, SRout);
  g_launches.fetch_add(1, std::memory_order_relaxed);
}

void adj_rho(int64_t n, int64_t ld, int nb, double a, const double* S, const double* delta, double* rho,
             cudaStream_t s) {
  k_adj_rho<<<dim3(blocks_for(n), nb), kThreads, 0, s>>>(n, ld, a, S, delta, rho);
  g_launches.fetch_add(1, std::memory_order_relaxed);
}

void adj_delta(int64_t n, int64_t ld, int nb, double beta, double c1, const double* xbar, double* delta, double* y,
               cudaStream_t s) {
  k_adj_delta<<<dim3(blocks_for(n), nb), kThreads, 0, s>>>(n, ld, beta, c1, xbar, delta, y);
  g_launches.fetch_add(1, std::memory_order_relaxed);
}

void lincomb(int64_t n, int64_t ld, int nb, double a, const double* x, double b, const double* y, double* out,
             cudaStream_t s) {
  k_lincomb<<<dim3(blocks_for(n), nb), kThreads, 0, s>>>(n, ld, a, x, b, y, out);
  g_launches.fetch_add(1, std::memory_order_relaxed);
}

void scale_rows(int64_t n, int64_t ld, int nb, const double* coef, const double* x, double* out, cudaStream_t s) {
  k_scale_rows<<<dim3(blocks_for(n), nb), kThreads, 0, s>>>(n, ld, coef, x, out);
  g_launches.fetch_add(1, std::memory_order_relaxed);
}

int adj_dot_scratch(int64_t n, int nb) { return dot_blocks(n) * nb; }

void dot_accumulate(int64_t n, int64_t ld, int nb, const double* a, const double* b, double coef, double* part,
                    double* acc, int slot, cudaStream_t s) {
  const int nblk = dot_blocks(n);
  k_dot_partial<<<dim3(nblk, nb), kThreads, 0, s>>>(n, ld, nblk, a, b, part);
  k_dot_accumulate<<<1, kThreads, 0, s>>>((int64_t)nblk * nb, part, coef, acc, slot);
  g_launches.fetch_add(2, std::memory_order_relaxed);
}

void dot_rows(int64_t n, int64_t ld, int nb, const double* a, const double* b, double* part, double* out,
              cudaStream_t s) {
  const int nblk = dot_blocks(n);
  k_dot_partial<<<dim3(nblk, nb), kThreads, 0, s>>>(n, ld, nblk, a, b, part);
  k_dot_rows<<<nb, kThreads, 0, s>>>(nblk, part, out);
  g_launches.fetch_add(2, std::memory_order_relaxed);
}

}  // namespace chebmg
