// Batched Krylov kernels: the outer flexible CG (Polak-Ribiere) and the coarse-grid PCG run
// on nb right-hand sides at once, each with its own scalars (Sec. 1: a sequence of Poisson
// problems with the same operator, setup amortised over them).
//
// Layout: vector q of a batch starts at q * ld.  Per right-hand side the device keeps a row
// of FP64 scalars (the Slot enum) and four status words: active, iterations, status, spare.
// A right-hand side that has converged (or broken down) is frozen: its step length is zero,
// so x and r no longer change while the others iterate, and the iteration counts equal those
// of separate solves.  All decisions are taken on the device, so one Krylov iteration is a
// fixed sequence of launches that a CUDA graph can capture.
#include <cuda_runtime.h>

#include <cmath>

#include "common.cuh"

namespace chebmg {

namespace {

constexpr int kThreads = 256;

__device__ __forceinline__ double wsum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  return v;
}

// Sum of two values over a block of kThreads; result in thread 0.
__device__ __forceinline__ void bsum2(double& a, double& b) {
  __shared__ double sa[kThreads / 32], sb[kThreads / 32];
  a = wsum(a);
  b = wsum(b);
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  if (l == 0) {
    sa[w] = a;
    sb[w] = b;
  }
  __syncthreads();
  if (w == 0) {
    a = l < kThreads / 32 ? sa[l] : 0.0;
    b = l < kThreads / 32 ? sb[l] : 0.0;
    a = wsum(a);
    b = wsum(b);
  }
}

__device__ __forceinline__ bool finite(double v) { return v == v && fabs(v) <= 1.79769313486231570e308; }

// grid (nblk, nb): partial sums of (a0, b0) and (a1, b1) of right-hand side blockIdx.y
__global__ void __launch_bounds__(kThreads)
k_bdot2_partial(int64_t n, int64_t ld, int nblk, const double* __restrict__ a0, const double* __restrict__ b0,
                const double* __restrict__ a1, const double* __restrict__ b1, double* __restrict__ part, int vec) {
  const int64_t off = (int64_t)blockIdx.y * ld;
  double s0 = 0.0, s1 = 0.0;
  const int64_t tid = blockIdx.x * (int64_t)kThreads + threadIdx.x, stride = (int64_t)nblk * kThreads;
  const int64_t n2 = vec ? n / 2 : 0;   // 16-byte pairs over the aligned body
  for (int64_t g = tid; g < n2; g += stride) {
    const double2 x = reinterpret_cast<const double2*>(a0 + off)[g], y = reinterpret_cast<const double2*>(b0 + off)[g];
    s0 = fma(x.y, y.y, fma(x.x, y.x, s0));
    if (a1) {
      const double2 u = reinterpret_cast<const double2*>(a1 + off)[g], w = reinterpret_cast<const double2*>(b1 + off)[g];
      s1 = fma(u.y, w.y, fma(u.x, w.x, s1));
    }
  }
  for (int64_t g = 2 * n2 + tid; g < n; g += stride) {
    s0 += a0[off + g] * b0[off + g];
    if (a1) s1 += a1[off + g] * b1[off + g];
  }
  bsum2(s0, s1);
  if (threadIdx.x == 0) {
    part[(2 * (int64_t)blockIdx.y) * nblk + blockIdx.x] = s0;
    part[(2 * (int64_t)blockIdx.y + 1) * nblk + blockIdx.x] = s1;
  }
}

__device__ void bpost(int post, double s0, double s1, double* sc, int* st, double rtol) {
  switch (post) {
    case BPOST_INIT:   // s0 = (b, b)
      sc[S_BB] = s0;
      sc[S_RR] = s0;
      sc[S_T0] = rtol * rtol * s0;
      st[1] = 0;
      if (!finite(s0)) {
        st[0] = 0;
        st[2] = BS_BREAKDOWN;
      } else if (s0 == 0.0) {
        st[0] = 0;
        st[2] = BS_OK;
      } else {
        st[0] = 1;
        st[2] = BS_RUNNING;
      }
      break;
    case BPOST_SET_RZ:   // s0 = (z, r)
      sc[S_ZR] = s0;
      sc[S_RZ] = s0;
      break;
    case BPOST_ALPHA: {   // s0 = (p, A p)
      sc[S_PQ] = s0;
      double alpha = 0.0;
      if (st[0]) {
        if (s0 > 0.0 && finite(s0)) {
          alpha = sc[S_RZ] / s0;
        } else {
          st[0] = 0;
          st[2] = BS_BREAKDOWN;
          st[1] += 1;
        }
      }
      sc[S_ALPHA] = alpha;
      break;
    }
    case BPOST_CHECK:   // s0 = (r, r) after the update
      if (st[0]) {
        sc[S_RR] = s0;
        st[1] += 1;
        if (!finite(s0)) {
          st[0] = 0;
          st[2] = BS_BREAKDOWN;
        } else if (s0 <= sc[S_T0]) {
          st[0] = 0;
          st[2] = BS_OK;
        }
      }
      break;
    case BPOST_BETA_Q:   // s0 = (z, r_new), s1 = (z, A p): (z, r_new - r_old) = -alpha (z, A p)
      if (st[0]) {
        sc[S_ZR] = s0;
        sc[S_ZQ] = s1;
        sc[S_BETA] = -sc[S_ALPHA] * s1 / sc[S_RZ];
        sc[S_RZ] = s0;
      } else {
        sc[S_BETA] = 0.0;
      }
      break;
    default: break;
  }
}

// grid nb: fixed-order sum of the partials of right-hand side blockIdx.x, then the post-op
__global__ void __launch_bounds__(kThreads)
k_bdot2_finish(int nblk, int post, const double* __restrict__ part, double* __restrict__ scal,
               int* __restrict__ stat, double rtol) {
  const int64_t q = blockIdx.x;
  double s0 = 0.0, s1 = 0.0;
  for (int k = threadIdx.x; k < nblk; k += kThreads) {
    s0 += part[(2 * q) * nblk + k];
    s1 += part[(2 * q + 1) * nblk + k];
  }
  bsum2(s0, s1);
  if (threadIdx.x == 0) bpost(post, s0, s1, scal + q * S_NSLOTS, stat + q * 4, rtol);
}

// x += alpha p; r -= alpha q; r32 = FP32 copy of r (if given); partial (r, r)
__global__ void __launch_bounds__(kThreads)
k_bfcg_update_xr32(int64_t n, int64_t ld, int nblk, double* __restrict__ x, double* __restrict__ r,
                   float* __restrict__ r32, const double* __restrict__ p, const double* __restrict__ q,
                   double* __restrict__ part, const double* __restrict__ scal, int vec) {
  const int64_t off = (int64_t)blockIdx.y * ld;
  const double alpha = scal[blockIdx.y * S_NSLOTS + S_ALPHA];
  double s0 = 0.0, s1 = 0.0;
  const int64_t tid = blockIdx.x * (int64_t)kThreads + threadIdx.x, stride = (int64_t)nblk * kThreads;
  const int64_t n2 = vec ? n / 2 : 0;   // 16-byte pairs (8-byte for r32) over the aligned body
  x += off;
  r += off;
  p += off;
  q += off;
  if (r32) r32 += off;
  for (int64_t g = tid; g < n2; g += stride) {
    double2 xv = reinterpret_cast<double2*>(x)[g], rv = reinterpret_cast<double2*>(r)[g];
    const double2 pv = reinterpret_cast<const double2*>(p)[g], qv = reinterpret_cast<const double2*>(q)[g];
    xv.x += alpha * pv.x;
    xv.y += alpha * pv.y;
    rv.x = rv.x - alpha * qv.x;
    rv.y = rv.y - alpha * qv.y;
    reinterpret_cast<double2*>(x)[g] = xv;
    reinterpret_cast<double2*>(r)[g] = rv;
    if (r32) reinterpret_cast<float2*>(r32)[g] = make_float2(narrow_f64(rv.x), narrow_f64(rv.y));
    s0 += rv.x * rv.x;
    s0 += rv.y * rv.y;
  }
  for (int64_t g = 2 * n2 + tid; g < n; g += stride) {
    x[g] += alpha * p[g];
    const double rn = r[g] - alpha * q[g];
    r[g] = rn;
    if (r32) r32[g] = narrow_f64(rn);
    s0 += rn * rn;
  }
  bsum2(s0, s1);
  if (threadIdx.x == 0) {
    part[(2 * (int64_t)blockIdx.y) * nblk + blockIdx.x] = s0;
    part[(2 * (int64_t)blockIdx.y + 1) * nblk + blockIdx.x] = 0.0;
  }
}

template <typename Tz>
__global__ void __launch_bounds__(kThreads)
k_bdot_zr_zq(int64_t n, int64_t ld, int nblk, const Tz* __restrict__ z, const double* __restrict__ r,
             const double* __restrict__ q, double* __restrict__ part) {
  const int64_t off = (int64_t)blockIdx.y * ld;
  double s0 = 0.0, s1 = 0.0;
  for (int64_t g = off + blockIdx.x * (int64_t)kThreads + threadIdx.x; g < off + n; g += (int64_t)nblk * kThreads) {
    const double zv = to_f64(z[g]);
    s0 += zv * r[g];
    if (q) s1 += zv * q[g];
  }
  bsum2(s0, s1);
  if (threadIdx.x == 0) {
    part[(2 * (int64_t)blockIdx.y) * nblk + blockIdx.x] = s0;
    part[(2 * (int64_t)blockIdx.y + 1) * nblk + blockIdx.x] = s1;
  }
}

// p = z + beta p per right-hand side (p = z first), and q = 0 when q is given (the next product
// accumulates into it).  VEC: four entries per thread with 16-byte accesses, scalar tail.
template <typename Tz, bool VEC>
__global__ void __launch_bounds__(kThreads)
k_bupdate_p_from(int64_t n, int64_t ld, const Tz* __restrict__ z, double* __restrict__ p,
                 const double* __restrict__ scal, int first, double* __restrict__ q) {
  const int64_t off = (int64_t)blockIdx.y * ld;
  const double beta = first ? 0.0 : scal[blockIdx.y * S_NSLOTS + S_BETA];
  z += off;
  p += off;
  if (q) q += off;
  const int64_t tid = blockIdx.x * (int64_t)kThreads + threadIdx.x, stride = (int64_t)gridDim.x * kThreads;
  const int64_t nq = VEC ? n / 4 : 0;
  for (int64_t g = tid; g < nq; g += stride) {
    double zv[4];
    if constexpr (sizeof(Tz) == 4) {
      const float4 z4 = reinterpret_cast<const float4*>(z)[g];
      zv[0] = widen_f32(z4.x); zv[1] = widen_f32(z4.y); zv[2] = widen_f32(z4.z); zv[3] = widen_f32(z4.w);
    } else {
      const double2 a = reinterpret_cast<const double2*>(z)[2 * g], b = reinterpret_cast<const double2*>(z)[2 * g + 1];
      zv[0] = a.x; zv[1] = a.y; zv[2] = b.x; zv[3] = b.y;
    }
    double2* p2 = reinterpret_cast<double2*>(p) + 2 * g;
    if (first) {
      p2[0] = make_double2(zv[0], zv[1]);
      p2[1] = make_double2(zv[2], zv[3]);
    } else {
      const double2 a = p2[0], b = p2[1];
      p2[0] = make_double2(fma(beta, a.x, zv[0]), fma(beta, a.y, zv[1]));
      p2[1] = make_double2(fma(beta, b.x, zv[2]), fma(beta, b.y, zv[3]));
    }
    if (q) {
      double2* q2 = reinterpret_cast<double2*>(q) + 2 * g;
      q2[0] = make_double2(0.0, 0.0);
      q2[1] = make_double2(0.0, 0.0);
    }
  }
  for (int64_t g = nq * 4 + tid; g < n; g += stride) {
    p[g] = first ? to_f64(z[g]) : fma(beta, p[g], to_f64(z[g]));
    if (q) q[g] = 0.0;
  }
}

// ---------------------------------------------------------------------------
// Coarse PCG, one thread block per right-hand side.  The block keeps RPT rows per thread in
// registers (rows tid, tid + blockDim, ...), the vector of each product in shared memory, and
// reduces with warp shuffles; no grid-wide synchronisation, so any number of these blocks
// (and other kernels) may run side by side.  Same method as the cooperative coarse kernel:
// CG preconditioned by one degree-m application of Algorithm 2 (beta = 1) from a zero guess.
// ---------------------------------------------------------------------------
constexpr int kCBThreads = 512;
constexpr int kCBMaxRows = 6;   // rows per thread (registers)

// Sum of three values over the block; every thread gets the totals.
__device__ __forceinline__ void cb_sum3(double& a, double& b, double& c) {
  __shared__ double sh[3][kCBThreads / 32];
  __shared__ double res[3];
  a = wsum(a);
  b = wsum(b);
  c = wsum(c);
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  __syncthreads();   // previous readers of res are done
  if (l == 0) {
    sh[0][w] = a;
    sh[1][w] = b;
    sh[2][w] = c;
  }
  __syncthreads();
  if (w == 0) {
    double t0 = l < kCBThreads / 32 ? sh[0][l] : 0.0;
    double t1 = l < kCBThreads / 32 ? sh[1][l] : 0.0;
    double t2 = l < kCBThreads / 32 ? sh[2][l] : 0.0;
    t0 = wsum(t0);
    t1 = wsum(t1);
    t2 = wsum(t2);
    if (l == 0) {
      res[0] = t0;
      res[1] = t1;
      res[2] = t2;
    }
  }
  __syncthreads();
  a = res[0];
  b = res[1];
  c = res[2];
}

template <int NS, int RPT>
__device__ __forceinline__ void cb_spmv(const CoarseBlock& a, const double* sv, double (&y)[RPT]) {
  const int64_t n = a.n;
  const int ns = NS > 0 ? NS : a.nslot;
#pragma unroll
  for (int q = 0; q < RPT; ++q) {
    const int64_t g = threadIdx.x + (int64_t)q * kCBThreads;
    double acc = 0.0;
    if (g < n) {
      if (NS > 0) {
#pragma unroll
        for (int k = 0; k < (NS > 0 ? NS : 1); ++k) acc += __ldg(&a.val[k * n + g]) * sv[__ldg(&a.col[k * n + g])];
      } else {
        for (int k = 0; k < ns; ++k) acc += __ldg(&a.val[k * n + g]) * sv[__ldg(&a.col[k * n + g])];
      }
    }
    y[q] = acc;
  }
}

template <int NS, int RPT>
__device__ __forceinline__ void cb_spmv_f(const CoarseBlock& a, const float* sv, float (&y)[RPT]) {
  const int64_t n = a.n;
  const int ns = NS > 0 ? NS : a.nslot;
#pragma unroll
  for (int q = 0; q < RPT; ++q) {
    const int64_t g = threadIdx.x + (int64_t)q * kCBThreads;
    float acc = 0.f;
    if (g < n) {
      if (NS > 0) {
#pragma unroll
        for (int k = 0; k < (NS > 0 ? NS : 1); ++k) acc = fmaf(__ldg(&a.valf[k * n + g]), sv[__ldg(&a.col[k * n + g])], acc);
      } else {
        for (int k = 0; k < ns; ++k) acc = fmaf(__ldg(&a.valf[k * n + g]), sv[__ldg(&a.col[k * n + g])], acc);
      }
    }
    y[q] = acc;
  }
}

template <int NS, int RPT, bool PF32>
__global__ void __launch_bounds__(kCBThreads) k_coarse_block(CoarseBlock a) {
  extern __shared__ double sv[];   // [n]: the vector of the current product
  const int64_t n = a.n;
  const int64_t off = (int64_t)blockIdx.x * a.ld;
  const double* b = a.b + off;
  double* xo = a.x + off;
  double x[RPT], r[RPT], p[RPT], z[RPT], d[RPT], rp[RPT], y[RPT], ro[RPT];
  bool live[RPT];
  // S = invD is re-read (L1) where needed instead of taking RPT more registers
  auto Sv = [&](int q) { return live[q] ? __ldg(&a.invD[threadIdx.x + q * kCBThreads]) : 0.0; };
#pragma unroll
  for (int q = 0; q < RPT; ++q) {
    const int64_t g = threadIdx.x + (int64_t)q * kCBThreads;
    live[q] = g < n;
    r[q] = (live[q] && Sv(q) != 0.0) ? b[g] : 0.0;
    x[q] = p[q] = 0.0;
  }
  auto product = [&](const double (&v)[RPT]) {
    __syncthreads();   // earlier readers of sv are done
#pragma unroll
    for (int q = 0; q < RPT; ++q)
      if (live[q]) sv[threadIdx.x + q * kCBThreads] = v[q];
    __syncthreads();
    cb_spmv<NS, RPT>(a, sv, y);
  };
  const double c0 = 4.0 / (3.0 * a.lmax);
  __shared__ CoarseCoef coef;
  __shared__ double s_alpha, s_beta;
  coarse_coef_fill(coef, a.degree, a.lmax);
  __syncthreads();
  // the same polynomial on FP32 copies (the vector of each product in the same shared memory)
  auto precond_f = [&]() {
    float* svf = reinterpret_cast<float*>(sv);
    float df[RPT], rf[RPT], zf[RPT], yf[RPT];
    auto Sf = [&](int q) { return live[q] ? __ldg(&a.invDf[threadIdx.x + q * kCBThreads]) : 0.f; };
    const float c0f = (float)c0;
#pragma unroll
    for (int q = 0; q < RPT; ++q) {
      rf[q] = (float)r[q];
      df[q] = c0f * Sf(q) * rf[q];
      zf[q] = 0.f;
    }
    for (int i = 1; i < a.degree; ++i) {
#pragma unroll
      for (int q = 0; q < RPT; ++q) zf[q] += df[q];
      __syncthreads();
#pragma unroll
      for (int q = 0; q < RPT; ++q)
        if (live[q]) svf[threadIdx.x + q * kCBThreads] = df[q];
      __syncthreads();
      cb_spmv_f<NS, RPT>(a, svf, yf);
      const float c1 = coef.c1f[i], c2 = coef.c2f[i];
#pragma unroll
      for (int q = 0; q < RPT; ++q) {
        rf[q] -= yf[q];
        df[q] = c1 * df[q] + c2 * Sf(q) * rf[q];
      }
    }
#pragma unroll
    for (int q = 0; q < RPT; ++q) z[q] = (double)(zf[q] + df[q]);
  };
  auto precond = [&]() {
    if (PF32) {
      precond_f();
      return;
    }
#pragma unroll
    for (int q = 0; q < RPT; ++q) {
      rp[q] = r[q];
      d[q] = c0 * Sv(q) * rp[q];
      z[q] = 0.0;
    }
    for (int i = 1; i < a.degree; ++i) {
#pragma unroll
      for (int q = 0; q < RPT; ++q) z[q] += d[q];
      product(d);
      const double c1 = coef.c1[i], c2 = coef.c2[i];
#pragma unroll
      for (int q = 0; q < RPT; ++q) {
        rp[q] -= y[q];
        d[q] = c1 * d[q] + c2 * Sv(q) * rp[q];
      }
    }
#pragma unroll
    for (int q = 0; q < RPT; ++q) z[q] += d[q];
  };
  auto finish = [&](int status, int it) {
#pragma unroll
    for (int q = 0; q < RPT; ++q)
      if (live[q]) xo[threadIdx.x + q * kCBThreads] = x[q];
    if (threadIdx.x == 0) {
      a.stat[2 * blockIdx.x] = (unsigned)status;
      a.stat[2 * blockIdx.x + 1] = (unsigned)it;
      if (status == CS_BREAKDOWN) atomicMax((int*)a.sticky, (int)CS_BREAKDOWN);
    }
  };
  precond();
  double gam = 0.0, bb = 0.0, t = 0.0;
#pragma unroll
  for (int q = 0; q < RPT; ++q) {
    p[q] = z[q];
    gam += r[q] * z[q];
    bb += r[q] * r[q];
  }
  cb_sum3(gam, bb, t);
  if (!(bb > 0.0) || !(gam >= 0.0)) {
    finish(bb == 0.0 ? CS_OK : CS_BREAKDOWN, 0);
    return;
  }
  const double tol2 = a.rtol * a.rtol * bb;
  for (int it = 1; it <= a.maxit; ++it) {
    product(p);
    double pq = 0.0, u1 = 0.0, u2 = 0.0;
#pragma unroll
    for (int q = 0; q < RPT; ++q) pq += p[q] * y[q];
    cb_sum3(pq, u1, u2);
    if (!(pq > 0.0)) {
      finish(CS_BREAKDOWN, it);
      return;
    }
    const double alpha = block_div(&s_alpha, gam, pq);
#pragma unroll
    for (int q = 0; q < RPT; ++q) {
      ro[q] = r[q];
      x[q] = fma(alpha, p[q], x[q]);
      r[q] = fma(-alpha, y[q], r[q]);
    }
    precond();
    double gnew = 0.0, rr = 0.0;
    u1 = 0.0;
#pragma unroll
    for (int q = 0; q < RPT; ++q) {
      gnew += r[q] * z[q];
      rr += r[q] * r[q];
      if (PF32) u1 += ro[q] * z[q];
    }
    cb_sum3(gnew, rr, u1);
    if (!(rr == rr)) {
      finish(CS_BREAKDOWN, it);
      return;
    }
    if (rr <= tol2) {
      finish(CS_OK, it);
      return;
    }
    const double beta = block_div(&s_beta, PF32 ? gnew - u1 : gnew, gam);   // flexible beta for FP32
    gam = gnew;
#pragma unroll
    for (int q = 0; q < RPT; ++q) p[q] = fma(beta, p[q], z[q]);
  }
  finish(CS_NOTCONV, a.maxit);
}

template <int NS, bool PF32>
const void* cb_kernel(int rpt) {
  switch (rpt) {
    case 1: return (const void*)k_coarse_block<NS, 1, PF32>;
    case 2: return (const void*)k_coarse_block<NS, 2, PF32>;
    case 3: return (const void*)k_coarse_block<NS, 3, PF32>;
    case 4: return (const void*)k_coarse_block<NS, 4, PF32>;
    default: return (const void*)k_coarse_block<NS, 6, PF32>;
  }
}

}  // namespace

int bred_blocks(int64_t n) {
  int64_t b = (n + 4095) / 4096;
  if (b < 1) b = 1;
  if (b > 256) b = 256;
  return (int)b;
}

void bdot2(int64_t n, int64_t ld, int nb, const double* a0, const double* b0, const double* a1, const double* b1,
           int post, double rtol, double* part, double* scal, int* stat, cudaStream_t s) {
  const int nblk = bred_blocks(n);
  const int vec = ((uintptr_t)a0 | (uintptr_t)b0 | (uintptr_t)a1 | (uintptr_t)b1) % 16 == 0 && ld % 2 == 0;
  k_bdot2_partial<<<dim3(nblk, nb), kThreads, 0, s>>>(n, ld, nblk, a0, b0, a1, b1, part, vec);
  k_bdot2_finish<<<nb, kThreads, 0, s>>>(nblk, post, part, scal, stat, rtol);
  g_launches.fetch_add(2, std::memory_order_relaxed);
}

void bfcg_update_xr32(int64_t n, int64_t ld, int nb, double* x, double* r, float* r32, const double* p,
                      const double* q, double* part, double* scal, int* stat, cudaStream_t s) {
  const int nblk = bred_blocks(n);
  const int vec = ((uintptr_t)x | (uintptr_t)r | (uintptr_t)p | (uintptr_t)q) % 16 == 0 && (uintptr_t)r32 % 8 == 0 &&
                  ld % 2 == 0;
  k_bfcg_update_xr32<<<dim3(nblk, nb), kThreads, 0, s>>>(n, ld, nblk, x, r, r32, p, q, part, scal, vec);
  k_bdot2_finish<<<nb, kThreads, 0, s>>>(nblk, BPOST_CHECK, part, scal, stat, 0.0);
  g_launches.fetch_add(2, std::memory_order_relaxed);
}

template <typename Tz>
void bdot_zr_zq(int64_t n, int64_t ld, int nb, const Tz* z, const double* r, const double* q, int post,
                double* part, double* scal, int* stat, cudaStream_t s) {
  const int nblk = bred_blocks(n);
  k_bdot_zr_zq<Tz><<<dim3(nblk, nb), kThreads, 0, s>>>(n, ld, nblk, z, r, q, part);
  k_bdot2_finish<<<nb, kThreads, 0, s>>>(nblk, post, part, scal, stat, 0.0);
  g_launches.fetch_add(2, std::memory_order_relaxed);
}
template void bdot_zr_zq<float>(int64_t, int64_t, int, const float*, const double*, const double*, int, double*,
                                double*, int*, cudaStream_t);
template void bdot_zr_zq<double>(int64_t, int64_t, int, const double*, const double*, const double*, int, double*,
                                 double*, int*, cudaStream_t);

template <typename Tz>
void bupdate_p_from(int64_t n, int64_t ld, int nb, const Tz* z, double* p, const double* scal, bool first,
                    cudaStream_t s, double* q) {
  const bool vec = ((uintptr_t)z | (uintptr_t)p | (uintptr_t)q) % 16 == 0 && (ld * sizeof(Tz)) % 16 == 0 &&
                   (ld * sizeof(double)) % 16 == 0;
  int64_t g = ((vec ? n / 4 + 1 : n) + kThreads - 1) / kThreads;
  if (g > 1024) g = 1024;
  if (vec)
    k_bupdate_p_from<Tz, true><<<dim3((unsigned)g, nb), kThreads, 0, s>>>(n, ld, z, p, scal, first ? 1 : 0, q);
  else
    k_bupdate_p_from<Tz, false><<<dim3((unsigned)g, nb), kThreads, 0, s>>>(n, ld, z, p, scal, first ? 1 : 0, q);
  g_launches.fetch_add(1, std::memory_order_relaxed);
}
template void bupdate_p_from<float>(int64_t, int64_t, int, const float*, double*, const double*, bool, cudaStream_t,
                                    double*);
template void bupdate_p_from<double>(int64_t, int64_t, int, const double*, double*, const double*, bool,
                                     cudaStream_t, double*);

bool coarse_block_supported(int64_t n) { return n >= 1 && n <= (int64_t)kCBThreads * kCBMaxRows; }

bool coarse_block_launch(const CoarseBlock& a, int nb, cudaStream_t s) {
  if (!coarse_block_supported(a.n) || nb < 1) return false;
  int rpt = (int)((a.n + kCBThreads - 1) / kCBThreads);
  if (rpt > 4) rpt = 6;
  const void* fn = a.pf32 ? (a.nslot == 27 ? cb_kernel<27, true>(rpt) : cb_kernel<0, true>(rpt))
                         : (a.nslot == 27 ? cb_kernel<27, false>(rpt) : cb_kernel<0, false>(rpt));
  const size_t smem = sizeof(double) * (size_t)a.n;
  if (smem > 48 * 1024) {
    if (cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess)
      return false;
  }
  CoarseBlock arg = a;
  void* params[] = {&arg};
  const cudaError_t e = cudaLaunchKernel(fn, dim3(nb), dim3(kCBThreads), params, smem, s);
  g_launches.fetch_add(1, std::memory_order_relaxed);
  return e == cudaSuccess;
}

}  // namespace chebmg
