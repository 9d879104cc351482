// Chebyshev recurrences (Algorithms 1 and 2) and the vector updates of the smoother: the
// elementwise pass that follows each operator application.  Every kernel also takes a batch
// of right-hand sides (vector q at q * ld; per-node data such as S shared).
#include <cuda_runtime.h>

#include <cstdint>

#include "common.cuh"

namespace chebmg {

namespace {

inline unsigned grid_for(int64_t n, int bs) {
  int64_t g = (n + bs - 1) / bs;
  if (g > 4096 * 152) g = 4096 * 152;
  if (g < 1) g = 1;
  return (unsigned)g;
}

}  // namespace

// ===========================================================================
// Chebyshev recurrences and vector updates
// ===========================================================================
// Vector type of 16 bytes for T (float4 / double2) and its lane count.
template <typename T>
struct V16;
template <>
struct V16<float> {
  using type = float4;
  static constexpr int L = 4;
};
template <>
struct V16<double> {
  using type = double2;
  static constexpr int L = 2;
};

// 4th-kind init.  mode 2: d = c0 S b only; 1: x = 0, r = b, d = c0 S r; 0: r = b - y, y = 0,
// d = c0 S r.  VEC: 16-byte accesses over the aligned body, scalar tail.
template <typename T, bool VEC>
__global__ void k_cheb4_init(int64_t n, const T* __restrict__ b, T* __restrict__ x, T* __restrict__ r,
                             T* __restrict__ d, T* __restrict__ y, const T* __restrict__ invD, T c0,
                             int x_is_zero, int64_t ld) {
  pdl_wait();
  { const int64_t off_ = (int64_t)blockIdx.y * ld; b += off_; x += off_; r += off_; d += off_; y += off_; }
  using VT = typename V16<T>::type;
  constexpr int L = V16<T>::L;
  const int64_t tid = blockIdx.x * (int64_t)blockDim.x + threadIdx.x, stride = (int64_t)gridDim.x * blockDim.x;
  const int64_t nv = VEC ? n / L : 0;
  for (int64_t q = tid; q < nv; q += stride) {
    const VT bv = reinterpret_cast<const VT*>(b)[q], sv = reinterpret_cast<const VT*>(invD)[q];
    const T* bs = reinterpret_cast<const T*>(&bv);
    const T* ss = reinterpret_cast<const T*>(&sv);
    VT rv, dv;
    T* rs = reinterpret_cast<T*>(&rv);
    T* ds = reinterpret_cast<T*>(&dv);
    if (x_is_zero == 2) {   // x = 0 and r = b are left to the first step, which reads b
#pragma unroll
      for (int l = 0; l < L; ++l) ds[l] = c0 * ss[l] * bs[l];
      reinterpret_cast<VT*>(d)[q] = dv;
      continue;
    }
    if (x_is_zero) {
#pragma unroll
      for (int l = 0; l < L; ++l) rs[l] = bs[l];
      reinterpret_cast<VT*>(x)[q] = VT{};
    } else {
      const VT yv = reinterpret_cast<const VT*>(y)[q];
      const T* ys = reinterpret_cast<const T*>(&yv);
#pragma unroll
      for (int l = 0; l < L; ++l) rs[l] = bs[l] - ys[l];
      reinterpret_cast<VT*>(y)[q] = VT{};
    }
#pragma unroll
    for (int l = 0; l < L; ++l) ds[l] = c0 * ss[l] * rs[l];
    reinterpret_cast<VT*>(r)[q] = rv;
    reinterpret_cast<VT*>(d)[q] = dv;
  }
  for (int64_t g = nv * L + tid; g < n; g += stride) {
    T rv;
    if (x_is_zero == 2) {
      d[g] = c0 * invD[g] * b[g];
      continue;
    }
    if (x_is_zero) {
      rv = b[g];
      x[g] = T(0);
    } else {
      rv = b[g] - y[g];
      y[g] = T(0);
    }
    r[g] = rv;
    d[g] = c0 * invD[g] * rv;
  }
}


template <typename T, bool FIRST = false>
__device__ __forceinline__ void cheb4_one(T& x, T& r, T& d, T& y, T s, T beta, T c1, T c2, T beta_next) {
  const T dv = d;
  const T rv = r - y;
  if (FIRST) x = beta * dv;    // first step from x = 0 (r holds b)
  else x += beta * dv;
  r = rv;
  d = c1 * dv + c2 * s * rv;
  y = T(0);
  if (beta_next != T(0)) x += beta_next * d;   // last step: the final update x += beta_k d_k
}

// x += beta d; r -= y; d = c1 d + c2 S r; y = 0 -- 16-byte vector accesses over the aligned
// body (every pointer comes from a 256-byte aligned allocation), scalar tail.
// 16-byte global accesses with an L2 eviction hint.  The update streams x, r and S (evict
// first) and keeps d and y in L2 (evict last): the next operator application gathers d and
// accumulates into y, so they should still be there when it runs.
__device__ __forceinline__ uint64_t l2_policy_first() {
  uint64_t p;
  asm volatile("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(p));
  return p;
}
__device__ __forceinline__ uint64_t l2_policy_last() {
  uint64_t p;
  asm volatile("createpolicy.fractional.L2::evict_last.b64 %0, 1.0;" : "=l"(p));
  return p;
}
template <typename VT>
__device__ __forceinline__ VT ld16(const VT* p, uint64_t pol) {
  uint4 v;
  asm volatile("ld.global.L2::cache_hint.v4.u32 {%0, %1, %2, %3}, [%4], %5;"
               : "=r"(v.x), "=r"(v.y), "=r"(v.z), "=r"(v.w)
               : "l"(p), "l"(pol));
  return *reinterpret_cast<VT*>(&v);
}
template <typename VT>
__device__ __forceinline__ void st16(VT* p, const VT& val, uint64_t pol) {
  const uint4 v = *reinterpret_cast<const uint4*>(&val);
  asm volatile("st.global.L2::cache_hint.v4.u32 [%0], {%1, %2, %3, %4}, %5;" ::"l"(p), "r"(v.x), "r"(v.y), "r"(v.z),
               "r"(v.w), "l"(pol)
               : "memory");
}

// FIRST: the first step of a smoother application from x = 0, after an init that wrote only d:
// r is read from b (rin) and x is not read (x = beta d), so the init writes neither x nor r.
// (rin is r itself in the other steps, so neither is declared __restrict__.)
template <typename T, bool VEC, bool FIRST = false>
__global__ void k_cheb4_step(int64_t n, T* __restrict__ x, T* r, T* __restrict__ d,
                             T* __restrict__ y, const T* __restrict__ invD, T beta, T c1, T c2, T beta_next,
                             int64_t ld, const T* rin) {
  // Everything read here is the operator kernel's output or older: wait for that kernel before
  // the first load.  (Triggering the next kernel early as well, griddepcontrol.launch_dependents,
  // was measured slower: its waiting blocks cost this grid's last wave more than they saved.)
  pdl_wait();
  { const int64_t off_ = (int64_t)blockIdx.y * ld; x += off_; r += off_; d += off_; y += off_; rin += off_; }
  using VT = typename V16<T>::type;
  constexpr int L = V16<T>::L;
  const int64_t nv = VEC ? n / L : 0;
  const int64_t tid = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  const uint64_t first = l2_policy_first(), last = l2_policy_last();
  for (int64_t q = tid; q < nv; q += stride) {
    VT xv = {}, rv = ld16(reinterpret_cast<const VT*>(rin) + q, first);
    if (!FIRST) xv = ld16(reinterpret_cast<VT*>(x) + q, first);
    VT dv = ld16(reinterpret_cast<VT*>(d) + q, last), yv = ld16(reinterpret_cast<VT*>(y) + q, last);
    const VT sv = ld16(reinterpret_cast<const VT*>(invD) + q, first);
    T* xs = reinterpret_cast<T*>(&xv);
    T* rs = reinterpret_cast<T*>(&rv);
    T* ds = reinterpret_cast<T*>(&dv);
    T* ys = reinterpret_cast<T*>(&yv);
    const T* ss = reinterpret_cast<const T*>(&sv);
#pragma unroll
    for (int l = 0; l < L; ++l) cheb4_one<T, FIRST>(xs[l], rs[l], ds[l], ys[l], ss[l], beta, c1, c2, beta_next);
    st16(reinterpret_cast<VT*>(x) + q, xv, first);
    st16(reinterpret_cast<VT*>(r) + q, rv, first);
    st16(reinterpret_cast<VT*>(d) + q, dv, last);
    st16(reinterpret_cast<VT*>(y) + q, yv, last);
  }
  for (int64_t g = nv * L + tid; g < n; g += stride) {
    T xg = FIRST ? T(0) : x[g], rg = rin[g];
    cheb4_one<T, FIRST>(xg, rg, d[g], y[g], invD[g], beta, c1, c2, beta_next);
    x[g] = xg;
    r[g] = rg;
  }
}

template <typename T>
__global__ void k_cheb1_init(int64_t n, const T* __restrict__ b, T* __restrict__ x, T* __restrict__ r,
                             T* __restrict__ d, T* __restrict__ y, const T* __restrict__ invD,
                             T inv_theta, int x_is_zero, int64_t ld) {
  pdl_wait();
  { const int64_t off_ = (int64_t)blockIdx.y * ld; b += off_; x += off_; r += off_; d += off_; y += off_; }
  for (int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; g < n; g += (int64_t)gridDim.x * blockDim.x) {
    T rv;
    if (x_is_zero) {
      rv = invD[g] * b[g];
      x[g] = T(0);
    } else {
      rv = invD[g] * (b[g] - y[g]);
      y[g] = T(0);
    }
    r[g] = rv;
    d[g] = rv * inv_theta;
  }
}

template <typename T>
__global__ void k_cheb1_step(int64_t n, T* __restrict__ x, T* __restrict__ r, T* __restrict__ d,
                             T* __restrict__ y, const T* __restrict__ invD, T c1, T c2, int64_t ld) {
  pdl_wait();
  { const int64_t off_ = (int64_t)blockIdx.y * ld; x += off_; r += off_; d += off_; y += off_; }
  for (int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; g < n; g += (int64_t)gridDim.x * blockDim.x) {
    const T dv = d[g];
    const T rv = r[g] - invD[g] * y[g];
    x[g] += dv;
    r[g] = rv;
    d[g] = c1 * dv + c2 * rv;
    y[g] = T(0);
  }
}

template <typename T>
__global__ void k_axpy(int64_t n, T a, const T* __restrict__ d, T* __restrict__ x, int64_t ld) {
  pdl_wait();
  { const int64_t off_ = (int64_t)blockIdx.y * ld; d += off_; x += off_; }
  for (int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; g < n; g += (int64_t)gridDim.x * blockDim.x)
    x[g] += a * d[g];
}

template <typename T, bool VEC>
__global__ void k_residual(int64_t n, const T* __restrict__ b, T* __restrict__ y, T* __restrict__ r, int64_t ld) {
  pdl_wait();
  { const int64_t off_ = (int64_t)blockIdx.y * ld; b += off_; y += off_; r += off_; }
  using VT = typename V16<T>::type;
  constexpr int L = V16<T>::L;
  const int64_t tid = blockIdx.x * (int64_t)blockDim.x + threadIdx.x, stride = (int64_t)gridDim.x * blockDim.x;
  const int64_t nv = VEC ? n / L : 0;
  for (int64_t q = tid; q < nv; q += stride) {
    const VT bv = reinterpret_cast<const VT*>(b)[q], yv = reinterpret_cast<const VT*>(y)[q];
    const T* bs = reinterpret_cast<const T*>(&bv);
    const T* ys = reinterpret_cast<const T*>(&yv);
    VT rv;
    T* rs = reinterpret_cast<T*>(&rv);
#pragma unroll
    for (int l = 0; l < L; ++l) rs[l] = bs[l] - ys[l];
    reinterpret_cast<VT*>(r)[q] = rv;
    reinterpret_cast<VT*>(y)[q] = VT{};
  }
  for (int64_t g = nv * L + tid; g < n; g += stride) {
    r[g] = b[g] - y[g];
    y[g] = T(0);
  }
}


template <typename Tin, typename Tout>
__global__ void k_cast(int64_t n, const Tin* __restrict__ in, Tout* __restrict__ out, int64_t ldi, int64_t ldo) {
  pdl_wait();
  in += (int64_t)blockIdx.y * ldi;
  out += (int64_t)blockIdx.y * ldo;
  for (int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; g < n; g += (int64_t)gridDim.x * blockDim.x)
    out[g] = convert_to<Tout>(in[g]);
}

__global__ void k_masked_copy(int64_t n, const double* __restrict__ in, const double* __restrict__ invD,
                              double* __restrict__ out, int64_t ldi, int64_t ldo) {
  pdl_wait();
  in += (int64_t)blockIdx.y * ldi;
  out += (int64_t)blockIdx.y * ldo;
  for (int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; g < n; g += (int64_t)gridDim.x * blockDim.x)
    out[g] = invD[g] != 0.0 ? in[g] : 0.0;
}

constexpr int kVecThreads = 256;

template <typename T>
void cheb4_init(int64_t n, const T* b, T* x, T* r, T* d, T* y, const T* invD, double c0, int x_is_zero,
                cudaStream_t s, int nb, int64_t ld) {
  if (!ld) ld = n;
  const uintptr_t align = (uintptr_t)b | (uintptr_t)x | (uintptr_t)r | (uintptr_t)d | (uintptr_t)y | (uintptr_t)invD;
  if (align % 16 == 0 && (nb == 1 || (ld * sizeof(T)) % 16 == 0))
    launch_dep(k_cheb4_init<T, true>, dim3(grid_for(n / V16<T>::L + 1, kVecThreads), nb), dim3(kVecThreads), 0, s,
               n, b, x, r, d, y, invD, (T)c0, x_is_zero, ld);
  else
    launch_dep(k_cheb4_init<T, false>, dim3(grid_for(n, kVecThreads), nb), dim3(kVecThreads), 0, s, n, b, x, r, d,
               y, invD, (T)c0, x_is_zero, ld);
}
template <typename T, bool FIRST>
static void launch_cheb4_step(int64_t n, T* x, T* r, T* d, T* y, const T* invD, double beta, double c1, double c2,
                              cudaStream_t s, int nb, int64_t ld, double beta_next, const T* rin) {
  const uintptr_t align =
      (uintptr_t)x | (uintptr_t)r | (uintptr_t)d | (uintptr_t)y | (uintptr_t)invD | (uintptr_t)rin;
  if (align % 16 == 0 && (nb == 1 || (ld * sizeof(T)) % 16 == 0))
    launch_dep(k_cheb4_step<T, true, FIRST>, dim3(grid_for(n / V16<T>::L + 1, kVecThreads), nb), dim3(kVecThreads),
               0, s, n, x, r, d, y, invD, (T)beta, (T)c1, (T)c2, (T)beta_next, ld, rin);
  else
    launch_dep(k_cheb4_step<T, false, FIRST>, dim3(grid_for(n, kVecThreads), nb), dim3(kVecThreads), 0, s, n, x, r,
               d, y, invD, (T)beta, (T)c1, (T)c2, (T)beta_next, ld, rin);
}
template <typename T>
void cheb4_step(int64_t n, T* x, T* r, T* d, T* y, const T* invD, double beta, double c1, double c2,
                cudaStream_t s, int nb, int64_t ld, double beta_next, const T* b_first) {
  if (!ld) ld = n;
  if (b_first)
    launch_cheb4_step<T, true>(n, x, r, d, y, invD, beta, c1, c2, s, nb, ld, beta_next, b_first);
  else
    launch_cheb4_step<T, false>(n, x, r, d, y, invD, beta, c1, c2, s, nb, ld, beta_next, r);
}
template <typename T>
void cheb1_init(int64_t n, const T* b, T* x, T* r, T* d, T* y, const T* invD, double inv_theta,
                int x_is_zero, cudaStream_t s, int nb, int64_t ld) {
  launch_dep(k_cheb1_init<T>, dim3(grid_for(n, kVecThreads), nb), dim3(kVecThreads), 0, s, n, b, x, r, d, y, invD,
             (T)inv_theta, x_is_zero, ld ? ld : n);
}
template <typename T>
void cheb1_step(int64_t n, T* x, T* r, T* d, T* y, const T* invD, double c1, double c2, cudaStream_t s, int nb,
                int64_t ld) {
  launch_dep(k_cheb1_step<T>, dim3(grid_for(n, kVecThreads), nb), dim3(kVecThreads), 0, s, n, x, r, d, y, invD,
             (T)c1, (T)c2, ld ? ld : n);
}
template <typename T>
void axpy(int64_t n, double a, const T* d, T* x, cudaStream_t s, int nb, int64_t ld) {
  launch_dep(k_axpy<T>, dim3(grid_for(n, kVecThreads), nb), dim3(kVecThreads), 0, s, n, (T)a, d, x, ld ? ld : n);
}
template <typename T>
void residual(int64_t n, const T* b, T* y, T* r, cudaStream_t s, int nb, int64_t ld) {
  if (!ld) ld = n;
  const uintptr_t align = (uintptr_t)b | (uintptr_t)y | (uintptr_t)r;
  if (align % 16 == 0 && (nb == 1 || (ld * sizeof(T)) % 16 == 0))
    launch_dep(k_residual<T, true>, dim3(grid_for(n / V16<T>::L + 1, kVecThreads), nb), dim3(kVecThreads), 0, s, n,
               b, y, r, ld);
  else
    launch_dep(k_residual<T, false>, dim3(grid_for(n, kVecThreads), nb), dim3(kVecThreads), 0, s, n, b, y, r, ld);
}
template <typename Tin, typename Tout>
void cast(int64_t n, const Tin* in, Tout* out, cudaStream_t s, int nb, int64_t ldi, int64_t ldo) {
  launch_dep(k_cast<Tin, Tout>, dim3(grid_for(n, kVecThreads), nb), dim3(kVecThreads), 0, s, n, in, out,
             ldi ? ldi : n, ldo ? ldo : n);
}
void masked_copy(int64_t n, const double* in, const double* invD, double* out, cudaStream_t s, int nb, int64_t ldi,
                 int64_t ldo) {
  launch_dep(k_masked_copy, dim3(grid_for(n, kVecThreads), nb), dim3(kVecThreads), 0, s, n, in, invD, out,
             ldi ? ldi : n, ldo ? ldo : n);
}


#define CHEBMG_CHEB_INST(T)                                                                                 \
  template void cheb4_init<T>(int64_t, const T*, T*, T*, T*, T*, const T*, double, int, cudaStream_t, int,    \
                              int64_t);                                                                 \
  template void cheb4_step<T>(int64_t, T*, T*, T*, T*, const T*, double, double, double, cudaStream_t, int,   \
                              int64_t, double, const T*);                                               \
  template void cheb1_init<T>(int64_t, const T*, T*, T*, T*, T*, const T*, double, int, cudaStream_t, int,    \
                              int64_t);                                                                 \
  template void cheb1_step<T>(int64_t, T*, T*, T*, T*, const T*, double, double, cudaStream_t, int, int64_t); \
  template void axpy<T>(int64_t, double, const T*, T*, cudaStream_t, int, int64_t);                     \
  template void residual<T>(int64_t, const T*, T*, T*, cudaStream_t, int, int64_t);

CHEBMG_CHEB_INST(float)
CHEBMG_CHEB_INST(double)
template void cast<double, float>(int64_t, const double*, float*, cudaStream_t, int, int64_t, int64_t);
template void cast<float, double>(int64_t, const float*, double*, cudaStream_t, int, int64_t, int64_t);
template void cast<double, double>(int64_t, const double*, double*, cudaStream_t, int, int64_t, int64_t);
template void cast<float, float>(int64_t, const float*, float*, cudaStream_t, int, int64_t, int64_t);

}  // namespace chebmg
