// CUDA kernels of the Jacobi-Chebyshev multigrid hot path (sm_103a).
//
// SEM operator (Sec. 1, Eq. 1.3): per element w_m = sum_n G_mn (Dhat_n u),
// y_e = sum_m Dhat_m^T w_m, then direct-stiffness summation into the global
// vector by atomics, skipping Dirichlet nodes.  p-multigrid transfers
// (Sec. 4.1) apply J x J x J per element.  FD (Sec. 3): a constant 3x3
// stencil per level (five-point on the finest, Galerkin nine-point below).
// Chebyshev recurrences: Algorithms 1 and 2 split into an operator pass and
// an elementwise pass (the elementwise kernels are in chebyshev.cu).
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>

#include "common.cuh"

namespace chebmg {

std::atomic<int64_t> g_launches{0};
thread_local bool g_pdl = false;

namespace {

inline unsigned grid_for(int64_t n, int bs) {
  int64_t g = (n + bs - 1) / bs;
  if (g > 4096 * 152) g = 4096 * 152;
  if (g < 1) g = 1;
  return (unsigned)g;
}

inline void count() { g_launches.fetch_add(1, std::memory_order_relaxed); }

constexpr int kVecThreads = 256;

}  // namespace

// ===========================================================================
// SEM element operator
// ===========================================================================
template <int Q>
struct SemShape {
  static constexpr int NP = Q * Q * Q;
  static constexpr int EPB = NP >= 512 ? 1 : 512 / NP;   // elements per block
  static constexpr int THREADS = EPB * NP;
};

template <typename T, int Q>
__global__ void __launch_bounds__(SemShape<Q>::THREADS)
k_sem_ax(int64_t E, const uint32_t* __restrict__ gid, const T* __restrict__ G,
         const T* __restrict__ Dg, const T* __restrict__ u, T* __restrict__ y, int64_t ld) {
  constexpr int NP = SemShape<Q>::NP;
  u += (int64_t)blockIdx.y * ld;   // right-hand side of a batch
  y += (int64_t)blockIdx.y * ld;
  constexpr int EPB = SemShape<Q>::EPB;
  __shared__ T sD[Q * Q];
  __shared__ T s_u[EPB * NP];
  __shared__ T s_r[EPB * NP];
  __shared__ T s_s[EPB * NP];
  __shared__ T s_t[EPB * NP];
  const int tid = threadIdx.x;
  const int le = tid / NP;
  const int p = tid - le * NP;
  const int i = p % Q, j = (p / Q) % Q, k = p / (Q * Q);
  const int64_t e = (int64_t)blockIdx.x * EPB + le;
  if (tid < Q * Q) sD[tid] = Dg[tid];
  const bool valid = e < E;
  // the geometric factors do not depend on the gather: their loads go out first, in flight
  // with the id and value loads instead of after them
  T g00 = 0, g01 = 0, g02 = 0, g11 = 0, g12 = 0, g22 = 0;
  if (valid) {
    const T* Ge = G + (size_t)e * 6 * NP + p;
    g00 = Ge[0];
    g01 = Ge[NP];
    g02 = Ge[2 * NP];
    g11 = Ge[3 * NP];
    g12 = Ge[4 * NP];
    g22 = Ge[5 * NP];
  }
  const uint32_t id = valid ? gid[e * NP + p] : kGidDirichlet;
  pdl_wait();   // u and y may come from the kernel before (programmatic dependent launch)
  T* su = s_u + le * NP;
  su[p] = (id & kGidDirichlet) ? T(0) : u[id & kGidMask];
  __syncthreads();
  T ur = 0, us = 0, ut = 0;
#pragma unroll
  for (int l = 0; l < Q; ++l) {
    ur += sD[i * Q + l] * su[(k * Q + j) * Q + l];
    us += sD[j * Q + l] * su[(k * Q + l) * Q + i];
    ut += sD[k * Q + l] * su[(l * Q + j) * Q + i];
  }
  T wr = 0, ws = 0, wt = 0;
  if (valid) {
    wr = g00 * ur + g01 * us + g02 * ut;
    ws = g01 * ur + g11 * us + g12 * ut;
    wt = g02 * ur + g12 * us + g22 * ut;
  }
  T* sr = s_r + le * NP;
  T* ss = s_s + le * NP;
  T* st = s_t + le * NP;
  sr[p] = wr;
  ss[p] = ws;
  st[p] = wt;
  __syncthreads();
  T acc = 0;
#pragma unroll
  for (int l = 0; l < Q; ++l) {
    acc += sD[l * Q + i] * sr[(k * Q + j) * Q + l];
    acc += sD[l * Q + j] * ss[(k * Q + l) * Q + i];
    acc += sD[l * Q + k] * st[(l * Q + j) * Q + i];
  }
  if (valid && !(id & kGidDirichlet)) atomicAdd(&y[id & kGidMask], acc);
}

template <typename T, int Q>
static void launch_sem_ax(int64_t E, const uint32_t* gid, const T* G, const T* D, const T* u, T* y,
                          cudaStream_t s, int nb, int64_t ld) {
  using S = SemShape<Q>;
  const unsigned blocks = (unsigned)((E + S::EPB - 1) / S::EPB);
  launch_dep(k_sem_ax<T, Q>, dim3(blocks, nb), dim3(S::THREADS), 0, s, E, gid, G, D, u, y, ld);
}

// Order-3 element operator (N = 3, 4 points per direction) by line passes: 16 threads per
// element, thread (a, b) owning one 4-point line in each pass -- its t-line (i = a, j = b) in
// registers for the gather, the t derivative, the geometric factors and the scatter; the r and
// s lines (j = a, k = b and i = a, k = b) through shared memory.  An element's 16 threads are
// half a warp, so the passes synchronise with __syncwarp() and the block has no barrier.  The
// factors of the t-line (24 values) and D (16) are loaded into registers before the gather
// (and, under programmatic dependent launch, before waiting for the kernel that wrote u).
// IMPLICIT: global ids from the box lattice (ids and Dirichlet flags computed, no map read).
constexpr int kAx4Threads = 256;                 // 16 elements per block
constexpr int kAx4Plane = 20;                    // padded k-plane stride: conflict-free s lines

template <typename T, bool IMPLICIT>
__global__ void __launch_bounds__(kAx4Threads)
k_sem_ax4(int64_t E, const uint32_t* __restrict__ gid, Lattice lat, const T* __restrict__ G,
          const T* __restrict__ Dg, const T* __restrict__ u, T* __restrict__ y, int64_t ld) {
  constexpr int PK = kAx4Plane, EL = 4 * kAx4Plane;
  __shared__ __align__(16) T sU[kAx4Threads / 16][EL];
  __shared__ __align__(16) T sR[kAx4Threads / 16][EL];
  __shared__ __align__(16) T sS[kAx4Threads / 16][EL];
  const int tid = threadIdx.x, le = tid >> 4, t = tid & 15, a = t & 3, b = t >> 2;
  const int64_t e = (int64_t)blockIdx.x * (kAx4Threads / 16) + le;
  const bool valid = e < E;
  T D[4][4];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int l = 0; l < 4; ++l) D[i][l] = __ldg(Dg + i * 4 + l);
  T gr[6][4];
  {
    const T* Ge = G + (valid ? e : 0) * 384 + b * 4 + a;
#pragma unroll
    for (int c = 0; c < 6; ++c)
#pragma unroll
      for (int k = 0; k < 4; ++k) gr[c][k] = __ldg(Ge + c * 64 + k * 16);
  }
  uint32_t g[4];
  if (!valid) {
#pragma unroll
    for (int k = 0; k < 4; ++k) g[k] = kGidDirichlet;
  } else if constexpr (IMPLICIT) {
    const uint32_t ee = (uint32_t)e, exy = (uint32_t)lat.nex * (uint32_t)lat.ney;
    const uint32_t ez = ee / exy, rem = ee - ez * exy, ey = rem / (uint32_t)lat.nex, ex = rem - ey * (uint32_t)lat.nex;
    const uint32_t gx = ex * 3 + a, gy = ey * 3 + b;
    const bool side = gx == 0 || gx == (uint32_t)lat.NX - 1 || gy == 0 || gy == (uint32_t)lat.NY - 1;
    const uint32_t plane = (uint32_t)lat.NX * (uint32_t)lat.NY;
    const uint32_t g0 = (ez * 3 * (uint32_t)lat.NY + gy) * (uint32_t)lat.NX + gx;
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      const uint32_t gz = ez * 3 + k;
      g[k] = (g0 + k * plane) | ((side || gz == 0 || gz == (uint32_t)lat.NZ - 1) ? kGidDirichlet : 0u);
    }
  } else {
#pragma unroll
    for (int k = 0; k < 4; ++k) g[k] = __ldg(gid + e * 64 + k * 16 + b * 4 + a);
  }
  u += (int64_t)blockIdx.y * ld;   // right-hand side of a batch
  y += (int64_t)blockIdx.y * ld;
  pdl_wait();   // u and y may come from the kernel before (programmatic dependent launch)
  T col[4];
#pragma unroll
  for (int k = 0; k < 4; ++k) col[k] = (g[k] & kGidDirichlet) ? T(0) : u[g[k] & kGidMask];
  T* su = sU[le];
  T* sr = sR[le];
  T* ss = sS[le];
  T ut[4];
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    su[k * PK + b * 4 + a] = col[k];
    T acc = D[k][0] * col[0];
#pragma unroll
    for (int l = 1; l < 4; ++l) acc = fma(D[k][l], col[l], acc);
    ut[k] = acc;
  }
  __syncwarp();
  {
    T v[4];
#pragma unroll
    for (int l = 0; l < 4; ++l) v[l] = su[b * PK + a * 4 + l];         // r-line (j = a, k = b)
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      T acc = D[i][0] * v[0];
#pragma unroll
      for (int l = 1; l < 4; ++l) acc = fma(D[i][l], v[l], acc);
      sr[b * PK + a * 4 + i] = acc;
    }
#pragma unroll
    for (int l = 0; l < 4; ++l) v[l] = su[b * PK + l * 4 + a];         // s-line (i = a, k = b)
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      T acc = D[j][0] * v[0];
#pragma unroll
      for (int l = 1; l < 4; ++l) acc = fma(D[j][l], v[l], acc);
      ss[b * PK + j * 4 + a] = acc;
    }
  }
  __syncwarp();
  T wt[4];
#pragma unroll
  for (int k = 0; k < 4; ++k) {                                         // own t-line points
    const int q = k * PK + b * 4 + a;
    const T ur = sr[q], us = ss[q], utk = ut[k];
    sr[q] = gr[0][k] * ur + gr[1][k] * us + gr[2][k] * utk;
    ss[q] = gr[1][k] * ur + gr[3][k] * us + gr[4][k] * utk;
    wt[k] = gr[2][k] * ur + gr[4][k] * us + gr[5][k] * utk;
  }
  T yt[4];
#pragma unroll
  for (int k = 0; k < 4; ++k) {                                         // D^T along t
    T acc = D[0][k] * wt[0];
#pragma unroll
    for (int l = 1; l < 4; ++l) acc = fma(D[l][k], wt[l], acc);
    yt[k] = acc;
  }
  __syncwarp();
  {
    T v[4];
#pragma unroll
    for (int l = 0; l < 4; ++l) v[l] = sr[b * PK + a * 4 + l];         // D^T along r
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      T acc = D[0][i] * v[0];
#pragma unroll
      for (int l = 1; l < 4; ++l) acc = fma(D[l][i], v[l], acc);
      su[b * PK + a * 4 + i] = acc;
    }
  }
  __syncwarp();
  {
    T v[4];
#pragma unroll
    for (int l = 0; l < 4; ++l) v[l] = ss[b * PK + l * 4 + a];         // D^T along s
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      T acc = D[0][j] * v[0];
#pragma unroll
      for (int l = 1; l < 4; ++l) acc = fma(D[l][j], v[l], acc);
      su[b * PK + j * 4 + a] += acc;
    }
  }
  __syncwarp();
#pragma unroll
  for (int k = 0; k < 4; ++k)
    if (!(g[k] & kGidDirichlet)) atomicAdd(&y[g[k] & kGidMask], su[k * PK + b * 4 + a] + yt[k]);
}

template <typename T>
void sem_ax4(int64_t E, const uint32_t* gid, const Lattice* lat, const T* G, const T* D, const T* u, T* y,
             cudaStream_t s, int nb, int64_t ld) {
  const dim3 blocks((unsigned)((E + kAx4Threads / 16 - 1) / (kAx4Threads / 16)), nb);
  if (lat)
    launch_dep(k_sem_ax4<T, true>, blocks, dim3(kAx4Threads), 0, s, E, gid, *lat, G, D, u, y, ld);
  else
    launch_dep(k_sem_ax4<T, false>, blocks, dim3(kAx4Threads), 0, s, E, gid, Lattice{}, G, D, u, y, ld);
}

template <typename T>
void sem_ax(int Q, int64_t E, const uint32_t* gid, const T* G, const T* D, const T* u, T* y,
            cudaStream_t s, int nb, int64_t ld) {
  switch (Q) {
    case 2: launch_sem_ax<T, 2>(E, gid, G, D, u, y, s, nb, ld); break;
    case 3: launch_sem_ax<T, 3>(E, gid, G, D, u, y, s, nb, ld); break;
    case 4: launch_sem_ax<T, 4>(E, gid, G, D, u, y, s, nb, ld); break;
    case 5: launch_sem_ax<T, 5>(E, gid, G, D, u, y, s, nb, ld); break;
    case 6: launch_sem_ax<T, 6>(E, gid, G, D, u, y, s, nb, ld); break;
    case 7: launch_sem_ax<T, 7>(E, gid, G, D, u, y, s, nb, ld); break;
    case 8: launch_sem_ax<T, 8>(E, gid, G, D, u, y, s, nb, ld); break;
    case 9: launch_sem_ax<T, 9>(E, gid, G, D, u, y, s, nb, ld); break;
    case 10: launch_sem_ax<T, 10>(E, gid, G, D, u, y, s, nb, ld); break;
    default: break;
  }
}

// ---------------------------------------------------------------------------
// p-multigrid transfers.  One block per element, runtime orders (Q <= 10).
// Restriction uses the owner copy of each fine node: P^T = Q_c^T J3^T O^T,
// which equals Q_c^T J3^T Q_f W because J3 Q_c maps into continuous fields.
// ---------------------------------------------------------------------------
constexpr int kTransferThreads = 256;

template <typename T>
__global__ void __launch_bounds__(kTransferThreads)
k_sem_restrict(int Qf, int Qc, const uint32_t* __restrict__ gidf, const uint32_t* __restrict__ gidc,
               const T* __restrict__ J, const T* __restrict__ rf, T* __restrict__ rc, int64_t ldf, int64_t ldc) {
  pdl_wait();
  rf += (int64_t)blockIdx.y * ldf;
  rc += (int64_t)blockIdx.y * ldc;
  extern __shared__ unsigned char smem_raw[];
  T* sJ = reinterpret_cast<T*>(smem_raw);      // [Qf][Qc]
  T* a = sJ + Qf * Qc;                         // [kf][jf][if]
  T* b = a + Qf * Qf * Qf;                     // [kf][jf][ic]
  T* c = b + Qf * Qf * Qc;                     // [kf][jc][ic]
  const int64_t e = blockIdx.x;
  const int NPf = Qf * Qf * Qf, NPc = Qc * Qc * Qc;
  for (int q = threadIdx.x; q < Qf * Qc; q += blockDim.x) sJ[q] = J[q];
  for (int p = threadIdx.x; p < NPf; p += blockDim.x) {
    const uint32_t id = gidf[e * NPf + p];
    a[p] = ((id & kGidOwner) && !(id & kGidDirichlet)) ? rf[id & kGidMask] : T(0);
  }
  __syncthreads();
  for (int q = threadIdx.x; q < Qf * Qf * Qc; q += blockDim.x) {
    const int ic = q % Qc, jf = (q / Qc) % Qf, kf = q / (Qc * Qf);
    T acc = 0;
    for (int l = 0; l < Qf; ++l) acc += sJ[l * Qc + ic] * a[(kf * Qf + jf) * Qf + l];
    b[q] = acc;
  }
  __syncthreads();
  for (int q = threadIdx.x; q < Qf * Qc * Qc; q += blockDim.x) {
    const int ic = q % Qc, jc = (q / Qc) % Qc, kf = q / (Qc * Qc);
    T acc = 0;
    for (int l = 0; l < Qf; ++l) acc += sJ[l * Qc + jc] * b[(kf * Qf + l) * Qc + ic];
    c[q] = acc;
  }
  __syncthreads();
  for (int q = threadIdx.x; q < NPc; q += blockDim.x) {
    const int ic = q % Qc, jc = (q / Qc) % Qc, kc = q / (Qc * Qc);
    T acc = 0;
    for (int l = 0; l < Qf; ++l) acc += sJ[l * Qc + kc] * c[(l * Qc + jc) * Qc + ic];
    const uint32_t id = gidc[e * NPc + q];
    if (!(id & kGidDirichlet)) atomicAdd(&rc[id & kGidMask], acc);
  }
}

template <typename T>
__global__ void __launch_bounds__(kTransferThreads)
k_sem_prolong(int Qf, int Qc, const uint32_t* __restrict__ gidf, const uint32_t* __restrict__ gidc,
              const T* __restrict__ J, const T* __restrict__ zc, T* __restrict__ zf, int accumulate, int64_t ldf,
              int64_t ldc) {
  pdl_wait();
  zf += (int64_t)blockIdx.y * ldf;
  zc += (int64_t)blockIdx.y * ldc;
  extern __shared__ unsigned char smem_raw[];
  T* sJ = reinterpret_cast<T*>(smem_raw);      // [Qf][Qc]
  T* a = sJ + Qf * Qc;                         // [kc][jc][ic]
  T* b = a + Qc * Qc * Qc;                     // [kc][jc][if]
  T* c = b + Qc * Qc * Qf;                     // [kc][jf][if]
  const int64_t e = blockIdx.x;
  const int NPf = Qf * Qf * Qf, NPc = Qc * Qc * Qc;
  for (int q = threadIdx.x; q < Qf * Qc; q += blockDim.x) sJ[q] = J[q];
  for (int p = threadIdx.x; p < NPc; p += blockDim.x) {
    const uint32_t id = gidc[e * NPc + p];
    a[p] = (id & kGidDirichlet) ? T(0) : zc[id & kGidMask];
  }
  __syncthreads();
  for (int q = threadIdx.x; q < Qc * Qc * Qf; q += blockDim.x) {
    const int iF = q % Qf, jc = (q / Qf) % Qc, kc = q / (Qf * Qc);
    T acc = 0;
    for (int l = 0; l < Qc; ++l) acc += sJ[iF * Qc + l] * a[(kc * Qc + jc) * Qc + l];
    b[q] = acc;
  }
  __syncthreads();
  for (int q = threadIdx.x; q < Qc * Qf * Qf; q += blockDim.x) {
    const int iF = q % Qf, jF = (q / Qf) % Qf, kc = q / (Qf * Qf);
    T acc = 0;
    for (int l = 0; l < Qc; ++l) acc += sJ[jF * Qc + l] * b[(kc * Qc + l) * Qf + iF];
    c[q] = acc;
  }
  __syncthreads();
  for (int q = threadIdx.x; q < NPf; q += blockDim.x) {
    const int iF = q % Qf, jF = (q / Qf) % Qf, kF = q / (Qf * Qf);
    const uint32_t id = gidf[e * NPf + q];
    if (!(id & kGidOwner)) continue;
    T* dst = &zf[id & kGidMask];
    if (id & kGidDirichlet) {
      if (!accumulate) *dst = T(0);
      continue;
    }
    T acc = 0;
    for (int l = 0; l < Qc; ++l) acc += sJ[kF * Qc + l] * c[(l * Qf + jF) * Qf + iF];
    *dst = accumulate ? *dst + acc : acc;
  }
}

template <typename T>
static size_t transfer_smem(int Qf, int Qc) {
  return sizeof(T) * (size_t)(Qf * Qc + Qf * Qf * Qf + Qf * Qf * Qc + Qf * Qc * Qc);
}

template <typename T>
void sem_restrict(int Qf, int Qc, int64_t E, const uint32_t* gidf, const uint32_t* gidc, const T* J,
                  const T* rf, T* rc, cudaStream_t s, int nb, int64_t ldf, int64_t ldc) {
  launch_dep(k_sem_restrict<T>, dim3((unsigned)E, nb), dim3(kTransferThreads), transfer_smem<T>(Qf, Qc), s, Qf, Qc,
             gidf, gidc, J, rf, rc, ldf, ldc);
}

template <typename T>
void sem_prolong(int Qf, int Qc, int64_t E, const uint32_t* gidf, const uint32_t* gidc, const T* J,
                 const T* zc, T* zf, int accumulate, cudaStream_t s, int nb, int64_t ldf, int64_t ldc) {
  launch_dep(k_sem_prolong<T>, dim3((unsigned)E, nb), dim3(kTransferThreads), transfer_smem<T>(Qf, Qc), s, Qf, Qc,
             gidf, gidc, J, zc, zf, accumulate, ldf, ldc);
}

// ===========================================================================
// FD kernels
// ===========================================================================
template <typename T>
__global__ void k_fd_apply(int mx, int my, Stencil9<T> st, const T* __restrict__ u, T* __restrict__ y,
                           int64_t ld) {
  pdl_wait();
  u += (int64_t)blockIdx.z * ld;   // right-hand side of a batch
  y += (int64_t)blockIdx.z * ld;
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const int j = blockIdx.y * blockDim.y + threadIdx.y;
  if (i >= mx || j >= my) return;
  T acc = 0;
#pragma unroll
  for (int a = -1; a <= 1; ++a) {
    const int jj = j + a;
    if (jj < 0 || jj >= my) continue;
#pragma unroll
    for (int b = -1; b <= 1; ++b) {
      const int ii = i + b;
      if (ii < 0 || ii >= mx) continue;
      acc += st.c[(a + 1) * 3 + (b + 1)] * u[(size_t)jj * mx + ii];
    }
  }
  y[(size_t)j * mx + i] = acc;
}

template <typename T>
void fd_apply(int mx, int my, const Stencil9<T>& st, const T* u, T* y, cudaStream_t s, int nb, int64_t ld) {
  dim3 bs(32, 8);
  dim3 gs((mx + 31) / 32, (my + 7) / 8, nb);
  launch_dep(k_fd_apply<T>, gs, bs, 0, s, mx, my, st, u, y, ld);
}

// rc(I,J) = sum_{|a|,|b| < c} w_a w_b rf(c(I+1)-1+b, c(J+1)-1+a), w_d = (c - |d|)/c
template <typename T>
__global__ void k_fd_restrict(int mfx, int mfy, int mcx, int mcy, int c, const T* __restrict__ rf,
                              T* __restrict__ rc, int64_t ldf, int64_t ldc) {
  pdl_wait();
  rf += (int64_t)blockIdx.z * ldf;
  rc += (int64_t)blockIdx.z * ldc;
  const int I = blockIdx.x * blockDim.x + threadIdx.x;
  const int Jc = blockIdx.y * blockDim.y + threadIdx.y;
  if (I >= mcx || Jc >= mcy) return;
  const int fi = c * (I + 1) - 1, fj = c * (Jc + 1) - 1;
  const T inv_c = T(1) / T(c);
  T acc = 0;
  for (int a = -(c - 1); a <= c - 1; ++a) {
    const int jj = fj + a;
    if (jj < 0 || jj >= mfy) continue;
    const T wa = T(c - (a < 0 ? -a : a)) * inv_c;
    T row = 0;
    for (int b = -(c - 1); b <= c - 1; ++b) {
      const int ii = fi + b;
      if (ii < 0 || ii >= mfx) continue;
      row += T(c - (b < 0 ? -b : b)) * inv_c * rf[(size_t)jj * mfx + ii];
    }
    acc += wa * row;
  }
  rc[(size_t)Jc * mcx + I] = acc;
}

template <typename T>
__global__ void k_fd_prolong(int mfx, int mfy, int mcx, int mcy, int c, const T* __restrict__ zc,
                             T* __restrict__ zf, int accumulate, int64_t ldf, int64_t ldc) {
  pdl_wait();
  zf += (int64_t)blockIdx.z * ldf;
  zc += (int64_t)blockIdx.z * ldc;
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const int j = blockIdx.y * blockDim.y + threadIdx.y;
  if (i >= mfx || j >= mfy) return;
  const T inv_c = T(1) / T(c);
  const int I0 = (i + 1) / c - 1, J0 = (j + 1) / c - 1;
  const int di = i - (c * (I0 + 1) - 1), dj = j - (c * (J0 + 1) - 1);
  T wi[2] = {T(c - di) * inv_c, T(di) * inv_c};
  T wj[2] = {T(c - dj) * inv_c, T(dj) * inv_c};
  T acc = 0;
  for (int a = 0; a < 2; ++a) {
    const int Jc = J0 + a;
    if (Jc < 0 || Jc >= mcy || wj[a] == T(0)) continue;
    for (int b = 0; b < 2; ++b) {
      const int I = I0 + b;
      if (I < 0 || I >= mcx || wi[b] == T(0)) continue;
      acc += wj[a] * wi[b] * zc[(size_t)Jc * mcx + I];
    }
  }
  T* dst = &zf[(size_t)j * mfx + i];
  *dst = accumulate ? *dst + acc : acc;
}

template <typename T>
void fd_restrict(int mfx, int mfy, int mcx, int mcy, int c, const T* rf, T* rc, cudaStream_t s, int nb,
                 int64_t ldf, int64_t ldc) {
  dim3 bs(16, 16);
  dim3 gs((mcx + 15) / 16, (mcy + 15) / 16, nb);
  launch_dep(k_fd_restrict<T>, gs, bs, 0, s, mfx, mfy, mcx, mcy, c, rf, rc, ldf, ldc);
}

template <typename T>
void fd_prolong(int mfx, int mfy, int mcx, int mcy, int c, const T* zc, T* zf, int accumulate,
                cudaStream_t s, int nb, int64_t ldf, int64_t ldc) {
  dim3 bs(32, 8);
  dim3 gs((mfx + 31) / 32, (mfy + 7) / 8, nb);
  launch_dep(k_fd_prolong<T>, gs, bs, 0, s, mfx, mfy, mcx, mcy, c, zc, zf, accumulate, ldf, ldc);
}

__global__ void k_dense_matvec(int n, const double* __restrict__ M, const double* __restrict__ x,
                               double* __restrict__ y, int64_t ld) {
  pdl_wait();
  x += (int64_t)blockIdx.y * ld;
  y += (int64_t)blockIdx.y * ld;
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  double acc = 0.0;
  for (int j = 0; j < n; ++j) acc += M[(size_t)i * n + j] * x[j];
  y[i] = acc;
}

void dense_matvec(int n, const double* M, const double* x, double* y, cudaStream_t s, int nb, int64_t ld) {
  launch_dep(k_dense_matvec, dim3((n + 127) / 128, nb), dim3(128), 0, s, n, M, x, y, ld);
}

// p[0 .. bytes) = 0, 16-byte stores over the aligned body: the zeroing of a work vector as a
// kernel, so that it joins a chain of programmatic dependent launches (a memset node would end it).
__global__ void k_zero_bytes(unsigned char* __restrict__ p, int64_t bytes) {
  pdl_wait();
  const int64_t tid = blockIdx.x * (int64_t)blockDim.x + threadIdx.x, stride = (int64_t)gridDim.x * blockDim.x;
  const int64_t n16 = bytes / 16;
  for (int64_t q = tid; q < n16; q += stride) reinterpret_cast<uint4*>(p)[q] = make_uint4(0u, 0u, 0u, 0u);
  for (int64_t g = n16 * 16 + tid; g < bytes; g += stride) p[g] = 0;
}

void zero_bytes(void* p, int64_t bytes, cudaStream_t s) {
  if ((uintptr_t)p % 16 != 0 || bytes <= 0) {
    cudaMemsetAsync(p, 0, (size_t)(bytes > 0 ? bytes : 0), s);
    return;
  }
  launch_dep(k_zero_bytes, dim3(grid_for(bytes / 16 + 1, kVecThreads)), dim3(kVecThreads), 0, s,
             static_cast<unsigned char*>(p), bytes);
}

// ===========================================================================
// Deterministic FP64 reductions: fixed kRedBlocks partials, fixed-order finish
// ===========================================================================
constexpr int kRedThreads = 256;

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  return v;
}

// Block-wide sum of two values; result valid in thread 0.
__device__ __forceinline__ void block_sum2(double& a, double& b) {
  __shared__ double sa[kRedThreads / 32], sb[kRedThreads / 32];
  a = warp_sum(a);
  b = warp_sum(b);
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  if (l == 0) {
    sa[w] = a;
    sb[w] = b;
  }
  __syncthreads();
  if (w == 0) {
    a = l < kRedThreads / 32 ? sa[l] : 0.0;
    b = l < kRedThreads / 32 ? sb[l] : 0.0;
    a = warp_sum(a);
    b = warp_sum(b);
  }
}

__global__ void __launch_bounds__(kRedThreads)
k_dot2_partial(int64_t n, const double* __restrict__ a0, const double* __restrict__ b0,
               const double* __restrict__ a1, const double* __restrict__ b1, double* __restrict__ partial) {
  pdl_wait();
  double s0 = 0.0, s1 = 0.0;
  for (int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; g < n; g += (int64_t)gridDim.x * blockDim.x) {
    s0 += a0[g] * b0[g];
    if (a1) s1 += a1[g] * b1[g];
  }
  block_sum2(s0, s1);
  if (threadIdx.x == 0) {
    partial[blockIdx.x] = s0;
    partial[kRedBlocks + blockIdx.x] = s1;
  }
}

__device__ void apply_post(int post, double* scal) {
  switch (post) {
    case POST_ALPHA: scal[S_ALPHA] = scal[S_RZ] / scal[S_PQ]; break;
    case POST_BETA_CG:     // Fletcher-Reeves for the coarse CG: beta = rz_new / rz_old
      scal[S_BETA] = scal[S_ZR] / scal[S_RZ];
      scal[S_RZ] = scal[S_ZR];
      break;
    case POST_SET_RZ_FROM_ZR: scal[S_RZ] = scal[S_ZR]; break;
    case POST_BETA_FLEX_Q:   // the same Polak-Ribiere beta with r_new - r_old = -alpha q
      scal[S_BETA] = -scal[S_ALPHA] * scal[S_ZQ] / scal[S_RZ];
      scal[S_RZ] = scal[S_ZR];
      break;
    default: break;
  }
}

// One block: sums the partials of two slots in a fixed order, then the post-op.
__global__ void __launch_bounds__(kRedThreads)
k_dot2_finish(const double* __restrict__ partial, int slot0, int slot1, int post, double* __restrict__ scal) {
  pdl_wait();
  double s0 = 0.0, s1 = 0.0;
  for (int q = threadIdx.x; q < kRedBlocks; q += blockDim.x) {
    s0 += partial[q];
    s1 += partial[kRedBlocks + q];
  }
  block_sum2(s0, s1);
  if (threadIdx.x == 0) {
    if (slot0 >= 0) scal[slot0] = s0;
    if (slot1 >= 0) scal[slot1] = s1;
    apply_post(post, scal);
  }
}

void dot2(int64_t n, const double* a0, const double* b0, const double* a1, const double* b1, int slot0,
          int slot1, int post, double* partial, double* scal, cudaStream_t s) {
  launch_dep(k_dot2_partial, dim3(kRedBlocks), dim3(kRedThreads), 0, s, n, a0, b0, a1, b1, partial);
  launch_dep(k_dot2_finish, dim3(1), dim3(kRedThreads), 0, s, (const double*)partial, slot0, a1 ? slot1 : -1, post,
             scal);
}

__global__ void __launch_bounds__(kRedThreads)
k_fcg_update_xr32(int64_t n, double* __restrict__ x, double* __restrict__ r, float* __restrict__ r32,
                  const double* __restrict__ p, const double* __restrict__ q, double* __restrict__ partial,
                  const double* __restrict__ scal) {
  pdl_wait();
  const double alpha = scal[S_ALPHA];
  double s0 = 0.0, s1 = 0.0;
  for (int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; g < n; g += (int64_t)gridDim.x * blockDim.x) {
    x[g] += alpha * p[g];
    const double rn = r[g] - alpha * q[g];
    r[g] = rn;
    if (r32) r32[g] = narrow_f64(rn);
    s0 += rn * rn;
  }
  block_sum2(s0, s1);
  if (threadIdx.x == 0) {
    partial[blockIdx.x] = s0;
    partial[kRedBlocks + blockIdx.x] = 0.0;
  }
}

void fcg_update_xr32(int64_t n, double* x, double* r, float* r32, const double* p, const double* q,
                     double* partial, double* scal, cudaStream_t s) {
  launch_dep(k_fcg_update_xr32, dim3(kRedBlocks), dim3(kRedThreads), 0, s, n, x, r, r32, p, q, partial,
             (const double*)scal);
  launch_dep(k_dot2_finish, dim3(1), dim3(kRedThreads), 0, s, (const double*)partial, (int)S_RR, -1, (int)POST_NONE,
             scal);
}

template <typename Tz>
__global__ void __launch_bounds__(kRedThreads)
k_dot_zr_zq(int64_t n, const Tz* __restrict__ z, const double* __restrict__ r, const double* __restrict__ q,
            double* __restrict__ partial) {
  pdl_wait();
  double s0 = 0.0, s1 = 0.0;
  for (int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; g < n; g += (int64_t)gridDim.x * blockDim.x) {
    const double zv = to_f64(z[g]);
    s0 += zv * r[g];
    if (q) s1 += zv * q[g];
  }
  block_sum2(s0, s1);
  if (threadIdx.x == 0) {
    partial[blockIdx.x] = s0;
    partial[kRedBlocks + blockIdx.x] = s1;
  }
}

template <typename Tz>
void dot_zr_zq(int64_t n, const Tz* z, const double* r, const double* q, int post, double* partial, double* scal,
               cudaStream_t s) {
  launch_dep(k_dot_zr_zq<Tz>, dim3(kRedBlocks), dim3(kRedThreads), 0, s, n, z, r, q, partial);
  launch_dep(k_dot2_finish, dim3(1), dim3(kRedThreads), 0, s, (const double*)partial, (int)S_ZR,
             q ? (int)S_ZQ : -1, post, scal);
}
template void dot_zr_zq<float>(int64_t, const float*, const double*, const double*, int, double*, double*,
                               cudaStream_t);
template void dot_zr_zq<double>(int64_t, const double*, const double*, const double*, int, double*, double*,
                                cudaStream_t);

// p = z + beta p (p = z first), and q = 0 when q is given (the next product accumulates into it).
// Vector path: four entries per thread (z as one 16-byte load for FP32), 16-byte p and q accesses.
template <typename Tz, bool VEC>
__global__ void k_update_p_from(int64_t n, const Tz* __restrict__ z, double* __restrict__ p,
                                const double* __restrict__ scal, int first, double* __restrict__ q) {
  pdl_wait();
  const double beta = first ? 0.0 : scal[S_BETA];
  const int64_t tid = blockIdx.x * (int64_t)blockDim.x + threadIdx.x, stride = (int64_t)gridDim.x * blockDim.x;
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

template <typename Tz>
void update_p_from(int64_t n, const Tz* z, double* p, const double* scal, bool first, cudaStream_t s, double* q) {
  const uintptr_t align = (uintptr_t)z | (uintptr_t)p | (uintptr_t)q;
  if (align % 16 == 0)
    launch_dep(k_update_p_from<Tz, true>, dim3(grid_for(n / 4 + 1, kVecThreads)), dim3(kVecThreads), 0, s, n, z, p,
               scal, first ? 1 : 0, q);
  else
    launch_dep(k_update_p_from<Tz, false>, dim3(grid_for(n, kVecThreads)), dim3(kVecThreads), 0, s, n, z, p, scal,
               first ? 1 : 0, q);
}
template void update_p_from<float>(int64_t, const float*, double*, const double*, bool, cudaStream_t, double*);
template void update_p_from<double>(int64_t, const double*, double*, const double*, bool, cudaStream_t, double*);

__global__ void k_update_p(int64_t n, const double* __restrict__ z, double* __restrict__ p,
                           const double* __restrict__ scal) {
  pdl_wait();
  const double beta = scal[S_BETA];
  for (int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; g < n; g += (int64_t)gridDim.x * blockDim.x)
    p[g] = z[g] + beta * p[g];
}

void update_p(int64_t n, const double* z, double* p, const double* scal, cudaStream_t s) {
  launch_dep(k_update_p, dim3(grid_for(n, kVecThreads)), dim3(kVecThreads), 0, s, n, z, p, scal);
}

__global__ void __launch_bounds__(kRedThreads)
k_cg_update(int64_t n, double* __restrict__ x, double* __restrict__ r, double* __restrict__ z,
            const double* __restrict__ p, const double* __restrict__ q, const double* __restrict__ invD,
            double* __restrict__ partial, const double* __restrict__ scal) {
  pdl_wait();
  const double alpha = scal[S_ALPHA];
  double s0 = 0.0, s1 = 0.0;
  for (int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; g < n; g += (int64_t)gridDim.x * blockDim.x) {
    x[g] += alpha * p[g];
    const double rn = r[g] - alpha * q[g];
    r[g] = rn;
    const double zn = invD[g] * rn;
    z[g] = zn;
    s0 += rn * rn;
    s1 += rn * zn;
  }
  block_sum2(s0, s1);
  if (threadIdx.x == 0) {
    partial[blockIdx.x] = s0;
    partial[kRedBlocks + blockIdx.x] = s1;
  }
}

void cg_update(int64_t n, double* x, double* r, double* z, const double* p, const double* q,
               const double* invD, double* partial, double* scal, cudaStream_t s) {
  launch_dep(k_cg_update, dim3(kRedBlocks), dim3(kRedThreads), 0, s, n, x, r, z, p, q, invD, partial,
             (const double*)scal);
  launch_dep(k_dot2_finish, dim3(1), dim3(kRedThreads), 0, s, (const double*)partial, (int)S_RR, (int)S_ZR,
             (int)POST_BETA_CG, scal);
}

// ===========================================================================
// Persistent coarse Jacobi-PCG: the whole solve in one cooperative launch.
// ELL SpMV, deterministic block partial sums read back by every block in the
// same order (so all blocks take identical alpha/beta/stop decisions), and a
// grid barrier whose waits are bounded: a block that waits too long records a
// timeout and returns, and every other block then also returns at its next
// (bounded) wait, so the kernel always finishes.
// ===========================================================================
constexpr int kCoarseThreads = 256;

__device__ __forceinline__ void block_allsum2(double& a, double& b) {
  __shared__ double sa[kCoarseThreads / 32], sb[kCoarseThreads / 32];
  __syncthreads();
  a = warp_sum(a);
  b = warp_sum(b);
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  if (l == 0) {
    sa[w] = a;
    sb[w] = b;
  }
  __syncthreads();
  double ta = 0.0, tb = 0.0;
#pragma unroll
  for (int q = 0; q < kCoarseThreads / 32; ++q) {   // same order in every thread
    ta += sa[q];
    tb += sb[q];
  }
  a = ta;
  b = tb;
}

// Block sum of three values: one warp adds the per-thread values through shared memory
// (few FP64 additions: GB300 issues about two FP64 operations per clock per SM).  Result in
// all threads; fixed order.
__device__ __forceinline__ void block_sum3(double& a, double& b, double& c) {
  __shared__ double sh[3][kCoarseThreads];
  __shared__ double res[3];
  __syncthreads();
  sh[0][threadIdx.x] = a;
  sh[1][threadIdx.x] = b;
  sh[2][threadIdx.x] = c;
  __syncthreads();
  if (threadIdx.x < 32) {
    double t0 = 0.0, t1 = 0.0, t2 = 0.0;
#pragma unroll
    for (int q = 0; q < kCoarseThreads / 32; ++q) {
      t0 += sh[0][threadIdx.x + 32 * q];
      t1 += sh[1][threadIdx.x + 32 * q];
      t2 += sh[2][threadIdx.x + 32 * q];
    }
    t0 = warp_sum(t0);
    t1 = warp_sum(t1);
    t2 = warp_sum(t2);
    if (threadIdx.x == 0) {
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

__device__ __forceinline__ unsigned ld_acquire(const unsigned* p) {
  unsigned v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ void red_release_add(unsigned* p, unsigned v) {
  asm volatile("red.release.gpu.global.add.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}
__device__ __forceinline__ uint64_t global_ns() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}
constexpr uint64_t kWaitNs = 1000000000ull;   // every wait gives up after about a second

// Spins until *p >= target (acquire); false after kWaitNs, with the timeout recorded.
__device__ __forceinline__ bool wait_at_least(const unsigned* p, unsigned target, unsigned* ctl) {
  if (ld_acquire(p) >= target) return true;
  const uint64_t t0 = global_ns();
  for (unsigned it = 1;; ++it) {
    __nanosleep(20);                     // back off: polling competes with the producers' stores
    if (ld_acquire(p) >= target) return true;
    if ((it & 63u) == 0 && global_ns() - t0 > kWaitNs) {
      atomicMax((int*)&ctl[4], (int)CS_TIMEOUT);
      return false;
    }
  }
}

// Grid-wide sum of three values (a, b, c: this block's totals, the same in every thread),
// replaced by the grid totals.  Each block posts its partials into the buffer of this
// generation's parity and arrives at a monotonic counter (release); once all `expected`
// blocks have arrived (acquire), every block sums all partials in the same fixed order, so
// the totals are bitwise identical everywhere.  Two buffers suffice: a block can only write a
// buffer again two reductions later, after every block has passed the reduction in between,
// i.e. after every block has finished reading it.
__device__ __forceinline__ bool allreduce3(unsigned* ctl, unsigned& gen, unsigned expected, double* part,
                                           double& a, double& b, double& c) {
  __shared__ int s_ok;
  const unsigned g1 = gen + 1;
  double* p = part + (size_t)(g1 & 1u) * 3 * gridDim.x;
  if (threadIdx.x == 0) {
    p[3 * blockIdx.x] = a;
    p[3 * blockIdx.x + 1] = b;
    p[3 * blockIdx.x + 2] = c;
    red_release_add(&ctl[0], 1u);
    s_ok = wait_at_least(&ctl[0], g1 * expected, ctl) ? 1 : 0;
  }
  __syncthreads();
  double A = 0.0, B = 0.0, C = 0.0;
  if (s_ok)
    for (int q = threadIdx.x; q < (int)gridDim.x; q += blockDim.x) {
      A += __ldcg(&p[3 * q]);
      B += __ldcg(&p[3 * q + 1]);
      C += __ldcg(&p[3 * q + 2]);
    }
  const bool ok = s_ok != 0;
  block_sum3(A, B, C);
  gen = g1;
  a = A;
  b = B;
  c = C;
  return ok;
}
// ---- tagged-word exchange ----
__device__ __forceinline__ void st_tagged(unsigned long long* p, unsigned long long w) {
  asm volatile("st.relaxed.gpu.global.b64 [%0], %1;" ::"l"(p), "l"(w) : "memory");
}
__device__ __forceinline__ void st_tagged2(unsigned long long* p, unsigned long long w0, unsigned long long w1) {
  asm volatile("st.relaxed.gpu.global.v2.b64 [%0], {%1, %2};" ::"l"(p), "l"(w0), "l"(w1) : "memory");
}
__device__ __forceinline__ unsigned long long ld_tagged(const unsigned long long* p) {
  unsigned long long w;
  asm volatile("ld.relaxed.gpu.global.b64 %0, [%1];" : "=l"(w) : "l"(p) : "memory");
  return w;
}
__device__ __forceinline__ void ld_tagged2(const unsigned long long* p, unsigned long long& w0,
                                           unsigned long long& w1) {
  asm volatile("ld.relaxed.gpu.global.v2.b64 {%0, %1}, [%2];" : "=l"(w0), "=l"(w1) : "l"(p) : "memory");
}
// Column index load that the compiler may not merge with an earlier one (keeps the reload
// loop from holding all column indices in registers).
__device__ __forceinline__ int ld_col(const int* p) {
  int v;
  asm volatile("ld.global.nc.b32 %0, [%1];" : "=r"(v) : "l"(p));
  return v;
}

// One exchanged value: FP32 in one tagged word, FP64 as two (high and low halves, loaded
// and stored together; each half carries the tag, so a torn pair is never accepted).
template <typename V>
struct Tagged;
template <>
struct Tagged<float> {
  struct W {
    unsigned long long w;
  };
  static __device__ __forceinline__ unsigned long long* buf(const CoarseCG& a, unsigned gx) {
    return a.exf[gx & 1u];
  }
  static __device__ __forceinline__ void store(unsigned long long* b, int64_t g, unsigned tag, float v) {
    st_tagged(b + g, ((unsigned long long)tag << 32) | __float_as_uint(v));
  }
  static __device__ __forceinline__ W load(const unsigned long long* b, int64_t g) { return {ld_tagged(b + g)}; }
  static __device__ __forceinline__ bool ready(const W& w, unsigned tag) { return (unsigned)(w.w >> 32) == tag; }
  static __device__ __forceinline__ float value(const W& w) { return __uint_as_float((unsigned)w.w); }
  static __device__ __forceinline__ float coef(const CoarseCG& a, int64_t i) { return __ldg(&a.valf[i]); }
};
template <>
struct Tagged<double> {
  struct W {
    unsigned long long hi, lo;
  };
  static __device__ __forceinline__ unsigned long long* buf(const CoarseCG& a, unsigned gx) {
    return a.exd[gx & 1u];
  }
  static __device__ __forceinline__ void store(unsigned long long* b, int64_t g, unsigned tag, double v) {
    const unsigned long long t = (unsigned long long)tag << 32;
    st_tagged2(b + 2 * g, t | (unsigned)__double2hiint(v), t | (unsigned)__double2loint(v));
  }
  static __device__ __forceinline__ W load(const unsigned long long* b, int64_t g) {
    W w;
    ld_tagged2(b + 2 * g, w.hi, w.lo);
    return w;
  }
  static __device__ __forceinline__ bool ready(const W& w, unsigned tag) {
    return (unsigned)(w.hi >> 32) == tag && (unsigned)(w.lo >> 32) == tag;
  }
  static __device__ __forceinline__ double value(const W& w) {
    return __hiloint2double((int)(unsigned)w.hi, (int)(unsigned)w.lo);
  }
  static __device__ __forceinline__ double coef(const CoarseCG& a, int64_t i) { return __ldg(&a.val[i]); }
};

// Publishes this block's rows under exchange gx.  No barrier first: every product ends with
// a block barrier, so this block has finished reading the buffer it overwrites (two exchanges
// ago), and a neighbour only moves on to it after reading values this block published after
// that barrier.
template <typename V, int RPT>
__device__ __forceinline__ void publish_tagged(const CoarseCG& a, unsigned gx, const V (&v)[RPT], int64_t base) {
  unsigned long long* b = Tagged<V>::buf(a, gx);
  const unsigned tag = a.gen0 + gx;
#pragma unroll
  for (int q = 0; q < RPT; ++q) {
    const int64_t g = base + threadIdx.x + (int64_t)q * blockDim.x;
    if (g < a.n && g < base + a.rows_per_block) Tagged<V>::store(b, g, tag, v[q]);
  }
}

// y = A v on this block's rows, v read from exchange gx: all column indices first, then all
// words, then every word whose tag is not there yet reloaded in the next round (one L2 round
// trip per round).  Ends with a block barrier; false in every thread if a wait ran out.
template <typename V, int NS, int RPT>
__device__ __forceinline__ bool coarse_spmv_tagged(const CoarseCG& a, unsigned gx, int64_t base, V (&y)[RPT]) {
  using TW = typename Tagged<V>::W;
  const unsigned long long* b = Tagged<V>::buf(a, gx);
  const unsigned tag = a.gen0 + gx;
  const int64_t n = a.n;
  const bool lat = NS == 27 && a.lat_nx > 0;
  // column of slot k: read from the ELL, or (box lattice) the row plus the slot's offset
  auto column = [&](int k, int64_t g) -> int {
    if (lat) return (int)g + (k / 9 - 1) * a.lat_nxy + ((k / 3) % 3 - 1) * a.lat_nx + (k % 3 - 1);
    return ld_col(&a.col[k * n + g]);
  };
  // Box lattice: slots whose column is a lattice-boundary (Dirichlet) node are absent, as in the
  // ELL, where those columns were removed.  Reading them would make a row depend on a node that
  // reads nothing in turn, and the exchange's double buffering relies on blocks that read each
  // other's rows doing so both ways.  Bit d of pmask[axis] is set when offset d - 1 along that
  // axis stays inside the interior.
  auto slot_present = [&](int k, const unsigned (&pm)[3]) -> bool {
    return ((pm[0] >> (k % 3)) & (pm[1] >> ((k / 3) % 3)) & (pm[2] >> (k / 9)) & 1u) != 0;
  };
  bool ok = true;
#pragma unroll
  for (int q = 0; q < RPT; ++q) {
    const int64_t g = base + threadIdx.x + (int64_t)q * blockDim.x;
    V acc = V(0);
    if (g < n && g < base + a.rows_per_block && (!lat || __ldg(&a.invD[g]) != 0.0)) {
      unsigned pm[3] = {7u, 7u, 7u};
      if (lat) {
        const int gi = (int)g, nz = (int)(n / a.lat_nxy);
        const int gz = gi / a.lat_nxy, rem = gi - gz * a.lat_nxy, gy = rem / a.lat_nx, gxx = rem - gy * a.lat_nx;
        const int c3[3] = {gxx, gy, gz}, e3[3] = {a.lat_nx, a.lat_nxy / a.lat_nx, nz};
#pragma unroll
        for (int d = 0; d < 3; ++d) pm[d] = (c3[d] - 1 >= 1 ? 1u : 0u) | 2u | (c3[d] + 1 <= e3[d] - 2 ? 4u : 0u);
      }
      if constexpr (NS > 0) {
        // FP64 words come in pairs: a third of the slots at a time keeps them in registers
        constexpr int CH = sizeof(V) == 4 ? NS : (NS + 2) / 3;
        static_assert(CH <= 32, "miss mask is 32 bits");
#pragma unroll
        for (int k0 = 0; k0 < NS; k0 += CH) {
          TW w[CH];
          unsigned absent = 0;   // slots not read (their coefficient is zero)
          {
            int c[CH];
#pragma unroll
            for (int k = 0; k < CH; ++k)
              if (k0 + k < NS) {
                if (lat && !slot_present(k0 + k, pm)) absent |= 1u << k;
                c[k] = column(k0 + k, g);
              }
#pragma unroll
            for (int k = 0; k < CH; ++k)
              if (k0 + k < NS) w[k] = (absent >> k & 1u) ? TW{} : Tagged<V>::load(b, c[k]);
          }
          unsigned miss = 0;
#pragma unroll
          for (int k = 0; k < CH; ++k)
            if (k0 + k < NS && !(absent >> k & 1u) && !Tagged<V>::ready(w[k], tag)) miss |= 1u << k;
          if (miss && ok) {
            const uint64_t t0 = global_ns();
            for (unsigned it = 1; miss; ++it) {
              if (it > 16) __nanosleep(32);
              int c[CH];
#pragma unroll
              for (int k = 0; k < CH; ++k)
                if (miss >> k & 1u) c[k] = column(k0 + k, g);
#pragma unroll
              for (int k = 0; k < CH; ++k)
                if (miss >> k & 1u) w[k] = Tagged<V>::load(b, c[k]);
              unsigned still = 0;
#pragma unroll
              for (int k = 0; k < CH; ++k)
                if ((miss >> k & 1u) && !Tagged<V>::ready(w[k], tag)) still |= 1u << k;
              miss = still;
              if (miss && (it & 63u) == 0 && global_ns() - t0 > kWaitNs) {
                atomicMax((int*)&a.ctl[4], (int)CS_TIMEOUT);
                ok = false;
                break;
              }
            }
          }
#pragma unroll
          for (int k = 0; k < CH; ++k)
            if (k0 + k < NS) acc = fma(Tagged<V>::coef(a, (k0 + k) * n + g), Tagged<V>::value(w[k]), acc);
        }
      } else {
        for (int k = 0; k < a.nslot && ok; ++k) {
          const int c = __ldg(&a.col[k * n + g]);
          TW w = Tagged<V>::load(b, c);
          const uint64_t t0 = global_ns();
          for (unsigned it = 1; !Tagged<V>::ready(w, tag); ++it) {
            if (it > 16) __nanosleep(32);
            w = Tagged<V>::load(b, c);
            if ((it & 63u) == 0 && !Tagged<V>::ready(w, tag) && global_ns() - t0 > kWaitNs) {
              atomicMax((int*)&a.ctl[4], (int)CS_TIMEOUT);
              ok = false;
              break;
            }
          }
          acc = fma(Tagged<V>::coef(a, k * n + g), Tagged<V>::value(w), acc);
        }
      }
    }
    y[q] = acc;
  }
  return __syncthreads_and(ok) != 0;
}

// Persistent preconditioned CG on the assembled coarse operator.  The preconditioner is one
// application of Algorithm 2 (4th kind, beta = 1) of degree m from a zero guess, Jacobi-
// scaled -- SPD for every m, and for m = 1 simply Jacobi.  Per CG iteration: m products,
// each reading the neighbouring blocks' rows through tagged words (no flags, no fences), and two grid-wide
// reductions (reduce-then-release barrier).  Owned rows live in registers.
template <int NS, int RPT, bool PF32>
__global__ void __launch_bounds__(kCoarseThreads) k_coarse_pcg(CoarseCG a) {
  const int64_t n = a.n;
  const int64_t base = (int64_t)blockIdx.x * a.rows_per_block;
  const unsigned expected = gridDim.x + a.phantom_blocks;
  const bool lead = blockIdx.x == 0 && threadIdx.x == 0;
  unsigned gb = 0, gx = 0;   // generations: grid barrier, neighbour exchange
  double x[RPT], r[RPT], p[RPT], z[RPT], S[RPT], d[RPT], rp[RPT], y[RPT], ro[RPT];
  bool live[RPT];
#pragma unroll
  for (int q = 0; q < RPT; ++q) {
    const int64_t g = base + threadIdx.x + (int64_t)q * blockDim.x;
    live[q] = g < n && g < base + a.rows_per_block;
    S[q] = live[q] ? __ldg(&a.invD[g]) : 0.0;
    r[q] = (live[q] && S[q] != 0.0) ? a.b[g] : 0.0;
    x[q] = p[q] = 0.0;
  }
  const double c0 = 4.0 / (3.0 * a.lmax);
  __shared__ CoarseCoef coef;
  __shared__ double s_alpha, s_beta;
  coarse_coef_fill(coef, a.degree, a.lmax);
  __syncthreads();
  // z = M r in FP32 (same recurrence on FP32 copies)
  auto precond_f = [&]() -> bool {
    float df[RPT], rf[RPT], zf[RPT], yf[RPT], sf[RPT];
    const float c0f = (float)c0;
#pragma unroll
    for (int q = 0; q < RPT; ++q) {
      const int64_t g = base + threadIdx.x + (int64_t)q * blockDim.x;
      sf[q] = live[q] ? __ldg(&a.invDf[g]) : 0.f;
      rf[q] = (float)r[q];
      df[q] = c0f * sf[q] * rf[q];
      zf[q] = 0.f;
    }
    for (int i = 1; i < a.degree; ++i) {
#pragma unroll
      for (int q = 0; q < RPT; ++q) zf[q] += df[q];
      publish_tagged<float, RPT>(a, ++gx, df, base);
      if (!coarse_spmv_tagged<float, NS, RPT>(a, gx, base, yf)) return false;
      const float c1 = coef.c1f[i], c2 = coef.c2f[i];
#pragma unroll
      for (int q = 0; q < RPT; ++q) {
        rf[q] -= yf[q];
        df[q] = c1 * df[q] + c2 * sf[q] * rf[q];
      }
    }
#pragma unroll
    for (int q = 0; q < RPT; ++q) z[q] = (double)(zf[q] + df[q]);
    return true;
  };
  // z = M r: Algorithm 2 from a zero guess; returns false on a failed exchange
  auto precond = [&]() -> bool {
    if constexpr (PF32) {
      return precond_f();
    } else {
#pragma unroll
      for (int q = 0; q < RPT; ++q) {
        rp[q] = r[q];
        d[q] = c0 * S[q] * rp[q];
        z[q] = 0.0;
      }
      for (int i = 1; i < a.degree; ++i) {
#pragma unroll
        for (int q = 0; q < RPT; ++q) z[q] += d[q];
        publish_tagged<double, RPT>(a, ++gx, d, base);
        if (!coarse_spmv_tagged<double, NS, RPT>(a, gx, base, y)) return false;
        const double c1 = coef.c1[i], c2 = coef.c2[i];
#pragma unroll
        for (int q = 0; q < RPT; ++q) {
          rp[q] -= y[q];
          d[q] = c1 * d[q] + c2 * S[q] * rp[q];
        }
      }
#pragma unroll
      for (int q = 0; q < RPT; ++q) z[q] += d[q];
      return true;
    }
  };
  auto finish = [&](int status, int it) {
#pragma unroll
    for (int q = 0; q < RPT; ++q) {
      const int64_t g = base + threadIdx.x + (int64_t)q * blockDim.x;
      if (live[q]) a.x[g] = x[q];
    }
    if (lead) {
      a.ctl[2] = (unsigned)status;
      a.ctl[3] = (unsigned)it;
      if (status == CS_BREAKDOWN) atomicMax((int*)&a.ctl[4], (int)CS_BREAKDOWN);
    }
  };
  if (!precond()) return;
  double rz = 0.0, rr = 0.0, zero = 0.0;
#pragma unroll
  for (int q = 0; q < RPT; ++q) {
    p[q] = z[q];
    rz += r[q] * z[q];
    rr += r[q] * r[q];
  }
  block_sum3(rz, rr, zero);
  if (!allreduce3(a.ctl, gb, expected, a.part, rz, rr, zero)) return;
  double gam = rz, bb = rr;
  if (!(bb > 0.0) || !(gam >= 0.0)) {
    finish(bb == 0.0 ? CS_OK : CS_BREAKDOWN, 0);
    return;
  }
  const double tol2 = a.rtol * a.rtol * bb;
  publish_tagged<double, RPT>(a, ++gx, p, base);
  for (int it = 1; it <= a.maxit; ++it) {
    if (!coarse_spmv_tagged<double, NS, RPT>(a, gx, base, y)) return;
    double pq = 0.0, z1 = 0.0, z2 = 0.0;
#pragma unroll
    for (int q = 0; q < RPT; ++q) pq += p[q] * y[q];
    block_sum3(pq, z1, z2);
    if (!allreduce3(a.ctl, gb, expected, a.part, pq, z1, z2)) return;
    const double pq_tot = pq;
    if (!(pq_tot > 0.0)) {
      finish(CS_BREAKDOWN, it);
      return;
    }
    const double alpha = block_div(&s_alpha, gam, pq_tot);
#pragma unroll
    for (int q = 0; q < RPT; ++q) {
      ro[q] = r[q];
      x[q] = fma(alpha, p[q], x[q]);
      r[q] = fma(-alpha, y[q], r[q]);
    }
    if (!precond()) return;
    double rz2 = 0.0, rr2 = 0.0;
    z1 = 0.0;
#pragma unroll
    for (int q = 0; q < RPT; ++q) {
      rz2 += r[q] * z[q];
      rr2 += r[q] * r[q];
      if (PF32) z1 += ro[q] * z[q];
    }
    block_sum3(rz2, rr2, z1);
    if (!allreduce3(a.ctl, gb, expected, a.part, rz2, rr2, z1)) return;
    const double gam_new = rz2, rr_tot = rr2;
    if (!(rr_tot == rr_tot)) {
      finish(CS_BREAKDOWN, it);
      return;
    }
    if (rr_tot <= tol2) {
      finish(CS_OK, it);
      return;
    }
    // Fletcher-Reeves for the exact (symmetric) FP64 preconditioner; Polak-Ribiere
    // (z_new, r_new - r_old) / (z_old, r_old) for the FP32 one
    const double beta = block_div(&s_beta, PF32 ? gam_new - z1 : gam_new, gam);
    gam = gam_new;
#pragma unroll
    for (int q = 0; q < RPT; ++q) p[q] = fma(beta, p[q], z[q]);
    publish_tagged<double, RPT>(a, ++gx, p, base);
  }
  finish(CS_NOTCONV, a.maxit);
}

template <int NS, bool PF32>
static const void* coarse_kernel(int rpt) {
  switch (rpt) {
    case 1: return (const void*)k_coarse_pcg<NS, 1, PF32>;
    case 2: return (const void*)k_coarse_pcg<NS, 2, PF32>;
    case 4: return (const void*)k_coarse_pcg<NS, 4, PF32>;
    default: return (const void*)k_coarse_pcg<NS, 8, PF32>;
  }
}

void coarse_pcg_shape(int64_t n, int rpt_min, int* grid, int* rows_per_block) {
  static int sms = -1;
  if (sms < 0) {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  }
  const int64_t per_block_min = (n + sms - 1) / sms;
  int rpt = 1;
  while (rpt < rpt_min && rpt < kCoarseMaxRowsPerThread) rpt *= 2;
  while ((int64_t)rpt * kCoarseThreads < per_block_min && rpt < kCoarseMaxRowsPerThread) rpt *= 2;
  const int64_t rb = (int64_t)rpt * kCoarseThreads;
  const int64_t g = (n + rb - 1) / rb;
  if (g > sms) {
    *grid = 0;
    *rows_per_block = 0;
    return;
  }
  *grid = (int)std::max<int64_t>(1, g);
  *rows_per_block = (int)rb;
}

bool coarse_pcg_launch(const CoarseCG& a, int grid, cudaStream_t s, cudaError_t* err) {
  CoarseCG arg = a;
  void* params[] = {&arg};
  const int rpt = a.rows_per_block / kCoarseThreads;
  if (grid <= 0 || rpt < 1) {
    if (err) *err = cudaErrorInvalidConfiguration;
    return false;
  }
  const void* fn = a.pf32 ? (a.nslot == 27 ? coarse_kernel<27, true>(rpt) : coarse_kernel<0, true>(rpt))
                         : (a.nslot == 27 ? coarse_kernel<27, false>(rpt) : coarse_kernel<0, false>(rpt));
  cudaError_t e = cudaLaunchCooperativeKernel(fn, dim3(grid), dim3(kCoarseThreads), params, 0, s);
  count();
  if (err) *err = e;
  return e == cudaSuccess;
}

// ===========================================================================
// Lanczos helpers
// ===========================================================================
__global__ void k_splitmix_fill(int64_t n, uint64_t seed, const double* __restrict__ invD, double* __restrict__ v) {
  for (int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; g < n; g += (int64_t)gridDim.x * blockDim.x) {
    // SplitMix64 (Steele, Lea & Flood 2014), output g of the stream seeded with `seed`
    uint64_t z = seed + (uint64_t)(g + 1) * 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    z = z ^ (z >> 31);
    const double u = (double)(z >> 11) * (1.0 / 9007199254740992.0);
    v[g] = invD[g] > 0.0 ? 2.0 * u - 1.0 : 0.0;
  }
}

void splitmix_fill(int64_t n, uint64_t seed, const double* invD, double* v, cudaStream_t s) {
  k_splitmix_fill<<<grid_for(n, kVecThreads), kVecThreads, 0, s>>>(n, seed, invD, v);
  count();
}

__global__ void k_sqrt_scale(int64_t n, const double* __restrict__ invD, const double* __restrict__ v,
                             double* __restrict__ t) {
  for (int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; g < n; g += (int64_t)gridDim.x * blockDim.x)
    t[g] = sqrt(invD[g]) * v[g];
}

void sqrt_scale(int64_t n, const double* invD, const double* v, double* t, cudaStream_t s) {
  k_sqrt_scale<<<grid_for(n, kVecThreads), kVecThreads, 0, s>>>(n, invD, v, t);
  count();
}

__global__ void k_lanczos_w(int64_t n, const double* __restrict__ invD, const double* __restrict__ y,
                            const double* __restrict__ v, const double* __restrict__ vprev, double alpha,
                            double beta, double* __restrict__ w) {
  for (int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; g < n; g += (int64_t)gridDim.x * blockDim.x)
    w[g] = sqrt(invD[g]) * y[g] - alpha * v[g] - beta * vprev[g];
}

void lanczos_w(int64_t n, const double* invD, const double* y, const double* v, const double* vprev,
               double alpha, double beta, double* w, cudaStream_t s) {
  k_lanczos_w<<<grid_for(n, kVecThreads), kVecThreads, 0, s>>>(n, invD, y, v, vprev, alpha, beta, w);
  count();
}

__global__ void k_scale(int64_t n, double a, const double* __restrict__ x, double* __restrict__ y) {
  for (int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; g < n; g += (int64_t)gridDim.x * blockDim.x)
    y[g] = a * x[g];
}

void scale(int64_t n, double a, const double* x, double* y, cudaStream_t s) {
  k_scale<<<grid_for(n, kVecThreads), kVecThreads, 0, s>>>(n, a, x, y);
  count();
}

// ===========================================================================
// explicit instantiations
// ===========================================================================
#define CHEBMG_INST(T)                                                                                \
  template void sem_ax4<T>(int64_t, const uint32_t*, const Lattice*, const T*, const T*, const T*, T*,           \
                           cudaStream_t, int, int64_t);                                                    \
  template void sem_ax<T>(int, int64_t, const uint32_t*, const T*, const T*, const T*, T*, cudaStream_t, int,  \
                          int64_t);                                                                   \
  template void sem_restrict<T>(int, int, int64_t, const uint32_t*, const uint32_t*, const T*, const T*,  \
                                T*, cudaStream_t, int, int64_t, int64_t);                              \
  template void sem_prolong<T>(int, int, int64_t, const uint32_t*, const uint32_t*, const T*, const T*,   \
                               T*, int, cudaStream_t, int, int64_t, int64_t);                          \
  template void fd_apply<T>(int, int, const Stencil9<T>&, const T*, T*, cudaStream_t, int, int64_t);    \
  template void fd_restrict<T>(int, int, int, int, int, const T*, T*, cudaStream_t, int, int64_t, int64_t); \
  template void fd_prolong<T>(int, int, int, int, int, const T*, T*, int, cudaStream_t, int, int64_t,     \
                              int64_t);

CHEBMG_INST(float)
CHEBMG_INST(double)

}  // namespace chebmg
