// p-multigrid interpolation and restriction (Sec. 4.1) for fixed order pairs (7->3, 3->1 and
// the 7->5->3 steps of the 7-5-3-1 schedule), on the box lattice of the library's meshes.
//
// P z_c = W Q_f^T (J x J x J) Q_c z_c and P^T r_f = Q_c^T (J^T x J^T x J^T) O^T r_f, where
// O^T keeps each fine node only in its owner element (equal to Q_f W on the continuous range
// of J3 Q_c).  One element per 64 threads, four elements per block; each 1-D contraction is
// done by one thread per grid line with compile-time extents; global ids, ownership and
// Dirichlet flags come from lattice coordinates.
#include <cuda_runtime.h>

#include "common.cuh"

namespace chebmg {

namespace {

// J[fine point][coarse point], one table per supported pair and precision.
__constant__ double c_J84_d[8 * 4];
__constant__ float c_J84_f[8 * 4];
__constant__ double c_J42_d[4 * 2];
__constant__ float c_J42_f[4 * 2];
__constant__ double c_J86_d[8 * 6];
__constant__ float c_J86_f[8 * 6];
__constant__ double c_J64_d[6 * 4];
__constant__ float c_J64_f[6 * 4];

template <typename T, int QF, int QC>
__device__ __forceinline__ T Jv(int f, int c);
template <>
__device__ __forceinline__ double Jv<double, 8, 4>(int f, int c) { return c_J84_d[f * 4 + c]; }
template <>
__device__ __forceinline__ float Jv<float, 8, 4>(int f, int c) { return c_J84_f[f * 4 + c]; }
template <>
__device__ __forceinline__ double Jv<double, 4, 2>(int f, int c) { return c_J42_d[f * 2 + c]; }
template <>
__device__ __forceinline__ float Jv<float, 4, 2>(int f, int c) { return c_J42_f[f * 2 + c]; }
template <>
__device__ __forceinline__ double Jv<double, 8, 6>(int f, int c) { return c_J86_d[f * 6 + c]; }
template <>
__device__ __forceinline__ float Jv<float, 8, 6>(int f, int c) { return c_J86_f[f * 6 + c]; }
template <>
__device__ __forceinline__ double Jv<double, 6, 4>(int f, int c) { return c_J64_d[f * 4 + c]; }
template <>
__device__ __forceinline__ float Jv<float, 6, 4>(int f, int c) { return c_J64_f[f * 4 + c]; }

constexpr int kEB = 4;   // elements per block

struct ElemCoord {
  int ex, ey, ez;
};

__device__ __forceinline__ ElemCoord elem_coord(int64_t e, const Lattice& L) {
  const uint32_t ee = (uint32_t)e;
  const uint32_t exy = (uint32_t)L.nex * (uint32_t)L.ney;
  const uint32_t ez = ee / exy;
  const uint32_t rem = ee - ez * exy;
  const uint32_t ey = rem / (uint32_t)L.nex;
  return {(int)(rem - ey * (uint32_t)L.nex), (int)ey, (int)ez};
}

// Global id of local node (i, j, k) of element (ex, ey, ez) at order N (box lattice L).
__device__ __forceinline__ uint32_t lattice_id(const Lattice& L, int N, ElemCoord c, int i, int j, int k,
                                               bool& dirichlet, bool& owner) {
  const int gx = c.ex * N + i, gy = c.ey * N + j, gz = c.ez * N + k;
  dirichlet = gx == 0 || gx == L.NX - 1 || gy == 0 || gy == L.NY - 1 || gz == 0 || gz == L.NZ - 1;
  owner = (i < N || c.ex == L.nex - 1) && (j < N || c.ey == L.ney - 1) && (k < N || c.ez == L.nez - 1);
  return (uint32_t)(((int64_t)gz * L.NY + gy) * L.NX + gx);
}

// rc += P^T rf (rc zeroed by the caller; coarse contributions summed by atomics)
template <typename T, int QF, int QC>
__global__ void __launch_bounds__(64 * kEB)
k_restrict_box(int64_t E, Lattice Lf, Lattice Lc, const T* __restrict__ rf, T* __restrict__ rc, int64_t ldf,
               int64_t ldc) {
  pdl_wait();   // rf (and the zeroed rc) may come from the kernel before
  rf += (int64_t)blockIdx.y * ldf;   // right-hand side of a batch
  rc += (int64_t)blockIdx.y * ldc;
  constexpr int NF = QF - 1, NC = QC - 1;
  __shared__ T sA[kEB][QF * QF * QF];
  __shared__ T sB[kEB][QF * QF * QC];
  __shared__ T sC[kEB][QF * QC * QC];
  const int le = threadIdx.x >> 6, t = threadIdx.x & 63;
  const int64_t e = (int64_t)blockIdx.x * kEB + le;
  const bool valid = e < E;
  const ElemCoord c = valid ? elem_coord(e, Lf) : ElemCoord{0, 0, 0};
  T* A = sA[le];
  T* B = sB[le];
  T* C = sC[le];
  // fine values at owned, non-Dirichlet copies: every load of the thread in flight at once
  constexpr int NP = (QF * QF * QF + 63) / 64;
  T fv[NP];
#pragma unroll
  for (int q = 0; q < NP; ++q) {
    const int p = t + 64 * q;
    fv[q] = T(0);
    if (p < QF * QF * QF) {
      const int i = p % QF, j = (p / QF) % QF, k = p / (QF * QF);
      bool dir, own;
      const uint32_t g = lattice_id(Lf, NF, c, i, j, k, dir, own);
      if (valid && own && !dir) fv[q] = rf[g];
    }
  }
#pragma unroll
  for (int q = 0; q < NP; ++q)
    if (t + 64 * q < QF * QF * QF) A[t + 64 * q] = fv[q];
  __syncthreads();
  // along i: line (j, k) -> QC outputs
  for (int l = t; l < QF * QF; l += 64) {
    const int j = l % QF, k = l / QF;
    T v[QF];
#pragma unroll
    for (int i = 0; i < QF; ++i) v[i] = A[(k * QF + j) * QF + i];
#pragma unroll
    for (int ic = 0; ic < QC; ++ic) {
      T acc = 0;
#pragma unroll
      for (int i = 0; i < QF; ++i) acc += Jv<T, QF, QC>(i, ic) * v[i];
      B[(k * QF + j) * QC + ic] = acc;
    }
  }
  __syncthreads();
  // along j: line (ic, k)
  for (int l = t; l < QC * QF; l += 64) {
    const int ic = l % QC, k = l / QC;
    T v[QF];
#pragma unroll
    for (int j = 0; j < QF; ++j) v[j] = B[(k * QF + j) * QC + ic];
#pragma unroll
    for (int jc = 0; jc < QC; ++jc) {
      T acc = 0;
#pragma unroll
      for (int j = 0; j < QF; ++j) acc += Jv<T, QF, QC>(j, jc) * v[j];
      C[(k * QC + jc) * QC + ic] = acc;
    }
  }
  __syncthreads();
  // along k: line (ic, jc) -> coarse column, summed into the coarse vector
  for (int l = t; l < QC * QC; l += 64) {
    const int ic = l % QC, jc = l / QC;
    T v[QF];
#pragma unroll
    for (int k = 0; k < QF; ++k) v[k] = C[(k * QC + jc) * QC + ic];
#pragma unroll
    for (int kc = 0; kc < QC; ++kc) {
      T acc = 0;
#pragma unroll
      for (int k = 0; k < QF; ++k) acc += Jv<T, QF, QC>(k, kc) * v[k];
      bool dir, own;
      const uint32_t g = lattice_id(Lc, NC, c, ic, jc, kc, dir, own);
      if (valid && !dir) atomicAdd(&rc[g], acc);
    }
  }
}

// zf (+)= P zc at the owned fine copies
template <typename T, int QF, int QC>
__global__ void __launch_bounds__(64 * kEB)
k_prolong_box(int64_t E, Lattice Lf, Lattice Lc, const T* __restrict__ zc, T* __restrict__ zf, int accumulate,
              int64_t ldf, int64_t ldc) {
  pdl_wait();   // zc and zf may come from the kernels before
  zf += (int64_t)blockIdx.y * ldf;
  zc += (int64_t)blockIdx.y * ldc;
  constexpr int NF = QF - 1, NC = QC - 1;
  __shared__ T sA[kEB][QC * QC * QC];
  __shared__ T sB[kEB][QC * QC * QF];
  __shared__ T sC[kEB][QC * QF * QF];
  const int le = threadIdx.x >> 6, t = threadIdx.x & 63;
  const int64_t e = (int64_t)blockIdx.x * kEB + le;
  const bool valid = e < E;
  const ElemCoord c = valid ? elem_coord(e, Lf) : ElemCoord{0, 0, 0};
  T* A = sA[le];
  T* B = sB[le];
  T* C = sC[le];
  for (int p = t; p < QC * QC * QC; p += 64) {
    const int i = p % QC, j = (p / QC) % QC, k = p / (QC * QC);
    bool dir, own;
    const uint32_t g = lattice_id(Lc, NC, c, i, j, k, dir, own);
    A[p] = (valid && !dir) ? zc[g] : T(0);
  }
  __syncthreads();
  for (int l = t; l < QC * QC; l += 64) {          // along i: line (jc, kc) -> QF outputs
    const int jc = l % QC, kc = l / QC;
    T v[QC];
#pragma unroll
    for (int i = 0; i < QC; ++i) v[i] = A[(kc * QC + jc) * QC + i];
#pragma unroll
    for (int iF = 0; iF < QF; ++iF) {
      T acc = 0;
#pragma unroll
      for (int i = 0; i < QC; ++i) acc += Jv<T, QF, QC>(iF, i) * v[i];
      B[(kc * QC + jc) * QF + iF] = acc;
    }
  }
  __syncthreads();
  for (int l = t; l < QF * QC; l += 64) {          // along j: line (iF, kc)
    const int iF = l % QF, kc = l / QF;
    T v[QC];
#pragma unroll
    for (int j = 0; j < QC; ++j) v[j] = B[(kc * QC + j) * QF + iF];
#pragma unroll
    for (int jF = 0; jF < QF; ++jF) {
      T acc = 0;
#pragma unroll
      for (int j = 0; j < QC; ++j) acc += Jv<T, QF, QC>(jF, j) * v[j];
      C[(kc * QF + jF) * QF + iF] = acc;
    }
  }
  __syncthreads();
  for (int l = t; l < QF * QF; l += 64) {          // along k: fine column (iF, jF)
    const int iF = l % QF, jF = l / QF;
    T v[QC];
#pragma unroll
    for (int k = 0; k < QC; ++k) v[k] = C[(k * QF + jF) * QF + iF];
    // the column's ids and (accumulate) old values first: all loads in flight at once instead
    // of one load-store round trip per output
    uint32_t g[QF];
    bool wr[QF], dz[QF];
    T old[QF];
#pragma unroll
    for (int kF = 0; kF < QF; ++kF) {
      bool dir, own;
      g[kF] = lattice_id(Lf, NF, c, iF, jF, kF, dir, own);
      wr[kF] = valid && own;
      dz[kF] = dir;
      old[kF] = (accumulate && wr[kF] && !dir) ? zf[g[kF]] : T(0);
    }
#pragma unroll
    for (int kF = 0; kF < QF; ++kF) {
      if (!wr[kF]) continue;
      if (dz[kF]) {
        if (!accumulate) zf[g[kF]] = T(0);
        continue;
      }
      T acc = 0;
#pragma unroll
      for (int k = 0; k < QC; ++k) acc += Jv<T, QF, QC>(kF, k) * v[k];
      zf[g[kF]] = accumulate ? old[kF] + acc : acc;
    }
  }
}

}  // namespace

template <int QF, int QC>
static cudaError_t set_J(const double* J, const void* sym_d, const void* sym_f) {
  float f[QF * QC];
  for (int q = 0; q < QF * QC; ++q) f[q] = (float)J[q];
  cudaError_t e = cudaMemcpyToSymbol(sym_d, J, sizeof(double) * QF * QC);
  return e != cudaSuccess ? e : cudaMemcpyToSymbol(sym_f, f, sizeof(f));
}

cudaError_t transfer_box_set_J(int Qf, int Qc, const double* J) {
  if (Qf == 8 && Qc == 4) return set_J<8, 4>(J, c_J84_d, c_J84_f);
  if (Qf == 4 && Qc == 2) return set_J<4, 2>(J, c_J42_d, c_J42_f);
  if (Qf == 8 && Qc == 6) return set_J<8, 6>(J, c_J86_d, c_J86_f);
  if (Qf == 6 && Qc == 4) return set_J<6, 4>(J, c_J64_d, c_J64_f);
  return cudaErrorInvalidValue;
}

bool transfer_box_supported(int Qf, int Qc) {
  return (Qf == 8 && Qc == 4) || (Qf == 4 && Qc == 2) || (Qf == 8 && Qc == 6) || (Qf == 6 && Qc == 4);
}

template <typename T>
void restrict_box(int Qf, int Qc, int64_t E, const Lattice& Lf, const Lattice& Lc, const T* rf, T* rc,
                  cudaStream_t s, int nb, int64_t ldf, int64_t ldc) {
  const dim3 blocks((unsigned)((E + kEB - 1) / kEB), nb);
  if (Qf == 8 && Qc == 4) launch_dep(k_restrict_box<T, 8, 4>, blocks, dim3(64 * kEB), 0, s, E, Lf, Lc, rf, rc, ldf, ldc);
  else if (Qf == 8 && Qc == 6)
    launch_dep(k_restrict_box<T, 8, 6>, blocks, dim3(64 * kEB), 0, s, E, Lf, Lc, rf, rc, ldf, ldc);
  else if (Qf == 6 && Qc == 4)
    launch_dep(k_restrict_box<T, 6, 4>, blocks, dim3(64 * kEB), 0, s, E, Lf, Lc, rf, rc, ldf, ldc);
  else launch_dep(k_restrict_box<T, 4, 2>, blocks, dim3(64 * kEB), 0, s, E, Lf, Lc, rf, rc, ldf, ldc);
}

template <typename T>
void prolong_box(int Qf, int Qc, int64_t E, const Lattice& Lf, const Lattice& Lc, const T* zc, T* zf,
                 int accumulate, cudaStream_t s, int nb, int64_t ldf, int64_t ldc) {
  const dim3 blocks((unsigned)((E + kEB - 1) / kEB), nb);
  if (Qf == 8 && Qc == 4)
    launch_dep(k_prolong_box<T, 8, 4>, blocks, dim3(64 * kEB), 0, s, E, Lf, Lc, zc, zf, accumulate, ldf, ldc);
  else if (Qf == 8 && Qc == 6)
    launch_dep(k_prolong_box<T, 8, 6>, blocks, dim3(64 * kEB), 0, s, E, Lf, Lc, zc, zf, accumulate, ldf, ldc);
  else if (Qf == 6 && Qc == 4)
    launch_dep(k_prolong_box<T, 6, 4>, blocks, dim3(64 * kEB), 0, s, E, Lf, Lc, zc, zf, accumulate, ldf, ldc);
  else
    launch_dep(k_prolong_box<T, 4, 2>, blocks, dim3(64 * kEB), 0, s, E, Lf, Lc, zc, zf, accumulate, ldf, ldc);
}

template void restrict_box<float>(int, int, int64_t, const Lattice&, const Lattice&, const float*, float*,
                                  cudaStream_t, int, int64_t, int64_t);
template void restrict_box<double>(int, int, int64_t, const Lattice&, const Lattice&, const double*, double*,
                                   cudaStream_t, int, int64_t, int64_t);
template void prolong_box<float>(int, int, int64_t, const Lattice&, const Lattice&, const float*, float*, int,
                                 cudaStream_t, int, int64_t, int64_t);
template void prolong_box<double>(int, int, int64_t, const Lattice&, const Lattice&, const double*, double*, int,
                                  cudaStream_t, int, int64_t, int64_t);

}  // namespace chebmg
