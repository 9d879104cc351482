// Building blocks of the order-7 element operator (N = 7, 8 GLL points per direction), shared
// by the operator kernels (sem_ax8.cu) and the fused smoother (sem_smooth8.cu): the shared-memory
// layout of one element, the even-odd line derivative and 8-point row loads / stores.
//
// Even-odd factorisation: the GLL derivative matrix is centro-antisymmetric,
// D[7-i][7-l] = -D[i][l], so (D u)[i] = E_i.(u_l + u_{7-l}) + O_i.(u_l - u_{7-l}) and
// (D u)[7-i] = O_i.(...) - E_i.(...) with 4 x 4 blocks E and O.  Each translation unit that
// includes this header has its own copy of the constant blocks and uploads them itself.
#pragma once
#include <cuda_runtime.h>

#include <cstdint>

namespace chebmg {
namespace {

// even-odd blocks: [0] E of D, [1] O of D, [2] E of D^T, [3] O of D^T, each [i][l], i,l < 4
__constant__ float c_eo_f[4][4][4];
__constant__ double c_eo_d[4][4][4];

template <typename T, int EB_ = 2>
struct Ax8 {
  static constexpr int EB = EB_;                       // elements per block
  static constexpr int R = sizeof(T) == 4 ? 12 : 10;   // padded row stride (16-B aligned rows)
  static constexpr int P = sizeof(T) == 4 ? 104 : 88;  // padded plane stride (bank spread)
  static constexpr int STAGE = 8 * P;
  static constexpr int GELEM = 6 * 512;
  static size_t smem_bytes() { return sizeof(T) * (size_t)EB * (GELEM + 3 * STAGE); }
};

template <typename T>
__device__ __forceinline__ T eo(int w, int i, int l);
template <>
__device__ __forceinline__ float eo<float>(int w, int i, int l) { return c_eo_f[w][i][l]; }
template <>
__device__ __forceinline__ double eo<double>(int w, int i, int l) { return c_eo_d[w][i][l]; }

// o = D u (W = 0) or o = D^T u (W = 1) along one line of 8 points.
template <typename T, int W>
__device__ __forceinline__ void line8(const T (&u)[8], T (&o)[8]) {
  T ue[4], uo[4];
#pragma unroll
  for (int l = 0; l < 4; ++l) {
    ue[l] = u[l] + u[7 - l];
    uo[l] = u[l] - u[7 - l];
  }
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    T se = eo<T>(2 * W, i, 0) * ue[0];
#pragma unroll
    for (int l = 1; l < 4; ++l) se = fma(eo<T>(2 * W, i, l), ue[l], se);
    if constexpr (sizeof(T) == 8) {
      // FP64 (bound by its FP64 issue rate): the odd chain continues from se, giving
      // o[i] = se + so directly, and o[7-i] = so - se = o[i] - 2 se in one more FMA
      // (9 operations per output pair instead of 10)
      T s = se;
#pragma unroll
      for (int l = 0; l < 4; ++l) s = fma(eo<T>(2 * W + 1, i, l), uo[l], s);
      o[i] = s;
      o[7 - i] = fma(T(-2), se, s);
    } else {
      T so = eo<T>(2 * W + 1, i, 0) * uo[0];
#pragma unroll
      for (int l = 1; l < 4; ++l) so = fma(eo<T>(2 * W + 1, i, l), uo[l], so);
      o[i] = se + so;
      o[7 - i] = so - se;
    }
  }
}

__device__ __forceinline__ void ld_row(const float* p, float (&v)[8]) {
  const float4 a = reinterpret_cast<const float4*>(p)[0], b = reinterpret_cast<const float4*>(p)[1];
  v[0] = a.x; v[1] = a.y; v[2] = a.z; v[3] = a.w; v[4] = b.x; v[5] = b.y; v[6] = b.z; v[7] = b.w;
}
__device__ __forceinline__ void st_row(float* p, const float (&v)[8]) {
  reinterpret_cast<float4*>(p)[0] = make_float4(v[0], v[1], v[2], v[3]);
  reinterpret_cast<float4*>(p)[1] = make_float4(v[4], v[5], v[6], v[7]);
}
__device__ __forceinline__ void ld_row(const double* p, double (&v)[8]) {
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    const double2 a = reinterpret_cast<const double2*>(p)[q];
    v[2 * q] = a.x;
    v[2 * q + 1] = a.y;
  }
}
__device__ __forceinline__ void st_row(double* p, const double (&v)[8]) {
#pragma unroll
  for (int q = 0; q < 4; ++q) reinterpret_cast<double2*>(p)[q] = make_double2(v[2 * q], v[2 * q + 1]);
}


}  // namespace
}  // namespace chebmg
