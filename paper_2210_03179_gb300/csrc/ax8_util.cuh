// Device helpers shared by the order-7 element kernels: shared-memory addresses, the bounded
// mbarrier wait, the TMA bulk copy of the geometric factors with an L2 evict-first hint, and
// the global ids of an element column (element-to-global map or box lattice).
#pragma once
#include <cuda_runtime.h>

#include <cstdint>

#include "common.cuh"

namespace chebmg {
namespace {

__device__ __forceinline__ uint32_t smem_addr(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(smem_addr(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}

constexpr uint32_t kWaitLimit = 1u << 22;

// L2 policy for the geometric factors: each byte is read once per operator application, so the
// copies are marked evict-first and leave the L2 to the vectors that the update kernel reads
// next (the gathered d and the accumulated y).
__device__ __forceinline__ uint64_t evict_first_policy() {
  uint64_t pol;
  asm volatile("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(pol));
  return pol;
}

// One bulk copy global -> shared, completion counted on `bar`, with the evict-first L2 hint.
__device__ __forceinline__ void bulk_copy_g(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes.L2::cache_hint [%0], [%1], %2, [%3], "
      "%4;" ::"r"(smem_addr(dst)),
      "l"(src), "r"(bytes), "r"(smem_addr(bar)), "l"(evict_first_policy())
      : "memory");
}

// Global ids (with the Dirichlet flag) of the column (i = a, j = b, k = 0..7) of element e:
// read from the element-to-global map, or (IMPLICIT) computed from the box lattice, which the
// library's meshes always have -- connectivity of a box, arbitrary vertex positions.  32-bit
// arithmetic (n < 2^30), one division pair per element.
template <bool IMPLICIT>
__device__ __forceinline__ void column_ids(const uint32_t* __restrict__ gid, const Lattice& L, int64_t e,
                                           bool valid, int a, int b, uint32_t (&g)[8]) {
  if (!valid) {
#pragma unroll
    for (int k = 0; k < 8; ++k) g[k] = kGidDirichlet;
    return;
  }
  if constexpr (IMPLICIT) {
    const uint32_t ee = (uint32_t)e;
    const uint32_t exy = (uint32_t)L.nex * (uint32_t)L.ney;
    const uint32_t ez = ee / exy;
    const uint32_t rem = ee - ez * exy;
    const uint32_t ey = rem / (uint32_t)L.nex;
    const uint32_t ex = rem - ey * (uint32_t)L.nex;
    const uint32_t gx = ex * 7 + a, gy = ey * 7 + b;
    const bool side = gx == 0 || gx == (uint32_t)L.NX - 1 || gy == 0 || gy == (uint32_t)L.NY - 1;
    const uint32_t plane = (uint32_t)L.NX * (uint32_t)L.NY;
    const uint32_t g0 = (ez * 7 * (uint32_t)L.NY + gy) * (uint32_t)L.NX + gx;
#pragma unroll
    for (int k = 0; k < 8; ++k) {
      const uint32_t gz = ez * 7 + k;
      const bool bnd = side || gz == 0 || gz == (uint32_t)L.NZ - 1;
      g[k] = (g0 + k * plane) | (bnd ? kGidDirichlet : 0u);
    }
  } else {
#pragma unroll
    for (int k = 0; k < 8; ++k) g[k] = gid[e * 512 + k * 64 + b * 8 + a];
  }
}

}  // namespace
}  // namespace chebmg
