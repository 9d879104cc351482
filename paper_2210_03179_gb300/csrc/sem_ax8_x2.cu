// The order-7 element operator in FP64-class arithmetic on FP32 pairs (f32x2.cuh), for the
// outer Krylov product of the mixed form.  GB300 executes FP32 at a large multiple of its FP64
// rate, and the FP64 operator runs at that FP64 roof; the same operator with every
// multiply-add on FP32 pairs (about 48 significant bits) costs about ten
// FP32 operations per FP64 one and runs faster, with errors near 1e-14 relative.
//
// Same structure as k_sem_ax8 (Sec. 1, Eq. 1.3): one element per 64 threads, line passes
// with the even-odd factorisation of D, geometric factors by one TMA bulk copy per block
// (stored as FP32 pairs, 8 bytes per value like FP64), gathered vector values converted from
// FP64, element results converted back to FP64 for the direct-stiffness atomics.
#include <cuda_runtime.h>

#include "ax8_util.cuh"
#include "common.cuh"
#include "f32x2.cuh"

namespace chebmg {

namespace {

// even-odd blocks as FP32 pairs: [0] E of D, [1] O of D, [2] E of D^T, [3] O of D^T
__constant__ f32x2 c_eo_x2[4][4][4];

constexpr int kR = 10, kP = 88, kStage = 8 * kP, kGElem = 6 * 512;   // same strides as FP64

template <int W>
__device__ __forceinline__ void line8_x2(const f32x2 (&u)[8], f32x2 (&o)[8]) {
  f32x2 ue[4], uo[4];
#pragma unroll
  for (int l = 0; l < 4; ++l) {
    ue[l] = x2_add(u[l], u[7 - l]);
    uo[l] = x2_sub(u[l], u[7 - l]);
  }
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    f32x2 se = x2_mul(c_eo_x2[2 * W][i][0], ue[0]);
    f32x2 so = x2_mul(c_eo_x2[2 * W + 1][i][0], uo[0]);
#pragma unroll
    for (int l = 1; l < 4; ++l) {
      se = x2_fma(c_eo_x2[2 * W][i][l], ue[l], se);
      so = x2_fma(c_eo_x2[2 * W + 1][i][l], uo[l], so);
    }
    o[i] = x2_add(se, so);
    o[7 - i] = x2_sub(so, se);
  }
}

// Applies the operator to right-hand sides q0 .. q1-1 of a batch (vector q at u + q * ld,
// y + q * ld): the geometric factors are staged once, and the gather of the next right-hand
// side is in flight while the current one is computed.  A single vector is the batch of one.
template <int EB, bool IMPLICIT>
__global__ void __launch_bounds__(64 * EB)
k_sem_ax8_x2(int64_t E, const uint32_t* __restrict__ gid, Lattice lat, const f32x2* __restrict__ G,
             const double* __restrict__ u, double* __restrict__ y, unsigned* __restrict__ err, int nb, int64_t ld,
             int rb) {
  extern __shared__ __align__(128) unsigned char smem_raw[];
  __shared__ __align__(8) uint64_t bar;
  f32x2* sG = reinterpret_cast<f32x2*>(smem_raw);
  f32x2* sU = sG + EB * kGElem;
  f32x2* sR = sU + EB * kStage;
  f32x2* sS = sR + EB * kStage;

  const int tid = threadIdx.x;
  const int le = tid >> 6, t = tid & 63, a = t & 7, b = t >> 3;
  const int64_t e0 = (int64_t)blockIdx.x * EB;
  const int nvalid = (int)((E - e0) < EB ? (E - e0) : EB);
  const bool valid = le < nvalid;
  const int64_t e = e0 + le;
  const int q0 = blockIdx.y * rb;
  const int q1 = q0 + rb < nb ? q0 + rb : nb;

  if (tid == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_addr(&bar)) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();
  if (tid == 0) {
    const uint32_t bytes = (uint32_t)(nvalid * kGElem * sizeof(f32x2));
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(&bar)), "r"(bytes)
                 : "memory");
    bulk_copy_g(sG, G + e0 * kGElem, bytes, &bar);
  }

  f32x2* su = sU + le * kStage;
  f32x2* sr = sR + le * kStage;
  f32x2* ss = sS + le * kStage;

  // gather: thread (i = a, j = b) owns the column along t
  uint32_t g[8];
  column_ids<IMPLICIT>(gid, lat, e, valid, a, b, g);
  auto gather = [&](int q, double (&v)[8]) {
    const double* uq = u + (int64_t)q * ld;
#pragma unroll
    for (int k = 0; k < 8; ++k) v[k] = (q < q1 && !(g[k] & kGidDirichlet)) ? uq[g[k] & kGidMask] : 0.0;
  };
  double cv[8];
  gather(q0, cv);
  for (int q = q0; q < q1; ++q) {
    f32x2 col[8];
#pragma unroll
    for (int k = 0; k < 8; ++k) {
      col[k] = x2_from(cv[k]);
      su[k * kP + b * kR + a] = col[k];
    }
    gather(q + 1, cv);   // next right-hand side's loads overlap this one's work
    f32x2 ut[8];
    line8_x2<0>(col, ut);
    __syncthreads();
    // r (thread (j = a, k = b) owns the row along i) and s (thread (i = a, k = b) owns the line
    // along j) in one loop: the pair arithmetic is long, and one copy of the pass keeps the
    // kernel's code within the instruction cache
#pragma unroll 1
    for (int d = 0; d < 2; ++d) {
      const int base = d == 0 ? b * kP + a * kR : b * kP + a, stride = d == 0 ? 1 : kR;
      f32x2 v[8], o[8];
#pragma unroll
      for (int j = 0; j < 8; ++j) v[j] = su[base + j * stride];
      line8_x2<0>(v, o);
      f32x2* dst = d == 0 ? sr : ss;
#pragma unroll
      for (int j = 0; j < 8; ++j) dst[base + j * stride] = o[j];
    }
    if (q == q0) {   // geometric factors must have landed (once per block)
      bool ok = false;
      for (uint32_t it = 0; it < kWaitLimit; ++it)
        if (mbar_try_wait(&bar, 0)) {
          ok = true;
          break;
        }
      if (!__syncthreads_and(ok ? 1 : 0)) {
        if (tid == 0) atomicExch(err, 1u);
        for (uint32_t it = 0; it < kWaitLimit; ++it)
          if (mbar_try_wait(&bar, 0)) break;
        return;
      }
    } else {
      __syncthreads();   // the line passes above wrote points other threads read next
    }
    f32x2 wt[8];
    const f32x2* gG = sG + le * kGElem;
#pragma unroll
    for (int k = 0; k < 8; ++k) {
      const int p = k * 64 + b * 8 + a;
      const int qq = k * kP + b * kR + a;
      const f32x2 ur = sr[qq], us = ss[qq], utk = ut[k];
      const f32x2 g00 = gG[p], g01 = gG[512 + p], g02 = gG[1024 + p];
      const f32x2 g11 = gG[1536 + p], g12 = gG[2048 + p], g22 = gG[2560 + p];
      sr[qq] = x2_fma(g02, utk, x2_fma(g01, us, x2_mul(g00, ur)));
      ss[qq] = x2_fma(g12, utk, x2_fma(g11, us, x2_mul(g01, ur)));
      wt[k] = x2_fma(g22, utk, x2_fma(g12, us, x2_mul(g02, ur)));
    }
    f32x2 yt[8];
    line8_x2<1>(wt, yt);
    __syncthreads();
    // transposed r into su, then transposed s added to it (the s lines cross the r rows that
    // other threads wrote: a barrier in between)
#pragma unroll 1
    for (int d = 0; d < 2; ++d) {
      const int base = d == 0 ? b * kP + a * kR : b * kP + a, stride = d == 0 ? 1 : kR;
      const f32x2* src = d == 0 ? sr : ss;
      f32x2 v[8], o[8];
#pragma unroll
      for (int j = 0; j < 8; ++j) v[j] = src[base + j * stride];
      line8_x2<1>(v, o);
#pragma unroll
      for (int j = 0; j < 8; ++j) su[base + j * stride] = d == 0 ? o[j] : x2_add(su[base + j * stride], o[j]);
      __syncthreads();
    }
    if (valid) {
      double* yq = y + (int64_t)q * ld;
#pragma unroll
      for (int k = 0; k < 8; ++k) {
        const f32x2 v = x2_add(su[k * kP + b * kR + a], yt[k]);
        if (!(g[k] & kGidDirichlet)) atomicAdd(&yq[g[k] & kGidMask], x2_to_double(v));
      }
    }
    __syncthreads();   // stage buffers free for the next right-hand side
  }
}

__global__ void k_to_x2(int64_t n, const double* __restrict__ in, f32x2* __restrict__ out) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    out[i] = x2_from(in[i]);
}

size_t smem_x2(int eb) { return sizeof(f32x2) * (size_t)eb * (kGElem + 3 * kStage); }

template <int EB, bool IM>
void launch_x2(int64_t E, const uint32_t* gid, const Lattice& lat, const f32x2* G, const double* u, double* y,
               unsigned* err, int nb, int64_t ld, int rb, cudaStream_t s) {
  static bool configured = false;
  if (!configured) {
    cudaFuncSetAttribute(k_sem_ax8_x2<EB, IM>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_x2(EB));
    configured = true;
  }
  if (rb < 1) rb = 1;
  const dim3 blocks((unsigned)((E + EB - 1) / EB), (unsigned)((nb + rb - 1) / rb));
  k_sem_ax8_x2<EB, IM><<<blocks, 64 * EB, smem_x2(EB), s>>>(E, gid, lat, G, u, y, err, nb, ld, rb);
  g_launches.fetch_add(1, std::memory_order_relaxed);
}

}  // namespace

cudaError_t sem_ax8_x2_set_eo(const double* h) {
  f32x2 t[64];
  for (int q = 0; q < 64; ++q) {
    const float hi = (float)h[q];
    t[q] = {hi, (float)(h[q] - (double)hi)};
  }
  return cudaMemcpyToSymbol(c_eo_x2, t, sizeof(t));
}

void sem_to_x2(int64_t n, const double* in, void* out, cudaStream_t s) {
  const int64_t want = (n + 255) / 256;
  k_to_x2<<<(unsigned)(want < 152 * 32 ? want : 152 * 32), 256, 0, s>>>(n, in, static_cast<f32x2*>(out));
  g_launches.fetch_add(1, std::memory_order_relaxed);
}

void sem_ax8_x2(int64_t E, const uint32_t* gid, const Lattice& lat, const void* G, const double* u, double* y,
                unsigned* err, int variant, cudaStream_t s, int nb, int64_t ld, int rb) {
  const f32x2* Gx = static_cast<const f32x2*>(G);
  const bool im = variant >= 100;
  const int eb = variant % 100;
  if (im) {
    if (eb == 1) launch_x2<1, true>(E, gid, lat, Gx, u, y, err, nb, ld, rb, s);
    else if (eb == 4) launch_x2<4, true>(E, gid, lat, Gx, u, y, err, nb, ld, rb, s);
    else launch_x2<2, true>(E, gid, lat, Gx, u, y, err, nb, ld, rb, s);
  } else {
    if (eb == 1) launch_x2<1, false>(E, gid, lat, Gx, u, y, err, nb, ld, rb, s);
    else if (eb == 4) launch_x2<4, false>(E, gid, lat, Gx, u, y, err, nb, ld, rb, s);
    else launch_x2<2, false>(E, gid, lat, Gx, u, y, err, nb, ld, rb, s);
  }
}

}  // namespace chebmg
