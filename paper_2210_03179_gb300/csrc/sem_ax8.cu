// Element operator for polynomial order N = 7 (8 GLL points per direction), the
// order of the finest p-multigrid level.
//
// Same operator as k_sem_ax (Sec. 1, Eq. 1.3: y_e = sum_m Dhat_m^T sum_n G_mn Dhat_n u_e,
// then direct-stiffness summation), organised for GB300:
//
// * Line passes.  64 threads per element; in each of the six 1-D contractions a thread owns
//   one whole grid line (a column along t, a row along r, a line along s), loads its 8 values
//   once and produces 8 outputs, so one shared-memory load feeds 8 FMAs.  The t-direction
//   line stays in registers.
// * Even-odd factorisation.  The GLL derivative matrix is centro-antisymmetric,
//   D[7-i][7-l] = -D[i][l], so (D u)[i] = E_i.(u_l + u_{7-l}) + O_i.(u_l - u_{7-l}) and
//   (D u)[7-i] = O_i.(...) - E_i.(...) with 4x4 blocks E, O: 48 instead of 64 operations per
//   line (44 in FP64, whose odd chain continues the even one), which matters for the FP64
//   form (GB300 issues few FP64 FMAs per clock).
// * Geometric factors by TMA.  G is stored [E][6][512], so the EB elements of a block are
//   one contiguous span; a single elected thread issues one cp.async.bulk into shared memory
//   at kernel start, completion tracked by an mbarrier, and the block overlaps it with the
//   gather and the first three contractions.  The wait is bounded: on timeout the block
//   records an error flag and skips its stores instead of hanging.
#include <cuda_runtime.h>

#include "ax8_core.cuh"
#include "ax8_util.cuh"
#include "common.cuh"

namespace chebmg {

namespace {

template <typename T, int EB_, bool IMPLICIT>
__global__ void __launch_bounds__(64 * EB_)
k_sem_ax8(int64_t E, const uint32_t* __restrict__ gid, Lattice lat, const T* __restrict__ G,
          const T* __restrict__ u, T* __restrict__ y, unsigned* __restrict__ err) {
  using C = Ax8<T, EB_>;
  constexpr int EB = C::EB, R = C::R, P = C::P;
  extern __shared__ __align__(128) unsigned char smem_raw[];
  __shared__ __align__(8) uint64_t bar;
  T* sG = reinterpret_cast<T*>(smem_raw);
  T* sU = sG + EB * C::GELEM;
  T* sR = sU + EB * C::STAGE;
  T* sS = sR + EB * C::STAGE;

  const int tid = threadIdx.x;
  const int le = tid >> 6, t = tid & 63, a = t & 7, b = t >> 3;
  const int64_t e0 = (int64_t)blockIdx.x * EB;
  const int nvalid = (int)((E - e0) < EB ? (E - e0) : EB);
  const bool valid = le < nvalid;
  const int64_t e = e0 + le;

  if (tid == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_addr(&bar)) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();
  if (tid == 0) {
    const uint32_t bytes = (uint32_t)(nvalid * C::GELEM * sizeof(T));
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(&bar)), "r"(bytes)
                 : "memory");
    bulk_copy_g(sG, G + e0 * C::GELEM, bytes, &bar);
  }
  pdl_wait();   // u and y may come from the kernel before (programmatic dependent launch)

  T* su = sU + le * C::STAGE;
  T* sr = sR + le * C::STAGE;
  T* ss = sS + le * C::STAGE;

  // gather: thread (i = a, j = b) owns the column along t
  uint32_t g[8];
  T col[8];
  column_ids<IMPLICIT>(gid, lat, e, valid, a, b, g);
#pragma unroll
  for (int k = 0; k < 8; ++k) {
    col[k] = (g[k] & kGidDirichlet) ? T(0) : u[g[k] & kGidMask];
    su[k * P + b * R + a] = col[k];
  }
  T ut[8];
  line8<T, 0>(col, ut);
  __syncthreads();
  {
    T v[8], o[8];
    // r: thread (j = a, k = b) owns the row along i
    ld_row(su + b * P + a * R, v);
    line8<T, 0>(v, o);
    st_row(sr + b * P + a * R, o);
    // s: thread (i = a, k = b) owns the line along j
#pragma unroll
    for (int j = 0; j < 8; ++j) v[j] = su[b * P + j * R + a];
    line8<T, 0>(v, o);
#pragma unroll
    for (int j = 0; j < 8; ++j) ss[b * P + j * R + a] = o[j];
  }
  // geometric factors must have landed
  bool ok = false;
  for (uint32_t it = 0; it < kWaitLimit; ++it)
    if (mbar_try_wait(&bar, 0)) {
      ok = true;
      break;
    }
  // every thread takes the same branch: the block agrees on the outcome
  if (!__syncthreads_and(ok ? 1 : 0)) {
    if (tid == 0) atomicExch(err, 1u);
    for (uint32_t it = 0; it < kWaitLimit; ++it)   // let the copy in flight finish before leaving
      if (mbar_try_wait(&bar, 0)) break;
    return;
  }
  T wt[8];
  const T* gG = sG + le * C::GELEM;
#pragma unroll
  for (int k = 0; k < 8; ++k) {
    const int p = k * 64 + b * 8 + a;
    const int q = k * P + b * R + a;
    const T ur = sr[q], us = ss[q], utk = ut[k];
    const T g00 = gG[p], g01 = gG[512 + p], g02 = gG[1024 + p];
    const T g11 = gG[1536 + p], g12 = gG[2048 + p], g22 = gG[2560 + p];
    sr[q] = g00 * ur + g01 * us + g02 * utk;
    ss[q] = g01 * ur + g11 * us + g12 * utk;
    wt[k] = g02 * ur + g12 * us + g22 * utk;
  }
  T yt[8];
  line8<T, 1>(wt, yt);
  __syncthreads();
  {
    T v[8], o[8];
    ld_row(sr + b * P + a * R, v);          // transposed r, thread (j = a, k = b)
    line8<T, 1>(v, o);
    st_row(su + b * P + a * R, o);
  }
  __syncthreads();
  {
    T v[8], o[8];
#pragma unroll
    for (int j = 0; j < 8; ++j) v[j] = ss[b * P + j * R + a];   // transposed s, thread (i = a, k = b)
    line8<T, 1>(v, o);
#pragma unroll
    for (int j = 0; j < 8; ++j) su[b * P + j * R + a] += o[j];
  }
  __syncthreads();
  if (valid) {
#pragma unroll
    for (int k = 0; k < 8; ++k) {
      const T v = su[k * P + b * R + a] + yt[k];
      if (!(g[k] & kGidDirichlet)) atomicAdd(&y[g[k] & kGidMask], v);
    }
  }
}

// Variant without the shared-memory copy of the geometric factors: each point's six factors
// are read from global memory in the step that uses them (coalesced across the element's
// threads).  Only the three stage buffers stay in shared memory, so several times more blocks
// are resident per SM -- for the FP64 form, bound by its FP64 issue rate, more warps ready to
// issue while others gather or scatter.
template <typename T, int EB_, bool IMPLICIT>
__global__ void __launch_bounds__(64 * EB_)
k_sem_ax8g(int64_t E, const uint32_t* __restrict__ gid, Lattice lat, const T* __restrict__ G,
           const T* __restrict__ u, T* __restrict__ y) {
  using C = Ax8<T, EB_>;
  constexpr int R = C::R, P = C::P;
  extern __shared__ __align__(128) unsigned char smem_raw[];
  T* sU = reinterpret_cast<T*>(smem_raw);
  T* sR = sU + EB_ * C::STAGE;
  T* sS = sR + EB_ * C::STAGE;
  const int tid = threadIdx.x;
  const int le = tid >> 6, t = tid & 63, a = t & 7, b = t >> 3;
  const int64_t e = (int64_t)blockIdx.x * EB_ + le;
  const bool valid = e < E;
  T* su = sU + le * C::STAGE;
  T* sr = sR + le * C::STAGE;
  T* ss = sS + le * C::STAGE;
  uint32_t g[8];
  T col[8];
  column_ids<IMPLICIT>(gid, lat, e, valid, a, b, g);
  pdl_wait();   // u and y may come from the kernel before (programmatic dependent launch)
#pragma unroll
  for (int k = 0; k < 8; ++k) {
    col[k] = (g[k] & kGidDirichlet) ? T(0) : u[g[k] & kGidMask];
    su[k * P + b * R + a] = col[k];
  }
  T ut[8];
  line8<T, 0>(col, ut);
  __syncthreads();
  {
    T v[8], o[8];
    ld_row(su + b * P + a * R, v);
    line8<T, 0>(v, o);
    st_row(sr + b * P + a * R, o);
#pragma unroll
    for (int j = 0; j < 8; ++j) v[j] = su[b * P + j * R + a];
    line8<T, 0>(v, o);
#pragma unroll
    for (int j = 0; j < 8; ++j) ss[b * P + j * R + a] = o[j];
  }
  __syncthreads();
  T wt[8];
  const T* gG = G + (valid ? e : 0) * C::GELEM;
#pragma unroll
  for (int k = 0; k < 8; ++k) {
    const int p = k * 64 + b * 8 + a;
    const int q = k * P + b * R + a;
    const T ur = sr[q], us = ss[q], utk = ut[k];
    const T g00 = __ldg(gG + p), g01 = __ldg(gG + 512 + p), g02 = __ldg(gG + 1024 + p);
    const T g11 = __ldg(gG + 1536 + p), g12 = __ldg(gG + 2048 + p), g22 = __ldg(gG + 2560 + p);
    sr[q] = g00 * ur + g01 * us + g02 * utk;
    ss[q] = g01 * ur + g11 * us + g12 * utk;
    wt[k] = g02 * ur + g12 * us + g22 * utk;
  }
  T yt[8];
  line8<T, 1>(wt, yt);
  __syncthreads();
  {
    T v[8], o[8];
    ld_row(sr + b * P + a * R, v);
    line8<T, 1>(v, o);
    st_row(su + b * P + a * R, o);
  }
  __syncthreads();
  {
    T v[8], o[8];
#pragma unroll
    for (int j = 0; j < 8; ++j) v[j] = ss[b * P + j * R + a];
    line8<T, 1>(v, o);
#pragma unroll
    for (int j = 0; j < 8; ++j) su[b * P + j * R + a] += o[j];
  }
  __syncthreads();
  if (valid) {
#pragma unroll
    for (int k = 0; k < 8; ++k) {
      const T v = su[k * P + b * R + a] + yt[k];
      if (!(g[k] & kGidDirichlet)) atomicAdd(&y[g[k] & kGidMask], v);
    }
  }
}

// Persistent, software-pipelined variant: each block walks batches of EB elements
// (blockIdx.x, blockIdx.x + gridDim.x, ...), and batch i+1's gather (element-to-global ids
// and u values) is in flight into registers while batch i is computed.  NB = 2: the TMA copy
// of batch i+1's geometric factors runs into the second buffer during all of batch i.  NB = 1
// (half the shared memory, so more blocks per SM): one buffer, refilled for batch i+1 as soon
// as batch i's factor multiply has read it, so the copy overlaps the transposed passes, the
// scatter and batch i+1's forward passes.  Waits on the copies are bounded like in k_sem_ax8.
template <typename T, int EB, bool IMPLICIT, int NB = 2>
__global__ void __launch_bounds__(64 * EB)
k_sem_ax8p(int64_t E, const uint32_t* __restrict__ gid, Lattice lat, const T* __restrict__ G,
           const T* __restrict__ u, T* __restrict__ y, unsigned* __restrict__ err) {
  static_assert(NB == 1 || NB == 2, "one or two geometric-factor buffers");
  using C = Ax8<T, EB>;
  constexpr int R = C::R, P = C::P;
  extern __shared__ __align__(128) unsigned char smem_raw[];
  __shared__ __align__(8) uint64_t bar[2];
  T* sG = reinterpret_cast<T*>(smem_raw);                 // [NB][EB * GELEM]
  T* sU = sG + NB * EB * C::GELEM;
  T* sR = sU + EB * C::STAGE;
  T* sS = sR + EB * C::STAGE;
  const int tid = threadIdx.x;
  const int le = tid >> 6, t = tid & 63, a = t & 7, b = t >> 3;
  const int64_t nbatch = (E + EB - 1) / EB;
  int64_t batch = blockIdx.x;
  if (batch >= nbatch) return;

  if (tid == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_addr(&bar[0])) : "memory");
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_addr(&bar[1])) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();
  auto issue = [&](int64_t bt, int buf) {
    const int64_t e0 = bt * EB;
    const int nv = (int)((E - e0) < EB ? (E - e0) : EB);
    const uint32_t bytes = (uint32_t)(nv * C::GELEM * sizeof(T));
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(&bar[buf])), "r"(bytes)
                 : "memory");
    bulk_copy_g(sG + buf * EB * C::GELEM, G + e0 * C::GELEM, bytes, &bar[buf]);
  };
  auto gather = [&](int64_t bt, uint32_t (&g)[8], T (&v)[8]) {
    const int64_t e = bt * EB + le;
    const bool valid = bt < nbatch && e < E;
    column_ids<IMPLICIT>(gid, lat, e, valid, a, b, g);
#pragma unroll
    for (int k = 0; k < 8; ++k) v[k] = (g[k] & kGidDirichlet) ? T(0) : u[g[k] & kGidMask];
  };
  if (tid == 0) issue(batch, 0);
  // u and y may come from the kernel before (programmatic dependent launch): wait for it now,
  // after the first geometric-factor copy (G is never written by the solve) is on its way.
  pdl_wait();
  uint32_t g[8];
  T col[8];
  gather(batch, g, col);
  uint32_t phase = 0;   // bit `buf`: parity of the next wait on bar[buf]
  T* su = sU + le * C::STAGE;
  T* sr = sR + le * C::STAGE;
  T* ss = sS + le * C::STAGE;
  for (int it = 0; batch < nbatch; ++it, batch += gridDim.x) {
    const int buf = NB == 2 ? (it & 1) : 0;
    const int64_t next = batch + gridDim.x;
    if (NB == 2 && tid == 0 && next < nbatch) issue(next, buf ^ 1);
#pragma unroll
    for (int k = 0; k < 8; ++k) su[k * P + b * R + a] = col[k];
    T ut[8];
    line8<T, 0>(col, ut);
    uint32_t gn[8];
    T cn[8];
    gather(next, gn, cn);        // next batch's loads overlap this batch's work
    __syncthreads();
    {
      T v[8], o[8];
      ld_row(su + b * P + a * R, v);
      line8<T, 0>(v, o);
      st_row(sr + b * P + a * R, o);
#pragma unroll
      for (int j = 0; j < 8; ++j) v[j] = su[b * P + j * R + a];
      line8<T, 0>(v, o);
#pragma unroll
      for (int j = 0; j < 8; ++j) ss[b * P + j * R + a] = o[j];
    }
    bool ok = false;
    const uint32_t par = (phase >> buf) & 1u;
    for (uint32_t w = 0; w < kWaitLimit; ++w)
      if (mbar_try_wait(&bar[buf], par)) {
        ok = true;
        break;
      }
    phase ^= 1u << buf;
    if (!__syncthreads_and(ok ? 1 : 0)) {
      if (tid == 0) atomicExch(err, 1u);
      // let copies still in flight finish before the block leaves
      for (uint32_t w = 0; w < kWaitLimit; ++w)
        if (mbar_try_wait(&bar[buf], par)) break;
      if (NB == 2 && next < nbatch)
        for (uint32_t w = 0; w < kWaitLimit; ++w)
          if (mbar_try_wait(&bar[buf ^ 1], (phase >> (buf ^ 1)) & 1u)) break;
      return;
    }
    T wt[8];
    const T* gG = sG + buf * EB * C::GELEM + le * C::GELEM;
#pragma unroll
    for (int k = 0; k < 8; ++k) {
      const int p = k * 64 + b * 8 + a;
      const int q = k * P + b * R + a;
      const T ur = sr[q], us = ss[q], utk = ut[k];
      const T g00 = gG[p], g01 = gG[512 + p], g02 = gG[1024 + p];
      const T g11 = gG[1536 + p], g12 = gG[2048 + p], g22 = gG[2560 + p];
      sr[q] = g00 * ur + g01 * us + g02 * utk;
      ss[q] = g01 * ur + g11 * us + g12 * utk;
      wt[k] = g02 * ur + g12 * us + g22 * utk;
    }
    T yt[8];
    line8<T, 1>(wt, yt);
    __syncthreads();
    // single buffer: every thread has read it (the barrier above), so batch i+1's copy starts
    if (NB == 1 && tid == 0 && next < nbatch) issue(next, 0);
    {
      T v[8], o[8];
      ld_row(sr + b * P + a * R, v);
      line8<T, 1>(v, o);
      st_row(su + b * P + a * R, o);
    }
    __syncthreads();
    {
      T v[8], o[8];
#pragma unroll
      for (int j = 0; j < 8; ++j) v[j] = ss[b * P + j * R + a];
      line8<T, 1>(v, o);
#pragma unroll
      for (int j = 0; j < 8; ++j) su[b * P + j * R + a] += o[j];
    }
    __syncthreads();
#pragma unroll
    for (int k = 0; k < 8; ++k) {
      const T v = su[k * P + b * R + a] + yt[k];
      if (!(g[k] & kGidDirichlet)) atomicAdd(&y[g[k] & kGidMask], v);
    }
    __syncthreads();             // stage buffers and this G buffer are free for reuse
#pragma unroll
    for (int k = 0; k < 8; ++k) {
      g[k] = gn[k];
      col[k] = cn[k];
    }
  }
}

// Batched variant: the block stages the geometric factors of its EB elements once (one TMA
// copy) and applies the element operator to RB right-hand sides in turn, RHS q of the batch
// at u + q * ld, y + q * ld.  The element-to-global ids are computed once per block, and the
// gather of the next right-hand side is in flight while the current one is computed.
template <typename T, int EB, bool IMPLICIT>
__global__ void __launch_bounds__(64 * EB)
k_sem_ax8b(int64_t E, const uint32_t* __restrict__ gid, Lattice lat, const T* __restrict__ G,
           const T* __restrict__ u, T* __restrict__ y, unsigned* __restrict__ err, int nb, int64_t ld, int rb) {
  using C = Ax8<T, EB>;
  constexpr int R = C::R, P = C::P;
  extern __shared__ __align__(128) unsigned char smem_raw[];
  __shared__ __align__(8) uint64_t bar;
  T* sG = reinterpret_cast<T*>(smem_raw);
  T* sU = sG + EB * C::GELEM;
  T* sR = sU + EB * C::STAGE;
  T* sS = sR + EB * C::STAGE;
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
    const uint32_t bytes = (uint32_t)(nvalid * C::GELEM * sizeof(T));
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(&bar)), "r"(bytes)
                 : "memory");
    bulk_copy_g(sG, G + e0 * C::GELEM, bytes, &bar);
  }
  T* su = sU + le * C::STAGE;
  T* sr = sR + le * C::STAGE;
  T* ss = sS + le * C::STAGE;
  uint32_t g[8];
  column_ids<IMPLICIT>(gid, lat, e, valid, a, b, g);
  auto gather = [&](int q, T (&v)[8]) {
    const T* uq = u + (int64_t)q * ld;
#pragma unroll
    for (int k = 0; k < 8; ++k) v[k] = (q < q1 && !(g[k] & kGidDirichlet)) ? uq[g[k] & kGidMask] : T(0);
  };
  T col[8];
  gather(q0, col);
  for (int q = q0; q < q1; ++q) {
#pragma unroll
    for (int k = 0; k < 8; ++k) su[k * P + b * R + a] = col[k];
    T ut[8];
    line8<T, 0>(col, ut);
    T cn[8];
    gather(q + 1, cn);           // next right-hand side's loads overlap this one's work
    __syncthreads();
    {
      T v[8], o[8];
      ld_row(su + b * P + a * R, v);
      line8<T, 0>(v, o);
      st_row(sr + b * P + a * R, o);
#pragma unroll
      for (int j = 0; j < 8; ++j) v[j] = su[b * P + j * R + a];
      line8<T, 0>(v, o);
#pragma unroll
      for (int j = 0; j < 8; ++j) ss[b * P + j * R + a] = o[j];
    }
    if (q == q0) {               // geometric factors must have landed (once per block)
      bool ok = false;
      for (uint32_t w = 0; w < kWaitLimit; ++w)
        if (mbar_try_wait(&bar, 0)) {
          ok = true;
          break;
        }
      if (!__syncthreads_and(ok ? 1 : 0)) {
        if (tid == 0) atomicExch(err, 1u);
        for (uint32_t w = 0; w < kWaitLimit; ++w)
          if (mbar_try_wait(&bar, 0)) break;
        return;
      }
    } else {
      __syncthreads();           // the line passes above wrote points other threads read next
    }
    T wt[8];
    const T* gG = sG + le * C::GELEM;
#pragma unroll
    for (int k = 0; k < 8; ++k) {
      const int p = k * 64 + b * 8 + a;
      const int qq = k * P + b * R + a;
      const T ur = sr[qq], us = ss[qq], utk = ut[k];
      const T g00 = gG[p], g01 = gG[512 + p], g02 = gG[1024 + p];
      const T g11 = gG[1536 + p], g12 = gG[2048 + p], g22 = gG[2560 + p];
      sr[qq] = g00 * ur + g01 * us + g02 * utk;
      ss[qq] = g01 * ur + g11 * us + g12 * utk;
      wt[k] = g02 * ur + g12 * us + g22 * utk;
    }
    T yt[8];
    line8<T, 1>(wt, yt);
    __syncthreads();
    {
      T v[8], o[8];
      ld_row(sr + b * P + a * R, v);
      line8<T, 1>(v, o);
      st_row(su + b * P + a * R, o);
    }
    __syncthreads();
    {
      T v[8], o[8];
#pragma unroll
      for (int j = 0; j < 8; ++j) v[j] = ss[b * P + j * R + a];
      line8<T, 1>(v, o);
#pragma unroll
      for (int j = 0; j < 8; ++j) su[b * P + j * R + a] += o[j];
    }
    __syncthreads();
    if (valid) {
      T* yq = y + (int64_t)q * ld;
#pragma unroll
      for (int k = 0; k < 8; ++k) {
        const T v = su[k * P + b * R + a] + yt[k];
        if (!(g[k] & kGidDirichlet)) atomicAdd(&yq[g[k] & kGidMask], v);
      }
    }
    __syncthreads();             // stage buffers free for the next right-hand side
#pragma unroll
    for (int k = 0; k < 8; ++k) col[k] = cn[k];
  }
}

// Batched variant with the geometric factors in registers: each thread loads the six factors
// of the eight points of its t-line once (48 values; for a given factor and point the 64
// threads of an element read 64 consecutive words) and keeps them for all the block's
// right-hand sides.  No shared-memory copy of G: the factor multiply reads only the staged
// derivatives (60 instead of 84 bytes of shared-memory traffic per point and right-hand side)
// and the block holds just the three stage buffers.
template <typename T, int EB, bool IMPLICIT>
__global__ void __launch_bounds__(64 * EB)
k_sem_ax8bg(int64_t E, const uint32_t* __restrict__ gid, Lattice lat, const T* __restrict__ G,
            const T* __restrict__ u, T* __restrict__ y, int nb, int64_t ld, int rb) {
  using C = Ax8<T, EB>;
  constexpr int R = C::R, P = C::P;
  extern __shared__ __align__(128) unsigned char smem_raw[];
  T* sU = reinterpret_cast<T*>(smem_raw);
  T* sR = sU + EB * C::STAGE;
  T* sS = sR + EB * C::STAGE;
  const int tid = threadIdx.x;
  const int le = tid >> 6, t = tid & 63, a = t & 7, b = t >> 3;
  const int64_t e = (int64_t)blockIdx.x * EB + le;
  const bool valid = e < E;
  const int q0 = blockIdx.y * rb;
  const int q1 = q0 + rb < nb ? q0 + rb : nb;
  T gr[6][8];
  {
    const T* gG = G + (valid ? e : 0) * C::GELEM + b * 8 + a;
#pragma unroll
    for (int c = 0; c < 6; ++c)
#pragma unroll
      for (int k = 0; k < 8; ++k) gr[c][k] = __ldg(gG + c * 512 + k * 64);
  }
  T* su = sU + le * C::STAGE;
  T* sr = sR + le * C::STAGE;
  T* ss = sS + le * C::STAGE;
  uint32_t g[8];
  column_ids<IMPLICIT>(gid, lat, e, valid, a, b, g);
  auto gather = [&](int q, T (&v)[8]) {
    const T* uq = u + (int64_t)q * ld;
#pragma unroll
    for (int k = 0; k < 8; ++k) v[k] = (q < q1 && !(g[k] & kGidDirichlet)) ? uq[g[k] & kGidMask] : T(0);
  };
  T col[8];
  gather(q0, col);
  for (int q = q0; q < q1; ++q) {
#pragma unroll
    for (int k = 0; k < 8; ++k) su[k * P + b * R + a] = col[k];
    T ut[8];
    line8<T, 0>(col, ut);
    T cn[8];
    gather(q + 1, cn);           // next right-hand side's loads overlap this one's work
    __syncthreads();
    {
      T v[8], o[8];
      ld_row(su + b * P + a * R, v);
      line8<T, 0>(v, o);
      st_row(sr + b * P + a * R, o);
#pragma unroll
      for (int j = 0; j < 8; ++j) v[j] = su[b * P + j * R + a];
      line8<T, 0>(v, o);
#pragma unroll
      for (int j = 0; j < 8; ++j) ss[b * P + j * R + a] = o[j];
    }
    __syncthreads();             // the line passes above wrote points other threads read next
    T wt[8];
#pragma unroll
    for (int k = 0; k < 8; ++k) {
      const int qq = k * P + b * R + a;
      const T ur = sr[qq], us = ss[qq], utk = ut[k];
      sr[qq] = gr[0][k] * ur + gr[1][k] * us + gr[2][k] * utk;
      ss[qq] = gr[1][k] * ur + gr[3][k] * us + gr[4][k] * utk;
      wt[k] = gr[2][k] * ur + gr[4][k] * us + gr[5][k] * utk;
    }
    T yt[8];
    line8<T, 1>(wt, yt);
    __syncthreads();
    {
      T v[8], o[8];
      ld_row(sr + b * P + a * R, v);
      line8<T, 1>(v, o);
      st_row(su + b * P + a * R, o);
    }
    __syncthreads();
    {
      T v[8], o[8];
#pragma unroll
      for (int j = 0; j < 8; ++j) v[j] = ss[b * P + j * R + a];
      line8<T, 1>(v, o);
#pragma unroll
      for (int j = 0; j < 8; ++j) su[b * P + j * R + a] += o[j];
    }
    __syncthreads();
    if (valid) {
      T* yq = y + (int64_t)q * ld;
#pragma unroll
      for (int k = 0; k < 8; ++k) {
        const T v = su[k * P + b * R + a] + yt[k];
        if (!(g[k] & kGidDirichlet)) atomicAdd(&yq[g[k] & kGidMask], v);
      }
    }
    __syncthreads();             // stage buffers free for the next right-hand side
#pragma unroll
    for (int k = 0; k < 8; ++k) col[k] = cn[k];
  }
}

// Paired batched variant: like k_sem_ax8b, but every line pass works on two right-hand sides
// at once (q and q + 1): each thread carries two independent lines through each contraction,
// the geometric factors read from shared memory serve both, and a block barrier covers two
// right-hand sides instead of one.  Stage buffers for both live in shared memory.
template <typename T, int EB, bool IMPLICIT>
__global__ void __launch_bounds__(64 * EB)
k_sem_ax8b2(int64_t E, const uint32_t* __restrict__ gid, Lattice lat, const T* __restrict__ G,
            const T* __restrict__ u, T* __restrict__ y, unsigned* __restrict__ err, int nb, int64_t ld, int rb) {
  using C = Ax8<T, EB>;
  constexpr int R = C::R, P = C::P;
  extern __shared__ __align__(128) unsigned char smem_raw[];
  __shared__ __align__(8) uint64_t bar;
  T* sG = reinterpret_cast<T*>(smem_raw);
  T* sStage = sG + EB * C::GELEM;   // [2 right-hand sides][3 stages][EB][STAGE]
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
    const uint32_t bytes = (uint32_t)(nvalid * C::GELEM * sizeof(T));
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(&bar)), "r"(bytes)
                 : "memory");
    bulk_copy_g(sG, G + e0 * C::GELEM, bytes, &bar);
  }
  T* su[2];
  T* sr[2];
  T* ss[2];
#pragma unroll
  for (int h = 0; h < 2; ++h) {
    su[h] = sStage + ((h * 3 + 0) * EB + le) * C::STAGE;
    sr[h] = sStage + ((h * 3 + 1) * EB + le) * C::STAGE;
    ss[h] = sStage + ((h * 3 + 2) * EB + le) * C::STAGE;
  }
  uint32_t g[8];
  column_ids<IMPLICIT>(gid, lat, e, valid, a, b, g);
  auto gather = [&](int q, T (&v)[8]) {
    const T* uq = u + (int64_t)q * ld;
#pragma unroll
    for (int k = 0; k < 8; ++k) v[k] = (q < q1 && !(g[k] & kGidDirichlet)) ? uq[g[k] & kGidMask] : T(0);
  };
  T col[2][8];
  gather(q0, col[0]);
  gather(q0 + 1, col[1]);
  for (int q = q0; q < q1; q += 2) {
    T ut[2][8], cn[2][8];
#pragma unroll
    for (int h = 0; h < 2; ++h) {
#pragma unroll
      for (int k = 0; k < 8; ++k) su[h][k * P + b * R + a] = col[h][k];
      line8<T, 0>(col[h], ut[h]);
    }
    gather(q + 2, cn[0]);        // the next pair's loads overlap this pair's work
    gather(q + 3, cn[1]);
    __syncthreads();
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      T v[8], o[8];
      ld_row(su[h] + b * P + a * R, v);
      line8<T, 0>(v, o);
      st_row(sr[h] + b * P + a * R, o);
#pragma unroll
      for (int j = 0; j < 8; ++j) v[j] = su[h][b * P + j * R + a];
      line8<T, 0>(v, o);
#pragma unroll
      for (int j = 0; j < 8; ++j) ss[h][b * P + j * R + a] = o[j];
    }
    if (q == q0) {               // geometric factors must have landed (once per block)
      bool ok = false;
      for (uint32_t w = 0; w < kWaitLimit; ++w)
        if (mbar_try_wait(&bar, 0)) {
          ok = true;
          break;
        }
      if (!__syncthreads_and(ok ? 1 : 0)) {
        if (tid == 0) atomicExch(err, 1u);
        for (uint32_t w = 0; w < kWaitLimit; ++w)
          if (mbar_try_wait(&bar, 0)) break;
        return;
      }
    } else {
      __syncthreads();           // the line passes above wrote points other threads read next
    }
    T wt[2][8];
    const T* gG = sG + le * C::GELEM;
#pragma unroll
    for (int k = 0; k < 8; ++k) {
      const int p = k * 64 + b * 8 + a;
      const int qq = k * P + b * R + a;
      const T g00 = gG[p], g01 = gG[512 + p], g02 = gG[1024 + p];
      const T g11 = gG[1536 + p], g12 = gG[2048 + p], g22 = gG[2560 + p];
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        const T ur = sr[h][qq], us = ss[h][qq], utk = ut[h][k];
        sr[h][qq] = g00 * ur + g01 * us + g02 * utk;
        ss[h][qq] = g01 * ur + g11 * us + g12 * utk;
        wt[h][k] = g02 * ur + g12 * us + g22 * utk;
      }
    }
    T yt[2][8];
#pragma unroll
    for (int h = 0; h < 2; ++h) line8<T, 1>(wt[h], yt[h]);
    __syncthreads();
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      T v[8], o[8];
      ld_row(sr[h] + b * P + a * R, v);
      line8<T, 1>(v, o);
      st_row(su[h] + b * P + a * R, o);
    }
    __syncthreads();
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      T v[8], o[8];
#pragma unroll
      for (int j = 0; j < 8; ++j) v[j] = ss[h][b * P + j * R + a];
      line8<T, 1>(v, o);
#pragma unroll
      for (int j = 0; j < 8; ++j) su[h][b * P + j * R + a] += o[j];
    }
    __syncthreads();
    if (valid) {
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        if (q + h >= q1) continue;
        T* yq = y + (int64_t)(q + h) * ld;
#pragma unroll
        for (int k = 0; k < 8; ++k) {
          const T v = su[h][k * P + b * R + a] + yt[h][k];
          if (!(g[k] & kGidDirichlet)) atomicAdd(&yq[g[k] & kGidMask], v);
        }
      }
    }
    __syncthreads();             // stage buffers free for the next pair
#pragma unroll
    for (int h = 0; h < 2; ++h)
#pragma unroll
      for (int k = 0; k < 8; ++k) col[h][k] = cn[h][k];
  }
}

}  // namespace

cudaError_t sem_ax8_set_D(const double* D) {
  // symmetrised even-odd blocks of D and D^T (D[7-i][7-l] = -D[i][l] exactly)
  double S[8][8];
  for (int i = 0; i < 8; ++i)
    for (int l = 0; l < 8; ++l) S[i][l] = 0.5 * (D[i * 8 + l] - D[(7 - i) * 8 + (7 - l)]);
  double h[4][4][4];
  float f[4][4][4];
  for (int i = 0; i < 4; ++i)
    for (int l = 0; l < 4; ++l) {
      h[0][i][l] = 0.5 * (S[i][l] + S[i][7 - l]);
      h[1][i][l] = 0.5 * (S[i][l] - S[i][7 - l]);
      h[2][i][l] = 0.5 * (S[l][i] + S[7 - l][i]);
      h[3][i][l] = 0.5 * (S[l][i] - S[7 - l][i]);
    }
  for (int w = 0; w < 4; ++w)
    for (int i = 0; i < 4; ++i)
      for (int l = 0; l < 4; ++l) f[w][i][l] = (float)h[w][i][l];
  cudaError_t e = cudaMemcpyToSymbol(c_eo_d, h, sizeof(h));
  if (e != cudaSuccess) return e;
  e = cudaMemcpyToSymbol(c_eo_f, f, sizeof(f));
  if (e != cudaSuccess) return e;
  e = sem_smooth8_set_eo(&h[0][0][0]);
  if (e != cudaSuccess) return e;
  return sem_ax8_x2_set_eo(&h[0][0][0]);
}

template <typename T, int EB, bool IM>
static void launch_ax8(int64_t E, const uint32_t* gid, const Lattice& lat, const T* G, const T* u, T* y,
                       unsigned* err, cudaStream_t s) {
  using C = Ax8<T, EB>;
  static bool configured = false;
  if (!configured) {
    cudaFuncSetAttribute(k_sem_ax8<T, EB, IM>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)C::smem_bytes());
    configured = true;
  }
  const unsigned blocks = (unsigned)((E + EB - 1) / EB);
  launch_dep(k_sem_ax8<T, EB, IM>, dim3(blocks), dim3(64 * EB), C::smem_bytes(), s, E, gid, lat, G, u, y, err);
}

template <typename T, int EB, bool IM>
static void launch_ax8g(int64_t E, const uint32_t* gid, const Lattice& lat, const T* G, const T* u, T* y,
                        cudaStream_t s) {
  using C = Ax8<T, EB>;
  const size_t smem = sizeof(T) * (size_t)EB * 3 * C::STAGE;
  static bool configured = false;
  if (!configured) {
    cudaFuncSetAttribute(k_sem_ax8g<T, EB, IM>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    configured = true;
  }
  const unsigned blocks = (unsigned)((E + EB - 1) / EB);
  launch_dep(k_sem_ax8g<T, EB, IM>, dim3(blocks), dim3(64 * EB), smem, s, E, gid, lat, G, u, y);
}

template <typename T, int EB, bool IM, int NB = 2>
static void launch_ax8p(int64_t E, const uint32_t* gid, const Lattice& lat, const T* G, const T* u, T* y,
                        unsigned* err, cudaStream_t s) {
  using C = Ax8<T, EB>;
  const size_t smem = sizeof(T) * (size_t)EB * (NB * C::GELEM + 3 * C::STAGE);
  static int grid = 0;
  if (grid == 0) {
    cudaFuncSetAttribute(k_sem_ax8p<T, EB, IM, NB>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    int dev = 0, sms = 0, per_sm = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_sem_ax8p<T, EB, IM, NB>, 64 * EB, smem);
    grid = sms * (per_sm > 0 ? per_sm : 1);
  }
  const int64_t nbatch = (E + EB - 1) / EB;
  const unsigned blocks = (unsigned)(nbatch < grid ? nbatch : grid);
  launch_dep(k_sem_ax8p<T, EB, IM, NB>, dim3(blocks), dim3(64 * EB), smem, s, E, gid, lat, G, u, y, err);
}

template <typename T, int EB, bool IM>
static void launch_ax8b(int64_t E, const uint32_t* gid, const Lattice& lat, const T* G, const T* u, T* y,
                        unsigned* err, int nb, int64_t ld, int rb, cudaStream_t s) {
  using C = Ax8<T, EB>;
  static bool configured = false;
  if (!configured) {
    cudaFuncSetAttribute(k_sem_ax8b<T, EB, IM>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)C::smem_bytes());
    configured = true;
  }
  if (rb < 1) rb = 1;
  const dim3 blocks((unsigned)((E + EB - 1) / EB), (unsigned)((nb + rb - 1) / rb));
  k_sem_ax8b<T, EB, IM><<<blocks, 64 * EB, C::smem_bytes(), s>>>(E, gid, lat, G, u, y, err, nb, ld, rb);
  g_launches.fetch_add(1, std::memory_order_relaxed);
}

template <typename T, int EB, bool IM>
static void launch_ax8b2(int64_t E, const uint32_t* gid, const Lattice& lat, const T* G, const T* u, T* y,
                         unsigned* err, int nb, int64_t ld, int rb, cudaStream_t s) {
  using C = Ax8<T, EB>;
  const size_t smem = sizeof(T) * (size_t)EB * (C::GELEM + 6 * C::STAGE);
  static bool configured = false;
  if (!configured) {
    cudaFuncSetAttribute(k_sem_ax8b2<T, EB, IM>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    configured = true;
  }
  if (rb < 2) rb = 2;
  const dim3 blocks((unsigned)((E + EB - 1) / EB), (unsigned)((nb + rb - 1) / rb));
  k_sem_ax8b2<T, EB, IM><<<blocks, 64 * EB, smem, s>>>(E, gid, lat, G, u, y, err, nb, ld, rb);
  g_launches.fetch_add(1, std::memory_order_relaxed);
}

template <typename T, int EB, bool IM>
static void launch_ax8bg(int64_t E, const uint32_t* gid, const Lattice& lat, const T* G, const T* u, T* y, int nb,
                         int64_t ld, int rb, cudaStream_t s) {
  using C = Ax8<T, EB>;
  const size_t smem = sizeof(T) * (size_t)EB * 3 * C::STAGE;
  static bool configured = false;
  if (!configured) {
    cudaFuncSetAttribute(k_sem_ax8bg<T, EB, IM>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    configured = true;
  }
  if (rb < 1) rb = 1;
  const dim3 blocks((unsigned)((E + EB - 1) / EB), (unsigned)((nb + rb - 1) / rb));
  k_sem_ax8bg<T, EB, IM><<<blocks, 64 * EB, smem, s>>>(E, gid, lat, G, u, y, nb, ld, rb);
  g_launches.fetch_add(1, std::memory_order_relaxed);
}

template <typename T>
size_t sem_ax8_smem(int eb) {
  eb %= 100;
  switch (eb) {
    case 1: return sizeof(T) * 1 * (Ax8<T, 1>::GELEM + 3 * Ax8<T, 1>::STAGE);
    case 2: return sizeof(T) * 2 * (Ax8<T, 2>::GELEM + 3 * Ax8<T, 2>::STAGE);
    case 4: return sizeof(T) * 4 * (Ax8<T, 4>::GELEM + 3 * Ax8<T, 4>::STAGE);
    case 12: return sizeof(T) * 2 * (2 * Ax8<T, 2>::GELEM + 3 * Ax8<T, 2>::STAGE);
    case 14: return sizeof(T) * 4 * (2 * Ax8<T, 4>::GELEM + 3 * Ax8<T, 4>::STAGE);
    case 31: return sizeof(T) * 1 * (Ax8<T, 1>::GELEM + 3 * Ax8<T, 1>::STAGE);
    case 32: return sizeof(T) * 2 * (Ax8<T, 2>::GELEM + 3 * Ax8<T, 2>::STAGE);
    case 21: return sizeof(T) * 1 * 3 * Ax8<T, 1>::STAGE;
    case 22: return sizeof(T) * 2 * 3 * Ax8<T, 2>::STAGE;
    default: return ~size_t(0);
  }
}

// Shared memory of the paired batched variant with eb elements per block (1 or 2).
template <typename T>
size_t sem_ax8b2_smem(int eb) {
  switch (eb) {
    case 1: return sizeof(T) * 1 * (Ax8<T, 1>::GELEM + 6 * Ax8<T, 1>::STAGE);
    case 2: return sizeof(T) * 2 * (Ax8<T, 2>::GELEM + 6 * Ax8<T, 2>::STAGE);
    default: return ~size_t(0);
  }
}

template <typename T>
bool sem_ax8_variant_fits(int eb) {
  int dev = 0, optin = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
  return sem_ax8_smem<T>(eb) + 256 <= (size_t)optin;   // + static shared (mbarriers)
}

template <typename T, bool IM>
static void dispatch_ax8(int64_t E, const uint32_t* gid, const Lattice& lat, const T* G, const T* u, T* y,
                         unsigned* err, int eb, cudaStream_t s) {
  switch (eb) {
    case 21: launch_ax8g<T, 1, IM>(E, gid, lat, G, u, y, s); break;
    case 22: launch_ax8g<T, 2, IM>(E, gid, lat, G, u, y, s); break;
    case 1: launch_ax8<T, 1, IM>(E, gid, lat, G, u, y, err, s); break;
    case 4: launch_ax8<T, 4, IM>(E, gid, lat, G, u, y, err, s); break;
    case 12: launch_ax8p<T, 2, IM>(E, gid, lat, G, u, y, err, s); break;
    case 14: launch_ax8p<T, 4, IM>(E, gid, lat, G, u, y, err, s); break;
    case 31: launch_ax8p<T, 1, IM, 1>(E, gid, lat, G, u, y, err, s); break;
    case 32: launch_ax8p<T, 2, IM, 1>(E, gid, lat, G, u, y, err, s); break;
    default: launch_ax8<T, 2, IM>(E, gid, lat, G, u, y, err, s); break;
  }
}

template <typename T>
void sem_ax8(int64_t E, const uint32_t* gid, const Lattice& lat, const T* G, const T* u, T* y, unsigned* err,
             int variant, cudaStream_t s) {
  if (variant >= 100) dispatch_ax8<T, true>(E, gid, lat, G, u, y, err, variant - 100, s);
  else dispatch_ax8<T, false>(E, gid, lat, G, u, y, err, variant, s);
}

template <typename T>
void sem_ax8_batched(int64_t E, const uint32_t* gid, const Lattice& lat, const T* G, const T* u, T* y,
                     unsigned* err, int variant, int nb, int64_t ld, cudaStream_t s) {
  const int rb = variant / 1000;
  const bool im = (variant % 1000) >= 100;
  const int form = (variant % 100) / 10;   // 0 single, 1 paired, 2 factors in registers
  const bool pair = form == 1;
  const int eb = variant % 10;
  if (form == 2) {
    // FP32 only: 48 FP64 factors per thread do not fit the register file
    if constexpr (sizeof(T) == 4) {
      if (im) {
        if (eb == 1) launch_ax8bg<T, 1, true>(E, gid, lat, G, u, y, nb, ld, rb, s);
        else launch_ax8bg<T, 2, true>(E, gid, lat, G, u, y, nb, ld, rb, s);
      } else {
        if (eb == 1) launch_ax8bg<T, 1, false>(E, gid, lat, G, u, y, nb, ld, rb, s);
        else launch_ax8bg<T, 2, false>(E, gid, lat, G, u, y, nb, ld, rb, s);
      }
    }
    return;
  }
  if (pair) {
    if (im) {
      if (eb == 1) launch_ax8b2<T, 1, true>(E, gid, lat, G, u, y, err, nb, ld, rb, s);
      else launch_ax8b2<T, 2, true>(E, gid, lat, G, u, y, err, nb, ld, rb, s);
    } else {
      if (eb == 1) launch_ax8b2<T, 1, false>(E, gid, lat, G, u, y, err, nb, ld, rb, s);
      else launch_ax8b2<T, 2, false>(E, gid, lat, G, u, y, err, nb, ld, rb, s);
    }
    return;
  }
  if (im) {
    if (eb == 1) launch_ax8b<T, 1, true>(E, gid, lat, G, u, y, err, nb, ld, rb, s);
    else if (eb == 4) launch_ax8b<T, 4, true>(E, gid, lat, G, u, y, err, nb, ld, rb, s);
    else launch_ax8b<T, 2, true>(E, gid, lat, G, u, y, err, nb, ld, rb, s);
  } else {
    if (eb == 1) launch_ax8b<T, 1, false>(E, gid, lat, G, u, y, err, nb, ld, rb, s);
    else if (eb == 4) launch_ax8b<T, 4, false>(E, gid, lat, G, u, y, err, nb, ld, rb, s);
    else launch_ax8b<T, 2, false>(E, gid, lat, G, u, y, err, nb, ld, rb, s);
  }
}

template <typename T>
bool sem_ax8_batched_fits(int variant) {
  const int rest = variant % 100;
  // factors in registers (21, 22: the stage buffers alone, like the single-vector variants 21
  // and 22) and single (1, 2, 4) forms
  if (rest >= 20) return sizeof(T) == 4 && sem_ax8_variant_fits<T>(rest);   // FP32 only
  if (rest < 10) return sem_ax8_variant_fits<T>(rest);
  int dev = 0, optin = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
  return sem_ax8b2_smem<T>(rest % 10) + 256 <= (size_t)optin;
}

template bool sem_ax8_batched_fits<float>(int);
template bool sem_ax8_batched_fits<double>(int);
template bool sem_ax8_variant_fits<float>(int);
template bool sem_ax8_variant_fits<double>(int);
template void sem_ax8<float>(int64_t, const uint32_t*, const Lattice&, const float*, const float*, float*,
                             unsigned*, int, cudaStream_t);
template void sem_ax8<double>(int64_t, const uint32_t*, const Lattice&, const double*, const double*, double*,
                              unsigned*, int, cudaStream_t);
template void sem_ax8_batched<float>(int64_t, const uint32_t*, const Lattice&, const float*, const float*, float*,
                                     unsigned*, int, int, int64_t, cudaStream_t);
template void sem_ax8_batched<double>(int64_t, const uint32_t*, const Lattice&, const double*, const double*,
                                      double*, unsigned*, int, int, int64_t, cudaStream_t);

}  // namespace chebmg
