// Fused smoother for the order-7 level of a box lattice: every step of Algorithm 1 or 2 (the
// element operator with its gather-scatter, Sec. 1 Eq. 1.3, then the Jacobi-scaled Chebyshev
// recurrence and the residual update) and the V-cycle's restriction residual (Eq. 2.2) run in
// one persistent launch.
//
// Why one launch.  The element operator sums the contributions of every element that shares a
// node with atomics into an accumulator y, so the update of a node can only run after all those
// elements are done.  Run as two kernels per step, y makes an extra round trip and every step
// pays two kernel tails.  Here the step is split into tasks over slabs of one element plane:
//
//   P1(p, s)  operator of phase p on the elements of plane s, accumulated into y: it reads the
//             source vector on node planes 7s .. 7s+7 and adds into y there;
//   P2(p, s)  pointwise operation of phase p over the nodes owned by slab s, the range
//             [a_s, a_{s+1}) with a_s = 7 s NX NY rounded down to a multiple of 4 (node planes
//             7s .. 7s+6, the last slab to the end); it reads y there and zeroes it.
//
// Dependencies (a task starts after the ones it names are complete):
//   P1(p, s) <- P2(p-1, s), P2(p-1, s+1)   its source vector is final, y is zero on its nodes;
//   P2(p, s) <- P1(p, s), P1(p, s-1)       every element touching the range has accumulated and
//                                          has read the old source values there;
//   P2(p, s) <- P2(p-1, s)                 (phases without an operator; implied otherwise).
// Work items (P1: EB elements; P2: `chunk` nodes) are numbered in the order of t = 3p + s for P1
// and t = 3p + s + 1 for P2, which puts every task after all tasks it depends on, and block b
// takes items b, b + grid, b + 2 grid, ... in turn.  The launch is cooperative (every block
// resident), so the oldest unfinished item is always held by a running block whose dependencies
// are done: no deadlock.  Phase p + 1 runs three planes behind phase p, so y and the vectors are
// read again soon after they were written.  A block knows its next item in advance: it starts
// the TMA copy of an operator item's geometric factors into a second buffer and reads the next
// item's dependency counters (relaxed loads) while it works on the current one, so a dependency
// that is complete by then costs no round trip.  Every wait is bounded (2 s): on timeout the
// block records the error and all blocks leave, after waiting (bounded) for their own copies in
// flight.
//
// Vectors written in this launch are read with ld.global.cg (L2, never a stale L1 line).  A work
// item's completion is published by a block barrier and one release increment of its task's
// counter, and observed by relaxed or acquire loads followed by an acquire fence and a block
// barrier.
#include <cuda_runtime.h>

#include <algorithm>

#include "ax8_core.cuh"
#include "ax8_util.cuh"
#include "common.cuh"

namespace chebmg {

namespace {

constexpr unsigned long long kFusedWaitNs = 2000000000ull;   // 2 s per wait

__device__ __forceinline__ unsigned long long global_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %globaltimer;" : "=l"(t));
  return t;
}

__device__ __forceinline__ unsigned ld_acquire(const unsigned* p) {
  unsigned v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

__device__ __forceinline__ unsigned ld_relaxed(const unsigned* p) {
  unsigned v;
  asm volatile("ld.relaxed.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

__device__ __forceinline__ void red_release_add(unsigned* p, unsigned v) {
  asm volatile("red.release.gpu.global.add.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

__device__ __forceinline__ void fence_acq_rel() { asm volatile("fence.acq_rel.gpu;" ::: "memory"); }

// Waits until *cnt >= target (thread 0 only).  False if the error flag is raised meanwhile or
// the wait runs out.
__device__ bool wait_count(const unsigned* cnt, unsigned target, const unsigned* err) {
  if (ld_acquire(cnt) >= target) return true;
  const unsigned long long t0 = global_ns();
  for (;;) {
    __nanosleep(100);
    if (ld_acquire(cnt) >= target) return true;
    if (*(volatile const unsigned*)err) return false;
    if (global_ns() - t0 > kFusedWaitNs) return false;
  }
}

__device__ __forceinline__ unsigned* cnt1(const FusedSmooth& a, int p, int s) {
  return a.ctl + 2 + 2 * (p * a.nslab + s);
}
__device__ __forceinline__ unsigned* cnt2(const FusedSmooth& a, int p, int s) {
  return a.ctl + 3 + 2 * (p * a.nslab + s);
}

// First node of slab s's range.
__device__ __forceinline__ int64_t slab_start(const FusedSmooth& a, int s) {
  if (s <= 0) return 0;
  if (s >= a.nslab) return a.n;
  return ((int64_t)7 * s * a.lat.NX * a.lat.NY) & ~int64_t(3);
}

// Work item w -> kind (0 none, 1 operator, 2 pointwise), phase, slab, index within the task.
struct Item {
  int kind, p, s, k;
};
__device__ Item decode(const FusedSmooth& a, uint32_t w) {
  Item it{0, 0, 0, 0};
  if (w >= a.total) return it;
  int lo = 0, hi = a.tsteps;
  while (hi - lo > 1) {
    const int mid = (lo + hi) >> 1;
    if (a.toff[mid] <= w) lo = mid;
    else hi = mid;
  }
  const int t = lo;
  uint32_t off = w - a.toff[t];
  for (int p = 0; p < a.nphase; ++p) {
    const int s2 = t - 3 * p - 1;
    if (s2 >= 0 && s2 < a.nslab) {
      if (off < (uint32_t)a.m2) return Item{2, p, s2, (int)off};
      off -= a.m2;
    }
    const int s1 = t - 3 * p;
    if (a.ph[p].src != FSRC_NONE && s1 >= 0 && s1 < a.nslab) {
      if (off < (uint32_t)a.m1) return Item{1, p, s1, (int)off};
      off -= a.m1;
    }
  }
  return it;
}

// The completion counters an item waits for (at most two) and their targets.
struct Deps {
  const unsigned* c[2];
  unsigned t[2];
};
__device__ Deps deps_of(const FusedSmooth& a, const Item& it) {
  Deps d{{nullptr, nullptr}, {0u, 0u}};
  if (it.kind == 1) {
    if (it.p > 0) {
      d.c[0] = cnt2(a, it.p - 1, it.s);
      d.t[0] = (unsigned)a.m2;
      if (it.s + 1 < a.nslab) {
        d.c[1] = cnt2(a, it.p - 1, it.s + 1);
        d.t[1] = (unsigned)a.m2;
      }
    }
  } else if (it.kind == 2) {
    if (a.ph[it.p].src != FSRC_NONE) {
      d.c[0] = cnt1(a, it.p, it.s);
      d.t[0] = (unsigned)a.m1;
      if (it.s > 0) {
        d.c[1] = cnt1(a, it.p, it.s - 1);
        d.t[1] = (unsigned)a.m1;
      }
    } else if (it.p > 0) {
      d.c[0] = cnt2(a, it.p - 1, it.s);
      d.t[0] = (unsigned)a.m2;
    }
  }
  return d;
}

template <typename T>
struct Vec16;
template <>
struct Vec16<float> {
  using type = float4;
  static constexpr int L = 4;
};
template <>
struct Vec16<double> {
  using type = double2;
  static constexpr int L = 2;
};

// The pointwise operation of a phase on one node; the loads it needs are done by the caller.
// Same arithmetic as the vector kernels (chebyshev.cu).
template <typename T>
struct PointOp {
  int op;
  T c0, c1, c2, c3;
  __device__ __forceinline__ void operator()(T& x, T& r, T& d, T& y, T s, T b) const {
    switch (op) {
      case FOP_ZERO_Y:
        y = T(0);
        break;
      case FOP_CHEB4_INIT_B:
        x = T(0);
        r = b;
        d = c0 * s * b;
        y = T(0);
        break;
      case FOP_CHEB4_INIT_BY: {
        const T rv = b - y;
        r = rv;
        d = c0 * s * rv;
        y = T(0);
        break;
      }
      case FOP_CHEB4_STEP: {
        const T dv = d;
        const T rv = r - y;
        x += c0 * dv;
        r = rv;
        d = c1 * dv + c2 * s * rv;
        y = T(0);
        if (c3 != T(0)) x += c3 * d;
        break;
      }
      case FOP_CHEB1_INIT_B: {
        const T rv = s * b;
        x = T(0);
        r = rv;
        d = rv * c0;
        y = T(0);
        break;
      }
      case FOP_CHEB1_INIT_BY: {
        const T rv = s * (b - y);
        r = rv;
        d = rv * c0;
        y = T(0);
        break;
      }
      case FOP_CHEB1_STEP: {
        const T dv = d;
        const T rv = r - s * y;
        x += dv;
        r = rv;
        d = c1 * dv + c2 * rv;
        y = T(0);
        if (c3 != T(0)) x += c3 * d;
        break;
      }
      case FOP_AXPY:
        x += c0 * d;
        break;
      default:   // FOP_RESIDUAL
        r = b - y;
        y = T(0);
        break;
    }
  }
};

// Which vectors an operation reads and writes (bit 0 x, 1 r, 2 d, 3 y, 4 S, 5 b).
__device__ __forceinline__ unsigned op_reads(int op) {
  switch (op) {
    case FOP_ZERO_Y: return 0u;
    case FOP_CHEB4_INIT_B: return 16u | 32u;
    case FOP_CHEB4_INIT_BY: return 8u | 16u | 32u;
    case FOP_CHEB4_STEP: return 1u | 2u | 4u | 8u | 16u;
    case FOP_CHEB1_INIT_B: return 16u | 32u;
    case FOP_CHEB1_INIT_BY: return 8u | 16u | 32u;
    case FOP_CHEB1_STEP: return 1u | 2u | 4u | 8u | 16u;
    case FOP_AXPY: return 1u | 4u;
    default: return 8u | 32u;
  }
}
__device__ __forceinline__ unsigned op_writes(int op) {
  switch (op) {
    case FOP_ZERO_Y: return 8u;
    case FOP_CHEB4_INIT_B: return 1u | 2u | 4u | 8u;
    case FOP_CHEB4_INIT_BY: return 2u | 4u | 8u;
    case FOP_CHEB4_STEP: return 1u | 2u | 4u | 8u;
    case FOP_CHEB1_INIT_B: return 1u | 2u | 4u | 8u;
    case FOP_CHEB1_INIT_BY: return 2u | 4u | 8u;
    case FOP_CHEB1_STEP: return 1u | 2u | 4u | 8u;
    case FOP_AXPY: return 1u;
    default: return 2u | 8u;
  }
}

// The pointwise operation over nodes [lo, hi) (lo a multiple of 4): 16-byte accesses over the
// aligned body, VPT vectors per thread per round, scalar tail.
template <typename T, int NT>
__device__ void pointwise(const FusedSmooth& a, const PointOp<T>& f, int64_t lo, int64_t hi) {
  using V = typename Vec16<T>::type;
  constexpr int L = Vec16<T>::L;
  constexpr int VPT = 4;
  const unsigned rd = op_reads(f.op), wr = op_writes(f.op);
  T* X = static_cast<T*>(a.x);
  T* Rv = static_cast<T*>(a.r);
  T* Dv = static_cast<T*>(a.d);
  T* Y = static_cast<T*>(a.y);
  const T* S = static_cast<const T*>(a.S);
  const T* B = static_cast<const T*>(a.b);
  const int64_t v0 = lo / L, v1 = hi / L;   // vectors [v0, v1)
  for (int64_t base = v0 + threadIdx.x; base < v1; base += (int64_t)NT * VPT) {
    V xv[VPT], rv[VPT], dv[VPT], yv[VPT], sv[VPT], bv[VPT];
#pragma unroll
    for (int u = 0; u < VPT; ++u) {
      const int64_t q = base + (int64_t)u * NT;
      if (q < v1) {
        if (rd & 1u) xv[u] = __ldcg(reinterpret_cast<const V*>(X) + q);
        if (rd & 2u) rv[u] = __ldcg(reinterpret_cast<const V*>(Rv) + q);
        if (rd & 4u) dv[u] = __ldcg(reinterpret_cast<const V*>(Dv) + q);
        if (rd & 8u) yv[u] = __ldcg(reinterpret_cast<const V*>(Y) + q);
        if (rd & 16u) sv[u] = __ldg(reinterpret_cast<const V*>(S) + q);
        if (rd & 32u) bv[u] = __ldg(reinterpret_cast<const V*>(B) + q);
      }
    }
#pragma unroll
    for (int u = 0; u < VPT; ++u) {
      const int64_t q = base + (int64_t)u * NT;
      if (q < v1) {
        T* xs = reinterpret_cast<T*>(&xv[u]);
        T* rs = reinterpret_cast<T*>(&rv[u]);
        T* ds = reinterpret_cast<T*>(&dv[u]);
        T* ys = reinterpret_cast<T*>(&yv[u]);
        const T* ss = reinterpret_cast<const T*>(&sv[u]);
        const T* bs = reinterpret_cast<const T*>(&bv[u]);
#pragma unroll
        for (int l = 0; l < L; ++l) f(xs[l], rs[l], ds[l], ys[l], ss[l], bs[l]);
        if (wr & 1u) __stcg(reinterpret_cast<V*>(X) + q, xv[u]);
        if (wr & 2u) __stcg(reinterpret_cast<V*>(Rv) + q, rv[u]);
        if (wr & 4u) __stcg(reinterpret_cast<V*>(Dv) + q, dv[u]);
        if (wr & 8u) __stcg(reinterpret_cast<V*>(Y) + q, yv[u]);
      }
    }
  }
  for (int64_t g = v1 * L + threadIdx.x; g < hi; g += NT) {   // tail (last slab only)
    T x = (rd & 1u) ? __ldcg(X + g) : T(0), r = (rd & 2u) ? __ldcg(Rv + g) : T(0);
    T d = (rd & 4u) ? __ldcg(Dv + g) : T(0), y = (rd & 8u) ? __ldcg(Y + g) : T(0);
    const T s = (rd & 16u) ? S[g] : T(0), b = (rd & 32u) ? B[g] : T(0);
    f(x, r, d, y, s, b);
    if (wr & 1u) X[g] = x;
    if (wr & 2u) Rv[g] = r;
    if (wr & 4u) Dv[g] = d;
    if (wr & 8u) Y[g] = y;
  }
}

template <typename T, int EB, bool PF>
__global__ void __launch_bounds__(64 * EB) k_sem_smooth8(const __grid_constant__ FusedSmooth a) {
  using C = Ax8<T, EB>;
  constexpr int R = C::R, P = C::P, NT = 64 * EB, NBUF = PF ? 2 : 1;
  extern __shared__ __align__(128) unsigned char smem_raw[];
  __shared__ __align__(8) uint64_t bar[2];
  __shared__ Item sh_item[2];   // [0] the item in progress, [1] the next one
  __shared__ int sh_ok;
  T* sG = reinterpret_cast<T*>(smem_raw);   // [NBUF][EB * GELEM]
  T* sU = sG + NBUF * EB * C::GELEM;
  T* sR = sU + EB * C::STAGE;
  T* sS = sR + EB * C::STAGE;
  const int tid = threadIdx.x;
  const int le = tid >> 6, tt = tid & 63, ca = tt & 7, cb = tt >> 3;
  const T* G = static_cast<const T*>(a.G);
  T* Y = static_cast<T*>(a.y);
  T* su = sU + le * C::STAGE;
  T* sr = sR + le * C::STAGE;
  T* ss = sS + le * C::STAGE;

  // thread 0: operator items decoded so far (their buffer is that count mod NBUF) and copies
  // issued but not yet waited for
  int p1dec = 0;
  unsigned pend = 0;   // bit q: a copy into buffer q is in flight
  // all threads: operator items processed so far, parity of the next wait on each buffer
  int p1seq = 0;
  uint32_t par = 0;

  auto issue = [&](const Item& it) {   // thread 0: TMA of the item's geometric factors
    const int buf = p1dec % NBUF;
    ++p1dec;
    const int64_t e0 = (int64_t)it.s * a.spp + (int64_t)it.k * EB;
    const int nv = min(EB, a.spp - it.k * EB);
    const uint32_t bytes = (uint32_t)(nv * C::GELEM * sizeof(T));
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(&bar[buf])), "r"(bytes)
                 : "memory");
    bulk_copy_g(sG + buf * EB * C::GELEM, G + e0 * C::GELEM, bytes, &bar[buf]);
    pend |= 1u << buf;
  };
  // thread 0: the work items of this block are blockIdx.x, blockIdx.x + gridDim.x, ... (every
  // block is resident: cooperative launch); the next item's dependency counters are read one
  // item ahead with relaxed loads, so a dependency that is already complete costs no round trip
  uint32_t w = blockIdx.x;
  Deps cd{{nullptr, nullptr}, {0u, 0u}}, nd = cd;
  unsigned cv[2] = {0u, 0u}, nv[2] = {0u, 0u};
  auto item_at = [&](uint32_t idx) -> Item {
    if (*(volatile const unsigned*)a.err) return Item{0, 0, 0, 0};   // another block gave up
    return decode(a, idx);
  };

  if (tid == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_addr(&bar[0])) : "memory");
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_addr(&bar[1])) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    const Item it = item_at(w);
    sh_item[0] = it;
    if (it.kind == 1) issue(it);
    cd = deps_of(a, it);
    for (int q = 0; q < 2; ++q) cv[q] = cd.c[q] ? ld_relaxed(cd.c[q]) : 0u;
  }
  __syncthreads();

  bool failed = false;
  for (;;) {
    const Item cur = sh_item[0];
    if (cur.kind == 0) break;
    if (tid == 0) {
      w += gridDim.x;
      const Item nx = item_at(w);
      sh_item[1] = nx;
      if (PF && nx.kind == 1) issue(nx);
      nd = deps_of(a, nx);
      for (int q = 0; q < 2; ++q) nv[q] = nd.c[q] ? ld_relaxed(nd.c[q]) : 0u;
      // this item's dependencies: complete when read one item ago, else poll
      bool ok = true;
      for (int q = 0; q < 2 && ok; ++q)
        if (cd.c[q] && cv[q] < cd.t[q]) ok = wait_count(cd.c[q], cd.t[q], a.err);
      fence_acq_rel();   // acquire side of the counters observed above
      sh_ok = ok ? 1 : 0;
    }
    __syncthreads();
    if (!sh_ok) {
      failed = true;
      break;
    }
    const FusedPhase& ph = a.ph[cur.p];
    if (cur.kind == 1) {
      // ---- operator on EB elements of plane cur.s: y += A v ----
      const T* src = static_cast<const T*>(ph.src == FSRC_X ? a.x : a.d);
      const int64_t e = (int64_t)cur.s * a.spp + (int64_t)cur.k * EB + le;
      const bool valid = cur.k * EB + le < a.spp;
      uint32_t g[8];
      column_ids<true>(nullptr, a.lat, e, valid, ca, cb, g);
      T col[8];
#pragma unroll
      for (int k = 0; k < 8; ++k) col[k] = (g[k] & kGidDirichlet) ? T(0) : __ldcg(src + (g[k] & kGidMask));
#pragma unroll
      for (int k = 0; k < 8; ++k) su[k * P + cb * R + ca] = col[k];
      T ut[8];
      line8<T, 0>(col, ut);
      __syncthreads();
      {
        T v[8], o[8];
        ld_row(su + cb * P + ca * R, v);
        line8<T, 0>(v, o);
        st_row(sr + cb * P + ca * R, o);
#pragma unroll
        for (int j = 0; j < 8; ++j) v[j] = su[cb * P + j * R + ca];
        line8<T, 0>(v, o);
#pragma unroll
        for (int j = 0; j < 8; ++j) ss[cb * P + j * R + ca] = o[j];
      }
      const int buf = p1seq % NBUF;
      const uint32_t pr = (par >> buf) & 1u;
      bool gok = false;
      for (uint32_t w = 0; w < kWaitLimit; ++w)
        if (mbar_try_wait(&bar[buf], pr)) {
          gok = true;
          break;
        }
      if (!__syncthreads_and(gok ? 1 : 0)) {
        failed = true;
        break;
      }
      par ^= 1u << buf;
      ++p1seq;
      if (tid == 0) pend &= ~(1u << buf);
      T wt[8];
      const T* gG = sG + buf * EB * C::GELEM + le * C::GELEM;
#pragma unroll
      for (int k = 0; k < 8; ++k) {
        const int p = k * 64 + cb * 8 + ca;
        const int q = k * P + cb * R + ca;
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
        ld_row(sr + cb * P + ca * R, v);
        line8<T, 1>(v, o);
        st_row(su + cb * P + ca * R, o);
      }
      __syncthreads();
      {
        T v[8], o[8];
#pragma unroll
        for (int j = 0; j < 8; ++j) v[j] = ss[cb * P + j * R + ca];
        line8<T, 1>(v, o);
#pragma unroll
        for (int j = 0; j < 8; ++j) su[cb * P + j * R + ca] += o[j];
      }
      __syncthreads();
#pragma unroll
      for (int k = 0; k < 8; ++k) {
        const T v = su[k * P + cb * R + ca] + yt[k];
        if (!(g[k] & kGidDirichlet)) atomicAdd(&Y[g[k] & kGidMask], v);
      }
      __syncthreads();   // every thread's additions precede the release below
      if (tid == 0) red_release_add(cnt1(a, cur.p, cur.s), 1u);
    } else {
      // ---- pointwise operation on chunk cur.k of slab cur.s's nodes ----
      const int64_t s0 = slab_start(a, cur.s), s1 = slab_start(a, cur.s + 1);
      const int64_t lo = s0 + (int64_t)cur.k * a.chunk;
      const int64_t hi = lo + a.chunk < s1 ? lo + a.chunk : s1;
      if (lo < hi) {
        PointOp<T> f{ph.op, (T)ph.c[0], (T)ph.c[1], (T)ph.c[2], (T)ph.c[3]};
        pointwise<T, NT>(a, f, lo, hi);
      }
      __syncthreads();   // every thread's stores precede the release below
      if (tid == 0) red_release_add(cnt2(a, cur.p, cur.s), 1u);
    }
    __syncthreads();   // the item is done in every thread; sh_item[1] is written
    if (tid == 0) {
      const Item nx = sh_item[1];
      sh_item[0] = nx;
      if (!PF && nx.kind == 1) issue(nx);
      cd = nd;
      cv[0] = nv[0];
      cv[1] = nv[1];
    }
    __syncthreads();
  }
  if (failed && tid == 0) {
    atomicExch(a.err, 1u);
    // copies still in flight land before the block's shared memory is released
    for (int q = 0; q < NBUF; ++q)
      if (pend & (1u << q))
        for (uint32_t w = 0; w < kWaitLimit; ++w)
          if (mbar_try_wait(&bar[q], (par >> q) & 1u)) break;
  }
}

template <typename T, int EB, bool PF>
bool launch_fused(FusedSmooth& a, cudaStream_t s) {
  using C = Ax8<T, EB>;
  const size_t smem = sizeof(T) * (size_t)EB * ((PF ? 2 : 1) * C::GELEM + 3 * C::STAGE);
  static int grid = 0;
  if (grid == 0) {
    cudaFuncSetAttribute(k_sem_smooth8<T, EB, PF>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    int dev = 0, sms = 0, per_sm = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_sem_smooth8<T, EB, PF>, 64 * EB, smem);
    grid = sms * (per_sm > 0 ? per_sm : 1);
  }
  cudaMemsetAsync(a.ctl, 0, sizeof(unsigned) * (size_t)fused_ctl_words(a.lat), s);
  const unsigned blocks = (unsigned)std::min<int64_t>(grid, std::max<int64_t>(a.total, 1));
  // cooperative: every block is resident, which the static schedule's waits rely on
  void* args[] = {(void*)&a};
  const cudaError_t e = cudaLaunchCooperativeKernel((const void*)k_sem_smooth8<T, EB, PF>, dim3(blocks),
                                                    dim3(64 * EB), args, smem, s);
  if (e != cudaSuccess) return false;
  g_launches.fetch_add(1, std::memory_order_relaxed);
  return true;
}

}  // namespace

int fused_ctl_words(const Lattice& lat) { return 2 + 2 * kFusedMaxPhases * std::max(lat.nez, 1); }

bool fused_plan(FusedSmooth& a, int variant) {
  const int EB = variant == 1 ? 2 : 1;
  const Lattice& L = a.lat;
  a.nslab = L.nez;
  a.spp = L.nex * L.ney;
  if (a.nphase < 1 || a.nphase > kFusedMaxPhases || a.ph[0].src != FSRC_NONE) return false;
  if (a.nslab < 1 || a.spp < 1 || a.E != (int64_t)a.spp * a.nslab) return false;
  if ((int64_t)L.NX * L.NY * L.NZ != a.n || L.NX != 7 * L.nex + 1 || L.NY != 7 * L.ney + 1 ||
      L.NZ != 7 * L.nez + 1)
    return false;
  a.m1 = (a.spp + EB - 1) / EB;
  a.chunk = 64 * EB * 32;
  const int64_t plane = (int64_t)L.NX * L.NY;
  int64_t maxr = 0;
  for (int s = 0; s < a.nslab; ++s) {
    const int64_t s0 = s == 0 ? 0 : ((7 * s * plane) & ~int64_t(3));
    const int64_t s1 = s + 1 == a.nslab ? a.n : ((7 * (int64_t)(s + 1) * plane) & ~int64_t(3));
    maxr = std::max(maxr, s1 - s0);
  }
  a.m2 = (int)((maxr + a.chunk - 1) / a.chunk);
  a.tsteps = 3 * (a.nphase - 1) + a.nslab + 1;
  if (a.tsteps > kFusedMaxT) return false;
  uint64_t acc = 0;
  for (int t = 0; t < a.tsteps; ++t) {
    a.toff[t] = (uint32_t)acc;
    for (int p = 0; p < a.nphase; ++p) {
      const int s2 = t - 3 * p - 1, s1 = t - 3 * p;
      if (s2 >= 0 && s2 < a.nslab) acc += (uint64_t)a.m2;
      if (a.ph[p].src != FSRC_NONE && s1 >= 0 && s1 < a.nslab) acc += (uint64_t)a.m1;
    }
  }
  a.toff[a.tsteps] = (uint32_t)acc;
  if (acc >= (uint64_t(1) << 31)) return false;
  a.total = (uint32_t)acc;
  return true;
}

template <>
bool sem_smooth8<float>(FusedSmooth& a, int variant, cudaStream_t s) {
  (void)variant;
  return launch_fused<float, 2, true>(a, s);
}

template <>
bool sem_smooth8<double>(FusedSmooth& a, int variant, cudaStream_t s) {
  if (variant == 3) return launch_fused<double, 1, true>(a, s);
  return launch_fused<double, 1, false>(a, s);
}

cudaError_t sem_smooth8_set_eo(const double* eo) {
  float f[64];
  for (int i = 0; i < 64; ++i) f[i] = (float)eo[i];
  cudaError_t e = cudaMemcpyToSymbol(c_eo_d, eo, sizeof(double) * 64);
  if (e != cudaSuccess) return e;
  return cudaMemcpyToSymbol(c_eo_f, f, sizeof(f));
}

}  // namespace chebmg
