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
// read again soon after they were written.
//
// Warp specialisation.  The compute warps of a block never wait on bookkeeping: one control
// lane (its own warp) reads dependency counters, starts the TMA copy of an operator item's
// geometric factors into one of two shared-memory buffers, hands items over through two
// mbarrier slots and publishes completions, up to two items ahead of the compute warps.  Every
// wait is bounded (2 s for a dependency, 4 s without progress): on timeout the error flag is
// raised, every block stops after its current item, and copies in flight are waited for
// (bounded) before a block leaves.
//
// Memory ordering.  Vectors written in this launch are read with ld.global.cg (L2, never a stale
// L1 line).  A finished item: compute warps' writes, named barrier, mbarrier arrival (release,
// CTA scope), the control lane's wait (acquire, CTA scope) and its release increment of the
// task counter at GPU scope.  A dependency: relaxed load of the counter, acquire fence, the
// descriptor written to shared memory and the slot's mbarrier arrival (release, CTA scope),
// the compute warps' wait (acquire, CTA scope).
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

__device__ __forceinline__ unsigned ld_relaxed(const unsigned* p) {
  unsigned v;
  asm volatile("ld.relaxed.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

__device__ __forceinline__ void red_release_add(unsigned* p, unsigned v) {
  asm volatile("red.release.gpu.global.add.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

__device__ __forceinline__ void fence_acq_rel() { asm volatile("fence.acq_rel.gpu;" ::: "memory"); }

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
__device__ void pointwise(const FusedSmooth& a, const PointOp<T>& f, int64_t lo, int64_t hi, int64_t off) {
  using V = typename Vec16<T>::type;
  constexpr int L = Vec16<T>::L;
  constexpr int VPT = 2;
  const unsigned rd = op_reads(f.op), wr = op_writes(f.op);
  T* X = static_cast<T*>(a.x) + off;   // right-hand side at offset off; S is shared
  T* Rv = static_cast<T*>(a.r) + off;
  T* Dv = static_cast<T*>(a.d) + off;
  T* Y = static_cast<T*>(a.y) + off;
  const T* S = static_cast<const T*>(a.S);
  const T* B = static_cast<const T*>(a.b) + off;
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

__device__ __forceinline__ void named_sync(int id, int nthreads) {
  asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(nthreads) : "memory");
}
// AND of `pred` over the nthreads threads of named barrier `id` (a barrier as well).
__device__ __forceinline__ bool named_and(int id, int nthreads, bool pred) {
  uint32_t r;
  asm volatile(
      "{\n\t.reg .pred p, q;\n\t"
      "setp.ne.u32 p, %1, 0;\n\t"
      "bar.red.and.pred q, %2, %3, p;\n\t"
      "selp.u32 %0, 1, 0, q;\n\t}"
      : "=r"(r)
      : "r"((uint32_t)pred), "r"(id), "r"(nthreads)
      : "memory");
  return r != 0;
}
__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_addr(bar)) : "memory");
}

// Warp roles: warps 0 .. 2 EB - 1 compute (64 threads per element), the last warp controls.
// Work items of block b: b, b + grid, b + 2 grid, ...; item j of the block goes through slot
// j mod 2: the control lane prepares it (dependencies complete, descriptor in shared memory,
// for an operator item the TMA copy of its geometric factors into the slot's buffer) and
// completes ready[slot] (its arrival plus the copy's bytes); the compute warps wait on
// ready[slot], do the item and complete done[slot]; the control lane then publishes the item's
// completion (release increment of its task counter).  The control lane never blocks on one
// condition: it publishes finished items and prepares the next ones as each becomes possible,
// so an item whose dependencies include this block's own earlier items cannot stall it.
template <typename T, int EB>
__global__ void __launch_bounds__(64 * EB + 32, 3) k_sem_smooth8(const __grid_constant__ FusedSmooth a) {
  using C = Ax8<T, EB>;
  constexpr int R = C::R, P = C::P, NC = 64 * EB;
  extern __shared__ __align__(128) unsigned char smem_raw[];
  __shared__ __align__(8) uint64_t ready[2], done[2];
  __shared__ Item sh_item[2];
  T* sG = reinterpret_cast<T*>(smem_raw);   // [2][EB * GELEM], buffer = slot
  T* sU = sG + 2 * EB * C::GELEM;
  T* sR = sU + EB * C::STAGE;
  T* sS = sR + EB * C::STAGE;
  const int tid = threadIdx.x;
  if (tid == 0) {
    for (int q = 0; q < 2; ++q) {
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_addr(&ready[q])) : "memory");
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_addr(&done[q])) : "memory");
    }
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();

  if (tid >= NC) {
    // ---------------- control lane ----------------
    if (tid != NC) return;
    const T* G = static_cast<const T*>(a.G);
    uint32_t w = blockIdx.x;
    uint32_t jp = 0, jr = 0;       // next item to prepare / to publish
    Item held[2] = {Item{0, 0, 0, 0}, Item{0, 0, 0, 0}};
    bool ended = false;            // the terminating empty item is prepared
    bool have_next = false;
    Item nx{0, 0, 0, 0};
    Deps nd{{nullptr, nullptr}, {0u, 0u}};
    unsigned long long idle_since = global_ns(), dep_since = 0;
    bool failed = false;
    for (;;) {
      bool progress = false;
      // publish the completion of the oldest item in the compute warps' hands
      if (jr < jp && held[jr & 1].kind != 0 && mbar_try_wait(&done[jr & 1], (jr >> 1) & 1u)) {
        const Item& it = held[jr & 1];
        red_release_add(it.kind == 1 ? cnt1(a, it.p, it.s) : cnt2(a, it.p, it.s), 1u);
        ++jr;
        progress = true;
      }
      // prepare the next item once its slot is free and its dependencies are complete
      if (!ended && jp < jr + 2) {
        if (!have_next) {
          nx = *(volatile const unsigned*)a.err ? Item{0, 0, 0, 0} : decode(a, w);
          w += gridDim.x;
          nd = deps_of(a, nx);
          have_next = true;
          dep_since = global_ns();
        }
        bool ok = true;
        for (int q = 0; q < 2; ++q)
          if (nd.c[q] && ld_relaxed(nd.c[q]) < nd.t[q]) ok = false;
        if (!ok && (global_ns() - dep_since > kFusedWaitNs || *(volatile const unsigned*)a.err)) {
          failed = true;   // give up: hand the compute warps the empty item
          nx = Item{0, 0, 0, 0};
          ok = true;
        }
        if (ok) {
          fence_acq_rel();   // acquire side of the counters observed above
          const int slot = jp & 1;
          sh_item[slot] = nx;
          held[slot] = nx;
          if (nx.kind == 1) {
            const int bt = nx.k / a.ngroups;   // element batch of the item
            const int64_t e0 = (int64_t)nx.s * a.spp + (int64_t)bt * EB;
            const int nv = min(EB, a.spp - bt * EB);
            const uint32_t bytes = (uint32_t)(nv * C::GELEM * sizeof(T));
            asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(&ready[slot])),
                         "r"(bytes)
                         : "memory");
            bulk_copy_g(sG + slot * EB * C::GELEM, G + e0 * C::GELEM, bytes, &ready[slot]);
          } else {
            mbar_arrive(&ready[slot]);
          }
          if (nx.kind == 0) ended = true;
          ++jp;
          have_next = false;
          progress = true;
        }
      }
      // done when every prepared item is published (the empty item needs none)
      if (ended && jr + 1 == jp) break;
      if (progress) {
        idle_since = global_ns();
      } else {
        if (global_ns() - idle_since > 2 * kFusedWaitNs) {   // the compute warps stopped answering
          failed = true;
          break;
        }
        __nanosleep(64);
      }
    }
    if (failed) {
      atomicExch(a.err, 1u);
      // copies still in flight land before the block's shared memory is released
      for (uint32_t j = jr; j < jp; ++j)
        if (held[j & 1].kind == 1)
          for (uint32_t t = 0; t < kWaitLimit; ++t)
            if (mbar_try_wait(&ready[j & 1], (j >> 1) & 1u)) break;
    }
    return;
  }

  // ---------------- compute warps ----------------
  const int le = tid >> 6, tt = tid & 63, ca = tt & 7, cb = tt >> 3;
  T* Y = static_cast<T*>(a.y);
  T* su = sU + le * C::STAGE;
  T* sr = sR + le * C::STAGE;
  T* ss = sS + le * C::STAGE;
  // ids of the item's element column and the values of its first right-hand side
  auto gather = [&](const Item& it, uint32_t (&g)[8], T (&col)[8]) {
    const int bt = it.k / a.ngroups, q0 = (it.k % a.ngroups) * a.gsz;
    const T* src = static_cast<const T*>(a.ph[it.p].src == FSRC_X ? a.x : a.d) + (int64_t)q0 * a.ld;
    const int64_t e = (int64_t)it.s * a.spp + (int64_t)bt * EB + le;
    column_ids<true>(nullptr, a.lat, e, bt * EB + le < a.spp, ca, cb, g);
#pragma unroll
    for (int k = 0; k < 8; ++k) col[k] = (g[k] & kGidDirichlet) ? T(0) : __ldcg(src + (g[k] & kGidMask));
  };
  for (uint32_t j = 0;; ++j) {
    const int slot = j & 1;
    bool ok = false;
    const unsigned long long t0 = global_ns();
    for (;;) {
      if (mbar_try_wait(&ready[slot], (j >> 1) & 1u)) {
        ok = true;
        break;
      }
      if (global_ns() - t0 > 2 * kFusedWaitNs) break;
    }
    if (!named_and(1, NC, ok)) {
      if (tid == 0) atomicExch(a.err, 1u);
      break;
    }
    const Item cur = sh_item[slot];
    if (cur.kind == 0) break;
    const FusedPhase& ph = a.ph[cur.p];
    if (cur.kind == 1) {
      // ---- operator on EB elements of plane cur.s, for the item's right-hand sides: y += A v ----
      const int bt = cur.k / a.ngroups, q0 = (cur.k % a.ngroups) * a.gsz;
      const int q1 = q0 + a.gsz < a.nb ? q0 + a.gsz : a.nb;
      const bool valid = bt * EB + le < a.spp;
      const T* srcb = static_cast<const T*>(ph.src == FSRC_X ? a.x : a.d);
      uint32_t g[8];
      T col[8];
      gather(cur, g, col);
      const T* gG = sG + slot * EB * C::GELEM + le * C::GELEM;
      for (int q = q0; q < q1; ++q) {
#pragma unroll
        for (int k = 0; k < 8; ++k) su[k * P + cb * R + ca] = col[k];
        T ut[8];
        line8<T, 0>(col, ut);
        T nxt[8];
        if (q + 1 < q1) {   // the next right-hand side's values, in flight during this one
          const T* src = srcb + (int64_t)(q + 1) * a.ld;
#pragma unroll
          for (int k = 0; k < 8; ++k) nxt[k] = (g[k] & kGidDirichlet) ? T(0) : __ldcg(src + (g[k] & kGidMask));
        }
        named_sync(1, NC);
        {
          T v[8], o[8];
          ld_row(su + cb * P + ca * R, v);
          line8<T, 0>(v, o);
          st_row(sr + cb * P + ca * R, o);
#pragma unroll
          for (int jj = 0; jj < 8; ++jj) v[jj] = su[cb * P + jj * R + ca];
          line8<T, 0>(v, o);
#pragma unroll
          for (int jj = 0; jj < 8; ++jj) ss[cb * P + jj * R + ca] = o[jj];
        }
        named_sync(1, NC);   // the r and s passes wrote points that other threads read next
        T wt[8];
#pragma unroll
        for (int k = 0; k < 8; ++k) {
          const int p = k * 64 + cb * 8 + ca;
          const int qq = k * P + cb * R + ca;
          const T ur = sr[qq], us = ss[qq], utk = ut[k];
          const T g00 = gG[p], g01 = gG[512 + p], g02 = gG[1024 + p];
          const T g11 = gG[1536 + p], g12 = gG[2048 + p], g22 = gG[2560 + p];
          sr[qq] = g00 * ur + g01 * us + g02 * utk;
          ss[qq] = g01 * ur + g11 * us + g12 * utk;
          wt[k] = g02 * ur + g12 * us + g22 * utk;
        }
        T yt[8];
        line8<T, 1>(wt, yt);
        named_sync(1, NC);
        {
          T v[8], o[8];
          ld_row(sr + cb * P + ca * R, v);
          line8<T, 1>(v, o);
          st_row(su + cb * P + ca * R, o);
        }
        named_sync(1, NC);
        {
          T v[8], o[8];
#pragma unroll
          for (int jj = 0; jj < 8; ++jj) v[jj] = ss[cb * P + jj * R + ca];
          line8<T, 1>(v, o);
#pragma unroll
          for (int jj = 0; jj < 8; ++jj) su[cb * P + jj * R + ca] += o[jj];
        }
        named_sync(1, NC);
        if (valid) {
          T* Yq = Y + (int64_t)q * a.ld;
#pragma unroll
          for (int k = 0; k < 8; ++k) {
            const T v = su[k * P + cb * R + ca] + yt[k];
            if (!(g[k] & kGidDirichlet)) atomicAdd(&Yq[g[k] & kGidMask], v);
          }
        }
        if (q + 1 < q1) {
          named_sync(1, NC);   // stage buffers free for the next right-hand side
#pragma unroll
          for (int k = 0; k < 8; ++k) col[k] = nxt[k];
        }
      }
    } else {
      // ---- pointwise operation on chunk cur.k of slab cur.s's nodes ----
      const int ck = cur.k / a.ngroups, q0 = (cur.k % a.ngroups) * a.gsz;
      const int q1 = q0 + a.gsz < a.nb ? q0 + a.gsz : a.nb;
      const int64_t s0 = slab_start(a, cur.s), s1 = slab_start(a, cur.s + 1);
      const int64_t lo = s0 + (int64_t)ck * a.chunk;
      const int64_t hi = lo + a.chunk < s1 ? lo + a.chunk : s1;
      if (lo < hi) {
        PointOp<T> f{ph.op, (T)ph.c[0], (T)ph.c[1], (T)ph.c[2], (T)ph.c[3]};
        for (int q = q0; q < q1; ++q) pointwise<T, NC>(a, f, lo, hi, (int64_t)q * a.ld);
      }
    }
    named_sync(1, NC);   // the item is done in every compute thread (stage buffers free)
    if (tid == 0) mbar_arrive(&done[slot]);
  }
}

template <typename T, int EB>
bool launch_fused(FusedSmooth& a, cudaStream_t s) {
  using C = Ax8<T, EB>;
  const size_t smem = sizeof(T) * (size_t)EB * (2 * C::GELEM + 3 * C::STAGE);
  static int grid = 0;
  if (grid == 0) {
    cudaFuncSetAttribute(k_sem_smooth8<T, EB>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    int dev = 0, sms = 0, per_sm = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_sem_smooth8<T, EB>, 64 * EB + 32, smem);
    grid = sms * (per_sm > 0 ? per_sm : 1);
  }
  cudaMemsetAsync(a.ctl, 0, sizeof(unsigned) * (size_t)fused_ctl_words(a.lat), s);
  const unsigned blocks = (unsigned)std::min<int64_t>(grid, std::max<int64_t>(a.total, 1));
  // cooperative: every block is resident, which the static schedule's waits rely on
  void* args[] = {(void*)&a};
  const cudaError_t e = cudaLaunchCooperativeKernel((const void*)k_sem_smooth8<T, EB>, dim3(blocks),
                                                    dim3(64 * EB + 32), args, smem, s);
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
  if (a.nb < 1 || a.gsz < 1 || (a.nb > 1 && a.ld % 4 != 0)) return false;
  a.ngroups = (a.nb + a.gsz - 1) / a.gsz;
  a.m1 = (a.spp + EB - 1) / EB * a.ngroups;
  a.chunk = 64 * EB * 32;
  const int64_t plane = (int64_t)L.NX * L.NY;
  int64_t maxr = 0;
  for (int s = 0; s < a.nslab; ++s) {
    const int64_t s0 = s == 0 ? 0 : ((7 * s * plane) & ~int64_t(3));
    const int64_t s1 = s + 1 == a.nslab ? a.n : ((7 * (int64_t)(s + 1) * plane) & ~int64_t(3));
    maxr = std::max(maxr, s1 - s0);
  }
  a.m2 = (int)((maxr + a.chunk - 1) / a.chunk) * a.ngroups;
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
  return launch_fused<float, 2>(a, s);
}

template <>
bool sem_smooth8<double>(FusedSmooth& a, int variant, cudaStream_t s) {
  (void)variant;
  return launch_fused<double, 1>(a, s);
}

cudaError_t sem_smooth8_set_eo(const double* eo) {
  float f[64];
  for (int i = 0; i < 64; ++i) f[i] = (float)eo[i];
  cudaError_t e = cudaMemcpyToSymbol(c_eo_d, eo, sizeof(double) * 64);
  if (e != cudaSuccess) return e;
  return cudaMemcpyToSymbol(c_eo_f, f, sizeof(f));
}

}  // namespace chebmg
