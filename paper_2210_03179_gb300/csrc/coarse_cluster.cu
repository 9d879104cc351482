// Coarse-grid CG on one thread-block cluster (box lattices at N = 1).
//
// The N = 1 coarse problem of a box mesh is a 27-point operator on the node lattice
// nx x ny x nz.  Its interior planes z = 1 .. nz-2 are split over the CTAs of one cluster
// (up to 16, one per SM); each CTA keeps its planes' rows in registers, the FP32 copy of the
// operator (forward half of the stencil, the other half read from the neighbour row by
// symmetry) in shared memory, and the vector each product reads in a shared-memory plane
// buffer with one halo plane below and above.  A product publishes its rows into the own
// buffer and pushes the first and last plane into the neighbours' halos through distributed
// shared memory; one hardware cluster barrier (release / acquire) then makes everything
// visible.  Dot products sum the CTAs' partials in rank order in every CTA, so all CTAs take
// identical decisions -- there is no spinning anywhere, only cluster barriers that every CTA
// reaches the same number of times.
//
// The method is the one of the grid-wide persistent kernel: FP64 CG (Polak-Ribiere beta for
// the FP32 preconditioner) preconditioned by one application of Algorithm 2 (4th kind,
// beta = 1) of degree m from a zero guess, Jacobi-scaled, in FP32.  The CG's own product
// A p is FP64 (values from global memory, in the same symmetric layout).
#include <cooperative_groups.h>

#include <algorithm>

#include "common.cuh"

namespace cg = cooperative_groups;

namespace chebmg {
namespace {

inline void count() { g_launches.fetch_add(1, std::memory_order_relaxed); }

constexpr int kCcThreads = 512;

__device__ __forceinline__ double cc_warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Sums three per-thread values over the block (fixed order); result in every thread.
__device__ __forceinline__ void cc_block_sum3(double* sh, double& a, double& b, double& c) {
  a = cc_warp_sum(a);
  b = cc_warp_sum(b);
  c = cc_warp_sum(c);
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  __syncthreads();   // scratch free (previous use finished)
  if (l == 0) {
    sh[3 * w] = a;
    sh[3 * w + 1] = b;
    sh[3 * w + 2] = c;
  }
  __syncthreads();
  double ta = 0.0, tb = 0.0, tc = 0.0;
#pragma unroll
  for (int q = 0; q < kCcThreads / 32; ++q) {
    ta += sh[3 * q];
    tb += sh[3 * q + 1];
    tc += sh[3 * q + 2];
  }
  a = ta;
  b = tb;
  c = tc;
}

// Cluster-wide sum of three values (each CTA's block totals, equal in all its threads):
// every CTA posts its totals into its own slot of this parity, a cluster barrier, then warp 0
// of every CTA adds the CTAs' totals in rank order.  Two parities suffice: a slot is written
// again two reductions later, after a barrier that every CTA reaches only once it has read it.
__device__ __forceinline__ void cc_cluster_sum3(cg::cluster_group& cl, double* red, double* bcast, int par,
                                                int ctas, double& a, double& b, double& c) {
  if (threadIdx.x == 0) {
    red[4 * par] = a;
    red[4 * par + 1] = b;
    red[4 * par + 2] = c;
  }
  cl.sync();
  if (threadIdx.x < 32) {
    double ta = 0.0, tb = 0.0, tc = 0.0;
    if ((int)threadIdx.x < ctas) {
      const double* r = cl.map_shared_rank(red, (unsigned)threadIdx.x);
      ta = r[4 * par];
      tb = r[4 * par + 1];
      tc = r[4 * par + 2];
    }
    // fixed shuffle tree over lanes = ranks: the same order in every CTA
    ta = cc_warp_sum(ta);
    tb = cc_warp_sum(tb);
    tc = cc_warp_sum(tc);
    if (threadIdx.x == 0) {
      bcast[0] = ta;
      bcast[1] = tb;
      bcast[2] = tc;
    }
  }
  __syncthreads();
  a = bcast[0];
  b = bcast[1];
  c = bcast[2];
  __syncthreads();   // bcast is reused by the next reduction
}

template <int RPT>
__global__ void __launch_bounds__(kCcThreads, 1) k_coarse_cluster(CoarseCluster a) {
  cg::cluster_group cl = cg::this_cluster();
  const int rank = (int)cl.block_rank();
  const int C = a.ctas;
  const int NX = a.nx, NY = a.ny, NXY = a.nx * a.ny;
  const int P = a.nz - 2;
  const int per = P / C, extra = P % C;
  const int np = per + (rank < extra ? 1 : 0);
  const int z0 = 1 + rank * per + min(rank, extra);
  const int np_dn = rank > 0 ? per + (rank - 1 < extra ? 1 : 0) : 0;   // planes of rank - 1
  const int rows = np * NXY;
  const int RM = a.rmax;                      // slot stride of the staged values
  const int PB = (a.rmax / NXY + 2) * NXY;    // plane-buffer length (halo planes included)
  const int64_t n = (int64_t)NXY * a.nz;
  const int64_t g0 = (int64_t)z0 * NXY;

  extern __shared__ __align__(16) unsigned char smem[];
  double* p64 = reinterpret_cast<double*>(smem);   // [PB] FP64 exchange (CG direction p)
  double* red = p64 + PB;                          // [2][4] cluster reduction slots
  double* bcast = red + 8;                         // [4]
  double* scratch = bcast + 4;                     // [3 * 16] block reduction
  float* vals = reinterpret_cast<float*>(scratch + 3 * (kCcThreads / 32));   // [14][RM]
  float* const xf0 = vals + 14 * RM;   // FP32 exchange, two buffers
  float* const xf1 = xf0 + PB;
  double* const xs = reinterpret_cast<double*>(xf1 + PB);   // [RM] the iterate (8-byte aligned: PB even)

  // zero the exchange buffers (halo planes of the lattice boundary stay zero), stage values
  for (int i = threadIdx.x; i < PB; i += kCcThreads) {
    p64[i] = 0.0;
    xf0[i] = 0.f;
    xf1[i] = 0.f;
  }
  for (int k = 0; k < 14; ++k)
    for (int i = threadIdx.x; i < rows; i += kCcThreads) vals[k * RM + i] = __ldg(&a.val32[k * n + g0 + i]);
  // neighbours' buffers (distributed shared memory); every CTA has started after this barrier
  cl.sync();
  const bool has_dn = rank > 0, has_up = rank + 1 < C;
  double* p64_dn = has_dn ? cl.map_shared_rank(p64, (unsigned)(rank - 1)) : p64;
  double* p64_up = has_up ? cl.map_shared_rank(p64, (unsigned)(rank + 1)) : p64;
  float* const xf0_dn = has_dn ? cl.map_shared_rank(xf0, (unsigned)(rank - 1)) : xf0;
  float* const xf1_dn = has_dn ? cl.map_shared_rank(xf1, (unsigned)(rank - 1)) : xf1;
  float* const xf0_up = has_up ? cl.map_shared_rank(xf0, (unsigned)(rank + 1)) : xf0;
  float* const xf1_up = has_up ? cl.map_shared_rank(xf1, (unsigned)(rank + 1)) : xf1;
  const float* vals_dn = has_dn ? cl.map_shared_rank(vals, (unsigned)(rank - 1)) : vals;

  // rows of this thread: local row l = threadIdx.x + q * kCcThreads
  bool act[RPT];
  float sf[RPT];
  double r[RPT], p[RPT], z[RPT], y[RPT];
#pragma unroll
  for (int q = 0; q < RPT; ++q) {
    const int l = threadIdx.x + q * kCcThreads;
    const int ip = l % NXY, ix = ip % NX, iy = ip / NX;
    const bool live = l < rows;
    sf[q] = live ? __ldg(&a.invDf[g0 + l]) : 0.f;
    act[q] = live && ix >= 1 && ix <= NX - 2 && iy >= 1 && iy <= NY - 2 && sf[q] != 0.f;
    r[q] = act[q] ? a.b[g0 + l] : 0.0;
    p[q] = z[q] = y[q] = 0.0;
    if (live) xs[l] = 0.0;
  }

  // y = A v for FP32 v published in exchange buffer `buf` (values staged in shared memory)
  auto spmv_f = [&](int buf, float (&yf)[RPT]) {
    const float* xb = buf ? xf1 : xf0;
#pragma unroll
    for (int q = 0; q < RPT; ++q) {
      float acc = 0.f;
      if (act[q]) {
        const int l = threadIdx.x + q * kCcThreads;
        const int pz = l / NXY, ip = l - pz * NXY;
        const float* xc = xb + (pz + 1) * NXY + ip;
        const float* v = vals + l;
        const float* vb = pz > 0 ? vals + (l - NXY) : (has_dn ? vals_dn + (np_dn - 1) * NXY + ip : vals + l);
        acc = v[0] * xc[0];
#pragma unroll
        for (int k = 1; k < 5; ++k) {
          const int o = cc_dy(k) * NX + cc_dx(k);
          acc = fmaf(v[k * RM], xc[o], acc);
          acc = fmaf(v[k * RM - o], xc[-o], acc);
        }
#pragma unroll
        for (int k = 5; k < 14; ++k) {
          const int o = cc_dy(k) * NX + cc_dx(k);
          acc = fmaf(v[k * RM], xc[NXY + o], acc);
          acc = fmaf(vb[k * RM - o], xc[-NXY - o], acc);
        }
      }
      yf[q] = acc;
    }
  };
  // publish FP32 rows into buffer `buf` (own planes and the neighbours' halo planes)
  auto publish_f = [&](int buf, const float (&v)[RPT]) {
    float* const own = buf ? xf1 : xf0;
    float* const dn = buf ? xf1_dn : xf0_dn;
    float* const up = buf ? xf1_up : xf0_up;
#pragma unroll
    for (int q = 0; q < RPT; ++q) {
      if (!act[q]) continue;
      const int l = threadIdx.x + q * kCcThreads;
      const int pz = l / NXY, ip = l - pz * NXY;
      own[(pz + 1) * NXY + ip] = v[q];
      if (pz == 0 && has_dn) dn[(np_dn + 1) * NXY + ip] = v[q];
      if (pz == np - 1 && has_up) up[ip] = v[q];
    }
  };
  auto publish_d = [&](const double (&v)[RPT]) {
#pragma unroll
    for (int q = 0; q < RPT; ++q) {
      if (!act[q]) continue;
      const int l = threadIdx.x + q * kCcThreads;
      const int pz = l / NXY, ip = l - pz * NXY;
      p64[(pz + 1) * NXY + ip] = v[q];
      if (pz == 0 && has_dn) p64_dn[(np_dn + 1) * NXY + ip] = v[q];
      if (pz == np - 1 && has_up) p64_up[ip] = v[q];
    }
  };
  // y = A p in FP64 (values from global memory, same symmetric layout)
  auto spmv_d = [&]() {
#pragma unroll
    for (int q = 0; q < RPT; ++q) {
      double acc = 0.0;
      if (act[q]) {
        const int l = threadIdx.x + q * kCcThreads;
        const int pz = l / NXY, ip = l - pz * NXY;
        const double* pc = p64 + (pz + 1) * NXY + ip;
        const double* v = a.val64 + g0 + l;
        acc = __ldg(v) * pc[0];
#pragma unroll
        for (int k = 1; k < 5; ++k) {
          const int o = cc_dy(k) * NX + cc_dx(k);
          acc = fma(__ldg(v + k * n), pc[o], acc);
          acc = fma(__ldg(v + k * n - o), pc[-o], acc);
        }
#pragma unroll
        for (int k = 5; k < 14; ++k) {
          const int o = cc_dy(k) * NX + cc_dx(k);
          acc = fma(__ldg(v + k * n), pc[NXY + o], acc);
          acc = fma(__ldg(v + k * n - NXY - o), pc[-NXY - o], acc);
        }
      }
      y[q] = acc;
    }
  };

  const double c0 = 4.0 / (3.0 * a.lmax);
  __shared__ CoarseCoef coef;
  __shared__ double s_alpha, s_beta;
  coarse_coef_fill(coef, a.degree, a.lmax);
  __syncthreads();
  int xpar = 0;   // FP32 exchange buffer parity
  // z = M r: Algorithm 2 of degree m from a zero guess in FP32 (Jacobi-scaled)
  auto precond = [&]() {
    float df[RPT], rf[RPT], zf[RPT], yf[RPT];
    const float c0f = (float)c0;
#pragma unroll
    for (int q = 0; q < RPT; ++q) {
      rf[q] = (float)r[q];
      df[q] = c0f * sf[q] * rf[q];
      zf[q] = 0.f;
    }
    for (int i = 1; i < a.degree; ++i) {
#pragma unroll
      for (int q = 0; q < RPT; ++q) zf[q] += df[q];
      publish_f(xpar, df);
      cl.sync();
      spmv_f(xpar, yf);
      xpar ^= 1;
      const float c1 = coef.c1f[i], c2 = coef.c2f[i];
#pragma unroll
      for (int q = 0; q < RPT; ++q) {
        rf[q] -= yf[q];
        df[q] = c1 * df[q] + c2 * sf[q] * rf[q];
      }
    }
#pragma unroll
    for (int q = 0; q < RPT; ++q) z[q] = (double)(zf[q] + df[q]);
  };
  int rpar = 0;   // reduction parity
  auto allsum3 = [&](double& s0, double& s1, double& s2) {
    cc_block_sum3(scratch, s0, s1, s2);
    cc_cluster_sum3(cl, red, bcast, rpar, C, s0, s1, s2);
    rpar ^= 1;
  };
  auto finish = [&](int status, int it) {
#pragma unroll
    for (int q = 0; q < RPT; ++q) {
      const int l = threadIdx.x + q * kCcThreads;
      if (l < rows) a.x[g0 + l] = xs[l];
    }
    // the lattice's bottom and top planes (Dirichlet) are zero
    if (rank == 0)
      for (int i = threadIdx.x; i < NXY; i += kCcThreads) a.x[i] = 0.0;
    if (rank == C - 1)
      for (int i = threadIdx.x; i < NXY; i += kCcThreads) a.x[(int64_t)(a.nz - 1) * NXY + i] = 0.0;
    if (rank == 0 && threadIdx.x == 0) {
      a.ctl[2] = (unsigned)status;
      a.ctl[3] = (unsigned)it;
      if (status == CS_BREAKDOWN) atomicMax((int*)&a.ctl[4], (int)CS_BREAKDOWN);
    }
    cl.sync();   // no CTA leaves while another may still read its shared memory
  };

  precond();
  double rz = 0.0, rr = 0.0, zero = 0.0;
#pragma unroll
  for (int q = 0; q < RPT; ++q) {
    p[q] = z[q];
    rz += r[q] * z[q];
    rr += r[q] * r[q];
  }
  allsum3(rz, rr, zero);
  double gam = rz;
  const double bb = rr;
  if (!(bb > 0.0) || !(gam >= 0.0)) {
    finish(bb == 0.0 ? CS_OK : CS_BREAKDOWN, 0);
    return;
  }
  const double tol2 = a.rtol * a.rtol * bb;
  for (int it = 1; it <= a.maxit; ++it) {
    publish_d(p);
    cl.sync();
    spmv_d();
    double pq = 0.0, u1 = 0.0, u2 = 0.0;
#pragma unroll
    for (int q = 0; q < RPT; ++q) pq += p[q] * y[q];
    allsum3(pq, u1, u2);
    if (!(pq > 0.0)) {
      finish(CS_BREAKDOWN, it);
      return;
    }
    const double alpha = block_div(&s_alpha, gam, pq);
#pragma unroll
    for (int q = 0; q < RPT; ++q) {
      const int l = threadIdx.x + q * kCcThreads;
      if (act[q]) xs[l] = fma(alpha, p[q], xs[l]);
      r[q] = fma(-alpha, y[q], r[q]);
    }
    precond();
    double rz2 = 0.0, rr2 = 0.0, zq = 0.0;
#pragma unroll
    for (int q = 0; q < RPT; ++q) {
      rz2 += r[q] * z[q];
      rr2 += r[q] * r[q];
      zq += z[q] * y[q];
    }
    allsum3(rz2, rr2, zq);
    if (!(rr2 == rr2)) {
      finish(CS_BREAKDOWN, it);
      return;
    }
    if (rr2 <= tol2) {
      finish(CS_OK, it);
      return;
    }
    // Polak-Ribiere (z_new, r_new - r_old) / (z_old, r_old) with r_new - r_old = -alpha A p:
    // the FP32 preconditioner is not exactly symmetric
    const double beta = block_div(&s_beta, -alpha * zq, gam);
    gam = rz2;
#pragma unroll
    for (int q = 0; q < RPT; ++q) p[q] = fma(beta, p[q], z[q]);
  }
  finish(CS_NOTCONV, a.maxit);
}

template <int RPT>
const void* cc_kernel() {
  return (const void*)k_coarse_cluster<RPT>;
}

const void* cc_kernel_for(int rpt) {
  switch (rpt) {
    case 1: return cc_kernel<1>();
    case 2: return cc_kernel<2>();
    case 3: return cc_kernel<3>();
    case 4: return cc_kernel<4>();
    case 5: return cc_kernel<5>();
    case 6: return cc_kernel<6>();
    default: return cc_kernel<8>();
  }
}

int cc_rpt(int rmax) {
  const int need = (rmax + kCcThreads - 1) / kCcThreads;
  if (need <= 6) return std::max(1, need);
  return need <= 8 ? 8 : 0;
}

}  // namespace

size_t coarse_cluster_smem(int nx, int ny, int rmax) {
  const size_t pb = (size_t)(rmax / (nx * ny) + 2) * nx * ny;
  return sizeof(double) * (pb + 8 + 4 + 3 * (kCcThreads / 32) + (size_t)rmax) +
         sizeof(float) * (14 * (size_t)rmax + 2 * pb);
}

bool coarse_cluster_plan(int nx, int ny, int nz, int* ctas, int* rmax, size_t* smem) {
  *ctas = 0;
  *rmax = 0;
  *smem = 0;
  const int P = nz - 2;
  if (nx < 3 || ny < 3 || P < 1) return false;
  const int C = std::min(16, P);
  const int pmax = (P + C - 1) / C;
  const int rm = pmax * nx * ny;
  if (cc_rpt(rm) == 0) return false;
  int dev = 0, optin = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return false;
  if (cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) != cudaSuccess) return false;
  const size_t sm = coarse_cluster_smem(nx, ny, rm);
  if (sm > (size_t)optin) return false;
  const void* fn = cc_kernel_for(cc_rpt(rm));
  if (cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm) != cudaSuccess ||
      cudaFuncSetAttribute(fn, cudaFuncAttributeNonPortableClusterSizeAllowed, 1) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  cudaLaunchConfig_t cfg = {};
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = (unsigned)C;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.gridDim = dim3((unsigned)C);
  cfg.blockDim = dim3(kCcThreads);
  cfg.dynamicSmemBytes = sm;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  int clusters = 0;
  if (cudaOccupancyMaxActiveClusters(&clusters, fn, &cfg) != cudaSuccess || clusters < 1) {
    cudaGetLastError();
    return false;
  }
  *ctas = C;
  *rmax = rm;
  *smem = sm;
  return true;
}

bool coarse_cluster_launch(const CoarseCluster& a, size_t smem, cudaStream_t s, cudaError_t* err) {
  const int rpt = cc_rpt(a.rmax);
  if (rpt == 0 || a.ctas < 1 || a.ctas > 16) {
    if (err) *err = cudaErrorInvalidConfiguration;
    return false;
  }
  cudaLaunchConfig_t cfg = {};
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = (unsigned)a.ctas;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.gridDim = dim3((unsigned)a.ctas);
  cfg.blockDim = dim3(kCcThreads);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  CoarseCluster arg = a;
  void* params[] = {&arg};
  const cudaError_t e = cudaLaunchKernelExC(&cfg, cc_kernel_for(rpt), params);
  count();
  if (err) *err = e;
  return e == cudaSuccess;
}

}  // namespace chebmg
