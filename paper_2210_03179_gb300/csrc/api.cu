// C-ABI entry points and host orchestration of the multigrid hot path.
//
// Host code here only sequences kernels (kernels.cu) on the context's stream:
// every arithmetic step of the smoother, the transfers, the coarse solves and
// the outer Krylov loop runs on the GPU.  The host reads back one or two FP64
// scalars per Krylov iteration to test convergence.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <stdexcept>
#include <string>
#include <vector>

#include "../../include/chebmg.h"
#include "common.cuh"
#include "setup_host.h"

using namespace chebmg;

namespace {

thread_local std::string g_last_error;

struct Error : std::runtime_error {
  int code;
  Error(int c, const std::string& m) : std::runtime_error(m), code(c) {}
};

#define CK(call)                                                                                    \
  do {                                                                                              \
    cudaError_t e_ = (call);                                                                        \
    if (e_ != cudaSuccess) {                                                                        \
      if (e_ == cudaErrorMemoryAllocation)                                                          \
        throw Error(CHEBMG_ENOMEM, std::string(#call) + ": " + cudaGetErrorString(e_));            \
      throw Error(CHEBMG_ECUDA, std::string(#call) + ": " + cudaGetErrorString(e_));               \
    }                                                                                               \
  } while (0)

inline void check_launch() {
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) throw Error(CHEBMG_ECUDA, std::string("kernel launch: ") + cudaGetErrorString(e));
}

// Optimized 4th-kind coefficients beta_i^{(k)}, k = 1..16 (Table 5, Sec. 8.1).
const double kBeta[16][16] = {
    {1.12500000000000},
    {1.02387287570313, 1.26408905371085},
    {1.00842544782028, 1.08867839208730, 1.33753125909618},
    {1.00391310427285, 1.04035811188593, 1.14863498546254, 1.38268869241000},
    {1.00212930146164, 1.02173711549260, 1.07872433192603, 1.19810065292663, 1.41322542791682},
    {1.00128517255940, 1.01304293035233, 1.04678215124113, 1.11616489419675, 1.23829020218444, 1.43524297106744},
    {1.00083464397912, 1.00843949430122, 1.03008707768713, 1.07408384092003, 1.15036186707366, 1.27116474046139, 1.45186658649364},
    {1.00057246631197, 1.00577427662415, 1.02050187922941, 1.05019803444565, 1.10115572984941, 1.18086042806856, 1.29838585382576, 1.46486073151099},
    {1.00040960072832, 1.00412439506106, 1.01460212148266, 1.03561113626671, 1.07139972529194, 1.12688273710962, 1.20785219140729, 1.32121930716746, 1.47529642820699},
    {1.00030312229652, 1.00304840660796, 1.01077022715387, 1.02619011597640, 1.05231724933755, 1.09255743207549, 1.15083376663972, 1.23172250870894, 1.34060802024460, 1.48386124407011},
    {1.00023058595209, 1.00231675024028, 1.00817245396304, 1.01982986566342, 1.03950210235324, 1.06965042700541, 1.11305754295742, 1.17290876275564, 1.25288300576792, 1.35725579919519, 1.49101672564139},
    {1.00017947200828, 1.00180189139619, 1.00634861907307, 1.01537864566306, 1.03056942830760, 1.05376019693943, 1.08699862592072, 1.13259183097913, 1.19316273358172, 1.27171293675110, 1.37169337969799, 1.49708418575562},
    {1.00014241921559, 1.00142906932629, 1.00503028986298, 1.01216910518495, 1.02414874342792, 1.04238158880820, 1.06842008128700, 1.10399010936759, 1.15102748242645, 1.21171811910125, 1.28854264865128, 1.38432619380991, 1.50229418757368},
    {1.00011490538261, 1.00115246376914, 1.00405357333264, 1.00979590573153, 1.01941300472994, 1.03401425035436, 1.05480599606629, 1.08311420301813, 1.12040891660892, 1.16833095655446, 1.22872122288238, 1.30365305707817, 1.39546814053678, 1.50681646209583},
    {1.00009404750752, 1.00094291696343, 1.00331449056444, 1.00800294833816, 1.01584236259140, 1.02772083317705, 1.04459535422831, 1.06750761206125, 1.09760092545889, 1.13613855366157, 1.18452361426236, 1.24432087304475, 1.31728069083392, 1.40536543893560, 1.51077872501845},
    {1.00007794828179, 1.00078126847253, 1.00274487974401, 1.00662291017015, 1.01309858836971, 1.02289448329337, 1.03678321409983, 1.05559875719896, 1.08024848405560, 1.11172607131497, 1.15112543431072, 1.19965584614973, 1.25865841744946, 1.32962412656664, 1.41421360695576, 1.51427891730346},
};

}  // namespace

namespace chebmg {

// Row k (1..16) of the optimized 4th-kind coefficient table, for other translation units.
const double* beta_row(int k) { return (k >= 1 && k <= 16) ? kBeta[k - 1] : nullptr; }
void set_last_error(const char* msg) { g_last_error = msg; }

enum { VB = 0, VX = 1, VR = 2, VD = 3, VY = 4, NV = 5 };
enum { TYPE_SEM = 0, TYPE_FD = 1 };

struct Level {
  int type = TYPE_SEM;
  int64_t n = 0;
  // SEM
  int N = 0, Q = 0, NP = 0;
  int64_t E = 0;
  uint32_t* gid = nullptr;
  // FD
  int mx = 0, my = 0, c_next = 2;
  double st[9] = {0};
  double lmax = 0.0;
  void* G[2] = {nullptr, nullptr};
  void* invD[2] = {nullptr, nullptr};
  void* D[2] = {nullptr, nullptr};
  void* Jn[2] = {nullptr, nullptr};   // interpolation from level+1 to this level, [Qf][Qc]
  void* v[2][NV] = {{nullptr}};
  int eb[2] = {2, 2};   // variant of the order-7 operator, per dtype (autotuned)
  Lattice lat = {0, 0, 0, 0, 0, 0};
};

}  // namespace chebmg

struct chebmg_ctx {
  chebmg_opts o;
  int type = TYPE_SEM;
  int dev = 0;
  bool fp32 = false;
  int pre = 0, post = 0;
  cudaStream_t s = nullptr;
  std::vector<Level> L;
  std::vector<void*> allocs;
  double* partial = nullptr;
  double* scal = nullptr;
  double* hscal = nullptr;      // pinned host copy of scal
  // the coarse CG runs inside every V-cycle, so it keeps its own scalars
  double* cpartial = nullptr;
  double* cscal = nullptr;
  double* hcscal = nullptr;
  double *kr = nullptr, *kz = nullptr, *kp = nullptr, *kq = nullptr, *kro = nullptr;
  double *cr = nullptr, *cz = nullptr, *cp = nullptr, *cq = nullptr, *cb = nullptr, *cx = nullptr;
  double* cinv = nullptr;       // FD coarsest dense inverse
  int last_coarse_iters = 0;
  // SEM coarsest level assembled in ELL form for the persistent coarse PCG kernel
  int* ell_col = nullptr;
  double* ell_val = nullptr;
  int nslot = 0;
  int coarse_grid = 0;
  bool coop_ok = false;
  unsigned* cctl = nullptr;     // [5] control words of the persistent kernel
  unsigned* hcctl = nullptr;    // pinned host copy
  double* cpart = nullptr;      // [3 * coarse_grid + 3]
  double* cxbuf[2] = {nullptr, nullptr};   // exchange buffers of the persistent coarse CG
  unsigned* cflag = nullptr;    // [coarse_grid] exchange flags
  int coarse_rows_per_block = 0;
  int coarse_halo = 0;
  int coarse_degree = 1;        // 4th-kind polynomial preconditioner degree (autotuned)
  double coarse_lmax = 0.0;
  unsigned* dstat = nullptr;    // [4] device-side error flags of the operator kernels
  unsigned* hdstat = nullptr;
};

namespace {

template <typename T>
T* dalloc(chebmg_ctx* c, int64_t n) {
  void* p = nullptr;
  CK(cudaMalloc(&p, sizeof(T) * (size_t)std::max<int64_t>(n, 1)));
  c->allocs.push_back(p);
  return static_cast<T*>(p);
}

template <typename T>
constexpr int dt_of() {
  return sizeof(T) == 8 ? CHEBMG_F64 : CHEBMG_F32;
}

template <typename T>
T* vec(Level& L, int w) {
  return static_cast<T*>(L.v[dt_of<T>()][w]);
}

template <typename T>
const T* invD_of(const Level& L) {
  return static_cast<const T*>(L.invD[dt_of<T>()]);
}

template <typename T>
Stencil9<T> stencil(const Level& L) {
  Stencil9<T> st;
  for (int q = 0; q < 9; ++q) st.c[q] = (T)L.st[q];
  return st;
}

void read_scal(chebmg_ctx* c) {
  CK(cudaMemcpyAsync(c->hscal, c->scal, sizeof(double) * S_NSLOTS, cudaMemcpyDeviceToHost, c->s));
  if (c->cctl) CK(cudaMemcpyAsync(c->hcctl, c->cctl, sizeof(unsigned) * 5, cudaMemcpyDeviceToHost, c->s));
  CK(cudaMemcpyAsync(c->hdstat, c->dstat, sizeof(unsigned) * 4, cudaMemcpyDeviceToHost, c->s));
  CK(cudaStreamSynchronize(c->s));
}

// Worst error recorded by persistent coarse solves since the last reset (0 if none).
int coarse_sticky_error(chebmg_ctx* c) {
  if (c->hdstat[0]) return CHEBMG_ETIMEOUT;     // an operator kernel's bounded wait ran out
  if (!c->cctl) return CHEBMG_OK;
  const unsigned w = c->hcctl[4];
  if (w == CS_TIMEOUT) return CHEBMG_ETIMEOUT;
  if (w == CS_BREAKDOWN) return CHEBMG_EBREAKDOWN;
  return CHEBMG_OK;
}

void reset_coarse_sticky(chebmg_ctx* c) {
  if (c->cctl) CK(cudaMemsetAsync(c->cctl + 4, 0, sizeof(unsigned), c->s));
}

void read_cscal(chebmg_ctx* c) {
  CK(cudaMemcpyAsync(c->hcscal, c->cscal, sizeof(double) * S_NSLOTS, cudaMemcpyDeviceToHost, c->s));
  CK(cudaStreamSynchronize(c->s));
}

// y = A x on level j; for SEM y must be zero on entry (element contributions accumulate).
template <typename T>
void apply_into(chebmg_ctx* c, int j, const T* x, T* y) {
  Level& L = c->L[j];
  const int dt = dt_of<T>();
  if (L.type == TYPE_SEM) {
    if (L.Q == 8)
      sem_ax8<T>(L.E, L.gid, L.lat, static_cast<const T*>(L.G[dt]), x, y, c->dstat, L.eb[dt], c->s);
    else
      sem_ax<T>(L.Q, L.E, L.gid, static_cast<const T*>(L.G[dt]), static_cast<const T*>(L.D[dt]), x, y, c->s);
  } else {
    fd_apply<T>(L.mx, L.my, stencil<T>(L), x, y, c->s);
  }
  check_launch();
}

template <typename T>
void zero(chebmg_ctx* c, T* p, int64_t n) {
  CK(cudaMemsetAsync(p, 0, sizeof(T) * (size_t)n, c->s));
}

// One smoother application (Algorithm 1 or 2) of the given order on level j.
template <typename T>
void smooth(chebmg_ctx* c, int j, const T* b, T* x, int order, bool x_zero) {
  Level& L = c->L[j];
  const int64_t n = L.n;
  T* r = vec<T>(L, VR);
  T* d = vec<T>(L, VD);
  T* y = vec<T>(L, VY);
  const T* S = invD_of<T>(L);
  const double lmax = L.lmax;
  zero<T>(c, y, n);
  if (!x_zero) apply_into<T>(c, j, x, y);
  if (c->o.kind == CHEBMG_CHEB_1ST) {
    const double lmin = c->o.lmin_ratio * lmax;
    const double theta = 0.5 * (lmax + lmin), delta = 0.5 * (lmax - lmin);
    const double sigma = theta / delta;
    double rho = 1.0 / sigma;
    cheb1_init<T>(n, b, x, r, d, y, S, 1.0 / theta, x_zero ? 1 : 0, c->s);
    for (int i = 1; i < order; ++i) {
      apply_into<T>(c, j, d, y);
      const double rho_new = 1.0 / (2.0 * sigma - rho);
      cheb1_step<T>(n, x, r, d, y, S, rho_new * rho, 2.0 * rho_new / delta, c->s);
      rho = rho_new;
    }
    axpy<T>(n, 1.0, d, x, c->s);
  } else {
    const double* beta = (c->o.kind == CHEBMG_CHEB_4TH_OPT) ? kBeta[order - 1] : nullptr;
    cheb4_init<T>(n, b, x, r, d, y, S, 4.0 / (3.0 * lmax), x_zero ? 1 : 0, c->s);
    for (int i = 1; i < order; ++i) {
      apply_into<T>(c, j, d, y);
      const double c1 = (2.0 * i - 1.0) / (2.0 * i + 3.0);
      const double c2 = (8.0 * i + 4.0) / ((2.0 * i + 3.0) * lmax);
      cheb4_step<T>(n, x, r, d, y, S, beta ? beta[i - 1] : 1.0, c1, c2, c->s);
    }
    axpy<T>(n, beta ? beta[order - 1] : 1.0, d, x, c->s);
  }
  check_launch();
}

// rc = P^T rf (level j -> j+1)
template <typename T>
void restrict_to(chebmg_ctx* c, int j, const T* rf, T* rc) {
  Level& F = c->L[j];
  Level& C = c->L[j + 1];
  const int dt = dt_of<T>();
  if (F.type == TYPE_SEM) {
    zero<T>(c, rc, C.n);
    if (transfer_box_supported(F.Q, C.Q))
      restrict_box<T>(F.Q, C.Q, F.E, F.lat, C.lat, rf, rc, c->s);
    else
      sem_restrict<T>(F.Q, C.Q, F.E, F.gid, C.gid, static_cast<const T*>(F.Jn[dt]), rf, rc, c->s);
  } else {
    fd_restrict<T>(F.mx, F.my, C.mx, C.my, F.c_next, rf, rc, c->s);
  }
  check_launch();
}

// zf (+)= P zc (level j+1 -> j)
template <typename T>
void prolong_to(chebmg_ctx* c, int j, const T* zc, T* zf, int accumulate) {
  Level& F = c->L[j];
  Level& C = c->L[j + 1];
  const int dt = dt_of<T>();
  if (F.type == TYPE_SEM) {
    if (transfer_box_supported(F.Q, C.Q))
      prolong_box<T>(F.Q, C.Q, F.E, F.lat, C.lat, zc, zf, accumulate, c->s);
    else
      sem_prolong<T>(F.Q, C.Q, F.E, F.gid, C.gid, static_cast<const T*>(F.Jn[dt]), zc, zf, accumulate, c->s);
  } else {
    fd_prolong<T>(F.mx, F.my, C.mx, C.my, F.c_next, zc, zf, accumulate, c->s);
  }
  check_launch();
}

CoarseCG coarse_args(chebmg_ctx* c, const double* b, double* x) {
  Level& C = c->L.back();
  CoarseCG a;
  a.n = C.n;
  a.nslot = c->nslot;
  a.col = c->ell_col;
  a.val = c->ell_val;
  a.invD = static_cast<const double*>(C.invD[CHEBMG_F64]);
  a.b = b;
  a.x = x;
  a.xbuf[0] = c->cxbuf[0];
  a.xbuf[1] = c->cxbuf[1];
  a.flag = c->cflag;
  a.rows_per_block = c->coarse_rows_per_block;
  a.halo = c->coarse_halo;
  a.part = c->cpart;
  a.tot = c->cpart + 3 * std::max(1, c->coarse_grid);
  a.ctl = c->cctl;
  a.rtol = c->o.coarse_rtol;
  a.maxit = c->o.coarse_maxit;
  a.degree = c->coarse_degree;
  a.lmax = c->coarse_lmax > 0.0 ? c->coarse_lmax : 1.0;
  a.phantom_blocks = 0;
  return a;
}

// Resets the control words and exchange flags of the persistent coarse kernel.
void coarse_reset(chebmg_ctx* c) {
  CK(cudaMemsetAsync(c->cctl, 0, sizeof(unsigned) * 4, c->s));
  CK(cudaMemsetAsync(c->cflag, 0, sizeof(unsigned) * std::max(1, c->coarse_grid), c->s));
}

// FP64 coarse solve on the last level: FD dense inverse, SEM Jacobi-PCG.
int coarse_solve64(chebmg_ctx* c, const double* b, double* x) {
  Level& C = c->L.back();
  const int64_t n = C.n;
  if (C.type == TYPE_FD) {
    dense_matvec((int)n, c->cinv, b, x, c->s);
    check_launch();
    c->last_coarse_iters = 1;
    return CHEBMG_OK;
  }
  const double* S = static_cast<const double*>(C.invD[CHEBMG_F64]);
  double *r = c->cr, *z = c->cz, *p = c->cp, *q = c->cq;
  if (c->coop_ok) {
    // whole PCG in one cooperative launch; no host round trip.  Status and iterations
    // land in cctl[2..3], errors also in the sticky cctl[4].
    coarse_reset(c);
    CoarseCG a = coarse_args(c, b, x);
    a.phantom_blocks = 0;
    cudaError_t e = cudaSuccess;
    if (coarse_pcg_launch(a, c->coarse_grid, c->s, &e)) return CHEBMG_OK;
    cudaGetLastError();
    c->coop_ok = false;   // cooperative launch refused: use the host-driven loop from now on
  }
  // x = 0, r = b, z = S r, p = z, RZ = (r, z), RR = (r, r): one CG update with alpha = 0, p = q = 0
  double* sc = c->cscal;
  double* part = c->cpartial;
  zero<double>(c, x, n);
  masked_copy(n, b, S, r, c->s);
  zero<double>(c, p, n);
  zero<double>(c, q, n);
  CK(cudaMemsetAsync(sc + S_ALPHA, 0, sizeof(double), c->s));
  cg_update(n, x, r, z, p, q, S, part, sc, c->s);
  CK(cudaMemcpyAsync(p, z, sizeof(double) * n, cudaMemcpyDeviceToDevice, c->s));
  read_cscal(c);
  const double bb = c->hcscal[S_RR];
  c->last_coarse_iters = 0;
  if (!(bb > 0.0)) return std::isfinite(bb) ? CHEBMG_OK : CHEBMG_EBREAKDOWN;
  const double tol2 = c->o.coarse_rtol * c->o.coarse_rtol * bb;
  for (int it = 1; it <= c->o.coarse_maxit; ++it) {
    zero<double>(c, q, n);
    apply_into<double>(c, (int)c->L.size() - 1, p, q);
    dot2(n, p, q, nullptr, nullptr, S_PQ, -1, POST_ALPHA, part, sc, c->s);
    cg_update(n, x, r, z, p, q, S, part, sc, c->s);   // RR, ZR; BETA = ZR/RZ; RZ = ZR
    read_cscal(c);
    c->last_coarse_iters = it;
    const double rr = c->hcscal[S_RR], pq = c->hcscal[S_PQ];
    if (!(pq > 0.0) || !std::isfinite(rr)) return CHEBMG_EBREAKDOWN;
    if (rr <= tol2) return CHEBMG_OK;
    update_p(n, z, p, sc, c->s);
  }
  return CHEBMG_ENOTCONV;
}

template <typename T>
int coarse(chebmg_ctx* c, const T* b, T* x) {
  if constexpr (sizeof(T) == 8) {
    return coarse_solve64(c, b, x);
  } else {
    Level& C = c->L.back();
    cast<float, double>(C.n, b, c->cb, c->s);
    int rc = coarse_solve64(c, c->cb, c->cx);
    cast<double, float>(C.n, c->cx, x, c->s);
    check_launch();
    return rc;
  }
}

// z = V-cycle(b) from level j (Eq. 2.2), in precision T.
template <typename T>
int vcycle_level(chebmg_ctx* c, int j, const T* b, T* x) {
  if (j == (int)c->L.size() - 1) return coarse<T>(c, b, x);
  Level& L = c->L[j];
  Level& C = c->L[j + 1];
  if (c->pre > 0) {
    smooth<T>(c, j, b, x, c->pre, true);
  } else {
    zero<T>(c, x, L.n);
  }
  T* y = vec<T>(L, VY);
  T* r = vec<T>(L, VR);
  zero<T>(c, y, L.n);
  apply_into<T>(c, j, x, y);
  residual<T>(L.n, b, y, r, c->s);
  restrict_to<T>(c, j, r, vec<T>(C, VB));
  int rc = vcycle_level<T>(c, j + 1, vec<T>(C, VB), vec<T>(C, VX));
  if (rc != CHEBMG_OK && rc != CHEBMG_ENOTCONV) return rc;
  prolong_to<T>(c, j, vec<T>(C, VX), x, 1);
  if (c->post > 0) smooth<T>(c, j, b, x, c->post, false);
  check_launch();
  return rc;
}

int vcycle_top(chebmg_ctx* c, const double* r, double* z) {
  if (c->L.size() == 1) return coarse_solve64(c, r, z);
  if (!c->fp32) return vcycle_level<double>(c, 0, r, z);
  Level& L = c->L[0];
  float* b32 = vec<float>(L, VB);
  float* x32 = vec<float>(L, VX);
  cast<double, float>(L.n, r, b32, c->s);
  int rc = vcycle_level<float>(c, 0, b32, x32);
  cast<float, double>(L.n, x32, z, c->s);
  check_launch();
  return rc;
}

// Largest eigenvalue of the symmetric tridiagonal (a, b) by Sturm-sequence bisection.
double tridiag_max_eig(const std::vector<double>& a, const std::vector<double>& b) {
  const int m = (int)a.size();
  double lo = 1e300, hi = -1e300;
  for (int i = 0; i < m; ++i) {
    const double off = (i > 0 ? std::fabs(b[i - 1]) : 0.0) + (i < m - 1 ? std::fabs(b[i]) : 0.0);
    lo = std::min(lo, a[i] - off);
    hi = std::max(hi, a[i] + off);
  }
  auto below = [&](double x) {   // number of eigenvalues < x
    int cnt = 0;
    double d = 1.0;
    for (int i = 0; i < m; ++i) {
      const double bb = i > 0 ? b[i - 1] * b[i - 1] : 0.0;
      d = (a[i] - x) - (i > 0 ? bb / d : 0.0);
      if (d == 0.0) d = -1e-300;
      if (d < 0.0) ++cnt;
    }
    return cnt;
  };
  for (int it = 0; it < 200 && hi - lo > 1e-15 * std::max(std::fabs(hi), 1e-300); ++it) {
    const double mid = 0.5 * (lo + hi);
    if (below(mid) >= m) hi = mid;
    else lo = mid;
  }
  return 0.5 * (lo + hi);
}

// lambda_max of S A on level j by Lanczos on S^{1/2} A S^{1/2} (FP64).
double lanczos(chebmg_ctx* c, int j, int steps) {
  Level& L = c->L[j];
  const int64_t n = L.n;
  const double* S = static_cast<const double*>(L.invD[CHEBMG_F64]);
  double* v = vec<double>(L, VB);
  double* vp = vec<double>(L, VX);
  double* t = vec<double>(L, VR);
  double* w = vec<double>(L, VD);
  double* y = vec<double>(L, VY);
  splitmix_fill(n, 42ull, S, v, c->s);
  dot2(n, v, v, nullptr, nullptr, S_T0, -1, POST_NONE, c->partial, c->scal, c->s);
  read_scal(c);
  scale(n, 1.0 / std::sqrt(c->hscal[S_T0]), v, v, c->s);
  zero<double>(c, vp, n);
  std::vector<double> al, be;
  double beta = 0.0;
  for (int k = 0; k < steps; ++k) {
    sqrt_scale(n, S, v, t, c->s);
    zero<double>(c, y, n);
    apply_into<double>(c, j, t, y);
    dot2(n, t, y, nullptr, nullptr, S_T0, -1, POST_NONE, c->partial, c->scal, c->s);
    read_scal(c);
    const double alpha = c->hscal[S_T0];
    lanczos_w(n, S, y, v, vp, alpha, beta, w, c->s);
    dot2(n, w, w, nullptr, nullptr, S_T1, -1, POST_NONE, c->partial, c->scal, c->s);
    read_scal(c);
    al.push_back(alpha);
    const double bn = std::sqrt(c->hscal[S_T1]);
    if (!std::isfinite(alpha) || !std::isfinite(bn)) throw Error(CHEBMG_EBREAKDOWN, "Lanczos produced NaN");
    if (bn <= 1e-14 * std::fabs(alpha)) break;
    be.push_back(bn);
    CK(cudaMemcpyAsync(vp, v, sizeof(double) * n, cudaMemcpyDeviceToDevice, c->s));
    scale(n, 1.0 / bn, w, v, c->s);
    beta = bn;
  }
  be.resize(al.size() > 0 ? al.size() - 1 : 0);
  check_launch();
  if (al.size() == 1) return al[0];
  return tridiag_max_eig(al, be);
}

void alloc_vectors(chebmg_ctx* c, Level& L, bool with32) {
  for (int w = 0; w < NV; ++w) L.v[CHEBMG_F64][w] = dalloc<double>(c, L.n);
  if (with32)
    for (int w = 0; w < NV; ++w) L.v[CHEBMG_F32][w] = dalloc<float>(c, L.n);
}

void common_alloc(chebmg_ctx* c) {
  c->dstat = dalloc<unsigned>(c, 4);
  CK(cudaMemsetAsync(c->dstat, 0, sizeof(unsigned) * 4, c->s));
  c->partial = dalloc<double>(c, 2 * kRedBlocks);
  c->scal = dalloc<double>(c, S_NSLOTS);
  CK(cudaMemsetAsync(c->scal, 0, sizeof(double) * S_NSLOTS, c->s));
  void* h = nullptr;
  CK(cudaMallocHost(&h, sizeof(double) * S_NSLOTS));
  c->hscal = static_cast<double*>(h);
  CK(cudaMallocHost(&h, sizeof(unsigned) * 4));
  c->hdstat = static_cast<unsigned*>(h);
  std::memset(c->hdstat, 0, sizeof(unsigned) * 4);
  c->cpartial = dalloc<double>(c, 2 * kRedBlocks);
  c->cscal = dalloc<double>(c, S_NSLOTS);
  CK(cudaMemsetAsync(c->cscal, 0, sizeof(double) * S_NSLOTS, c->s));
  CK(cudaMallocHost(&h, sizeof(double) * S_NSLOTS));
  c->hcscal = static_cast<double*>(h);
  const int64_t n0 = c->L[0].n;
  c->kr = dalloc<double>(c, n0);
  c->kz = dalloc<double>(c, n0);
  c->kp = dalloc<double>(c, n0);
  c->kq = dalloc<double>(c, n0);
  c->kro = dalloc<double>(c, n0);
  const int64_t nc = c->L.back().n;
  c->cr = dalloc<double>(c, nc);
  c->cz = dalloc<double>(c, nc);
  c->cp = dalloc<double>(c, nc);
  c->cq = dalloc<double>(c, nc);
  c->cb = dalloc<double>(c, nc);
  c->cx = dalloc<double>(c, nc);
  if (c->ell_col) {
    int coop = 0;
    CK(cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, c->dev));
    int grid = 0, rb = 0;
    coarse_pcg_shape(nc, &grid, &rb);
    c->coarse_grid = grid;
    c->coarse_rows_per_block = rb;
    c->coop_ok = coop != 0 && grid > 0;
    c->cctl = dalloc<unsigned>(c, 5);
    CK(cudaMemsetAsync(c->cctl, 0, sizeof(unsigned) * 5, c->s));
    CK(cudaMallocHost(&h, sizeof(unsigned) * 5));
    c->hcctl = static_cast<unsigned*>(h);
    std::memset(c->hcctl, 0, sizeof(unsigned) * 5);
    c->cpart = dalloc<double>(c, 3 * std::max(1, grid) + 3);
    c->cxbuf[0] = dalloc<double>(c, nc);
    c->cxbuf[1] = dalloc<double>(c, nc);
    c->cflag = dalloc<unsigned>(c, std::max(1, grid));
  }
}

template <typename T>
T* upload(chebmg_ctx* c, const std::vector<double>& h) {
  std::vector<T> tmp(h.begin(), h.end());
  T* d = dalloc<T>(c, (int64_t)tmp.size());
  CK(cudaMemcpy(d, tmp.data(), sizeof(T) * tmp.size(), cudaMemcpyHostToDevice));
  return d;
}

// Picks the elements-per-block of the order-7 operator by timing each candidate on the
// level's own data (3 launches each, best of them) -- a small autotuner run once at setup.
template <typename T>
void autotune_ax8(chebmg_ctx* c, int j) {
  Level& L = c->L[j];
  const int dt = dt_of<T>();
  if (L.type != TYPE_SEM || L.Q != 8 || !L.G[dt]) return;
  T* x = vec<T>(L, VB);
  T* y = vec<T>(L, VY);
  CK(cudaMemsetAsync(x, 0, sizeof(T) * L.n, c->s));
  cudaEvent_t e0, e1;
  CK(cudaEventCreate(&e0));
  CK(cudaEventCreate(&e1));
  float best = 1e30f;
  int best_eb = 2;
  for (int eb : {1, 2, 4, 12, 14, 101, 102, 104, 112, 114}) {
    if (!sem_ax8_variant_fits<T>(eb)) continue;
    L.eb[dt] = eb;
    apply_into<T>(c, j, x, y);   // warm-up / first-launch configuration
    float t_min = 1e30f;
    for (int rep = 0; rep < 3; ++rep) {
      CK(cudaEventRecord(e0, c->s));
      apply_into<T>(c, j, x, y);
      CK(cudaEventRecord(e1, c->s));
      CK(cudaEventSynchronize(e1));
      float ms = 0.f;
      CK(cudaEventElapsedTime(&ms, e0, e1));
      t_min = std::min(t_min, ms);
    }
    if (t_min < best) {
      best = t_min;
      best_eb = eb;
    }
  }
  L.eb[dt] = best_eb;
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  CK(cudaMemsetAsync(y, 0, sizeof(T) * L.n, c->s));
}

// Picks the degree of the coarse CG's polynomial preconditioner by timing full coarse solves
// of a seeded right-hand side (degree 1 = Jacobi-PCG).
void autotune_coarse_degree(chebmg_ctx* c) {
  Level& C = c->L.back();
  const int64_t n = C.n;
  double* b = vec<double>(C, VB);
  double* x = vec<double>(C, VX);
  splitmix_fill(n, 7ull, static_cast<const double*>(C.invD[CHEBMG_F64]), b, c->s);
  cudaEvent_t e0, e1;
  CK(cudaEventCreate(&e0));
  CK(cudaEventCreate(&e1));
  float best = 1e30f;
  int best_m = 1;
  for (int m : {1, 2, 4, 8, 12, 16}) {
    c->coarse_degree = m;
    float t_min = 1e30f;
    bool ok = true;
    for (int rep = 0; rep < 2 && ok; ++rep) {
      CK(cudaEventRecord(e0, c->s));
      if (coarse_solve64(c, b, x) != CHEBMG_OK) ok = false;
      CK(cudaEventRecord(e1, c->s));
      CK(cudaEventSynchronize(e1));
      read_scal(c);
      if (c->hcctl[2] != CS_OK) ok = false;
      float ms = 0.f;
      CK(cudaEventElapsedTime(&ms, e0, e1));
      t_min = std::min(t_min, ms);
    }
    if (ok && t_min < best) {
      best = t_min;
      best_m = m;
    }
  }
  c->coarse_degree = best_m;
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  CK(cudaMemsetAsync(c->cctl + 4, 0, sizeof(unsigned), c->s));
}

void finish_setup(chebmg_ctx* c) {
  const int nl = (int)c->L.size();
  for (int j = 0; j < nl; ++j) {
    autotune_ax8<double>(c, j);
    if (c->fp32) autotune_ax8<float>(c, j);
  }
  c->pre = c->o.sided == CHEBMG_ONE_SIDED ? 2 * c->o.order : c->o.order;
  c->post = c->o.sided == CHEBMG_ONE_SIDED ? 0 : c->o.order;
  for (int j = 0; j + 1 < nl; ++j) {
    double lm;
    if (c->o.lmax_override) lm = c->o.lmax_override[j];
    else lm = c->o.lmax_scale * lanczos(c, j, c->o.lanczos_steps);
    if (!(lm > 0.0) || !std::isfinite(lm)) throw Error(CHEBMG_EBREAKDOWN, "non-positive lambda_max");
    c->L[j].lmax = lm;
  }
  if (c->coop_ok) {
    // lambda_max of S A on the coarse level (same Lanczos), then the preconditioner degree
    c->coarse_lmax = lanczos(c, nl - 1, c->o.lanczos_steps);
    autotune_coarse_degree(c);
  }
  CK(cudaStreamSynchronize(c->s));
}

void validate_opts(const chebmg_opts* o) {
  if (!o) throw Error(CHEBMG_EINVAL, "opts is NULL");
  if (o->kind != CHEBMG_CHEB_1ST && o->kind != CHEBMG_CHEB_4TH && o->kind != CHEBMG_CHEB_4TH_OPT)
    throw Error(CHEBMG_EINVAL, "unknown smoother kind");
  if (o->order < 1) throw Error(CHEBMG_EINVAL, "order must be >= 1");
  const int maxorder = o->sided == CHEBMG_ONE_SIDED ? 2 * o->order : o->order;
  if (o->kind == CHEBMG_CHEB_4TH_OPT && maxorder > 16)
    throw Error(CHEBMG_EINVAL, "optimized 4th-kind coefficients are tabulated up to order 16");
  if (o->sided != CHEBMG_SYMMETRIC && o->sided != CHEBMG_ONE_SIDED) throw Error(CHEBMG_EINVAL, "bad sided");
  if (o->prec != CHEBMG_FP64 && o->prec != CHEBMG_FP32_SMOOTHER) throw Error(CHEBMG_EINVAL, "bad prec");
  if (o->kind == CHEBMG_CHEB_1ST && !(o->lmin_ratio > 0.0 && o->lmin_ratio < 1.0))
    throw Error(CHEBMG_EINVAL, "lmin_ratio must be in (0, 1)");
  if (!(o->lmax_scale > 0.0)) throw Error(CHEBMG_EINVAL, "lmax_scale must be > 0");
  if (o->lanczos_steps < 1 && !o->lmax_override) throw Error(CHEBMG_EINVAL, "lanczos_steps must be >= 1");
  if (!(o->coarse_rtol > 0.0) || o->coarse_maxit < 1) throw Error(CHEBMG_EINVAL, "bad coarse tolerance");
}

template <typename F>
int guard(F&& f) {
  try {
    return f();
  } catch (const Error& e) {
    g_last_error = e.what();
    return e.code;
  } catch (const std::bad_alloc&) {
    g_last_error = "host allocation failed";
    return CHEBMG_ENOMEM;
  } catch (const std::exception& e) {
    g_last_error = e.what();
    return CHEBMG_ECUDA;
  } catch (...) {
    g_last_error = "unknown error";
    return CHEBMG_ECUDA;
  }
}

void destroy_ctx(chebmg_ctx* c) {
  if (!c) return;
  cudaSetDevice(c->dev);
  if (c->s) cudaStreamSynchronize(c->s);
  for (void* p : c->allocs) cudaFree(p);
  if (c->hscal) cudaFreeHost(c->hscal);
  if (c->hcscal) cudaFreeHost(c->hcscal);
  if (c->hcctl) cudaFreeHost(c->hcctl);
  if (c->hdstat) cudaFreeHost(c->hdstat);
  delete c;
}

chebmg_ctx* new_ctx(const chebmg_opts* o) {
  validate_opts(o);
  chebmg_ctx* c = new chebmg_ctx();
  c->o = *o;
  c->s = static_cast<cudaStream_t>(o->stream);
  c->fp32 = o->prec == CHEBMG_FP32_SMOOTHER;
  cudaError_t e = cudaGetDevice(&c->dev);
  if (e != cudaSuccess) {
    delete c;
    throw Error(CHEBMG_ECUDA, std::string("cudaGetDevice: ") + cudaGetErrorString(e));
  }
  return c;
}

Level& level_checked(chebmg_ctx* c, int level) {
  if (!c) throw Error(CHEBMG_EINVAL, "ctx is NULL");
  if (level < 0 || level >= (int)c->L.size()) throw Error(CHEBMG_EINVAL, "level out of range");
  return c->L[level];
}

void check_dtype(chebmg_ctx* c, int dtype) {
  if (dtype == CHEBMG_F64) return;
  if (dtype == CHEBMG_F32 && c->fp32) return;
  throw Error(CHEBMG_EINVAL, "dtype not available in this context");
}

void enter(chebmg_ctx* c) {
  if (!c) throw Error(CHEBMG_EINVAL, "ctx is NULL");
  CK(cudaSetDevice(c->dev));
}

}  // namespace

// ===========================================================================
// C ABI
// ===========================================================================
extern "C" {

void chebmg_default_opts(chebmg_opts* o) {
  if (!o) return;
  std::memset(o, 0, sizeof(*o));
  o->kind = CHEBMG_CHEB_4TH_OPT;
  o->order = 2;
  o->sided = CHEBMG_ONE_SIDED;
  o->prec = CHEBMG_FP64;
  o->lmin_ratio = 0.1;
  o->lmax_scale = 1.0;
  o->lanczos_steps = 30;
  o->lmax_override = nullptr;
  o->coarse_rtol = 1e-10;
  o->coarse_maxit = 5000;
  o->stream = nullptr;
}

int chebmg_setup_fd2d(int m, double Lx, double Ly, int coarsening, int coarsest, const chebmg_opts* opts,
                      chebmg_ctx** out) {
  return guard([&]() -> int {
    if (!out) throw Error(CHEBMG_EINVAL, "ctx output is NULL");
    *out = nullptr;
    if (m < 1 || coarsening < 2 || coarsest < 1 || !(Lx > 0.0) || !(Ly > 0.0))
      throw Error(CHEBMG_EINVAL, "bad FD sizes");
    std::vector<int> sizes{m};
    while (sizes.back() > coarsest) {
      const int mf = sizes.back();
      if ((mf + 1) % coarsening != 0) throw Error(CHEBMG_EINVAL, "m+1 not divisible by the coarsening factor");
      const int mc = (mf + 1) / coarsening - 1;
      if (mc < 1) throw Error(CHEBMG_EINVAL, "coarsening below one unknown");
      sizes.push_back(mc);
    }
    chebmg_ctx* c = new_ctx(opts);
    try {
      c->type = TYPE_FD;
      double st[9];
      fd_fine_stencil(Lx / (m + 1), Ly / (m + 1), st);
      for (size_t j = 0; j < sizes.size(); ++j) {
        Level L;
        L.type = TYPE_FD;
        L.mx = L.my = sizes[j];
        L.n = (int64_t)sizes[j] * sizes[j];
        L.c_next = coarsening;
        std::memcpy(L.st, st, sizeof(st));
        std::vector<double> invd((size_t)L.n, 1.0 / st[4]);
        L.invD[CHEBMG_F64] = upload<double>(c, invd);
        if (c->fp32) L.invD[CHEBMG_F32] = upload<float>(c, invd);
        c->L.push_back(L);
        alloc_vectors(c, c->L.back(), c->fp32);
        double cst[9];
        fd_galerkin_stencil(st, coarsening, cst);
        std::memcpy(st, cst, sizeof(st));
      }
      Level& C = c->L.back();
      std::vector<double> inv;
      if (!fd_dense_inverse(C.st, C.mx, C.my, inv)) throw Error(CHEBMG_EBREAKDOWN, "coarse Cholesky failed");
      c->cinv = upload<double>(c, inv);
      common_alloc(c);
      finish_setup(c);
    } catch (...) {
      destroy_ctx(c);
      throw;
    }
    *out = c;
    return CHEBMG_OK;
  });
}

int chebmg_setup_sem(int nex, int ney, int nez, const double* verts, const int* orders, int nlevels,
                     const chebmg_opts* opts, chebmg_ctx** out) {
  return guard([&]() -> int {
    if (!out) throw Error(CHEBMG_EINVAL, "ctx output is NULL");
    *out = nullptr;
    if (nex < 1 || ney < 1 || nez < 1 || !verts || !orders || nlevels < 1)
      throw Error(CHEBMG_EINVAL, "bad SEM arguments");
    for (int j = 0; j < nlevels; ++j) {
      if (orders[j] < 1 || orders[j] > 9) throw Error(CHEBMG_EINVAL, "orders must be in 1..9");
      if (j > 0 && orders[j] >= orders[j - 1]) throw Error(CHEBMG_EINVAL, "orders must decrease");
    }
    const int64_t nmax = ((int64_t)nex * orders[0] + 1) * ((int64_t)ney * orders[0] + 1) * ((int64_t)nez * orders[0] + 1);
    if (nmax >= (int64_t)kGidMask) throw Error(CHEBMG_EINVAL, "mesh too large for 30-bit global ids");
    chebmg_ctx* c = new_ctx(opts);
    try {
      c->type = TYPE_SEM;
      std::vector<SemHostLevel> H(nlevels);
      for (int j = 0; j < nlevels; ++j) {
        if (!build_sem_level(nex, ney, nez, verts, orders[j], H[j]))
          throw Error(CHEBMG_EMESH, "mesh has a non-positive Jacobian");
      }
      for (int j = 0; j < nlevels; ++j) {
        SemHostLevel& h = H[j];
        Level L;
        L.type = TYPE_SEM;
        L.N = h.N;
        L.Q = h.NQ;
        L.lat = {nex, ney, nez, (int)(nex * h.N + 1), (int)(ney * h.N + 1), (int)(nez * h.N + 1)};
        L.NP = h.NP;
        L.E = h.E;
        L.n = h.n;
        L.gid = dalloc<uint32_t>(c, (int64_t)h.gid.size());
        CK(cudaMemcpy(L.gid, h.gid.data(), sizeof(uint32_t) * h.gid.size(), cudaMemcpyHostToDevice));
        std::vector<double> invd((size_t)h.n, 0.0);
        for (int64_t g = 0; g < h.n; ++g)
          if (!h.dirichlet[g]) invd[g] = 1.0 / h.diag[g];
        const bool smoothed32 = c->fp32 && j + 1 < nlevels;
        L.G[CHEBMG_F64] = upload<double>(c, h.G);
        L.invD[CHEBMG_F64] = upload<double>(c, invd);
        L.D[CHEBMG_F64] = upload<double>(c, h.Dm);
        if (h.N == 7) CK(sem_ax8_set_D(h.Dm.data()));
        if (smoothed32) {
          L.G[CHEBMG_F32] = upload<float>(c, h.G);
          L.invD[CHEBMG_F32] = upload<float>(c, invd);
          L.D[CHEBMG_F32] = upload<float>(c, h.Dm);
        }
        if (j + 1 < nlevels) {
          std::vector<double> J;
          lagrange_interp(H[j + 1].x, h.x, J);
          if (transfer_box_supported(h.NQ, H[j + 1].NQ)) CK(transfer_box_set_J(h.NQ, H[j + 1].NQ, J.data()));
          L.Jn[CHEBMG_F64] = upload<double>(c, J);
          if (c->fp32) L.Jn[CHEBMG_F32] = upload<float>(c, J);
        }
        if (j + 1 == nlevels) {
          std::vector<int> col;
          std::vector<double> val;
          assemble_ell(h, c->nslot, col, val);
          int grid = 0, rb = 0;
          coarse_pcg_shape(h.n, &grid, &rb);
          int halo = 0;
          if (rb > 0)
            for (int64_t g = 0; g < h.n; ++g)
              for (int k = 0; k < c->nslot; ++k) {
                const int64_t cc = col[(size_t)k * h.n + g];
                halo = std::max<int>(halo, (int)std::llabs(cc / rb - g / rb));
              }
          c->coarse_halo = halo;
          c->ell_col = dalloc<int>(c, (int64_t)col.size());
          CK(cudaMemcpy(c->ell_col, col.data(), sizeof(int) * col.size(), cudaMemcpyHostToDevice));
          c->ell_val = upload<double>(c, val);
        }
        c->L.push_back(L);
        alloc_vectors(c, c->L.back(), c->fp32);
        std::vector<double>().swap(h.G);
      }
      common_alloc(c);
      finish_setup(c);
    } catch (...) {
      destroy_ctx(c);
      throw;
    }
    *out = c;
    return CHEBMG_OK;
  });
}

void chebmg_destroy(chebmg_ctx* c) { destroy_ctx(c); }

int chebmg_num_levels(const chebmg_ctx* c, int* nl) {
  if (!c || !nl) return CHEBMG_EINVAL;
  *nl = (int)c->L.size();
  return CHEBMG_OK;
}

int chebmg_level_size(const chebmg_ctx* c, int level, int64_t* n) {
  if (!c || !n || level < 0 || level >= (int)c->L.size()) return CHEBMG_EINVAL;
  *n = c->L[level].n;
  return CHEBMG_OK;
}

int chebmg_lambda_max(const chebmg_ctx* c, int level, double* out) {
  if (!c || !out || level < 0 || level + 1 >= (int)c->L.size()) return CHEBMG_EINVAL;
  *out = c->L[level].lmax;
  return CHEBMG_OK;
}

int chebmg_tile_choice(const chebmg_ctx* c, int level, int dtype, int* elements_per_block) {
  if (!c || !elements_per_block || level < 0 || level >= (int)c->L.size() || (dtype != 0 && dtype != 1))
    return CHEBMG_EINVAL;
  const Level& L = c->L[level];
  *elements_per_block = (L.type == TYPE_SEM && L.Q == 8) ? L.eb[dtype] : 0;
  return CHEBMG_OK;
}

int chebmg_coarse_info(const chebmg_ctx* c, int* degree, double* lmax) {
  if (!c || !degree || !lmax) return CHEBMG_EINVAL;
  *degree = (c->coop_ok && c->L.back().type == TYPE_SEM) ? c->coarse_degree : 1;
  *lmax = c->coarse_lmax;
  return CHEBMG_OK;
}

int chebmg_set_coarse_degree(chebmg_ctx* c, int degree) {
  if (!c || degree < 1 || degree > 64) return CHEBMG_EINVAL;
  c->coarse_degree = degree;
  return CHEBMG_OK;
}

int chebmg_set_tile_choice(chebmg_ctx* c, int level, int dtype, int variant) {
  if (!c || level < 0 || level >= (int)c->L.size() || (dtype != 0 && dtype != 1)) return CHEBMG_EINVAL;
  Level& L = c->L[level];
  if (L.type != TYPE_SEM || L.Q != 8) return CHEBMG_EINVAL;
  const int base = variant % 100;
  if ((variant != base && variant != base + 100) ||
      (base != 1 && base != 2 && base != 4 && base != 12 && base != 14))
    return CHEBMG_EINVAL;
  const bool fits = dtype == CHEBMG_F64 ? sem_ax8_variant_fits<double>(variant) : sem_ax8_variant_fits<float>(variant);
  if (!fits) return CHEBMG_EINVAL;
  L.eb[dtype] = variant;
  return CHEBMG_OK;
}

int chebmg_launch_count(const chebmg_ctx* c, int64_t* count) {
  (void)c;
  if (!count) return CHEBMG_EINVAL;
  *count = g_launches.load();
  return CHEBMG_OK;
}

int chebmg_apply_A(chebmg_ctx* c, int level, int dtype, const void* x, void* y) {
  return guard([&]() -> int {
    enter(c);
    Level& L = level_checked(c, level);
    check_dtype(c, dtype);
    if (!x || !y) throw Error(CHEBMG_EINVAL, "NULL vector");
    if (dtype == CHEBMG_F64) {
      zero<double>(c, static_cast<double*>(y), L.n);
      apply_into<double>(c, level, static_cast<const double*>(x), static_cast<double*>(y));
    } else {
      if (!L.G[CHEBMG_F32] && L.type == TYPE_SEM) throw Error(CHEBMG_EINVAL, "no FP32 data on this level");
      zero<float>(c, static_cast<float*>(y), L.n);
      apply_into<float>(c, level, static_cast<const float*>(x), static_cast<float*>(y));
    }
    return CHEBMG_OK;
  });
}

int chebmg_inv_diagonal(chebmg_ctx* c, int level, int dtype, void* out) {
  return guard([&]() -> int {
    enter(c);
    Level& L = level_checked(c, level);
    check_dtype(c, dtype);
    if (!out || !L.invD[dtype]) throw Error(CHEBMG_EINVAL, "no data");
    const size_t bytes = (dtype == CHEBMG_F64 ? 8 : 4) * (size_t)L.n;
    CK(cudaMemcpyAsync(out, L.invD[dtype], bytes, cudaMemcpyDeviceToDevice, c->s));
    return CHEBMG_OK;
  });
}

int chebmg_smooth(chebmg_ctx* c, int level, int dtype, const void* b, void* x, int order, int x_is_zero) {
  return guard([&]() -> int {
    enter(c);
    Level& L = level_checked(c, level);
    check_dtype(c, dtype);
    if (level + 1 >= (int)c->L.size()) throw Error(CHEBMG_EINVAL, "the coarsest level is not smoothed");
    if (!b || !x || order < 1) throw Error(CHEBMG_EINVAL, "bad smoother arguments");
    if (c->o.kind == CHEBMG_CHEB_4TH_OPT && order > 16) throw Error(CHEBMG_EINVAL, "order > 16");
    if (dtype == CHEBMG_F64)
      smooth<double>(c, level, static_cast<const double*>(b), static_cast<double*>(x), order, x_is_zero != 0);
    else {
      if (!L.G[CHEBMG_F32] && L.type == TYPE_SEM) throw Error(CHEBMG_EINVAL, "no FP32 data on this level");
      smooth<float>(c, level, static_cast<const float*>(b), static_cast<float*>(x), order, x_is_zero != 0);
    }
    return CHEBMG_OK;
  });
}

int chebmg_restrict(chebmg_ctx* c, int level, int dtype, const void* rf, void* rc) {
  return guard([&]() -> int {
    enter(c);
    level_checked(c, level);
    check_dtype(c, dtype);
    if (level + 1 >= (int)c->L.size()) throw Error(CHEBMG_EINVAL, "no coarser level");
    if (!rf || !rc) throw Error(CHEBMG_EINVAL, "NULL vector");
    if (dtype == CHEBMG_F64) restrict_to<double>(c, level, static_cast<const double*>(rf), static_cast<double*>(rc));
    else restrict_to<float>(c, level, static_cast<const float*>(rf), static_cast<float*>(rc));
    return CHEBMG_OK;
  });
}

int chebmg_prolong(chebmg_ctx* c, int level, int dtype, const void* zc, void* zf, int accumulate) {
  return guard([&]() -> int {
    enter(c);
    level_checked(c, level);
    check_dtype(c, dtype);
    if (level + 1 >= (int)c->L.size()) throw Error(CHEBMG_EINVAL, "no coarser level");
    if (!zc || !zf) throw Error(CHEBMG_EINVAL, "NULL vector");
    if (dtype == CHEBMG_F64)
      prolong_to<double>(c, level, static_cast<const double*>(zc), static_cast<double*>(zf), accumulate ? 1 : 0);
    else
      prolong_to<float>(c, level, static_cast<const float*>(zc), static_cast<float*>(zf), accumulate ? 1 : 0);
    return CHEBMG_OK;
  });
}

int chebmg_coarse_solve(chebmg_ctx* c, const double* r, double* z, int* iters) {
  return guard([&]() -> int {
    enter(c);
    if (!r || !z) throw Error(CHEBMG_EINVAL, "NULL vector");
    reset_coarse_sticky(c);
    int rc = coarse_solve64(c, r, z);
    CK(cudaStreamSynchronize(c->s));
    if (c->coop_ok && c->L.back().type == TYPE_SEM) {
      read_scal(c);
      c->last_coarse_iters = (int)c->hcctl[3];
      const unsigned st = c->hcctl[2];
      rc = st == CS_OK ? CHEBMG_OK : st == CS_NOTCONV ? CHEBMG_ENOTCONV
           : coarse_sticky_error(c) != CHEBMG_OK ? coarse_sticky_error(c) : CHEBMG_EBREAKDOWN;
    }
    if (iters) *iters = c->last_coarse_iters;
    return rc;
  });
}

int chebmg_vcycle(chebmg_ctx* c, const double* r, double* z) {
  return guard([&]() -> int {
    enter(c);
    if (!r || !z) throw Error(CHEBMG_EINVAL, "NULL vector");
    reset_coarse_sticky(c);
    int rc = vcycle_top(c, r, z);
    check_launch();
    read_scal(c);
    if (rc == CHEBMG_OK || rc == CHEBMG_ENOTCONV) rc = coarse_sticky_error(c);
    return rc;
  });
}

int chebmg_pcg_solve(chebmg_ctx* c, const double* b, double* u, double rtol, int maxit, int* iters,
                     double* relres, double* history) {
  return guard([&]() -> int {
    enter(c);
    if (!b || !u || maxit < 0 || !(rtol > 0.0)) throw Error(CHEBMG_EINVAL, "bad solve arguments");
    Level& L = c->L[0];
    const int64_t n = L.n;
    const double* S = static_cast<const double*>(L.invD[CHEBMG_F64]);
    double *r = c->kr, *z = c->kz, *p = c->kp, *q = c->kq, *ro = c->kro;
    if (iters) *iters = 0;
    reset_coarse_sticky(c);
    masked_copy(n, b, S, r, c->s);
    zero<double>(c, u, n);
    dot2(n, r, r, nullptr, nullptr, S_BB, -1, POST_NONE, c->partial, c->scal, c->s);
    read_scal(c);
    const double bb = c->hscal[S_BB];
    if (history) history[0] = 1.0;
    if (!std::isfinite(bb)) return CHEBMG_EBREAKDOWN;
    if (bb == 0.0) {
      if (relres) *relres = 0.0;
      return CHEBMG_OK;
    }
    int rc = vcycle_top(c, r, z);
    if (rc != CHEBMG_OK && rc != CHEBMG_ENOTCONV) return rc;
    CK(cudaMemcpyAsync(p, z, sizeof(double) * n, cudaMemcpyDeviceToDevice, c->s));
    dot2(n, z, r, nullptr, nullptr, S_ZR, -1, POST_SET_RZ_FROM_ZR, c->partial, c->scal, c->s);
    double rel = 1.0;
    for (int it = 1; it <= maxit; ++it) {
      zero<double>(c, q, n);
      apply_into<double>(c, 0, p, q);
      dot2(n, p, q, nullptr, nullptr, S_PQ, -1, POST_ALPHA, c->partial, c->scal, c->s);
      fcg_update_xr(n, u, r, ro, p, q, c->partial, c->scal, c->s);
      read_scal(c);
      const double pq = c->hscal[S_PQ], rr = c->hscal[S_RR];
      const int crc = coarse_sticky_error(c);
      if (crc != CHEBMG_OK) {
        if (iters) *iters = it;
        g_last_error = "coarse solve inside the V-cycle failed";
        return crc;
      }
      if (!(pq > 0.0) || !std::isfinite(rr)) {
        if (iters) *iters = it;
        if (relres) *relres = std::sqrt(rr / bb);
        g_last_error = "FCG breakdown: p^T A p <= 0 or non-finite residual";
        return CHEBMG_EBREAKDOWN;
      }
      rel = std::sqrt(rr / bb);
      if (history) history[it] = rel;
      if (iters) *iters = it;
      if (relres) *relres = rel;
      if (rel <= rtol) return CHEBMG_OK;
      rc = vcycle_top(c, r, z);
      if (rc != CHEBMG_OK && rc != CHEBMG_ENOTCONV) return rc;
      dot2(n, z, r, z, ro, S_ZR, S_ZRO, POST_BETA_FLEX, c->partial, c->scal, c->s);
      update_p(n, z, p, c->scal, c->s);
      check_launch();
    }
    g_last_error = "FCG did not reach the tolerance";
    return CHEBMG_ENOTCONV;
  });
}

int chebmg_pcg_solve_host(chebmg_ctx* c, const double* b_host, double* u_host, double rtol, int maxit,
                          int* iters, double* relres) {
  return guard([&]() -> int {
    enter(c);
    if (!b_host || !u_host) throw Error(CHEBMG_EINVAL, "NULL vector");
    const int64_t n = c->L[0].n;
    // stage through the level-0 FP64 work vectors that a solve does not use
    double* b = vec<double>(c->L[0], VB);
    double* u = vec<double>(c->L[0], VX);
    CK(cudaMemcpyAsync(b, b_host, sizeof(double) * n, cudaMemcpyHostToDevice, c->s));
    int rc = chebmg_pcg_solve(c, b, u, rtol, maxit, iters, relres, nullptr);
    CK(cudaMemcpyAsync(u_host, u, sizeof(double) * n, cudaMemcpyDeviceToHost, c->s));
    CK(cudaStreamSynchronize(c->s));
    return rc;
  });
}

int chebmg_selftest_coarse_timeout(chebmg_ctx* c, int* status) {
  return guard([&]() -> int {
    enter(c);
    if (!status) throw Error(CHEBMG_EINVAL, "status is NULL");
    if (!c->cctl || !c->coop_ok) throw Error(CHEBMG_EINVAL, "no persistent coarse solver in this context");
    Level& C = c->L.back();
    const int64_t n = C.n;
    coarse_reset(c);
    CK(cudaMemsetAsync(c->cctl + 4, 0, sizeof(unsigned), c->s));
    CoarseCG a = coarse_args(c, c->cb, c->cx);
    a.phantom_blocks = 1;    // one arrival that never comes: every barrier wait runs out
    cudaError_t e = cudaSuccess;
    if (!coarse_pcg_launch(a, c->coarse_grid, c->s, &e)) throw Error(CHEBMG_ECUDA, cudaGetErrorString(e));
    read_scal(c);
    *status = coarse_sticky_error(c);
    CK(cudaMemsetAsync(c->cctl, 0, sizeof(unsigned) * 5, c->s));
    CK(cudaStreamSynchronize(c->s));
    return CHEBMG_OK;
  });
}

const char* chebmg_strerror(int code) {
  switch (code) {
    case CHEBMG_OK: return "ok";
    case CHEBMG_EINVAL: return "invalid argument";
    case CHEBMG_ECUDA: return "CUDA error";
    case CHEBMG_ENOTCONV: return "not converged";
    case CHEBMG_EBREAKDOWN: return "breakdown";
    case CHEBMG_ETIMEOUT: return "device wait timed out";
    case CHEBMG_ENOMEM: return "out of device memory";
    case CHEBMG_EMESH: return "invalid mesh";
    default: return "unknown status";
  }
}

const char* chebmg_last_error(void) { return g_last_error.c_str(); }

}  // extern "C"
