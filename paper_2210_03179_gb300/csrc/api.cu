// C-ABI entry points and host orchestration of the multigrid hot path.
//
// Host code here only sequences kernels (kernels.cu) on the context's stream:
// every arithmetic step of the smoother, the transfers, the coarse solves and
// the outer Krylov loop runs on the GPU.  The host reads back one or two FP64
// scalars per Krylov iteration to test convergence.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <limits>
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
  int ax4[2] = {41, 41};   // order-3 operator: 40 one thread per point, 41 line passes (+100 lattice ids)
  int beb[2] = {2002, 2002};   // variant of the batched order-7 operator (autotuned per batch size)
  Lattice lat = {0, 0, 0, 0, 0, 0};
  bool boxed = true;    // SEM: the level carries the box lattice (lattice-indexed kernels usable)
  // fused smoother (one persistent launch per smoother application) per dtype: 0 = the separate
  // operator and update kernels, else the sem_smooth8 variant; control words of its launches
  int fused[2] = {0, 0};
  int fused_b[2] = {0, 0};     // the same for batches of the size tuned last
  int fused_gsz[2] = {8, 8};   // right-hand sides per work item in batches
  unsigned* fctl = nullptr;
  int64_t ld = 0;       // leading dimension of batched vectors: n rounded up to 64
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
  double *kr = nullptr, *kz = nullptr, *kp = nullptr, *kq = nullptr;
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
  double* cpart = nullptr;      // [2][3 * coarse_grid] block partials, by generation parity
  unsigned long long* cexf[2] = {nullptr, nullptr};   // tagged exchange of the persistent coarse CG: FP32
  unsigned long long* cexd[2] = {nullptr, nullptr};   // and FP64
  uint64_t coarse_gen = 0;      // exchange tags used so far (advanced per launch)
  float* ell_valf = nullptr;    // FP32 copies for the FP32 preconditioner
  float* coarse_invDf = nullptr;
  bool coarse_pf32 = false;     // coarse CG preconditioner in FP32
  int coarse_rows_per_block = 0;
  // the outer Krylov product of the finest level: 0 FP64, 1 FP64-class arithmetic on FP32 pairs
  int outer_op = 0;
  void* G_x2 = nullptr;         // level-0 geometric factors as FP32 pairs
  int eb_x2 = 2;                // variant of the pair-arithmetic kernel (autotuned)
  // coarse CG on one thread-block cluster (box lattice at N = 1, FP32 preconditioner)
  int coarse_kernel = 0;        // 0 grid-wide persistent kernel, 1 cluster kernel
  float* cc_val32 = nullptr;    // [14][n] symmetric stencil layout
  double* cc_val64 = nullptr;
  // the same operator with 27 slots in lattice order (grid-wide kernel, box lattices)
  double* lat_val = nullptr;
  float* lat_valf = nullptr;
  int cc_nx = 0, cc_ny = 0, cc_nz = 0, cc_ctas = 0, cc_rmax = 0;
  size_t cc_smem = 0;
  bool cc_ok = false;
  int coarse_degree = 1;        // 4th-kind polynomial preconditioner degree (autotuned)
  double coarse_lmax = 0.0;
  unsigned* dstat = nullptr;    // [4] device-side error flags: [0] operator wait, [1] batched coarse
  unsigned* hdstat = nullptr;
  // ---- batches of right-hand sides ----
  int nb = 1;                   // right-hand sides of the operation in progress
  bool batched = false;         // inside a batched or grouped solve (device-side decisions only)
  int64_t gen = 0;              // bumped whenever captured graphs of this context go stale
  int bcap = 1;                 // capacity of the work vectors (right-hand sides)
  int btuned = 0;               // batch size the batched variants were tuned for
  double* kx = nullptr;         // batched FCG solution
  double* bpart = nullptr;      // batched reduction partials
  double* bscal = nullptr;      // [bcap][S_NSLOTS]
  int* bstat = nullptr;         // [bcap][4]
  double* hbscal = nullptr;
  int* hbstat = nullptr;
  unsigned* bcstat = nullptr;   // [bcap][2] batched coarse status
  int bcoarse_degree = 1;
  cudaStream_t gs = nullptr;    // private stream for graph capture
  cudaGraphExec_t gexec[2] = {nullptr, nullptr};
  int gexec_nb = 0;
  int64_t glaunches[2] = {0, 0};   // kernels per replay of each graph
  // ---- smoother parameter overrides (weight tuning) ----
  std::vector<double> lmin_opt;  // optimal lambda_min / lambda_max per smoothing order (1st kind)
  std::vector<double> beta_ovr;  // weights of Algorithm 2 for smoothing order beta_ovr.size()
  double lscale = 1.0;           // every level smooths with lscale * lambda_max
  // ---- adjoint workspace ----
  struct GradWork {
    int nb = 0, kmax = 0, steps = 0;
    std::vector<std::vector<double*>> lv;   // per level: the vectors of enum GW
    std::vector<double*> D, SR;             // recorded d_i and S r_i of one smoother call
    std::vector<double*> Et;                // e_0 .. e_steps
    double *W = nullptr, *Z = nullptr, *EB = nullptr, *ZB = nullptr, *WB = nullptr;
    double *part = nullptr, *acc = nullptr, *rows = nullptr, *coef = nullptr;
  } gw;
  // ---- GMRES workspace ----
  struct GmresWork {
    int m = 0;
    double *V = nullptr, *Z = nullptr, *w = nullptr, *bm = nullptr, *part = nullptr, *h = nullptr;
    double* hh = nullptr;   // pinned host copy of a Hessenberg column
  } gm;
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

// Leading dimension and total length of a level's work vectors for the current batch.
int64_t ldv(const chebmg_ctx* c, const Level& L) { return c->nb > 1 ? L.ld : L.n; }
int64_t span(const chebmg_ctx* c, const Level& L) { return c->nb > 1 ? (int64_t)c->nb * L.ld : L.n; }

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
void apply_into_ld(chebmg_ctx* c, int j, const T* x, T* y, int nb, int64_t ld) {
  Level& L = c->L[j];
  const int dt = dt_of<T>();
  if (L.type == TYPE_SEM) {
    if (L.Q == 8 && nb > 1)
      sem_ax8_batched<T>(L.E, L.gid, L.lat, static_cast<const T*>(L.G[dt]), x, y, c->dstat, L.beb[dt], nb, ld,
                         c->s);
    else if (L.Q == 8)
      sem_ax8<T>(L.E, L.gid, L.lat, static_cast<const T*>(L.G[dt]), x, y, c->dstat, L.eb[dt], c->s);
    else if (L.Q == 4 && L.ax4[dt] % 100 == 41)
      sem_ax4<T>(L.E, L.gid, L.ax4[dt] >= 100 ? &L.lat : nullptr, static_cast<const T*>(L.G[dt]),
                 static_cast<const T*>(L.D[dt]), x, y, c->s, nb, ld);
    else
      sem_ax<T>(L.Q, L.E, L.gid, static_cast<const T*>(L.G[dt]), static_cast<const T*>(L.D[dt]), x, y, c->s, nb,
                ld);
  } else {
    fd_apply<T>(L.mx, L.my, stencil<T>(L), x, y, c->s, nb, ld);
  }
  check_launch();
}

// y = A x on level j for the current batch (y zero on entry for SEM).
template <typename T>
void apply_into(chebmg_ctx* c, int j, const T* x, T* y) {
  apply_into_ld<T>(c, j, x, y, c->nb, ldv(c, c->L[j]));
}

template <typename T>
void zero(chebmg_ctx* c, T* p, int64_t n) {
  // inside a chain of programmatic dependent launches a zeroing kernel keeps the chain going
  if (pdl_on(c->s)) zero_bytes(p, (int64_t)sizeof(T) * n, c->s);
  else CK(cudaMemsetAsync(p, 0, sizeof(T) * (size_t)n, c->s));
}

// lambda_min / lambda_max of the 1st-kind smoother of the given order: the option's fixed ratio,
// or (option <= 0) the ratio that maximises gamma^{-1} for that order (computed once).
double lmin_ratio_for(chebmg_ctx* c, int order) {
  if (c->o.lmin_ratio > 0.0) return c->o.lmin_ratio;
  if ((int)c->lmin_opt.size() <= order) c->lmin_opt.resize(order + 1, 0.0);
  if (c->lmin_opt[order] == 0.0) c->lmin_opt[order] = cheb1_optimal_lmin_ratio(order);
  return c->lmin_opt[order];
}

// Whether level j can run the fused smoother at all (order-7 box lattice).
bool fused_eligible(const chebmg_ctx* c, int j) {
  const Level& L = c->L[j];
  return L.type == TYPE_SEM && L.Q == 8 && L.boxed && L.fctl != nullptr;
}

// The smoother of smooth() -- and, with_residual, the restriction residual r = b - A x after it
// -- as one launch of the fused kernel (sem_smooth8.cu): the same steps and coefficients as the
// separate kernels, written as phases (operator application, then a pointwise update).  Returns
// false, having done nothing, where the fused kernel does not apply.
template <typename T>
bool smooth_fused(chebmg_ctx* c, int j, const T* b, T* x, int order, bool x_zero, bool with_residual) {
  Level& L = c->L[j];
  const int dt = dt_of<T>();
  const int variant = c->nb > 1 ? L.fused_b[dt] : L.fused[dt];
  if (!fused_eligible(c, j) || variant == 0 || order < 1) return false;
  // the pointwise phases use 16-byte accesses on b and x as well (caller vectors may be views)
  if (reinterpret_cast<uintptr_t>(b) % 16 != 0 || reinterpret_cast<uintptr_t>(x) % 16 != 0) return false;
  FusedSmooth a{};
  a.E = L.E;
  a.n = L.n;
  a.lat = L.lat;
  a.G = L.G[dt];
  a.S = invD_of<T>(L);
  a.b = b;
  a.x = x;
  a.r = vec<T>(L, VR);
  a.d = vec<T>(L, VD);
  a.y = vec<T>(L, VY);
  a.ctl = L.fctl;
  a.err = c->dstat;
  a.nb = c->nb;
  a.ld = ldv(c, L);
  a.gsz = c->nb > 1 ? std::max(1, L.fused_gsz[dt]) : 1;
  const double lmax = L.lmax * c->lscale;
  int np = 0;
  bool fits = true;
  auto add = [&](int op, int src, double c0 = 0.0, double c1 = 0.0, double c2 = 0.0, double c3 = 0.0) {
    if (np >= kFusedMaxPhases) {
      fits = false;
      return;
    }
    a.ph[np++] = FusedPhase{op, src, {c0, c1, c2, c3}};
  };
  if (!x_zero) add(FOP_ZERO_Y, FSRC_NONE);   // the first operator application accumulates into y
  if (c->o.kind == CHEBMG_CHEB_1ST) {
    const double lmin = lmin_ratio_for(c, order) * lmax;
    const double theta = 0.5 * (lmax + lmin), delta = 0.5 * (lmax - lmin);
    const double sigma = theta / delta;
    double rho = 1.0 / sigma;
    if (x_zero) add(FOP_CHEB1_INIT_B, FSRC_NONE, 1.0 / theta);
    else add(FOP_CHEB1_INIT_BY, FSRC_X, 1.0 / theta);
    for (int i = 1; i < order; ++i) {
      const double rho_new = 1.0 / (2.0 * sigma - rho);
      // the last step also applies the final update x += d
      add(FOP_CHEB1_STEP, FSRC_D, 0.0, rho_new * rho, 2.0 * rho_new / delta, i + 1 == order ? 1.0 : 0.0);
      rho = rho_new;
    }
    if (order == 1) add(FOP_AXPY, FSRC_NONE, 1.0);
  } else {
    const double* beta = (c->o.kind == CHEBMG_CHEB_4TH_OPT) ? kBeta[order - 1] : nullptr;
    if (!c->beta_ovr.empty() && (int)c->beta_ovr.size() == order) beta = c->beta_ovr.data();
    if (x_zero) add(FOP_CHEB4_INIT_B, FSRC_NONE, 4.0 / (3.0 * lmax));
    else add(FOP_CHEB4_INIT_BY, FSRC_X, 4.0 / (3.0 * lmax));
    const double beta_k = beta ? beta[order - 1] : 1.0;
    for (int i = 1; i < order; ++i) {
      const double c1 = (2.0 * i - 1.0) / (2.0 * i + 3.0);
      const double c2 = (8.0 * i + 4.0) / ((2.0 * i + 3.0) * lmax);
      add(FOP_CHEB4_STEP, FSRC_D, beta ? beta[i - 1] : 1.0, c1, c2, i + 1 == order ? beta_k : 0.0);
    }
    if (order == 1 || beta_k == 0.0) add(FOP_AXPY, FSRC_NONE, beta_k);
  }
  if (with_residual) add(FOP_RESIDUAL, FSRC_X);
  if (!fits) return false;
  a.nphase = np;
  if (!fused_plan(a, variant)) return false;
  if (!sem_smooth8<T>(a, variant, c->s)) {
    cudaGetLastError();   // a refused cooperative launch leaves no other trace: separate kernels
    return false;
  }
  check_launch();
  return true;
}

// One smoother application (Algorithm 1 or 2) of the given order on level j.
template <typename T>
void smooth(chebmg_ctx* c, int j, const T* b, T* x, int order, bool x_zero) {
  if (smooth_fused<T>(c, j, b, x, order, x_zero, false)) return;
  Level& L = c->L[j];
  const int64_t n = L.n;
  const int nb = c->nb;
  // one right-hand side: the step kernels launch as programmatic dependents of each other
  const PdlScope pdl_(g_pdl || nb == 1);
  const int64_t ld = ldv(c, L);
  T* r = vec<T>(L, VR);
  T* d = vec<T>(L, VD);
  T* y = vec<T>(L, VY);
  const T* S = invD_of<T>(L);
  const double lmax = L.lmax * c->lscale;
  zero<T>(c, y, span(c, L));
  if (!x_zero) apply_into<T>(c, j, x, y);
  if (c->o.kind == CHEBMG_CHEB_1ST) {
    const double lmin = lmin_ratio_for(c, order) * lmax;
    const double theta = 0.5 * (lmax + lmin), delta = 0.5 * (lmax - lmin);
    const double sigma = theta / delta;
    double rho = 1.0 / sigma;
    cheb1_init<T>(n, b, x, r, d, y, S, 1.0 / theta, x_zero ? 1 : 0, c->s, nb, ld);
    for (int i = 1; i < order; ++i) {
      apply_into<T>(c, j, d, y);
      const double rho_new = 1.0 / (2.0 * sigma - rho);
      cheb1_step<T>(n, x, r, d, y, S, rho_new * rho, 2.0 * rho_new / delta, c->s, nb, ld);
      rho = rho_new;
    }
    axpy<T>(n, 1.0, d, x, c->s, nb, ld);
  } else {
    const double* beta = (c->o.kind == CHEBMG_CHEB_4TH_OPT) ? kBeta[order - 1] : nullptr;
    if (!c->beta_ovr.empty() && (int)c->beta_ovr.size() == order) beta = c->beta_ovr.data();
    // from x = 0 with more than one step, the init writes only d and the first step reads b
    // for r and writes x (two vector writes and a read fewer than x = 0, r = b in the init)
    const bool lean = x_zero && order > 1;
    cheb4_init<T>(n, b, x, r, d, y, S, 4.0 / (3.0 * lmax), lean ? 2 : x_zero ? 1 : 0, c->s, nb, ld);
    const double beta_k = beta ? beta[order - 1] : 1.0;
    for (int i = 1; i < order; ++i) {
      apply_into<T>(c, j, d, y);
      const double c1 = (2.0 * i - 1.0) / (2.0 * i + 3.0);
      const double c2 = (8.0 * i + 4.0) / ((2.0 * i + 3.0) * lmax);
      // the last step also applies the final update x += beta_k d_k (one pass fewer)
      cheb4_step<T>(n, x, r, d, y, S, beta ? beta[i - 1] : 1.0, c1, c2, c->s, nb, ld,
                    i + 1 == order ? beta_k : 0.0, lean && i == 1 ? b : nullptr);
    }
    if (order == 1 || beta_k == 0.0) axpy<T>(n, beta_k, d, x, c->s, nb, ld);
  }
  check_launch();
}

// rc = P^T rf (level j -> j+1)
template <typename T>
void restrict_to(chebmg_ctx* c, int j, const T* rf, T* rc) {
  Level& F = c->L[j];
  Level& C = c->L[j + 1];
  const int dt = dt_of<T>();
  const int nb = c->nb;
  const int64_t ldf = ldv(c, F), ldc = ldv(c, C);
  if (F.type == TYPE_SEM) {
    zero<T>(c, rc, span(c, C));
    if (F.boxed && transfer_box_supported(F.Q, C.Q))
      restrict_box<T>(F.Q, C.Q, F.E, F.lat, C.lat, rf, rc, c->s, nb, ldf, ldc);
    else
      sem_restrict<T>(F.Q, C.Q, F.E, F.gid, C.gid, static_cast<const T*>(F.Jn[dt]), rf, rc, c->s, nb, ldf, ldc);
  } else {
    fd_restrict<T>(F.mx, F.my, C.mx, C.my, F.c_next, rf, rc, c->s, nb, ldf, ldc);
  }
  check_launch();
}

// zf (+)= P zc (level j+1 -> j)
template <typename T>
void prolong_to(chebmg_ctx* c, int j, const T* zc, T* zf, int accumulate) {
  Level& F = c->L[j];
  Level& C = c->L[j + 1];
  const int dt = dt_of<T>();
  const int nb = c->nb;
  const int64_t ldf = ldv(c, F), ldc = ldv(c, C);
  if (F.type == TYPE_SEM) {
    if (F.boxed && transfer_box_supported(F.Q, C.Q))
      prolong_box<T>(F.Q, C.Q, F.E, F.lat, C.lat, zc, zf, accumulate, c->s, nb, ldf, ldc);
    else
      sem_prolong<T>(F.Q, C.Q, F.E, F.gid, C.gid, static_cast<const T*>(F.Jn[dt]), zc, zf, accumulate, c->s, nb,
                     ldf, ldc);
  } else {
    fd_prolong<T>(F.mx, F.my, C.mx, C.my, F.c_next, zc, zf, accumulate, c->s, nb, ldf, ldc);
  }
  check_launch();
}

// Shape of the persistent coarse kernel: at least rpt_min rows per thread.
void set_coarse_shape(chebmg_ctx* c, int rpt_min) {
  int grid = 0, rb = 0;
  coarse_pcg_shape(c->L.back().n, rpt_min, &grid, &rb);
  c->coarse_grid = grid;
  c->coarse_rows_per_block = rb;
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
  a.rows_per_block = c->coarse_rows_per_block;
  a.part = c->cpart;
  a.ctl = c->cctl;
  a.rtol = c->o.coarse_rtol;
  a.maxit = c->o.coarse_maxit;
  a.degree = c->coarse_degree;
  a.lmax = c->coarse_lmax > 0.0 ? c->coarse_lmax : 1.0;
  a.phantom_blocks = 0;
  a.pf32 = c->coarse_pf32 ? 1 : 0;
  a.valf = c->ell_valf;
  a.invDf = c->coarse_invDf;
  a.lat_nx = 0;
  a.lat_nxy = 0;
  if (c->lat_val) {   // box lattice: values in lattice slot order, columns computed
    a.nslot = 27;
    a.val = c->lat_val;
    a.valf = c->lat_valf;
    a.lat_nx = c->cc_nx;
    a.lat_nxy = c->cc_nx * c->cc_ny;
  }
  a.exf[0] = c->cexf[0];
  a.exf[1] = c->cexf[1];
  a.exd[0] = c->cexd[0];
  a.exd[1] = c->cexd[1];
  // exchanges one launch can make: (degree - 1) per preconditioner application, one more per
  // CG iteration, maxit + 1 applications
  const uint64_t tags = (uint64_t)(std::max(1, a.degree) + 1) * (uint64_t)(std::max(0, a.maxit) + 2) + 4;
  if (tags >= 0x7fffffffull) throw Error(CHEBMG_EINVAL, "coarse degree x iterations too large");
  if (c->coarse_gen + tags >= 0xffffffffull) {   // tags would wrap: clear the buffers, restart
    for (int q = 0; q < 2; ++q) {
      CK(cudaMemsetAsync(c->cexf[q], 0, sizeof(unsigned long long) * a.n, c->s));
      CK(cudaMemsetAsync(c->cexd[q], 0, sizeof(unsigned long long) * 2 * a.n, c->s));
    }
    c->coarse_gen = 0;
  }
  a.gen0 = (unsigned)c->coarse_gen;
  c->coarse_gen += tags;
  return a;
}

// Resets the control words of the persistent coarse kernels (the exchange needs no reset:
// each launch takes fresh tags).
void coarse_reset(chebmg_ctx* c) { zero<unsigned>(c, c->cctl, 4); }

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
  if (c->coarse_kernel == 1 && c->cc_ok && c->coarse_pf32) {
    // whole PCG on one thread-block cluster (status words as below)
    coarse_reset(c);
    CoarseCluster a;
    a.nx = c->cc_nx;
    a.ny = c->cc_ny;
    a.nz = c->cc_nz;
    a.ctas = c->cc_ctas;
    a.rmax = c->cc_rmax;
    a.val32 = c->cc_val32;
    a.val64 = c->cc_val64;
    a.invDf = c->coarse_invDf;
    a.b = b;
    a.x = x;
    a.rtol = c->o.coarse_rtol;
    a.maxit = c->o.coarse_maxit;
    a.degree = c->coarse_degree;
    a.lmax = c->coarse_lmax > 0.0 ? c->coarse_lmax : 1.0;
    a.ctl = c->cctl;
    cudaError_t e = cudaSuccess;
    if (coarse_cluster_launch(a, c->cc_smem, c->s, &e)) return CHEBMG_OK;
    cudaGetLastError();
    c->cc_ok = false;   // cluster launch refused: grid-wide kernel from now on
    c->coarse_kernel = 0;
  }
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

// Whether the coarse solve of a batch runs without host decisions (so it can be captured).
bool coarse_batch_capturable(const chebmg_ctx* c) {
  const Level& C = c->L.back();
  return C.type == TYPE_FD || (c->ell_col && coarse_block_supported(C.n));
}

// FP64 coarse solve of the current batch (c->nb right-hand sides at the coarse leading dimension).
int coarse_solve64_batched(chebmg_ctx* c, const double* b, double* x) {
  Level& C = c->L.back();
  const int64_t ld = ldv(c, C);
  if (C.type == TYPE_FD) {
    dense_matvec((int)C.n, c->cinv, b, x, c->s, c->nb, ld);
    check_launch();
    return CHEBMG_OK;
  }
  if (coarse_block_supported(C.n)) {
    CoarseBlock a;
    a.n = C.n;
    a.nslot = c->nslot;
    a.col = c->ell_col;
    a.val = c->ell_val;
    a.invD = static_cast<const double*>(C.invD[CHEBMG_F64]);
    a.b = b;
    a.x = x;
    a.ld = ld;
    a.rtol = c->o.coarse_rtol;
    a.maxit = c->o.coarse_maxit;
    a.degree = c->bcoarse_degree;
    a.lmax = c->coarse_lmax > 0.0 ? c->coarse_lmax : 1.0;
    a.stat = c->bcstat;
    a.sticky = c->dstat + 1;
    a.pf32 = c->coarse_pf32 ? 1 : 0;
    a.valf = c->ell_valf;
    a.invDf = c->coarse_invDf;
    if (!coarse_block_launch(a, c->nb, c->s)) throw Error(CHEBMG_ECUDA, "batched coarse launch failed");
    check_launch();
    return CHEBMG_OK;
  }
  // larger coarse problems: one persistent solve per right-hand side
  const int nb = c->nb;
  c->nb = 1;
  int rc = CHEBMG_OK;
  for (int q = 0; q < nb && (rc == CHEBMG_OK || rc == CHEBMG_ENOTCONV); ++q)
    rc = coarse_solve64(c, b + q * ld, x + q * ld);
  c->nb = nb;
  return rc;
}

template <typename T>
int coarse(chebmg_ctx* c, const T* b, T* x) {
  if constexpr (sizeof(T) == 8) {
    return c->batched ? coarse_solve64_batched(c, b, x) : coarse_solve64(c, b, x);
  } else {
    Level& C = c->L.back();
    const int64_t ld = ldv(c, C);
    cast<float, double>(C.n, b, c->cb, c->s, c->nb, ld, ld);
    int rc = c->batched ? coarse_solve64_batched(c, c->cb, c->cx) : coarse_solve64(c, c->cb, c->cx);
    cast<double, float>(C.n, c->cx, x, c->s, c->nb, ld, ld);
    check_launch();
    return rc;
  }
}

// q = A p on the finest level for the outer Krylov method (q zero on entry): FP64, or the
// order-7 operator in FP64-class FP32-pair arithmetic when the context selected it.
void apply_outer(chebmg_ctx* c, const double* p, double* q) {
  Level& L = c->L[0];
  if (c->outer_op == 1 && c->G_x2) {
    sem_ax8_x2(L.E, L.gid, L.lat, c->G_x2, p, q, c->dstat, c->eb_x2, c->s);
    check_launch();
    return;
  }
  apply_into<double>(c, 0, p, q);
}

// z = V-cycle(b) from level j (Eq. 2.2), in precision T.
template <typename T>
int vcycle_level(chebmg_ctx* c, int j, const T* b, T* x) {
  if (j == (int)c->L.size() - 1) return coarse<T>(c, b, x);
  Level& L = c->L[j];
  Level& C = c->L[j + 1];
  // the fused kernel computes the restriction residual in the same launch as the pre-smoother
  bool have_r = false;
  if (c->pre > 0) {
    have_r = smooth_fused<T>(c, j, b, x, c->pre, true, true);
    if (!have_r) smooth<T>(c, j, b, x, c->pre, true);
  } else {
    zero<T>(c, x, span(c, L));
  }
  T* y = vec<T>(L, VY);
  T* r = vec<T>(L, VR);
  if (!have_r) {
    if (c->pre == 0) zero<T>(c, y, span(c, L));   // the smoothers leave y = 0
    apply_into<T>(c, j, x, y);
    residual<T>(L.n, b, y, r, c->s, c->nb, ldv(c, L));
  }
  restrict_to<T>(c, j, r, vec<T>(C, VB));
  int rc = vcycle_level<T>(c, j + 1, vec<T>(C, VB), vec<T>(C, VX));
  if (rc != CHEBMG_OK && rc != CHEBMG_ENOTCONV) return rc;
  prolong_to<T>(c, j, vec<T>(C, VX), x, 1);
  if (c->post > 0) smooth<T>(c, j, b, x, c->post, false);
  check_launch();
  return rc;
}

int vcycle_top(chebmg_ctx* c, const double* r, double* z) {
  if (c->L.size() == 1) return coarse<double>(c, r, z);
  if (!c->fp32) return vcycle_level<double>(c, 0, r, z);
  Level& L = c->L[0];
  float* b32 = vec<float>(L, VB);
  float* x32 = vec<float>(L, VX);
  const int64_t ld = ldv(c, L);
  cast<double, float>(L.n, r, b32, c->s, c->nb, ld, ld);
  int rc = vcycle_level<float>(c, 0, b32, x32);
  cast<float, double>(L.n, x32, z, c->s, c->nb, ld, ld);
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
  if (!(c->hscal[S_T0] > 0.0)) return 1.0;   // no free node on this level: nothing to smooth or solve
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
  for (int w = 0; w < NV; ++w) L.v[CHEBMG_F64][w] = dalloc<double>(c, L.ld);
  if (with32)
    for (int w = 0; w < NV; ++w) L.v[CHEBMG_F32][w] = dalloc<float>(c, L.ld);
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
    coarse_pcg_shape(nc, 1, &grid, &rb);   // the widest shape: buffers are sized for it
    set_coarse_shape(c, 1);
    c->coop_ok = coop != 0 && grid > 0;
    if (c->cc_val64)
      c->cc_ok = coarse_cluster_plan(c->cc_nx, c->cc_ny, c->cc_nz, &c->cc_ctas, &c->cc_rmax, &c->cc_smem);
    c->cctl = dalloc<unsigned>(c, 5);
    CK(cudaMemsetAsync(c->cctl, 0, sizeof(unsigned) * 5, c->s));
    CK(cudaMallocHost(&h, sizeof(unsigned) * 5));
    c->hcctl = static_cast<unsigned*>(h);
    std::memset(c->hcctl, 0, sizeof(unsigned) * 5);
    c->cpart = dalloc<double>(c, 6 * std::max(1, grid));   // two generations of 3 partials per block
    for (int q = 0; q < 2; ++q) {   // tag 0 (zeroed words) is never used
      c->cexf[q] = dalloc<unsigned long long>(c, nc);
      c->cexd[q] = dalloc<unsigned long long>(c, 2 * nc);
      CK(cudaMemsetAsync(c->cexf[q], 0, sizeof(unsigned long long) * nc, c->s));
      CK(cudaMemsetAsync(c->cexd[q], 0, sizeof(unsigned long long) * 2 * nc, c->s));
    }
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
// level's own data (6 launches each, best of them: variants within a few per cent of each other
// are told apart more reliably than by 3) -- a small autotuner run once at setup.
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
  for (int eb : {1, 2, 4, 12, 14, 21, 22, 31, 32, 101, 102, 104, 112, 114, 121, 122, 131, 132}) {
    if (!sem_ax8_variant_fits<T>(eb)) continue;
    if (eb >= 100 && !L.boxed) continue;   // lattice ids need the box lattice
    L.eb[dt] = eb;
    apply_into<T>(c, j, x, y);   // warm-up / first-launch configuration
    float t_min = 1e30f;
    for (int rep = 0; rep < 6; ++rep) {
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

// Picks the order-3 operator (one thread per point, or line passes with map or lattice ids)
// by timing each on the level's own data, like autotune_ax8.
template <typename T>
void autotune_ax4(chebmg_ctx* c, int j) {
  Level& L = c->L[j];
  const int dt = dt_of<T>();
  if (L.type != TYPE_SEM || L.Q != 4 || !L.G[dt]) return;
  T* x = vec<T>(L, VB);
  T* y = vec<T>(L, VY);
  CK(cudaMemsetAsync(x, 0, sizeof(T) * L.n, c->s));
  cudaEvent_t e0, e1;
  CK(cudaEventCreate(&e0));
  CK(cudaEventCreate(&e1));
  float best = 1e30f;
  int best_v = L.boxed ? 141 : 41;
  for (int v : {40, 41, 141}) {
    if (v >= 100 && !L.boxed) continue;
    L.ax4[dt] = v;
    apply_into<T>(c, j, x, y);   // warm-up
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
      best_v = v;
    }
  }
  L.ax4[dt] = best_v;
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  CK(cudaMemsetAsync(y, 0, sizeof(T) * L.n, c->s));
}

// Picks the coarse CG's kernel, the degree of its polynomial preconditioner and (grid-wide
// kernel) the rows per thread by timing full coarse solves of a seeded right-hand side
// (degree 1 = Jacobi-PCG).  More rows per thread means fewer blocks: cheaper exchanges and
// reductions, but more FP64 work per block in each product.  The cluster kernel (box lattices,
// FP32 preconditioner) exchanges through distributed shared memory at a fraction of the
// grid-wide latency but has 16 SMs for the FP64 products.
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
  int best_m = 1, best_rpt = 1, last_rb = -1, best_kernel = 0;
  const bool try_cluster = c->cc_ok && c->coarse_pf32;
  for (int rpt = 1; rpt <= 2 * kCoarseMaxRowsPerThread; rpt *= 2) {
    const bool cluster = rpt > kCoarseMaxRowsPerThread;   // last round: the cluster kernel
    if (cluster && !try_cluster) break;
    c->coarse_kernel = cluster ? 1 : 0;
    if (!cluster) {
      set_coarse_shape(c, rpt);
      if (c->coarse_grid <= 0 || c->coarse_rows_per_block == last_rb) continue;
      last_rb = c->coarse_rows_per_block;
    }
  for (int m : {1, 2, 4, 8, 12, 16, 24, 32}) {
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
      best_rpt = rpt;
      best_kernel = c->coarse_kernel;
    }
  }
  }
  c->coarse_degree = best_m;
  c->coarse_kernel = best_kernel;
  set_coarse_shape(c, best_kernel == 1 ? 1 : best_rpt);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  CK(cudaMemsetAsync(c->cctl + 4, 0, sizeof(unsigned), c->s));
}

// Time of x0 = 0 smoother applications of order 4 on level j in precision T: five back to back
// per sample (so the host's launch overhead overlaps the device work, as in a solve), best of 3.
template <typename T>
float time_smooth(chebmg_ctx* c, int j, cudaEvent_t e0, cudaEvent_t e1) {
  Level& L = c->L[j];
  T* b = vec<T>(L, VB);
  T* x = vec<T>(L, VX);
  smooth<T>(c, j, b, x, 4, true);   // warm-up, first-launch configuration
  float t_min = 1e30f;
  for (int rep = 0; rep < 3; ++rep) {
    CK(cudaEventRecord(e0, c->s));
    for (int k = 0; k < 5; ++k) smooth<T>(c, j, b, x, 4, true);
    CK(cudaEventRecord(e1, c->s));
    CK(cudaEventSynchronize(e1));
    float ms = 0.f;
    CK(cudaEventElapsedTime(&ms, e0, e1));
    t_min = std::min(t_min, ms);
  }
  return t_min;
}

// On an order-7 box-lattice level: allocates the fused smoother's control words and picks, per
// precision the context uses, the fused kernel (variant) or the separate kernels (0) by timing
// a smoother application of each on the level's own data.
void autotune_fused(chebmg_ctx* c, int j) {
  Level& L = c->L[j];
  if (!(L.type == TYPE_SEM && L.Q == 8 && L.boxed)) return;
  if (!L.fctl) L.fctl = dalloc<unsigned>(c, fused_ctl_words(L.lat));
  cudaEvent_t e0, e1;
  CK(cudaEventCreate(&e0));
  CK(cudaEventCreate(&e1));
  for (int dt : {CHEBMG_F64, CHEBMG_F32}) {
    if (dt == CHEBMG_F32 && (!c->fp32 || !L.G[CHEBMG_F32])) continue;
    const size_t w = dt == CHEBMG_F64 ? sizeof(double) : sizeof(float);
    CK(cudaMemsetAsync(L.v[dt][VB], 0, w * (size_t)L.n, c->s));
    float best = 1e30f;
    int best_v = 0;
    const std::vector<int> cand = dt == CHEBMG_F32 ? std::vector<int>{0, 1} : std::vector<int>{0, 2};
    for (int v : cand) {
      L.fused[dt] = v;
      const float t = dt == CHEBMG_F64 ? time_smooth<double>(c, j, e0, e1) : time_smooth<float>(c, j, e0, e1);
      if (t < best) {
        best = t;
        best_v = v;
      }
    }
    L.fused[dt] = best_v;
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
}

void finish_setup(chebmg_ctx* c) {
  const int nl = (int)c->L.size();
  for (int j = 0; j < nl; ++j) {
    autotune_ax8<double>(c, j);
    if (c->fp32) autotune_ax8<float>(c, j);
    autotune_ax4<double>(c, j);
    if (c->fp32) autotune_ax4<float>(c, j);
  }
  c->pre = c->o.sided == CHEBMG_ONE_SIDED ? 2 * c->o.order : c->o.order;
  c->post = c->o.sided == CHEBMG_ONE_SIDED ? 0 : c->o.order;
  if (c->o.kind == CHEBMG_CHEB_1ST) {
    lmin_ratio_for(c, c->pre);
    if (c->post > 0) lmin_ratio_for(c, c->post);
  }
  for (int j = 0; j + 1 < nl; ++j) {
    double lm;
    if (c->o.lmax_override) lm = c->o.lmax_override[j];
    else lm = c->o.lmax_scale * lanczos(c, j, c->o.lanczos_steps);
    if (!(lm > 0.0) || !std::isfinite(lm)) throw Error(CHEBMG_EBREAKDOWN, "non-positive lambda_max");
    c->L[j].lmax = lm;
  }
  for (int j = 0; j + 1 < nl; ++j) autotune_fused(c, j);
  if (c->ell_col) {
    // lambda_max of S A on the coarse level (same Lanczos), then the preconditioner degree.
    // The mixed form evaluates the coarse CG's preconditioner in FP32 as well (the CG stays
    // FP64); the FP64 form keeps it in FP64.
    c->coarse_lmax = lanczos(c, nl - 1, c->o.lanczos_steps >= 1 ? c->o.lanczos_steps : 30);
    c->coarse_pf32 = c->fp32;
    if (c->coop_ok) autotune_coarse_degree(c);
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
  if (o->kind == CHEBMG_CHEB_1ST && !(o->lmin_ratio < 1.0) )
    throw Error(CHEBMG_EINVAL, "lmin_ratio must be below 1 (<= 0: optimal per order)");
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
  if (c->hbscal) cudaFreeHost(c->hbscal);
  if (c->hbstat) cudaFreeHost(c->hbstat);
  for (auto& g : c->gexec)
    if (g) cudaGraphExecDestroy(g);
  if (c->gs) cudaStreamDestroy(c->gs);
  if (c->gm.hh) cudaFreeHost(c->gm.hh);
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

// ===========================================================================
// Batches of right-hand sides
// ===========================================================================
void replace_alloc(chebmg_ctx* c, void*& p, size_t bytes) {
  if (p) {
    auto it = std::find(c->allocs.begin(), c->allocs.end(), p);
    if (it != c->allocs.end()) c->allocs.erase(it);
    CK(cudaFree(p));
    p = nullptr;
  }
  CK(cudaMalloc(&p, std::max<size_t>(bytes, 8)));
  c->allocs.push_back(p);
}
template <typename T>
void replace_vec(chebmg_ctx* c, T*& p, int64_t count) {
  void* v = p;
  replace_alloc(c, v, sizeof(T) * (size_t)count);
  p = static_cast<T*>(v);
}

void drop_graphs(chebmg_ctx* c) {
  for (auto& g : c->gexec)
    if (g) {
      cudaGraphExecDestroy(g);
      g = nullptr;
    }
  c->gexec_nb = 0;
  ++c->gen;
}

// Grows every work vector to `nrhs` right-hand sides at the levels' leading dimensions and
// allocates the per-right-hand-side scalars and status words.
void reserve_batch(chebmg_ctx* c, int nrhs) {
  if (nrhs <= c->bcap && c->bscal) return;
  const int cap = std::max(nrhs, c->bcap);
  CK(cudaStreamSynchronize(c->s));
  drop_graphs(c);
  if (cap > c->bcap) {
    for (Level& L : c->L)
      for (int dt = 0; dt < 2; ++dt)
        for (int w = 0; w < NV; ++w)
          if (L.v[dt][w]) replace_alloc(c, L.v[dt][w], (dt == CHEBMG_F64 ? 8 : 4) * (size_t)cap * L.ld);
    const int64_t ld0 = c->L[0].ld, ldc = c->L.back().ld;
    for (double** p : {&c->kr, &c->kz, &c->kp, &c->kq}) replace_vec(c, *p, (int64_t)cap * ld0);
    for (double** p : {&c->cb, &c->cx}) replace_vec(c, *p, (int64_t)cap * ldc);
  }
  const int64_t ld0 = c->L[0].ld;
  replace_vec(c, c->kx, (int64_t)cap * ld0);
  replace_vec(c, c->bpart, 2 * (int64_t)cap * std::max(bred_blocks(c->L[0].n), bred_blocks(c->L.back().n)));
  replace_vec(c, c->bscal, (int64_t)cap * S_NSLOTS);
  replace_vec(c, c->bstat, (int64_t)cap * 4);
  replace_vec(c, c->bcstat, (int64_t)cap * 2);
  CK(cudaMemsetAsync(c->bscal, 0, sizeof(double) * cap * S_NSLOTS, c->s));
  CK(cudaMemsetAsync(c->bstat, 0, sizeof(int) * cap * 4, c->s));
  CK(cudaMemsetAsync(c->bcstat, 0, sizeof(unsigned) * cap * 2, c->s));
  if (c->hbscal) cudaFreeHost(c->hbscal);
  if (c->hbstat) cudaFreeHost(c->hbstat);
  c->hbscal = nullptr;
  c->hbstat = nullptr;
  void* h = nullptr;
  CK(cudaMallocHost(&h, sizeof(double) * cap * S_NSLOTS));
  c->hbscal = static_cast<double*>(h);
  CK(cudaMallocHost(&h, sizeof(int) * cap * 4));
  c->hbstat = static_cast<int*>(h);
  c->bcap = cap;
  CK(cudaStreamSynchronize(c->s));
}

// Times the batched order-7 variants (elements per block x right-hand sides per block x id
// source) and the batched coarse preconditioner degree on the context's own data for a batch
// of nrhs right-hand sides -- run once per batch size.
void autotune_batch(chebmg_ctx* c, int nrhs) {
  if (c->btuned == nrhs) return;
  drop_graphs(c);
  cudaEvent_t e0, e1;
  CK(cudaEventCreate(&e0));
  CK(cudaEventCreate(&e1));
  auto time_it = [&](auto&& fn, int reps) {
    fn();
    float best = 1e30f;
    for (int r = 0; r < reps; ++r) {
      CK(cudaEventRecord(e0, c->s));
      fn();
      CK(cudaEventRecord(e1, c->s));
      CK(cudaEventSynchronize(e1));
      float ms = 0.f;
      CK(cudaEventElapsedTime(&ms, e0, e1));
      best = std::min(best, ms);
    }
    return best;
  };
  const int saved_nb = c->nb;
  const bool saved_batched = c->batched;
  c->nb = nrhs;
  c->batched = true;
  if (nrhs > 1) {
    for (int j = 0; j < (int)c->L.size(); ++j) {
      Level& L = c->L[j];
      if (L.type != TYPE_SEM || L.Q != 8) continue;
      for (int dt = 0; dt < 2; ++dt) {
        if (!L.G[dt]) continue;
        void* x = L.v[dt][VB];
        void* y = L.v[dt][VY];
        const size_t es = dt == CHEBMG_F64 ? 8 : 4;
        CK(cudaMemsetAsync(x, 0, es * (size_t)nrhs * L.ld, c->s));
        float best = 1e30f;
        int best_v = L.beb[dt];
        for (int rb : {1, 2, 4, 8, 16}) {
          if (rb > nrhs) break;
          for (int eb : {1, 2, 4, 101, 102, 104, 11, 12, 111, 112, 21, 22, 121, 122}) {
            if (eb >= 100 && !L.boxed) continue;
            if (eb % 100 >= 10 && rb < 2) continue;   // pairs of right-hand sides
            const int v = 1000 * rb + eb;
            if (dt == CHEBMG_F64 ? !sem_ax8_batched_fits<double>(v) : !sem_ax8_batched_fits<float>(v)) continue;
            L.beb[dt] = v;
            const float t = time_it(
                [&]() {
                  if (dt == CHEBMG_F64) apply_into<double>(c, j, static_cast<double*>(x), static_cast<double*>(y));
                  else apply_into<float>(c, j, static_cast<float*>(x), static_cast<float*>(y));
                },
                2);
            if (t < best) {
              best = t;
              best_v = v;
            }
          }
        }
        L.beb[dt] = best_v;
        CK(cudaMemsetAsync(y, 0, es * (size_t)nrhs * L.ld, c->s));
      }
    }
  }
  // fused smoother for this batch size: off, or on with 4, 8 or 16 right-hand sides per work
  // item (order-7 box-lattice levels that smooth), timed on one order-4 application
  if (nrhs > 1) {
    for (int j = 0; j + 1 < (int)c->L.size(); ++j) {
      Level& L = c->L[j];
      if (!(L.type == TYPE_SEM && L.Q == 8 && L.boxed && L.fctl)) continue;
      for (int dt : {CHEBMG_F64, CHEBMG_F32}) {
        if (dt == CHEBMG_F32 && (!c->fp32 || !L.G[CHEBMG_F32])) continue;
        const size_t es = dt == CHEBMG_F64 ? 8 : 4;
        CK(cudaMemsetAsync(L.v[dt][VB], 0, es * (size_t)nrhs * L.ld, c->s));
        float best = 1e30f;
        int best_v = 0, best_g = 8;
        for (int g : {0, 4, 8, 16}) {
          if (g > nrhs) continue;
          L.fused_b[dt] = g == 0 ? 0 : (dt == CHEBMG_F32 ? 1 : 2);
          L.fused_gsz[dt] = g == 0 ? 8 : g;
          const float t = time_it(
              [&]() {
                for (int k = 0; k < 3; ++k) {   // back to back, as in a solve
                  if (dt == CHEBMG_F64) smooth<double>(c, j, vec<double>(L, VB), vec<double>(L, VX), 4, true);
                  else smooth<float>(c, j, vec<float>(L, VB), vec<float>(L, VX), 4, true);
                }
              },
              2);
          if (t < best) {
            best = t;
            best_v = L.fused_b[dt];
            best_g = L.fused_gsz[dt];
          }
        }
        L.fused_b[dt] = best_v;
        L.fused_gsz[dt] = best_g;
      }
    }
  }
  Level& C = c->L.back();
  if (C.type == TYPE_SEM && c->ell_col && coarse_block_supported(C.n)) {
    const int64_t ldc = ldv(c, C);
    splitmix_fill(C.n, 7ull, static_cast<const double*>(C.invD[CHEBMG_F64]), c->cb, c->s);
    for (int q = 1; q < nrhs; ++q)
      CK(cudaMemcpyAsync(c->cb + q * ldc, c->cb, sizeof(double) * C.n, cudaMemcpyDeviceToDevice, c->s));
    std::vector<unsigned> st(2 * (size_t)nrhs);
    float best = 1e30f;
    int best_m = 1;
    for (int m : {1, 2, 4, 8, 12, 16, 24}) {
      c->bcoarse_degree = m;
      const float t = time_it([&]() { coarse_solve64_batched(c, c->cb, c->cx); }, 2);
      CK(cudaMemcpy(st.data(), c->bcstat, sizeof(unsigned) * st.size(), cudaMemcpyDeviceToHost));
      bool ok = true;
      for (int q = 0; q < nrhs; ++q) ok = ok && st[2 * q] == CS_OK;
      if (ok && t < best) {
        best = t;
        best_m = m;
      }
    }
    c->bcoarse_degree = best_m;
    CK(cudaMemsetAsync(c->dstat + 1, 0, sizeof(unsigned), c->s));
  }
  c->nb = saved_nb;
  c->batched = saved_batched;
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  CK(cudaStreamSynchronize(c->s));
  c->btuned = nrhs;
}

// ---- batched flexible CG, split into launch sequences without host decisions ----
// Mixed form: the V-cycle reads the FP32 copy of r that the x/r update writes, and its FP32
// output feeds the dots and the p update directly (as in the single solve).
bool bfcg_mixed(const chebmg_ctx* c) { return c->fp32 && c->L.size() > 1; }

int bfcg_precondition(chebmg_ctx* c, bool r32_ready) {
  if (!bfcg_mixed(c)) return vcycle_top(c, c->kr, c->kz);
  Level& L = c->L[0];
  float* r32 = vec<float>(L, VB);
  const int64_t ld = ldv(c, L);
  if (!r32_ready) cast<double, float>(L.n, c->kr, r32, c->s, c->nb, ld, ld);
  return vcycle_level<float>(c, 0, r32, vec<float>(L, VX));
}

void bfcg_start(chebmg_ctx* c, const double* B, int64_t ldb, double rtol) {
  Level& L = c->L[0];
  const int nb = c->nb;
  const int64_t n = L.n, ld = ldv(c, L);
  const double* S = static_cast<const double*>(L.invD[CHEBMG_F64]);
  CK(cudaMemsetAsync(c->dstat, 0, sizeof(unsigned) * 2, c->s));
  masked_copy(n, B, S, c->kr, c->s, nb, ldb, ld);
  zero<double>(c, c->kx, span(c, L));
  bdot2(n, ld, nb, c->kr, c->kr, nullptr, nullptr, BPOST_INIT, rtol, c->bpart, c->bscal, c->bstat, c->s);
  const int rc = bfcg_precondition(c, false);
  if (rc != CHEBMG_OK && rc != CHEBMG_ENOTCONV) throw Error(rc, "V-cycle failed");
  if (bfcg_mixed(c)) {
    const float* z32 = vec<float>(L, VX);
    bupdate_p_from<float>(n, ld, nb, z32, c->kp, c->bscal, true, c->s, c->kq);
    bdot_zr_zq<float>(n, ld, nb, z32, c->kr, nullptr, BPOST_SET_RZ, c->bpart, c->bscal, c->bstat, c->s);
  } else {
    bupdate_p_from<double>(n, ld, nb, c->kz, c->kp, c->bscal, true, c->s, c->kq);
    bdot_zr_zq<double>(n, ld, nb, c->kz, c->kr, nullptr, BPOST_SET_RZ, c->bpart, c->bscal, c->bstat, c->s);
  }
  check_launch();
}

// q = A p; alpha; x += alpha p; r -= alpha q; convergence test
void bfcg_body1(chebmg_ctx* c) {
  Level& L = c->L[0];
  const int nb = c->nb;
  const int64_t n = L.n, ld = ldv(c, L);
  // q was zeroed by the p update that precedes every body1
  if (c->outer_op == 1 && c->G_x2) {
    // the FP32-pair operator with the batched FP64 kernel's elements and right-hand sides per block
    const int v = L.beb[CHEBMG_F64];
    sem_ax8_x2(L.E, L.gid, L.lat, c->G_x2, c->kp, c->kq, c->dstat, v % 1000, c->s, nb, ld, v / 1000);
  } else {
    apply_into<double>(c, 0, c->kp, c->kq);
  }
  bdot2(n, ld, nb, c->kp, c->kq, nullptr, nullptr, BPOST_ALPHA, 0.0, c->bpart, c->bscal, c->bstat, c->s);
  bfcg_update_xr32(n, ld, nb, c->kx, c->kr, bfcg_mixed(c) ? vec<float>(L, VB) : nullptr, c->kp, c->kq, c->bpart,
                   c->bscal, c->bstat, c->s);
  check_launch();
}

// z = V-cycle(r); Polak-Ribiere beta; p = z + beta p
void bfcg_body2(chebmg_ctx* c) {
  Level& L = c->L[0];
  const int nb = c->nb;
  const int64_t n = L.n, ld = ldv(c, L);
  const int rc = bfcg_precondition(c, true);
  if (rc != CHEBMG_OK && rc != CHEBMG_ENOTCONV) throw Error(rc, "V-cycle failed");
  if (bfcg_mixed(c)) {
    const float* z32 = vec<float>(L, VX);
    bdot_zr_zq<float>(n, ld, nb, z32, c->kr, c->kq, BPOST_BETA_Q, c->bpart, c->bscal, c->bstat, c->s);
    bupdate_p_from<float>(n, ld, nb, z32, c->kp, c->bscal, false, c->s, c->kq);
  } else {
    bdot_zr_zq<double>(n, ld, nb, c->kz, c->kr, c->kq, BPOST_BETA_Q, c->bpart, c->bscal, c->bstat, c->s);
    bupdate_p_from<double>(n, ld, nb, c->kz, c->kp, c->bscal, false, c->s, c->kq);
  }
  check_launch();
}

// Queues the read-back of the status words (and device error flags) on stream s.
void bfcg_queue_read(chebmg_ctx* c, cudaStream_t s) {
  CK(cudaMemcpyAsync(c->hbstat, c->bstat, sizeof(int) * 4 * c->nb, cudaMemcpyDeviceToHost, s));
  CK(cudaMemcpyAsync(c->hdstat, c->dstat, sizeof(unsigned) * 4, cudaMemcpyDeviceToHost, s));
}

int bfcg_active(const chebmg_ctx* c) {
  int a = 0;
  for (int q = 0; q < c->nb; ++q) a += c->hbstat[4 * q] != 0;
  return a;
}

// Copies the solutions out and fills the per-right-hand-side results; returns the worst status.
int bfcg_finish(chebmg_ctx* c, double* U, int64_t ldu, int* iters, double* relres) {
  Level& L = c->L[0];
  cast<double, double>(L.n, c->kx, U, c->s, c->nb, ldv(c, L), ldu);
  CK(cudaMemcpyAsync(c->hbscal, c->bscal, sizeof(double) * S_NSLOTS * c->nb, cudaMemcpyDeviceToHost, c->s));
  bfcg_queue_read(c, c->s);
  CK(cudaStreamSynchronize(c->s));
  check_launch();
  int worst = CHEBMG_OK;
  for (int q = 0; q < c->nb; ++q) {
    const double* sc = c->hbscal + q * S_NSLOTS;
    const int* st = c->hbstat + 4 * q;
    if (iters) iters[q] = st[1];
    if (relres) relres[q] = sc[S_BB] > 0.0 ? std::sqrt(sc[S_RR] / sc[S_BB]) : 0.0;
    int rc = CHEBMG_OK;
    if (st[2] == BS_BREAKDOWN) rc = CHEBMG_EBREAKDOWN;
    else if (st[0] != 0 || st[2] != BS_OK) rc = CHEBMG_ENOTCONV;
    if (rc == CHEBMG_EBREAKDOWN || (rc == CHEBMG_ENOTCONV && worst == CHEBMG_OK)) worst = rc;
  }
  if (c->hdstat[0]) return CHEBMG_ETIMEOUT;
  if (c->hdstat[1] == CS_BREAKDOWN) return CHEBMG_EBREAKDOWN;
  return worst;
}

// Captures fn (a launch sequence on c->s) into an executable graph; launches counted per replay.
template <typename F>
cudaGraphExec_t capture(chebmg_ctx* c, F&& fn, int64_t* launches) {
  cudaGraph_t g = nullptr;
  CK(cudaStreamBeginCapture(c->s, cudaStreamCaptureModeThreadLocal));
  const int64_t l0 = g_launches.load();
  try {
    fn();
  } catch (...) {
    cudaStreamEndCapture(c->s, &g);
    if (g) cudaGraphDestroy(g);
    throw;
  }
  const int64_t l1 = g_launches.load();
  CK(cudaStreamEndCapture(c->s, &g));
  g_launches.fetch_sub(l1 - l0);
  *launches = l1 - l0;
  cudaGraphExec_t ex = nullptr;
  const cudaError_t e = cudaGraphInstantiate(&ex, g, 0);
  cudaGraphDestroy(g);
  if (e != cudaSuccess) throw Error(CHEBMG_ECUDA, std::string("cudaGraphInstantiate: ") + cudaGetErrorString(e));
  return ex;
}

void replay(chebmg_ctx* c, int k) {
  CK(cudaGraphLaunch(c->gexec[k], c->s));
  g_launches.fetch_add(c->glaunches[k]);
}

// Runs on the context's private stream (needed for capture) and restores the caller's stream.
struct PrivateStream {
  chebmg_ctx* c;
  cudaStream_t saved;
  explicit PrivateStream(chebmg_ctx* cc) : c(cc), saved(cc->s) {
    if (!c->gs) CK(cudaStreamCreateWithFlags(&c->gs, cudaStreamNonBlocking));
    CK(cudaStreamSynchronize(saved));
    c->s = c->gs;
  }
  ~PrivateStream() {
    cudaStreamSynchronize(c->gs);
    c->s = saved;
  }
};

struct BatchScope {
  chebmg_ctx* c;
  BatchScope(chebmg_ctx* cc, int nb) : c(cc) {
    c->nb = nb;
    c->batched = true;
  }
  ~BatchScope() {
    c->nb = 1;
    c->batched = false;
  }
};

int pcg_batched(chebmg_ctx* c, int nrhs, const double* B, int64_t ldb, double* U, int64_t ldu, double rtol,
                int maxit, int* iters, double* relres, bool graphs) {
  reserve_batch(c, nrhs);
  autotune_batch(c, nrhs);
  PrivateStream ps(c);
  BatchScope bs(c, nrhs);
  const bool use_graph = graphs && coarse_batch_capturable(c);
  bfcg_start(c, B, ldb, rtol);
  bfcg_queue_read(c, c->s);
  CK(cudaStreamSynchronize(c->s));
  if (bfcg_active(c) == 0 || maxit == 0) return bfcg_finish(c, U, ldu, iters, relres);
  if (use_graph && c->gexec_nb != nrhs) {
    drop_graphs(c);
    // first iteration eagerly (first-launch configuration happens outside capture)
    bfcg_body1(c);
    bfcg_queue_read(c, c->s);
    CK(cudaStreamSynchronize(c->s));
    if (bfcg_active(c) == 0 || maxit == 1) return bfcg_finish(c, U, ldu, iters, relres);
    bfcg_body2(c);
    c->gexec[0] = capture(c, [&]() { bfcg_body1(c); }, &c->glaunches[0]);
    c->gexec[1] = capture(c, [&]() { bfcg_body2(c); }, &c->glaunches[1]);
    c->gexec_nb = nrhs;
    for (int it = 2; it <= maxit; ++it) {
      replay(c, 0);
      bfcg_queue_read(c, c->s);
      CK(cudaStreamSynchronize(c->s));
      if (bfcg_active(c) == 0 || c->hdstat[0]) break;
      if (it < maxit) replay(c, 1);
    }
    return bfcg_finish(c, U, ldu, iters, relres);
  }
  for (int it = 1; it <= maxit; ++it) {
    if (use_graph) replay(c, 0);
    else bfcg_body1(c);
    bfcg_queue_read(c, c->s);
    CK(cudaStreamSynchronize(c->s));
    if (bfcg_active(c) == 0 || c->hdstat[0]) break;
    if (it < maxit) {
      if (use_graph) replay(c, 1);
      else bfcg_body2(c);
    }
  }
  return bfcg_finish(c, U, ldu, iters, relres);
}

// ===========================================================================
// Adjoint of the smoothed V-cycle (gradient of the error-reduction ratio)
// ===========================================================================
enum GW { GW_XB = 0, GW_BB, GW_X0B, GW_RB, GW_RHO, GW_DEL, GW_YA, GW_XM, GW_XS, GW_N };

void grad_alloc(chebmg_ctx* c, int nb, int kmax, int steps) {
  auto& g = c->gw;
  if (g.nb >= nb && g.kmax >= kmax && g.steps >= steps) return;
  CK(cudaStreamSynchronize(c->s));
  auto take = [&](double*& p, int64_t count) {
    void* v = p;
    replace_alloc(c, v, sizeof(double) * (size_t)count);
    p = static_cast<double*>(v);
  };
  nb = std::max(nb, g.nb);
  kmax = std::max(kmax, g.kmax);
  steps = std::max(steps, g.steps);
  const int nl = (int)c->L.size();
  g.lv.resize(nl);
  for (int j = 0; j < nl; ++j) {
    g.lv[j].resize(GW_N, nullptr);
    for (int w = 0; w < GW_N; ++w) take(g.lv[j][w], (int64_t)nb * c->L[j].ld);
  }
  const int64_t v0 = (int64_t)nb * c->L[0].ld;
  g.D.resize(kmax, nullptr);
  g.SR.resize(kmax, nullptr);
  for (int i = 0; i < kmax; ++i) {
    take(g.D[i], v0);
    take(g.SR[i], v0);
  }
  g.Et.resize(steps + 1, nullptr);
  for (auto& p : g.Et) take(p, v0);
  for (double** p : {&g.W, &g.Z, &g.EB, &g.ZB, &g.WB}) take(*p, v0);
  take(g.part, adj_dot_scratch(c->L[0].n, nb));
  take(g.acc, kmax + nl);
  take(g.rows, 2 * (int64_t)nb);
  take(g.coef, nb);
  g.nb = nb;
  g.kmax = kmax;
  g.steps = steps;
}

// Forward V-cycle in FP64 (Eq. 2.2) that also keeps each level's iterate before the
// post-smoother (the input of that smoother call, needed by its adjoint).
int vcycle_store(chebmg_ctx* c, int j, const double* b, double* x) {
  const int last = (int)c->L.size() - 1;
  if (j == last) return coarse<double>(c, b, x);
  Level& L = c->L[j];
  Level& C = c->L[j + 1];
  if (c->pre > 0) smooth<double>(c, j, b, x, c->pre, true);
  else zero<double>(c, x, span(c, L));
  double* y = vec<double>(L, VY);
  double* r = vec<double>(L, VR);
  zero<double>(c, y, span(c, L));
  apply_into<double>(c, j, x, y);
  residual<double>(L.n, b, y, r, c->s, c->nb, ldv(c, L));
  restrict_to<double>(c, j, r, vec<double>(C, VB));
  const int rc = vcycle_store(c, j + 1, vec<double>(C, VB), vec<double>(C, VX));
  if (rc != CHEBMG_OK && rc != CHEBMG_ENOTCONV) return rc;
  prolong_to<double>(c, j, vec<double>(C, VX), x, 1);
  if (c->post > 0) {
    CK(cudaMemcpyAsync(c->gw.lv[j][GW_XM], x, sizeof(double) * span(c, L), cudaMemcpyDeviceToDevice, c->s));
    smooth<double>(c, j, b, x, c->post, false);
  }
  check_launch();
  return rc;
}

// Adjoint of one Algorithm-2 smoother call on level j (inputs b and x0, x0 = null for a zero
// guess) for the output adjoint xbar: bbar += b-bar, x0bar = x0-bar (if x0), and the weight
// and lambda adjoints accumulate into gw.acc[0 .. order-1] and gw.acc[kmax + j].
void smooth_adj(chebmg_ctx* c, int j, const double* b, const double* x0, int order, const double* xbar,
                double* bbar, double* x0bar) {
  auto& g = c->gw;
  Level& L = c->L[j];
  const int nb = c->nb;
  const int64_t n = L.n, ld = ldv(c, L), sp = span(c, L);
  const double* S = static_cast<const double*>(L.invD[CHEBMG_F64]);
  const double lam = L.lmax * c->lscale;
  const std::vector<double>& beta = c->beta_ovr;
  double* r = vec<double>(L, VR);
  double* d = vec<double>(L, VD);
  double* y = vec<double>(L, VY);
  double* xs = g.lv[j][GW_XS];
  // forward recomputation, recording d_i and S r_i
  zero<double>(c, y, sp);
  if (x0) {
    CK(cudaMemcpyAsync(xs, x0, sizeof(double) * sp, cudaMemcpyDeviceToDevice, c->s));
    apply_into<double>(c, j, xs, y);
  }
  cheb4_init<double>(n, b, xs, r, d, y, S, 4.0 / (3.0 * lam), x0 ? 0 : 1, c->s, nb, ld);
  adj_record(n, ld, nb, d, r, S, g.D[0], g.SR[0], c->s);
  for (int i = 1; i < order; ++i) {
    zero<double>(c, y, sp);
    apply_into<double>(c, j, d, y);
    const double c1 = (2.0 * i - 1.0) / (2.0 * i + 3.0);
    const double c2 = (8.0 * i + 4.0) / ((2.0 * i + 3.0) * lam);
    cheb4_step<double>(n, xs, r, d, y, S, beta[i - 1], c1, c2, c->s, nb, ld);
    adj_record(n, ld, nb, d, r, S, g.D[i], g.SR[i], c->s);
  }
  // backward
  const int lslot = g.kmax + j;
  for (int i = 1; i <= order; ++i) dot_accumulate(n, ld, nb, xbar, g.D[i - 1], 1.0, g.part, g.acc, i - 1, c->s);
  double* rho = g.lv[j][GW_RHO];
  double* del = g.lv[j][GW_DEL];
  double* ya = g.lv[j][GW_YA];
  lincomb(n, ld, nb, beta[order - 1], xbar, 0.0, nullptr, del, c->s);
  zero<double>(c, rho, sp);
  zero<double>(c, ya, sp);
  for (int i = order - 1; i >= 1; --i) {
    const double c1 = (2.0 * i - 1.0) / (2.0 * i + 3.0);
    const double c2 = (8.0 * i + 4.0) / (2.0 * i + 3.0);
    adj_rho(n, ld, nb, c2 / lam, S, del, rho, c->s);
    dot_accumulate(n, ld, nb, del, g.SR[i], -c2 / (lam * lam), g.part, g.acc, lslot, c->s);
    apply_into<double>(c, j, rho, ya);
    adj_delta(n, ld, nb, beta[i - 1], c1, xbar, del, ya, c->s);
  }
  adj_rho(n, ld, nb, 4.0 / (3.0 * lam), S, del, rho, c->s);
  dot_accumulate(n, ld, nb, del, g.SR[0], -4.0 / (3.0 * lam * lam), g.part, g.acc, lslot, c->s);
  lincomb(n, ld, nb, 1.0, bbar, 1.0, rho, bbar, c->s);
  if (x0) {
    zero<double>(c, ya, sp);
    apply_into<double>(c, j, rho, ya);
    lincomb(n, ld, nb, 1.0, xbar, -1.0, ya, x0bar, c->s);
  }
  check_launch();
}

// Transposed V-cycle from level j: bbar = B_j^T xbar, with the parameter adjoints accumulated.
// Uses the forward state of the last vcycle_store (each level's right-hand side in VB, the
// pre-post-smoother iterates in gw XM); b is level j's forward right-hand side.
int vcycle_adj(chebmg_ctx* c, int j, const double* b, const double* xbar, double* bbar) {
  auto& g = c->gw;
  const int last = (int)c->L.size() - 1;
  if (j == last) return coarse<double>(c, xbar, bbar);   // A_c^{-1} is symmetric
  Level& L = c->L[j];
  Level& C = c->L[j + 1];
  const int nb = c->nb;
  const int64_t n = L.n, ld = ldv(c, L), sp = span(c, L);
  double* x0bar = g.lv[j][GW_X0B];
  zero<double>(c, bbar, sp);
  if (c->post > 0) smooth_adj(c, j, b, g.lv[j][GW_XM], c->post, xbar, bbar, x0bar);
  else CK(cudaMemcpyAsync(x0bar, xbar, sizeof(double) * sp, cudaMemcpyDeviceToDevice, c->s));
  // x_mid = x_pre + P x_c
  restrict_to<double>(c, j, x0bar, g.lv[j + 1][GW_XB]);
  const int rc = vcycle_adj(c, j + 1, vec<double>(C, VB), g.lv[j + 1][GW_XB], g.lv[j + 1][GW_BB]);
  if (rc != CHEBMG_OK && rc != CHEBMG_ENOTCONV) return rc;
  // r_c = P^T (b - A x_pre)
  double* rb = g.lv[j][GW_RB];
  prolong_to<double>(c, j, g.lv[j + 1][GW_BB], rb, 0);
  lincomb(n, ld, nb, 1.0, bbar, 1.0, rb, bbar, c->s);
  double* ya = g.lv[j][GW_YA];
  zero<double>(c, ya, sp);
  apply_into<double>(c, j, rb, ya);
  lincomb(n, ld, nb, 1.0, x0bar, -1.0, ya, x0bar, c->s);
  if (c->pre > 0) smooth_adj(c, j, b, nullptr, c->pre, x0bar, bbar, nullptr);
  check_launch();
  return rc;
}

// f = mean_q ||(I - B A)^steps e0_q||^2 / ||e0_q||^2 and its gradient with respect to the
// weights and the lambda_max scale, for nrhs initial errors E0 [nrhs][n] (device).
int cycle_error_grad(chebmg_ctx* c, int nrhs, const double* E0, int steps, const double* betas, int nbeta,
                     double scale, double* f_out, double* gbeta, double* gscale, double* f_each) {
  if (c->o.kind == CHEBMG_CHEB_1ST) throw Error(CHEBMG_EINVAL, "the weights belong to the 4th-kind smoother");
  if (nbeta != c->pre || (c->post != 0 && c->post != c->pre))
    throw Error(CHEBMG_EINVAL, "one weight per smoothing step: nbeta must equal the smoothing order");
  if (c->L.size() < 2) throw Error(CHEBMG_EINVAL, "need at least two levels");
  reserve_batch(c, nrhs);
  autotune_batch(c, nrhs);
  grad_alloc(c, nrhs, nbeta, steps);
  auto& g = c->gw;
  struct Restore {
    chebmg_ctx* c;
    std::vector<double> b;
    double s;
    ~Restore() {
      c->beta_ovr = b;
      c->lscale = s;
    }
  } restore{c, c->beta_ovr, c->lscale};
  c->beta_ovr.assign(betas, betas + nbeta);
  c->lscale = scale;
  BatchScope bs(c, nrhs);
  Level& L = c->L[0];
  const int64_t n = L.n, ld = ldv(c, L), sp = span(c, L);
  const double* S = static_cast<const double*>(L.invD[CHEBMG_F64]);
  CK(cudaMemsetAsync(c->dstat, 0, sizeof(unsigned) * 2, c->s));
  masked_copy(n, E0, S, g.Et[0], c->s, nrhs, n, ld);
  dot_rows(n, ld, nrhs, g.Et[0], g.Et[0], g.part, g.rows, c->s);
  int rc = CHEBMG_OK;
  for (int t = 0; t < steps; ++t) {
    zero<double>(c, g.W, sp);
    apply_into<double>(c, 0, g.Et[t], g.W);
    rc = vcycle_store(c, 0, g.W, g.Z);
    if (rc != CHEBMG_OK && rc != CHEBMG_ENOTCONV) return rc;
    lincomb(n, ld, nrhs, 1.0, g.Et[t], -1.0, g.Z, g.Et[t + 1], c->s);
  }
  dot_rows(n, ld, nrhs, g.Et[steps], g.Et[steps], g.part, g.rows + nrhs, c->s);
  std::vector<double> rows(2 * (size_t)nrhs);
  CK(cudaMemcpyAsync(rows.data(), g.rows, sizeof(double) * rows.size(), cudaMemcpyDeviceToHost, c->s));
  CK(cudaStreamSynchronize(c->s));
  double f = 0.0;
  std::vector<double> coef(nrhs);
  for (int q = 0; q < nrhs; ++q) {
    if (!(rows[q] > 0.0)) throw Error(CHEBMG_EINVAL, "an initial error is zero");
    const double fq = rows[nrhs + q] / rows[q];
    if (f_each) f_each[q] = fq;
    f += fq / nrhs;
    coef[q] = 2.0 / (nrhs * rows[q]);
  }
  *f_out = f;
  if (!gbeta) return CHEBMG_OK;   // objective only
  CK(cudaMemcpyAsync(g.coef, coef.data(), sizeof(double) * nrhs, cudaMemcpyHostToDevice, c->s));
  scale_rows(n, ld, nrhs, g.coef, g.Et[steps], g.EB, c->s);
  CK(cudaMemsetAsync(g.acc, 0, sizeof(double) * (g.kmax + c->L.size()), c->s));
  for (int t = steps - 1; t >= 0; --t) {
    lincomb(n, ld, nrhs, -1.0, g.EB, 0.0, nullptr, g.ZB, c->s);
    zero<double>(c, g.W, sp);
    apply_into<double>(c, 0, g.Et[t], g.W);
    rc = vcycle_store(c, 0, g.W, g.Z);                  // recomputed forward state of cycle t
    if (rc != CHEBMG_OK && rc != CHEBMG_ENOTCONV) return rc;
    rc = vcycle_adj(c, 0, g.W, g.ZB, g.WB);
    if (rc != CHEBMG_OK && rc != CHEBMG_ENOTCONV) return rc;
    double* ya = g.lv[0][GW_YA];
    zero<double>(c, ya, sp);
    apply_into<double>(c, 0, g.WB, ya);
    lincomb(n, ld, nrhs, 1.0, g.EB, 1.0, ya, g.EB, c->s);
  }
  std::vector<double> acc(g.kmax + c->L.size());
  CK(cudaMemcpyAsync(acc.data(), g.acc, sizeof(double) * acc.size(), cudaMemcpyDeviceToHost, c->s));
  CK(cudaMemcpyAsync(c->hdstat, c->dstat, sizeof(unsigned) * 4, cudaMemcpyDeviceToHost, c->s));
  CK(cudaStreamSynchronize(c->s));
  check_launch();
  if (c->hdstat[0]) return CHEBMG_ETIMEOUT;
  if (c->hdstat[1] == CS_BREAKDOWN) return CHEBMG_EBREAKDOWN;
  for (int i = 0; i < nbeta; ++i) gbeta[i] = acc[i];
  double gs = 0.0;
  for (size_t j = 0; j + 1 < c->L.size(); ++j) gs += acc[g.kmax + j] * c->L[j].lmax;
  *gscale = gs;
  return CHEBMG_OK;
}

// ===========================================================================
// Restarted flexible GMRES(m) preconditioned by one V-cycle (Sec. 6.1; Table 1 of Sec. 3)
// ===========================================================================
int gmres_solve(chebmg_ctx* c, const double* b, double* u, double rtol, int m, int maxit, int* iters,
                double* relres, double* history) {
  Level& L = c->L[0];
  const int64_t n = L.n, ld = L.ld;
  auto& g = c->gm;
  if (g.m < m) {
    CK(cudaStreamSynchronize(c->s));
    replace_vec(c, g.V, (int64_t)(m + 1) * ld);
    replace_vec(c, g.Z, (int64_t)m * ld);
    replace_vec(c, g.w, ld);
    replace_vec(c, g.bm, ld);
    replace_vec(c, g.part, gmres_part_size(n));
    replace_vec(c, g.h, m + 2);
    if (g.hh) cudaFreeHost(g.hh);
    g.hh = nullptr;
    void* hp = nullptr;
    CK(cudaMallocHost(&hp, sizeof(double) * (m + 2)));
    g.hh = static_cast<double*>(hp);
    g.m = m;
  }
  const double* S = static_cast<const double*>(L.invD[CHEBMG_F64]);
  reset_coarse_sticky(c);
  CK(cudaMemsetAsync(c->dstat, 0, sizeof(unsigned), c->s));
  masked_copy(n, b, S, g.bm, c->s);
  zero<double>(c, u, n);
  double* r = g.w;
  CK(cudaMemcpyAsync(r, g.bm, sizeof(double) * n, cudaMemcpyDeviceToDevice, c->s));
  auto read_norm = [&]() {
    CK(cudaMemcpyAsync(g.hh, g.h, sizeof(double), cudaMemcpyDeviceToHost, c->s));
    CK(cudaStreamSynchronize(c->s));
    return g.hh[0];
  };
  gmres_norm_scale(n, r, g.part, g.h, nullptr, c->s);
  const double bnorm = read_norm();
  if (iters) *iters = 0;
  if (history) history[0] = 1.0;
  if (!std::isfinite(bnorm)) return CHEBMG_EBREAKDOWN;
  if (bnorm == 0.0) {
    if (relres) *relres = 0.0;
    return CHEBMG_OK;
  }
  double beta = bnorm;
  int its = 0;
  std::vector<double> R((size_t)m * (m + 1)), cs(m), sn(m), gv(m + 1), y(m);
  while (its < maxit) {
    // v_0 = r / beta
    gmres_norm_scale(n, r, g.part, g.h, g.V, c->s);
    std::fill(gv.begin(), gv.end(), 0.0);
    gv[0] = beta;
    int jd = 0;
    double est = 1.0;
    for (int j = 0; j < m; ++j) {
      double* vj = g.V + (int64_t)j * ld;
      double* zj = g.Z + (int64_t)j * ld;
      const int rc = vcycle_top(c, vj, zj);
      if (rc != CHEBMG_OK && rc != CHEBMG_ENOTCONV) return rc;
      zero<double>(c, g.w, n);
      apply_into<double>(c, 0, zj, g.w);
      gmres_mdot(n, ld, j + 1, g.V, g.w, g.part, g.h, c->s);
      gmres_maxpy_norm(n, ld, j + 1, g.V, g.h, -1.0, g.w, g.part, g.h + j + 1, g.V + (int64_t)(j + 1) * ld, c->s);
      check_launch();
      CK(cudaMemcpyAsync(g.hh, g.h, sizeof(double) * (j + 2), cudaMemcpyDeviceToHost, c->s));
      CK(cudaMemcpyAsync(c->hdstat, c->dstat, sizeof(unsigned) * 4, cudaMemcpyDeviceToHost, c->s));
      if (c->cctl) CK(cudaMemcpyAsync(c->hcctl, c->cctl, sizeof(unsigned) * 5, cudaMemcpyDeviceToHost, c->s));
      CK(cudaStreamSynchronize(c->s));
      ++its;
      const int crc = coarse_sticky_error(c);
      if (crc != CHEBMG_OK) {
        if (iters) *iters = its;
        return crc;
      }
      double* col = R.data() + (size_t)j * (m + 1);
      for (int i = 0; i <= j + 1; ++i) col[i] = g.hh[i];
      if (!std::isfinite(col[j + 1])) {
        if (iters) *iters = its;
        return CHEBMG_EBREAKDOWN;
      }
      const double hlast = col[j + 1];
      for (int i = 0; i < j; ++i) {
        const double t = cs[i] * col[i] + sn[i] * col[i + 1];
        col[i + 1] = -sn[i] * col[i] + cs[i] * col[i + 1];
        col[i] = t;
      }
      const double den = std::hypot(col[j], col[j + 1]);
      cs[j] = den > 0.0 ? col[j] / den : 1.0;
      sn[j] = den > 0.0 ? col[j + 1] / den : 0.0;
      col[j] = den;
      col[j + 1] = 0.0;
      gv[j + 1] = -sn[j] * gv[j];
      gv[j] = cs[j] * gv[j];
      est = std::fabs(gv[j + 1]) / bnorm;
      if (history) history[its] = est;
      jd = j + 1;
      if (est <= rtol || hlast == 0.0 || its >= maxit) break;
    }
    // y = R^{-1} g, u += Z y
    for (int i = jd - 1; i >= 0; --i) {
      double t = gv[i];
      for (int k = i + 1; k < jd; ++k) t -= R[(size_t)k * (m + 1) + i] * y[k];
      const double d = R[(size_t)i * (m + 1) + i];
      y[i] = d != 0.0 ? t / d : 0.0;
    }
    CK(cudaMemcpyAsync(g.h, y.data(), sizeof(double) * jd, cudaMemcpyHostToDevice, c->s));
    gmres_maxpy_norm(n, ld, jd, g.Z, g.h, 1.0, u, nullptr, nullptr, nullptr, c->s);
    // true residual r = b - A u
    zero<double>(c, g.w, n);
    apply_into<double>(c, 0, u, g.w);
    lincomb(n, n, 1, 1.0, g.bm, -1.0, g.w, g.w, c->s);   // w = b - A u
    gmres_norm_scale(n, r, g.part, g.h, nullptr, c->s);
    beta = read_norm();
    const double rel = beta / bnorm;
    if (iters) *iters = its;
    if (relres) *relres = rel;
    if (!std::isfinite(rel)) return CHEBMG_EBREAKDOWN;
    if (rel <= rtol) return CHEBMG_OK;
  }
  return CHEBMG_ENOTCONV;
}

}  // namespace

// A fixed set of contexts (meshes of different sizes and orders) solved together: one
// right-hand side each, every context on its own stream, each Krylov half-iteration of all
// of them captured as one CUDA graph (fork/join over the contexts' streams).
struct chebmg_group {
  std::vector<chebmg_ctx*> c;
  int dev = 0;
  cudaStream_t s = nullptr;
  cudaEvent_t fork = nullptr;
  std::vector<cudaEvent_t> join;
  cudaGraphExec_t g[2] = {nullptr, nullptr};
  int64_t launches[2] = {0, 0};
  std::vector<int64_t> gens;   // contexts' graph generations when captured
};

namespace {

void group_drop(chebmg_group* g) {
  for (auto& x : g->g)
    if (x) {
      cudaGraphExecDestroy(x);
      x = nullptr;
    }
  g->gens.clear();
}

// Every context on its private stream in batched mode with one right-hand side; restored on exit.
struct GroupScope {
  chebmg_group* g;
  std::vector<cudaStream_t> saved;
  explicit GroupScope(chebmg_group* gg) : g(gg) {
    for (chebmg_ctx* c : g->c) {
      if (!c->gs) CK(cudaStreamCreateWithFlags(&c->gs, cudaStreamNonBlocking));
      CK(cudaStreamSynchronize(c->s));
      saved.push_back(c->s);
      c->s = c->gs;
      c->nb = 1;
      c->batched = true;
    }
  }
  ~GroupScope() {
    for (size_t k = 0; k < saved.size(); ++k) {
      chebmg_ctx* c = g->c[k];
      cudaStreamSynchronize(c->gs);
      c->s = saved[k];
      c->nb = 1;
      c->batched = false;
    }
  }
};

template <typename F>
cudaGraphExec_t group_capture(chebmg_group* g, F&& body, int64_t* launches) {
  cudaGraph_t graph = nullptr;
  CK(cudaStreamBeginCapture(g->s, cudaStreamCaptureModeThreadLocal));
  const int64_t l0 = g_launches.load();
  try {
    CK(cudaEventRecord(g->fork, g->s));
    for (size_t k = 0; k < g->c.size(); ++k) {
      chebmg_ctx* c = g->c[k];
      CK(cudaStreamWaitEvent(c->s, g->fork, 0));
      body(c);
      CK(cudaEventRecord(g->join[k], c->s));
      CK(cudaStreamWaitEvent(g->s, g->join[k], 0));
    }
  } catch (...) {
    cudaStreamEndCapture(g->s, &graph);
    if (graph) cudaGraphDestroy(graph);
    throw;
  }
  const int64_t l1 = g_launches.load();
  CK(cudaStreamEndCapture(g->s, &graph));
  g_launches.fetch_sub(l1 - l0);
  *launches = l1 - l0;
  cudaGraphExec_t ex = nullptr;
  const cudaError_t e = cudaGraphInstantiate(&ex, graph, 0);
  cudaGraphDestroy(graph);
  if (e != cudaSuccess) throw Error(CHEBMG_ECUDA, std::string("cudaGraphInstantiate: ") + cudaGetErrorString(e));
  return ex;
}

int group_active(chebmg_group* g, cudaStream_t s) {
  for (chebmg_ctx* c : g->c) bfcg_queue_read(c, s ? s : c->s);
  if (s) CK(cudaStreamSynchronize(s));
  else
    for (chebmg_ctx* c : g->c) CK(cudaStreamSynchronize(c->s));
  int a = 0;
  for (chebmg_ctx* c : g->c) {
    if (c->hdstat[0]) return 0;
    a += bfcg_active(c);
  }
  return a;
}

int group_solve(chebmg_group* g, const double* const* B, double* const* U, double rtol, int maxit, bool graphs,
                int* iters, double* relres) {
  for (chebmg_ctx* c : g->c) {
    reserve_batch(c, 1);
    autotune_batch(c, 1);
  }
  bool use_graph = graphs;
  for (chebmg_ctx* c : g->c) use_graph = use_graph && coarse_batch_capturable(c);
  if (use_graph && !g->gens.empty())
    for (size_t k = 0; k < g->c.size(); ++k)
      if (g->gens[k] != g->c[k]->gen) group_drop(g);
  GroupScope scope(g);
  auto finish = [&]() {
    int worst = CHEBMG_OK;
    for (size_t k = 0; k < g->c.size(); ++k) {
      const int rc = bfcg_finish(g->c[k], U[k], g->c[k]->L[0].n, iters ? iters + k : nullptr,
                                 relres ? relres + k : nullptr);
      if (rc == CHEBMG_ETIMEOUT || rc == CHEBMG_EBREAKDOWN) worst = rc;
      else if (rc != CHEBMG_OK && worst == CHEBMG_OK) worst = rc;
    }
    return worst;
  };
  for (size_t k = 0; k < g->c.size(); ++k) bfcg_start(g->c[k], B[k], g->c[k]->L[0].n, rtol);
  if (group_active(g, nullptr) == 0 || maxit == 0) return finish();
  int it = 1;
  if (use_graph && !g->g[0]) {
    for (chebmg_ctx* c : g->c) bfcg_body1(c);   // first iteration eagerly
    if (group_active(g, nullptr) == 0 || maxit == 1) return finish();
    for (chebmg_ctx* c : g->c) bfcg_body2(c);
    for (chebmg_ctx* c : g->c) CK(cudaStreamSynchronize(c->s));
    g->g[0] = group_capture(g, [](chebmg_ctx* c) { bfcg_body1(c); }, &g->launches[0]);
    g->g[1] = group_capture(g, [](chebmg_ctx* c) { bfcg_body2(c); }, &g->launches[1]);
    g->gens.clear();
    for (chebmg_ctx* c : g->c) g->gens.push_back(c->gen);
    it = 2;
  }
  for (; it <= maxit; ++it) {
    if (use_graph) {
      CK(cudaGraphLaunch(g->g[0], g->s));
      g_launches.fetch_add(g->launches[0]);
      if (group_active(g, g->s) == 0) break;
      if (it < maxit) {
        CK(cudaGraphLaunch(g->g[1], g->s));
        g_launches.fetch_add(g->launches[1]);
      }
    } else {
      for (chebmg_ctx* c : g->c) bfcg_body1(c);
      if (group_active(g, nullptr) == 0) break;
      if (it < maxit)
        for (chebmg_ctx* c : g->c) bfcg_body2(c);
    }
  }
  if (use_graph) CK(cudaStreamSynchronize(g->s));
  return finish();
}

// Uploads the host-built SEM levels (finest first) and assembles the coarsest level's ELL
// form; boxed = the levels carry the box lattice (lattice kernels usable).
// The N = 1 box operator in the symmetric 27-point stencil layout of the cluster coarse
// kernel: row g keeps the 14 forward-half entries (slot k <-> lattice offset cc_d*(k)), each
// the mean of A(g, g + o) and A(g + o, g).  Leaves the cluster kernel off if an entry is not
// a lattice neighbour (cannot happen for a box).
void stencil_layout(chebmg_ctx* c, const SemHostLevel& h, const std::vector<int>& col,
                    const std::vector<double>& val) {
  const int nx = h.nex + 1, ny = h.ney + 1, nz = h.nez + 1;
  const int64_t n = h.n;
  if ((int64_t)nx * ny * nz != n) return;
  std::vector<double> v64((size_t)kCcSlots * n, 0.0);
  auto slot_of = [](int dx, int dy, int dz) {
    for (int k = 0; k < kCcSlots; ++k)
      if (cc_dx(k) == dx && cc_dy(k) == dy && cc_dz(k) == dz) return k;
    return -1;
  };
  for (int64_t g = 0; g < n; ++g) {
    const int gx = (int)(g % nx), gy = (int)((g / nx) % ny), gz = (int)(g / ((int64_t)nx * ny));
    for (int s = 0; s < c->nslot; ++s) {
      const int64_t cc = col[(size_t)s * n + g];
      const double v = val[(size_t)s * n + g];
      const int dx = (int)(cc % nx) - gx, dy = (int)((cc / nx) % ny) - gy,
                dz = (int)(cc / ((int64_t)nx * ny)) - gz;
      if (std::abs(dx) > 1 || std::abs(dy) > 1 || std::abs(dz) > 1) {
        if (v != 0.0) return;
        continue;
      }
      const int kf = slot_of(dx, dy, dz), kb = slot_of(-dx, -dy, -dz);
      if (kf >= 0) v64[(size_t)kf * n + g] += 0.5 * v;       // stored in row g
      if (kb >= 0) v64[(size_t)kb * n + cc] += 0.5 * v;      // stored in row cc (mirror)
    }
  }
  c->cc_val64 = upload<double>(c, v64);
  c->cc_val32 = upload<float>(c, v64);
  c->cc_nx = nx;
  c->cc_ny = ny;
  c->cc_nz = nz;
  // 27 slots in lattice order for the grid-wide kernel: slot k <-> (dx, dy, dz) =
  // (k % 3 - 1, (k / 3) % 3 - 1, k / 9 - 1), the ELL entry A(g, g + offset) or zero
  std::vector<double> v27((size_t)27 * n, 0.0);
  for (int64_t g = 0; g < n; ++g) {
    const int gx = (int)(g % nx), gy = (int)((g / nx) % ny), gz = (int)(g / ((int64_t)nx * ny));
    for (int s = 0; s < c->nslot; ++s) {
      const int64_t cc = col[(size_t)s * n + g];
      const double v = val[(size_t)s * n + g];
      if (v == 0.0) continue;
      const int dx = (int)(cc % nx) - gx, dy = (int)((cc / nx) % ny) - gy,
                dz = (int)(cc / ((int64_t)nx * ny)) - gz;
      v27[(size_t)((dz + 1) * 9 + (dy + 1) * 3 + (dx + 1)) * n + g] = v;
    }
  }
  c->lat_val = upload<double>(c, v27);
  c->lat_valf = upload<float>(c, v27);
}

void upload_sem_levels(chebmg_ctx* c, std::vector<SemHostLevel>& H, bool boxed) {
  const int nlevels = (int)H.size();
  for (int j = 0; j < nlevels; ++j) {
    SemHostLevel& h = H[j];
    Level L;
    L.type = TYPE_SEM;
    L.N = h.N;
    L.Q = h.NQ;
    L.boxed = boxed;
    if (boxed)
      L.lat = {h.nex, h.ney, h.nez, (int)(h.nex * h.N + 1), (int)(h.ney * h.N + 1), (int)(h.nez * h.N + 1)};
    L.NP = h.NP;
    L.E = h.E;
    L.n = h.n;
    L.ld = (L.n + 63) / 64 * 64;
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
      if (boxed && transfer_box_supported(h.NQ, H[j + 1].NQ))
        CK(transfer_box_set_J(h.NQ, H[j + 1].NQ, J.data()));
      L.Jn[CHEBMG_F64] = upload<double>(c, J);
      if (c->fp32) L.Jn[CHEBMG_F32] = upload<float>(c, J);
    }
    if (j + 1 == nlevels) {
      std::vector<int> col;
      std::vector<double> val;
      assemble_ell(h, c->nslot, col, val);
      if (boxed && h.N == 1) stencil_layout(c, h, col, val);
      c->ell_col = dalloc<int>(c, (int64_t)col.size());
      CK(cudaMemcpy(c->ell_col, col.data(), sizeof(int) * col.size(), cudaMemcpyHostToDevice));
      c->ell_val = upload<double>(c, val);
      c->ell_valf = upload<float>(c, val);
      c->coarse_invDf = upload<float>(c, invd);
    }
    c->L.push_back(L);
    alloc_vectors(c, c->L.back(), c->fp32);
    std::vector<double>().swap(h.G);
  }
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
        L.ld = (L.n + 63) / 64 * 64;
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
      upload_sem_levels(c, H, true);
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

int chebmg_setup_sem_mesh(int64_t E, int N, const double* coords, const int64_t* gid, int64_t n,
                          const uint8_t* dirichlet, const int* orders, int nlevels, const chebmg_opts* opts,
                          chebmg_ctx** out) {
  return guard([&]() -> int {
    if (!out) throw Error(CHEBMG_EINVAL, "ctx output is NULL");
    *out = nullptr;
    if (E < 1 || N < 1 || N > 9 || !coords || !gid || n < 1 || !dirichlet || !orders || nlevels < 1)
      throw Error(CHEBMG_EINVAL, "bad SEM mesh arguments");
    if (orders[0] != N) throw Error(CHEBMG_EINVAL, "orders[0] must be the mesh order N");
    for (int j = 0; j < nlevels; ++j) {
      if (orders[j] < 1 || orders[j] > 9) throw Error(CHEBMG_EINVAL, "orders must be in 1..9");
      if (j > 0 && orders[j] >= orders[j - 1]) throw Error(CHEBMG_EINVAL, "orders must decrease");
    }
    if (n >= (int64_t)kGidMask) throw Error(CHEBMG_EINVAL, "mesh too large for 30-bit global ids");
    const int64_t NP = (int64_t)(N + 1) * (N + 1) * (N + 1);
    for (int64_t q = 0; q < E * NP; ++q)
      if (gid[q] < 0 || gid[q] >= n) throw Error(CHEBMG_EINVAL, "global id out of range");
    SemMeshInput in;
    in.E = E;
    in.N = N;
    in.coords = coords;
    in.gid = gid;
    in.n = n;
    in.dirichlet = dirichlet;
    chebmg_ctx* c = new_ctx(opts);
    try {
      c->type = TYPE_SEM;
      std::vector<SemHostLevel> H(nlevels);
      for (int j = 0; j < nlevels; ++j) {
        std::string err;
        if (!build_sem_level_mesh(in, orders[j], H[j], err))
          throw Error(err.find("Jacobian") != std::string::npos ? CHEBMG_EMESH : CHEBMG_EINVAL, err);
      }
      upload_sem_levels(c, H, false);
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
  *elements_per_block = L.type != TYPE_SEM ? 0 : L.Q == 8 ? L.eb[dtype] : L.Q == 4 ? L.ax4[dtype] : 0;
  return CHEBMG_OK;
}

int chebmg_coarse_info(const chebmg_ctx* c, int* degree, double* lmax) {
  if (!c || !degree || !lmax) return CHEBMG_EINVAL;
  *degree = (c->coop_ok && c->L.back().type == TYPE_SEM) ? c->coarse_degree : 1;
  *lmax = c->coarse_lmax;
  return CHEBMG_OK;
}

int chebmg_coarse_shape(const chebmg_ctx* c, int* kernel, int* blocks, int* rows_per_block) {
  if (!c || !kernel || !blocks || !rows_per_block) return CHEBMG_EINVAL;
  const bool sem = c->L.back().type == TYPE_SEM && c->ell_col;
  const bool cluster = sem && c->coarse_kernel == 1 && c->cc_ok && c->coarse_pf32;
  const bool grid = sem && !cluster && c->coop_ok;
  *kernel = cluster ? CHEBMG_COARSE_CLUSTER : grid ? CHEBMG_COARSE_GRID : CHEBMG_COARSE_HOST;
  *blocks = cluster ? c->cc_ctas : grid ? c->coarse_grid : 0;
  *rows_per_block = cluster ? c->cc_rmax : grid ? c->coarse_rows_per_block : 0;
  return CHEBMG_OK;
}

int chebmg_set_coarse_kernel(chebmg_ctx* c, int kernel) {
  return guard([&]() -> int {
    enter(c);
    if (kernel == CHEBMG_COARSE_CLUSTER) {
      if (!c->cc_ok || !c->coarse_pf32)
        throw Error(CHEBMG_EINVAL, "cluster coarse kernel needs a box lattice at N = 1 and an FP32 preconditioner");
      c->coarse_kernel = 1;
    } else if (kernel == CHEBMG_COARSE_GRID) {
      if (!c->coop_ok) throw Error(CHEBMG_EINVAL, "no grid-wide persistent coarse kernel in this context");
      c->coarse_kernel = 0;
    } else {
      throw Error(CHEBMG_EINVAL, "bad coarse kernel");
    }
    drop_graphs(c);
    return CHEBMG_OK;
  });
}

int chebmg_lambda_min_ratio(chebmg_ctx* c, int order, double* ratio) {
  return guard([&]() -> int {
    if (!c || !ratio || order < 1 || order > 256) throw Error(CHEBMG_EINVAL, "bad arguments");
    *ratio = lmin_ratio_for(c, order);
    return CHEBMG_OK;
  });
}

int chebmg_set_coarse_precond_dtype(chebmg_ctx* c, int dtype, int retune) {
  return guard([&]() -> int {
    enter(c);
    if (dtype != CHEBMG_F64 && dtype != CHEBMG_F32) throw Error(CHEBMG_EINVAL, "bad dtype");
    if (!c->ell_col) throw Error(CHEBMG_EINVAL, "no SEM coarse CG in this context");
    c->coarse_pf32 = dtype == CHEBMG_F32;
    if (!c->coarse_pf32) c->coarse_kernel = 0;   // the cluster kernel has an FP32 preconditioner only
    if (retune && c->coop_ok) autotune_coarse_degree(c);
    drop_graphs(c);
    CK(cudaStreamSynchronize(c->s));
    return CHEBMG_OK;
  });
}

int chebmg_set_coarse_degree(chebmg_ctx* c, int degree) {
  if (!c || degree < 1 || degree > kCoarseMaxDegree) return CHEBMG_EINVAL;
  c->coarse_degree = degree;
  c->bcoarse_degree = degree;
  drop_graphs(c);
  return CHEBMG_OK;
}

int chebmg_set_tile_choice(chebmg_ctx* c, int level, int dtype, int variant) {
  if (!c || level < 0 || level >= (int)c->L.size() || (dtype != 0 && dtype != 1)) return CHEBMG_EINVAL;
  Level& L = c->L[level];
  if (L.type == TYPE_SEM && L.Q == 4) {
    if ((variant != 40 && variant != 41 && variant != 141) || (variant == 141 && !L.boxed)) return CHEBMG_EINVAL;
    L.ax4[dtype] = variant;
    drop_graphs(c);
    return CHEBMG_OK;
  }
  if (L.type != TYPE_SEM || L.Q != 8) return CHEBMG_EINVAL;
  const int base = variant % 100;
  if ((variant != base && variant != base + 100) ||
      (base != 1 && base != 2 && base != 4 && base != 12 && base != 14 && base != 21 && base != 22 && base != 31 &&
       base != 32))
    return CHEBMG_EINVAL;
  const bool fits = dtype == CHEBMG_F64 ? sem_ax8_variant_fits<double>(variant) : sem_ax8_variant_fits<float>(variant);
  if (!fits || (variant >= 100 && !L.boxed)) return CHEBMG_EINVAL;
  L.eb[dtype] = variant;
  drop_graphs(c);
  return CHEBMG_OK;
}

int chebmg_fused_smoother(const chebmg_ctx* c, int level, int dtype, int* variant) {
  return guard([&]() -> int {
    if (!c || !variant) throw Error(CHEBMG_EINVAL, "NULL argument");
    if (level < 0 || level >= (int)c->L.size()) throw Error(CHEBMG_EINVAL, "bad level");
    if (dtype != CHEBMG_F64 && dtype != CHEBMG_F32) throw Error(CHEBMG_EINVAL, "bad dtype");
    *variant = c->L[level].fused[dtype];
    return CHEBMG_OK;
  });
}

int chebmg_set_fused_smoother(chebmg_ctx* c, int level, int dtype, int variant) {
  return guard([&]() -> int {
    enter(c);
    Level& L = level_checked(c, level);
    check_dtype(c, dtype);
    if (variant != 0) {
      if (!(L.type == TYPE_SEM && L.Q == 8 && L.boxed && L.fctl))
        throw Error(CHEBMG_EINVAL, "the fused smoother needs an order-7 box-lattice level that smooths");
      const bool ok = dtype == CHEBMG_F32 ? variant == 1 : variant == 2;
      if (!ok) throw Error(CHEBMG_EINVAL, "fused smoother variant: 1 for FP32, 2 for FP64");
    }
    L.fused[dtype] = variant;
    drop_graphs(c);
    return CHEBMG_OK;
  });
}

int chebmg_batch_fused_smoother(chebmg_ctx* c, int nrhs, int level, int dtype, int* variant, int* rhs_per_item) {
  return guard([&]() -> int {
    enter(c);
    if (!variant || !rhs_per_item) throw Error(CHEBMG_EINVAL, "NULL argument");
    Level& L = level_checked(c, level);
    check_dtype(c, dtype);
    if (nrhs < 2 || nrhs > 65535) throw Error(CHEBMG_EINVAL, "batches have 2 to 65535 right-hand sides");
    reserve_batch(c, nrhs);
    autotune_batch(c, nrhs);
    *variant = L.fused_b[dtype];
    *rhs_per_item = L.fused_b[dtype] ? L.fused_gsz[dtype] : 0;
    return CHEBMG_OK;
  });
}

int chebmg_set_batch_fused_smoother(chebmg_ctx* c, int nrhs, int level, int dtype, int variant, int rhs_per_item) {
  return guard([&]() -> int {
    enter(c);
    Level& L = level_checked(c, level);
    check_dtype(c, dtype);
    if (nrhs < 2 || nrhs > 65535) throw Error(CHEBMG_EINVAL, "batches have 2 to 65535 right-hand sides");
    if (variant != 0) {
      if (!(L.type == TYPE_SEM && L.Q == 8 && L.boxed && L.fctl))
        throw Error(CHEBMG_EINVAL, "the fused smoother needs an order-7 box-lattice level that smooths");
      const bool ok = dtype == CHEBMG_F32 ? variant == 1 : variant == 2;
      if (!ok || rhs_per_item < 1 || rhs_per_item > 64)
        throw Error(CHEBMG_EINVAL, "fused smoother variant: 1 for FP32, 2 for FP64; 1 to 64 right-hand sides per item");
    }
    reserve_batch(c, nrhs);
    autotune_batch(c, nrhs);
    L.fused_b[dtype] = variant;
    if (variant != 0) L.fused_gsz[dtype] = rhs_per_item;
    drop_graphs(c);
    return CHEBMG_OK;
  });
}

int chebmg_convert(const void* in, int in_dtype, void* out, int out_dtype, int64_t n, void* stream) {
  return guard([&]() -> int {
    if (n < 0 || (n > 0 && (!in || !out))) throw Error(CHEBMG_EINVAL, "bad conversion arguments");
    if ((in_dtype != CHEBMG_F32 && in_dtype != CHEBMG_F64) || (out_dtype != CHEBMG_F32 && out_dtype != CHEBMG_F64))
      throw Error(CHEBMG_EINVAL, "dtype must be CHEBMG_F32 or CHEBMG_F64");
    if (n == 0) return CHEBMG_OK;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    if (in_dtype == CHEBMG_F32 && out_dtype == CHEBMG_F64)
      cast<float, double>(n, static_cast<const float*>(in), static_cast<double*>(out), s);
    else if (in_dtype == CHEBMG_F64 && out_dtype == CHEBMG_F32)
      cast<double, float>(n, static_cast<const double*>(in), static_cast<float*>(out), s);
    else if (in_dtype == CHEBMG_F32)
      cast<float, float>(n, static_cast<const float*>(in), static_cast<float*>(out), s);
    else
      cast<double, double>(n, static_cast<const double*>(in), static_cast<double*>(out), s);
    check_launch();
    return CHEBMG_OK;
  });
}

int chebmg_launch_count(const chebmg_ctx* c, int64_t* count) {
  (void)c;
  if (!count) return CHEBMG_EINVAL;
  *count = g_launches.load();
  return CHEBMG_OK;
}

int chebmg_set_outer_operator(chebmg_ctx* c, int kind) {
  return guard([&]() -> int {
    enter(c);
    if (kind == CHEBMG_OUTER_FP64) {
      c->outer_op = 0;
      drop_graphs(c);
      return CHEBMG_OK;
    }
    if (kind != CHEBMG_OUTER_F32X2) throw Error(CHEBMG_EINVAL, "bad outer operator kind");
    Level& L = c->L[0];
    if (L.type != TYPE_SEM || L.Q != 8) throw Error(CHEBMG_EINVAL, "FP32-pair operator needs an order-7 finest level");
    if (!c->G_x2) {
      c->G_x2 = dalloc<double>(c, L.E * 6 * 512);   // 8 bytes per value, like FP64
      sem_to_x2(L.E * 6 * 512, static_cast<const double*>(L.G[CHEBMG_F64]), c->G_x2, c->s);
      check_launch();
      // variant: 1, 2 or 4 elements per block (box lattice ids where available), timed
      double* x = vec<double>(L, VB);
      double* y = vec<double>(L, VY);
      splitmix_fill(L.n, 11ull, static_cast<const double*>(L.invD[CHEBMG_F64]), x, c->s);
      cudaEvent_t e0, e1;
      CK(cudaEventCreate(&e0));
      CK(cudaEventCreate(&e1));
      float best = 1e30f;
      for (int eb : {1, 2, 4}) {
        const int v = eb + (L.boxed ? 100 : 0);
        float t_min = 1e30f;
        for (int rep = 0; rep < 3; ++rep) {
          CK(cudaEventRecord(e0, c->s));
          sem_ax8_x2(L.E, L.gid, L.lat, c->G_x2, x, y, c->dstat, v, c->s);
          CK(cudaEventRecord(e1, c->s));
          CK(cudaEventSynchronize(e1));
          float ms = 0.f;
          CK(cudaEventElapsedTime(&ms, e0, e1));
          t_min = std::min(t_min, ms);
        }
        if (t_min < best) {
          best = t_min;
          c->eb_x2 = v;
        }
      }
      cudaEventDestroy(e0);
      cudaEventDestroy(e1);
      check_launch();
    }
    c->outer_op = 1;
    drop_graphs(c);
    return CHEBMG_OK;
  });
}

int chebmg_apply_outer(chebmg_ctx* c, const double* x, double* y) {
  return guard([&]() -> int {
    enter(c);
    if (!x || !y) throw Error(CHEBMG_EINVAL, "NULL vector");
    zero<double>(c, y, c->L[0].n);
    apply_outer(c, x, y);
    CK(cudaStreamSynchronize(c->s));
    return CHEBMG_OK;
  });
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
    const PdlScope pdl_(c->nb == 1);
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
    const PdlScope pdl_(c->nb == 1);
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
    const PdlScope pdl_(c->nb == 1);   // the solve's kernels launch as programmatic dependents
    if (!b || !u || maxit < 0 || !(rtol > 0.0)) throw Error(CHEBMG_EINVAL, "bad solve arguments");
    Level& L = c->L[0];
    const int64_t n = L.n;
    const double* S = static_cast<const double*>(L.invD[CHEBMG_F64]);
    double *r = c->kr, *z = c->kz, *p = c->kp, *q = c->kq;
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
    // Mixed form: the V-cycle reads an FP32 copy of r, written by the x/r update, and its FP32
    // output z32 feeds the dots and the p update directly (no FP64 copy of z).  The flexible
    // (Polak-Ribiere) beta uses r_new - r_old = -alpha A p, so no copy of r_old is kept.
    const bool mixed = c->fp32 && c->L.size() > 1;
    float* r32 = mixed ? vec<float>(L, VB) : nullptr;
    float* z32 = mixed ? vec<float>(L, VX) : nullptr;
    auto precondition = [&](bool r32_ready) -> int {
      if (!mixed) return vcycle_top(c, r, z);
      if (!r32_ready) cast<double, float>(n, r, r32, c->s);
      return vcycle_level<float>(c, 0, r32, z32);
    };
    int rc = precondition(false);
    if (rc != CHEBMG_OK && rc != CHEBMG_ENOTCONV) return rc;
    // the p updates also zero q, which the next product accumulates into
    if (mixed) {
      update_p_from<float>(n, z32, p, c->scal, true, c->s, q);
      dot_zr_zq<float>(n, z32, r, nullptr, POST_SET_RZ_FROM_ZR, c->partial, c->scal, c->s);
    } else {
      update_p_from<double>(n, z, p, c->scal, true, c->s, q);
      dot_zr_zq<double>(n, z, r, nullptr, POST_SET_RZ_FROM_ZR, c->partial, c->scal, c->s);
    }
    double rel = 1.0;
    for (int it = 1; it <= maxit; ++it) {
      apply_outer(c, p, q);
      dot2(n, p, q, nullptr, nullptr, S_PQ, -1, POST_ALPHA, c->partial, c->scal, c->s);
      fcg_update_xr32(n, u, r, r32, p, q, c->partial, c->scal, c->s);
      read_scal(c);
      const double pq = c->hscal[S_PQ], rr = c->hscal[S_RR];
      const int crc = coarse_sticky_error(c);
      if (crc != CHEBMG_OK) {
        if (iters) *iters = it;
        if (crc == CHEBMG_ETIMEOUT) {   // the iterate may hold the output of an unfinished kernel
          zero<double>(c, u, n);
          CK(cudaStreamSynchronize(c->s));
          if (relres) *relres = std::numeric_limits<double>::quiet_NaN();
        }
        g_last_error = crc == CHEBMG_ETIMEOUT ? "a bounded device wait ran out inside the solve; u discarded"
                                              : "coarse solve inside the V-cycle failed";
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
      rc = precondition(true);
      if (rc != CHEBMG_OK && rc != CHEBMG_ENOTCONV) return rc;
      if (mixed) {
        dot_zr_zq<float>(n, z32, r, q, POST_BETA_FLEX_Q, c->partial, c->scal, c->s);
        update_p_from<float>(n, z32, p, c->scal, false, c->s, q);
      } else {
        dot_zr_zq<double>(n, z, r, q, POST_BETA_FLEX_Q, c->partial, c->scal, c->s);
        update_p_from<double>(n, z, p, c->scal, false, c->s, q);
      }
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

int chebmg_pcg_solve_batched(chebmg_ctx* c, int nrhs, const double* B, double* U, double rtol, int maxit,
                             int flags, int* iters, double* relres) {
  return guard([&]() -> int {
    enter(c);
    if (!B || !U || nrhs < 1 || nrhs > 65535 || maxit < 0 || !(rtol > 0.0) || (flags & ~CHEBMG_BATCH_GRAPH))
      throw Error(CHEBMG_EINVAL, "bad batched solve arguments");
    const int64_t n = c->L[0].n;
    return pcg_batched(c, nrhs, B, n, U, n, rtol, maxit, iters, relres, (flags & CHEBMG_BATCH_GRAPH) != 0);
  });
}

int chebmg_apply_A_batched(chebmg_ctx* c, int level, int dtype, int nrhs, const void* X, void* Y) {
  return guard([&]() -> int {
    enter(c);
    Level& L = level_checked(c, level);
    check_dtype(c, dtype);
    if (!X || !Y || nrhs < 1 || nrhs > 65535) throw Error(CHEBMG_EINVAL, "bad batched apply arguments");
    if (dtype == CHEBMG_F32 && !L.G[CHEBMG_F32] && L.type == TYPE_SEM)
      throw Error(CHEBMG_EINVAL, "no FP32 data on this level");
    if (nrhs > 1) {
      reserve_batch(c, nrhs);
      autotune_batch(c, nrhs);
    }
    const size_t es = dtype == CHEBMG_F64 ? 8 : 4;
    CK(cudaMemsetAsync(Y, 0, es * (size_t)nrhs * L.n, c->s));
    if (dtype == CHEBMG_F64)
      apply_into_ld<double>(c, level, static_cast<const double*>(X), static_cast<double*>(Y), nrhs, L.n);
    else
      apply_into_ld<float>(c, level, static_cast<const float*>(X), static_cast<float*>(Y), nrhs, L.n);
    return CHEBMG_OK;
  });
}

int chebmg_vcycle_batched(chebmg_ctx* c, int nrhs, const double* R, double* Z) {
  return guard([&]() -> int {
    enter(c);
    if (!R || !Z || nrhs < 1 || nrhs > 65535) throw Error(CHEBMG_EINVAL, "bad batched V-cycle arguments");
    reserve_batch(c, nrhs);
    autotune_batch(c, nrhs);
    Level& L = c->L[0];
    BatchScope bs(c, nrhs);
    CK(cudaMemsetAsync(c->dstat, 0, sizeof(unsigned) * 2, c->s));
    cast<double, double>(L.n, R, c->kr, c->s, nrhs, L.n, L.ld);
    int rc = vcycle_top(c, c->kr, c->kz);
    cast<double, double>(L.n, c->kz, Z, c->s, nrhs, L.ld, L.n);
    check_launch();
    CK(cudaMemcpyAsync(c->hdstat, c->dstat, sizeof(unsigned) * 4, cudaMemcpyDeviceToHost, c->s));
    CK(cudaStreamSynchronize(c->s));
    if (c->hdstat[0]) return CHEBMG_ETIMEOUT;
    if (c->hdstat[1] == CS_BREAKDOWN) return CHEBMG_EBREAKDOWN;
    return rc == CHEBMG_ENOTCONV ? CHEBMG_OK : rc;
  });
}

int chebmg_cycle_error_grad(chebmg_ctx* c, int nrhs, const double* E0, int steps, const double* betas,
                            int nbeta, double lmax_scale, double* f, double* grad_betas, double* grad_scale,
                            double* f_each) {
  return guard([&]() -> int {
    enter(c);
    if (!E0 || !betas || !f || (!grad_betas) != (!grad_scale) || nrhs < 1 || nrhs > 65535 || steps < 1 ||
        steps > 64 || nbeta < 1 || nbeta > 64 || !(lmax_scale > 0.0))
      throw Error(CHEBMG_EINVAL, "bad gradient arguments");
    return cycle_error_grad(c, nrhs, E0, steps, betas, nbeta, lmax_scale, f, grad_betas, grad_scale, f_each);
  });
}

int chebmg_set_smoother_weights(chebmg_ctx* c, const double* betas, int nbeta, double lmax_scale) {
  return guard([&]() -> int {
    enter(c);
    if (nbeta < 0 || nbeta > 64 || (nbeta > 0 && !betas) || !(lmax_scale > 0.0))
      throw Error(CHEBMG_EINVAL, "bad smoother weights");
    if (nbeta > 0 && c->o.kind == CHEBMG_CHEB_1ST) throw Error(CHEBMG_EINVAL, "weights need the 4th kind");
    c->beta_ovr.assign(betas, betas + nbeta);
    c->lscale = lmax_scale;
    drop_graphs(c);
    return CHEBMG_OK;
  });
}

int chebmg_batch_info(chebmg_ctx* c, int nrhs, int level, int dtype, int* variant, int* coarse_degree) {
  return guard([&]() -> int {
    enter(c);
    Level& L = level_checked(c, level);
    check_dtype(c, dtype);
    if (!variant || !coarse_degree || nrhs < 1 || nrhs > 65535) throw Error(CHEBMG_EINVAL, "bad arguments");
    reserve_batch(c, nrhs);
    autotune_batch(c, nrhs);
    *variant = (L.type == TYPE_SEM && L.Q == 8 && nrhs > 1) ? L.beb[dtype] : 0;
    *coarse_degree = (c->ell_col && coarse_block_supported(c->L.back().n)) ? c->bcoarse_degree : 0;
    return CHEBMG_OK;
  });
}

int chebmg_set_batch_tile_choice(chebmg_ctx* c, int nrhs, int level, int dtype, int variant) {
  return guard([&]() -> int {
    enter(c);
    Level& L = level_checked(c, level);
    check_dtype(c, dtype);
    if (L.type != TYPE_SEM || L.Q != 8 || nrhs < 2 || nrhs > 65535) throw Error(CHEBMG_EINVAL, "no batched variant");
    const int rb = variant / 1000, rest = variant % 1000, eb = rest % 100;
    const bool paired = eb == 11 || eb == 12, in_regs = eb == 21 || eb == 22;
    if (rb < 1 || rb > 64 || (rest != eb && rest != eb + 100) ||
        (eb != 1 && eb != 2 && eb != 4 && !paired && !in_regs) || (paired && rb < 2))
      throw Error(CHEBMG_EINVAL, "bad batched variant");
    const bool fits = dtype == CHEBMG_F64 ? sem_ax8_batched_fits<double>(variant) : sem_ax8_batched_fits<float>(variant);
    if (!fits || (dtype == CHEBMG_F32 && !L.G[CHEBMG_F32]) || (rest >= 100 && !L.boxed))
      throw Error(CHEBMG_EINVAL, "variant not available");
    reserve_batch(c, nrhs);
    autotune_batch(c, nrhs);
    L.beb[dtype] = variant;
    drop_graphs(c);
    return CHEBMG_OK;
  });
}

int chebmg_group_create(chebmg_ctx* const* ctxs, int nctx, chebmg_group** out) {
  return guard([&]() -> int {
    if (!out) throw Error(CHEBMG_EINVAL, "group output is NULL");
    *out = nullptr;
    if (!ctxs || nctx < 1) throw Error(CHEBMG_EINVAL, "no contexts");
    for (int k = 0; k < nctx; ++k) {
      if (!ctxs[k]) throw Error(CHEBMG_EINVAL, "NULL context");
      if (ctxs[k]->dev != ctxs[0]->dev) throw Error(CHEBMG_EINVAL, "contexts on different devices");
      for (int q = 0; q < k; ++q)
        if (ctxs[q] == ctxs[k]) throw Error(CHEBMG_EINVAL, "a context appears twice");
    }
    CK(cudaSetDevice(ctxs[0]->dev));
    chebmg_group* g = new chebmg_group();
    g->dev = ctxs[0]->dev;
    g->c.assign(ctxs, ctxs + nctx);
    g->join.assign(nctx, nullptr);
    cudaError_t e = cudaStreamCreateWithFlags(&g->s, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&g->fork, cudaEventDisableTiming);
    for (int k = 0; k < nctx && e == cudaSuccess; ++k) e = cudaEventCreateWithFlags(&g->join[k], cudaEventDisableTiming);
    if (e != cudaSuccess) {
      chebmg_group_destroy(g);
      throw Error(CHEBMG_ECUDA, std::string("group resources: ") + cudaGetErrorString(e));
    }
    *out = g;
    return CHEBMG_OK;
  });
}

int chebmg_group_pcg_solve(chebmg_group* g, const double* const* B, double* const* U, double rtol, int maxit,
                           int flags, int* iters, double* relres) {
  return guard([&]() -> int {
    if (!g || !B || !U || maxit < 0 || !(rtol > 0.0) || (flags & ~CHEBMG_BATCH_GRAPH))
      throw Error(CHEBMG_EINVAL, "bad group solve arguments");
    for (size_t k = 0; k < g->c.size(); ++k)
      if (!B[k] || !U[k]) throw Error(CHEBMG_EINVAL, "NULL vector");
    CK(cudaSetDevice(g->dev));
    return group_solve(g, B, U, rtol, maxit, (flags & CHEBMG_BATCH_GRAPH) != 0, iters, relres);
  });
}

void chebmg_group_destroy(chebmg_group* g) {
  if (!g) return;
  cudaSetDevice(g->dev);
  if (g->s) cudaStreamSynchronize(g->s);
  group_drop(g);
  for (cudaEvent_t e : g->join)
    if (e) cudaEventDestroy(e);
  if (g->fork) cudaEventDestroy(g->fork);
  if (g->s) cudaStreamDestroy(g->s);
  delete g;
}

int chebmg_gmres_solve(chebmg_ctx* c, const double* b, double* u, double rtol, int restart, int maxit, int* iters,
                       double* relres, double* history) {
  return guard([&]() -> int {
    enter(c);
    if (!b || !u || maxit < 0 || !(rtol > 0.0) || restart < 1 || restart + 1 > gmres_max_basis())
      throw Error(CHEBMG_EINVAL, "bad GMRES arguments");
    const PdlScope pdl_(c->nb == 1);
    return gmres_solve(c, b, u, rtol, restart, maxit, iters, relres, history);
  });
}

int chebmg_selftest_coarse_timeout(chebmg_ctx* c, int* status) {
  return guard([&]() -> int {
    enter(c);
    if (!status) throw Error(CHEBMG_EINVAL, "status is NULL");
    if (!c->cctl || !c->coop_ok) throw Error(CHEBMG_EINVAL, "no persistent coarse solver in this context");
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
