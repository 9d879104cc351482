// Internal declarations shared by the CUDA translation units of libchebmg.
#pragma once
#include <cuda_runtime.h>

#include <atomic>
#include <cstdint>

#include "setup_host.h"

namespace chebmg {

// Number of kernel launches issued by this library in this process.
extern std::atomic<int64_t> g_launches;

// Programmatic dependent launch.  While g_pdl is set on the calling host thread (single
// right-hand-side solves, V-cycles and smoother applications set it while they enqueue), the
// kernels of the solve path are launched as programmatic dependents of the kernel before them
// in the stream: their blocks may be scheduled while that kernel drains, and each of them
// executes pdl_wait() -- which returns once the preceding grid has completed and its memory
// operations are visible -- before its first global memory access.  Launches into a stream
// that is being captured are ordinary launches.
extern thread_local bool g_pdl;
struct PdlScope {
  bool old;
  explicit PdlScope(bool on) : old(g_pdl) { g_pdl = on; }
  ~PdlScope() { g_pdl = old; }
  PdlScope(const PdlScope&) = delete;
  PdlScope& operator=(const PdlScope&) = delete;
};
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
inline bool pdl_on(cudaStream_t s) {
  if (!g_pdl) return false;
  cudaStreamCaptureStatus st = cudaStreamCaptureStatusNone;
  return cudaStreamIsCapturing(s, &st) == cudaSuccess && st == cudaStreamCaptureStatusNone;
}
// Launches kernel k (which must begin with pdl_wait()) as a programmatic dependent when
// pdl_on(s), else as an ordinary launch; counts the launch.
template <typename... KArgs, typename... Args>
inline void launch_dep(void (*k)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t s, Args&&... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cudaLaunchAttribute attr;
  attr.id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr.val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = &attr;
  cfg.numAttrs = pdl_on(s) ? 1 : 0;
  cudaLaunchKernelEx(&cfg, k, static_cast<Args&&>(args)...);
  g_launches.fetch_add(1, std::memory_order_relaxed);
}

// Scalar slots of the device-side reduction buffer (FP64).
enum Slot {
  S_RZ = 0,      // (r, z) of the current Krylov iteration
  S_PQ,          // (p, A p)
  S_RR,          // (r, r)
  S_ZR,          // (z_new, r_new)
  S_ZRO,         // (z_new, r_old)
  S_BB,          // (b, b)
  S_ALPHA,
  S_BETA,
  S_T0,          // scratch
  S_T1,
  S_ZQ,          // (z_new, q) with q = A p of the same iteration
  S_NSLOTS
};
enum PostOp { POST_NONE = 0, POST_ALPHA, POST_BETA_CG, POST_SET_RZ_FROM_ZR, POST_BETA_FLEX_Q };

constexpr int kRedBlocks = 1216;   // 152 SMs x 8: partial sums per reduction pass (full occupancy)

template <typename T>
struct Stencil9 {
  T c[9];
};

// p[0 .. bytes) = 0 by a kernel (programmatic dependent launch when g_pdl is set; 16-byte
// aligned p), else by a memset.
void zero_bytes(void* p, int64_t bytes, cudaStream_t s);

// ---- SEM kernels (y must be zeroed by the caller; results accumulate) ----
// Every operator, transfer and vector kernel also runs on a batch of nb right-hand sides:
// vector b of the batch starts at offset b * ld (ld = 0 means n; per-node data shared).
template <typename T>
void sem_ax(int Q, int64_t E, const uint32_t* gid, const T* G, const T* D, const T* u, T* y,
            cudaStream_t s, int nb = 1, int64_t ld = 0);
template <typename T>
void sem_restrict(int Qf, int Qc, int64_t E, const uint32_t* gidf, const uint32_t* gidc,
                  const T* J, const T* rf, T* rc, cudaStream_t s, int nb = 1, int64_t ldf = 0, int64_t ldc = 0);
template <typename T>
void sem_prolong(int Qf, int Qc, int64_t E, const uint32_t* gidf, const uint32_t* gidc,
                 const T* J, const T* zc, T* zf, int accumulate, cudaStream_t s, int nb = 1, int64_t ldf = 0,
                 int64_t ldc = 0);

// Order-7 element operator (line passes, even-odd D, TMA-staged geometric factors).
// sem_ax8_set_D uploads the even-odd blocks of the 8x8 GLL derivative matrix (row-major).
cudaError_t sem_ax8_set_D(const double* D);
// Box lattice of a level (element counts and global node counts per direction).
struct Lattice {
  int nex, ney, nez;
  int NX, NY, NZ;
};
// Order-3 element operator by line passes (16 threads per element, no block barrier): as
// sem_ax for Q = 4; ids from the box lattice when lat is given, else from gid.
template <typename T>
void sem_ax4(int64_t E, const uint32_t* gid, const Lattice* lat, const T* G, const T* D, const T* u, T* y,
             cudaStream_t s, int nb = 1, int64_t ld = 0);
// The order-7 operator in FP64-class arithmetic on FP32 pairs (sem_ax8_x2.cu): G in that
// format (sem_to_x2 converts an FP64 array of n values), u and y FP64; variant as sem_ax8's
// non-persistent codes (1, 2, 4; +100 box lattice ids); batches of nb vectors at stride ld,
// rb of them per thread block (the factors staged once per block).
cudaError_t sem_ax8_x2_set_eo(const double* eo_blocks);   // [4][4][4], as uploaded by sem_ax8_set_D
void sem_to_x2(int64_t n, const double* in, void* out, cudaStream_t s);
void sem_ax8_x2(int64_t E, const uint32_t* gid, const Lattice& lat, const void* G, const double* u, double* y,
                unsigned* err, int variant, cudaStream_t s, int nb = 1, int64_t ld = 0, int rb = 1);
// variant chosen per level by a setup-time autotuner: 1, 2 or 4 elements per thread block,
// or 12 / 14 for the persistent software-pipelined kernel with 2 / 4 elements, 31 / 32 for that
// kernel with 1 / 2 elements and a single geometric-factor buffer, 21 / 22 for factors read
// where used; +100 computes global ids from the box lattice instead of reading the
// element-to-global map.  Programmatic dependent launch (g_pdl) on every single-vector variant;
// the persistent ones start their first geometric-factor copy before pdl_wait().
template <typename T>
void sem_ax8(int64_t E, const uint32_t* gid, const Lattice& lat, const T* G, const T* u, T* y,
             unsigned* err, int variant, cudaStream_t s);
// Batched form: nb right-hand sides at leading dimension ld.  variant = 1000 * RB + (100 if
// implicit ids) + EB: a block stages the geometric factors of EB elements once and applies them
// to RB right-hand sides; EB + 10 (EB 1 or 2) takes the right-hand sides two at a time through
// each line pass (RB at least 2); EB + 20 (EB 1 or 2) keeps the factors in registers instead.
template <typename T>
void sem_ax8_batched(int64_t E, const uint32_t* gid, const Lattice& lat, const T* G, const T* u, T* y,
                     unsigned* err, int variant, int nb, int64_t ld, cudaStream_t s);
// Whether variant `eb` fits the device's per-block shared-memory limit.
template <typename T>
bool sem_ax8_variant_fits(int eb);
// The same for a batched variant code.
template <typename T>
bool sem_ax8_batched_fits(int variant);

// ---- fused smoother on an order-7 box-lattice level (sem_smooth8.cu) ----
// One persistent launch runs a sequence of phases; a phase is an optional element operator
// application y += A v (v = d or x, Sec. 1 Eq. 1.3) followed by one pointwise operation over all
// nodes that reads and zeroes y.  The pointwise operations are those of the vector kernels below,
// with the same arithmetic.
enum FusedOp {
  FOP_ZERO_Y = 0,     // y = 0
  FOP_CHEB4_INIT_B,   // x = 0, r = b, d = c0 S r, y = 0                      (Algorithm 2, x0 = 0)
  FOP_CHEB4_INIT_BY,  // r = b - y, d = c0 S r, y = 0                         (Algorithm 2, y = A x0)
  FOP_CHEB4_STEP,     // x += c0 d; r -= y; d = c1 d + c2 S r; y = 0; x += c3 d  (c3 = 0 except last)
  FOP_CHEB1_INIT_B,   // x = 0, r = S b, d = c0 r, y = 0                      (Algorithm 1, x0 = 0)
  FOP_CHEB1_INIT_BY,  // r = S (b - y), d = c0 r, y = 0                       (Algorithm 1, y = A x0)
  FOP_CHEB1_STEP,     // x += d; r -= S y; d = c1 d + c2 r; y = 0; x += c3 d      (c3 = 0 except last)
  FOP_AXPY,           // x += c0 d
  FOP_RESIDUAL        // r = b - y, y = 0                                      (restriction residual)
};
enum FusedSrc { FSRC_NONE = 0, FSRC_D = 1, FSRC_X = 2 };
struct FusedPhase {
  int op;             // FusedOp
  int src;            // FusedSrc: the vector the phase's operator application reads
  double c[4];
};
constexpr int kFusedMaxPhases = 24;
constexpr int kFusedMaxT = 700;   // queue steps: 3 (phases - 1) + element planes + 1 at most
struct FusedSmooth {
  int64_t E, n;
  Lattice lat;
  int nphase;
  FusedPhase ph[kFusedMaxPhases];
  const void *G, *S, *b;
  void *x, *r, *d, *y;
  unsigned* ctl;      // fused_ctl_words(lat) words, zeroed by the launcher
  unsigned* err;      // set to 1 when a bounded wait runs out
  int nb;             // right-hand sides: vector q of x, r, d, y, b at q * ld (S shared)
  int64_t ld;
  int gsz;            // right-hand sides per work item
  // derived by fused_plan
  int nslab;          // element planes (slabs)
  int spp;            // elements per slab
  int ngroups;        // right-hand-side groups: item k of a task covers group k % ngroups
  int m1, m2;         // work items per operator task / per pointwise task
  int chunk;          // nodes per pointwise work item
  int tsteps;
  uint32_t total;
  uint32_t toff[kFusedMaxT + 1];
};
// Variants: 1 = FP32, 2 elements per work item; 2 = FP64, 1 element per work item.
int fused_ctl_words(const Lattice& lat);
// Fills the derived fields; false if the level or the program is beyond the kernel's limits
// (the caller then runs the separate kernels).
bool fused_plan(FusedSmooth& a, int variant);
// Launches the fused kernel (cooperative); false, with nothing launched, if that is impossible.
template <typename T>
bool sem_smooth8(FusedSmooth& a, int variant, cudaStream_t s);
cudaError_t sem_smooth8_set_eo(const double* eo_blocks);   // [4][4][4], as for sem_ax8_x2_set_eo

// p-multigrid transfers on the box lattice for the order pairs (7,3), (3,1), (7,5), (5,3)
// (Q 8->4, 4->2, 8->6, 6->4).
cudaError_t transfer_box_set_J(int Qf, int Qc, const double* J);
bool transfer_box_supported(int Qf, int Qc);
template <typename T>
void restrict_box(int Qf, int Qc, int64_t E, const Lattice& Lf, const Lattice& Lc, const T* rf, T* rc,
                  cudaStream_t s, int nb = 1, int64_t ldf = 0, int64_t ldc = 0);
template <typename T>
void prolong_box(int Qf, int Qc, int64_t E, const Lattice& Lf, const Lattice& Lc, const T* zc, T* zf,
                 int accumulate, cudaStream_t s, int nb = 1, int64_t ldf = 0, int64_t ldc = 0);

// ---- FD kernels ----
template <typename T>
void fd_apply(int mx, int my, const Stencil9<T>& st, const T* u, T* y, cudaStream_t s, int nb = 1,
              int64_t ld = 0);
template <typename T>
void fd_restrict(int mfx, int mfy, int mcx, int mcy, int c, const T* rf, T* rc, cudaStream_t s, int nb = 1,
                 int64_t ldf = 0, int64_t ldc = 0);
template <typename T>
void fd_prolong(int mfx, int mfy, int mcx, int mcy, int c, const T* zc, T* zf, int accumulate,
                cudaStream_t s, int nb = 1, int64_t ldf = 0, int64_t ldc = 0);
void dense_matvec(int n, const double* M, const double* x, double* y, cudaStream_t s, int nb = 1, int64_t ld = 0);

// ---- Chebyshev recurrences (Algorithms 1 and 2), elementwise over n ----
// 4th kind init: x_is_zero 1: x = 0, r = b; 0: r = b - y, y = 0; then d = c0 S r.  x_is_zero 2:
// d = c0 S b only (x = 0 and r = b are left to the first cheb4_step, given b_first = b).
template <typename T>
void cheb4_init(int64_t n, const T* b, T* x, T* r, T* d, T* y, const T* invD, double c0,
                int x_is_zero, cudaStream_t s, int nb = 1, int64_t ld = 0);
// 4th kind step: x += beta d; r -= y; d = c1 d + c2 S r; y = 0; then, if beta_next != 0 (the
// last step), the final update x += beta_next d with the new d.  b_first: the first step from
// x = 0 after cheb4_init with x_is_zero = 2 (d only): r = b_first - y and x = beta d.
template <typename T>
void cheb4_step(int64_t n, T* x, T* r, T* d, T* y, const T* invD, double beta, double c1,
                double c2, cudaStream_t s, int nb = 1, int64_t ld = 0, double beta_next = 0.0,
                const T* b_first = nullptr);
// 1st kind init: r = S (b - y) (or S b), d = r / theta, y = 0 (x = 0 if x_is_zero).
template <typename T>
void cheb1_init(int64_t n, const T* b, T* x, T* r, T* d, T* y, const T* invD, double inv_theta,
                int x_is_zero, cudaStream_t s, int nb = 1, int64_t ld = 0);
// 1st kind step: x += d; r -= S y; d = c1 d + c2 r; y = 0.
template <typename T>
void cheb1_step(int64_t n, T* x, T* r, T* d, T* y, const T* invD, double c1, double c2,
                cudaStream_t s, int nb = 1, int64_t ld = 0);
// x += a * d
template <typename T>
void axpy(int64_t n, double a, const T* d, T* x, cudaStream_t s, int nb = 1, int64_t ld = 0);
// r = b - y; y = 0
template <typename T>
void residual(int64_t n, const T* b, T* y, T* r, cudaStream_t s, int nb = 1, int64_t ld = 0);
// Batched forms: nb vectors at leading dimension ld (0 = n); per-node data (S) shared.
template <typename Tin, typename Tout>
void cast(int64_t n, const Tin* in, Tout* out, cudaStream_t s, int nb = 1, int64_t ldi = 0, int64_t ldo = 0);
// out = mask(invD) ? in : 0   (mask: invD != 0)
void masked_copy(int64_t n, const double* in, const double* invD, double* out, cudaStream_t s, int nb = 1,
                 int64_t ldi = 0, int64_t ldo = 0);

// ---- FP64 reductions into scal[slot] (deterministic two-pass) ----
// out slots: scal[slot0] = (a0, b0), scal[slot1] = (a1, b1) if a1 != nullptr; then post-op.
void dot2(int64_t n, const double* a0, const double* b0, const double* a1, const double* b1,
          int slot0, int slot1, int post, double* partial, double* scal, cudaStream_t s);

// ---- Krylov vector updates with device scalars ----
// p = z + scal[BETA] p
void update_p(int64_t n, const double* z, double* p, const double* scal, cudaStream_t s);
// The flexible CG loop's fused forms.  FCG: x += alpha p; r -= alpha q; partial (r, r) ->
// scal[RR]; r32 (if not NULL) = FP32 copy of the new r (the V-cycle's right-hand side).
void fcg_update_xr32(int64_t n, double* x, double* r, float* r32, const double* p, const double* q,
                     double* partial, double* scal, cudaStream_t s);
// scal[ZR] = (z, r), scal[ZQ] = (z, q), then post (z in FP32 or FP64)
template <typename Tz>
void dot_zr_zq(int64_t n, const Tz* z, const double* r, const double* q, int post, double* partial, double* scal,
               cudaStream_t s);
// p = z + scal[BETA] p, or p = z (first); q_zero, if given, is set to 0 in the same pass
template <typename Tz>
void update_p_from(int64_t n, const Tz* z, double* p, const double* scal, bool first, cudaStream_t s,
                   double* q_zero = nullptr);
// CG (coarse): x += alpha p; r -= alpha q; z = S r; partials (r, r) and (r, z)
void cg_update(int64_t n, double* x, double* r, double* z, const double* p, const double* q,
               const double* invD, double* partial, double* scal, cudaStream_t s);

// ---- persistent coarse solve (one cooperative launch per solve) ----
// Control words: ctl[0] reduction arrivals (monotonic within a launch), ctl[1] unused, ctl[2]
// status of the last solve, ctl[3] its iterations, ctl[4] sticky worst error since the caller
// reset it.
enum CoarseStatus { CS_NONE = 0, CS_OK = 1, CS_NOTCONV = 2, CS_BREAKDOWN = 3, CS_TIMEOUT = 4 };
struct CoarseCG {
  int64_t n;
  int nslot;
  const int* col;        // ELL, slot-major
  const double* val;
  const double* invD;
  const double* b;
  double* x;
  int rows_per_block;    // block q owns rows [q * rows_per_block, (q + 1) * rows_per_block)
  double* part;          // [2][3 * gridDim] block partials, double-buffered by reduction parity
  unsigned* ctl;         // [5], ctl[0] (monotonic arrival counter) zero at launch
  double rtol;
  int maxit;
  int degree;            // degree of the 4th-kind Chebyshev preconditioner (1 = Jacobi)
  double lmax;           // lambda_max of S A on the coarse level
  unsigned phantom_blocks;   // self-test only: barrier also waits for this many blocks that never come
  // preconditioner in FP32 (pf32 != 0): the polynomial's products, recurrence and exchanges
  // run on FP32 copies; the CG itself (iterate, residual, products A p, dots) stays FP64 and
  // takes the flexible (Polak-Ribiere) beta, since rounded FP32 arithmetic makes the
  // preconditioner slightly non-symmetric.
  int pf32;
  const float* valf;     // ELL values, FP32
  const float* invDf;    // Jacobi diagonal, FP32
  // Box lattice (lat_nx > 0): 27 slots in lattice order, slot k of row g the entry for column
  // g + (k / 9 - 1) lat_nxy + ((k / 3) % 3 - 1) lat_nx + (k % 3 - 1), so no column indices are
  // read; rows with a zero Jacobi entry (the lattice boundary) are skipped.
  int lat_nx, lat_nxy;
  // Products exchange the vector they read through tagged words: each value travels with its
  // exchange tag in one 64-bit word (single-copy atomic; FP64 values as two such words), so a
  // reader needs no flag and no fence -- it reloads the words whose tag is not there yet.
  // Buffers alternate with the parity of the kernel's exchange counter; the tags of one launch
  // are gen0 + 1, gen0 + 2, ..., and the host moves gen0 past every tag a launch can use, so
  // words left by an earlier launch never match.
  unsigned long long* exf[2];   // [n] FP32 values
  unsigned long long* exd[2];   // [2 n] FP64 values
  unsigned gen0;
};
// Step coefficients of the coarse CG's polynomial preconditioner (Algorithm 2, beta = 1):
// step i (1 <= i < degree) updates d = c1[i] d + c2[i] S r.  The coarse kernels fill this table
// once per launch, one thread per entry, instead of dividing in every thread at every step:
// FP64 runs at a small fraction of the FP32 rate on this GPU, and a block-wide FP64 division
// costs about as much as a short product.
constexpr int kCoarseMaxDegree = 64;
struct CoarseCoef {
  double c1[kCoarseMaxDegree], c2[kCoarseMaxDegree];
  float c1f[kCoarseMaxDegree], c2f[kCoarseMaxDegree];
};
#ifdef __CUDACC__
__device__ __forceinline__ void coarse_coef_fill(CoarseCoef& t, int degree, double lmax) {
  for (int i = threadIdx.x; i < degree && i < kCoarseMaxDegree; i += blockDim.x) {
    const double c1 = (2.0 * i - 1.0) / (2.0 * i + 3.0), c2 = (8.0 * i + 4.0) / ((2.0 * i + 3.0) * lmax);
    t.c1[i] = c1;
    t.c2[i] = c2;
    t.c1f[i] = (float)c1;
    t.c2f[i] = (float)c2;
  }
}
// num / den divided by one thread and shared with the block through *slot.  The caller must
// not write *slot again before a later block barrier.
__device__ __forceinline__ double block_div(double* slot, double num, double den) {
  if (threadIdx.x == 0) *slot = num / den;
  __syncthreads();
  return *slot;
}
#endif

// Conversions between FP32 and FP64 in integer arithmetic.  GB300 issues FP64 instructions --
// the hardware conversions F2F included -- at a small fraction of its FP32 and integer rates, so
// the FP64 vector kernels of the Krylov loop, which convert every FP32 value they touch, are
// bound by the FP64 pipe.  These give the hardware conversion's exact result: widening re-biases
// the exponent and shifts the mantissa (exact for every finite float); narrowing rounds the
// 52-bit mantissa to 23 bits to nearest, ties to even, a carry running into the exponent (and to
// infinity above the largest float).  Values outside the normal range (zeros and subnormals on
// the float side, infinities and NaN) take the hardware conversion.
#ifdef __CUDACC__
__device__ __forceinline__ double widen_f32(float v) {
  const uint32_t u = __float_as_uint(v);
  const uint32_t e = (u >> 23) & 0xffu;
  if (e == 0u || e == 0xffu) return (double)v;
  const uint32_t hi = (u & 0x80000000u) | ((e + 896u) << 20) | ((u & 0x7fffffu) >> 3);
  return __hiloint2double((int)hi, (int)(u << 29));
}
__device__ __forceinline__ float narrow_f64(double v) {
  const unsigned long long u = (unsigned long long)__double_as_longlong(v);
  const uint32_t e = (uint32_t)(u >> 52) & 0x7ffu;
  if (e < 897u || e > 1150u) return (float)v;
  const unsigned long long m = u & 0xfffffffffffffull;
  uint32_t f = ((e - 896u) << 23) | (uint32_t)(m >> 29);
  const unsigned long long rem = m & 0x1fffffffull;
  f += (rem > 0x10000000ull || (rem == 0x10000000ull && (f & 1u))) ? 1u : 0u;
  return __uint_as_float(f | ((uint32_t)(u >> 32) & 0x80000000u));
}
__device__ __forceinline__ double to_f64(float v) { return widen_f32(v); }
__device__ __forceinline__ double to_f64(double v) { return v; }
template <typename Tout>
__device__ __forceinline__ Tout convert_to(float v);
template <typename Tout>
__device__ __forceinline__ Tout convert_to(double v);
template <>
__device__ __forceinline__ double convert_to<double>(float v) { return widen_f32(v); }
template <>
__device__ __forceinline__ float convert_to<float>(double v) { return narrow_f64(v); }
template <>
__device__ __forceinline__ float convert_to<float>(float v) { return v; }
template <>
__device__ __forceinline__ double convert_to<double>(double v) { return v; }
#endif

// Rows per thread the persistent coarse kernel can keep in registers.
constexpr int kCoarseMaxRowsPerThread = 8;
constexpr int kCoarseThreadsPerBlock = 256;
// Returns false (nothing launched) if a cooperative launch is not possible.
bool coarse_pcg_launch(const CoarseCG& a, int grid, cudaStream_t s, cudaError_t* err);
// Grid size (blocks) and rows per block for a coarse problem of n rows, at least rpt_min rows
// per thread (a power of two up to kCoarseMaxRowsPerThread); grid 0 = not possible.
void coarse_pcg_shape(int64_t n, int rpt_min, int* grid, int* rows_per_block);

// ---- coarse CG on one thread-block cluster (coarse_cluster.cu; box lattice at N = 1) ----
// Forward half of the 27-point lattice stencil, slot k -> offset (dx, dy, dz): slot 0 the
// diagonal, 1-4 the in-plane neighbours (1,0), (-1,1), (0,1), (1,1), 5-13 the plane above
// with (dx, dy) in {-1,0,1}^2, dx fastest.  The other half is the mirror image: A is
// symmetric, so entry (i, i - o) is stored as entry (i - o, i) in row i - o.
__host__ __device__ constexpr int cc_dx(int k) {
  return k == 0 ? 0 : k == 1 ? 1 : k == 2 ? -1 : k <= 4 ? k - 3 : (k - 5) % 3 - 1;
}
__host__ __device__ constexpr int cc_dy(int k) { return k <= 1 ? 0 : k <= 4 ? 1 : (k - 5) / 3 - 1; }
__host__ __device__ constexpr int cc_dz(int k) { return k <= 4 ? 0 : 1; }
constexpr int kCcSlots = 14;
struct CoarseCluster {
  int nx, ny, nz;        // node lattice (boundary planes and rings included; they are Dirichlet)
  int ctas;              // cluster size: interior planes 1 .. nz-2 split over the CTAs
  int rmax;              // rows of the largest CTA (planes x nx x ny)
  const float* val32;    // [14][n] stencil values (symmetrised), FP32, lattice numbering
  const double* val64;   // [14][n] FP64
  const float* invDf;    // Jacobi diagonal, 0 on Dirichlet nodes
  const double* b;
  double* x;
  double rtol;
  int maxit;
  int degree;
  double lmax;
  unsigned* ctl;         // as CoarseCG::ctl ([2] status, [3] iterations, [4] sticky error)
};
// Cluster size, largest CTA and shared memory for an nx x ny x nz lattice; false if the
// problem does not fit one cluster on this device (nothing changed then).
bool coarse_cluster_plan(int nx, int ny, int nz, int* ctas, int* rmax, size_t* smem);
bool coarse_cluster_launch(const CoarseCluster& a, size_t smem, cudaStream_t s, cudaError_t* err);

// ---- batched Krylov (batched.cu): nb right-hand sides at leading dimension ld ----
// Per right-hand side: scal[q * S_NSLOTS + slot] and stat[q * 4 + {0 active, 1 iterations,
// 2 status, 3 spare}].
enum BatchStatus { BS_RUNNING = 0, BS_OK = 1, BS_NOTCONV = 2, BS_BREAKDOWN = 3 };
enum BatchPost {
  BPOST_NONE = 0,
  BPOST_INIT,      // s0 = (b, b): BB, tolerance rtol^2 BB in S_T0, active unless b = 0
  BPOST_SET_RZ,    // s0 = (z, r): ZR = RZ = s0
  BPOST_ALPHA,     // s0 = (p, A p): ALPHA = RZ / PQ while active (breakdown freezes), else 0
  BPOST_CHECK,     // s0 = (r, r): iteration count, converged when RR <= S_T0
  BPOST_BETA_Q     // s0 = (z, r), s1 = (z, A p): Polak-Ribiere BETA while active (else 0), with
                   // r_new - r_old = -ALPHA A p
};
int bred_blocks(int64_t n);
// part needs 2 * nb * bred_blocks(n) doubles
void bdot2(int64_t n, int64_t ld, int nb, const double* a0, const double* b0, const double* a1, const double* b1,
           int post, double rtol, double* part, double* scal, int* stat, cudaStream_t s);
// Fused forms of the batched flexible CG: x += alpha p; r -= alpha q; r32 (if not NULL) = FP32
// copy of r, then BPOST_CHECK; (z, r) and (z, q) with z in FP32 or FP64, then post; p = z +
// beta p (first: p = z).
void bfcg_update_xr32(int64_t n, int64_t ld, int nb, double* x, double* r, float* r32, const double* p,
                      const double* q, double* part, double* scal, int* stat, cudaStream_t s);
template <typename Tz>
void bdot_zr_zq(int64_t n, int64_t ld, int nb, const Tz* z, const double* r, const double* q, int post,
                double* part, double* scal, int* stat, cudaStream_t s);
template <typename Tz>
void bupdate_p_from(int64_t n, int64_t ld, int nb, const Tz* z, double* p, const double* scal, bool first,
                    cudaStream_t s, double* q_zero = nullptr);

// Coarse PCG with one thread block per right-hand side (no grid-wide synchronisation).
struct CoarseBlock {
  int64_t n;
  int nslot;
  const int* col;        // ELL, slot-major
  const double* val;
  const double* invD;
  const double* b;       // [nb][ld]
  double* x;             // [nb][ld]
  int64_t ld;
  double rtol;
  int maxit;
  int degree;
  double lmax;
  unsigned* stat;        // [nb][2]: status (CoarseStatus), iterations
  unsigned* sticky;      // worst error (atomicMax), reset by the caller
  int pf32;              // preconditioner in FP32 (as CoarseCG::pf32)
  const float* valf;
  const float* invDf;
};
bool coarse_block_supported(int64_t n);
bool coarse_block_launch(const CoarseBlock& a, int nb, cudaStream_t s);

// ---- adjoint V-cycle (adjoint.cu), FP64, batched at leading dimension ld ----
// Dout = d, SRout = S r
void adj_record(int64_t n, int64_t ld, int nb, const double* d, const double* r, const double* S, double* Dout,
                double* SRout, cudaStream_t s);
// rho += a S delta
void adj_rho(int64_t n, int64_t ld, int nb, double a, const double* S, const double* delta, double* rho,
             cudaStream_t s);
// delta = beta xbar + c1 delta - y; y = 0
void adj_delta(int64_t n, int64_t ld, int nb, double beta, double c1, const double* xbar, double* delta, double* y,
               cudaStream_t s);
// out = a x + b y (y may be null); out may alias x or y
void lincomb(int64_t n, int64_t ld, int nb, double a, const double* x, double b, const double* y, double* out,
             cudaStream_t s);
// out_q = coef[q] x_q (coef on the device)
void scale_rows(int64_t n, int64_t ld, int nb, const double* coef, const double* x, double* out, cudaStream_t s);
// scratch doubles needed by the two dot routines below
int adj_dot_scratch(int64_t n, int nb);
// acc[slot] += coef * sum_q <a_q, b_q>  (deterministic order)
void dot_accumulate(int64_t n, int64_t ld, int nb, const double* a, const double* b, double coef, double* part,
                    double* acc, int slot, cudaStream_t s);
// out[q] = <a_q, b_q>
void dot_rows(int64_t n, int64_t ld, int nb, const double* a, const double* b, double* part, double* out,
              cudaStream_t s);

// ---- restarted flexible GMRES (gmres.cu), FP64; V, Z: [nv][ld] ----
int gmres_max_basis();                 // restart + 1 at most
int gmres_part_size(int64_t n);        // doubles of scratch for the routines below
// h[i] = <V_i, w>, i < nv (device h)
void gmres_mdot(int64_t n, int64_t ld, int nv, const double* V, const double* w, double* part, double* h,
                cudaStream_t s);
// w += sign * sum_i h[i] V_i; if hn: *hn = ||w|| (device), and if wn: wn = w / ||w||
void gmres_maxpy_norm(int64_t n, int64_t ld, int nv, const double* V, const double* h, double sign, double* w,
                      double* part, double* hn, double* wn, cudaStream_t s);
// *hn = ||w|| and (if wn) wn = w / ||w||
void gmres_norm_scale(int64_t n, const double* w, double* part, double* hn, double* wn, cudaStream_t s);

// ---- Lanczos helpers ----
void splitmix_fill(int64_t n, uint64_t seed, const double* invD, double* v, cudaStream_t s);
// t = sqrt(invD) * v
void sqrt_scale(int64_t n, const double* invD, const double* v, double* t, cudaStream_t s);
// w = sqrt(invD) * y - alpha v - beta vprev  (alpha, beta from host)
void lanczos_w(int64_t n, const double* invD, const double* y, const double* v,
               const double* vprev, double alpha, double beta, double* w, cudaStream_t s);
void scale(int64_t n, double a, const double* x, double* y, cudaStream_t s);

// Defined in api.cu: row k of the optimized-beta table (nullptr outside 1..16) and the
// per-thread message returned by chebmg_last_error().
const double* beta_row(int k);
void set_last_error(const char* msg);

}  // namespace chebmg
