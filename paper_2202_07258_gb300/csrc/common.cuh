// Internal declarations shared by the CUDA translation units of the solver.
//
// Arithmetic conventions
//   * A is float32, column-major, padded to lda_pad = roundup(m, 32) rows (pad rows are 0).
//   * The iterate x, the correlations g = A^T r and every scalar of the screening step are
//     float64.  float64 runs at a small fraction of the float32 rate on this part, so the
//     two O(m |A|) products never use it: in the FP32X2 mode they multiply with error-free
//     float32 products (fmaf) and accumulate in double-float pairs (hi, lo) with the
//     TwoSum transformation, which carries about 48 significant bits.
//   * Vectors of length m that feed the products (the folded data y' and the residual r)
//     are stored as two float32 arrays, hi and lo; their value is defined as hi + lo.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace bvls {

constexpr int kFwdRows = 128;     // rows per block of the A_S x_S kernel (32 lanes x float4)
constexpr int kFwdWarps = 4;      // column groups per block of that kernel
constexpr int kFwdThreads = kFwdRows / 4 * kFwdWarps;
constexpr int kFwdStage = 256;    // columns staged in shared memory at a time
constexpr int kTrWarps = 16;      // warps per block of the A_S^T r kernel
constexpr int kTrThreads = kTrWarps * 32;
constexpr int kRedThreads = 256;  // blocks of the O(|A|) epilogue kernels
constexpr int kCompactThreads = 1024;
constexpr int kMaxRows = 24576;   // r is staged in shared memory: 8 bytes per row
constexpr int kPassDot = 8;       // dot warps of the fused pass
constexpr int kLanczosSteps = 20; // Lanczos steps of the setup's step-constant estimate
constexpr int kPassTmax = 8;      // float4 row chunks owned by one lane of a q warp
constexpr int kPassMaxStages = 32;
constexpr int kMaxGridFlags = 1024;  // grid barrier words of the persistent pass
constexpr long long kGridWaitCycles = 4000000000LL;  // bounded grid-barrier wait (about 2 s)
// The persistent pass gives each CTA at least this many preserved columns: when screening
// has left fewer than kItersColsMin x (launched CTAs) columns, only ceil(|S| / kItersColsMin)
// CTAs take part (the others return at entry).  Measured on the Table-2 BVLS shape
// (1000 x 2000, about a fifth of the columns preserved on average): 16 columns per CTA made
// the screened solve 1.3x slower than one column (its iteration time is a per-CTA latency
// chain, not the barriers), so only CTAs that would own no column stay out.
constexpr int kItersColsMin = 1;

// CTAs of the persistent pass that take part for n_act preserved columns and `grid` launched.
__host__ __device__ inline int iters_active_ctas(int n_act, int grid) {
  const int want = (n_act + kItersColsMin - 1) / kItersColsMin;
  return want < 1 ? 1 : (want < grid ? want : grid);
}
// Columns one CTA of the persistent pass may own for n columns and `grid` CTAs.
__host__ __device__ inline int iters_idx_cap(int n, int grid) {
  const int per = (n + grid - 1) / grid;
  const int cap = per > kItersColsMin ? per : kItersColsMin;
  return cap < n ? cap : n;
}

enum DualMode { kScaling = 0, kTranslation = 1, kZero = 2 };
// kMix: float32 correlations a_j^T r, double-float forward product A_S x (the values of the
// public BVLS_PREC_* constants)
enum Precision { kX2 = 0, kF32 = 1, kMix = 2 };
enum Algorithm { kFista = 0, kChambollePock = 1 };

// Scalars of one solve, in device memory.  Written by the last block of a kernel (the
// others signal completion through the counters) and read by the next kernel.
struct DevState {
  int k;              // iterations completed
  int done;           // 1: stop; every kernel returns at entry
  int stop;           // set by the gap kernel, turned into done after the screening step
  int converged;
  int n_active;       // |preserved set|
  int n_pins;         // coordinates fixed by the current screening step
  int n_fold;         // of which with a nonzero bound value (their columns are folded into y')
  int out_slot;       // which x buffer holds the returned iterate
  int gap_evals;
  int nonfinite;
  int error;          // a bounded device wait gave up (nonzero: results invalid)
  int chunks;         // chunks run by the device-side loop of the solve graph
  double t;           // FISTA momentum parameter t_k
  int ti;             // steps since the last restart (t_k = T[ti] of the momentum table)
  int pad_ti;
  double P[2];        // 1/2 ||r_k||^2 in slot k & 1 (r = rh + rl)
  double eps;         // translation step of the last evaluation
  double gap;         // gap upper bound of the last evaluation
  double radius;      // sqrt(2 gap)
  double eta;         // per-unit-norm rounding margin of a_j^T theta
  double E_fold;      // bound on || y' (stored) - y' (exact) ||_2
  double S_fold;      // sum over folded columns of |b_j| ||a_j||
  double y_norm;      // ||y||_2
  double sum_active;  // sum of |preserved set| over the A_S^T r passes
  double sum_nnz;     // sum of nonzero preserved x_j over the A_S x_S passes
  double theta_r2;    // ||theta - r_k||^2 for a fixed dual point (computed by the pass at gap iterations)
  unsigned long long gbase;  // the persistent pass's grid-barrier count at the start of its next launch
  unsigned int cnt_tr, cnt_gap, cnt_fwd, cnt_resid;
};

// Momentum table of the persistent pass: with T[0] = 1 and T[i+1] = (1 + sqrt(1 + 4 T[i]^2)) / 2
// (the t_k recursion restarted at t = 1), entry i holds T[i], T[i+1] and beta = (T[i] - 1) /
// T[i+1] as double-float pairs, computed on the host in float64 so the step needs no float64.
struct MomEntry {
  double t, tn;
  float2 beta2, onepb2;   // beta and 1 + beta
};
constexpr int kMomTable = 1 << 16;

// Per-solve constants passed by value to the kernels.
struct Params {
  const float* A;          // padded copy, column-major
  int m, n, lda;           // lda = padded rows
  int m4;                  // m rounded up to a multiple of 4
  const double* l;         // lower bounds
  const double* u;         // upper bounds (+inf allowed)
  const double* nrm;       // ||a_j||_2
  const double* w;         // a_j^T t (translation mode)
  const uint8_t* jinf;     // 1 if u_j = +inf
  const float2* l2;        // l and u as double-float pairs (for the step's clip)
  const float2* u2;
  double invL;             // 1 / L
  float2 invL2;            // 1 / L as a double-float pair
  double t_norm;           // ||t||_2
  double gamma_w;          // |w_j (stored) - a_j^T t| <= gamma_w ||a_j|| ||t||
  double Cg;               // |g (computed) - a_j^T r| <= Cg ||a_j|| ||r||
  double Cf;               // |q (computed) - A_S x_S| <= Cf sum |x_j| ||a_j|| (per row, in 2-norm)
  double Csub;             // rounding of y' - q and of a fold, relative
  double tol;
  int max_iter;
  int dual_mode;
  int screening;
  int restart;
  // fixed dual point (the oracle-dual-point experiment of Section 5); wstar == null: Theta(x_k)
  const double* wstar;     // a_j^T theta_fixed (float64)
  const double* theta;     // theta_fixed (m)
  const double* tvec;      // the translation direction t (m), used with eps_star
  double eps_star;         // translation step that puts theta_fixed + eps_star t in F_D
  double eta_star;         // rounding bound of wstar_j + eps_star w_j per unit ||a_j||
  // primal-dual (Chambolle-Pock) iteration: steps and the bound of its residual recurrence
  int alg;                 // kFista or kChambollePock
  float2 tau2;             // primal step tau
  float2 sigma2;           // dual step sigma
  float2 inv1ps2;          // 1 / (1 + sigma)
  double E_cp;             // |r (stored) - r (exact)| from the recurrence r_{k+1} = (r_k + y' - A xbar) / 2
  const MomEntry* mom;     // momentum table (kMomTable entries)
  long long grid_wait;     // bound of the persistent pass's grid-barrier waits, in SM cycles
  int fwd_chunks;          // grid.y of the A_S x_S kernel
  int fwd_tiles;           // grid.x of the A_S x_S kernel
};

// ---------------------------------------------------------------- double-float helpers
// Error-free transformations (Knuth's TwoSum, FMA-based TwoProd).  Kept as separate
// statements; nvcc does not reassociate floating-point additions.
__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
  s = a + b;
  float bb = s - a;
  e = (a - (s - bb)) + (b - bb);
}

__device__ __forceinline__ void fast_two_sum(float a, float b, float& s, float& e) {
  // requires |a| >= |b| or a == 0
  s = a + b;
  e = b - (s - a);
}

// (s, c) += a * (xh + xl): exact product of a*xh, rounded a*xl, TwoSum into s, error into c.
__device__ __forceinline__ void df_fma(float& s, float& c, float a, float xh, float xl) {
  float p = a * xh;
  float e = fmaf(a, xh, -p);
  e = fmaf(a, xl, e);
  float t, err;
  two_sum(s, p, t, err);
  s = t;
  c += err + e;
}

// (s, c) += (s2, c2)
__device__ __forceinline__ void df_add(float& s, float& c, float s2, float c2) {
  float t, err;
  two_sum(s, s2, t, err);
  s = t;
  c += err + c2;
}

__device__ __forceinline__ double df_to_double(float s, float c) {
  return (double)s + (double)c;
}

__device__ __forceinline__ void split_double(double x, float& h, float& l) {
  h = (float)x;
  l = (float)(x - (double)h);
}

// ---- double-float values as float2 (x = hi, y = lo), float32 arithmetic only ----------
// The per-iteration path keeps x and g in this form: float64 runs at a small fraction of
// the float32 rate on this part, and these pairs carry about 48 significant bits.
__device__ __forceinline__ float2 df2_norm(float s, float c) {
  float h, l;
  two_sum(s, c, h, l);
  return make_float2(h, l);
}

__device__ __forceinline__ float2 df2_add(float2 a, float2 b) {
  float s, e;
  two_sum(a.x, b.x, s, e);
  e += a.y + b.y;
  float h, l;
  two_sum(s, e, h, l);
  return make_float2(h, l);
}

__device__ __forceinline__ float2 df2_sub(float2 a, float2 b) {
  return df2_add(a, make_float2(-b.x, -b.y));
}

__device__ __forceinline__ float2 df2_mul(float2 a, float2 b) {
  const float p = a.x * b.x;
  float e = fmaf(a.x, b.x, -p);
  e = fmaf(a.x, b.y, e);
  e = fmaf(a.y, b.x, e);
  float h, l;
  fast_two_sum(p, e, h, l);
  return make_float2(h, l);
}

// a < b for normalised pairs (|lo| <= ulp(hi)/2); infinities carry lo = 0
__device__ __forceinline__ bool df2_lt(float2 a, float2 b) {
  return a.x < b.x || (a.x == b.x && a.y < b.y);
}

__device__ __forceinline__ bool df2_eq(float2 a, float2 b) { return a.x == b.x && a.y == b.y; }

__device__ __forceinline__ bool df2_nonzero(float2 a) { return a.x != 0.0f || a.y != 0.0f; }

__device__ __forceinline__ double df2_to_double(float2 a) { return (double)a.x + (double)a.y; }

// float64 -> pair; +-inf map to (+-inf, 0)
__host__ __device__ __forceinline__ float2 df2_from_double(double x) {
  const float h = (float)x;
  if (isinf(h) || isinf(x)) return make_float2(h, 0.0f);
  return make_float2(h, (float)(x - (double)h));
}

__device__ __forceinline__ double warp_sum_d(double v) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

__device__ __forceinline__ unsigned ld_acquire_u32(const unsigned* p) {
  unsigned v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

__device__ __forceinline__ unsigned long long ld_relaxed_u64(const unsigned long long* p) {
  unsigned long long v;
  asm volatile("ld.relaxed.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
  return v;
}

__device__ __forceinline__ unsigned long long ld_acquire_u64(const unsigned long long* p) {
  unsigned long long v;
  asm volatile("ld.acquire.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
  return v;
}

// Grid barrier on a monotonic arrival count: each CTA adds 1 (release) once its threads have
// synchronised, then waits (bounded) until the count reaches `target` (the number of CTAs
// times the barriers passed so far).  No last arrival hands anything on, so a barrier costs
// one reduction and the polls.
// The release reduction orders the CTA's earlier writes (the caller synchronised the CTA's
// threads first, as for a fence by one thread); the polls are relaxed loads, and one acquire
// load after the count is reached orders the CTA's later reads.
__device__ inline bool grid_count_sync(unsigned long long* cnt, unsigned long long target, long long limit) {
  asm volatile("red.release.gpu.global.add.u64 [%0], 1;" ::"l"(cnt) : "memory");
  if (ld_acquire_u64(cnt) >= target) return true;
  const long long t0 = clock64();
  while (ld_relaxed_u64(cnt) < target) {
    if (clock64() - t0 > limit) return false;
  }
  (void)ld_acquire_u64(cnt);
  return true;
}

// All lanes of a warp agree on the outcome of a bounded wait.
__device__ __forceinline__ bool warp_all(bool ok) { return __all_sync(0xffffffffu, ok) != 0; }

// Sum of v[0..count) by one warp: each lane issues 8 loads before adding them, so every
// 256 entries cost one round trip to L2.  Result in every lane.
__device__ __forceinline__ double warp_load_sum(const double* v, int count) {
  double a = 0.0;
  for (int t0 = 0; t0 < count; t0 += 256) {
    double part[8];
#pragma unroll
    for (int k = 0; k < 8; ++k) {
      const int t = t0 + (threadIdx.x & 31) + 32 * k;
      part[k] = t < count ? __ldcg(v + t) : 0.0;
    }
#pragma unroll
    for (int k = 0; k < 8; ++k) a += part[k];
  }
  for (int o = 16; o > 0; o >>= 1) a += __shfl_xor_sync(0xffffffffu, a, o);
  return a;
}

__device__ __forceinline__ double warp_max_d(double v) {
  for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
  return v;
}

// ---------------------------------------------------------------- launch wrappers
// Iteration kernels (iter_kernels.cu).
struct Buffers {
  float2* x[2];           // iterates x_k (slot k & 1), double-float
  float2* g[2];           // correlations g_k = A_S^T r_k (slot k & 1), double-float
  int* idx;
  int* idx_tmp;
  int* fold;
  uint8_t* flags;
  float* yh;
  float* yl;
  float* rh;
  float* rl;
  float2* part;
  double* tileP;
  double* tileR;          // fused pass: block partials of P from the residual kernel
  double* tileD;          // primal-dual: block partials of ||z + r||^2 (theta = -z)
  double* tileZ;          // primal-dual: block partials of ||z||^2
  float* crh;             // primal-dual: the residual r(x_k) = y' - A_S x_S (hi, lo), kept by
  float* crl;             // the recurrence while rh / rl hold the dual iterate z
  unsigned int* tile_cnt;
  double* blk;            // per-block partials of the epilogue kernels (4 doubles each)
  float2* qpart;          // fused pass: per-CTA double-float partials of A_S x_S (grid x m4)
  unsigned int* gbar;     // persistent pass: grid-barrier words (the first two hold its 64-bit arrival count)
  double* xout;           // float64 copy of the returned iterate (n)
  DevState* st;
  const float* y_in;      // device copy of y
  const double* x0_in;    // device copy of x0 or null
};

cudaError_t launch_init(const Params& p, const Buffers& b, cudaStream_t s);
// Last node of a chunk inside the solve graph's while loop: clears the loop condition once
// the solve has stopped, a wait gave up, or max_chunks chunks have run.
cudaError_t launch_loop_ctl(const Buffers& b, cudaGraphConditionalHandle h, int max_chunks, cudaStream_t s);
cudaError_t launch_fwd(const Params& p, const Buffers& b, int slot, int precision, bool fold,
                       cudaStream_t s);
cudaError_t launch_tr(const Params& p, const Buffers& b, int slot, int precision, bool gap_iter,
                      int tr_blocks, cudaStream_t s);
cudaError_t launch_gap(const Params& p, const Buffers& b, int slot, bool finalize, int red_blocks,
                       cudaStream_t s);
cudaError_t launch_test(const Params& p, const Buffers& b, int slot, int red_blocks, cudaStream_t s);
cudaError_t launch_compact(const Params& p, const Buffers& b, int slot, cudaStream_t s);
size_t tr_smem_bytes(int m4);
// Fused single-pass iteration (pass_kernel.cu).
int pass_configure(int lda, int m4, int idx_cap, int smem_optin, int* qwarps, int* cps);
cudaError_t launch_pass(const Params& p, const Buffers& b, int slot, int precision, bool gap_iter,
                        int grid, int nstages, int cps, int qwarps, cudaStream_t s);
cudaError_t launch_resid(const Params& p, const Buffers& b, int slot, int nparts, cudaStream_t s);
// Persistent form: niter iterations (the last one a gap iteration when gap_last) in one
// cooperative launch of grid CTAs; same outputs as niter x (launch_pass + launch_resid).
// iters_configure returns true when the launch shape fits one CTA per SM.
bool iters_configure(int lda, int m4, int nstages, int cps, int idx_cap, int grid);
cudaError_t launch_iters(const Params& p, const Buffers& b, int slot0, int niter, bool gap_last, int precision,
                         int grid, int nstages, int cps, int qwarps, cudaStream_t s);
cudaError_t launch_export(const Params& p, const Buffers& b, int slot, cudaStream_t s);
// primal-dual start: r_0 (in rh / rl from the forward kernel) moves to crh / crl and
// z_1 = A x_0 - y' = -r_0 takes its place
cudaError_t launch_cp_init(const Params& p, const Buffers& b, cudaStream_t s);
cudaError_t tr_configure(int m4, int* blocks_per_sm);

// Record the text returned by bvls_last_error() on this thread (capi.cu).
void record_error(const char* msg);

// Setup kernels (setup_kernels.cu).
cudaError_t launch_check_finite(const float* A, int lda, int m, int n, int* flag, cudaStream_t s);
// l2, u2 as double-float pairs and jinf[j] = (u_j == +inf) from the device bounds l, u
cudaError_t launch_bound_pairs(const double* l, const double* u, float2* l2, float2* u2, uint8_t* jinf, int n,
                               cudaStream_t s);
// ||a_j|| rounded up (never below the exact norm); with wneg1, also a_j^T (-1) (the
// direction t = -1) in the same pass, bounded as launch_col_dots.
cudaError_t launch_col_norms(const float* A, int lda, int m, int n, double* nrm, cudaStream_t s,
                             double* wneg1 = nullptr);
// w_j = -c_j * inv
cudaError_t launch_scale_neg(const double* c, int n, double inv, double* w, cudaStream_t s);
// t (float64, m) as double-float pairs t2 = (float(t), float(t - float(t)))
cudaError_t launch_split_pairs(const double* t, float2* t2, int m, cudaStream_t s);
// w_j = a_j^T t for t given by launch_split_pairs, double-float accumulation
cudaError_t launch_col_dots(const float* A, int lda, int m, int n, const float2* t2, double* w,
                            cudaStream_t s);
// Bound of those products relative to ||a_j|| ||t||: a lane chain of d = ceil(m / 32) + 5
// TwoSum steps (2 (d+2)^2 u^2), the pair split of t and the rounded low products (4 u^2),
// the float64 lane tree, a scaling of w and the float64 norm of t (12 float64 units), with
// 1% for second-order terms.
inline double setup_dot_gamma(int m) {
  const double d = (double)((m + 31) / 32 + 5);
  return 1.01 * (2.0 * (d + 2.0) * (d + 2.0) * 0x1p-48 + 4.0 * 0x1p-48 + 12.0 * 0x1p-53);
}
// out_i = sum_j a_ij (deterministic); part: row_sums_scratch(m, n) doubles.
size_t row_sums_scratch(int m, int n);
cudaError_t launch_row_sums(const float* A, int lda, int m, int n, double* part, double* out, cudaStream_t s);
cudaError_t launch_power_step(const float* A, int lda, int m, int n, float* v, float* q, float* v2,
                              double* scal, cudaStream_t s);
cudaError_t launch_power_init(float* v, int n, cudaStream_t s);
// K Lanczos steps on A^T A from v0 (any nonzero vector) in one cooperative launch (one CTA
// per SM, lda <= 8192): ab[2 i] = alpha_i and ab[2 i + 1] = beta_i for i = 1..K (2 K + 2
// doubles); scal[1] = -1 if a grid-barrier wait gave up.  gb: two zeroed words (grid
// barrier); part: grid x lda floats; q: lda floats; wn2: grid doubles; qn2: lda / 32
// doubles.  Returns cudaErrorNotSupported when the launch shape does not fit.
cudaError_t launch_lanczos_coop(const float* A, int lda, int m, int n, const float* v0, float* part, float* q,
                                double* wn2, double* qn2, double* ab, double* scal, unsigned* gb, int K, int grid,
                                cudaStream_t s);

}  // namespace bvls
