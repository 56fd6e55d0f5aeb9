// Internal declarations of the batched solver: many right-hand sides y_b sharing one A.
//
// Every instance b runs the same screened FISTA iteration as the single-instance solver
// (Algorithm 1 / Algorithm 2 with the dual points of Section 4), in lockstep with the
// others; finished instances leave the active list at the next evaluation.
//
// Iteration kinds (k = iteration index, K = screening period):
//   k % K == 0   evaluation: exact correlation g_k = A^T (y - A x_k) in float32 (or
//                double-float) products, the dual point, the gap, the sphere test, the
//                stop test, and the step to x_{k+1} from that exact g_k.
//   otherwise    tensor-core step: g_k = g_{k-1} - H~ d_k with H~ = bf16(A^T A) and
//                d_k = bf16(x_k - x_{k-1}), one tcgen05 GEMM over all active instances
//                with the step fused into its epilogue.
// The iterates are double-float pairs: with float32 iterates a coordinate stops moving once
// |g_j| / L falls below half an ulp of x_j, which floors the gap far above 1e-6 when L is
// in the hundreds.  Correlations and momentum stay float32.
// The Gram form gives A^T (y - A x_k) = A^T (y - A x_{k-1}) - A^T A (x_k - x_{k-1}) exactly;
// with bf16 operands the error of a step is proportional to |x_k - x_{k-1}|, so it vanishes
// as the iteration converges, and every evaluation restarts the recurrence from the exact
// correlation.  The certificates (gap, radius, test) only ever use evaluation quantities.
#pragma once

#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

namespace bvls {

constexpr int kBTile = 128;        // coordinates per M tile = instances per N tile
constexpr int kBChunk = 64;        // K elements per shared-memory stage (128 bytes of bf16)
constexpr int kBStages = 4;        // stages in flight
constexpr int kBStepThreads = 512;  // 16 warps: 4 TMEM lane quarters x 4 column groups
constexpr int kBCopyWarps = 4;     // warps of the step that copy the D rows of a chunk
constexpr int kBEvalInst = 8;      // instances per CTA of the evaluation kernel
constexpr int kBEvalThreads = 256;
constexpr int kBEvalIlvF32 = 2;    // interleaved sums per correlation in the evaluation's A^T r
constexpr int kBEvalIlvX2 = 2;
constexpr int kBEvalRing = 4;      // steps of 8 rows in the evaluation's copy ring (RING - 1 in flight)
constexpr int kBMaxRows = 1024;    // m limit: the residuals of a CTA's instances sit in shared memory
constexpr int kBMaxCols = 4096;    // n limit: the Gram matrix has npad^2 bf16 entries
constexpr int kBMaxBatch = 1 << 20;

struct BState {
  int kbase;          // iterations completed before the running chunk
  int n_act;          // instances still iterating (length of the active list)
  int done;           // every instance finished
  int error;          // a bounded wait gave up
  int nonfinite;      // Y or X0 held NaN/Inf
  int gap_evals;      // evaluations run
  int chunks;         // chunks run by the device-side loop of the solve graph
  int pad0;
  double sum_step;    // sum over tensor-core steps of the active instance count
  double sum_eval;    // sum over evaluations of the active instance count
  double sum_pres;    // sum over evaluations and instances of the preserved coordinates
};

struct BParams {
  const float* A;          // padded float32 copy of the handle, column-major
  int m, n, lda;
  int npad;                // n rounded up to kBTile: row pitch of every B x n array
  int B;
  const __nv_bfloat16* H;  // npad x npad, bf16(A^T A), zero outside n x n
  const double* l;
  const double* u;
  const double* nrm;       // ||a_j||
  const float* nrmf;       // ||a_j|| rounded up to float32
  const float* wf;         // a_j^T t rounded to float32
  const double* w;         // a_j^T t (translation mode)
  const uint8_t* jinf;
  const float2* l2;        // bounds as double-float pairs (clip of the iterates)
  const float2* u2;
  double invL;
  float2 invL2;            // 1 / L as a double-float pair
  double t_norm, gamma_w;
  double Cg;               // |computed a_j^T r - a_j^T r| <= Cg ||a_j|| ||r|| (evaluation precision)
  double Cg2;              // the same for double-float correlations
  double Cf;               // residual rounding: <= Cf sum_j |x_j| ||a_j|| (2-norm)
  double Csub;
  double tol;
  int erb;                 // rows per block of the evaluation's correlation sums (beval_chain)
  int max_iter;
  int dual_mode;
  int screening;
  int restart;
  int K;
  // tensor map of the step's operand H~ (bf16, 128-byte swizzle, 64 x 128 box)
  CUtensorMap tmH;
};

struct BBuffers {
  float2* X[2];            // B x npad: x_k in slot k & 1 (x_{k-1} in the other), double-float
  float* G[2];             // B x npad: g_k in slot k & 1
  __nv_bfloat16* D[2];     // (B + 1) x npad: bf16(x_k - x_{k-1}) in slot k & 1; row B is zero
  float2* Ge;              // B x npad: correlations of the last evaluation (double-float)
  uint8_t* flags;          // B x npad: 0 preserved, 1 fixed at l_j, 2 fixed at u_j
  float* tval[2];          // B: FISTA parameter t_k in slot k & 1
  float* dotp[2];          // (npad / kBTile) x B: restart-test partials per M tile, slot k & 1
  const float* Y;          // B x lda, zero-padded rows
  const double* X0;        // B x n or null
  int* act;                // active instances (first n_act entries)
  int* act_tmp;
  int* fin;                // B: 1 once the instance has finished
  double* xout;            // B x n: returned iterates
  double* gap;             // B
  double* primal;          // B: P(x) of the returned iterate
  int* iters;              // B
  int* status;             // B: 0 converged, 4 max_iter reached (bvls_status values)
  int* npres;              // B: preserved coordinates at the finish
  BState* st;
};

// Summation order of the evaluation's correlations a_j^T r: one thread owns (column, instance)
// and walks the rows in blocks of `rows` (a multiple of 8) with `ilv` interleaved sums (row i
// into sum i mod ilv), merged pairwise at the end of each block and added to a running total.
// `depth` bounds the roundings any product passes through: rows / ilv + log2(ilv) + blocks.
struct BEvalChain {
  int rows;
  int depth;
};
__host__ __device__ inline BEvalChain beval_chain(int m, int ilv) {
  const int lg = ilv >= 4 ? 2 : ilv >= 2 ? 1 : 0;
  BEvalChain best{8, 1 << 30};
  for (int r = 8; r <= 1024; r += 8) {
    const int d = r / ilv + lg + (m + r - 1) / r;
    if (d < best.depth) best = BEvalChain{r, d};
  }
  return best;
}

cudaError_t launch_bgram(const float* A, int lda, int m, int n, int npad, __nv_bfloat16* H, cudaStream_t s);
cudaError_t launch_binit(const BParams& p, const BBuffers& b, cudaStream_t s);
cudaError_t launch_bstep(const BParams& p, const BBuffers& b, int j, cudaStream_t s);
// The steps j0 .. j0 + nsteps - 1 of a chunk (all tensor-core steps) in one cluster launch
// with the iteration state on chip; only when bsteps_supported(npad) (npad <= 512).  Same
// arithmetic in the same order as launch_bstep per step.
bool bsteps_supported(int npad);
size_t bsteps_smem_bytes(int npad);
cudaError_t launch_bsteps(const BParams& p, const BBuffers& b, int j0, int nsteps, cudaStream_t s);
cudaError_t launch_beval(const BParams& p, const BBuffers& b, int j, int precision, cudaStream_t s);
cudaError_t launch_bcompact(const BParams& p, const BBuffers& b, cudaStream_t s);
cudaError_t launch_bchunk_end(const BBuffers& b, int chunk_len, cudaStream_t s);
// Last node of a chunk inside the batched solve graph's while loop (see launch_loop_ctl).
cudaError_t launch_bloop_ctl(const BBuffers& b, cudaGraphConditionalHandle h, int max_chunks, cudaStream_t s);
size_t bstep_smem_bytes();
cudaError_t batch_configure(int m, int npad);  // shared-memory attributes of the step and evaluation kernels
size_t beval_smem_bytes(int m, int npad, int prec, int ring);

}  // namespace bvls
