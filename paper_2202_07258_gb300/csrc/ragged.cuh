// Internal declarations of the ragged batch: B independent problems, each with its own A_k
// (m_k x n_k), y_k and box, solved together (the mixed NNLS/BVLS batch of uneven sizes).
//
// Every instance runs the single-instance iteration (FISTA + restart with the screening of
// Algorithm 1 / 2 every K iterations, dual scaling or translation with t = -1), in lockstep
// with the others.  One iteration is two launches over all active instances:
//   k_rpass   a work list of tiles (instance, up to tw preserved columns): the tile's
//             columns are staged in shared memory, then a_j^T r_k in double-float, the FISTA
//             step, and the tile's partial of A x_{k+1} (double-float, per row);
//   k_rresid  per instance: r_{k+1} = y' - sum of its tiles' partials, P_{k+1}, and the
//             instance scalars (restart test, translation step).
// Every K iterations k_rgap evaluates the gap, runs the sphere test, compacts the preserved
// list, folds fixed columns into y', and retires converged instances; k_rtiles rebuilds the
// work list.  Power iterations for L_k reuse k_rpass / k_rresid in a power mode.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace bvls {

constexpr int kRTileMin = 8;        // columns per tile: tw in {8, 16, 32}, picked by the autotuner
constexpr int kRTileMax = 32;
constexpr int kRThreads = 256;
constexpr int kRMaxRows = 1024;     // m_k limit (r_k in shared memory)
constexpr int kRRowBlocks = kRMaxRows / 32;   // row blocks of the residual kernel per instance

struct RInst {                      // per instance, fixed at setup
  long long a_off;                  // offset of A_k in the float arena (column-major, lda)
  long long c_off;                  // offset of the instance's columns in per-column arrays
  long long r_off;                  // offset of the instance's rows in per-row arrays
  long long p_off;                  // offset of the instance's tile partials (tiles_max x m)
  long long t_off;                  // offset of the instance's per-tile scalars
  int m, n, lda, tiles_max;         // tiles_max = ceil(n / kRTileMin)
  int dual_mode;                    // kScaling, kTranslation (t = -1) or kZero
  int pad;
  double invL;
  double t_norm;                    // ||t|| = sqrt(m) for t = -1
  double gamma_w;
  double Cg, Cf, Csub;
};

struct RState {                     // per instance, changes while solving
  int k, done, converged, n_active, n_pins, out_slot, gap_evals, nonfinite;
  double t, P, P_prev, eps, gap, radius, eta, y_norm, E_fold, S_fold;
  double pw_scale;                  // power iteration: the norm that scales the next iterate
  double pw_lambda;                 // power iteration: the latest estimate of ||A||^2
  double dot;                       // restart test of the last iteration
};

struct RTileRef {                   // one entry of the work list
  int inst, tile;                   // tile index within the instance's preserved list
};

struct RBuf {
  const float* A;                   // arena
  const RInst* inst;
  RState* st;
  // per column (concatenated over instances)
  float2* x[2];
  float2* g[2];
  const float2* l2;
  const float2* u2;
  const double* l;
  const double* u;
  double* nrm;
  double* w;                        // a_j^T t (t = -1)
  const uint8_t* jinf;
  uint8_t* flags;
  int* idx;                         // preserved list (instance-local column indices)
  int* idx_tmp;
  // per row
  float* yh;
  float* yl;
  float* rh;
  float* rl;
  float2* part;                     // tile partials: per instance, tiles_max x m
  double* tdot;                     // per (instance, tile): restart-test partial
  double* teps;                     // per (instance, tile): translation-step candidate
  // work list
  RTileRef* tiles;
  int* n_tiles;
  int* n_act_inst;
  int* act;                         // active instances
  // outputs
  double* xout;                     // per column
  int B;
  int K;
  int max_iter;
  double tol;
  int screening;
  int restart;
  int power;                        // 1: the pass runs power iterations (x <- A^T A x / scale)
  unsigned int* err;                // bit 0: NaN or Inf in A or y
  int* chunks;                      // chunks run by the device-side loop of the solve graph
  int tw;                           // columns per tile of the work list (kRTileMin..kRTileMax)
  double* work;                     // sum over iterations of sum_k m_k |S_k| (A elements read), or null
  double* rblkP;                    // per (instance, row block): partial of P of the residual kernel
  unsigned int* rcnt;               // per instance: row blocks of the residual kernel done (zeroed)
};

cudaError_t launch_rnorms(const RBuf& b, long long total_cols, cudaStream_t s);
cudaError_t launch_rinit(const RBuf& b, long long total_cols, int power, cudaStream_t s);
cudaError_t launch_rtiles(const RBuf& b, cudaStream_t s);
cudaError_t launch_rfwd(const RBuf& b, cudaStream_t s);
cudaError_t launch_rpass(const RBuf& b, int max_tiles, int slot, int gap_iter, cudaStream_t s);
cudaError_t launch_rresid(const RBuf& b, int slot, cudaStream_t s);
cudaError_t launch_rgap(const RBuf& b, int slot, cudaStream_t s);
cudaError_t launch_rexport(const RBuf& b, cudaStream_t s);
size_t rpass_smem_bytes(int tw);
cudaError_t ragged_configure();  // shared-memory attribute of the tile kernel (before any launch; widest tile)
// Last node of a chunk in the ragged solve graph's while loop: ends the loop once no instance
// is active or max_chunks chunks have run.
cudaError_t launch_rloop_ctl(const RBuf& b, cudaGraphConditionalHandle h, int max_chunks, cudaStream_t s);

}  // namespace bvls
