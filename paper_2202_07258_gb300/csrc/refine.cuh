// Internal declarations of the free-set refinement (refine.cu).
//
// After a solve has certified its gap, the optimality conditions of Section 3.2
// (Eq. (optimality2)) describe the optimum exactly: the coordinates strictly inside the box
// (the free set F) satisfy a_j^T (y - A x) = 0, the others sit at a bound with the sign
// condition on a_j^T (y - A x).  With F known, x_F solves the restricted normal equations
// A_F^T A_F x_F = A_F^T (y - A_B x_B).  The refinement takes F from the solver's iterate and
// solves those equations by mixed-precision iterative refinement: the residual and the
// correlations in float64, the correction by conjugate gradients in float32; a coordinate
// that leaves the box is clipped onto its bound and a bound coordinate whose correlation has
// the wrong sign joins F, round after round, until the conditions hold within their rounding
// bounds.  Coordinates fixed by the safe rule are certified at their bounds and stay there.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace bvls {

constexpr int kRefThreads = 512;
constexpr int kRefMaxRows = 8192;   // the residual sits in shared memory (12 bytes per row)
constexpr int kRefMaxFree = 2048;   // free-set limit (five 4-byte vectors in shared memory)

// One instance.  Column j of A starts at A + j * lda (float32); y has m entries; l, u, x,
// g and xsave have n entries; flags (may be null) marks coordinates fixed by the safe rule.
struct RefDesc {
  const float* A;
  const float* y;
  const double* l;
  const double* u;
  double* x;           // in: the solver's iterate; out: refined (or unchanged if declined)
  const uint8_t* flags;
  double* g;           // scratch: a_j^T (y - A x) of the preserved coordinates
  double* xsave;       // scratch: the solver's iterate, restored when the refinement declines
  double step;         // 1/L of the solve (> 0): the proximal-gradient prediction of step 2
  int m, n, lda;
  int pad;
};

// Per-instance result.
struct RefOut {
  int refined;         // 1: the returned x satisfies the optimality conditions (below)
  int rounds;          // refinement rounds run
  int nfree;           // |F| at the end
  int cg_iters;        // conjugate-gradient iterations over all rounds
  int reason;          // 0 ok, 1 rounds exhausted, 2 |F| > kRefMaxFree or > m, 3 m > kRefMaxRows
  int pad;
  double kkt;          // max over preserved j of |x_j - clip(x_j + a_j^T (y - A x), l_j, u_j)|
  double viol;         // largest violation of the sign / stationarity tests, in units of its bound
};

struct RefParams {
  const RefDesc* desc; // B descriptors (device memory)
  RefOut* out;         // B results (device memory)
  int B;
  int max_rounds;      // rounds of residual, tests and correction (10 in the entry points)
  int cg_max_iter;     // per round
  float cg_tol;        // relative residual of the float32 correction solve
  double tau;          // free-set margin: l_j + tau (1 + |l_j|) < x_j < u_j - tau (1 + |u_j|)
  double zeta;         // stationarity: |a_j^T r| <= eta_j + zeta ||a_j|| ||r|| on F
};

size_t refine_smem_bytes(int m_max, int free_max);
// Descriptors of B instances that share A, l, u: instance b uses Y + b*ldy, X + b*ldx,
// flags + b*ldf (flags may be null), G + b*n, XS + b*n.
cudaError_t launch_ref_desc_strided(RefDesc* out, int B, const float* A, int m, int n, int lda, const float* Y,
                                    int ldy, const double* l, const double* u, double* X, int ldx,
                                    const uint8_t* flags, int ldf, double* G, double* XS, double step,
                                    cudaStream_t s);
// One CTA per instance; m_max, free_max size the shared memory (m_max <= kRefMaxRows).
cudaError_t launch_refine(const RefParams& p, int m_max, int free_max, cudaStream_t s);

}  // namespace bvls
