// Internal declarations of the backward pass (backward.cu).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace bvls {

constexpr int kBwdThreads = 256;
constexpr int kBwdMaxFree = 1024;  // free-set size limit (w, r, p, s sit in shared memory)

struct BwdParams {
  const float* A;        // padded float32 copy of the handle, column-major
  int m, n, lda, B;
  const double* l;
  const double* u;
  const double* X;       // B x n solutions
  const float* Y;        // B x ldy right-hand sides
  int ldy;
  const double* dLdX;    // B x n
  double* dLdY;          // B x m or null
  double* W;             // B x n scratch: w (zero off the free set), or null
  double* Q;             // B x m scratch: A_F w, or null
  double* R;             // B x m scratch: y - A x, or null
  int* status;           // B: 0 converged, 1 CG iteration limit, 2 free set too large, 3 |F| > m
  int* iters;            // B: CG iterations
  int* nfree;            // B: |F|
  double free_tol;
  double cg_tol;
  int cg_max_iter;
};

size_t bwd_smem_bytes(int m);
cudaError_t launch_bwd(const BwdParams& p, cudaStream_t s);
cudaError_t launch_bwd_da(const BwdParams& p, double* dLdA, cudaStream_t s);

}  // namespace bvls
