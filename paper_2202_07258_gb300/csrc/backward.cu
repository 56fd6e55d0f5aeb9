// Backward pass through the solution map (y, A) -> x*(y, A) of the box-constrained
// least-squares problem, for B instances that share the handle's A and box.
//
// At a non-degenerate optimum (strict complementarity; A_F of full column rank on the free
// set F) the optimality conditions of Section 3.2 fix the coordinates outside F at their
// bounds, and x_F solves the restricted normal equations A_F^T A_F x_F = A_F^T (y - A_B x_B).
// Differentiating them, with v = dL/dx and w = (A_F^T A_F)^{-1} v_F (zero off F):
//     dL/dy = A_F w,            dL/dA = r w^T - (A_F w) x^T,    r = y - A x.
// k_bwd solves for w by conjugate gradients on the free set (one CTA per instance) and
// writes dL/dy and the factors of dL/dA; k_bwd_da sums the rank-2 terms over the batch.
// Both run in float64: the backward is off the iteration's hot path and the solution map's
// derivative needs the accuracy (the finite-difference checks compare at 1e-6).
#include "backward.cuh"

namespace bvls {

namespace {

constexpr unsigned kFull = 0xffffffffu;

__device__ __forceinline__ double warp_sum(double v) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(kFull, v, o);
  return v;
}

// Sum over the block (kBwdThreads threads); every thread gets the result.
__device__ double block_sum(double v, double* sh) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  v = warp_sum(v);
  __syncthreads();
  if (lane == 0) sh[warp] = v;
  __syncthreads();
  double t = 0.0;
#pragma unroll
  for (int w = 0; w < kBwdThreads / 32; ++w) t += sh[w];
  return t;
}

}  // namespace

__global__ void __launch_bounds__(kBwdThreads) k_bwd(BwdParams p) {
  extern __shared__ double sm[];
  // shared: free-set list, then w, r, p, s (length <= kBwdMaxFree each) and q (m)
  int* sF = reinterpret_cast<int*>(sm);
  double* sw = sm + kBwdMaxFree / 2;
  double* sr = sw + kBwdMaxFree;
  double* sp = sr + kBwdMaxFree;
  double* ss = sp + kBwdMaxFree;
  double* sq = ss + kBwdMaxFree;
  __shared__ double sh[kBwdThreads / 32];
  __shared__ int s_cnt[kBwdThreads / 32 + 1];

  const int b = blockIdx.x;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const double* x = p.X + (size_t)b * p.n;
  const double* v = p.dLdX + (size_t)b * p.n;

  // ---- free set F (ordered): l_j + tau (1 + |l_j|) < x_j < u_j - tau (1 + |u_j|)
  int nf = 0;
  for (int j0 = 0; j0 < p.n; j0 += kBwdThreads) {
    const int j = j0 + tid;
    bool fr = false;
    if (j < p.n) {
      const double xj = x[j], lj = p.l[j], uj = p.u[j];
      fr = xj > lj + p.free_tol * (1.0 + fabs(lj)) && (isinf(uj) || xj < uj - p.free_tol * (1.0 + fabs(uj)));
    }
    const unsigned m = __ballot_sync(kFull, fr);
    if (lane == 0) s_cnt[warp] = __popc(m);
    __syncthreads();
    int before = 0, total = 0;
    for (int w = 0; w < kBwdThreads / 32; ++w) {
      if (w < warp) before += s_cnt[w];
      total += s_cnt[w];
    }
    const int pos = nf + before + __popc(m & ((1u << lane) - 1u));
    if (fr && pos < kBwdMaxFree) sF[pos] = j;
    nf += total;
    __syncthreads();
  }
  const bool too_big = nf > kBwdMaxFree;
  // |F| > m: A_F (m x |F|) cannot have full column rank, so A_F^T A_F is singular, the
  // optimum is not unique and the solution map has no derivative to follow
  const bool no_rank = !too_big && nf > p.m;
  if (too_big || no_rank) {
    if (tid == 0) {
      p.status[b] = too_big ? 2 : 3;
      p.iters[b] = 0;
      p.nfree[b] = nf;
    }
    nf = 0;  // the outputs below become zero gradients
  }

  // ---- conjugate gradients on (A_F^T A_F) w = v_F
  for (int k = tid; k < nf; k += kBwdThreads) {
    const double vk = v[sF[k]];
    sw[k] = 0.0;
    sr[k] = vk;
    sp[k] = vk;
  }
  __syncthreads();
  double rs = 0.0;
  for (int k = tid; k < nf; k += kBwdThreads) rs += sr[k] * sr[k];
  rs = block_sum(rs, sh);
  const double target = p.cg_tol * p.cg_tol * rs;
  int it = 0;
  bool conv = rs <= target || nf == 0;
  while (!conv && it < p.cg_max_iter) {
    // q = A_F p (thread per row)
    for (int i = tid; i < p.m; i += kBwdThreads) {
      double acc = 0.0;
      for (int k = 0; k < nf; ++k) acc = fma((double)p.A[(size_t)sF[k] * p.lda + i], sp[k], acc);
      sq[i] = acc;
    }
    __syncthreads();
    // s = A_F^T q (warp per column)
    for (int k = warp; k < nf; k += kBwdThreads / 32) {
      const float* col = p.A + (size_t)sF[k] * p.lda;
      double acc = 0.0;
      for (int i = lane; i < p.m; i += 32) acc = fma((double)col[i], sq[i], acc);
      acc = warp_sum(acc);
      if (lane == 0) ss[k] = acc;
    }
    __syncthreads();
    double pAp = 0.0;
    for (int k = tid; k < nf; k += kBwdThreads) pAp += sp[k] * ss[k];
    pAp = block_sum(pAp, sh);
    if (!(pAp > 0.0)) break;  // singular direction: A_F is rank deficient
    const double alpha = rs / pAp;
    double rn = 0.0;
    for (int k = tid; k < nf; k += kBwdThreads) {
      sw[k] = fma(alpha, sp[k], sw[k]);
      sr[k] = fma(-alpha, ss[k], sr[k]);
      rn += sr[k] * sr[k];
    }
    rn = block_sum(rn, sh);
    ++it;
    conv = rn <= target;
    const double beta = rn / rs;
    rs = rn;
    for (int k = tid; k < nf; k += kBwdThreads) sp[k] = fma(beta, sp[k], sr[k]);
    __syncthreads();
  }

  // ---- dL/dy = A_F w; the factors of dL/dA: w (zero off F), q = A_F w, r = y - A x
  for (int i = tid; i < p.m; i += kBwdThreads) {
    double acc = 0.0;
    for (int k = 0; k < nf; ++k) acc = fma((double)p.A[(size_t)sF[k] * p.lda + i], sw[k], acc);
    sq[i] = acc;
    if (p.dLdY) p.dLdY[(size_t)b * p.m + i] = acc;
    if (p.Q) p.Q[(size_t)b * p.m + i] = acc;
  }
  if (p.W) {
    double* wrow = p.W + (size_t)b * p.n;
    for (int j = tid; j < p.n; j += kBwdThreads) wrow[j] = 0.0;
    __syncthreads();
    for (int k = tid; k < nf; k += kBwdThreads) wrow[sF[k]] = sw[k];
  }
  if (p.R) {
    for (int i = tid; i < p.m; i += kBwdThreads) {
      double acc = (double)p.Y[(size_t)b * p.ldy + i];
      for (int j = 0; j < p.n; ++j) {
        const double xj = x[j];
        if (xj != 0.0) acc = fma(-(double)p.A[(size_t)j * p.lda + i], xj, acc);
      }
      p.R[(size_t)b * p.m + i] = acc;
    }
  }
  if (tid == 0 && !too_big && !no_rank) {
    p.status[b] = conv ? 0 : 1;
    p.iters[b] = it;
    p.nfree[b] = nf;
  }
}

// dL/dA[i][j] = sum_b R[b][i] W[b][j] - Q[b][i] X[b][j]; column-major output (leading
// dimension m), 32 x 32 outputs per block, the batch in chunks of 32.
__global__ void __launch_bounds__(256) k_bwd_da(BwdParams p, double* dLdA) {
  __shared__ double sR[32][33], sQ[32][33], sW[32][33], sX[32][33];
  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
  const int i0 = blockIdx.y * 32, j0 = blockIdx.x * 32;
  double acc[4] = {0.0, 0.0, 0.0, 0.0};  // rows i0 + tx, columns j0 + ty + 8 q
  for (int b0 = 0; b0 < p.B; b0 += 32) {
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int bb = ty + 8 * q;
      const int b = b0 + bb;
      const bool ok = b < p.B;
      sR[bb][tx] = ok && i0 + tx < p.m ? p.R[(size_t)b * p.m + i0 + tx] : 0.0;
      sQ[bb][tx] = ok && i0 + tx < p.m ? p.Q[(size_t)b * p.m + i0 + tx] : 0.0;
      sW[bb][tx] = ok && j0 + tx < p.n ? p.W[(size_t)b * p.n + j0 + tx] : 0.0;
      sX[bb][tx] = ok && j0 + tx < p.n ? p.X[(size_t)b * p.n + j0 + tx] : 0.0;
    }
    __syncthreads();
    for (int bb = 0; bb < 32; ++bb) {
      const double r = sR[bb][tx], qv = sQ[bb][tx];
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const int jj = ty + 8 * q;
        acc[q] = fma(r, sW[bb][jj], acc[q]);
        acc[q] = fma(-qv, sX[bb][jj], acc[q]);
      }
    }
    __syncthreads();
  }
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    const int i = i0 + tx, j = j0 + ty + 8 * q;
    if (i < p.m && j < p.n) dLdA[(size_t)j * p.m + i] = acc[q];
  }
}

size_t bwd_smem_bytes(int m) {
  return (size_t)(kBwdMaxFree / 2 + 4 * kBwdMaxFree + m) * sizeof(double);
}

cudaError_t launch_bwd(const BwdParams& p, cudaStream_t s) {
  const size_t sm = bwd_smem_bytes(p.m);
  cudaError_t e = cudaFuncSetAttribute(k_bwd, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
  if (e != cudaSuccess) return e;
  k_bwd<<<p.B, kBwdThreads, sm, s>>>(p);
  return cudaGetLastError();
}

cudaError_t launch_bwd_da(const BwdParams& p, double* dLdA, cudaStream_t s) {
  dim3 grid((p.n + 31) / 32, (p.m + 31) / 32);
  k_bwd_da<<<grid, 256, 0, s>>>(p, dLdA);
  return cudaGetLastError();
}

}  // namespace bvls
