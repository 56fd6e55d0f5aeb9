// Free-set refinement of a certified iterate (the optimality conditions of Section 3.2,
// Eq. (optimality2)), one CTA per instance.
//
// Round structure (at most max_rounds rounds):
//   1. r = y - A x and a bound on its rounding, in float64 over the nonzero x_j;
//   2. g_j = a_j^T r for the preserved coordinates, float64, with the rounding bound
//      eta_j = ||a_j|| (gamma_d ||r|| + ||e_r||); classification: a free coordinate
//      (l_j < x_j < u_j) must have |g_j| <= eta_j + zeta ||a_j|| ||r||; a coordinate at l_j
//      must have g_j <= eta_j, one at u_j g_j >= -eta_j.  When every test holds, the round
//      accepts x.  A free coordinate whose projected-gradient step x_j + g_j / L leaves the
//      box is moved onto that bound (the solver's iterate still carries coordinates that are
//      drifting to a bound), and the round ends there.  Otherwise F = {free} U {bound
//      coordinates that fail their sign test};
//   3. the correction d of the restricted normal equations A_F^T A_F d = g_F by conjugate
//      gradients in float32 (right-hand side normalised by its largest entry);
//   4. x_F <- clip(x_F + d, l, u): a coordinate that leaves the box stops on its bound.
// Steps 1-2 are the float64 residual of classical mixed-precision iterative refinement, so
// the float32 solve only has to reduce the error by a constant factor per round.  An instance
// whose rounds run out, whose free set exceeds m (A_F cannot have full column rank: the
// optimum is not unique) or the shared-memory capacity, keeps the solver's iterate.
#include "refine.cuh"

#include <cfloat>

namespace bvls {

namespace {

constexpr unsigned kFull = 0xffffffffu;
constexpr int kRefWarps = kRefThreads / 32;
constexpr int kChunk = kRefThreads;      // columns scanned per step of the column loops
constexpr double kU64 = 1.1102230246251565e-16;

__device__ __forceinline__ double warp_sum(double v) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(kFull, v, o);
  return v;
}
__device__ __forceinline__ float warp_sumf(float v) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(kFull, v, o);
  return v;
}
__device__ __forceinline__ double warp_max(double v) {
  for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(kFull, v, o));
  return v;
}

// Block-wide sum / max in a fixed order (every thread gets the same value).
__device__ double block_sum(double v, double* sh) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  v = warp_sum(v);
  __syncthreads();
  if (lane == 0) sh[warp] = v;
  __syncthreads();
  double t = 0.0;
#pragma unroll
  for (int w = 0; w < kRefWarps; ++w) t += sh[w];
  return t;
}
__device__ double block_max(double v, double* sh) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  v = warp_max(v);
  __syncthreads();
  if (lane == 0) sh[warp] = v;
  __syncthreads();
  double t = -DBL_MAX;
#pragma unroll
  for (int w = 0; w < kRefWarps; ++w) t = fmax(t, sh[w]);
  return t;
}

// Exclusive position of this thread's flag among the block's set flags, in thread order;
// *total receives the count.  Uses cnt[kRefWarps].
__device__ int block_rank(bool f, int* cnt, int* total) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const unsigned b = __ballot_sync(kFull, f);
  __syncthreads();
  if (lane == 0) cnt[warp] = __popc(b);
  __syncthreads();
  int before = 0, tot = 0;
#pragma unroll
  for (int w = 0; w < kRefWarps; ++w) {
    before += w < warp ? cnt[w] : 0;
    tot += cnt[w];
  }
  *total = tot;
  return before + __popc(b & ((1u << lane) - 1u));
}

__device__ __forceinline__ double gamma_n(double d) { return d * kU64 / (1.0 - d * kU64); }

}  // namespace

// Classification bits of a preserved coordinate in step 2.
constexpr uint8_t kInF = 1;     // solved for in step 3
constexpr uint8_t kFail = 2;    // fails its optimality test
constexpr uint8_t kSnap = 4;    // moved onto a bound in this round

__global__ void __launch_bounds__(kRefThreads) k_refine(RefParams p, int m_cap, int f_cap) {
  extern __shared__ __align__(16) unsigned char smem[];
  double* r = reinterpret_cast<double*>(smem);                 // m_cap
  float* q = reinterpret_cast<float*>(r + m_cap);              // m_cap
  int* F = reinterpret_cast<int*>(q + m_cap);                  // f_cap
  float* cp = reinterpret_cast<float*>(F + f_cap);             // f_cap each
  float* cr = cp + f_cap;
  float* cd = cr + f_cap;
  float* cs = cd + f_cap;
  int* nzj = reinterpret_cast<int*>(cs + f_cap);               // kChunk
  double* nzx = reinterpret_cast<double*>(nzj + kChunk);       // kChunk
  uint8_t* cls = reinterpret_cast<uint8_t*>(nzx + kChunk);     // kChunk
  __shared__ double sh[kRefWarps];
  __shared__ int cnt[kRefWarps];

  const int b = blockIdx.x;
  if (b >= p.B) return;
  const RefDesc d = p.desc[b];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int m = d.m, n = d.n;
  RefOut res{};
  if (m > m_cap || m > kRefMaxRows) {
    res.reason = 3;
    if (tid == 0) p.out[b] = res;
    return;
  }

  // Save the solver's iterate and snap the preserved coordinates within tau of a bound.
  for (int j = tid; j < n; j += kRefThreads) {
    const double xj = d.x[j];
    d.xsave[j] = xj;
    if (d.flags && d.flags[j]) continue;
    const double lj = d.l[j], uj = d.u[j];
    if (xj <= lj + p.tau * (1.0 + fabs(lj))) d.x[j] = lj;
    else if (isfinite(uj) && xj >= uj - p.tau * (1.0 + fabs(uj))) d.x[j] = uj;
  }
  __syncthreads();

  int accepted = 0;
  int cg_total = 0;
  int nf = 0;
  int rd = 0;
  double kkt = 0.0, viol = 0.0;
  for (; rd < p.max_rounds; ++rd) {
    // ---- 1. r = y - A x over the nonzero x_j (float64), and |y_i| + sum_j |a_ij x_j| (in q,
    // float32: an upper estimate within a relative 2^-24 per term, covered by the 1.01 below)
    for (int i = tid; i < m; i += kRefThreads) {
      const double yi = (double)d.y[i];
      r[i] = yi;
      q[i] = fabsf(d.y[i]);
    }
    int nnz = 0;
    for (int j0 = 0; j0 < n; j0 += kChunk) {
      const int j = j0 + tid;
      const double xj = j < n ? d.x[j] : 0.0;
      int tot = 0;
      const int pos = block_rank(xj != 0.0, cnt, &tot);
      if (xj != 0.0) {
        nzj[pos] = j;
        nzx[pos] = xj;
      }
      __syncthreads();
      nnz += tot;
      for (int i = tid; i < m; i += kRefThreads) {
        double a0 = r[i];
        float s0 = q[i];
        for (int k = 0; k < tot; ++k) {
          const float a = d.A[(size_t)nzj[k] * d.lda + i];
          const double xv = nzx[k];
          a0 = fma(-(double)a, xv, a0);
          s0 = fmaf(fabsf(a), (float)fabs(xv), s0);
        }
        r[i] = a0;
        q[i] = s0;
      }
      __syncthreads();
    }
    double rr = 0.0, ss = 0.0;
    for (int i = tid; i < m; i += kRefThreads) {
      rr = fma(r[i], r[i], rr);
      ss = fma((double)q[i], (double)q[i], ss);
    }
    rr = block_sum(rr, sh);
    ss = block_sum(ss, sh);
    const double nr = sqrt(rr) * (1.0 + 1e-12);
    // |r_i (computed) - r_i| <= gamma_{nnz+1} (|y_i| + sum_j |a_ij x_j|), summed in 2-norm
    const double er = 1.01 * gamma_n((double)nnz + 2.0) * sqrt(ss) * (1.0 + 1e-6 * (nnz + 2));
    const double gd = gamma_n((double)((m + 31) / 32) + 6.0);
    __syncthreads();

    // ---- 2. correlations, tests and the free set (in index order)
    nf = 0;
    int fails = 0, snaps = 0;
    bool overflow = false;
    kkt = 0.0;
    viol = 0.0;
    for (int j0 = 0; j0 < n; j0 += kChunk) {
      const int len = min(kChunk, n - j0);
      double wk = 0.0, wv = 0.0;
      int wf = 0, ws = 0;
      for (int jj = warp; jj < len; jj += kRefWarps) {
        const int j = j0 + jj;
        uint8_t c = 0;
        if (!(d.flags && d.flags[j])) {
          const float* col = d.A + (size_t)j * d.lda;
          double g = 0.0;
          float na2 = 0.f;
          for (int i = lane; i < m; i += 32) {
            const float a = col[i];
            g = fma((double)a, r[i], g);
            na2 = fmaf(a, a, na2);
          }
          g = warp_sum(g);
          na2 = warp_sumf(na2);
          const double na = sqrt((double)na2) * 1.001;
          const double eta = 1.01 * na * (gd * nr + er) + 1e-300;
          const double xj = d.x[j], lj = d.l[j], uj = d.u[j];
          double ex;
          if (xj == lj) {
            ex = g - eta;
            c = ex > 0.0 ? (kInF | kFail) : 0;
          } else if (xj == uj) {
            ex = -g - eta;
            c = ex > 0.0 ? (kInF | kFail) : 0;
          } else {
            ex = fabs(g) - eta - p.zeta * na * nr;
            c = kInF | (ex > 0.0 ? kFail : 0);
            const double xp = xj + d.step * g;
            if (ex > 0.0 && (xp <= lj || xp >= uj)) {
              // the projected-gradient step leaves the box: move x_j onto that bound
              c = kFail | kSnap;
              if (lane == 0) d.x[j] = xp <= lj ? lj : uj;
            }
          }
          const double xs = fmin(fmax(xj + g, lj), uj);
          wk = fmax(wk, fabs(xj - xs));
          wv = fmax(wv, (ex + eta) / eta);
          wf += (c & kFail) ? 1 : 0;
          ws += (c & kSnap) ? 1 : 0;
          if (lane == 0) d.g[j] = g;
        }
        if (lane == 0) cls[jj] = c;
      }
      kkt = fmax(kkt, wk);
      viol = fmax(viol, wv);
      fails += wf;
      snaps += ws;
      __syncthreads();
      const bool inF = tid < len && (cls[tid] & kInF);
      int tot = 0;
      const int pos = block_rank(inF, cnt, &tot);
      if (inF && nf + pos < f_cap) F[nf + pos] = j0 + tid;
      nf += tot;
      overflow |= nf > f_cap;
      __syncthreads();
    }
    kkt = block_max(kkt, sh);
    viol = block_max(viol, sh);
    // warps counted their own fails (lane values agree within a warp): one per warp
    const int fails_all = (int)block_sum(lane == 0 ? (double)fails : 0.0, sh);
    const int snaps_all = (int)block_sum(lane == 0 ? (double)snaps : 0.0, sh);
    if (fails_all == 0) {
      accepted = 1;
      break;
    }
    if (rd == p.max_rounds - 1) {
      res.reason = 1;
      break;
    }
    if (snaps_all > 0) {
      __syncthreads();
      continue;   // residual and correlations again at the moved point
    }
    if (overflow || nf > m) {
      res.reason = 2;
      break;
    }

    // ---- 3. A_F^T A_F c = g_F / s by conjugate gradients (float32), s = max |g_F|
    double gmax = 0.0;
    for (int k = tid; k < nf; k += kRefThreads) gmax = fmax(gmax, fabs(d.g[F[k]]));
    gmax = block_max(gmax, sh);
    const double sc = gmax > 0.0 ? gmax : 1.0;
    double rs = 0.0;
    for (int k = tid; k < nf; k += kRefThreads) {
      const float v = (float)(d.g[F[k]] / sc);
      cr[k] = v;
      cp[k] = v;
      cd[k] = 0.f;
      rs += (double)v * v;
    }
    rs = block_sum(rs, sh);
    const double target = (double)p.cg_tol * (double)p.cg_tol * rs;
    const int itmax = min(p.cg_max_iter, 3 * nf + 50);
    int it = 0;
    while (rs > target && it < itmax) {
      // q = A_F c_p, one thread per row
      for (int i = tid; i < m; i += kRefThreads) {
        float a0 = 0.f;
        for (int k = 0; k < nf; ++k) a0 = fmaf(d.A[(size_t)F[k] * d.lda + i], cp[k], a0);
        q[i] = a0;
      }
      __syncthreads();
      // c_s = A_F^T q, one warp per column
      for (int k = warp; k < nf; k += kRefWarps) {
        const float* col = d.A + (size_t)F[k] * d.lda;
        float a0 = 0.f;
        for (int i = lane; i < m; i += 32) a0 = fmaf(col[i], q[i], a0);
        a0 = warp_sumf(a0);
        if (lane == 0) cs[k] = a0;
      }
      __syncthreads();
      double pap = 0.0;
      for (int k = tid; k < nf; k += kRefThreads) pap += (double)cp[k] * cs[k];
      pap = block_sum(pap, sh);
      if (!(pap > 0.0)) break;
      const float alpha = (float)(rs / pap);
      double rn = 0.0;
      for (int k = tid; k < nf; k += kRefThreads) {
        cd[k] = fmaf(alpha, cp[k], cd[k]);
        cr[k] = fmaf(-alpha, cs[k], cr[k]);
        rn += (double)cr[k] * cr[k];
      }
      rn = block_sum(rn, sh);
      ++it;
      const float beta = (float)(rn / rs);
      rs = rn;
      for (int k = tid; k < nf; k += kRefThreads) cp[k] = fmaf(beta, cp[k], cr[k]);
      __syncthreads();
    }
    cg_total += it;

    // ---- 4. x_F <- clip(x_F + s c, l, u)
    for (int k = tid; k < nf; k += kRefThreads) {
      const int j = F[k];
      const double xn = d.x[j] + sc * (double)cd[k];
      d.x[j] = fmin(fmax(xn, d.l[j]), d.u[j]);
    }
    __syncthreads();
  }

  if (!accepted) {
    for (int j = tid; j < n; j += kRefThreads) d.x[j] = d.xsave[j];
  }
  if (tid == 0) {
    res.refined = accepted;
    res.rounds = min(rd + 1, p.max_rounds);
    res.nfree = nf;
    res.cg_iters = cg_total;
    res.kkt = kkt;
    res.viol = viol;
    p.out[b] = res;
  }
}

__global__ void k_ref_desc_strided(RefDesc* out, int B, const float* A, int m, int n, int lda, const float* Y,
                                   int ldy, const double* l, const double* u, double* X, int ldx,
                                   const uint8_t* flags, int ldf, double* G, double* XS, double step) {
  for (int b = blockIdx.x * blockDim.x + threadIdx.x; b < B; b += gridDim.x * blockDim.x) {
    RefDesc d{};
    d.A = A;
    d.y = Y + (size_t)b * ldy;
    d.l = l;
    d.u = u;
    d.x = X + (size_t)b * ldx;
    d.flags = flags ? flags + (size_t)b * ldf : nullptr;
    d.g = G + (size_t)b * n;
    d.xsave = XS + (size_t)b * n;
    d.step = step;
    d.m = m;
    d.n = n;
    d.lda = lda;
    out[b] = d;
  }
}

cudaError_t launch_ref_desc_strided(RefDesc* out, int B, const float* A, int m, int n, int lda, const float* Y,
                                    int ldy, const double* l, const double* u, double* X, int ldx,
                                    const uint8_t* flags, int ldf, double* G, double* XS, double step,
                                    cudaStream_t s) {
  k_ref_desc_strided<<<(B + 255) / 256, 256, 0, s>>>(out, B, A, m, n, lda, Y, ldy, l, u, X, ldx, flags, ldf, G, XS,
                                                     step);
  return cudaGetLastError();
}

size_t refine_smem_bytes(int m_max, int free_max) {
  return (size_t)m_max * (sizeof(double) + sizeof(float)) + (size_t)free_max * (sizeof(int) + 4 * sizeof(float)) +
         (size_t)kChunk * (sizeof(int) + sizeof(double) + 1) + 64;
}

cudaError_t launch_refine(const RefParams& p, int m_max, int free_max, cudaStream_t s) {
  if (m_max > kRefMaxRows) m_max = kRefMaxRows;
  m_max = (m_max + 1) / 2 * 2;
  free_max = (free_max + 3) / 4 * 4;
  const size_t sm = refine_smem_bytes(m_max, free_max);
  cudaError_t e = cudaFuncSetAttribute(k_refine, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
  if (e != cudaSuccess) return e;
  k_refine<<<p.B, kRefThreads, sm, s>>>(p, m_max, free_max);
  return cudaGetLastError();
}

}  // namespace bvls
