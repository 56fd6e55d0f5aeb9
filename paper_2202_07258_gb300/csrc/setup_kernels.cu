// Kernels run once per matrix by bvls_setup: finiteness check, column norms ||a_j||_2
// (used by the sphere test of Eq. (safe_rule)), w = A^T t for the dual translation of
// Section 4.2, the row sums used to build candidate directions t, and a power iteration
// for the step constant L ~ ||A||_2^2.  These run once per matrix; the power iteration,
// a hundred passes over A, runs in one cooperative launch when its shape fits.
#include "common.cuh"

namespace bvls {

__global__ void k_check_finite(const float* __restrict__ A, int lda, int m, int n, int* flag) {
  const size_t total = (size_t)m * n;
  const size_t stride = (size_t)gridDim.x * blockDim.x;
  int bad = 0;
  for (size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += stride) {
    const size_t j = e / m, i = e % m;
    if (!isfinite(A[j * lda + i])) bad = 1;
  }
  if (__syncthreads_or(bad) && threadIdx.x == 0) atomicOr(flag, 1);
}

cudaError_t launch_check_finite(const float* A, int lda, int m, int n, int* flag, cudaStream_t s) {
  k_check_finite<<<1024, 256, 0, s>>>(A, lda, m, n, flag);
  return cudaGetLastError();
}

// one warp per column, float64 accumulation
// ||a_j||_2 and, when wneg1 is given, a_j^T (-1) = -sum_i a_ij in the same pass (the
// summation order of k_col_dots with t = -1, so the same values bit for bit).
__global__ void k_col_norms(const float* __restrict__ A, int lda, int m, int n, double* nrm, double* wneg1) {
  const int lane = threadIdx.x & 31;
  const int w = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int nw = (gridDim.x * blockDim.x) >> 5;
  for (int j = w; j < n; j += nw) {
    const float* a = A + (size_t)j * lda;
    double s = 0.0, c = 0.0;
    for (int i = lane; i < m; i += 32) {
      const double v = (double)a[i];
      s = fma(v, v, s);
      c = fma(v, -1.0, c);
    }
    s = warp_sum_d(s);
    c = warp_sum_d(c);
    if (lane == 0) {
      nrm[j] = sqrt(s);
      if (wneg1) wneg1[j] = c;
    }
  }
}

cudaError_t launch_col_norms(const float* A, int lda, int m, int n, double* nrm, cudaStream_t s,
                             double* wneg1) {
  k_col_norms<<<1024, 256, 0, s>>>(A, lda, m, n, nrm, wneg1);
  return cudaGetLastError();
}

// w_j = -c_j / n (the minus-mean-column direction from c = A^T (sum_k a_k)).
__global__ void k_scale_neg(const double* c, int n, double inv, double* w) {
  for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < n; j += gridDim.x * blockDim.x) w[j] = -c[j] * inv;
}

cudaError_t launch_scale_neg(const double* c, int n, double inv, double* w, cudaStream_t s) {
  k_scale_neg<<<(n + 255) / 256, 256, 0, s>>>(c, n, inv, w);
  return cudaGetLastError();
}

__global__ void k_col_dots(const float* __restrict__ A, int lda, int m, int n, const double* t,
                           double* w) {
  const int lane = threadIdx.x & 31;
  const int wi = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int nw = (gridDim.x * blockDim.x) >> 5;
  for (int j = wi; j < n; j += nw) {
    const float* a = A + (size_t)j * lda;
    double s = 0.0;
    for (int i = lane; i < m; i += 32) s = fma((double)a[i], t[i], s);
    s = warp_sum_d(s);
    if (lane == 0) w[j] = s;
  }
}

cudaError_t launch_col_dots(const float* A, int lda, int m, int n, const double* t, double* w,
                            cudaStream_t s) {
  k_col_dots<<<1024, 256, 0, s>>>(A, lda, m, n, t, w);
  return cudaGetLastError();
}

// out_i = sum_j a_ij, deterministic: column chunks of 64 give per-chunk partials (threads
// over rows, columns in order), then the partials are summed in chunk order.
constexpr int kRowSumCols = 64;

__global__ void k_row_sums_part(const float* __restrict__ A, int lda, int m, int n, double* part) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= m) return;
  const int j0 = blockIdx.y * kRowSumCols, j1 = min(n, j0 + kRowSumCols);
  double s = 0.0;
  for (int j = j0; j < j1; ++j) s += (double)A[(size_t)j * lda + i];
  part[(size_t)blockIdx.y * m + i] = s;
}

__global__ void k_row_sums_reduce(const double* part, int m, int nchunks, double* out) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= m) return;
  double s = 0.0;
  for (int c = 0; c < nchunks; ++c) s += part[(size_t)c * m + i];
  out[i] = s;
}

size_t row_sums_scratch(int m, int n) { return (size_t)m * ((n + kRowSumCols - 1) / kRowSumCols); }

cudaError_t launch_row_sums(const float* A, int lda, int m, int n, double* part, double* out, cudaStream_t s) {
  const int nchunks = (n + kRowSumCols - 1) / kRowSumCols;
  k_row_sums_part<<<dim3((m + 127) / 128, nchunks), 128, 0, s>>>(A, lda, m, n, part);
  k_row_sums_reduce<<<(m + 127) / 128, 128, 0, s>>>(part, m, nchunks, out);
  return cudaGetLastError();
}

// ---------------------------------------------------------------- power iteration
// v <- A^T A v / ||A^T A v||; the Rayleigh quotient ||A v||^2 (||v|| = 1) increases to
// ||A||_2^2.  scal[0] holds the largest quotient seen, scal[1] the scale for the next v.
__global__ void k_power_init(float* v, int n) {
  const int stride = gridDim.x * blockDim.x;
  const float inv = rsqrtf((float)n);
  for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < n; j += stride) {
    unsigned h = (unsigned)j * 2654435761u;
    h ^= h >> 15;
    const float r = (float)(h & 0xffff) / 65536.0f;   // [0, 1)
    v[j] = inv * (0.75f + 0.5f * r);
  }
}

cudaError_t launch_power_init(float* v, int n, cudaStream_t s) {
  k_power_init<<<256, 256, 0, s>>>(v, n);
  return cudaGetLastError();
}

__global__ void k_gemv_n_atomic(const float* __restrict__ A, int lda, int m, int n,
                                const float* __restrict__ v, float* q) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const int nch = gridDim.y;
  const int per = (n + nch - 1) / nch;
  const int j0 = blockIdx.y * per, j1 = min(n, j0 + per);
  if (i >= m) return;
  float s = 0.f;
  for (int j = j0; j < j1; ++j) s = fmaf(A[(size_t)j * lda + i], v[j], s);
  atomicAdd(&q[i], s);
}

__global__ void k_gemv_t_warp(const float* __restrict__ A, int lda, int m, int n,
                              const float* __restrict__ q, float* v2) {
  const int lane = threadIdx.x & 31;
  const int wi = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int nw = (gridDim.x * blockDim.x) >> 5;
  for (int j = wi; j < n; j += nw) {
    const float* a = A + (size_t)j * lda;
    float s = 0.f;
    for (int i = lane; i < m; i += 32) s = fmaf(a[i], q[i], s);
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (lane == 0) v2[j] = s;
  }
}

__global__ void k_power_norms(const float* q, int m, const float* v2, int n, double* scal) {
  __shared__ double sh[2][32];
  double a = 0.0, b = 0.0;
  for (int i = threadIdx.x; i < m; i += blockDim.x) a += (double)q[i] * q[i];
  for (int j = threadIdx.x; j < n; j += blockDim.x) b += (double)v2[j] * v2[j];
  a = warp_sum_d(a);
  b = warp_sum_d(b);
  if ((threadIdx.x & 31) == 0) {
    sh[0][threadIdx.x >> 5] = a;
    sh[1][threadIdx.x >> 5] = b;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double qa = 0.0, vb = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) {
      qa += sh[0][w];
      vb += sh[1][w];
    }
    scal[0] = fmax(scal[0], qa);
    scal[1] = vb > 0.0 ? 1.0 / sqrt(vb) : 0.0;
  }
}

__global__ void k_power_scale(float* v, const float* v2, int n, const double* scal) {
  const int stride = gridDim.x * blockDim.x;
  const float sc = (float)scal[1];
  for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < n; j += stride) v[j] = v2[j] * sc;
}

cudaError_t launch_power_step(const float* A, int lda, int m, int n, float* v, float* q, float* v2,
                              double* scal, cudaStream_t s) {
  cudaError_t e = cudaMemsetAsync(q, 0, sizeof(float) * m, s);
  if (e != cudaSuccess) return e;
  const int nch = max(1, min(256, n / 64));
  k_gemv_n_atomic<<<dim3((m + 127) / 128, nch), 128, 0, s>>>(A, lda, m, n, v, q);
  k_gemv_t_warp<<<1024, 256, 0, s>>>(A, lda, m, n, q, v2);
  k_power_norms<<<1, 1024, 0, s>>>(q, m, v2, n, scal);
  k_power_scale<<<256, 256, 0, s>>>(v, v2, n, scal);
  return cudaGetLastError();
}


// ---------------------------------------------------------------- Lanczos on A^T A, one launch
// The step constant needs the largest eigenvalue of M = A^T A.  Lanczos (Golub & Van Loan,
// Matrix Computations, Algorithm 10.1.1) builds the tridiagonal T_K = tridiag(beta; alpha;
// beta) of M on the Krylov space of the start vector; the largest eigenvalue of T_K is a
// Rayleigh quotient of M, so it never exceeds lambda_max(M), and it converges much faster
// in K than the power method's quotient.  One CTA per SM owns a contiguous range of
// columns and keeps its parts of v_k, v_{k-1} and w in shared memory.  Iteration it has two
// phases, each ended by a grid barrier:
//   columns  for it > 0: u = A^T q_it (q_it = A v_it in shared memory; warp per column),
//            alpha_it = ||q_it||^2 = v_it^T M v_it, w = u - alpha_it v_it - beta_{it-1} v_{it-1};
//            at it = 0 w is the start vector.  Then the CTA's partial of ||w||^2 and of A w
//            over its columns (threads over rows, eight column loads in flight);
//   rows     every CTA sums the ||w||^2 partials in the same order: beta_it = ||w||,
//            v_{it+1} = w / beta_it, q_{it+1} = A v_{it+1} = (sum of the partials) / beta_it,
//            formed in 32-row slices over the CTAs with the slice partials of ||q||^2.
// float32 vectors and products, float64 reductions; ab[2 i] = alpha_i and ab[2 i + 1] =
// beta_i (i = 1..K) are written for the host, which bounds the largest eigenvalue of T_K.
// No reorthogonalisation: the lost orthogonality only adds copies of converged Ritz values.
constexpr int kPowThreads = 512;
constexpr int kPowChunks = 4;   // float4 row chunks per thread: lda <= 4 * 4 * 512 = 8192

__global__ void __launch_bounds__(kPowThreads, 1)
    k_lanczos_coop(const float* __restrict__ A, int lda, int m, int n, const float* v0, float* part, float* q,
                   double* wn2, double* qn2, double* ab, double* scal, unsigned* gb, int K) {
  extern __shared__ __align__(16) float psm[];
  const int lda4 = lda >> 2;
  const int per = (n + gridDim.x - 1) / gridDim.x;
  const int j0 = min(n, (int)blockIdx.x * per), j1 = min(n, j0 + per);
  float* sq = psm;               // q (lda)
  float* sv = psm + lda;         // v_it of the CTA's columns (per)
  float* svp = sv + per;         // v_{it-1}
  float* sw = svp + per;         // w
  __shared__ double s_red[kPowThreads / 32];
  __shared__ float s_part[kPowThreads / 32][32];
  __shared__ int s_ok;
  __shared__ double s_alpha, s_beta;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  constexpr int NW = kPowThreads / 32;
  const int nslices = lda / 32;
  const float4* A4 = reinterpret_cast<const float4*>(A);
  // grid barriers on a monotonic 64-bit arrival count (gb[0..1], zeroed before the launch):
  // barrier number nb completes when the count reaches gridDim.x * nb
  unsigned long long* gcount = reinterpret_cast<unsigned long long*>(gb);
  unsigned long long nbar = 0ull;
  if (tid == 0) {
    s_ok = 1;
    s_beta = 0.0;
  }
  for (int j = j0 + tid; j < j1; j += kPowThreads) {
    sw[j - j0] = v0[j];
    sv[j - j0] = 0.f;
    svp[j - j0] = 0.f;
  }
  __syncthreads();
  auto barrier = [&]() -> bool {
    __syncthreads();
    if (tid == 0 && !grid_count_sync(gcount, (unsigned long long)gridDim.x * ++nbar, kGridWaitCycles)) s_ok = 0;
    __syncthreads();
    return s_ok != 0;
  };
  for (int it = 0; it <= K; ++it) {
    // ---- columns
    if (it > 0) {
      if (warp == 0) {   // alpha_it = ||q_it||^2 from the slice partials, same order in every CTA
        double t = 0.0;
        for (int c = lane; c < nslices; c += 32) t += __ldcg(qn2 + c);
        t = warp_sum_d(t);
        if (lane == 0) s_alpha = t;
      }
      for (int i = tid; i < lda; i += kPowThreads) sq[i] = __ldcg(q + i);
      __syncthreads();
      const float alpha = (float)s_alpha, beta = (float)s_beta;
      if (blockIdx.x == 0 && tid == 0) ab[2 * it] = s_alpha;
      if (it == K) break;   // alpha_K is the last coefficient
      const float4* sq4 = reinterpret_cast<const float4*>(sq);
      for (int j = j0 + warp; j < j1; j += NW) {
        const float4* a = A4 + (size_t)j * lda4;
        float s0 = 0.f, s1 = 0.f;
        for (int c = lane; c < lda4; c += 32) {
          const float4 av = a[c], qv = sq4[c];
          s0 = fmaf(av.x, qv.x, s0);
          s1 = fmaf(av.y, qv.y, s1);
          s0 = fmaf(av.z, qv.z, s0);
          s1 = fmaf(av.w, qv.w, s1);
        }
        float s = s0 + s1;
        for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
        if (lane == 0) sw[j - j0] = s - alpha * sv[j - j0] - beta * svp[j - j0];
      }
      __syncthreads();
    }
    {
      double w2 = 0.0;
      for (int j = j0 + tid; j < j1; j += kPowThreads) w2 += (double)sw[j - j0] * (double)sw[j - j0];
      w2 = warp_sum_d(w2);
      if (lane == 0) s_red[warp] = w2;
      __syncthreads();
      if (tid == 0) {
        double t = 0.0;
        for (int w = 0; w < NW; ++w) t += s_red[w];
        wn2[blockIdx.x] = t;
      }
    }
    float4 acc[kPowChunks];
#pragma unroll
    for (int k = 0; k < kPowChunks; ++k) acc[k] = make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
    for (int k = 0; k < kPowChunks; ++k) {
      const int c = tid + k * kPowThreads;
      if (c >= lda4) continue;
      int j = j0;
      for (; j + 8 <= j1; j += 8) {
        float4 a[8];
#pragma unroll
        for (int u = 0; u < 8; ++u) a[u] = A4[(size_t)(j + u) * lda4 + c];
#pragma unroll
        for (int u = 0; u < 8; ++u) {
          const float vj = sw[j + u - j0];
          acc[k].x = fmaf(a[u].x, vj, acc[k].x);
          acc[k].y = fmaf(a[u].y, vj, acc[k].y);
          acc[k].z = fmaf(a[u].z, vj, acc[k].z);
          acc[k].w = fmaf(a[u].w, vj, acc[k].w);
        }
      }
      for (; j < j1; ++j) {
        const float4 a = A4[(size_t)j * lda4 + c];
        const float vj = sw[j - j0];
        acc[k].x = fmaf(a.x, vj, acc[k].x);
        acc[k].y = fmaf(a.y, vj, acc[k].y);
        acc[k].z = fmaf(a.z, vj, acc[k].z);
        acc[k].w = fmaf(a.w, vj, acc[k].w);
      }
    }
    float4* p4 = reinterpret_cast<float4*>(part + (size_t)blockIdx.x * lda);
#pragma unroll
    for (int k = 0; k < kPowChunks; ++k) {
      const int c = tid + k * kPowThreads;
      if (c < lda4) p4[c] = acc[k];
    }
    if (!barrier()) break;
    // ---- rows: beta_it = ||w||, v_{it+1} = w / beta_it, q_{it+1} = A v_{it+1}
    if (warp == 0) {
      double t = 0.0;
      for (int c = lane; c < (int)gridDim.x; c += 32) t += __ldcg(wn2 + c);
      t = warp_sum_d(t);
      if (lane == 0) {
        const double bt = sqrt(t);
        if (it > 0) s_beta = bt;
        if (it > 0 && blockIdx.x == 0) ab[2 * it + 1] = bt;
        s_red[0] = bt > 0.0 ? 1.0 / bt : 0.0;   // an invariant subspace: v and q become zero
      }
    }
    __syncthreads();
    const float sc = (float)s_red[0];
    for (int j = j0 + tid; j < j1; j += kPowThreads) {
      svp[j - j0] = sv[j - j0];
      sv[j - j0] = sc * sw[j - j0];
    }
    for (int sl = blockIdx.x; sl < nslices; sl += gridDim.x) {
      const int row = sl * 32 + lane;
      float sum = 0.f;
      for (int t = warp; t < (int)gridDim.x; t += NW) sum += __ldcg(part + (size_t)t * lda + row);
      s_part[warp][lane] = sum;
      __syncthreads();
      if (warp == 0) {
        float qi = 0.f;
        for (int w = 0; w < NW; ++w) qi += s_part[w][lane];
        qi *= sc;
        q[row] = qi;
        double q2 = (double)qi * (double)qi;
        q2 = warp_sum_d(q2);
        if (lane == 0) qn2[sl] = q2;
      }
      __syncthreads();
    }
    if (!barrier()) break;
  }
  if (blockIdx.x == 0 && tid == 0 && !s_ok) scal[1] = -1.0;   // a barrier wait gave up: the caller reports it
}

cudaError_t launch_lanczos_coop(const float* A, int lda, int m, int n, const float* v0, float* part, float* q,
                                double* wn2, double* qn2, double* ab, double* scal, unsigned* gb, int K, int grid,
                                cudaStream_t s) {
  if (lda > 4 * kPowChunks * kPowThreads || lda % 32 != 0 || grid < 1 || K < 1) return cudaErrorNotSupported;
  const int per = (n + grid - 1) / grid;
  const size_t sm = sizeof(float) * ((size_t)lda + 3 * (size_t)per);
  cudaError_t e = cudaFuncSetAttribute(k_lanczos_coop, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
  if (e != cudaSuccess) return e;
  int per_sm = 0, dev = 0, sms = 0;
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_lanczos_coop, kPowThreads, sm);
  if (e == cudaSuccess) e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (e != cudaSuccess) return e;
  if (per_sm < 1 || grid > per_sm * sms) return cudaErrorNotSupported;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(grid);
  cfg.blockDim = dim3(kPowThreads);
  cfg.dynamicSmemBytes = sm;
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeCooperative;
  attr[0].val.cooperative = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, k_lanczos_coop, A, lda, m, n, v0, part, q, wn2, qn2, ab, scal, gb, K);
}

}  // namespace bvls
