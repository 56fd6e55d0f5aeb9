// Kernels run once per matrix by bvls_setup: finiteness check, column norms ||a_j||_2
// (used by the sphere test of Eq. (safe_rule)), w = A^T t for the dual translation of
// Section 4.2, the row sums used to build candidate directions t, and a power iteration
// for the step constant L ~ ||A||_2^2.  These run once per matrix; the power iteration,
// a hundred passes over A, runs in one cooperative launch when its shape fits.
//
// The column passes accumulate in double-float (float32 pairs): float64 runs at about one
// operation per clock per SM on this part, so a float64 pass over a 2000 x 10000 matrix
// took ~90 us against a few us for the float32 pairs.  Each lane sums its rows (float4
// chunks lane, lane + 32, ... of a 16-byte aligned column, then the ragged tail; single
// rows otherwise): a chain of at most d = ceil(m / 32) + 5 TwoSum steps, exact up to
// 2 (d+2)^2 u^2 sum |terms|, u = 2^-24; the 32 lane sums meet in a float64 tree.
#include <algorithm>

#include "common.cuh"

namespace bvls {

// With m == lda (every stored row checked) and a 16-byte aligned, float4-divisible array, a
// flat grid-stride sweep with four float4 loads in flight per thread; otherwise a block per
// column (grid-stride) with threads over its rows.  No branch per element, so the loads of a
// thread are not serialised behind one another.
__device__ __forceinline__ int not_finite4(float4 v) {
  return !isfinite(v.x) | !isfinite(v.y) | !isfinite(v.z) | !isfinite(v.w);
}

__global__ void k_check_finite(const float* __restrict__ A, int lda, int m, int n, int* flag) {
  int bad = 0;
  if (m == lda && (lda & 3) == 0 && (reinterpret_cast<uintptr_t>(A) & 15) == 0) {
    const float4* A4 = reinterpret_cast<const float4*>(A);
    const size_t total = (size_t)lda * n / 4;
    const size_t stride = (size_t)gridDim.x * blockDim.x;
    size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    for (; e + 3 * stride < total; e += 4 * stride) {
      float4 v[4];
#pragma unroll
      for (int k = 0; k < 4; ++k) v[k] = A4[e + k * stride];
#pragma unroll
      for (int k = 0; k < 4; ++k) bad |= not_finite4(v[k]);
    }
    for (; e < total; e += stride) bad |= not_finite4(A4[e]);
  } else {
    for (int j = blockIdx.x; j < n; j += gridDim.x) {
      const float* a = A + (size_t)j * lda;
      for (int i = threadIdx.x; i < m; i += blockDim.x) bad |= !isfinite(a[i]);
    }
  }
  if (__syncthreads_or(bad) && threadIdx.x == 0) atomicOr(flag, 1);
}

// l2, u2 (double-float pairs) and jinf (u_j = +inf) from the float64 bounds
__global__ void k_bound_pairs(const double* l, const double* u, float2* l2, float2* u2, uint8_t* jinf, int n) {
  for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < n; j += gridDim.x * blockDim.x) {
    const double uj = u[j];
    l2[j] = df2_from_double(l[j]);
    u2[j] = df2_from_double(uj);
    jinf[j] = isinf(uj) ? 1 : 0;
  }
}

cudaError_t launch_bound_pairs(const double* l, const double* u, float2* l2, float2* u2, uint8_t* jinf, int n,
                               cudaStream_t s) {
  k_bound_pairs<<<std::max(1, std::min(256, (n + 255) / 256)), 256, 0, s>>>(l, u, l2, u2, jinf, n);
  return cudaGetLastError();
}

cudaError_t launch_check_finite(const float* A, int lda, int m, int n, int* flag, cudaStream_t s) {
  k_check_finite<<<1024, 256, 0, s>>>(A, lda, m, n, flag);
  return cudaGetLastError();
}

// one warp per column, double-float accumulation
// ||a_j||_2, stored rounded up: the lane sums carry at most 2 (d+2)^2 u^2 of the sum of
// squares, the float64 tree and square root a few float64 units more, and every use of the
// norm (the sphere test's threshold, the margins of the gap, the translation step) stays
// safe when it is overestimated.  With wneg1, also a_j^T (-1) = -sum_i a_ij in the same
// pass (the operations of k_col_dots with t = -1, so the same values bit for bit).
__global__ void k_col_norms(const float* __restrict__ A, int lda, int m, int n, double* nrm, double* wneg1) {
  const int lane = threadIdx.x & 31;
  const int w = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int nw = (gridDim.x * blockDim.x) >> 5;
  const double d = (double)((m + 31) / 32 + 5);
  const double up = 1.0 + 2.0 * (d + 2.0) * (d + 2.0) * 0x1p-48 + 16.0 * 0x1p-53;
  for (int j = w; j < n; j += nw) {
    const float* a = A + (size_t)j * lda;
    float s = 0.f, c = 0.f, ts = 0.f, tc = 0.f;
    int i0 = 0;
    if ((reinterpret_cast<uintptr_t>(a) & 15) == 0) {
      const float4* a4 = reinterpret_cast<const float4*>(a);
      for (int q = lane; q < (m >> 2); q += 32) {
        const float4 v = a4[q];
        df_fma(s, c, v.x, v.x, 0.f);
        df_fma(ts, tc, v.x, -1.f, 0.f);
        df_fma(s, c, v.y, v.y, 0.f);
        df_fma(ts, tc, v.y, -1.f, 0.f);
        df_fma(s, c, v.z, v.z, 0.f);
        df_fma(ts, tc, v.z, -1.f, 0.f);
        df_fma(s, c, v.w, v.w, 0.f);
        df_fma(ts, tc, v.w, -1.f, 0.f);
      }
      i0 = m & ~3;
    }
    for (int i = i0 + lane; i < m; i += 32) {
      const float v = a[i];
      df_fma(s, c, v, v, 0.f);
      df_fma(ts, tc, v, -1.f, 0.f);
    }
    const double ss = warp_sum_d(df_to_double(s, c));
    const double tt = warp_sum_d(df_to_double(ts, tc));
    if (lane == 0) {
      nrm[j] = sqrt(ss) * up;
      if (wneg1) wneg1[j] = tt;
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

// w_j = a_j^T t with t given as double-float pairs (launch_split_pairs); one warp per
// column, the lane order of k_col_norms.  |w_j - a_j^T t| <= setup_dot_gamma(m) ||a_j|| ||t||.
__global__ void k_col_dots(const float* __restrict__ A, int lda, int m, int n, const float2* __restrict__ t2,
                           double* w) {
  const int lane = threadIdx.x & 31;
  const int wi = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int nw = (gridDim.x * blockDim.x) >> 5;
  const bool t_al = (reinterpret_cast<uintptr_t>(t2) & 15) == 0;
  for (int j = wi; j < n; j += nw) {
    const float* a = A + (size_t)j * lda;
    float s = 0.f, c = 0.f;
    int i0 = 0;
    if (t_al && (reinterpret_cast<uintptr_t>(a) & 15) == 0) {
      const float4* a4 = reinterpret_cast<const float4*>(a);
      const float4* t4 = reinterpret_cast<const float4*>(t2);
      for (int q = lane; q < (m >> 2); q += 32) {
        const float4 v = a4[q], t01 = t4[2 * q], t23 = t4[2 * q + 1];
        df_fma(s, c, v.x, t01.x, t01.y);
        df_fma(s, c, v.y, t01.z, t01.w);
        df_fma(s, c, v.z, t23.x, t23.y);
        df_fma(s, c, v.w, t23.z, t23.w);
      }
      i0 = m & ~3;
    }
    for (int i = i0 + lane; i < m; i += 32) {
      const float2 t = t2[i];
      df_fma(s, c, a[i], t.x, t.y);
    }
    const double v = warp_sum_d(df_to_double(s, c));
    if (lane == 0) w[j] = v;
  }
}

cudaError_t launch_col_dots(const float* A, int lda, int m, int n, const float2* t2, double* w,
                            cudaStream_t s) {
  k_col_dots<<<1024, 256, 0, s>>>(A, lda, m, n, t2, w);
  return cudaGetLastError();
}

__global__ void k_split_pairs(const double* t, float2* t2, int m) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < m; i += gridDim.x * blockDim.x) {
    const double v = t[i];
    const float h = (float)v;
    t2[i] = make_float2(h, (float)(v - (double)h));
  }
}

cudaError_t launch_split_pairs(const double* t, float2* t2, int m, cudaStream_t s) {
  k_split_pairs<<<(m + 255) / 256, 256, 0, s>>>(t, t2, m);
  return cudaGetLastError();
}

// out_i = sum_j a_ij, deterministic: column chunks of 64 give per-chunk partials (threads
// over rows, columns in order, double-float), then the partials are summed in chunk order
// in float64.  The sums only shape a candidate direction t, whose products A^T t are then
// computed and bounded on their own, so they carry no rounding bound.
constexpr int kRowSumCols = 64;

__global__ void k_row_sums_part(const float* __restrict__ A, int lda, int m, int n, double* part) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= m) return;
  const int j0 = blockIdx.y * kRowSumCols, j1 = min(n, j0 + kRowSumCols);
  float s = 0.f, c = 0.f;
  for (int j = j0; j < j1; ++j) df_add(s, c, A[(size_t)j * lda + i], 0.f);
  part[(size_t)blockIdx.y * m + i] = df_to_double(s, c);
}

// warp per row: lane k sums chunks k, k + 32, ..., then a shuffle tree
__global__ void k_row_sums_reduce(const double* part, int m, int nchunks, double* out) {
  const int i = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
  if (i >= m) return;   // the whole warp
  double s = 0.0;
  for (int c = lane; c < nchunks; c += 32) s += part[(size_t)c * m + i];
  s = warp_sum_d(s);
  if (lane == 0) out[i] = s;
}

size_t row_sums_scratch(int m, int n) { return (size_t)m * ((n + kRowSumCols - 1) / kRowSumCols); }

cudaError_t launch_row_sums(const float* A, int lda, int m, int n, double* part, double* out, cudaStream_t s) {
  const int nchunks = (n + kRowSumCols - 1) / kRowSumCols;
  k_row_sums_part<<<dim3((m + 127) / 128, nchunks), 128, 0, s>>>(A, lda, m, n, part);
  k_row_sums_reduce<<<(m + 7) / 8, 256, 0, s>>>(part, m, nchunks, out);
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
//   columns  for it > 0: u = A^T q_it (q_it = A v_it in shared memory), alpha_it = ||q_it||^2
//            = v_it^T M v_it, w = u - alpha_it v_it - beta_{it-1} v_{it-1}, and the CTA's
//            partial of A w, from one read of its columns: groups of 8 / KC columns are held
//            in registers (threads over rows, KC float4 row chunks per thread, the next group
//            loading meanwhile), their products with q summed over the block give w_j, and
//            the same registers add a_j w_j into the thread's rows of A w.  At it = 0 w is the
//            start vector and only A w is formed.  Then the CTA's partial of ||w||^2;
//   rows     every CTA sums the ||w||^2 partials in the same order: beta_it = ||w||,
//            v_{it+1} = w / beta_it, q_{it+1} = A v_{it+1} = (sum of the partials) / beta_it,
//            formed in 32-row slices over the CTAs with the slice partials of ||q||^2.
// float32 vectors and products, float64 reductions; ab[2 i] = alpha_i and ab[2 i + 1] =
// beta_i (i = 1..K) are written for the host, which bounds the largest eigenvalue of T_K.
// No reorthogonalisation: the lost orthogonality only adds copies of converged Ritz values.
constexpr int kPowThreads = 512;
constexpr int kPowChunks = 4;   // float4 row chunks per thread at most: lda <= 4 * 4 * 512 = 8192

template <int KC>
__global__ void __launch_bounds__(kPowThreads, 1)
    k_lanczos_coop(const float* __restrict__ A, int lda, int m, int n, const float* v0, float* part, float* q,
                   double* wn2, double* qn2, double* ab, double* scal, unsigned* gb, int K) {
  constexpr int G = 8 / KC;   // columns per register group
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
  __shared__ float s_pd[kPowThreads / 32][G];   // warp partials of a group's products with q
  __shared__ float s_w[G];
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
        const double t = warp_load_sum(qn2, nslices);   // loads batched: one L2 round trip
        if (lane == 0) s_alpha = t;
      }
      {
        float4 qv[kPowChunks];
#pragma unroll
        for (int k = 0; k < kPowChunks; ++k) {
          const int c = tid + k * kPowThreads;
          qv[k] = c < lda4 ? __ldcg(reinterpret_cast<const float4*>(q) + c) : make_float4(0.f, 0.f, 0.f, 0.f);
        }
#pragma unroll
        for (int k = 0; k < kPowChunks; ++k) {
          const int c = tid + k * kPowThreads;
          if (c < lda4) reinterpret_cast<float4*>(sq)[c] = qv[k];
        }
      }
      __syncthreads();
      if (blockIdx.x == 0 && tid == 0) ab[2 * it] = s_alpha;
      if (it == K) break;   // alpha_K is the last coefficient
    }
    float4 acc[KC];
#pragma unroll
    for (int k = 0; k < KC; ++k) acc[k] = make_float4(0.f, 0.f, 0.f, 0.f);
    if (it > 0) {
      const float alpha = (float)s_alpha, beta = (float)s_beta;
      const float4* sq4 = reinterpret_cast<const float4*>(sq);
      float4 qr[KC];
#pragma unroll
      for (int k = 0; k < KC; ++k) {
        const int c = tid + k * kPowThreads;
        qr[k] = c < lda4 ? sq4[c] : make_float4(0.f, 0.f, 0.f, 0.f);
      }
      float4 cur[G][KC], nxt[G][KC];
      auto load_group = [&](int jg, float4 (&r)[G][KC]) {
#pragma unroll
        for (int u = 0; u < G; ++u)
#pragma unroll
          for (int k = 0; k < KC; ++k) {
            const int c = tid + k * kPowThreads;
            r[u][k] = (jg + u < j1 && c < lda4) ? A4[(size_t)(jg + u) * lda4 + c] : make_float4(0.f, 0.f, 0.f, 0.f);
          }
      };
      if (j0 < j1) load_group(j0, cur);
      for (int jg = j0; jg < j1; jg += G) {
        if (jg + G < j1) load_group(jg + G, nxt);
        float pd[G];
#pragma unroll
        for (int u = 0; u < G; ++u) {
          float t = 0.f;
#pragma unroll
          for (int k = 0; k < KC; ++k) {
            t = fmaf(cur[u][k].x, qr[k].x, t);
            t = fmaf(cur[u][k].y, qr[k].y, t);
            t = fmaf(cur[u][k].z, qr[k].z, t);
            t = fmaf(cur[u][k].w, qr[k].w, t);
          }
#pragma unroll
          for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
          pd[u] = t;
        }
        if (lane == 0) {
#pragma unroll
          for (int u = 0; u < G; ++u) s_pd[warp][u] = pd[u];
        }
        __syncthreads();
        if (tid < G) {
          const int j = jg + tid;
          float wj = 0.f;
          if (j < j1) {
            float u = 0.f;
            for (int w = 0; w < NW; ++w) u += s_pd[w][tid];
            wj = u - alpha * sv[j - j0] - beta * svp[j - j0];
            sw[j - j0] = wj;
          }
          s_w[tid] = wj;
        }
        __syncthreads();
#pragma unroll
        for (int u = 0; u < G; ++u) {
          const float wj = s_w[u];
#pragma unroll
          for (int k = 0; k < KC; ++k) {
            acc[k].x = fmaf(cur[u][k].x, wj, acc[k].x);
            acc[k].y = fmaf(cur[u][k].y, wj, acc[k].y);
            acc[k].z = fmaf(cur[u][k].z, wj, acc[k].z);
            acc[k].w = fmaf(cur[u][k].w, wj, acc[k].w);
          }
        }
#pragma unroll
        for (int u = 0; u < G; ++u)
#pragma unroll
          for (int k = 0; k < KC; ++k) cur[u][k] = nxt[u][k];
      }
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
    if (it == 0) {   // w = v0: the CTA's partial of A w (eight column loads in flight)
#pragma unroll
      for (int k = 0; k < KC; ++k) {
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
    }
    float4* p4 = reinterpret_cast<float4*>(part + (size_t)blockIdx.x * lda);
#pragma unroll
    for (int k = 0; k < KC; ++k) {
      const int c = tid + k * kPowThreads;
      if (c < lda4) p4[c] = acc[k];
    }
    if (!barrier()) break;
    // ---- rows: beta_it = ||w||, v_{it+1} = w / beta_it, q_{it+1} = A v_{it+1}
    if (warp == 0) {
      const double t = warp_load_sum(wn2, gridDim.x);
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
      for (int t0 = warp; t0 < (int)gridDim.x; t0 += NW * 10) {   // ten loads in flight per lane
        float v[10];
#pragma unroll
        for (int k = 0; k < 10; ++k) {
          const int t = t0 + NW * k;
          v[k] = t < (int)gridDim.x ? __ldcg(part + (size_t)t * lda + row) : 0.f;
        }
#pragma unroll
        for (int k = 0; k < 10; ++k) sum += v[k];
      }
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

// The same iteration for lda <= 2048 with a warp per column: a lane holds rows lane + 32 k
// (float4 chunks, k < 16) of one column in registers, sums its products with q over the warp,
// forms w_j and adds a_j w_j into its own rows of the warp's partial of A w; the next column
// of the warp loads meanwhile.  No block barrier per column: the eight warps' partials meet
// in shared memory once per iteration.  256 threads, up to 255 registers each.
constexpr int kWcThreads = 256;
constexpr int kWcChunks = 16;   // float4 row chunks per lane: lda <= 4 * 32 * 16 = 2048

__global__ void __launch_bounds__(kWcThreads, 1)
    k_lanczos_wc(const float* __restrict__ A, int lda, int m, int n, const float* v0, float* part, float* q,
                 double* wn2, double* qn2, double* ab, double* scal, unsigned* gb, int K) {
  constexpr int NW = kWcThreads / 32;
  constexpr int RC = kWcChunks;
  extern __shared__ __align__(16) float psm[];
  const int lda4 = lda >> 2;
  const int per = (n + gridDim.x - 1) / gridDim.x;
  const int j0 = min(n, (int)blockIdx.x * per), j1 = min(n, j0 + per);
  float* sq = psm;                                              // q (lda)
  float4* sacc = reinterpret_cast<float4*>(psm + lda);          // the warps' partials of A w (NW x lda4)
  float* sv = psm + (size_t)(NW + 1) * lda;                     // v_it of the CTA's columns (per)
  float* svp = sv + per;                                        // v_{it-1}
  float* sw = svp + per;                                        // w
  __shared__ double s_red[NW];
  __shared__ float s_part[NW][32];
  __shared__ int s_ok;
  __shared__ double s_alpha, s_beta;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int nslices = lda / 32;
  const float4* A4 = reinterpret_cast<const float4*>(A);
  unsigned long long* gcount = reinterpret_cast<unsigned long long*>(gb);
  unsigned long long nbar = 0ull;
  if (tid == 0) {
    s_ok = 1;
    s_beta = 0.0;
    s_alpha = 0.0;
  }
  for (int j = j0 + tid; j < j1; j += kWcThreads) {
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
        const double t = warp_load_sum(qn2, nslices);
        if (lane == 0) s_alpha = t;
      }
      {
        float4 qv[2];
#pragma unroll
        for (int k = 0; k < 2; ++k) {
          const int c = tid + k * kWcThreads;
          qv[k] = c < lda4 ? __ldcg(reinterpret_cast<const float4*>(q) + c) : make_float4(0.f, 0.f, 0.f, 0.f);
        }
#pragma unroll
        for (int k = 0; k < 2; ++k) {
          const int c = tid + k * kWcThreads;
          if (c < lda4) reinterpret_cast<float4*>(sq)[c] = qv[k];
        }
      }
      __syncthreads();
      if (blockIdx.x == 0 && tid == 0) ab[2 * it] = s_alpha;
      if (it == K) break;   // alpha_K is the last coefficient
    }
    const float alpha = (float)s_alpha, beta = (float)s_beta;
    const float4* sq4 = reinterpret_cast<const float4*>(sq);
    float4 acc[RC];
#pragma unroll
    for (int k = 0; k < RC; ++k) acc[k] = make_float4(0.f, 0.f, 0.f, 0.f);
    auto load_col = [&](int j, float4 (&r)[RC]) {
#pragma unroll
      for (int k = 0; k < RC; ++k) {
        const int c = lane + 32 * k;
        r[k] = c < lda4 ? A4[(size_t)j * lda4 + c] : make_float4(0.f, 0.f, 0.f, 0.f);
      }
    };
    auto body = [&](int j, const float4 (&r)[RC]) {
      float wj;
      if (it > 0) {
        float d0 = 0.f, d1 = 0.f;
#pragma unroll
        for (int k = 0; k < RC; ++k) {
          const int c = lane + 32 * k;
          if (c < lda4) {
            const float4 qk = sq4[c];
            d0 = fmaf(r[k].x, qk.x, d0);
            d1 = fmaf(r[k].y, qk.y, d1);
            d0 = fmaf(r[k].z, qk.z, d0);
            d1 = fmaf(r[k].w, qk.w, d1);
          }
        }
        float u = d0 + d1;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) u += __shfl_xor_sync(0xffffffffu, u, o);
        wj = u - alpha * sv[j - j0] - beta * svp[j - j0];
        if (lane == 0) sw[j - j0] = wj;
      } else {
        wj = sw[j - j0];   // w = v0
      }
#pragma unroll
      for (int k = 0; k < RC; ++k) {
        acc[k].x = fmaf(r[k].x, wj, acc[k].x);
        acc[k].y = fmaf(r[k].y, wj, acc[k].y);
        acc[k].z = fmaf(r[k].z, wj, acc[k].z);
        acc[k].w = fmaf(r[k].w, wj, acc[k].w);
      }
    };
    {
      float4 ca[RC], cb[RC];
      int j = j0 + warp;
      if (j < j1) load_col(j, ca);
      for (; j < j1; j += 2 * NW) {
        if (j + NW < j1) load_col(j + NW, cb);
        body(j, ca);
        if (j + NW >= j1) break;
        if (j + 2 * NW < j1) load_col(j + 2 * NW, ca);
        body(j + NW, cb);
      }
    }
#pragma unroll
    for (int k = 0; k < RC; ++k) {
      const int c = lane + 32 * k;
      if (c < lda4) sacc[(size_t)warp * lda4 + c] = acc[k];
    }
    __syncthreads();
    {
      double w2 = 0.0;
      for (int j = j0 + tid; j < j1; j += kWcThreads) w2 += (double)sw[j - j0] * (double)sw[j - j0];
      w2 = warp_sum_d(w2);
      if (lane == 0) s_red[warp] = w2;
    }
    float4* p4 = reinterpret_cast<float4*>(part + (size_t)blockIdx.x * lda);
    for (int c = tid; c < lda4; c += kWcThreads) {   // the warps' partials, in warp order
      float4 t = sacc[c];
#pragma unroll
      for (int w = 1; w < NW; ++w) {
        const float4 o = sacc[(size_t)w * lda4 + c];
        t.x += o.x;
        t.y += o.y;
        t.z += o.z;
        t.w += o.w;
      }
      p4[c] = t;
    }
    __syncthreads();
    if (tid == 0) {
      double t = 0.0;
      for (int w = 0; w < NW; ++w) t += s_red[w];
      wn2[blockIdx.x] = t;
    }
    if (!barrier()) break;
    // ---- rows: beta_it = ||w||, v_{it+1} = w / beta_it, q_{it+1} = A v_{it+1}
    if (warp == 0) {
      const double t = warp_load_sum(wn2, gridDim.x);
      if (lane == 0) {
        const double bt = sqrt(t);
        if (it > 0) s_beta = bt;
        if (it > 0 && blockIdx.x == 0) ab[2 * it + 1] = bt;
        s_red[0] = bt > 0.0 ? 1.0 / bt : 0.0;   // an invariant subspace: v and q become zero
      }
    }
    __syncthreads();
    const float sc = (float)s_red[0];
    for (int j = j0 + tid; j < j1; j += kWcThreads) {
      svp[j - j0] = sv[j - j0];
      sv[j - j0] = sc * sw[j - j0];
    }
    for (int sl = blockIdx.x; sl < nslices; sl += gridDim.x) {
      const int row = sl * 32 + lane;
      float sum = 0.f;
      for (int t0 = warp; t0 < (int)gridDim.x; t0 += NW * 10) {   // ten loads in flight per lane
        float v[10];
#pragma unroll
        for (int k = 0; k < 10; ++k) {
          const int t = t0 + NW * k;
          v[k] = t < (int)gridDim.x ? __ldcg(part + (size_t)t * lda + row) : 0.f;
        }
#pragma unroll
        for (int k = 0; k < 10; ++k) sum += v[k];
      }
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

// Cooperative launch of a Lanczos kernel: one CTA per SM at most (grid <= what fits).
static cudaError_t lanczos_launch(const void* fn, int threads, size_t sm, const float* A, int lda, int m, int n,
                                  const float* v0, float* part, float* q, double* wn2, double* qn2, double* ab,
                                  double* scal, unsigned* gb, int K, int grid, cudaStream_t s) {
  cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
  if (e != cudaSuccess) return e;
  int per_sm = 0, dev = 0, sms = 0;
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, threads, sm);
  if (e == cudaSuccess) e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (e != cudaSuccess) return e;
  if (per_sm < 1 || grid > per_sm * sms) return cudaErrorNotSupported;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(grid);
  cfg.blockDim = dim3(threads);
  cfg.dynamicSmemBytes = sm;
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeCooperative;
  attr[0].val.cooperative = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  void* args[] = {&A, &lda, &m, &n, &v0, &part, &q, &wn2, &qn2, &ab, &scal, &gb, &K};
  return cudaLaunchKernelExC(&cfg, fn, args);
}

cudaError_t launch_lanczos_coop(const float* A, int lda, int m, int n, const float* v0, float* part, float* q,
                                double* wn2, double* qn2, double* ab, double* scal, unsigned* gb, int K, int grid,
                                cudaStream_t s) {
  if (lda > 4 * kPowChunks * kPowThreads || lda % 32 != 0 || grid < 1 || K < 1) return cudaErrorNotSupported;
  const int lda4 = lda / 4;
  const int per = (n + grid - 1) / grid;
  if (lda4 <= 32 * kWcChunks) {
    const size_t sm = sizeof(float) * ((size_t)(kWcThreads / 32 + 1) * lda + 3 * (size_t)per);
    return lanczos_launch(reinterpret_cast<const void*>(k_lanczos_wc), kWcThreads, sm, A, lda, m, n, v0, part, q,
                          wn2, qn2, ab, scal, gb, K, grid, s);
  }
  const size_t sm = sizeof(float) * ((size_t)lda + 3 * (size_t)per);
  const void* fn = lda4 <= 2 * kPowThreads ? reinterpret_cast<const void*>(k_lanczos_coop<2>)
                                           : reinterpret_cast<const void*>(k_lanczos_coop<4>);
  return lanczos_launch(fn, kPowThreads, sm, A, lda, m, n, v0, part, q, wn2, qn2, ab, scal, gb, K, grid, s);
}

}  // namespace bvls
