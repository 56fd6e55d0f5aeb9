// Kernels run once per matrix by bvls_setup: finiteness check, column norms ||a_j||_2
// (used by the sphere test of Eq. (safe_rule)), w = A^T t for the dual translation of
// Section 4.2, the row sums used to build candidate directions t, and a power iteration
// for the step constant L ~ ||A||_2^2.  These run once, so they favour plainness (float64
// accumulation, simple mappings) over speed.
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
__global__ void k_col_norms(const float* __restrict__ A, int lda, int m, int n, double* nrm) {
  const int lane = threadIdx.x & 31;
  const int w = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int nw = (gridDim.x * blockDim.x) >> 5;
  for (int j = w; j < n; j += nw) {
    const float* a = A + (size_t)j * lda;
    double s = 0.0;
    for (int i = lane; i < m; i += 32) s = fma((double)a[i], (double)a[i], s);
    s = warp_sum_d(s);
    if (lane == 0) nrm[j] = sqrt(s);
  }
}

cudaError_t launch_col_norms(const float* A, int lda, int m, int n, double* nrm, cudaStream_t s) {
  k_col_norms<<<1024, 256, 0, s>>>(A, lda, m, n, nrm);
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

// out_i = sum_j a_ij, deterministic: thread per row, columns in order.
__global__ void k_row_sums(const float* __restrict__ A, int lda, int m, int n, double* out) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= m) return;
  double s = 0.0;
  for (int j = 0; j < n; ++j) s += (double)A[(size_t)j * lda + i];
  out[i] = s;
}

cudaError_t launch_row_sums(const float* A, int lda, int m, int n, double* out, cudaStream_t s) {
  k_row_sums<<<(m + 127) / 128, 128, 0, s>>>(A, lda, m, n, out);
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

}  // namespace bvls
