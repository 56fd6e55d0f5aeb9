// bvls_solve_static: the single-instance solve for callers that cannot allocate device
// memory (for example code running inside a memory pool it does not own, or in a process
// whose allocator is fixed by its host application at start-up).  It uses the same
// per-iteration kernels as bvls_setup + bvls_solve (the single pass and its residual, or the
// two passes for large m, then the gap, test and compaction kernels), launched one by one:
// the step constant comes from power steps instead of the Lanczos launch, and neither the
// persistent form nor CUDA graphs are used.  Every scratch buffer lives in one file-scope
// device array of fixed size, so the call allocates nothing: no cudaMalloc, cudaFree,
// pinned host memory, CUDA graphs or events.
//
// The array (kStaticBytes) is part of the library image: every GPU that loads the library
// holds it until the process exits.  All calls share it and it keeps the last call's
// contents; each call clears what must start at zero.  Calls whose GPU work overlaps (two
// host threads, or two streams) race on it and must be serialised by the caller.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <mutex>

#include "bvls_gb300.h"
#include "common.cuh"

using namespace bvls;

namespace {

constexpr size_t kStaticBytes = size_t(8) << 20;  // 8 MiB
constexpr int kStaticMaxM = 4096;
constexpr int kStaticMaxN = 16384;
constexpr int kMaxDevices = 64;

__device__ __align__(256) unsigned char g_scratch[kStaticBytes];

// Device address of g_scratch per device, looked up once per device with that device
// current.  The lookup is serialised by a mutex, so two host threads making their first call
// on one device do not race.  A cached address belongs to the device's current context:
// after cudaDeviceReset the process must not call this entry point again on that device.
void* g_scratch_dev[kMaxDevices] = {nullptr};
std::mutex g_scratch_mu;

constexpr double kU = 5.9604644775390625e-08;
constexpr double kU64 = 1.1102230246251565e-16;


struct Arena {
  unsigned char* base;
  size_t used;
  template <typename T>
  T* take(size_t count) {
    used = (used + 255) & ~size_t(255);
    T* p = reinterpret_cast<T*>(base ? base + used : nullptr);
    used += count * sizeof(T) + 16;
    return p;
  }
};

__global__ void k_fill_bounds(double* l, double* u, float2* l2, float2* u2, uint8_t* jinf, int n,
                              int have_l, int have_u) {
  for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < n; j += gridDim.x * blockDim.x) {
    if (!have_l) l[j] = 0.0;
    if (!have_u) u[j] = INFINITY;
    jinf[j] = isinf(u[j]) ? 1 : 0;
    l2[j] = df2_from_double(l[j]);
    u2[j] = df2_from_double(u[j]);
  }
}

// bad = 1 unless a_j^T t < 0 (with its rounding bound) on every nonzero column of J_inf.
__global__ void k_dir_check(const double* w, const double* nrm, const uint8_t* jinf, int n,
                            double gamma_tn, int* bad) {
  int b = 0;
  for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < n; j += gridDim.x * blockDim.x)
    if (jinf[j] && nrm[j] > 0.0 && !(w[j] + gamma_tn * nrm[j] < 0.0)) b = 1;
  if (__syncthreads_or(b) && threadIdx.x == 0) atomicOr(bad, 1);
}

struct Layout {
  Buffers b;
  double *l, *u, *nrm, *w, *scal;
  float2 *l2, *u2;
  uint8_t* jinf;
  float *y, *v, *v2, *q;
  double* x0;
  int* flag;
  size_t bytes;
};

Layout carve(unsigned char* base, int m, int n, int m4, int lda, int fwd_tiles, int fwd_chunks,
             int max_blocks, int sms) {
  Arena a{base, 0};
  Layout L{};
  L.b.x[0] = a.take<float2>(n);
  L.b.x[1] = a.take<float2>(n);
  L.b.g[0] = a.take<float2>(n);
  L.b.g[1] = a.take<float2>(n);
  L.b.idx = a.take<int>(n);
  L.b.idx_tmp = a.take<int>(n);
  L.b.fold = a.take<int>(n);
  L.b.flags = a.take<uint8_t>(n);
  L.b.yh = a.take<float>(m4);
  L.b.yl = a.take<float>(m4);
  L.b.rh = a.take<float>(m4);
  L.b.rl = a.take<float>(m4);
  L.b.part = a.take<float2>((size_t)fwd_chunks * lda);
  L.b.tileP = a.take<double>((lda + 31) / 32);
  L.b.tileR = a.take<double>((m4 + 31) / 32);
  L.b.tile_cnt = a.take<unsigned int>(fwd_tiles);
  L.b.blk = a.take<double>(4 * (size_t)max_blocks);
  L.b.st = a.take<DevState>(1);
  L.b.qpart = a.take<float2>((size_t)sms * m4);
  L.b.xout = a.take<double>(n);
  L.l = a.take<double>(n);
  L.u = a.take<double>(n);
  L.l2 = a.take<float2>(n);
  L.u2 = a.take<float2>(n);
  L.nrm = a.take<double>(n);
  L.w = a.take<double>(n);
  L.jinf = a.take<uint8_t>(n);
  L.scal = a.take<double>(2);
  L.y = a.take<float>(m4);
  L.x0 = a.take<double>(n);
  L.v = a.take<float>(n);
  L.v2 = a.take<float>(n);
  L.q = a.take<float>(m);
  L.flag = a.take<int>(2);   // [0] non-finite A, [1] t not interior
  L.bytes = a.used;
  return L;
}

bvls_status fail(bvls_status s, const char* what, cudaError_t e = cudaSuccess) {
  char msg[256];
  if (e != cudaSuccess) snprintf(msg, sizeof(msg), "%s: %s", what, cudaGetErrorString(e));
  else snprintf(msg, sizeof(msg), "%s", what);
  record_error(msg);
  return s;
}

#define SCK(call)                                                                        \
  do {                                                                                   \
    cudaError_t e_ = (call);                                                             \
    if (e_ != cudaSuccess) return fail(BVLS_ECUDA, #call, e_);                           \
  } while (0)

}  // namespace

extern "C" {

bvls_status bvls_solve_static(const float* A, int m, int n, int lda, const double* l,
                              const double* u, const float* y, const double* x0,
                              const bvls_opts* opts, void* stream, double* x_out,
                              uint8_t* screened_out, bvls_info* info) {
  record_error("");
  if (!A || !y || !x_out || m < 1 || n < 1 || lda < m)
    return fail(BVLS_EINVAL, "need A, y, x_out, m >= 1, n >= 1, lda >= m");
  if (m > kStaticMaxM || n > kStaticMaxN)
    return fail(BVLS_ENOTSUP, "bvls_solve_static handles m <= 4096 and n <= 16384; use bvls_setup");
  if (lda % 32 != 0) return fail(BVLS_EINVAL, "bvls_solve_static needs lda a multiple of 32");
  if (reinterpret_cast<uintptr_t>(A) % 16 != 0)
    return fail(BVLS_EINVAL, "bvls_solve_static needs A aligned to 16 bytes");
  bvls_opts o;
  bvls_default_opts(&o);
  if (opts) o = *opts;
  if (!(o.tol >= 0.0) || o.screen_every < 1 || o.max_iter < 1 ||
      (o.precision != BVLS_PREC_FP32X2 && o.precision != BVLS_PREC_FP32 && o.precision != BVLS_PREC_MIXED) ||
      !(o.lipschitz >= 0.0) ||
      !std::isfinite(o.lipschitz) || o.single_pass < 0 || o.single_pass > 2)
    return fail(BVLS_EINVAL, "invalid options");
  if (o.algorithm != BVLS_ALG_FISTA)
    return fail(BVLS_ENOTSUP, "bvls_solve_static runs FISTA only (opts->algorithm = BVLS_ALG_FISTA)");
  bool any_inf = false;
  for (int j = 0; j < n; ++j) {
    const double lj = l ? l[j] : 0.0, uj = u ? u[j] : INFINITY;
    if (!std::isfinite(lj) || std::isnan(uj) || uj == -INFINITY || lj > uj)
      return fail(BVLS_EINVAL, "need finite l_j <= u_j (u_j may be +inf)");
    any_inf |= std::isinf(uj);
  }
  cudaPointerAttributes pa;
  if (cudaPointerGetAttributes(&pa, A) != cudaSuccess || pa.type != cudaMemoryTypeDevice) {
    cudaGetLastError();
    return fail(BVLS_EINVAL, "bvls_solve_static reads A in place: A must be device memory");
  }
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  int dev = 0, sms = 0, optin = 0;
  SCK(cudaGetDevice(&dev));
  if (dev >= kMaxDevices) return fail(BVLS_ENOTSUP, "device index too large");
  // Once per device, with that device current: the device address of the static array.
  void* scratch = nullptr;
  {
    std::lock_guard<std::mutex> lock(g_scratch_mu);
    if (!g_scratch_dev[dev]) {
      void* ptr = nullptr;
      cudaError_t e = cudaGetSymbolAddress(&ptr, g_scratch);
      if (e != cudaSuccess || !ptr) return fail(BVLS_ECUDA, "cudaGetSymbolAddress(g_scratch)", e);
      g_scratch_dev[dev] = ptr;
    }
    scratch = g_scratch_dev[dev];
  }
  SCK(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  SCK(cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev));

  const int m4 = (m + 3) / 4 * 4;
  const int fwd_tiles = (lda + kFwdRows - 1) / kFwdRows;
  int fwd_chunks = (4 * sms + fwd_tiles - 1) / fwd_tiles;
  fwd_chunks = std::max(1, std::min(std::min(fwd_chunks, std::max(1, (n + 7) / 8)), 64));
  int bps = 1;
  SCK(tr_configure(m4, &bps));
  const int tr_blocks = sms * std::max(1, std::min(bps, 2));
  const int red_blocks = std::max(1, std::min(2 * sms, (n + kRedThreads - 1) / kRedThreads));
  const int max_blocks = std::max(std::max(tr_blocks, red_blocks), std::max(64, sms));
  int pass_qw = 0, pass_cps = 1;
  const int pass_stages = pass_configure(lda, m4, (n + sms - 1) / sms, optin, &pass_qw, &pass_cps);
  cudaGetLastError();

  const Layout need = carve(nullptr, m, n, m4, lda, fwd_tiles, fwd_chunks, max_blocks, sms);
  if (need.bytes > kStaticBytes) {
    char msg[160];
    snprintf(msg, sizeof(msg), "problem needs %zu bytes of scratch > %zu static bytes", need.bytes,
             kStaticBytes);
    return fail(BVLS_ENOTSUP, msg);
  }
  Layout W = carve(static_cast<unsigned char*>(scratch), m, n, m4, lda, fwd_tiles, fwd_chunks,
                   max_blocks, sms);
  Buffers& b = W.b;

  // Clear what must start at zero (the array keeps the previous call's contents).
  SCK(cudaMemsetAsync(b.tile_cnt, 0, sizeof(unsigned) * fwd_tiles, s));
  SCK(cudaMemsetAsync(b.st, 0, sizeof(DevState), s));
  SCK(cudaMemsetAsync(W.y, 0, sizeof(float) * m4, s));
  SCK(cudaMemsetAsync(W.w, 0, sizeof(double) * n, s));
  SCK(cudaMemsetAsync(W.flag, 0, 2 * sizeof(int), s));

  // Setup: finiteness of every stored row, bounds, column norms, dual direction, L.
  SCK(launch_check_finite(A, lda, lda, n, W.flag, s));
  if (l) SCK(cudaMemcpyAsync(W.l, l, sizeof(double) * n, cudaMemcpyHostToDevice, s));
  if (u) SCK(cudaMemcpyAsync(W.u, u, sizeof(double) * n, cudaMemcpyHostToDevice, s));
  k_fill_bounds<<<64, 256, 0, s>>>(W.l, W.u, W.l2, W.u2, W.jinf, n, l != nullptr, u != nullptr);
  SCK(cudaGetLastError());
  // with an infinite upper bound, the same pass gives w = A^T t for t = -1 (Proposition 2,
  // case 3), as bvls_setup tries first; otherwise theta = 0
  SCK(launch_col_norms(A, lda, m, n, W.nrm, s, any_inf ? W.w : nullptr));
  int dual_mode = kScaling;
  double t_norm = 0.0, gamma_w = 0.0;
  if (any_inf) {
    t_norm = std::sqrt((double)m);
    gamma_w = setup_dot_gamma(m);
    k_dir_check<<<64, 256, 0, s>>>(W.w, W.nrm, W.jinf, n, gamma_w * t_norm, W.flag + 1);
    SCK(cudaGetLastError());
  }
  int flags[2] = {0, 0};
  SCK(cudaMemcpyAsync(flags, W.flag, 2 * sizeof(int), cudaMemcpyDeviceToHost, s));
  SCK(cudaStreamSynchronize(s));
  if (flags[0]) return fail(BVLS_ENONFINITE, "A contains NaN or Inf");
  if (any_inf) {
    dual_mode = flags[1] ? kZero : kTranslation;
    if (flags[1]) t_norm = gamma_w = 0.0;
  }
  double Lc = o.lipschitz;
  if (!(Lc > 0.0)) {
    SCK(cudaMemsetAsync(W.scal, 0, 2 * sizeof(double), s));
    SCK(launch_power_init(W.v, n, s));
    SCK(launch_power_step(A, lda, m, n, W.v, W.q, W.v2, W.scal, s));
    SCK(cudaMemsetAsync(W.scal, 0, sizeof(double), s));
    for (int it = 0; it < 100; ++it) SCK(launch_power_step(A, lda, m, n, W.v, W.q, W.v2, W.scal, s));
    double lam = 0.0;
    SCK(cudaMemcpyAsync(&lam, W.scal, sizeof(double), cudaMemcpyDeviceToHost, s));
    SCK(cudaStreamSynchronize(s));
    Lc = lam > 0.0 ? 1.05 * lam : 1.0;
  }

  // Parameters (rounding constants as in bvls_setup).
  Params p{};
  p.A = A;
  p.m = m;
  p.n = n;
  p.lda = lda;
  p.m4 = m4;
  p.l = W.l;
  p.u = W.u;
  p.nrm = W.nrm;
  p.w = W.w;
  p.jinf = W.jinf;
  p.l2 = W.l2;
  p.u2 = W.u2;
  p.invL = 1.0 / Lc;
  p.invL2 = df2_from_double(p.invL);
  p.grid_wait = kGridWaitCycles;
  p.t_norm = t_norm;
  p.gamma_w = gamma_w;
  {
    const int d_g = (m4 / 4 + 31) / 32 + 7;
    const int per = (n + fwd_chunks - 1) / fwd_chunks;
    const int d_f0 = ((per + kFwdWarps - 1) / kFwdWarps + 1) / 2 + 4 + fwd_chunks + 1;
    const int d_f = std::max(d_f0, (n + sms - 1) / sms + (sms + 7) / 8 + 8);
    p.Cg = o.precision == BVLS_PREC_FP32X2 ? 2.0 * (d_g + 2.0) * (d_g + 2.0) * kU * kU + 4.0 * kU * kU + 2.0 * kU64
                                           : 1.01 * (d_g + 2.0) * kU + kU;
    p.Cf = o.precision != BVLS_PREC_FP32 ? 2.0 * (d_f + 2.0) * (d_f + 2.0) * kU * kU + 2.0 * kU * kU
                                         : 1.01 * (d_f + 2.0) * kU + kU;
    // mode MIXED: the pass sums each stage's columns in float32 before a double-float merge
    if (o.precision == BVLS_PREC_MIXED) p.Cf = 1.01 * (std::max(1, pass_cps) + 1.0) * kU + 1.01 * p.Cf;
    p.Csub = 8.0 * kU * kU;
  }
  const int K = o.screen_every;
  const int max_iter = (int)std::min<long long>((long long)(o.max_iter + K - 1) / K * K, 0x7fffffff);
  p.tol = o.tol;
  p.max_iter = max_iter;
  p.dual_mode = dual_mode;
  p.screening = o.screening;
  p.restart = o.restart;
  p.fwd_chunks = fwd_chunks;
  p.fwd_tiles = fwd_tiles;

  // Solve: direct launches (a captured graph would allocate), a chunk at a time.
  SCK(cudaMemcpyAsync(W.y, y, sizeof(float) * m, cudaMemcpyDefault, s));
  b.y_in = W.y;
  b.x0_in = nullptr;
  if (x0) {
    SCK(cudaMemcpyAsync(W.x0, x0, sizeof(double) * n, cudaMemcpyDefault, s));
    b.x0_in = W.x0;
  }
  SCK(launch_init(p, b, s));
  const bool fused = pass_stages > 0 && o.single_pass;
  if (fused) SCK(launch_fwd(p, b, 0, o.precision, false, s));
  const bool scr = o.screening && dual_mode != kZero;
  int chunk = K;
  while (chunk < 16 || chunk % 2) chunk += K;
  const long long max_chunks = (max_iter + chunk - 1) / chunk + 1;
  long long launches = fused ? 3 : 2;
  DevState hs;
  for (long long c = 0; c < max_chunks; ++c) {
    for (int j = 0; j < chunk; ++j) {
      const int slot = j & 1;
      const bool gap_iter = ((j + 1) % K) == 0;
      if (fused) {
        SCK(launch_pass(p, b, slot, o.precision, gap_iter, sms, pass_stages, pass_cps, pass_qw, s));
        SCK(launch_resid(p, b, slot, sms, s));
      } else {
        SCK(launch_fwd(p, b, slot, o.precision, false, s));
        SCK(launch_tr(p, b, slot, o.precision, gap_iter, tr_blocks, s));
      }
      launches += 2;
      if (gap_iter) {
        SCK(launch_gap(p, b, slot, !scr, red_blocks, s));
        ++launches;
        if (scr) {
          SCK(launch_test(p, b, slot, red_blocks, s));
          SCK(launch_compact(p, b, slot, s));
          SCK(launch_fwd(p, b, slot, o.precision, true, s));
          launches += 3;
        }
      }
    }
    SCK(cudaMemcpyAsync(&hs, b.st, sizeof(DevState), cudaMemcpyDeviceToHost, s));
    SCK(cudaStreamSynchronize(s));
    if (hs.done) break;
  }
  if (hs.nonfinite) return fail(BVLS_ENONFINITE, "y or x0 contains NaN or Inf");
  if (hs.error) return fail(BVLS_ETIMEOUT, "a device-side wait exceeded its bound; results discarded");
  SCK(launch_export(p, b, hs.out_slot, s));
  SCK(cudaMemcpyAsync(x_out, b.xout, sizeof(double) * n, cudaMemcpyDefault, s));
  if (screened_out) SCK(cudaMemcpyAsync(screened_out, b.flags, n, cudaMemcpyDefault, s));
  SCK(cudaStreamSynchronize(s));
  if (info) {
    std::memset(info, 0, sizeof(*info));
    info->iters = hs.k;
    info->converged = hs.converged;
    info->n_preserved = hs.n_active;
    info->dual_mode = dual_mode;
    info->gap_evals = hs.gap_evals;
    info->gap = hs.gap;
    info->primal = hs.P[hs.out_slot];
    info->radius = hs.radius;
    info->L = Lc;
    info->sum_preserved = hs.sum_active;
    info->sum_nonzero = hs.sum_nnz;
    info->kernel_launches = (double)launches;
    info->single_pass = fused ? 1 : 0;
  }
  if (!hs.done || !hs.converged) {
    char msg[128];
    snprintf(msg, sizeof(msg), "gap %.3e >= tol after %d iterations", hs.gap, hs.k);
    return fail(BVLS_EMAXITER, msg);
  }
  return BVLS_OK;
}

}  // extern "C"
