// C ABI: handle management, setup and the solve loop (CUDA-graph chunks of iterations).
#include <algorithm>
#include <map>
#include <mutex>
#include <tuple>
#include <chrono>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include <cudaTypedefs.h>

#include "backward.cuh"
#include "batch.cuh"
#include "ragged.cuh"
#include "refine.cuh"
#include "bvls_gb300.h"
#include "common.cuh"

using namespace bvls;

namespace {

thread_local std::string g_err;

bvls_status set_err(bvls_status s, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof(buf), fmt, ap);
  va_end(ap);
  g_err = buf;
  return s;
}

#define CK(call)                                                                          \
  do {                                                                                    \
    cudaError_t e_ = (call);                                                              \
    if (e_ != cudaSuccess)                                                                \
      return set_err(e_ == cudaErrorMemoryAllocation ? BVLS_ENOMEM : BVLS_ECUDA,         \
                     "%s failed: %s (line %d)", #call, cudaGetErrorString(e_), __LINE__); \
  } while (0)

constexpr double kU = 5.9604644775390625e-08;   // 2^-24, unit roundoff of float32
constexpr double kU64 = 1.1102230246251565e-16; // 2^-53

constexpr int kGraphCache = 4;   // solve graphs kept per handle

struct GraphKey {
  int K, screening, precision, restart, max_iter, single_pass, algorithm;
  double tol, invL, eps_star, eta_star;
  bool fixed_dual;
  bool operator==(const GraphKey& o) const {
    return K == o.K && screening == o.screening && precision == o.precision &&
           restart == o.restart && max_iter == o.max_iter && single_pass == o.single_pass &&
           algorithm == o.algorithm &&
           tol == o.tol && invL == o.invL && eps_star == o.eps_star && eta_star == o.eta_star &&
           fixed_dual == o.fixed_dual;
  }
};

}  // namespace

struct bvls_handle {
  int m = 0, n = 0, lda = 0, m4 = 0, num_sms = 0;
  cudaStream_t user = nullptr, s = nullptr;
  cudaEvent_t ev_in = nullptr;
  float* A = nullptr;
  double *l = nullptr, *u = nullptr, *nrm = nullptr, *w = nullptr, *t = nullptr;
  float2 *l2 = nullptr, *u2 = nullptr, *t2 = nullptr;   // t2: t as double-float pairs
  uint8_t* jinf = nullptr;
  double t_norm = 0.0, gamma_w = 0.0, L = 0.0;
  double xbox = -1.0;  // sum_j max(|l_j|, |u_j|) ||a_j|| (primal-dual error bound), once computed
  int dual_mode = kScaling;
  int t_choice = -1;   // translation direction: 0 caller's, 1 -1, 2 minus the mean column, 3 -a_+, 4 case 1
  Buffers b{};
  float* y_dev = nullptr;
  double* x0_dev = nullptr;
  double *theta_dev = nullptr, *wstar_dev = nullptr;  // fixed dual point and A^T theta
  float2* theta2_dev = nullptr;                        // theta as double-float pairs
  int fwd_tiles = 0, fwd_chunks = 0, tr_blocks = 0, red_blocks = 0;
  int pass_stages = 0, pass_qw = 0, pass_cps = 1;  // fused single-pass iteration when pass_stages > 0
  bool pass_coop = false;                          // its persistent (cooperative) launch fits
  MomEntry* mom = nullptr;                          // momentum table of the persistent pass
  double Cg[3] = {0, 0, 0}, Cf[3] = {0, 0, 0}, Csub = 0.0;
  // instantiated solve graphs, one per option set (at most kGraphCache, oldest evicted), so
  // callers that alternate options do not rebuild a graph on every call
  struct CachedGraph {
    GraphKey key;
    int chunk;
    cudaGraphExec_t exec;
  };
  std::vector<CachedGraph> graphs;
  bool own_stream = false;
  std::vector<cudaEvent_t> prof;
  std::vector<void*> allocs;
  // batched solve (shared A): bf16 Gram matrix, float32 bounds, workspace of capacity b_cap
  int b_npad = 0;
  __nv_bfloat16* bH = nullptr;
  int b_cap = 0;
  float *b_nrmf = nullptr, *b_wf = nullptr;
  BBuffers bb{};
  CUtensorMap b_tmH{};  // tensor map of the step's operand H~
  float* bY = nullptr;
  double* bX0 = nullptr;
  std::vector<void*> b_allocs;
  bool b_have_graph = false;
  double b_key[10] = {0};
  cudaGraphExec_t b_exec = nullptr;
  // refinement (opts.refine): scratch for ref_cap instances (correlations, saved iterate),
  // their descriptors and results, and two events around the kernel
  int ref_cap = 0;
  double *ref_g = nullptr, *ref_xs = nullptr;
  RefDesc* ref_desc = nullptr;
  RefOut* ref_out = nullptr;
  cudaEvent_t ref_ev[2] = {nullptr, nullptr};
  long long grid_wait = kGridWaitCycles;  // bound of the persistent pass's grid-barrier waits
  unsigned char* pool_cur = nullptr;       // device pool of dalloc
  size_t pool_left = 0;
};

namespace {

// Handle-owned device buffers: carved (256-byte aligned, 16 bytes of slack each) from pool
// chunks of kPoolChunk bytes, a request larger than that in a chunk of its own; setup makes
// a few dozen small buffers, and one cudaMalloc per buffer cost a few tenths of a ms.
constexpr size_t kPoolChunk = size_t(4) << 20;
// The chunks come, stream-ordered on the handle's stream, from one memory pool per device
// owned by the library, which keeps up to kPoolKeep bytes of freed chunks for reuse: a setup
// after a destroy then takes its memory (the padded A included) without a cudaMalloc, which
// cost ~0.1 ms for an 80 MB matrix.
constexpr uint64_t kPoolKeep = uint64_t(1) << 30;

cudaError_t device_pool(cudaMemPool_t* out) {
  static std::mutex mu;
  static std::map<int, cudaMemPool_t> pools;
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  std::lock_guard<std::mutex> lock(mu);
  auto it = pools.find(dev);
  if (it != pools.end()) {
    *out = it->second;
    return cudaSuccess;
  }
  cudaMemPoolProps props{};
  props.allocType = cudaMemAllocationTypePinned;
  props.location.type = cudaMemLocationTypeDevice;
  props.location.id = dev;
  cudaMemPool_t pool = nullptr;
  e = cudaMemPoolCreate(&pool, &props);
  if (e != cudaSuccess) return e;
  uint64_t keep = kPoolKeep;
  e = cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &keep);
  if (e != cudaSuccess) {
    cudaMemPoolDestroy(pool);
    return e;
  }
  pools[dev] = pool;
  *out = pool;
  return cudaSuccess;
}

template <typename T>
bvls_status dalloc(bvls_handle* h, T** p, size_t count) {
  const size_t bytes = (count * sizeof(T) + 16 + 255) & ~size_t(255);
  if (bytes > h->pool_left) {
    const size_t chunk = std::max(bytes, kPoolChunk);
    void* q = nullptr;
    cudaMemPool_t pool = nullptr;
    CK(device_pool(&pool));
    CK(cudaMallocFromPoolAsync(&q, chunk, pool, h->s));
    h->allocs.push_back(q);
    if (bytes >= kPoolChunk) {   // a large buffer keeps its chunk; the current pool stays
      *p = static_cast<T*>(q);
      return BVLS_OK;
    }
    h->pool_cur = static_cast<unsigned char*>(q);
    h->pool_left = chunk;
  }
  *p = reinterpret_cast<T*>(h->pool_cur);
  h->pool_cur += bytes;
  h->pool_left -= bytes;
  return BVLS_OK;
}

#define TRY(expr)                      \
  do {                                 \
    bvls_status st_ = (expr);          \
    if (st_ != BVLS_OK) return st_;    \
  } while (0)

void free_handle(bvls_handle* h) {
  if (!h) return;
  for (auto& c : h->graphs) cudaGraphExecDestroy(c.exec);
  if (h->b_exec) cudaGraphExecDestroy(h->b_exec);
  for (void* p : h->b_allocs) cudaFree(p);
  for (auto e : h->prof) cudaEventDestroy(e);
  // the pool chunks go back to the library's pool in stream order, after the handle's work
  for (void* p : h->allocs) cudaFreeAsync(p, h->s);
  for (void* p : {(void*)h->ref_g, (void*)h->ref_xs, (void*)h->ref_desc, (void*)h->ref_out})
    if (p) cudaFree(p);
  for (cudaEvent_t e : h->ref_ev)
    if (e) cudaEventDestroy(e);
  if (h->ev_in) cudaEventDestroy(h->ev_in);
  if (h->s && h->own_stream) cudaStreamDestroy(h->s);
  delete h;
}

// The momentum table of the persistent pass (T[0] = 1, T[i+1] = (1 + sqrt(1 + 4 T[i]^2)) / 2),
// computed once per process in float64, in page-locked host memory where that can be had
// (its 2 MB then reach each new handle by an asynchronous copy instead of a staged one).
struct MomTable {
  const MomEntry* data;
  bool pinned;
};

const MomTable& momentum_table() {
  static const MomTable tab = [] {
    MomEntry* v = nullptr;
    bool pinned = cudaHostAlloc(reinterpret_cast<void**>(&v), sizeof(MomEntry) * kMomTable, cudaHostAllocDefault) ==
                  cudaSuccess;
    if (!pinned) {
      cudaGetLastError();
      v = new MomEntry[kMomTable];
    }
    double t = 1.0;
    for (int i = 0; i < kMomTable; ++i) {
      const double tn = 0.5 * (1.0 + std::sqrt(1.0 + 4.0 * t * t));
      const double beta = (t - 1.0) / tn;
      v[i].t = t;
      v[i].tn = tn;
      v[i].beta2 = df2_from_double(beta);
      v[i].onepb2 = df2_from_double(1.0 + beta);
      t = tn;
    }
    return MomTable{v, pinned};
  }();
  return tab;
}

// w = A^T t for a host direction t (or, with w_ready, the w already in h->w); returns whether
// a_j^T t < 0 (with its rounding bound) on every nonzero column with u_j = +inf.
bvls_status try_direction(bvls_handle* h, const std::vector<double>& t,
                          const std::vector<uint8_t>& jinf, const std::vector<double>& nrm,
                          bool* ok, bool w_ready = false) {
  CK(cudaMemcpyAsync(h->t, t.data(), sizeof(double) * h->m, cudaMemcpyHostToDevice, h->s));
  CK(launch_split_pairs(h->t, h->t2, h->m, h->s));
  if (!w_ready) CK(launch_col_dots(h->A, h->lda, h->m, h->n, h->t2, h->w, h->s));
  std::vector<double> w(h->n);
  CK(cudaMemcpyAsync(w.data(), h->w, sizeof(double) * h->n, cudaMemcpyDeviceToHost, h->s));
  CK(cudaStreamSynchronize(h->s));
  double tn = 0.0;
  for (double v : t) tn += v * v;
  tn = std::sqrt(tn);
  const double gamma = setup_dot_gamma(h->m);
  *ok = true;
  for (int j = 0; j < h->n; ++j) {
    if (!jinf[j] || !(nrm[j] > 0.0)) continue;
    if (!(w[j] + gamma * nrm[j] * tn < 0.0)) {
      *ok = false;
      break;
    }
  }
  if (*ok) {
    h->t_norm = tn;
    h->gamma_w = gamma;
  }
  return BVLS_OK;
}

// t = A (A^T A)^{-1} (-1) for n <= min(m, kBwdMaxFree) (Proposition 2, case 1), through the
// backward pass's free-set solver with every coordinate free.  Scratch is freed on return.
bvls_status case1_direction(bvls_handle* h, std::vector<double>* t) {
  const int m = h->m, n = h->n;
  std::vector<double> half(n, 0.5), zero(n, 0.0), one(n, 1.0), minus(n, -1.0);
  double *dx = nullptr, *dl = nullptr, *du = nullptr, *dv = nullptr, *dt = nullptr;
  int* di = nullptr;
  auto release = [&]() {
    for (void* p : {(void*)dx, (void*)dl, (void*)du, (void*)dv, (void*)dt, (void*)di})
      if (p) cudaFree(p);
  };
  cudaError_t e = cudaMalloc(&dx, sizeof(double) * n);
  if (e == cudaSuccess) e = cudaMalloc(&dl, sizeof(double) * n);
  if (e == cudaSuccess) e = cudaMalloc(&du, sizeof(double) * n);
  if (e == cudaSuccess) e = cudaMalloc(&dv, sizeof(double) * n);
  if (e == cudaSuccess) e = cudaMalloc(&dt, sizeof(double) * m);
  if (e == cudaSuccess) e = cudaMalloc(&di, sizeof(int) * 3);
  if (e == cudaSuccess) e = cudaMemcpyAsync(dx, half.data(), sizeof(double) * n, cudaMemcpyHostToDevice, h->s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(dl, zero.data(), sizeof(double) * n, cudaMemcpyHostToDevice, h->s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(du, one.data(), sizeof(double) * n, cudaMemcpyHostToDevice, h->s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(dv, minus.data(), sizeof(double) * n, cudaMemcpyHostToDevice, h->s);
  if (e == cudaSuccess) {
    BwdParams bp{};
    bp.A = h->A;
    bp.m = m;
    bp.n = n;
    bp.lda = h->lda;
    bp.B = 1;
    bp.l = dl;
    bp.u = du;
    bp.X = dx;
    bp.Y = nullptr;   // read only for r = y - A x, which this call does not request
    bp.ldy = m;
    bp.dLdX = dv;
    bp.dLdY = dt;
    bp.status = di;
    bp.iters = di + 1;
    bp.nfree = di + 2;
    bp.free_tol = 1e-9;
    bp.cg_tol = 1e-13;
    bp.cg_max_iter = 20000;
    e = launch_bwd(bp, h->s);
  }
  t->assign(m, 0.0);
  if (e == cudaSuccess) e = cudaMemcpyAsync(t->data(), dt, sizeof(double) * m, cudaMemcpyDeviceToHost, h->s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(h->s);
  release();
  if (e != cudaSuccess) return set_err(BVLS_ECUDA, "case-1 direction: %s", cudaGetErrorString(e));
  return BVLS_OK;
}

Params make_params(const bvls_handle* h, const bvls_opts& o, int max_iter) {
  Params p{};
  p.A = h->A;
  p.m = h->m;
  p.n = h->n;
  p.lda = h->lda;
  p.m4 = h->m4;
  p.l = h->l;
  p.u = h->u;
  p.nrm = h->nrm;
  p.w = h->w;
  p.jinf = h->jinf;
  p.l2 = h->l2;
  p.u2 = h->u2;
  const double L = o.lipschitz > 0.0 ? o.lipschitz : h->L;
  p.invL = 1.0 / L;
  p.invL2 = df2_from_double(p.invL);
  p.t_norm = h->t_norm;
  p.gamma_w = h->gamma_w;
  p.Cg = h->Cg[o.precision];
  p.Cf = h->Cf[o.precision];
  p.Csub = h->Csub;
  p.tol = o.tol;
  p.max_iter = max_iter;
  p.dual_mode = h->dual_mode;
  p.screening = o.screening;
  p.restart = o.restart;
  p.alg = o.algorithm == BVLS_ALG_CHAMBOLLE_POCK ? kChambollePock : kFista;
  if (p.alg == kChambollePock) {
    const double st = 0.99 / std::sqrt(L);
    p.tau2 = df2_from_double(st);
    p.sigma2 = df2_from_double(st);
    p.inv1ps2 = df2_from_double(1.0 / (1.0 + st));
    // the recurrence's error: each step adds the rounding of A xbar (|xbar_j| <= 3 max(|l_j|,|u_j|))
    // and halves what came before, so it stays below one step's bound
    p.E_cp = (p.Cf + 2.0 * p.Csub) * 3.0 * std::max(0.0, h->xbox);
  }
  p.fwd_chunks = h->fwd_chunks;
  p.fwd_tiles = h->fwd_tiles;
  p.mom = h->mom;
  p.grid_wait = h->grid_wait;
  return p;
}

// The single-pass iterations run as persistent launches (K iterations each).
bool persistent_form(const bvls_handle* h, const bvls_opts& o) {
  return h->pass_stages > 0 && h->pass_coop && o.single_pass == 1;
}

// Refinement parameters shared by the entry points (opts.refine).
RefParams ref_params(const RefDesc* desc, RefOut* out, int B) {
  RefParams rp{};
  rp.desc = desc;
  rp.out = out;
  rp.B = B;
  rp.max_rounds = 10;
  rp.cg_max_iter = 4000;
  rp.cg_tol = 1e-5f;
  rp.tau = 1e-9;
  rp.zeta = 1e-12;
  return rp;
}

// Scratch of the refinement for B instances of n coordinates (kept by the handle, grown on
// demand) and its two timing events.
bvls_status ref_reserve(bvls_handle* h, int B) {
  if (!h->ref_ev[0]) {
    CK(cudaEventCreate(&h->ref_ev[0]));
    CK(cudaEventCreate(&h->ref_ev[1]));
  }
  if (B <= h->ref_cap) return BVLS_OK;
  for (void** p : {(void**)&h->ref_g, (void**)&h->ref_xs, (void**)&h->ref_desc, (void**)&h->ref_out}) {
    if (*p) cudaFree(*p);
    *p = nullptr;
  }
  h->ref_cap = 0;
  CK(cudaMalloc(&h->ref_g, sizeof(double) * (size_t)B * h->n));
  CK(cudaMalloc(&h->ref_xs, sizeof(double) * (size_t)B * h->n));
  CK(cudaMalloc(&h->ref_desc, sizeof(RefDesc) * (size_t)B));
  CK(cudaMalloc(&h->ref_out, sizeof(RefOut) * (size_t)B));
  h->ref_cap = B;
  return BVLS_OK;
}

// Refine B instances sharing the handle's A and box: Y (pitch ldy floats), X (pitch ldx
// doubles, in place), flags (pitch ldf bytes, or null).  Results land in out (host, B).
bvls_status refine_shared(bvls_handle* h, int B, const float* Y, int ldy, double* X, int ldx, const uint8_t* flags,
                          int ldf, double step, std::vector<RefOut>* out, float* ms) {
  TRY(ref_reserve(h, B));
  CK(launch_ref_desc_strided(h->ref_desc, B, h->A, h->m, h->n, h->lda, Y, ldy, h->l, h->u, X, ldx, flags, ldf,
                             h->ref_g, h->ref_xs, step, h->s));
  CK(cudaEventRecord(h->ref_ev[0], h->s));
  CK(launch_refine(ref_params(h->ref_desc, h->ref_out, B), h->m, std::min(std::min(h->n, h->m), kRefMaxFree),
                   h->s));
  CK(cudaEventRecord(h->ref_ev[1], h->s));
  out->resize(B);
  CK(cudaMemcpyAsync(out->data(), h->ref_out, sizeof(RefOut) * B, cudaMemcpyDeviceToHost, h->s));
  CK(cudaStreamSynchronize(h->s));
  CK(cudaEventElapsedTime(ms, h->ref_ev[0], h->ref_ev[1]));
  return BVLS_OK;
}

// Enqueue chunk_len iterations (the chunk starts at an even k, so slot = j & 1).
// With ev != nullptr, records ev[3j], ev[3j+1], ev[3j+2] around the two products.
cudaError_t enqueue_chunk(bvls_handle* h, const Params& p, const bvls_opts& o, int chunk_len,
                          cudaEvent_t* ev) {
  const bool scr = o.screening && h->dual_mode != kZero;
  cudaError_t e = cudaSuccess;
  if (persistent_form(h, o)) {
    // one cooperative launch per K iterations (ending at a gap iteration), then the gap
    // evaluation and the screening step; with ev: ev[3 b] and ev[3 b + 1] around launch b
    const int K = o.screen_every;
    for (int j0 = 0, blk = 0; j0 < chunk_len && e == cudaSuccess; j0 += K, ++blk) {
      const int slot = j0 & 1;
      const int last = (j0 + K - 1) & 1;
      if (ev) cudaEventRecordWithFlags(ev[3 * blk], h->s, cudaEventRecordExternal);
      e = launch_iters(p, h->b, slot, K, true, o.precision, h->num_sms, h->pass_stages, h->pass_cps, h->pass_qw,
                       h->s);
      if (e != cudaSuccess) break;
      if (ev) cudaEventRecordWithFlags(ev[3 * blk + 1], h->s, cudaEventRecordExternal);
      e = launch_gap(p, h->b, last, !scr, h->red_blocks, h->s);
      if (e == cudaSuccess && scr) {
        e = launch_test(p, h->b, last, h->red_blocks, h->s);
        if (e == cudaSuccess) e = launch_compact(p, h->b, last, h->s);
        if (e == cudaSuccess) e = launch_fwd(p, h->b, last, o.precision, true, h->s);
      }
    }
    return e;
  }
  for (int j = 0; j < chunk_len && e == cudaSuccess; ++j) {
    const int slot = j & 1;
    const bool gap_iter = ((j + 1) % o.screen_every) == 0;
    // External records: inside a captured graph they become event-record nodes that time
    // the kernels (a plain record would only become a dependency edge).
    if (ev) cudaEventRecordWithFlags(ev[3 * j], h->s, cudaEventRecordExternal);
    if (h->pass_stages > 0 && o.single_pass) {
      // fused: one read of A_S gives g_k and q_{k+1}; then r_{k+1} = y' - q_{k+1}
      e = launch_pass(p, h->b, slot, o.precision, gap_iter, h->num_sms, h->pass_stages, h->pass_cps, h->pass_qw,
                      h->s);
      if (e != cudaSuccess) break;
      if (ev) cudaEventRecordWithFlags(ev[3 * j + 1], h->s, cudaEventRecordExternal);
      e = launch_resid(p, h->b, slot, h->num_sms, h->s);
    } else {
      e = launch_fwd(p, h->b, slot, o.precision, false, h->s);
      if (e != cudaSuccess) break;
      if (ev) cudaEventRecordWithFlags(ev[3 * j + 1], h->s, cudaEventRecordExternal);
      e = launch_tr(p, h->b, slot, o.precision, gap_iter, h->tr_blocks, h->s);
    }
    if (e != cudaSuccess) break;
    if (ev) cudaEventRecordWithFlags(ev[3 * j + 2], h->s, cudaEventRecordExternal);
    if (gap_iter) {
      e = launch_gap(p, h->b, slot, !scr, h->red_blocks, h->s);
      if (e == cudaSuccess && scr) {
        e = launch_test(p, h->b, slot, h->red_blocks, h->s);
        if (e == cudaSuccess) e = launch_compact(p, h->b, slot, h->s);
        if (e == cudaSuccess) e = launch_fwd(p, h->b, slot, o.precision, true, h->s);
      }
    }
  }
  return e;
}

int chunk_length(int K) {
  int c = 1;
  while (K * c < 16 || (K * c) % 2) ++c;
  return K * c;
}

bvls_status validate_opts(const bvls_opts& o) {
  if (o.algorithm != BVLS_ALG_FISTA && o.algorithm != BVLS_ALG_CHAMBOLLE_POCK)
    return set_err(BVLS_EINVAL, "algorithm must be BVLS_ALG_FISTA or BVLS_ALG_CHAMBOLLE_POCK");
  if (!(o.tol >= 0.0) || o.screen_every < 1 || o.max_iter < 1 ||
      (o.precision != BVLS_PREC_FP32X2 && o.precision != BVLS_PREC_FP32 && o.precision != BVLS_PREC_MIXED) ||
      !(o.lipschitz >= 0.0) || !std::isfinite(o.lipschitz))
    return set_err(BVLS_EINVAL, "invalid options (tol >= 0, screen_every >= 1, max_iter >= 1, "
                                "precision 0/1/2, lipschitz >= 0 finite)");
  if (o.single_pass < 0 || o.single_pass > 2) return set_err(BVLS_EINVAL, "single_pass must be 0, 1 or 2");
  if (o.refine < 0 || o.refine > 1) return set_err(BVLS_EINVAL, "refine must be 0 or 1");
  if (o.profile < 0 || o.profile > 2) return set_err(BVLS_EINVAL, "profile must be 0, 1 or 2");
  return BVLS_OK;
}

// sum_j max(|l_j|, |u_j|) ||a_j|| for the primal-dual error bound (host, once per handle).
bvls_status compute_xbox(bvls_handle* h) {
  std::vector<double> l(h->n), u(h->n), nr(h->n);
  CK(cudaMemcpyAsync(l.data(), h->l, sizeof(double) * h->n, cudaMemcpyDeviceToHost, h->s));
  CK(cudaMemcpyAsync(u.data(), h->u, sizeof(double) * h->n, cudaMemcpyDeviceToHost, h->s));
  CK(cudaMemcpyAsync(nr.data(), h->nrm, sizeof(double) * h->n, cudaMemcpyDeviceToHost, h->s));
  CK(cudaStreamSynchronize(h->s));
  double s = 0.0;
  for (int j = 0; j < h->n; ++j) s += std::max(std::fabs(l[j]), std::fabs(u[j])) * nr[j];
  h->xbox = s * (1.0 + 1e-12);
  return BVLS_OK;
}

// The fixed dual point of the oracle-dual-point experiment: copies theta, forms
// w* = A^T theta in float64 and the translation step that puts theta in F_D.
bvls_status prepare_fixed_dual(bvls_handle* h, const double* theta, Params* p) {
  if (!(h->pass_stages > 0)) return set_err(BVLS_ENOTSUP, "dual_point needs the single-pass form (m <= 8192)");
  if (h->dual_mode == kZero)
    return set_err(BVLS_EINVAL, "dual_point needs an interior translation direction (dual mode zero)");
  const int m = h->m, n = h->n;
  if (!h->theta_dev) {
    TRY(dalloc(h, &h->theta_dev, m));
    TRY(dalloc(h, &h->theta2_dev, m));
    TRY(dalloc(h, &h->wstar_dev, n));
  }
  std::vector<double> th(m), ws(n), nr(n), w(n);
  CK(cudaMemcpyAsync(h->theta_dev, theta, sizeof(double) * m, cudaMemcpyDefault, h->s));
  CK(cudaMemcpyAsync(th.data(), h->theta_dev, sizeof(double) * m, cudaMemcpyDeviceToHost, h->s));
  CK(launch_split_pairs(h->theta_dev, h->theta2_dev, m, h->s));
  CK(launch_col_dots(h->A, h->lda, m, n, h->theta2_dev, h->wstar_dev, h->s));
  CK(cudaMemcpyAsync(ws.data(), h->wstar_dev, sizeof(double) * n, cudaMemcpyDeviceToHost, h->s));
  CK(cudaMemcpyAsync(nr.data(), h->nrm, sizeof(double) * n, cudaMemcpyDeviceToHost, h->s));
  CK(cudaMemcpyAsync(w.data(), h->w, sizeof(double) * n, cudaMemcpyDeviceToHost, h->s));
  std::vector<uint8_t> jinf(n);
  CK(cudaMemcpyAsync(jinf.data(), h->jinf, n, cudaMemcpyDeviceToHost, h->s));
  CK(cudaStreamSynchronize(h->s));
  double tn = 0.0;
  for (double v : th) {
    if (!std::isfinite(v)) return set_err(BVLS_ENONFINITE, "dual_point contains NaN or Inf");
    tn += v * v;
  }
  tn = std::sqrt(tn);
  const double eta0 = setup_dot_gamma(m) * tn;  // the product a_j^T theta, per unit ||a_j||
  double eps = 0.0;
  if (h->dual_mode == kTranslation) {
    for (int j = 0; j < n; ++j) {
      if (!jinf[j] || !(nr[j] > 0.0)) continue;
      const double den = -w[j] - h->gamma_w * nr[j] * h->t_norm;
      eps = std::max(eps, std::max(ws[j] + eta0 * nr[j], 0.0) / den);
    }
    eps *= 1.0 + 1e-12;
  }
  p->wstar = h->wstar_dev;
  p->theta = h->theta_dev;
  p->tvec = h->t;
  p->eps_star = eps;
  p->eta_star = eta0 + eps * h->gamma_w * h->t_norm;
  return BVLS_OK;
}

}  // namespace

void bvls::record_error(const char* msg) { g_err = msg; }

extern "C" {

void bvls_default_opts(bvls_opts* o) {
  if (!o) return;
  o->tol = 1e-6;
  o->screen_every = 10;
  o->max_iter = 100000;
  o->screening = 1;
  o->precision = BVLS_PREC_FP32X2;
  o->restart = 1;
  o->lipschitz = 0.0;
  o->profile = 0;
  o->single_pass = 1;
  o->dual_point = nullptr;
  o->algorithm = BVLS_ALG_FISTA;
  o->refine = 0;
}

const char* bvls_last_error(void) { return g_err.c_str(); }

void bvls_destroy(bvls_handle* h) { free_handle(h); }

bvls_status bvls_set_grid_wait(bvls_handle* h, long long cycles) {
  if (!h) return set_err(BVLS_EINVAL, "handle is required");
  h->grid_wait = cycles > 0 ? cycles : kGridWaitCycles;
  // the bound is a kernel argument baked into the instantiated solve graphs
  CK(cudaStreamSynchronize(h->s));
  for (auto& c : h->graphs) cudaGraphExecDestroy(c.exec);
  h->graphs.clear();
  return BVLS_OK;
}

// Largest eigenvalue of the symmetric tridiagonal matrix with diagonal alpha and off-diagonal
// beta, by bisection on the Sturm count (the number of eigenvalues below x is the number of
// negative pivots of the LDL^T factorisation of T - x I; Golub & Van Loan, Section 8.4.1).
double tridiag_max_eig(const std::vector<double>& alpha, const std::vector<double>& beta) {
  const int K = (int)alpha.size();
  if (K == 0) return 0.0;
  double lo = 0.0, hi = 0.0;  // Gershgorin bounds
  for (int i = 0; i < K; ++i) {
    const double r = (i > 0 ? std::fabs(beta[i - 1]) : 0.0) + (i + 1 < K ? std::fabs(beta[i]) : 0.0);
    lo = std::min(lo, alpha[i] - r);
    hi = std::max(hi, alpha[i] + r);
  }
  auto below = [&](double x) {  // eigenvalues < x
    int cnt = 0;
    double d = 1.0;
    for (int i = 0; i < K; ++i) {
      const double b2 = i > 0 ? beta[i - 1] * beta[i - 1] : 0.0;
      d = alpha[i] - x - (i > 0 ? b2 / d : 0.0);
      if (d == 0.0) d = -1e-300;
      if (d < 0.0) ++cnt;
    }
    return cnt;
  };
  for (int it = 0; it < 200 && hi - lo > 1e-15 * std::max(1.0, std::fabs(hi)); ++it) {
    const double mid = 0.5 * (lo + hi);
    if (below(mid) >= K) hi = mid;   // every eigenvalue is below mid
    else lo = mid;
  }
  return hi;
}

static bvls_status setup_impl(bvls_handle* h, const float* A, int lda, const double* l,
                              const double* u, const double* t) {
  const int m = h->m, n = h->n;
  // Host-side validation of the box.
  std::vector<double> lv(n, 0.0), uv(n, INFINITY);
  if (l) std::memcpy(lv.data(), l, sizeof(double) * n);
  if (u) std::memcpy(uv.data(), u, sizeof(double) * n);
  std::vector<uint8_t> jinf(n);
  bool any_inf = false;
  for (int j = 0; j < n; ++j) {
    if (!std::isfinite(lv[j]) || std::isnan(uv[j]) || uv[j] == -INFINITY || lv[j] > uv[j])
      return set_err(BVLS_EINVAL, "bound %d: need finite l_j <= u_j (u_j may be +inf)", j);
    jinf[j] = std::isinf(uv[j]) ? 1 : 0;
    any_inf |= jinf[j] != 0;
  }
  int dev = 0;
  CK(cudaGetDevice(&dev));
  CK(cudaDeviceGetAttribute(&h->num_sms, cudaDevAttrMultiProcessorCount, dev));
  // Work runs on the caller's stream; the legacy default stream cannot be captured into a
  // graph, so for stream 0 the handle owns a stream ordered after it by events.
  if (h->user) {
    h->s = h->user;
  } else {
    CK(cudaStreamCreateWithFlags(&h->s, cudaStreamNonBlocking));
    h->own_stream = true;
  }
  CK(cudaEventCreateWithFlags(&h->ev_in, cudaEventDisableTiming));
  if (h->own_stream) {
    CK(cudaEventRecord(h->ev_in, h->user));
    CK(cudaStreamWaitEvent(h->s, h->ev_in, 0));
  }

  TRY(dalloc(h, &h->A, (size_t)h->lda * n));
  if (h->lda > m)   // the padding rows m..lda-1 of every column are zero
    CK(cudaMemset2DAsync(h->A + m, sizeof(float) * h->lda, 0, sizeof(float) * (h->lda - m), n, h->s));
  CK(cudaMemcpy2DAsync(h->A, sizeof(float) * h->lda, A, sizeof(float) * lda, sizeof(float) * m, n,
                       cudaMemcpyDefault, h->s));
  int* flag = nullptr;
  TRY(dalloc(h, &flag, 4));
  CK(cudaMemsetAsync(flag, 0, sizeof(int), h->s));
  // every stored row (the padding rows are zero), read back with the column norms
  CK(launch_check_finite(h->A, h->lda, h->lda, n, flag, h->s));

  // l and u in one buffer and one copy; their double-float pairs and J_inf formed on the device
  double* lu = nullptr;
  TRY(dalloc(h, &lu, 2 * (size_t)n));
  h->l = lu;
  h->u = lu + n;
  TRY(dalloc(h, &h->nrm, n));
  TRY(dalloc(h, &h->w, n));
  TRY(dalloc(h, &h->jinf, n));
  TRY(dalloc(h, &h->t, m));
  TRY(dalloc(h, &h->t2, m));
  {
    std::vector<double> luv(2 * (size_t)n);
    std::memcpy(luv.data(), lv.data(), sizeof(double) * n);
    std::memcpy(luv.data() + n, uv.data(), sizeof(double) * n);
    // a pageable copy: the call returns once the source is staged, so luv may go
    CK(cudaMemcpyAsync(lu, luv.data(), sizeof(double) * 2 * (size_t)n, cudaMemcpyHostToDevice, h->s));
  }
  TRY(dalloc(h, &h->l2, n));
  TRY(dalloc(h, &h->u2, n));
  CK(launch_bound_pairs(h->l, h->u, h->l2, h->u2, h->jinf, n, h->s));
  CK(cudaMemsetAsync(h->w, 0, sizeof(double) * n, h->s));
  // with no caller t, the first candidate t = -1 gets its products w = A^T t in this pass
  CK(launch_col_norms(h->A, h->lda, m, n, h->nrm, h->s, (any_inf && !t) ? h->w : nullptr));
  std::vector<double> nrm(n);
  int bad = 0;
  CK(cudaMemcpyAsync(&bad, flag, sizeof(int), cudaMemcpyDeviceToHost, h->s));
  CK(cudaMemcpyAsync(nrm.data(), h->nrm, sizeof(double) * n, cudaMemcpyDeviceToHost, h->s));
  CK(cudaStreamSynchronize(h->s));
  if (bad) return set_err(BVLS_ENONFINITE, "A contains NaN or Inf");

  // Dual point of Section 4.
  if (!any_inf) {
    h->dual_mode = kScaling;
  } else if (t) {
    std::vector<double> tv(t, t + m);
    for (double v : tv)
      if (!std::isfinite(v)) return set_err(BVLS_EINVAL, "t must be finite");
    bool ok = false;
    TRY(try_direction(h, tv, jinf, nrm, &ok));
    if (!ok) return set_err(BVLS_EINVAL, "the given t is not an interior direction (a_j^T t < 0)");
    h->dual_mode = kTranslation;
    h->t_choice = 0;
  } else {
    bool ok = false;
    std::vector<double> tv(m, -1.0);  // Proposition 2, case 3 (w from the column-norm pass)
    TRY(try_direction(h, tv, jinf, nrm, &ok, true));
    if (ok) h->t_choice = 1;
    if (!ok) {
      // s = sum_k a_k and c = A^T s serve the next two candidates: minus the mean column has
      // w = -c / n, and the column most correlated with all others is argmax_j c_j
      double *rs = nullptr, *rs_part = nullptr, *corr_d = nullptr;
      float2* rs2 = nullptr;
      TRY(dalloc(h, &rs, m));
      TRY(dalloc(h, &rs2, m));
      TRY(dalloc(h, &rs_part, row_sums_scratch(m, n)));
      TRY(dalloc(h, &corr_d, n));
      CK(launch_row_sums(h->A, h->lda, m, n, rs_part, rs, h->s));
      CK(launch_split_pairs(rs, rs2, m, h->s));
      CK(launch_col_dots(h->A, h->lda, m, n, rs2, corr_d, h->s));
      CK(launch_scale_neg(corr_d, n, 1.0 / n, h->w, h->s));
      std::vector<double> s(m), corr(n);
      CK(cudaMemcpyAsync(s.data(), rs, sizeof(double) * m, cudaMemcpyDeviceToHost, h->s));
      CK(cudaMemcpyAsync(corr.data(), corr_d, sizeof(double) * n, cudaMemcpyDeviceToHost, h->s));
      CK(cudaStreamSynchronize(h->s));
      for (int i = 0; i < m; ++i) tv[i] = -s[i] / n;  // minus the mean column
      TRY(try_direction(h, tv, jinf, nrm, &ok, true));
      if (ok) h->t_choice = 2;
      if (!ok) {
        // minus the column most correlated with all others: argmax_j a_j^T sum_k a_k
        int jb = 0;
        for (int j = 1; j < n; ++j)
          if (corr[j] > corr[jb]) jb = j;
        std::vector<float> col(m);
        CK(cudaMemcpyAsync(col.data(), h->A + (size_t)jb * h->lda, sizeof(float) * m,
                           cudaMemcpyDeviceToHost, h->s));
        CK(cudaStreamSynchronize(h->s));
        for (int i = 0; i < m; ++i) tv[i] = -(double)col[i];
        TRY(try_direction(h, tv, jinf, nrm, &ok));
        if (ok) h->t_choice = 3;
      }
      if (!ok && n <= m && n <= kBwdMaxFree && bwd_smem_bytes(m) <= 227u * 1024u) {
        // Proposition 2, case 1: with rank(A) = n <= m, A^T t = -1 has the least-squares
        // (minimum-norm) solution t = A (A^T A)^{-1} (-1).  The backward pass's solver
        // computes exactly that shape, A_F (A_F^T A_F)^{-1} v, by conjugate gradients in
        // float64: here with every coordinate free (x = 1/2 in the box [0, 1]) and v = -1.
        TRY(case1_direction(h, &tv));
        TRY(try_direction(h, tv, jinf, nrm, &ok));
        if (ok) h->t_choice = 4;
      }
    }
    h->dual_mode = ok ? kTranslation : kZero;
    if (!ok) {
      h->t_norm = 0.0;
      h->gamma_w = 0.0;
    }
  }

  // Step constant: L = 1.05 x the largest eigenvalue of A^T A, estimated by K Lanczos steps
  // (one cooperative launch) or, where that launch does not fit, by 100 power steps (one
  // unnormalised warm-up step discarded).
  {
    float *v = nullptr, *q = nullptr, *v2 = nullptr;
    double* scal = nullptr;
    TRY(dalloc(h, &v, n));
    TRY(dalloc(h, &v2, n));
    TRY(dalloc(h, &q, m));
    TRY(dalloc(h, &scal, 2));
    CK(cudaMemsetAsync(scal, 0, 2 * sizeof(double), h->s));
    CK(launch_power_init(v, n, h->s));
    bool done = false;
    {
      const int K = std::min(kLanczosSteps, n);
      float *part = nullptr, *qc = nullptr;
      double *wn2 = nullptr, *qn2 = nullptr, *ab = nullptr;
      unsigned* gb = nullptr;
      TRY(dalloc(h, &part, (size_t)h->num_sms * h->lda));
      TRY(dalloc(h, &qc, h->lda));
      TRY(dalloc(h, &wn2, h->num_sms));
      TRY(dalloc(h, &qn2, h->lda / 32));
      TRY(dalloc(h, &ab, 2 * (size_t)K + 2));
      TRY(dalloc(h, &gb, 2));
      CK(cudaMemsetAsync(gb, 0, 2 * sizeof(unsigned), h->s));
      CK(cudaMemsetAsync(ab, 0, sizeof(double) * (2 * (size_t)K + 2), h->s));
      const cudaError_t e = launch_lanczos_coop(h->A, h->lda, m, n, v, part, qc, wn2, qn2, ab, scal, gb, K,
                                                h->num_sms, h->s);
      if (e == cudaSuccess) {
        double sc[2] = {0.0, 0.0};
        std::vector<double> hab(2 * (size_t)K + 2);
        CK(cudaMemcpyAsync(sc, scal, 2 * sizeof(double), cudaMemcpyDeviceToHost, h->s));
        CK(cudaMemcpyAsync(hab.data(), ab, sizeof(double) * hab.size(), cudaMemcpyDeviceToHost, h->s));
        CK(cudaStreamSynchronize(h->s));
        if (sc[1] >= 0.0) {
          std::vector<double> alpha(K), beta(K > 1 ? K - 1 : 0);
          for (int i = 0; i < K; ++i) alpha[i] = hab[2 * (i + 1)];
          for (int i = 0; i + 1 < K; ++i) beta[i] = hab[2 * (i + 1) + 1];
          const double lam = tridiag_max_eig(alpha, beta);
          h->L = lam > 0.0 ? 1.05 * lam : 1.0;
          done = true;
        } else {
          return set_err(BVLS_ETIMEOUT, "a device-side wait of the Lanczos steps exceeded its bound");
        }
      } else if (e != cudaErrorNotSupported) {
        CK(e);
      } else {
        cudaGetLastError();
      }
    }
    if (!done) {
      CK(launch_power_step(h->A, h->lda, m, n, v, q, v2, scal, h->s));
      CK(cudaMemsetAsync(scal, 0, sizeof(double), h->s));
      for (int it = 0; it < 100; ++it) CK(launch_power_step(h->A, h->lda, m, n, v, q, v2, scal, h->s));
      double lam = 0.0;
      CK(cudaMemcpyAsync(&lam, scal, sizeof(double), cudaMemcpyDeviceToHost, h->s));
      CK(cudaStreamSynchronize(h->s));
      h->L = lam > 0.0 ? 1.05 * lam : 1.0;
    }
  }

  // Workspace of the solve loop and launch shapes.
  h->fwd_tiles = (h->lda + kFwdRows - 1) / kFwdRows;
  {
    int chunks = (4 * h->num_sms + h->fwd_tiles - 1) / h->fwd_tiles;
    chunks = std::max(1, std::min(chunks, std::max(1, (n + 7) / 8)));
    h->fwd_chunks = std::min(chunks, 1024);
  }
  int bps = 1;
  CK(tr_configure(h->m4, &bps));
  {
    int optin = 0;
    CK(cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev));
    h->pass_stages = pass_configure(h->lda, h->m4, iters_idx_cap(n, h->num_sms), optin, &h->pass_qw,
                                    &h->pass_cps);
    h->pass_coop = h->pass_stages > 0 &&
                   iters_configure(h->lda, h->m4, h->pass_stages, h->pass_cps, iters_idx_cap(n, h->num_sms),
                                   h->num_sms);
    cudaGetLastError();
  }
  h->tr_blocks = h->num_sms * std::max(1, std::min(bps, 2));
  h->red_blocks = std::max(1, std::min(2 * h->num_sms, (n + kRedThreads - 1) / kRedThreads));
  const int max_blocks = std::max(std::max(h->tr_blocks, h->red_blocks), 64);

  Buffers& b = h->b;
  TRY(dalloc(h, &b.x[0], n));
  TRY(dalloc(h, &b.x[1], n));
  TRY(dalloc(h, &b.g[0], n));
  TRY(dalloc(h, &b.g[1], n));
  TRY(dalloc(h, &b.idx, n));
  TRY(dalloc(h, &b.idx_tmp, n));
  TRY(dalloc(h, &b.fold, n));
  TRY(dalloc(h, &b.flags, n));
  TRY(dalloc(h, &b.yh, h->m4));
  TRY(dalloc(h, &b.yl, h->m4));
  TRY(dalloc(h, &b.rh, h->m4));
  TRY(dalloc(h, &b.rl, h->m4));
  TRY(dalloc(h, &b.part, (size_t)h->fwd_chunks * h->lda));
  TRY(dalloc(h, &b.tileP, (h->lda + 31) / 32));   // >= fwd_tiles
  TRY(dalloc(h, &b.tileR, (h->m4 + 31) / 32));    // the residual kernel's grid
  TRY(dalloc(h, &b.tileD, (h->m4 + 31) / 32));
  TRY(dalloc(h, &b.tileZ, (h->m4 + 31) / 32));
  TRY(dalloc(h, &b.crh, h->m4));
  TRY(dalloc(h, &b.crl, h->m4));
  TRY(dalloc(h, &b.tile_cnt, h->fwd_tiles));
  TRY(dalloc(h, &b.blk, 4 * (size_t)max_blocks));
  TRY(dalloc(h, &b.st, 1));
  TRY(dalloc(h, &b.qpart, (size_t)h->num_sms * h->m4));
  TRY(dalloc(h, &b.gbar, kMaxGridFlags));
  TRY(dalloc(h, &h->mom, kMomTable));
  CK(cudaMemcpyAsync(h->mom, momentum_table().data, sizeof(MomEntry) * kMomTable, cudaMemcpyHostToDevice, h->s));
  TRY(dalloc(h, &b.xout, n));
  TRY(dalloc(h, &h->y_dev, h->m4));
  TRY(dalloc(h, &h->x0_dev, n));
  CK(cudaMemsetAsync(b.tile_cnt, 0, sizeof(unsigned) * h->fwd_tiles, h->s));
  CK(cudaMemsetAsync(b.gbar, 0, kMaxGridFlags * sizeof(unsigned), h->s));
  CK(cudaMemsetAsync(b.st, 0, sizeof(DevState), h->s));
  CK(cudaMemsetAsync(h->y_dev, 0, sizeof(float) * h->m4, h->s));
  b.y_in = h->y_dev;
  b.x0_in = nullptr;

  // Rounding constants of the double-float products (see the header of common.cuh): a
  // tree of depth d of TwoSum steps is exact up to 2 (d+2)^2 u^2 sum |terms|.
  {
    const int m4q = h->m4 / 4;
    const int d_g = (m4q + 31) / 32 + 7;
    h->Cg[kX2] = 2.0 * (d_g + 2.0) * (d_g + 2.0) * kU * kU + 4.0 * kU * kU + 2.0 * kU64;
    h->Cg[kF32] = 1.01 * (d_g + 2.0) * kU + kU;
    const int per = (n + h->fwd_chunks - 1) / h->fwd_chunks;
    const int d_f = ((per + kFwdWarps - 1) / kFwdWarps + 1) / 2 + 4 + h->fwd_chunks + 1;
    // the fused pass: a q-warp lane sums its CTA's columns (at most iters_idx_cap of them when
    // the persistent pass shrinks its grid), then 8 warps x nparts/8 partials
    const int d_p = iters_idx_cap(n, h->num_sms) + (h->num_sms + 7) / 8 + 8;
    const int d = std::max(d_f, d_p);
    h->Cf[kX2] = 2.0 * (d + 2.0) * (d + 2.0) * kU * kU + 2.0 * kU * kU;
    h->Cf[kF32] = 1.01 * (d + 2.0) * kU + kU;
    h->Cg[kMix] = h->Cg[kF32];
    // mode MIXED: the fused pass sums each stage's (at most pass_cps) columns in float32 with
    // the high part of x_j before one double-float merge: gamma_cps + u for the stage sums
    // (the dropped low parts), then the double-float bound of the merges
    h->Cf[kMix] = 1.01 * (std::max(1, h->pass_cps) + 1.0) * kU + 1.01 * h->Cf[kX2];
    h->Csub = 8.0 * kU * kU;
  }
  CK(cudaStreamSynchronize(h->s));
  return BVLS_OK;
}

bvls_status bvls_setup(const float* A, int m, int n, int lda, const double* l, const double* u,
                       const double* t, void* stream, bvls_handle** out) {
  if (!out) return set_err(BVLS_EINVAL, "out is NULL");
  *out = nullptr;
  if (!A || m < 1 || n < 1 || lda < m) return set_err(BVLS_EINVAL, "need A != NULL, m >= 1, n >= 1, lda >= m");
  if (m > kMaxRows) return set_err(BVLS_ENOTSUP, "m = %d exceeds %d", m, kMaxRows);
  bvls_handle* h = new (std::nothrow) bvls_handle();
  if (!h) return set_err(BVLS_ENOMEM, "host allocation failed");
  h->m = m;
  h->n = n;
  h->lda = (m + 31) / 32 * 32;
  h->m4 = (m + 3) / 4 * 4;
  h->user = static_cast<cudaStream_t>(stream);
  bvls_status st = setup_impl(h, A, lda, l, u, t);
  if (st != BVLS_OK) {
    free_handle(h);
    return st;
  }
  g_err.clear();
  *out = h;
  return BVLS_OK;
}

bvls_status bvls_solve(bvls_handle* h, const float* y, const double* x0, const bvls_opts* opts,
                       double* x_out, uint8_t* screened_out, bvls_info* info) {
  if (!h || !y || !x_out) return set_err(BVLS_EINVAL, "handle, y and x_out are required");
  bvls_opts o;
  bvls_default_opts(&o);
  if (opts) o = *opts;
  TRY(validate_opts(o));
  const int K = o.screen_every;
  const int max_iter = (int)std::min<long long>((long long)(o.max_iter + K - 1) / K * K, 0x7fffffff);
  const int chunk = chunk_length(K);
  Params p = make_params(h, o, max_iter);
  if (o.dual_point) {
    if (!o.single_pass) return set_err(BVLS_ENOTSUP, "dual_point needs the single-pass form (single_pass = 1)");
    if (o.algorithm != BVLS_ALG_FISTA) return set_err(BVLS_ENOTSUP, "dual_point is a FISTA option");
    TRY(prepare_fixed_dual(h, o.dual_point, &p));
  }
  if (o.algorithm == BVLS_ALG_CHAMBOLLE_POCK && h->xbox < 0.0) {
    TRY(compute_xbox(h));
    p = make_params(h, o, max_iter);
  }

  if (h->own_stream) {
    CK(cudaEventRecord(h->ev_in, h->user));
    CK(cudaStreamWaitEvent(h->s, h->ev_in, 0));
  }
  CK(cudaMemcpyAsync(h->y_dev, y, sizeof(float) * h->m, cudaMemcpyDefault, h->s));
  h->b.x0_in = nullptr;
  if (x0) {
    CK(cudaMemcpyAsync(h->x0_dev, x0, sizeof(double) * h->n, cudaMemcpyDefault, h->s));
    h->b.x0_in = h->x0_dev;
  }
  const bool fused = h->pass_stages > 0 && o.single_pass;
  if (o.algorithm == BVLS_ALG_CHAMBOLLE_POCK && (!fused || h->dual_mode != kScaling))
    return set_err(BVLS_ENOTSUP, "the primal-dual solver covers BVLS (every u_j finite) in the single-pass form");
  CK(launch_init(p, h->b, h->s));
  if (fused) CK(launch_fwd(p, h->b, 0, o.precision, false, h->s));  // r_0, P_0
  if (p.alg == kChambollePock) CK(launch_cp_init(p, h->b, h->s));  // z_1 = -r_0

  const long long max_chunks = (max_iter + chunk - 1) / chunk + 1;
  const bool scr = o.screening && h->dual_mode != kZero;
  const bool pers = persistent_form(h, o);
  const long long per_chunk = (pers ? 0LL : 2LL * chunk) + (long long)(chunk / K) * ((scr ? 4 : 1) + (pers ? 1 : 0));
  long long chunks_run = 0;
  double fwd_ms = 0.0, tr_ms = 0.0;
  int fwd_launches = 0, tr_launches = 0;
  if (o.profile == 2) {
    // Every kernel launched directly from the host, a chunk at a time, until the stop flag.
    for (long long c = 0; c < max_chunks; ++c) {
      CK(enqueue_chunk(h, p, o, chunk, nullptr));
      ++chunks_run;
      DevState hs;
      CK(cudaMemcpyAsync(&hs, h->b.st, sizeof(DevState), cudaMemcpyDeviceToHost, h->s));
      CK(cudaStreamSynchronize(h->s));
      if (hs.done || hs.error) break;
    }
  } else if (o.profile) {
    // The chunk, with event-record nodes around the product kernels, is captured into a
    // graph so the events time the kernels without host launch gaps in between.
    while ((int)h->prof.size() < 3 * chunk) {
      cudaEvent_t e;
      CK(cudaEventCreate(&e));
      h->prof.push_back(e);
    }
    cudaGraph_t g = nullptr;
    cudaGraphExec_t gx = nullptr;
    CK(cudaStreamBeginCapture(h->s, cudaStreamCaptureModeThreadLocal));
    cudaError_t e1 = enqueue_chunk(h, p, o, chunk, h->prof.data());
    cudaError_t e2 = cudaStreamEndCapture(h->s, &g);
    CK(e1);
    CK(e2);
    cudaError_t e3 = cudaGraphInstantiate(&gx, g, 0);
    cudaGraphDestroy(g);
    CK(e3);
    int k_before = 0;
    bvls_status pst = BVLS_OK;
    for (long long c = 0; c < max_chunks && pst == BVLS_OK; ++c) {
      cudaError_t e = cudaGraphLaunch(gx, h->s);
      ++chunks_run;
      DevState hs;
      if (e == cudaSuccess) e = cudaMemcpyAsync(&hs, h->b.st, sizeof(DevState), cudaMemcpyDeviceToHost, h->s);
      if (e == cudaSuccess) e = cudaStreamSynchronize(h->s);
      if (e != cudaSuccess) {
        pst = set_err(BVLS_ECUDA, "profile chunk: %s", cudaGetErrorString(e));
        break;
      }
      const int ran = std::min(chunk, hs.k - k_before);
      if (pers) {
        for (int blk = 0; blk < ran / K; ++blk) {   // launches that ran their K iterations
          float a = 0.f;
          CK(cudaEventElapsedTime(&a, h->prof[3 * blk], h->prof[3 * blk + 1]));
          tr_ms += a;
          ++tr_launches;
        }
      } else {
        for (int j = 0; j < ran; ++j) {
          float a = 0.f, b2 = 0.f;
          CK(cudaEventElapsedTime(&a, h->prof[3 * j], h->prof[3 * j + 1]));
          CK(cudaEventElapsedTime(&b2, h->prof[3 * j + 1], h->prof[3 * j + 2]));
          tr_ms += fused ? a : b2;
          fwd_ms += fused ? b2 : a;
        }
        fwd_launches += ran;
        tr_launches += ran;
      }
      k_before = hs.k;
      if (hs.done) break;
    }
    cudaGraphExecDestroy(gx);
    if (pst != BVLS_OK) return pst;
  } else {
    GraphKey key{K, o.screening, o.precision, o.restart, max_iter, o.single_pass, o.algorithm, o.tol, p.invL,
                 p.eps_star, p.eta_star, p.wstar != nullptr};
    cudaGraphExec_t exec = nullptr;
    for (auto& c : h->graphs)
      if (c.key == key && c.chunk == chunk) exec = c.exec;
    if (!exec) {
      if ((int)h->graphs.size() >= kGraphCache) {
        cudaGraphExecDestroy(h->graphs.front().exec);
        h->graphs.erase(h->graphs.begin());
      }
      // One graph for the whole solve: a while node whose body is one chunk of iterations
      // followed by the loop-control kernel, which ends the loop on the device once the stop
      // flag is set (no host polling, no chunk launched after the stop).
      cudaGraph_t g = nullptr;
      CK(cudaGraphCreate(&g, 0));
      cudaGraphConditionalHandle hc;
      cudaError_t e = cudaGraphConditionalHandleCreate(&hc, g, 1, cudaGraphCondAssignDefault);
      cudaGraphNodeParams np = {};
      np.type = cudaGraphNodeTypeConditional;
      np.conditional.handle = hc;
      np.conditional.type = cudaGraphCondTypeWhile;
      np.conditional.size = 1;
      cudaGraphNode_t node;
      if (e == cudaSuccess) e = cudaGraphAddNode(&node, g, nullptr, nullptr, 0, &np);
      cudaGraph_t body = e == cudaSuccess ? np.conditional.phGraph_out[0] : nullptr;
      if (e == cudaSuccess) e = cudaStreamBeginCaptureToGraph(h->s, body, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal);
      if (e == cudaSuccess) {
        cudaError_t e1 = enqueue_chunk(h, p, o, chunk, nullptr);
        if (e1 == cudaSuccess) e1 = launch_loop_ctl(h->b, hc, (int)std::min<long long>(max_chunks, 0x7fffffff), h->s);
        cudaError_t e2 = cudaStreamEndCapture(h->s, &body);
        e = e1 != cudaSuccess ? e1 : e2;
      }
      if (e == cudaSuccess) e = cudaGraphInstantiate(&exec, g, 0);
      cudaGraphDestroy(g);
      CK(e);
      h->graphs.push_back({key, chunk, exec});
    }
    CK(cudaGraphLaunch(exec, h->s));
    chunks_run = -1;  // counted on the device
  }
  CK(cudaStreamSynchronize(h->s));
  DevState hs;
  CK(cudaMemcpy(&hs, h->b.st, sizeof(DevState), cudaMemcpyDeviceToHost));
  if (hs.nonfinite) return set_err(BVLS_ENONFINITE, "y or x0 contains NaN or Inf");
  if (hs.error) return set_err(BVLS_ETIMEOUT, "a device-side wait exceeded its bound; results discarded");
  CK(launch_export(p, h->b, hs.out_slot, h->s));
  std::vector<RefOut> rout;
  float ref_ms = 0.f;
  if (o.refine) TRY(refine_shared(h, 1, h->y_dev, h->m, h->b.xout, h->n, h->b.flags, h->n, p.invL, &rout, &ref_ms));
  CK(cudaMemcpyAsync(x_out, h->b.xout, sizeof(double) * h->n, cudaMemcpyDefault, h->s));
  if (screened_out)
    CK(cudaMemcpyAsync(screened_out, h->b.flags, h->n, cudaMemcpyDefault, h->s));
  CK(cudaStreamSynchronize(h->s));
  if (info) {
    std::memset(info, 0, sizeof(*info));
    info->iters = hs.k;
    info->converged = hs.converged;
    info->n_preserved = hs.n_active;
    info->dual_mode = h->dual_mode;
    info->gap_evals = hs.gap_evals;
    info->gap = hs.gap;
    info->primal = hs.P[hs.out_slot];
    info->radius = hs.radius;
    info->L = 1.0 / p.invL;
    info->sum_preserved = hs.sum_active;
    info->sum_nonzero = hs.sum_nnz;
    info->fwd_ms = fwd_ms;
    info->tr_ms = tr_ms;
    info->fwd_launches = fwd_launches;
    info->tr_launches = tr_launches;
    const double chunks_done = chunks_run >= 0 ? (double)chunks_run : (double)hs.chunks;
    info->kernel_launches = (fused ? 3.0 : 2.0) + chunks_done * (double)(per_chunk + (chunks_run >= 0 ? 0 : 1));
    info->single_pass = fused ? (pers ? 2 : 1) : 0;
    info->t_choice = h->t_choice;
    if (!rout.empty()) {
      info->refined = rout[0].refined;
      info->refine_rounds = rout[0].rounds;
      info->n_free = rout[0].nfree;
      info->refine_cg_iters = rout[0].cg_iters;
      info->kkt = rout[0].kkt;
      info->refine_ms = ref_ms;
      info->refine_reason = rout[0].refined ? 0 : rout[0].reason;
      info->kernel_launches += 2.0;
    }
  }
  if (!hs.done) return set_err(BVLS_EMAXITER, "stopped after %lld chunks without the stop flag", max_chunks);
  if (!hs.converged) return set_err(BVLS_EMAXITER, "gap %.3e >= tol after %d iterations", hs.gap, hs.k);
  g_err.clear();
  return BVLS_OK;
}

}  // extern "C"

// ------------------------------------------------------------------ batched solve
namespace {

template <typename T>
bvls_status balloc(bvls_handle* h, T** p, size_t count) {
  void* q = nullptr;
  CK(cudaMalloc(&q, count * sizeof(T) + 256));
  h->b_allocs.push_back(q);
  *p = static_cast<T*>(q);
  return BVLS_OK;
}

// cuTensorMapEncodeTiled through the runtime's driver entry point: a 2D bf16 tensor of `rows`
// rows of `cols` contiguous elements, 128-byte swizzle, box_cols x box_rows.
bool encode_bf16_2d(CUtensorMap* map, const void* base, uint64_t cols, uint64_t rows, uint32_t box_cols,
                    uint32_t box_rows) {
  static const PFN_cuTensorMapEncodeTiled_v12000 fn = [] {
    void* f = nullptr;
    cudaDriverEntryPointQueryResult q = cudaDriverEntryPointSymbolNotFound;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &f, 12000, cudaEnableDefault, &q) != cudaSuccess ||
        q != cudaDriverEntryPointSuccess)
      return static_cast<PFN_cuTensorMapEncodeTiled_v12000>(nullptr);
    return reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(f);
  }();
  if (!fn) return false;
  const cuuint64_t dims[2] = {cols, rows};
  const cuuint64_t strides[1] = {cols * 2};
  const cuuint32_t box[2] = {box_cols, box_rows};
  const cuuint32_t es[2] = {1, 1};
  return fn(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<void*>(base), dims, strides, box, es,
            CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
            CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

// Gram matrix and the workspace for B instances.
bvls_status batch_prepare(bvls_handle* h, int B) {
  const int n = h->n;
  if (!h->bH) {
    h->b_npad = (n + kBTile - 1) / kBTile * kBTile;
    CK(batch_configure(h->m, h->b_npad));
    TRY(dalloc(h, &h->bH, (size_t)h->b_npad * h->b_npad));
    CK(launch_bgram(h->A, h->lda, h->m, n, h->b_npad, h->bH, h->s));
    if (!encode_bf16_2d(&h->b_tmH, h->bH, (uint64_t)h->b_npad, (uint64_t)h->b_npad, kBChunk, kBTile))
      return set_err(BVLS_ECUDA, "tensor map of the Gram matrix could not be encoded");
    std::vector<double> nrm(n), w(n);
    CK(cudaMemcpyAsync(nrm.data(), h->nrm, sizeof(double) * n, cudaMemcpyDeviceToHost, h->s));
    CK(cudaMemcpyAsync(w.data(), h->w, sizeof(double) * n, cudaMemcpyDeviceToHost, h->s));
    CK(cudaStreamSynchronize(h->s));
    std::vector<float> nrmf(n), wf(n);
    for (int j = 0; j < n; ++j) {
      float f = (float)nrm[j];
      if ((double)f < nrm[j]) f = std::nextafter(f, INFINITY);
      nrmf[j] = f;
      wf[j] = (float)w[j];
    }
    TRY(dalloc(h, &h->b_nrmf, n));
    TRY(dalloc(h, &h->b_wf, n));
    CK(cudaMemcpyAsync(h->b_nrmf, nrmf.data(), sizeof(float) * n, cudaMemcpyHostToDevice, h->s));
    CK(cudaMemcpyAsync(h->b_wf, wf.data(), sizeof(float) * n, cudaMemcpyHostToDevice, h->s));
    CK(cudaStreamSynchronize(h->s));
  }
  if (B <= h->b_cap) return BVLS_OK;
  if (h->b_exec) {
    cudaGraphExecDestroy(h->b_exec);
    h->b_exec = nullptr;
  }
  h->b_have_graph = false;
  CK(cudaStreamSynchronize(h->s));
  for (void* q : h->b_allocs) cudaFree(q);
  h->b_allocs.clear();
  h->b_cap = 0;
  const size_t np = (size_t)h->b_npad, MT = np / kBTile;
  BBuffers& b = h->bb;
  b = BBuffers{};
  for (int q = 0; q < 2; ++q) {
    TRY(balloc(h, &b.X[q], (size_t)B * np));
    TRY(balloc(h, &b.G[q], (size_t)B * np));
    TRY(balloc(h, &b.D[q], (size_t)(B + 1) * np));
    TRY(balloc(h, &b.tval[q], (size_t)B));
    TRY(balloc(h, &b.dotp[q], MT * B));
  }
  TRY(balloc(h, &b.Ge, (size_t)B * np));
  TRY(balloc(h, &b.flags, (size_t)B * np));
  TRY(balloc(h, &b.act, (size_t)B));
  TRY(balloc(h, &b.act_tmp, (size_t)B));
  TRY(balloc(h, &b.fin, (size_t)B));
  TRY(balloc(h, &b.xout, (size_t)B * n));
  TRY(balloc(h, &b.gap, (size_t)B));
  TRY(balloc(h, &b.primal, (size_t)B));
  TRY(balloc(h, &b.iters, (size_t)B));
  TRY(balloc(h, &b.status, (size_t)B));
  TRY(balloc(h, &b.npres, (size_t)B));
  TRY(balloc(h, &b.st, 1));
  TRY(balloc(h, &h->bY, (size_t)B * h->lda));
  TRY(balloc(h, &h->bX0, (size_t)B * n));
  h->b_cap = B;
  return BVLS_OK;
}

BParams make_bparams(bvls_handle* h, const bvls_opts& o, int max_iter, int B) {
  BParams p{};
  p.A = h->A;
  p.m = h->m;
  p.n = h->n;
  p.lda = h->lda;
  p.npad = h->b_npad;
  p.B = B;
  p.H = h->bH;
  p.l = h->l;
  p.u = h->u;
  p.nrm = h->nrm;
  p.w = h->w;
  p.nrmf = h->b_nrmf;
  p.wf = h->b_wf;
  p.jinf = h->jinf;
  p.l2 = h->l2;
  p.u2 = h->u2;
  const double L = o.lipschitz > 0.0 ? o.lipschitz : h->L;
  p.invL = 1.0 / L;
  p.invL2 = df2_from_double(p.invL);
  p.t_norm = h->t_norm;
  p.gamma_w = h->gamma_w;
  // Rounding of the evaluation products (see common.cuh for the double-float bound).  The
  // double-float recomputation of selected correlations: a lane sums ceil(m/32) products,
  // then 5 shuffle levels; the residual sums up to n products per row in double-float.
  const double dg = (h->m + 31) / 32 + 5;
  p.Cg2 = 2.0 * (dg + 2.0) * (dg + 2.0) * kU * kU + 4.0 * kU * kU + 2.0 * kU64;
  // the evaluation's correlations: blocked, interleaved sums (beval_chain)
  const BEvalChain ch = beval_chain(h->m, o.precision == BVLS_PREC_FP32X2 ? kBEvalIlvX2 : kBEvalIlvF32);
  p.erb = ch.rows;
  const double de = ch.depth;
  p.Cg = o.precision == BVLS_PREC_FP32X2 ? 2.0 * (de + 2.0) * (de + 2.0) * kU * kU + 4.0 * kU * kU + 2.0 * kU64
                                         : 1.01 * (de + 2.0) * kU + kU;
  const double df = h->n;
  p.Cf = 2.0 * (df + 2.0) * (df + 2.0) * kU * kU + 2.0 * kU * kU;
  p.Csub = 8.0 * kU * kU;
  p.tol = o.tol;
  p.max_iter = max_iter;
  p.dual_mode = h->dual_mode;
  p.screening = o.screening;
  p.restart = o.restart;
  p.K = o.screen_every;
  p.tmH = h->b_tmH;
  return p;
}

// Whether the batched solve runs the tensor-core steps between two evaluations as one
// persistent cluster launch (single_pass 1, npad <= 512) or one launch per step.
bool bsteps_persistent(const bvls_handle* h, const bvls_opts& o) {
  return o.single_pass == 1 && bsteps_supported(h->b_npad);
}

// One chunk of iterations k = kbase + j (kbase a multiple of K and even): evaluations at
// j % K == 0 (followed by the retirement of finished instances), tensor-core steps otherwise:
// the K - 1 steps after an evaluation in one launch when bsteps_persistent, else one launch
// each.  With events (profile), a persistent launch is timed as a whole and its later steps
// get empty intervals.
cudaError_t enqueue_bchunk(bvls_handle* h, const BParams& p, const bvls_opts& o, int chunk, cudaEvent_t* ev) {
  cudaError_t e = cudaSuccess;
  const int K = o.screen_every;
  const bool persist = bsteps_persistent(h, o);
  for (int j = 0; j < chunk && e == cudaSuccess; ++j) {
    if (ev) cudaEventRecordWithFlags(ev[2 * j], h->s, cudaEventRecordExternal);
    if (j % K == 0) {
      e = launch_beval(p, h->bb, j, o.precision, h->s);
      if (e == cudaSuccess) e = launch_bcompact(p, h->bb, h->s);
    } else if (!persist) {
      e = launch_bstep(p, h->bb, j, h->s);
    } else if (j % K == 1) {
      e = launch_bsteps(p, h->bb, j, std::min(K - 1, chunk - j), h->s);
    }
    if (ev) cudaEventRecordWithFlags(ev[2 * j + 1], h->s, cudaEventRecordExternal);
  }
  if (e == cudaSuccess) e = launch_bchunk_end(h->bb, chunk, h->s);
  return e;
}

}  // namespace

extern "C" bvls_status bvls_solve_batched(bvls_handle* h, int B, const float* Y, int ldy, const double* X0,
                                          const bvls_opts* opts, double* X_out, uint8_t* screened_out,
                                          double* gaps_out, int* iters_out, int* status_out,
                                          bvls_batch_info* info) {
  if (!h || !Y || !X_out) return set_err(BVLS_EINVAL, "handle, Y and X_out are required");
  if (B < 1 || B > kBMaxBatch) return set_err(BVLS_EINVAL, "B = %d outside [1, %d]", B, kBMaxBatch);
  if (ldy < h->m) return set_err(BVLS_EINVAL, "ldy = %d < m = %d", ldy, h->m);
  if (h->m > kBMaxRows || h->n > kBMaxCols)
    return set_err(BVLS_ENOTSUP, "batched solve supports m <= %d and n <= %d (got %d x %d)", kBMaxRows,
                   kBMaxCols, h->m, h->n);
  bvls_opts o;
  bvls_default_opts(&o);
  if (opts) o = *opts;
  TRY(validate_opts(o));
  const int K = o.screen_every;
  const int max_iter = (int)std::min<long long>((long long)(o.max_iter + K - 1) / K * K, 0x3fffffff);
  const int chunk = chunk_length(K);
  TRY(batch_prepare(h, B));
  const BParams p = make_bparams(h, o, max_iter, B);

  if (h->own_stream) {
    CK(cudaEventRecord(h->ev_in, h->user));
    CK(cudaStreamWaitEvent(h->s, h->ev_in, 0));
  }
  CK(cudaMemcpy2DAsync(h->bY, sizeof(float) * h->lda, Y, sizeof(float) * ldy, sizeof(float) * h->m, B,
                       cudaMemcpyDefault, h->s));
  BBuffers& bb = h->bb;
  bb.Y = h->bY;
  bb.X0 = nullptr;
  if (X0) {
    CK(cudaMemcpyAsync(h->bX0, X0, sizeof(double) * (size_t)B * h->n, cudaMemcpyDefault, h->s));
    bb.X0 = h->bX0;
  }
  CK(cudaMemsetAsync(bb.st, 0, sizeof(BState), h->s));
  CK(launch_binit(p, bb, h->s));

  const long long max_chunks = (max_iter + chunk - 1) / chunk + 2;
  // per chunk: chunk / K evaluations with their compaction, the steps (one launch per run of
  // K - 1 when persistent), the chunk-end kernel
  const long long per_chunk =
      (long long)(chunk / K) * (bsteps_persistent(h, o) ? (K > 1 ? 3 : 2) : K + 1) + 1;
  long long chunks_run = 0;
  double step_ms = 0.0, eval_ms = 0.0;
  int step_launches = 0, eval_launches = 0;
  if (o.profile) {
    while ((int)h->prof.size() < 2 * chunk) {
      cudaEvent_t e;
      CK(cudaEventCreate(&e));
      h->prof.push_back(e);
    }
    cudaGraph_t g = nullptr;
    cudaGraphExec_t gx = nullptr;
    CK(cudaStreamBeginCapture(h->s, cudaStreamCaptureModeThreadLocal));
    cudaError_t e1 = enqueue_bchunk(h, p, o, chunk, h->prof.data());
    cudaError_t e2 = cudaStreamEndCapture(h->s, &g);
    CK(e1);
    CK(e2);
    cudaError_t e3 = cudaGraphInstantiate(&gx, g, 0);
    cudaGraphDestroy(g);
    CK(e3);
    bvls_status pst = BVLS_OK;
    for (long long c = 0; c < max_chunks; ++c) {
      BState before;
      cudaError_t e = cudaMemcpyAsync(&before, bb.st, sizeof(BState), cudaMemcpyDeviceToHost, h->s);
      if (e == cudaSuccess) e = cudaGraphLaunch(gx, h->s);
      ++chunks_run;
      BState hs;
      if (e == cudaSuccess) e = cudaMemcpyAsync(&hs, bb.st, sizeof(BState), cudaMemcpyDeviceToHost, h->s);
      if (e == cudaSuccess) e = cudaStreamSynchronize(h->s);
      if (e != cudaSuccess) {
        pst = set_err(BVLS_ECUDA, "profile chunk: %s", cudaGetErrorString(e));
        break;
      }
      // iterations that ran with instances still active: up to the evaluation that ended
      // the solve (a finished solve leaves the rest of the chunk's kernels returning at entry)
      int ran = chunk;
      if (hs.done) ran = std::min(chunk, (hs.gap_evals - before.gap_evals - 1) * K + 1);
      for (int j = 0; j < ran; ++j) {
        float a = 0.f;
        CK(cudaEventElapsedTime(&a, h->prof[2 * j], h->prof[2 * j + 1]));
        if (j % K == 0) {
          eval_ms += a;
          ++eval_launches;
        } else {
          step_ms += a;
          ++step_launches;
        }
      }
      if (hs.done) break;
    }
    cudaGraphExecDestroy(gx);
    if (pst != BVLS_OK) return pst;
  } else {
    const double key[10] = {(double)K,  (double)chunk,    (double)o.precision, (double)o.screening,
                            (double)o.restart, o.tol, (double)max_iter, p.invL, (double)B,
                            bsteps_persistent(h, o) ? 3.0 : 2.0};
    if (!h->b_have_graph || std::memcmp(key, h->b_key, sizeof(key)) != 0) {
      if (h->b_exec) {
        cudaGraphExecDestroy(h->b_exec);
        h->b_exec = nullptr;
      }
      h->b_have_graph = false;
      // one graph for the whole batched solve: a while node around one chunk and the
      // loop-control kernel (ends the loop on the device when every instance has finished)
      cudaGraph_t g = nullptr;
      CK(cudaGraphCreate(&g, 0));
      cudaGraphConditionalHandle hc;
      cudaError_t e = cudaGraphConditionalHandleCreate(&hc, g, 1, cudaGraphCondAssignDefault);
      cudaGraphNodeParams np = {};
      np.type = cudaGraphNodeTypeConditional;
      np.conditional.handle = hc;
      np.conditional.type = cudaGraphCondTypeWhile;
      np.conditional.size = 1;
      cudaGraphNode_t node;
      if (e == cudaSuccess) e = cudaGraphAddNode(&node, g, nullptr, nullptr, 0, &np);
      cudaGraph_t body = e == cudaSuccess ? np.conditional.phGraph_out[0] : nullptr;
      if (e == cudaSuccess) e = cudaStreamBeginCaptureToGraph(h->s, body, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal);
      if (e == cudaSuccess) {
        cudaError_t e1 = enqueue_bchunk(h, p, o, chunk, nullptr);
        if (e1 == cudaSuccess) e1 = launch_bloop_ctl(bb, hc, (int)std::min<long long>(max_chunks, 0x7fffffff), h->s);
        cudaError_t e2 = cudaStreamEndCapture(h->s, &body);
        e = e1 != cudaSuccess ? e1 : e2;
      }
      if (e == cudaSuccess) e = cudaGraphInstantiate(&h->b_exec, g, 0);
      cudaGraphDestroy(g);
      CK(e);
      h->b_have_graph = true;
      std::memcpy(h->b_key, key, sizeof(key));
    }
    CK(cudaGraphLaunch(h->b_exec, h->s));
    chunks_run = -1;  // counted on the device
  }
  CK(cudaStreamSynchronize(h->s));
  BState hs;
  CK(cudaMemcpy(&hs, bb.st, sizeof(BState), cudaMemcpyDeviceToHost));
  if (hs.nonfinite) return set_err(BVLS_ENONFINITE, "Y or X0 contains NaN or Inf");
  if (hs.error) return set_err(BVLS_ETIMEOUT, "a device-side wait exceeded its bound; results discarded");
  if (!hs.done) return set_err(BVLS_ECUDA, "batched solve stopped after %d chunks without finishing", hs.chunks);
  std::vector<int> st_h(B), it_h(B);
  std::vector<RefOut> rout;
  float ref_ms = 0.f;
  if (o.refine)
    TRY(refine_shared(h, B, h->bY, h->lda, bb.xout, h->n, bb.flags, h->b_npad, p.invL, &rout, &ref_ms));
  CK(cudaMemcpyAsync(X_out, bb.xout, sizeof(double) * (size_t)B * h->n, cudaMemcpyDefault, h->s));
  if (screened_out)
    CK(cudaMemcpy2DAsync(screened_out, h->n, bb.flags, h->b_npad, h->n, B, cudaMemcpyDefault, h->s));
  if (gaps_out) CK(cudaMemcpyAsync(gaps_out, bb.gap, sizeof(double) * B, cudaMemcpyDefault, h->s));
  if (iters_out) CK(cudaMemcpyAsync(iters_out, bb.iters, sizeof(int) * B, cudaMemcpyDefault, h->s));
  if (status_out) CK(cudaMemcpyAsync(status_out, bb.status, sizeof(int) * B, cudaMemcpyDefault, h->s));
  CK(cudaMemcpyAsync(st_h.data(), bb.status, sizeof(int) * B, cudaMemcpyDeviceToHost, h->s));
  CK(cudaMemcpyAsync(it_h.data(), bb.iters, sizeof(int) * B, cudaMemcpyDeviceToHost, h->s));
  CK(cudaStreamSynchronize(h->s));
  int nconv = 0, itmax = 0;
  for (int q = 0; q < B; ++q) {
    nconv += st_h[q] == BVLS_OK;
    itmax = std::max(itmax, it_h[q]);
  }
  if (info) {
    std::memset(info, 0, sizeof(*info));
    info->iters_max = itmax;
    info->n_converged = nconv;
    info->gap_evals = hs.gap_evals;
    info->dual_mode = h->dual_mode;
    info->L = 1.0 / p.invL;
    info->sum_step = hs.sum_step;
    info->sum_eval = hs.sum_eval;
    info->sum_preserved = hs.sum_pres;
    info->step_ms = step_ms;
    info->eval_ms = eval_ms;
    info->step_launches = step_launches;
    info->eval_launches = eval_launches;
    info->kernel_launches =
        1.0 + (chunks_run >= 0 ? (double)chunks_run * (double)per_chunk : (double)hs.chunks * (double)(per_chunk + 1));
    info->steps_persistent = bsteps_persistent(h, o) ? 1 : 0;
    if (!rout.empty()) {
      for (const RefOut& r : rout) {
        info->refine_out_of_rounds += r.reason == 1;
        info->refine_not_unique += r.reason == 2;
        if (!r.refined) continue;
        ++info->n_refined;
        info->refine_free_max = std::max(info->refine_free_max, r.nfree);
        info->kkt_max = std::max(info->kkt_max, r.kkt);
      }
      info->refine_ms = ref_ms;
      info->kernel_launches += 2.0;
    }
  }
  if (nconv < B) return set_err(BVLS_EMAXITER, "%d of %d instances reached max_iter with gap >= tol", B - nconv, B);
  g_err.clear();
  return BVLS_OK;
}

// ------------------------------------------------------------------ backward
extern "C" void bvls_backward_default_opts(bvls_backward_opts* o) {
  if (!o) return;
  o->free_tol = 1e-9;
  o->cg_tol = 1e-12;
  o->cg_max_iter = 4000;
}

extern "C" bvls_status bvls_backward(bvls_handle* h, int B, const double* X, const float* Y, int ldy,
                                     const double* dLdX, const bvls_backward_opts* opts, double* dLdY,
                                     double* dLdA, int* status_out, bvls_backward_info* info) {
  if (!h || !X || !Y || !dLdX) return set_err(BVLS_EINVAL, "handle, X, Y and dLdX are required");
  if (B < 1 || ldy < h->m) return set_err(BVLS_EINVAL, "need B >= 1 and ldy >= m");
  bvls_backward_opts o;
  bvls_backward_default_opts(&o);
  if (opts) o = *opts;
  if (!(o.free_tol >= 0.0) || !(o.cg_tol >= 0.0) || o.cg_max_iter < 1)
    return set_err(BVLS_EINVAL, "invalid backward options");
  const int m = h->m, n = h->n;
  std::vector<void*> mem;
  auto alloc = [&](void** ptr, size_t bytes) -> cudaError_t {
    cudaError_t e = cudaMalloc(ptr, bytes + 16);
    if (e == cudaSuccess) mem.push_back(*ptr);
    return e;
  };
  auto release = [&]() {
    cudaStreamSynchronize(h->s);
    for (void* q : mem) cudaFree(q);
    mem.clear();
  };
#define BCK(call)                                                                              \
  do {                                                                                         \
    cudaError_t e_ = (call);                                                                   \
    if (e_ != cudaSuccess) {                                                                   \
      release();                                                                               \
      return set_err(e_ == cudaErrorMemoryAllocation ? BVLS_ENOMEM : BVLS_ECUDA, "%s failed: %s", \
                     #call, cudaGetErrorString(e_));                                           \
    }                                                                                          \
  } while (0)
  BwdParams p{};
  p.A = h->A;
  p.m = m;
  p.n = n;
  p.lda = h->lda;
  p.B = B;
  p.l = h->l;
  p.u = h->u;
  p.ldy = h->lda;
  p.free_tol = o.free_tol;
  p.cg_tol = o.cg_tol;
  p.cg_max_iter = o.cg_max_iter;
  double *dX = nullptr, *dV = nullptr, *dDY = nullptr, *dW = nullptr, *dQ = nullptr, *dR = nullptr, *dDA = nullptr;
  float* dY = nullptr;
  int *dSt = nullptr, *dIt = nullptr, *dNf = nullptr;
  BCK(alloc((void**)&dX, sizeof(double) * (size_t)B * n));
  BCK(alloc((void**)&dV, sizeof(double) * (size_t)B * n));
  BCK(alloc((void**)&dY, sizeof(float) * (size_t)B * h->lda));
  BCK(alloc((void**)&dDY, sizeof(double) * (size_t)B * m));
  BCK(alloc((void**)&dSt, sizeof(int) * (size_t)B));
  BCK(alloc((void**)&dIt, sizeof(int) * (size_t)B));
  BCK(alloc((void**)&dNf, sizeof(int) * (size_t)B));
  if (dLdA) {
    BCK(alloc((void**)&dW, sizeof(double) * (size_t)B * n));
    BCK(alloc((void**)&dQ, sizeof(double) * (size_t)B * m));
    BCK(alloc((void**)&dR, sizeof(double) * (size_t)B * m));
    BCK(alloc((void**)&dDA, sizeof(double) * (size_t)m * n));
  }
  if (h->own_stream) {
    BCK(cudaEventRecord(h->ev_in, h->user));
    BCK(cudaStreamWaitEvent(h->s, h->ev_in, 0));
  }
  BCK(cudaMemcpyAsync(dX, X, sizeof(double) * (size_t)B * n, cudaMemcpyDefault, h->s));
  BCK(cudaMemcpyAsync(dV, dLdX, sizeof(double) * (size_t)B * n, cudaMemcpyDefault, h->s));
  BCK(cudaMemcpy2DAsync(dY, sizeof(float) * h->lda, Y, sizeof(float) * ldy, sizeof(float) * m, B,
                        cudaMemcpyDefault, h->s));
  p.X = dX;
  p.dLdX = dV;
  p.Y = dY;
  p.dLdY = dDY;
  p.W = dW;
  p.Q = dQ;
  p.R = dR;
  p.status = dSt;
  p.iters = dIt;
  p.nfree = dNf;
  struct EventPair {   // destroyed on every return
    cudaEvent_t a = nullptr, b = nullptr;
    ~EventPair() {
      if (a) cudaEventDestroy(a);
      if (b) cudaEventDestroy(b);
    }
  } ev;
  if (info) {
    BCK(cudaEventCreate(&ev.a));
    BCK(cudaEventCreate(&ev.b));
    BCK(cudaEventRecord(ev.a, h->s));
  }
  BCK(launch_bwd(p, h->s));
  if (dLdA) BCK(launch_bwd_da(p, dDA, h->s));
  if (info) BCK(cudaEventRecord(ev.b, h->s));
  std::vector<int> st(B), it(B), nf(B);
  BCK(cudaMemcpyAsync(st.data(), dSt, sizeof(int) * B, cudaMemcpyDeviceToHost, h->s));
  BCK(cudaMemcpyAsync(it.data(), dIt, sizeof(int) * B, cudaMemcpyDeviceToHost, h->s));
  BCK(cudaMemcpyAsync(nf.data(), dNf, sizeof(int) * B, cudaMemcpyDeviceToHost, h->s));
  if (dLdY) BCK(cudaMemcpyAsync(dLdY, dDY, sizeof(double) * (size_t)B * m, cudaMemcpyDefault, h->s));
  if (dLdA) BCK(cudaMemcpyAsync(dLdA, dDA, sizeof(double) * (size_t)m * n, cudaMemcpyDefault, h->s));
  if (status_out) BCK(cudaMemcpyAsync(status_out, dSt, sizeof(int) * B, cudaMemcpyDefault, h->s));
  BCK(cudaStreamSynchronize(h->s));
  float kms = 0.f;
  if (info) BCK(cudaEventElapsedTime(&kms, ev.a, ev.b));
  release();
#undef BCK
  if (info) {
    std::memset(info, 0, sizeof(*info));
    for (int b = 0; b < B; ++b) {
      info->n_converged += st[b] == 0;
      info->n_iter_limit += st[b] == 1;
      info->n_too_large += st[b] == 2;
      info->n_not_unique += st[b] == 3;
      info->max_free = std::max(info->max_free, nf[b]);
      info->max_cg_iters = std::max(info->max_cg_iters, it[b]);
      info->cg_work += (double)it[b] * (double)nf[b];
    }
    info->kernel_ms = kms;
  }
  g_err.clear();
  return BVLS_OK;
}

// ------------------------------------------------------------------ ragged batch
// Autotuner choices of the ragged solve, per batch shape (process-wide, thread-safe).
struct RaggedTuneKey {
  long long B, cols, rows, elems;
  int screening, restart, auto_k;
  bool operator<(const RaggedTuneKey& o) const {
    return std::tie(B, cols, rows, elems, screening, restart, auto_k) <
           std::tie(o.B, o.cols, o.rows, o.elems, o.screening, o.restart, o.auto_k);
  }
};
struct RaggedTune {
  int tw, K;
};
std::mutex g_tune_mu;
std::map<RaggedTuneKey, RaggedTune>& tune_cache() {
  static std::map<RaggedTuneKey, RaggedTune> c;
  return c;
}
bool ragged_tune_lookup(const RaggedTuneKey& k, RaggedTune* t) {
  std::lock_guard<std::mutex> g(g_tune_mu);
  auto it = tune_cache().find(k);
  if (it == tune_cache().end()) return false;
  *t = it->second;
  return true;
}
void ragged_tune_store(const RaggedTuneKey& k, const RaggedTune& t) {
  std::lock_guard<std::mutex> g(g_tune_mu);
  tune_cache()[k] = t;
}

extern "C" bvls_status bvls_solve_ragged(int B, const bvls_problem* probs, const bvls_opts* opts, void* stream,
                                         double* const* x_out, uint8_t* const* screened_out, double* gaps_out,
                                         int* iters_out, int* status_out, bvls_ragged_info* info) {
  using clk = std::chrono::steady_clock;
  const auto t_start = clk::now();
  if (B < 1 || !probs || !x_out) return set_err(BVLS_EINVAL, "need B >= 1, probs and x_out");
  bvls_opts o;
  bvls_default_opts(&o);
  if (opts) o = *opts;
  const bool auto_k = o.screen_every == 0;   // the autotuner picks the screening period
  if (auto_k) o.screen_every = 10;
  TRY(validate_opts(o));
  // ---- layout
  std::vector<RInst> in(B);
  long long a_tot = 0, c_tot = 0, r_tot = 0, p_tot = 0, t_tot = 0;
  for (int k = 0; k < B; ++k) {
    const bvls_problem& q = probs[k];
    if (!q.A || !q.y || q.m < 1 || q.n < 1 || q.lda < q.m)
      return set_err(BVLS_EINVAL, "problem %d: need A, y, m >= 1, n >= 1, lda >= m", k);
    if (q.m > kRMaxRows) return set_err(BVLS_ENOTSUP, "problem %d: m = %d exceeds %d", k, q.m, kRMaxRows);
    RInst& r = in[k];
    std::memset(&r, 0, sizeof(r));
    r.m = q.m;
    r.n = q.n;
    r.lda = (q.m + 3) / 4 * 4;
    r.tiles_max = (q.n + kRTileMin - 1) / kRTileMin;   // room for the narrowest tiles
    r.a_off = a_tot;
    r.c_off = c_tot;
    r.r_off = r_tot;
    r.p_off = p_tot;
    r.t_off = t_tot;
    a_tot += (long long)r.lda * q.n;
    c_tot += q.n;
    r_tot += q.m;
    p_tot += (long long)r.tiles_max * q.m;
    t_tot += r.tiles_max;
  }
  std::vector<double> l(c_tot), u(c_tot);
  std::vector<float2> l2(c_tot), u2(c_tot);
  std::vector<uint8_t> jinf(c_tot);
  for (int k = 0; k < B; ++k) {
    for (int j = 0; j < in[k].n; ++j) {
      const long long c = in[k].c_off + j;
      const double lv = probs[k].l ? probs[k].l[j] : 0.0, uv = probs[k].u ? probs[k].u[j] : INFINITY;
      if (!std::isfinite(lv) || std::isnan(uv) || uv == -INFINITY || lv > uv)
        return set_err(BVLS_EINVAL, "problem %d, coordinate %d: need finite l <= u", k, j);
      l[c] = lv;
      u[c] = uv;
      l2[c] = df2_from_double(lv);
      u2[c] = df2_from_double(uv);
      jinf[c] = std::isinf(uv) ? 1 : 0;
    }
  }
  // ---- workspace
  std::vector<void*> mem;
  cudaStream_t s = nullptr;
  cudaEvent_t ev = nullptr;
  cudaGraphExec_t gx = nullptr;
  auto release = [&]() {
    if (s) cudaStreamSynchronize(s);
    if (gx) cudaGraphExecDestroy(gx);
    for (void* q : mem) cudaFree(q);
    if (ev) cudaEventDestroy(ev);
    if (s) cudaStreamDestroy(s);
  };
#define RCK(call)                                                                              \
  do {                                                                                         \
    cudaError_t e_ = (call);                                                                   \
    if (e_ != cudaSuccess) {                                                                   \
      release();                                                                               \
      return set_err(e_ == cudaErrorMemoryAllocation ? BVLS_ENOMEM : BVLS_ECUDA, "%s failed: %s", \
                     #call, cudaGetErrorString(e_));                                           \
    }                                                                                          \
  } while (0)
  auto alloc = [&](auto** ptr, size_t count) -> cudaError_t {
    void* q = nullptr;
    cudaError_t e = cudaMalloc(&q, count * sizeof(**ptr) + 256);
    if (e == cudaSuccess) {
      mem.push_back(q);
      *ptr = static_cast<std::remove_reference_t<decltype(*ptr)>>(q);
    }
    return e;
  };
  RCK(ragged_configure());
  RCK(cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking));
  RCK(cudaEventCreateWithFlags(&ev, cudaEventDisableTiming));
  RCK(cudaEventRecord(ev, static_cast<cudaStream_t>(stream)));
  RCK(cudaStreamWaitEvent(s, ev, 0));
  RBuf b{};
  float* A = nullptr;
  RInst* d_in = nullptr;
  float2 *d_l2 = nullptr, *d_u2 = nullptr;
  double *d_l = nullptr, *d_u = nullptr;
  uint8_t* d_jinf = nullptr;
  RCK(alloc(&A, (size_t)a_tot));
  RCK(alloc(&d_in, (size_t)B));
  RCK(alloc(&b.st, (size_t)B));
  for (int q = 0; q < 2; ++q) {
    RCK(alloc(&b.x[q], (size_t)c_tot));
    RCK(alloc(&b.g[q], (size_t)c_tot));
  }
  RCK(alloc(&d_l2, (size_t)c_tot));
  RCK(alloc(&d_u2, (size_t)c_tot));
  RCK(alloc(&d_l, (size_t)c_tot));
  RCK(alloc(&d_u, (size_t)c_tot));
  RCK(alloc(&b.nrm, (size_t)c_tot));
  RCK(alloc(&b.w, (size_t)c_tot));
  RCK(alloc(&d_jinf, (size_t)c_tot));
  RCK(alloc(&b.flags, (size_t)c_tot));
  RCK(alloc(&b.idx, (size_t)c_tot));
  RCK(alloc(&b.idx_tmp, (size_t)c_tot));
  RCK(alloc(&b.xout, (size_t)c_tot));
  RCK(alloc(&b.yh, (size_t)r_tot));
  RCK(alloc(&b.yl, (size_t)r_tot));
  RCK(alloc(&b.rh, (size_t)r_tot));
  RCK(alloc(&b.rl, (size_t)r_tot));
  RCK(alloc(&b.part, (size_t)p_tot));
  RCK(alloc(&b.tdot, (size_t)t_tot));
  RCK(alloc(&b.teps, (size_t)t_tot));
  RCK(alloc(&b.tiles, (size_t)t_tot));
  RCK(alloc(&b.n_tiles, 1));
  RCK(alloc(&b.n_act_inst, 1));
  RCK(alloc(&b.chunks, 1));
  RCK(alloc(&b.act, (size_t)B));
  RCK(alloc(&b.err, 1));
  RCK(alloc(&b.work, 1));
  RCK(alloc(&b.rblkP, (size_t)B * kRRowBlocks));
  RCK(alloc(&b.rcnt, (size_t)B));
  // refinement: the original y_k (y' is folded during the solve), scratch, descriptors
  float* y_orig = nullptr;
  double *ref_g = nullptr, *ref_xs = nullptr;
  RefDesc* ref_desc = nullptr;
  RefOut* ref_out = nullptr;
  if (o.refine) {
    RCK(alloc(&y_orig, (size_t)r_tot));
    RCK(alloc(&ref_g, (size_t)c_tot));
    RCK(alloc(&ref_xs, (size_t)c_tot));
    RCK(alloc(&ref_desc, (size_t)B));
    RCK(alloc(&ref_out, (size_t)B));
  }
  b.A = A;
  b.inst = d_in;
  b.l2 = d_l2;
  b.u2 = d_u2;
  b.l = d_l;
  b.u = d_u;
  b.jinf = d_jinf;
  b.B = B;
  b.tw = 16;
  b.screening = o.screening;
  b.restart = o.restart;
  b.tol = o.tol;
  int K = o.screen_every;
  b.K = K;
  b.max_iter = (int)std::min<long long>((long long)(o.max_iter + K - 1) / K * K, 0x3fffffff);
  // ---- copies
  RCK(cudaMemsetAsync(A, 0, sizeof(float) * (size_t)a_tot, s));
  RCK(cudaMemsetAsync(b.yl, 0, sizeof(float) * (size_t)r_tot, s));
  RCK(cudaMemsetAsync(b.err, 0, sizeof(unsigned), s));
  RCK(cudaMemsetAsync(b.chunks, 0, sizeof(int), s));
  RCK(cudaMemsetAsync(b.rcnt, 0, sizeof(unsigned) * B, s));
  for (int k = 0; k < B; ++k) {
    const bvls_problem& q = probs[k];
    RCK(cudaMemcpy2DAsync(A + in[k].a_off, sizeof(float) * in[k].lda, q.A, sizeof(float) * q.lda,
                          sizeof(float) * q.m, q.n, cudaMemcpyDefault, s));
    RCK(cudaMemcpyAsync(b.yh + in[k].r_off, q.y, sizeof(float) * q.m, cudaMemcpyDefault, s));
    if (y_orig) RCK(cudaMemcpyAsync(y_orig + in[k].r_off, q.y, sizeof(float) * q.m, cudaMemcpyDefault, s));
  }
  RCK(cudaMemcpyAsync(d_l, l.data(), sizeof(double) * c_tot, cudaMemcpyHostToDevice, s));
  RCK(cudaMemcpyAsync(d_u, u.data(), sizeof(double) * c_tot, cudaMemcpyHostToDevice, s));
  RCK(cudaMemcpyAsync(d_l2, l2.data(), sizeof(float2) * c_tot, cudaMemcpyHostToDevice, s));
  RCK(cudaMemcpyAsync(d_u2, u2.data(), sizeof(float2) * c_tot, cudaMemcpyHostToDevice, s));
  RCK(cudaMemcpyAsync(d_jinf, jinf.data(), c_tot, cudaMemcpyHostToDevice, s));
  RCK(cudaMemcpyAsync(d_in, in.data(), sizeof(RInst) * B, cudaMemcpyHostToDevice, s));
  // ---- column norms, w = A^T (-1), dual modes
  RCK(launch_rnorms(b, c_tot, s));
  std::vector<double> nrm(c_tot), w(c_tot);
  RCK(cudaMemcpyAsync(nrm.data(), b.nrm, sizeof(double) * c_tot, cudaMemcpyDeviceToHost, s));
  RCK(cudaMemcpyAsync(w.data(), b.w, sizeof(double) * c_tot, cudaMemcpyDeviceToHost, s));
  unsigned herr = 0;
  RCK(cudaMemcpyAsync(&herr, b.err, sizeof(unsigned), cudaMemcpyDeviceToHost, s));
  RCK(cudaStreamSynchronize(s));
  if (herr) {
    release();
    return set_err(BVLS_ENONFINITE, "an A_k contains NaN or Inf");
  }
  int n_trans = 0, n_zero = 0;
  for (int k = 0; k < B; ++k) {
    RInst& r = in[k];
    bool any_inf = false, ok = true;
    const double gamma = 1.01 * (r.m + 8) * kU64;
    r.t_norm = std::sqrt((double)r.m);
    for (int j = 0; j < r.n; ++j) {
      const long long c = r.c_off + j;
      if (!jinf[c]) continue;
      any_inf = true;
      if (nrm[c] > 0.0 && !(w[c] + gamma * nrm[c] * r.t_norm < 0.0)) ok = false;
    }
    r.dual_mode = !any_inf ? kScaling : ok ? kTranslation : kZero;
    r.gamma_w = gamma;
    n_trans += r.dual_mode == kTranslation;
    n_zero += r.dual_mode == kZero;
    const double dg = ((r.m + 3) / 4 + 31) / 32 + 7;
    r.Cg = 2.0 * (dg + 2.0) * (dg + 2.0) * kU * kU + 4.0 * kU * kU + 2.0 * kU64;
    const double df = kRTileMax + r.tiles_max + 2;   // any tile width: <= 32 columns, <= tiles_max tiles
    r.Cf = 2.0 * (df + 2.0) * (df + 2.0) * kU * kU + 2.0 * kU * kU;
    r.Csub = 8.0 * kU * kU;
    r.invL = 1.0;
  }
  RCK(cudaMemcpyAsync(d_in, in.data(), sizeof(RInst) * B, cudaMemcpyHostToDevice, s));
  // ---- step constants: 40 power iterations on every instance at once
  const int max_tiles = (int)t_tot;
  b.power = 1;
  RCK(launch_rinit(b, c_tot, 1, s));
  RCK(launch_rfwd(b, s));
  RCK(launch_rtiles(b, s));
  for (int it = 0; it < 40; ++it) {
    RCK(launch_rpass(b, max_tiles, it & 1, 0, s));
    RCK(launch_rresid(b, it & 1, s));
  }
  std::vector<RState> hs(B);
  RCK(cudaMemcpyAsync(hs.data(), b.st, sizeof(RState) * B, cudaMemcpyDeviceToHost, s));
  RCK(cudaStreamSynchronize(s));
  for (int k = 0; k < B; ++k) in[k].invL = hs[k].pw_lambda > 0.0 ? 1.0 / (1.05 * hs[k].pw_lambda) : 1.0;
  RCK(cudaMemcpyAsync(d_in, in.data(), sizeof(RInst) * B, cudaMemcpyHostToDevice, s));
  // ---- autotuner
  const auto t_tune0 = clk::now();
  b.power = 0;
  bool tuned_now = false;
  {
    RaggedTuneKey key{B, c_tot, r_tot, a_tot, o.screening, o.restart, auto_k ? 1 : 0};
    RaggedTune t{};
    if (ragged_tune_lookup(key, &t)) {
      b.tw = t.tw;
      if (auto_k) K = t.K;
    } else {
      tuned_now = true;
      cudaEvent_t e0 = nullptr, e1 = nullptr;
      RCK(cudaEventCreate(&e0));
      RCK(cudaEventCreate(&e1));
      auto timed = [&](auto&& body) -> float {
        float ms = -1.f;
        if (cudaEventRecord(e0, s) != cudaSuccess) return ms;
        if (body() != cudaSuccess) return ms;
        if (cudaEventRecord(e1, s) != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess) return ms;
        cudaEventElapsedTime(&ms, e0, e1);
        return ms;
      };
      // tile width: eight plain iterations from the start point per width (the iterates do
      // not depend on it, only the tile kernel's speed does)
      float best = 0.f;
      for (int cand : {8, 16, 32}) {
        b.tw = cand;
        RCK(launch_rinit(b, c_tot, 0, s));
        RCK(launch_rfwd(b, s));
        RCK(launch_rtiles(b, s));
        RCK(launch_rpass(b, max_tiles, 0, 0, s));
        RCK(launch_rresid(b, 0, s));
        const float ms = timed([&]() {
          cudaError_t e = cudaSuccess;
          for (int it = 1; it <= 8 && e == cudaSuccess; ++it) {
            e = launch_rpass(b, max_tiles, it & 1, 0, s);
            if (e == cudaSuccess) e = launch_rresid(b, it & 1, s);
          }
          return e;
        });
        if (ms < 0.f) {
          const cudaError_t e = cudaGetLastError();
          RCK(e != cudaSuccess ? e : cudaErrorUnknown);
        }
        if (cand == 8 || ms < best) {
          best = ms;
          t.tw = cand;
        }
      }
      b.tw = t.tw;
      t.K = K;
      if (auto_k) {
        // screening period: 20 iterations (gap, test, compaction, folds included) from the
        // start point per candidate, each as one plain graph; the folds change y', which is
        // restored afterwards
        float* y0 = nullptr;
        RCK(alloc(&y0, (size_t)r_tot));
        RCK(cudaMemcpyAsync(y0, b.yh, sizeof(float) * r_tot, cudaMemcpyDeviceToDevice, s));
        for (int cand : {5, 10, 20}) {
          RCK(cudaMemcpyAsync(b.yh, y0, sizeof(float) * r_tot, cudaMemcpyDeviceToDevice, s));
          RCK(cudaMemsetAsync(b.yl, 0, sizeof(float) * r_tot, s));
          RCK(launch_rinit(b, c_tot, 0, s));
          RCK(launch_rfwd(b, s));
          RCK(launch_rtiles(b, s));
          cudaGraph_t g = nullptr;
          cudaGraphExec_t px = nullptr;
          RCK(cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal));
          cudaError_t e1 = cudaSuccess;
          for (int j = 0; j < 20 && e1 == cudaSuccess; ++j) {
            const bool gap_iter = ((j + 1) % cand) == 0;
            e1 = launch_rpass(b, max_tiles, j & 1, gap_iter ? 1 : 0, s);
            if (e1 == cudaSuccess) e1 = launch_rresid(b, j & 1, s);
            if (e1 == cudaSuccess && gap_iter) e1 = launch_rgap(b, j & 1, s);
            if (e1 == cudaSuccess && gap_iter) e1 = launch_rtiles(b, s);
          }
          const cudaError_t e2 = cudaStreamEndCapture(s, &g);
          RCK(e1);
          RCK(e2);
          const cudaError_t e3 = cudaGraphInstantiate(&px, g, 0);
          cudaGraphDestroy(g);
          RCK(e3);
          const float ms = timed([&]() { return cudaGraphLaunch(px, s); });
          cudaGraphExecDestroy(px);
          if (ms < 0.f) {
            const cudaError_t e = cudaGetLastError();
            RCK(e != cudaSuccess ? e : cudaErrorUnknown);
          }
          if (cand == 5 || ms < best) {
            best = ms;
            t.K = cand;
          }
        }
        RCK(cudaMemcpyAsync(b.yh, y0, sizeof(float) * r_tot, cudaMemcpyDeviceToDevice, s));
        RCK(cudaMemsetAsync(b.yl, 0, sizeof(float) * r_tot, s));
        K = t.K;
      }
      cudaEventDestroy(e0);
      cudaEventDestroy(e1);
      ragged_tune_store(key, t);
    }
    b.K = K;
    b.max_iter = (int)std::min<long long>((long long)(o.max_iter + K - 1) / K * K, 0x3fffffff);
  }
  const auto t_setup = clk::now();
  // ---- solve: one graph, a while node around one chunk
  b.power = 0;
  RCK(cudaMemsetAsync(b.work, 0, sizeof(double), s));
  RCK(launch_rinit(b, c_tot, 0, s));
  RCK(launch_rfwd(b, s));
  RCK(launch_rtiles(b, s));
  const int chunk = chunk_length(K);
  const long long max_chunks = (b.max_iter + chunk - 1) / chunk + 2;
  auto enqueue_rchunk = [&]() -> cudaError_t {
    cudaError_t e1 = cudaSuccess;
    for (int j = 0; j < chunk && e1 == cudaSuccess; ++j) {
      const bool gap_iter = ((j + 1) % K) == 0;
      e1 = launch_rpass(b, max_tiles, j & 1, gap_iter ? 1 : 0, s);
      if (e1 == cudaSuccess) e1 = launch_rresid(b, j & 1, s);
      if (e1 == cudaSuccess && gap_iter) e1 = launch_rgap(b, j & 1, s);
      if (e1 == cudaSuccess && gap_iter) e1 = launch_rtiles(b, s);
    }
    return e1;
  };
  if (o.profile == 2) {
    // every kernel launched directly from the host, a chunk at a time, until no instance is
    // active (no CUDA graph, so a profiler sees each launch)
    for (long long c = 0; c < max_chunks; ++c) {
      RCK(enqueue_rchunk());
      int act = 0;
      unsigned e = 0;
      RCK(cudaMemcpyAsync(&act, b.n_act_inst, sizeof(int), cudaMemcpyDeviceToHost, s));
      RCK(cudaMemcpyAsync(&e, b.err, sizeof(unsigned), cudaMemcpyDeviceToHost, s));
      RCK(cudaStreamSynchronize(s));
      if (act == 0 || e) break;
    }
  } else {
    cudaGraph_t g = nullptr;
    RCK(cudaGraphCreate(&g, 0));
    cudaGraphConditionalHandle hc;
    cudaError_t e = cudaGraphConditionalHandleCreate(&hc, g, 1, cudaGraphCondAssignDefault);
    cudaGraphNodeParams np = {};
    np.type = cudaGraphNodeTypeConditional;
    np.conditional.handle = hc;
    np.conditional.type = cudaGraphCondTypeWhile;
    np.conditional.size = 1;
    cudaGraphNode_t node;
    if (e == cudaSuccess) e = cudaGraphAddNode(&node, g, nullptr, nullptr, 0, &np);
    cudaGraph_t body = e == cudaSuccess ? np.conditional.phGraph_out[0] : nullptr;
    if (e == cudaSuccess) e = cudaStreamBeginCaptureToGraph(s, body, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal);
    if (e == cudaSuccess) {
      cudaError_t e1 = enqueue_rchunk();
      if (e1 == cudaSuccess) e1 = launch_rloop_ctl(b, hc, (int)std::min<long long>(max_chunks, 0x7fffffff), s);
      cudaError_t e2 = cudaStreamEndCapture(s, &body);
      e = e1 != cudaSuccess ? e1 : e2;
    }
    if (e == cudaSuccess) e = cudaGraphInstantiate(&gx, g, 0);
    cudaGraphDestroy(g);
    RCK(e);
    RCK(cudaGraphLaunch(gx, s));
  }
  RCK(launch_rexport(b, s));
  RCK(cudaMemcpyAsync(hs.data(), b.st, sizeof(RState) * B, cudaMemcpyDeviceToHost, s));
  int hchunks = 0;
  double hwork = 0.0;
  RCK(cudaMemcpyAsync(&hchunks, b.chunks, sizeof(int), cudaMemcpyDeviceToHost, s));
  RCK(cudaMemcpyAsync(&hwork, b.work, sizeof(double), cudaMemcpyDeviceToHost, s));
  RCK(cudaMemcpyAsync(&herr, b.err, sizeof(unsigned), cudaMemcpyDeviceToHost, s));
  RCK(cudaStreamSynchronize(s));
  const auto t_solve = clk::now();
  if (herr) {
    release();
    return set_err(BVLS_ENONFINITE, "a y_k contains NaN or Inf");
  }
  int nconv = 0, itmax = 0;
  for (int k = 0; k < B; ++k) {
    if (!hs[k].done) {
      release();
      return set_err(BVLS_ECUDA, "instance %d did not finish after %d chunks", k, hchunks);
    }
    nconv += hs[k].converged;
    itmax = std::max(itmax, hs[k].k);
  }
  std::vector<RefOut> rout;
  float ref_ms = 0.f;
  if (o.refine) {
    std::vector<RefDesc> dh(B);
    int m_max = 1, f_max = 1;
    for (int k = 0; k < B; ++k) {
      RefDesc& d = dh[k];
      d.A = A + in[k].a_off;
      d.y = y_orig + in[k].r_off;
      d.l = d_l + in[k].c_off;
      d.u = d_u + in[k].c_off;
      d.x = b.xout + in[k].c_off;
      d.flags = b.flags + in[k].c_off;
      d.g = ref_g + in[k].c_off;
      d.xsave = ref_xs + in[k].c_off;
      d.step = in[k].invL;
      d.m = in[k].m;
      d.n = in[k].n;
      d.lda = in[k].lda;
      m_max = std::max(m_max, in[k].m);
      f_max = std::max(f_max, std::min(in[k].m, in[k].n));
    }
    RCK(cudaMemcpyAsync(ref_desc, dh.data(), sizeof(RefDesc) * B, cudaMemcpyHostToDevice, s));
    cudaEvent_t r0 = nullptr, r1 = nullptr;
    RCK(cudaEventCreate(&r0));
    RCK(cudaEventCreate(&r1));
    cudaError_t e = cudaEventRecord(r0, s);
    if (e == cudaSuccess) e = launch_refine(ref_params(ref_desc, ref_out, B), m_max, std::min(f_max, kRefMaxFree), s);
    if (e == cudaSuccess) e = cudaEventRecord(r1, s);
    rout.resize(B);
    if (e == cudaSuccess) e = cudaMemcpyAsync(rout.data(), ref_out, sizeof(RefOut) * B, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ref_ms, r0, r1);
    cudaEventDestroy(r0);
    cudaEventDestroy(r1);
    RCK(e);
  }
  for (int k = 0; k < B; ++k) {
    RCK(cudaMemcpyAsync(x_out[k], b.xout + in[k].c_off, sizeof(double) * in[k].n, cudaMemcpyDefault, s));
    if (screened_out && screened_out[k])
      RCK(cudaMemcpyAsync(screened_out[k], b.flags + in[k].c_off, in[k].n, cudaMemcpyDefault, s));
    if (gaps_out) gaps_out[k] = hs[k].gap;
    if (iters_out) iters_out[k] = hs[k].k;
    if (status_out) status_out[k] = hs[k].converged ? BVLS_OK : BVLS_EMAXITER;
  }
  RCK(cudaStreamSynchronize(s));
  release();
#undef RCK
  if (info) {
    std::memset(info, 0, sizeof(*info));
    info->iters_max = itmax;
    info->n_converged = nconv;
    info->n_translation = n_trans;
    info->n_zero = n_zero;
    info->chunks = hchunks;
    info->tiles_max = max_tiles;
    info->tile_cols = b.tw;
    info->screen_every = K;
    info->tuned = tuned_now ? 1 : 0;
    info->tune_ms = std::chrono::duration<double, std::milli>(t_setup - t_tune0).count();
    info->setup_ms = std::chrono::duration<double, std::milli>(t_setup - t_start).count();
    info->solve_ms = std::chrono::duration<double, std::milli>(t_solve - t_setup).count();
    for (const RefOut& r : rout) {
      info->refine_out_of_rounds += r.reason == 1;
      info->refine_not_unique += r.reason == 2;
      if (!r.refined) continue;
      ++info->n_refined;
      info->refine_free_max = std::max(info->refine_free_max, r.nfree);
      info->kkt_max = std::max(info->kkt_max, r.kkt);
    }
    info->refine_ms = ref_ms;
    info->sum_rows_cols = hwork;
  }
  if (nconv < B) return set_err(BVLS_EMAXITER, "%d of %d instances reached max_iter with gap >= tol", B - nconv, B);
  g_err.clear();
  return BVLS_OK;
}

