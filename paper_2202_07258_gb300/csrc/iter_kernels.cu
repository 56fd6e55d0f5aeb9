// Kernels of one iteration of the screened accelerated projected-gradient solver.
//
// Per iteration k, on the preserved set S (index list idx[0..n_active)):
//   k_fwd   q = A_S x_S (column-parallel partial sums, last block per row tile reduces),
//           r = y' - q, P = 1/2 ||r||^2.                           (Eq. (decmposition_fwd))
//   k_tr    g = A_S^T r (one warp per two columns, r staged in shared memory) with the
//           FISTA step fused in its epilogue: g_v = (1+b) g_k - b g_{k-1} = A_S^T (y' - A v),
//           x_{k+1} = clip(v + g_v / L, l, u), the restart test and the translation step
//           candidate of Section 4.2.
// Every K-th iteration (Algorithm 1's screening step, evaluated at x_k):
//   k_gap     duality gap of Eq. (Dual_Gap) in its nonnegative-sum form plus rounding
//             bounds, radius of Eq. (GAP_Safe_sph), stop test.
//   k_test    sphere test of Eq. (safe_rule) with the rounding margin added to the radius;
//             fixes the coordinates that pass and already sit at that bound in x_k and x_{k+1}.
//   k_compact stable compaction of the preserved index list; list of fixed columns with a
//             nonzero bound, folded into y' by k_fwd<fold> (remark after Eq. (decmposition_fwd)).
#include "common.cuh"

namespace bvls {

// ------------------------------------------------------------------ small helpers
template <int PREC>
__device__ __forceinline__ void acc4(float* s, float* c, const float4 a, float xh, float xl) {
  if (PREC == kX2) {
    df_fma(s[0], c[0], a.x, xh, xl);
    df_fma(s[1], c[1], a.y, xh, xl);
    df_fma(s[2], c[2], a.z, xh, xl);
    df_fma(s[3], c[3], a.w, xh, xl);
  } else {
    s[0] = fmaf(a.x, xh, s[0]);
    s[1] = fmaf(a.y, xh, s[1]);
    s[2] = fmaf(a.z, xh, s[2]);
    s[3] = fmaf(a.w, xh, s[3]);
  }
}

// per-component products with a vector: (s_c, c_c) += a_c * (h_c + l_c)
template <int PREC>
__device__ __forceinline__ void acc4v(float* s, float* c, const float4 a, const float4 h, const float4 l) {
  if (PREC == kX2) {
    df_fma(s[0], c[0], a.x, h.x, l.x);
    df_fma(s[1], c[1], a.y, h.y, l.y);
    df_fma(s[2], c[2], a.z, h.z, l.z);
    df_fma(s[3], c[3], a.w, h.w, l.w);
  } else {
    s[0] = fmaf(a.x, h.x, s[0]);
    s[1] = fmaf(a.y, h.y, s[1]);
    s[2] = fmaf(a.z, h.z, s[2]);
    s[3] = fmaf(a.w, h.w, s[3]);
  }
}

template <int PREC>
__device__ __forceinline__ void merge(float& s, float& c, float s2, float c2) {
  if (PREC == kX2) {
    df_add(s, c, s2, c2);
  } else {
    s += s2;
  }
}

// Block-wide sum of up to 4 doubles; result valid in thread 0.  blockDim.x multiple of 32.
template <int N>
__device__ __forceinline__ void block_sum(double (&v)[N], double* sh /* >= 32*N */) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
#pragma unroll
  for (int q = 0; q < N; ++q) v[q] = warp_sum_d(v[q]);
  if (lane == 0) {
#pragma unroll
    for (int q = 0; q < N; ++q) sh[warp * N + q] = v[q];
  }
  __syncthreads();
  if (warp == 0) {
#pragma unroll
    for (int q = 0; q < N; ++q) {
      double t = lane < nw ? sh[lane * N + q] : 0.0;
      v[q] = warp_sum_d(t);
    }
  }
  __syncthreads();
}

// Returns true in every thread of the block that arrived last at *cnt (and resets it).
__device__ __forceinline__ bool last_block(unsigned int* cnt, unsigned int total) {
  __shared__ int s_last;
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) {
    unsigned int prev = atomicAdd(cnt, 1u);
    s_last = (prev == total - 1);
    if (s_last) *cnt = 0u;
  }
  __syncthreads();
  if (s_last) __threadfence();
  return s_last;
}

// ------------------------------------------------------------------ init
__global__ void k_init_state(Params p, Buffers b) {
  DevState* st = b.st;
  __shared__ double sh[32];
  double acc = 0.0;
  int bad = 0;
  for (int i = threadIdx.x; i < p.m; i += blockDim.x) {
    float v = b.y_in[i];
    if (!isfinite(v)) bad = 1;
    acc += (double)v * (double)v;
  }
  acc = warp_sum_d(acc);
  bad = __syncthreads_or(bad);
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    double s = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) s += sh[w];
    st->k = 0;
    st->done = bad;
    st->stop = 0;
    st->converged = 0;
    st->n_active = p.n;
    st->n_pins = 0;
    st->n_fold = 0;
    st->out_slot = 0;
    st->gap_evals = 0;
    st->nonfinite = bad;
    st->chunks = 0;
    st->t = 1.0;
    st->ti = 0;
    st->P[0] = 0.0;
    st->P[1] = 0.0;
    st->error = 0;
    st->eps = 0.0;
    st->gap = INFINITY;
    st->radius = INFINITY;
    st->eta = 0.0;
    st->E_fold = 0.0;
    st->S_fold = 0.0;
    st->y_norm = sqrt(s);
    st->sum_active = 0.0;
    st->sum_nnz = 0.0;
    st->cnt_tr = st->cnt_gap = st->cnt_fwd = st->cnt_resid = 0u;
    st->gbase = 0ull;
  }
  if (b.gbar)   // the persistent pass counts its grid barriers from 0 in every solve
    for (int i = threadIdx.x; i < kMaxGridFlags; i += blockDim.x) b.gbar[i] = 0u;
}

__global__ void k_init_arrays(Params p, Buffers b) {
  const int stride = gridDim.x * blockDim.x;
  for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < p.n; j += stride) {
    double x = b.x0_in ? b.x0_in[j] : 0.0;
    if (!isfinite(x)) {
      atomicOr(&b.st->nonfinite, 1);
      atomicOr(&b.st->done, 1);
      x = 0.0;
    }
    x = fmin(fmax(x, p.l[j]), p.u[j]);
    float2 x2 = df2_from_double(x);
    if (df2_lt(x2, p.l2[j])) x2 = p.l2[j];   // keep the pair inside the box exactly
    if (df2_lt(p.u2[j], x2)) x2 = p.u2[j];
    b.x[0][j] = x2;
    b.x[1][j] = x2;
    b.g[0][j] = make_float2(0.f, 0.f);
    b.g[1][j] = make_float2(0.f, 0.f);
    b.idx[j] = j;
    b.flags[j] = 0;
  }
  // y' = y (exact as a double-float); r padding rows stay zero.
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < p.m4; i += stride) {
    float v = i < p.m ? b.y_in[i] : 0.0f;
    b.yh[i] = v;
    b.yl[i] = 0.0f;
    b.rh[i] = 0.0f;
    b.rl[i] = 0.0f;
  }
}

__global__ void k_loop_ctl(DevState* st, cudaGraphConditionalHandle h, int max_chunks) {
  if (threadIdx.x == 0 && blockIdx.x == 0) {
    const int c = ++st->chunks;
    if (st->done || st->error || c >= max_chunks) cudaGraphSetConditional(h, 0);
  }
}

cudaError_t launch_loop_ctl(const Buffers& b, cudaGraphConditionalHandle h, int max_chunks, cudaStream_t s) {
  k_loop_ctl<<<1, 32, 0, s>>>(b.st, h, max_chunks);
  return cudaGetLastError();
}

cudaError_t launch_init(const Params& p, const Buffers& b, cudaStream_t s) {
  k_init_state<<<1, 1024, 0, s>>>(p, b);
  int blocks = (max(p.n, p.m4) + 255) / 256;
  blocks = min(blocks, 4096);
  k_init_arrays<<<blocks, 256, 0, s>>>(p, b);
  return cudaGetLastError();
}

// ------------------------------------------------------------------ q = A_S x_S
// grid (fwd_tiles, fwd_chunks), block kFwdThreads.  Column chunk c of the list is split
// over kFwdWarps warps; each lane owns 4 consecutive rows (one float4 per column) and two
// accumulator sets (alternate columns).  Columns whose x_j is exactly 0 are skipped: they
// add exact zeros.  FOLD=true folds y' <- y' - A_F b_F for the list of fixed columns.
template <int PREC, bool FOLD>
__global__ void __launch_bounds__(kFwdThreads) k_fwd(Params p, Buffers b, int slot) {
  DevState* st = b.st;
  if (st->done) return;
  const int cnt = FOLD ? st->n_fold : st->n_active;
  if (FOLD && cnt == 0) return;
  const int* list = FOLD ? b.fold : b.idx;
  const float2* __restrict__ xv = b.x[slot];
  const int nch = gridDim.y;
  const int per = (cnt + nch - 1) / nch;
  const int cb = blockIdx.y * per;
  const int ce = min(cnt, cb + per);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int row = blockIdx.x * kFwdRows + 4 * lane;
  const bool live = row < p.lda;

  __shared__ int s_col[kFwdStage];
  __shared__ float s_xh[kFwdStage];
  __shared__ float s_xl[kFwdStage];
  __shared__ int s_wcnt[kFwdThreads / 32];
  __shared__ float2 s_red[kFwdWarps - 1][kFwdRows];

  float s0[4] = {0.f, 0.f, 0.f, 0.f}, c0[4] = {0.f, 0.f, 0.f, 0.f};
  float s1[4] = {0.f, 0.f, 0.f, 0.f}, c1[4] = {0.f, 0.f, 0.f, 0.f};

  for (int base = cb; base < ce; base += kFwdStage) {
    const int nb = min(kFwdStage, ce - base);
    __syncthreads();
    // Stage the nonzero entries of this batch: two candidates per thread, block prefix
    // over warp ballots keeps the list order.
    int pos[2];
    bool keep[2];
    int j_c[2];
    float2 x_c[2];
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const int q = threadIdx.x + h * kFwdThreads;
      keep[h] = false;
      if (q < nb) {
        j_c[h] = list[base + q];
        x_c[h] = xv[j_c[h]];
        keep[h] = df2_nonzero(x_c[h]);
      }
    }
    int total = 0;
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const unsigned bal = __ballot_sync(0xffffffffu, keep[h]);
      if (lane == 0) s_wcnt[warp] = __popc(bal);
      __syncthreads();
      int before = total;
      for (int w = 0; w < warp; ++w) before += s_wcnt[w];
      int all = total;
      for (int w = 0; w < kFwdThreads / 32; ++w) all += s_wcnt[w];
      pos[h] = before + __popc(bal & ((1u << lane) - 1u));
      total = all;
      __syncthreads();
    }
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      if (keep[h]) {
        s_col[pos[h]] = j_c[h];
        s_xh[pos[h]] = x_c[h].x;
        s_xl[pos[h]] = PREC == kX2 ? x_c[h].y : 0.0f;
      }
    }
    __syncthreads();
    if (!FOLD && blockIdx.x == 0 && threadIdx.x == 0) atomicAdd(&st->sum_nnz, (double)total);
    if (live) {
      int q = warp;
#pragma unroll 2
      for (; q + kFwdWarps < total; q += 2 * kFwdWarps) {
        const float4 a0 = __ldg(reinterpret_cast<const float4*>(p.A + (size_t)s_col[q] * p.lda + row));
        const float4 a1 = __ldg(reinterpret_cast<const float4*>(p.A + (size_t)s_col[q + kFwdWarps] * p.lda + row));
        acc4<PREC>(s0, c0, a0, s_xh[q], s_xl[q]);
        acc4<PREC>(s1, c1, a1, s_xh[q + kFwdWarps], s_xl[q + kFwdWarps]);
      }
      if (q < total) {
        const float4 a0 = __ldg(reinterpret_cast<const float4*>(p.A + (size_t)s_col[q] * p.lda + row));
        acc4<PREC>(s0, c0, a0, s_xh[q], s_xl[q]);
      }
    }
  }

  // merge the two sets, then the warps (warp 0 collects), then write the chunk partial
#pragma unroll
  for (int i = 0; i < 4; ++i) merge<PREC>(s0[i], c0[i], s1[i], c1[i]);
  __syncthreads();
  if (warp > 0) {
#pragma unroll
    for (int i = 0; i < 4; ++i) s_red[warp - 1][4 * lane + i] = make_float2(s0[i], c0[i]);
  }
  __syncthreads();
  if (warp == 0) {
    for (int w = 0; w < kFwdWarps - 1; ++w) {
#pragma unroll
      for (int i = 0; i < 4; ++i) {
        const float2 v = s_red[w][4 * lane + i];
        merge<PREC>(s0[i], c0[i], v.x, v.y);
      }
    }
    if (live) {
#pragma unroll
      for (int i = 0; i < 4; ++i)
        b.part[(size_t)blockIdx.y * p.lda + row + i] = make_float2(s0[i], PREC == kX2 ? c0[i] : 0.f);
    }
  }

  if (!last_block(&b.tile_cnt[blockIdx.x], nch)) return;

  // Last block of this row tile: reduce the chunk partials, r = y' - q (or fold into y').
  double pv[1] = {0.0};
  const int r_ = blockIdx.x * kFwdRows + threadIdx.x;
  if (r_ < p.m) {
    float s = 0.f, c = 0.f;
    for (int ch = 0; ch < nch; ++ch) {
      const float2 v = __ldcg(&b.part[(size_t)ch * p.lda + r_]);
      df_add(s, c, v.x, v.y);
    }
    const float yh = b.yh[r_], yl = b.yl[r_];
    float dh, de;
    two_sum(yh, -s, dh, de);
    de += yl - c;
    float rh, rl;
    two_sum(dh, de, rh, rl);
    if (FOLD) {
      b.yh[r_] = rh;
      b.yl[r_] = rl;
    } else {
      b.rh[r_] = rh;
      b.rl[r_] = rl;
      const double rv = (double)rh + (double)rl;
      pv[0] = 0.5 * rv * rv;
    }
  }
  if (FOLD) return;
  __shared__ double sh[32];
  block_sum<1>(pv, sh);
  if (threadIdx.x == 0) b.tileP[blockIdx.x] = pv[0];
  if (!last_block(&st->cnt_fwd, gridDim.x)) return;
  if (threadIdx.x < 32) {
    const double a = warp_load_sum(b.tileP, gridDim.x);
    if (threadIdx.x == 0) st->P[slot] = a;
  }
}

cudaError_t launch_fwd(const Params& p, const Buffers& b, int slot, int precision, bool fold,
                       cudaStream_t s) {
  dim3 grid(p.fwd_tiles, p.fwd_chunks);
  if (precision != kF32) {   // kX2 and kMix: double-float forward product
    if (fold) k_fwd<kX2, true><<<grid, kFwdThreads, 0, s>>>(p, b, slot);
    else k_fwd<kX2, false><<<grid, kFwdThreads, 0, s>>>(p, b, slot);
  } else {
    if (fold) k_fwd<kF32, true><<<grid, kFwdThreads, 0, s>>>(p, b, slot);
    else k_fwd<kF32, false><<<grid, kFwdThreads, 0, s>>>(p, b, slot);
  }
  return cudaGetLastError();
}

// ------------------------------------------------------------------ g = A_S^T r + step
size_t tr_smem_bytes(int m4) { return (size_t)m4 * 2 * sizeof(float); }

template <int PREC>
__global__ void __launch_bounds__(kTrThreads, 1) k_tr(Params p, Buffers b, int slot, int gap_iter) {
  DevState* st = b.st;
  if (st->done) return;
  extern __shared__ float4 sm4[];
  const int m4q = p.m4 >> 2;
  float4* srh = sm4;
  float4* srl = sm4 + m4q;
  for (int i = threadIdx.x; i < m4q; i += kTrThreads) {
    srh[i] = __ldcg(reinterpret_cast<const float4*>(b.rh) + i);
    srl[i] = __ldcg(reinterpret_cast<const float4*>(b.rl) + i);
  }
  __syncthreads();

  const int n_act = st->n_active;
  __shared__ double s_scal[3];   // float64 is slow here: scalars once per block
  if (threadIdx.x == 0) {
    const double tk = st->t;
    const double tn0 = 0.5 * (1.0 + sqrt(1.0 + 4.0 * tk * tk));
    s_scal[0] = (tk - 1.0) / tn0;
    s_scal[1] = tn0;
    s_scal[2] = p.Cg * sqrt(2.0 * st->P[slot]) * (1.0 + 1e-6);
  }
  __syncthreads();
  const double tn = s_scal[1];
  const double eta_g = s_scal[2];
  const float2 bb = df2_from_double(s_scal[0]);
  const float2 onepb = df2_from_double(1.0 + s_scal[0]);
  const bool want_eps = gap_iter && p.dual_mode == kTranslation;
  const float2* __restrict__ xc = b.x[slot];
  float2* xn = b.x[slot ^ 1];
  const float2* __restrict__ gp = b.g[slot ^ 1];
  float2* gc = b.g[slot];

  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int gw = blockIdx.x * kTrWarps + warp;
  const int nw = gridDim.x * kTrWarps;
  float2 dot = make_float2(0.f, 0.f);
  double epsm = 0.0;

  for (int pp = 2 * gw; pp < n_act; pp += 2 * nw) {
    const int j0 = b.idx[pp];
    const int j1 = (pp + 1 < n_act) ? b.idx[pp + 1] : -1;
    const float4* c0p = reinterpret_cast<const float4*>(p.A + (size_t)j0 * p.lda);
    const float4* c1p = reinterpret_cast<const float4*>(p.A + (size_t)(j1 < 0 ? j0 : j1) * p.lda);
    float sA[4] = {0.f, 0.f, 0.f, 0.f}, cA[4] = {0.f, 0.f, 0.f, 0.f};
    float sB[4] = {0.f, 0.f, 0.f, 0.f}, cB[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll 4
    for (int i = lane; i < m4q; i += 32) {
      const float4 h = srh[i];
      const float4 l = srl[i];
      const float4 a0 = __ldg(c0p + i);
      const float4 a1 = __ldg(c1p + i);
      acc4v<PREC>(sA, cA, a0, h, l);
      acc4v<PREC>(sB, cB, a1, h, l);
    }
    merge<PREC>(sA[0], cA[0], sA[1], cA[1]);
    merge<PREC>(sA[2], cA[2], sA[3], cA[3]);
    merge<PREC>(sA[0], cA[0], sA[2], cA[2]);
    merge<PREC>(sB[0], cB[0], sB[1], cB[1]);
    merge<PREC>(sB[2], cB[2], sB[3], cB[3]);
    merge<PREC>(sB[0], cB[0], sB[2], cB[2]);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      const float a_s = __shfl_xor_sync(0xffffffffu, sA[0], o);
      const float a_c = __shfl_xor_sync(0xffffffffu, cA[0], o);
      const float b_s = __shfl_xor_sync(0xffffffffu, sB[0], o);
      const float b_c = __shfl_xor_sync(0xffffffffu, cB[0], o);
      merge<PREC>(sA[0], cA[0], a_s, a_c);
      merge<PREC>(sB[0], cB[0], b_s, b_c);
    }
    if (lane < 2) {
      const int j = lane == 0 ? j0 : j1;
      if (j >= 0) {
        const float2 g = lane == 0 ? df2_norm(sA[0], PREC == kX2 ? cA[0] : 0.f)
                                   : df2_norm(sB[0], PREC == kX2 ? cB[0] : 0.f);
        const float2 xk = xc[j];
        const float2 xp = xn[j];
        const float2 gv = df2_sub(df2_mul(onepb, g), df2_mul(bb, gp[j]));   // a_j^T (y' - A v_k)
        const float2 v = df2_add(xk, df2_mul(bb, df2_sub(xk, xp)));
        float2 xnew = df2_add(v, df2_mul(gv, p.invL2));
        if (df2_lt(xnew, p.l2[j])) xnew = p.l2[j];
        if (df2_lt(p.u2[j], xnew)) xnew = p.u2[j];
        xn[j] = xnew;
        gc[j] = g;
        dot = df2_add(dot, df2_mul(gv, df2_sub(xnew, xk)));
        if (want_eps && p.jinf[j]) {
          const double nr = p.nrm[j];
          if (nr > 0.0) {
            const double den = -p.w[j] - p.gamma_w * nr * p.t_norm;
            epsm = fmax(epsm, fmax(df2_to_double(g) + eta_g * nr, 0.0) / den);
          }
        }
      }
    }
  }

  // block reduction of (dot, eps) and the grid-wide finish in the last block
  __shared__ float2 shd[32][2];
  __shared__ double she[32];
  {
    const float2 o = make_float2(__shfl_down_sync(0xffffffffu, dot.x, 1), __shfl_down_sync(0xffffffffu, dot.y, 1));
    if (lane == 0) dot = df2_add(dot, o);   // lanes 0 and 1 carry the values
  }
  epsm = warp_max_d(epsm);
  if (lane == 0) {
    shd[warp][0] = dot;
    she[warp] = epsm;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    float2 d = make_float2(0.f, 0.f);
    double e = 0.0;
    for (int w = 0; w < kTrWarps; ++w) {
      d = df2_add(d, shd[w][0]);
      e = fmax(e, she[w]);
    }
    b.blk[4 * blockIdx.x + 0] = df2_to_double(d);
    b.blk[4 * blockIdx.x + 1] = e;
  }
  if (!last_block(&st->cnt_tr, gridDim.x)) return;
  if (threadIdx.x < 32) {
    double d = 0.0, e = 0.0;
    for (int t0 = 0; t0 < (int)gridDim.x; t0 += 256) {
      double dv[8], ev[8];
#pragma unroll
      for (int k = 0; k < 8; ++k) {   // loads first: one L2 round trip per 256 blocks
        const int t = t0 + threadIdx.x + 32 * k;
        dv[k] = t < (int)gridDim.x ? __ldcg(&b.blk[4 * t + 0]) : 0.0;
        ev[k] = t < (int)gridDim.x ? __ldcg(&b.blk[4 * t + 1]) : 0.0;
      }
#pragma unroll
      for (int k = 0; k < 8; ++k) {
        d += dv[k];
        e = fmax(e, ev[k]);
      }
    }
    d = warp_sum_d(d);
    e = warp_max_d(e);
    if (threadIdx.x == 0) {
      st->t = (p.restart && d < 0.0) ? 1.0 : tn;
      st->eps = e;
      st->k += 1;
      st->sum_active += (double)n_act;
    }
  }
}

cudaError_t launch_tr(const Params& p, const Buffers& b, int slot, int precision, bool gap_iter,
                      int tr_blocks, cudaStream_t s) {
  const size_t sm = tr_smem_bytes(p.m4);
  if (precision == kX2) k_tr<kX2><<<tr_blocks, kTrThreads, sm, s>>>(p, b, slot, gap_iter ? 1 : 0);
  else k_tr<kF32><<<tr_blocks, kTrThreads, sm, s>>>(p, b, slot, gap_iter ? 1 : 0);
  return cudaGetLastError();
}

// ------------------------------------------------------------------ gap and radius
// Gap(x, theta) for theta = r + eps t (eps = 0 in the scaling mode), written as
//   sum_j [ (u_j - x_j)(gt_j)^+ + (x_j - l_j)(-gt_j)^+ ] + 1/2 ||theta - r_exact||^2,
// gt_j = a_j^T theta.  This equals P(x) - D(theta) of Eqs. (Dual_Gap), (Dual_obj) for the
// least-squares loss; every term is nonnegative, so no cancellation.  The bound adds the
// rounding of gt_j (eta ||a_j|| per column, times the Lipschitz constant of the term in
// gt_j) and of the residual (E_r).  theta = 0 (no interior direction): Gap = P(x).
__global__ void __launch_bounds__(kRedThreads) k_gap(Params p, Buffers b, int slot, int finalize) {
  DevState* st = b.st;
  if (st->done) return;
  const int n_act = st->n_active;
  const bool trans = p.dual_mode == kTranslation;
  const double eps = trans ? st->eps : 0.0;
  // FISTA: the pair (x_k, Theta(x_k)); primal-dual: (x_{k+1}, theta = -z_{k+1}), whose
  // correlations a_j^T z_{k+1} the pass stored with the opposite sign
  const bool cp = p.alg == kChambollePock;
  const float2* __restrict__ xc = b.x[cp ? slot ^ 1 : slot];
  const float2* __restrict__ gc = b.g[slot];
  const double gsign = cp ? -1.0 : 1.0;
  double v[3] = {0.0, 0.0, 0.0};  // sum h_j, sum c_j ||a_j||, sum |x_j| ||a_j||
  const int stride = gridDim.x * blockDim.x;
  for (int pp = blockIdx.x * blockDim.x + threadIdx.x; pp < n_act; pp += stride) {
    const int j = b.idx[pp];
    const double x = df2_to_double(xc[j]);
    const double nr = p.nrm[j];
    v[2] += fabs(x) * nr;
    if (p.dual_mode != kZero) {
      const double gt = p.wstar ? p.wstar[j] + (trans ? p.eps_star * p.w[j] : 0.0)
                                : gsign * df2_to_double(gc[j]) + (trans ? eps * p.w[j] : 0.0);
      const double lj = p.l[j];
      if (p.jinf[j]) {
        v[0] += (x - lj) * fmax(-gt, 0.0);
        v[1] += (x - lj) * nr;
      } else {
        const double uj = p.u[j];
        v[0] += (uj - x) * fmax(gt, 0.0) + (x - lj) * fmax(-gt, 0.0);
        v[1] += fmax(uj - x, x - lj) * nr;
      }
    }
  }
  __shared__ double sh[96];
  block_sum<3>(v, sh);
  if (threadIdx.x == 0) {
    b.blk[4 * blockIdx.x + 0] = v[0];
    b.blk[4 * blockIdx.x + 1] = v[1];
    b.blk[4 * blockIdx.x + 2] = v[2];
  }
  if (!last_block(&st->cnt_gap, gridDim.x)) return;
  if (threadIdx.x < 32) {
    double a = 0.0, c = 0.0, x = 0.0;
    for (int t0 = 0; t0 < (int)gridDim.x; t0 += 256) {
      double av[8], cv[8], xv[8];
#pragma unroll
      for (int k = 0; k < 8; ++k) {   // loads first: one L2 round trip per 256 blocks
        const int t = t0 + threadIdx.x + 32 * k;
        const bool ok = t < (int)gridDim.x;
        av[k] = ok ? __ldcg(&b.blk[4 * t + 0]) : 0.0;
        cv[k] = ok ? __ldcg(&b.blk[4 * t + 1]) : 0.0;
        xv[k] = ok ? __ldcg(&b.blk[4 * t + 2]) : 0.0;
      }
#pragma unroll
      for (int k = 0; k < 8; ++k) {
        a += av[k];
        c += cv[k];
        x += xv[k];
      }
    }
    a = warp_sum_d(a);
    c = warp_sum_d(c);
    x = warp_sum_d(x);
    double P_cp = 0.0, dist2 = 0.0, z2 = 0.0;
    if (cp) {  // the residual kernel's block partials of 1/2||r||^2, ||z + r||^2, ||z||^2
      const int nres = (p.m4 + 31) / 32;
      P_cp = warp_load_sum(b.tileR, nres);
      dist2 = warp_load_sum(b.tileD, nres);
      z2 = warp_load_sum(b.tileZ, nres);
    }
    if (threadIdx.x == 0) {
      const double rnorm = sqrt(2.0 * (cp ? P_cp : st->P[slot])) * (1.0 + 1e-6);
      // rounding of a_j^T theta per unit ||a_j||: the correlation is taken with r (FISTA) or z
      const double eta = p.wstar ? p.eta_star
                                 : p.Cg * (cp ? sqrt(z2) * (1.0 + 1e-6) : rnorm) + (trans ? eps * p.gamma_w * p.t_norm : 0.0);
      const double E_r = cp ? st->E_fold + p.E_cp + p.Csub * (st->y_norm + st->S_fold)
                            : st->E_fold + p.Cf * x + p.Csub * (rnorm + st->y_norm + st->S_fold + x);
      double gap;
      if (cp) {
        // theta = -z: 1/2 ||theta - r (exact)||^2 <= 1/2 (||z + r (stored)|| + E_r)^2
        const double d = sqrt(dist2) * (1.0 + 1e-12) + E_r;
        gap = a + eta * c + 0.5 * d * d;
        st->P[slot ^ 1] = P_cp;
      } else if (p.wstar) {
        // fixed dual point: 1/2 ||theta - r||^2 with the stored residual's own error
        const double d = sqrt(st->theta_r2) * (1.0 + 1e-12) + E_r;
        gap = a + eta * c + 0.5 * d * d;
      } else if (p.dual_mode == kZero) {
        gap = 0.5 * (rnorm + E_r) * (rnorm + E_r);
      } else {
        const double d = E_r + eps * p.t_norm;
        gap = a + eta * c + 0.5 * d * d;
      }
      gap *= (1.0 + 1e-12);
      st->gap = gap;
      st->radius = sqrt(2.0 * gap);
      st->eta = eta;
      st->gap_evals += 1;
      const bool conv = gap < p.tol;
      if (conv || st->k >= p.max_iter) {
        st->converged = conv ? 1 : 0;
        st->out_slot = cp ? slot ^ 1 : slot;
        if (finalize) st->done = 1;
        else st->stop = 1;
      }
    }
  }
}

cudaError_t launch_gap(const Params& p, const Buffers& b, int slot, bool finalize, int red_blocks,
                       cudaStream_t s) {
  k_gap<<<red_blocks, kRedThreads, 0, s>>>(p, b, slot, finalize ? 1 : 0);
  return cudaGetLastError();
}

// ------------------------------------------------------------------ sphere test
// Eq. (safe_rule) with exact-arithmetic safety: a column is fixed at l_j when the computed
// gt_j < -(radius + eta) ||a_j|| (both inflated by 1e-12 relative), at u_j (finite) when
// gt_j > (radius + eta) ||a_j||.  Zero columns are never fixed.
__global__ void __launch_bounds__(kRedThreads) k_test(Params p, Buffers b, int slot) {
  DevState* st = b.st;
  if (st->done) return;
  const int n_act = st->n_active;
  const bool trans = p.dual_mode == kTranslation;
  const double eps = trans ? st->eps : 0.0;
  const double rr = st->radius * (1.0 + 1e-12) + st->eta;
  const float2* __restrict__ xc = b.x[slot];
  const float2* __restrict__ xn = b.x[slot ^ 1];
  const float2* __restrict__ gc = b.g[slot];
  int cnt = 0;
  const int stride = gridDim.x * blockDim.x;
  for (int pp = blockIdx.x * blockDim.x + threadIdx.x; pp < n_act; pp += stride) {
    const int j = b.idx[pp];
    const double nr = p.nrm[j];
    if (!(nr > 0.0)) continue;
    const double gt = p.wstar ? p.wstar[j] + (trans ? p.eps_star * p.w[j] : 0.0)
                              : (p.alg == kChambollePock ? -1.0 : 1.0) * df2_to_double(gc[j]) +
                                    (trans ? eps * p.w[j] : 0.0);
    const double thr = rr * nr * (1.0 + 1e-12);
    int pin = 0;
    float2 bnd = make_float2(0.f, 0.f);
    if (gt < -thr) {
      pin = 1;
      bnd = p.l2[j];
    } else if (!p.jinf[j] && gt > thr) {
      pin = 2;
      bnd = p.u2[j];
    }
    // Fixed once x_k and x_{k+1} both sit at that bound: the stored g_k then stays the
    // gradient of the reduced problem and the momentum needs no correction.
    if (pin && df2_eq(xc[j], bnd) && df2_eq(xn[j], bnd)) {
      b.flags[j] = (uint8_t)pin;
      ++cnt;
    }
  }
  for (int o = 16; o > 0; o >>= 1) cnt += __shfl_xor_sync(0xffffffffu, cnt, o);
  if ((threadIdx.x & 31) == 0 && cnt) atomicAdd(&st->n_pins, cnt);
}

cudaError_t launch_test(const Params& p, const Buffers& b, int slot, int red_blocks, cudaStream_t s) {
  k_test<<<red_blocks, kRedThreads, 0, s>>>(p, b, slot);
  return cudaGetLastError();
}

// ------------------------------------------------------------------ compaction
// One block.  Stable: the preserved list keeps its order, so the summation order of the
// products (and hence every rounding) is reproducible run to run.
__device__ __forceinline__ int block_excl_scan(int v, int* sh, int& total) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  int x = v;
  for (int o = 1; o < 32; o <<= 1) {
    const int y = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= o) x += y;
  }
  if (lane == 31) sh[warp] = x;
  __syncthreads();
  if (warp == 0) {
    int w = lane < nw ? sh[lane] : 0;
    for (int o = 1; o < 32; o <<= 1) {
      const int y = __shfl_up_sync(0xffffffffu, w, o);
      if (lane >= o) w += y;
    }
    sh[32 + lane] = w;
  }
  __syncthreads();
  const int warp_off = warp > 0 ? sh[32 + warp - 1] : 0;
  total = sh[32 + nw - 1];
  __syncthreads();
  return warp_off + x - v;
}

__global__ void __launch_bounds__(kCompactThreads) k_compact(Params p, Buffers b, int slot) {
  DevState* st = b.st;
  if (st->done) return;
  __shared__ int sh[64];
  __shared__ double shd[32];
  const int npins = st->n_pins;
  const int stop = st->stop;
  __syncthreads();
  if (npins == 0) {
    if (threadIdx.x == 0) {
      st->n_fold = 0;
      if (stop) st->done = 1;
    }
    return;
  }
  const int n_act = st->n_active;
  const float2* xc = b.x[slot];
  const int per = (n_act + kCompactThreads - 1) / kCompactThreads;
  const int q0 = min(n_act, threadIdx.x * per), q1 = min(n_act, q0 + per);
  int keep = 0, fold = 0;
  for (int q = q0; q < q1; ++q) {
    const int j = b.idx[q];
    if (!b.flags[j]) ++keep;
    else if (df2_nonzero(xc[j])) ++fold;
  }
  int nkeep, nfold;
  int ok = block_excl_scan(keep, sh, nkeep);
  int of = block_excl_scan(fold, sh, nfold);
  double sabs = 0.0;
  for (int q = q0; q < q1; ++q) {
    const int j = b.idx[q];
    if (!b.flags[j]) {
      b.idx_tmp[ok++] = j;
    } else if (df2_nonzero(xc[j])) {
      b.fold[of++] = j;
      sabs += fabs(df2_to_double(xc[j])) * p.nrm[j];
    }
  }
  sabs = warp_sum_d(sabs);
  if ((threadIdx.x & 31) == 0) shd[threadIdx.x >> 5] = sabs;
  __syncthreads();
  for (int q = threadIdx.x; q < nkeep; q += kCompactThreads) b.idx[q] = b.idx_tmp[q];
  if (threadIdx.x == 0) {
    double s = 0.0;
    for (int w = 0; w < kCompactThreads / 32; ++w) s += shd[w];
    st->n_active = nkeep;
    st->n_fold = nfold;
    st->S_fold += s;
    st->E_fold += p.Cf * s + p.Csub * (st->y_norm + st->S_fold);
    st->n_pins = 0;
    if (stop) st->done = 1;
  }
}

cudaError_t launch_compact(const Params& p, const Buffers& b, int slot, cudaStream_t s) {
  k_compact<<<1, kCompactThreads, 0, s>>>(p, b, slot);
  return cudaGetLastError();
}

}  // namespace bvls

namespace bvls {

// Opt the A_S^T r kernels into the dynamic shared memory a given m needs and return how
// many blocks of it fit on one SM.
cudaError_t tr_configure(int m4, int* blocks_per_sm) {
  const size_t sm = tr_smem_bytes(m4);
  cudaError_t e = cudaFuncSetAttribute(k_tr<kX2>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
  if (e != cudaSuccess) return e;
  e = cudaFuncSetAttribute(k_tr<kF32>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
  if (e != cudaSuccess) return e;
  int a = 0, b = 0;
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&a, k_tr<kX2>, kTrThreads, sm);
  if (e != cudaSuccess) return e;
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, k_tr<kF32>, kTrThreads, sm);
  if (e != cudaSuccess) return e;
  *blocks_per_sm = a < b ? a : b;
  return cudaSuccess;
}

}  // namespace bvls
