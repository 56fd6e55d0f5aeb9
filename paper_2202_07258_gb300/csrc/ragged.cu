// Ragged batch kernels: B problems with their own A_k, y_k and boxes (see ragged.cuh).
#include "common.cuh"
#include "ragged.cuh"

#include <algorithm>

namespace bvls {

namespace {

constexpr unsigned kFull = 0xffffffffu;

__device__ __forceinline__ double wsum(double v) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(kFull, v, o);
  return v;
}
__device__ __forceinline__ double wmax(double v) {
  for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(kFull, v, o));
  return v;
}

// block of kRThreads: sum (or max) over the block, result in every thread
__device__ double bsum(double v, double* sh) {
  v = wsum(v);
  __syncthreads();
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = v;
  __syncthreads();
  double t = 0.0;
  for (int w = 0; w < kRThreads / 32; ++w) t += sh[w];
  __syncthreads();
  return t;
}
__device__ double bmax(double v, double* sh) {
  v = wmax(v);
  __syncthreads();
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = v;
  __syncthreads();
  double t = 0.0;
  for (int w = 0; w < kRThreads / 32; ++w) t = fmax(t, sh[w]);
  __syncthreads();
  return t;
}

// exclusive block scan of 0/1 flags (kRThreads threads); total in *tot
__device__ int bscan(int v, int* sh, int* tot) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  int x = v;
  for (int o = 1; o < 32; o <<= 1) {
    const int y = __shfl_up_sync(kFull, x, o);
    if (lane >= o) x += y;
  }
  __syncthreads();
  if (lane == 31) sh[warp] = x;
  __syncthreads();
  int before = 0, total = 0;
  for (int w = 0; w < kRThreads / 32; ++w) {
    if (w < warp) before += sh[w];
    total += sh[w];
  }
  *tot = total;
  __syncthreads();
  return before + x - v;
}

}  // namespace

// ---------------------------------------------------------------- setup
// ||a_j|| and w_j = a_j^T t with t = -1, float64, one warp per column.
__global__ void k_rnorms(RBuf b, long long total_cols) {
  const int lane = threadIdx.x & 31;
  const long long wid = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const long long nw = ((long long)gridDim.x * blockDim.x) >> 5;
  for (long long c = wid; c < total_cols; c += nw) {
    // the instance of column c: binary search over c_off
    int lo = 0, hi = b.B - 1;
    while (lo < hi) {
      const int mid = (lo + hi + 1) >> 1;
      if (b.inst[mid].c_off <= c) lo = mid;
      else hi = mid - 1;
    }
    const RInst in = b.inst[lo];
    const int j = (int)(c - in.c_off);
    const float* col = b.A + in.a_off + (long long)j * in.lda;
    double s2 = 0.0, s1 = 0.0;
    for (int i = lane; i < in.m; i += 32) {
      const double a = col[i];
      s2 = fma(a, a, s2);
      s1 += a;
    }
    s2 = wsum(s2);
    s1 = wsum(s1);
    if (lane == 0) {
      b.nrm[c] = sqrt(s2);
      b.w[c] = -s1;
      if (!isfinite(s2) || !isfinite(s1)) atomicOr(b.err, 1u);
    }
  }
}

cudaError_t launch_rnorms(const RBuf& b, long long total_cols, cudaStream_t s) {
  const long long blocks = std::min<long long>((total_cols * 32 + 255) / 256, 65535 * 4);
  k_rnorms<<<(int)std::max<long long>(blocks, 1), 256, 0, s>>>(b, total_cols);
  return cudaGetLastError();
}

// Iterates, flags and the preserved lists; per-instance state.  Power mode starts from the
// unit vector 1/sqrt(n_k).
__global__ void k_rinit(RBuf b, long long total_cols, int power) {
  for (long long c = (long long)blockIdx.x * blockDim.x + threadIdx.x; c < total_cols;
       c += (long long)gridDim.x * blockDim.x) {
    int lo = 0, hi = b.B - 1;
    while (lo < hi) {
      const int mid = (lo + hi + 1) >> 1;
      if (b.inst[mid].c_off <= c) lo = mid;
      else hi = mid - 1;
    }
    const RInst& in = b.inst[lo];
    const int j = (int)(c - in.c_off);
    float2 x;
    if (power) {
      x = df2_from_double(1.0 / sqrt((double)in.n));
    } else {
      x = make_float2(0.f, 0.f);
      if (df2_lt(x, b.l2[c])) x = b.l2[c];
      if (df2_lt(b.u2[c], x)) x = b.u2[c];
    }
    b.x[0][c] = x;
    b.x[1][c] = x;
    b.g[0][c] = make_float2(0.f, 0.f);
    b.g[1][c] = make_float2(0.f, 0.f);
    b.flags[c] = 0;
    b.idx[c] = j;
  }
  for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < b.B; k += gridDim.x * blockDim.x) {
    RState& st = b.st[k];
    st.k = 0;
    st.done = 0;
    st.converged = 0;
    st.n_active = b.inst[k].n;
    st.n_pins = 0;
    st.out_slot = 0;
    st.gap_evals = 0;
    st.t = 1.0;
    st.eps = 0.0;
    st.gap = INFINITY;
    st.radius = INFINITY;
    st.eta = 0.0;
    st.E_fold = 0.0;
    st.S_fold = 0.0;
    st.dot = 0.0;
    if (power) {
      st.pw_scale = 1.0;
      st.pw_lambda = 0.0;
    }
  }
}

cudaError_t launch_rinit(const RBuf& b, long long total_cols, int power, cudaStream_t s) {
  const long long blocks = std::min<long long>((total_cols + 255) / 256, 65535 * 4);
  k_rinit<<<(int)std::max<long long>(blocks, 1), 256, 0, s>>>(b, total_cols, power);
  return cudaGetLastError();
}

// Work list over the active instances: ceil(n_active / tw) tiles each.  One block.
__global__ void __launch_bounds__(kRThreads) k_rtiles(RBuf b) {
  __shared__ int sh[kRThreads / 32];
  __shared__ double shd[kRThreads / 32];
  __shared__ int s_base, s_ibase;
  if (threadIdx.x == 0) {
    s_base = 0;
    s_ibase = 0;
  }
  __syncthreads();
  double work = 0.0;   // sum over the live instances of m_k |S_k|: A elements one iteration reads
  for (int k0 = 0; k0 < b.B; k0 += kRThreads) {
    const int k = k0 + threadIdx.x;
    const bool live = k < b.B && !b.st[k].done;
    const int nt = live ? (b.st[k].n_active + b.tw - 1) / b.tw : 0;
    if (live) work += (double)b.inst[k].m * (double)b.st[k].n_active;
    int tot = 0;
    // tiles: exclusive scan of nt (counts up to kRThreads * tiles_max fit an int)
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    int x = nt;
    for (int o = 1; o < 32; o <<= 1) {
      const int y = __shfl_up_sync(kFull, x, o);
      if (lane >= o) x += y;
    }
    if (lane == 31) sh[warp] = x;
    __syncthreads();
    int before = 0;
    for (int w = 0; w < kRThreads / 32; ++w) {
      if (w < warp) before += sh[w];
      tot += sh[w];
    }
    const int base = s_base + before + x - nt;
    for (int t = 0; t < nt; ++t) b.tiles[base + t] = RTileRef{k, t};
    __syncthreads();
    int itot = 0;
    const int ipos = bscan(live ? 1 : 0, sh, &itot);
    if (live) b.act[s_ibase + ipos] = k;
    __syncthreads();
    if (threadIdx.x == 0) {
      s_base += tot;
      s_ibase += itot;
    }
    __syncthreads();
  }
  work = bsum(work, shd);
  if (threadIdx.x == 0) {
    *b.n_tiles = s_base;
    *b.n_act_inst = s_ibase;
    // the work list stays until the next gap iteration: the next K iterations read this much
    if (b.work && !b.power) *b.work += work * (double)b.K;
  }
}

cudaError_t launch_rtiles(const RBuf& b, cudaStream_t s) {
  k_rtiles<<<1, kRThreads, 0, s>>>(b);
  return cudaGetLastError();
}

// r_0 = y' - A x_0 (or A v_0 in power mode) per instance, and P_0.  Block per instance.
__global__ void __launch_bounds__(kRThreads) k_rfwd(RBuf b) {
  __shared__ double sh[kRThreads / 32];
  const int k = blockIdx.x;
  const RInst in = b.inst[k];
  RState& st = b.st[k];
  double p2 = 0.0, y2 = 0.0;
  for (int i = threadIdx.x; i < in.m; i += kRThreads) {
    float s = 0.f, c = 0.f;
    for (int j = 0; j < in.n; ++j) {
      const float2 x = b.x[0][in.c_off + j];
      if (x.x != 0.f || x.y != 0.f) df_fma(s, c, b.A[in.a_off + (long long)j * in.lda + i], x.x, x.y);
    }
    float rh, rl;
    if (b.power) {
      two_sum(s, c, rh, rl);
    } else {
      float dh, de;
      two_sum(b.yh[in.r_off + i], -s, dh, de);
      de += b.yl[in.r_off + i] - c;
      two_sum(dh, de, rh, rl);
      const double y = (double)b.yh[in.r_off + i] + (double)b.yl[in.r_off + i];
      if (!isfinite(y)) atomicOr(b.err, 1u);
      y2 += y * y;
    }
    b.rh[in.r_off + i] = rh;
    b.rl[in.r_off + i] = rl;
    const double r = (double)rh + (double)rl;
    p2 += 0.5 * r * r;
  }
  p2 = bsum(p2, sh);
  y2 = bsum(y2, sh);
  if (threadIdx.x == 0) {
    st.P = p2;
    if (b.power) st.pw_scale = fmax(2.0 * p2, 1e-300);
    else st.y_norm = sqrt(y2);
  }
}

cudaError_t launch_rfwd(const RBuf& b, cudaStream_t s) {
  k_rfwd<<<b.B, kRThreads, 0, s>>>(b);
  return cudaGetLastError();
}

// ---------------------------------------------------------------- one iteration
// Tile = (instance k, tile t): preserved columns q in [t tw, min((t+1) tw, n_active)).
size_t rpass_smem_bytes(int tw) {
  return (size_t)kRMaxRows * 2 * sizeof(float) + (size_t)tw * kRMaxRows * sizeof(float);
}

// The grid walks the work list (a CTA takes tiles blockIdx.x, blockIdx.x + gridDim.x, ...), so
// a launch over few live tiles costs a few CTAs per SM, not one CTA per possible tile.
__global__ void __launch_bounds__(kRThreads) k_rpass(RBuf b, int slot, int gap_iter) {
  const int ntiles = *b.n_tiles;
  extern __shared__ __align__(16) float rsm[];
  float* srh = rsm;                      // r (hi), m4 floats
  float* srl = rsm + kRMaxRows;          // r (lo)
  float* sa = rsm + 2 * kRMaxRows;       // tile columns: [c][m4]
  __shared__ int s_col[kRTileMax];
  __shared__ float2 s_xn[kRTileMax];
  __shared__ double s_dot[kRTileMax], s_eps[kRTileMax], s_v2[kRTileMax];
  __shared__ float2 s_bb, s_onepb, s_invL2;
  __shared__ double s_etag;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  for (int wt = blockIdx.x; wt < ntiles; wt += gridDim.x) {
  const RTileRef tr = b.tiles[wt];
  const int k = tr.inst;
  const RInst in = b.inst[k];
  const RState& st = b.st[k];
  const int m4 = (in.m + 3) & ~3;
  const int q0 = tr.tile * b.tw;
  const int nc = min(b.tw, st.n_active - q0);
  if (tid < kRTileMax) {
    s_col[tid] = tid < nc ? b.idx[in.c_off + q0 + tid] : -1;
    s_dot[tid] = 0.0;
    s_eps[tid] = 0.0;
    s_v2[tid] = 0.0;
  }
  if (tid == 0) {
    // FISTA parameters of the instance (t_k stored), once per tile: float64 runs at a small
    // fraction of the float32 rate on this part, so one thread computes them while the
    // others stage the tile
    const double tk = st.t;
    const double tn = 0.5 * (1.0 + sqrt(1.0 + 4.0 * tk * tk));
    const double beta = (tk - 1.0) / tn;
    s_bb = df2_from_double(beta);
    s_onepb = df2_from_double(1.0 + beta);
    s_invL2 = df2_from_double(in.invL);
    s_etag = in.Cg * sqrt(2.0 * st.P) * (1.0 + 1e-6);
  }
  for (int i = tid; i < m4; i += kRThreads) {
    srh[i] = i < in.m ? b.rh[in.r_off + i] : 0.f;
    srl[i] = i < in.m ? b.rl[in.r_off + i] : 0.f;
  }
  __syncthreads();
  // stage the tile's columns (float4 when lda is a multiple of 4, which setup guarantees)
  const int m4q = m4 >> 2;
  for (int e = tid; e < nc * m4q; e += kRThreads) {
    const int c = e / m4q, i4 = e - c * m4q;
    const float4 v = *reinterpret_cast<const float4*>(b.A + in.a_off + (long long)s_col[c] * in.lda + 4 * i4);
    reinterpret_cast<float4*>(sa + (size_t)c * m4)[i4] = v;
  }
  __syncthreads();

  // FISTA parameters of the instance (from thread 0), or the power iteration's scale
  const float2 bb = s_bb, onepb = s_onepb;
  const float2 invL2 = s_invL2;
  const double eta_g = s_etag;
  const bool want_eps = gap_iter && in.dual_mode == kTranslation && !b.power;
  const float2* __restrict__ xc = b.x[slot];
  float2* xn = b.x[slot ^ 1];
  const float2* __restrict__ gp = b.g[slot ^ 1];
  float2* gc = b.g[slot];

  // dots: warp w takes columns w, w + 8 (lanes over float4 rows)
  for (int c = warp; c < nc; c += kRThreads / 32) {
    const float4* col = reinterpret_cast<const float4*>(sa + (size_t)c * m4);
    const float4* rh4 = reinterpret_cast<const float4*>(srh);
    const float4* rl4 = reinterpret_cast<const float4*>(srl);
    float s[4] = {0.f, 0.f, 0.f, 0.f}, e[4] = {0.f, 0.f, 0.f, 0.f};
    for (int i = lane; i < m4q; i += 32) {
      const float4 a = col[i], h = rh4[i], l = rl4[i];
      df_fma(s[0], e[0], a.x, h.x, l.x);
      df_fma(s[1], e[1], a.y, h.y, l.y);
      df_fma(s[2], e[2], a.z, h.z, l.z);
      df_fma(s[3], e[3], a.w, h.w, l.w);
    }
    df_add(s[0], e[0], s[1], e[1]);
    df_add(s[2], e[2], s[3], e[3]);
    df_add(s[0], e[0], s[2], e[2]);
    for (int o = 16; o > 0; o >>= 1) {
      const float os = __shfl_xor_sync(kFull, s[0], o);
      const float oe = __shfl_xor_sync(kFull, e[0], o);
      df_add(s[0], e[0], os, oe);
    }
    if (lane == 0) {
      const long long gcol = in.c_off + s_col[c];
      const float2 g2 = df2_norm(s[0], e[0]);
      const float2 xk = xc[gcol];
      float2 xnew;
      if (b.power) {
        // v_{i+1} = A^T A v_i / ||A v_i||^2 keeps the iterate's norm bounded
        xnew = df2_mul(g2, df2_from_double(1.0 / st.pw_scale));
        s_v2[c] = df2_to_double(xnew) * df2_to_double(xnew);
      } else {
        const float2 gv = df2_sub(df2_mul(onepb, g2), df2_mul(bb, gp[gcol]));
        const float2 v = df2_add(xk, df2_mul(bb, df2_sub(xk, xn[gcol])));
        xnew = df2_add(v, df2_mul(gv, invL2));
        if (df2_lt(xnew, b.l2[gcol])) xnew = b.l2[gcol];
        if (df2_lt(b.u2[gcol], xnew)) xnew = b.u2[gcol];
        s_dot[c] = df2_to_double(gv) * df2_to_double(df2_sub(xnew, xk));
        if (want_eps && b.jinf[gcol]) {
          const double nr = b.nrm[gcol];
          if (nr > 0.0) {
            const double den = -b.w[gcol] - in.gamma_w * nr * in.t_norm;
            s_eps[c] = fmax(df2_to_double(g2) + eta_g * nr, 0.0) / den;
          }
        }
      }
      s_xn[c] = xnew;
      xn[gcol] = xnew;
      gc[gcol] = g2;
    }
  }
  __syncthreads();
  // the tile's partial of A x_{k+1} (double-float, per row)
  float2* part = b.part + in.p_off + (long long)tr.tile * in.m;
  for (int i = tid; i < in.m; i += kRThreads) {
    float s = 0.f, e = 0.f;
    for (int c = 0; c < nc; ++c) {
      const float2 x = s_xn[c];
      if (x.x != 0.f || x.y != 0.f) df_fma(s, e, sa[(size_t)c * m4 + i], x.x, x.y);
    }
    part[i] = make_float2(s, e);
  }
  if (tid == 0) {
    double d = 0.0, ep = 0.0, v2 = 0.0;
    for (int c = 0; c < nc; ++c) {
      d += s_dot[c];
      ep = fmax(ep, s_eps[c]);
      v2 += s_v2[c];
    }
    const long long ti = in.t_off + tr.tile;
    b.tdot[ti] = b.power ? v2 : d;
    b.teps[ti] = ep;
  }
  __syncthreads();   // the next tile reuses the shared staging
  }
}

cudaError_t ragged_configure() {
  return cudaFuncSetAttribute(k_rpass, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              (int)rpass_smem_bytes(kRTileMax));
}

cudaError_t launch_rpass(const RBuf& b, int max_tiles, int slot, int gap_iter, cudaStream_t s) {
  if (b.tw < kRTileMin || b.tw > kRTileMax) return cudaErrorInvalidValue;
  // resident CTAs per SM for this tile width on the current device (the work list is walked
  // by a grid of that many CTAs per SM); the occupancy query is cheap next to the solve
  int dev = 0, sms = 0, per_sm = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (e == cudaSuccess)
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_rpass, kRThreads, rpass_smem_bytes(b.tw));
  if (e != cudaSuccess) return e;
  const int grid = std::max(1, std::min(max_tiles, std::max(1, per_sm) * sms));
  k_rpass<<<grid, kRThreads, rpass_smem_bytes(b.tw), s>>>(b, slot, gap_iter);
  return cudaGetLastError();
}

// Per instance: r_{k+1} = y' - sum of the tile partials (power mode: A v_{i+1}), P_{k+1}, and
// the scalars of the iteration.  Grid (row block, instance): a block takes 32 rows, a lane
// one row, and its 8 warps split the tiles (each sums every 8th tile, loads batched), then
// the warps' sums are merged in warp order.  The instance's last block to finish (a counter
// per instance) adds the blocks' P partials in block order and the tiles' restart terms,
// and updates the instance's scalars.
__global__ void __launch_bounds__(kRThreads) k_rresid(RBuf b, int slot) {
  __shared__ double sh[kRThreads / 32];
  __shared__ float2 s_part[kRThreads / 32][32];
  __shared__ int s_last;
  const int k = blockIdx.y;
  RState& st = b.st[k];
  if (st.done) return;
  const RInst in = b.inst[k];
  const int rb = blockIdx.x;
  const int nrb = (in.m + 31) / 32;
  if (rb >= nrb) return;
  const int nt = (st.n_active + b.tw - 1) / b.tw;
  const float2* part = b.part + in.p_off;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int i = rb * 32 + lane;
  float s = 0.f, c = 0.f;
  if (i < in.m) {
    int t = warp;
    for (; t + 3 * (kRThreads / 32) < nt; t += 4 * (kRThreads / 32)) {
      float2 v[4];
#pragma unroll
      for (int q = 0; q < 4; ++q) v[q] = __ldcg(part + (long long)(t + q * (kRThreads / 32)) * in.m + i);
#pragma unroll
      for (int q = 0; q < 4; ++q) df_add(s, c, v[q].x, v[q].y);
    }
    for (; t < nt; t += kRThreads / 32) {
      const float2 v = __ldcg(part + (long long)t * in.m + i);
      df_add(s, c, v.x, v.y);
    }
  }
  s_part[warp][lane] = make_float2(s, c);
  __syncthreads();
  if (warp == 0) {
    for (int w = 1; w < kRThreads / 32; ++w) df_add(s, c, s_part[w][lane].x, s_part[w][lane].y);
    double p2 = 0.0;
    if (i < in.m) {
      float rh, rl;
      if (b.power) {
        two_sum(s, c, rh, rl);
      } else {
        float dh, de;
        two_sum(b.yh[in.r_off + i], -s, dh, de);
        de += b.yl[in.r_off + i] - c;
        two_sum(dh, de, rh, rl);
      }
      b.rh[in.r_off + i] = rh;
      b.rl[in.r_off + i] = rl;
      const double r = (double)rh + (double)rl;
      p2 = 0.5 * r * r;
    }
    p2 = wsum(p2);
    if (lane == 0) {
      b.rblkP[(long long)k * kRRowBlocks + rb] = p2;
      __threadfence();
      const unsigned prev = atomicAdd(&b.rcnt[k], 1u);
      s_last = prev == (unsigned)nrb - 1u;
    }
  }
  __syncthreads();
  if (!s_last) return;
  __threadfence();
  // the instance's last block: P in block order, the restart terms and translation steps
  double p2 = 0.0;
  for (int q = threadIdx.x; q < nrb; q += kRThreads) p2 += __ldcg(b.rblkP + (long long)k * kRRowBlocks + q);
  p2 = bsum(p2, sh);
  const long long t0 = in.t_off;
  double d = 0.0, ep = 0.0;
  for (int t = threadIdx.x; t < nt; t += kRThreads) {
    d += b.tdot[t0 + t];
    ep = fmax(ep, b.teps[t0 + t]);
  }
  d = bsum(d, sh);
  ep = bmax(ep, sh);
  if (threadIdx.x == 0) {
    b.rcnt[k] = 0u;
    st.eps = ep;
    st.dot = d;
    if (b.power) {
      // lambda ~ ||A v||^2 / ||v||^2 for v = v_{i+1}
      st.pw_lambda = d > 0.0 ? 2.0 * p2 / d : 0.0;
      st.pw_scale = fmax(2.0 * p2, 1e-300);
      st.P = p2;
    } else {
      const double tk = st.t;
      const double tn = 0.5 * (1.0 + sqrt(1.0 + 4.0 * tk * tk));
      st.t = (b.restart && d < 0.0) ? 1.0 : tn;
      st.P_prev = st.P;  // P_k, for the gap of this iteration
      st.P = p2;
    }
    st.k += 1;
  }
}

cudaError_t launch_rresid(const RBuf& b, int slot, cudaStream_t s) {
  k_rresid<<<dim3(kRRowBlocks, b.B), kRThreads, 0, s>>>(b, slot);
  return cudaGetLastError();
}

// ---------------------------------------------------------------- screening step
// Block per instance: gap at x_k (P_k saved by the residual kernel), radius, sphere test,
// stable compaction of the preserved list, folding of fixed columns into y', stop.
__global__ void __launch_bounds__(kRThreads) k_rgap(RBuf b, int slot) {
  __shared__ double sh[kRThreads / 32];
  __shared__ int shi[kRThreads / 32];
  __shared__ int s_fold[kRThreads];
  __shared__ int s_nfold, s_keep;
  const int k = blockIdx.x;
  RState& st = b.st[k];
  if (st.done) return;
  const RInst in = b.inst[k];
  const int n_act = st.n_active;
  const bool trans = in.dual_mode == kTranslation;
  const double eps = trans ? st.eps : 0.0;
  const double Pk = st.P_prev;  // P_k, saved by the residual kernel
  const float2* __restrict__ xc = b.x[slot];
  const float2* __restrict__ xn = b.x[slot ^ 1];
  const float2* __restrict__ gc = b.g[slot];
  double va = 0.0, vc = 0.0, vx = 0.0;
  for (int q = threadIdx.x; q < n_act; q += kRThreads) {
    const long long c = in.c_off + b.idx[in.c_off + q];
    const double x = df2_to_double(xc[c]);
    const double nr = b.nrm[c];
    vx += fabs(x) * nr;
    if (in.dual_mode != kZero) {
      const double gt = df2_to_double(gc[c]) + (trans ? eps * b.w[c] : 0.0);
      const double lj = b.l[c];
      if (b.jinf[c]) {
        va += (x - lj) * fmax(-gt, 0.0);
        vc += (x - lj) * nr;
      } else {
        const double uj = b.u[c];
        va += (uj - x) * fmax(gt, 0.0) + (x - lj) * fmax(-gt, 0.0);
        vc += fmax(uj - x, x - lj) * nr;
      }
    }
  }
  va = bsum(va, sh);
  vc = bsum(vc, sh);
  vx = bsum(vx, sh);
  const double rnorm = sqrt(2.0 * Pk) * (1.0 + 1e-6);
  const double eta = in.Cg * rnorm + (trans ? eps * in.gamma_w * in.t_norm : 0.0);
  const double E_r = st.E_fold + in.Cf * vx + in.Csub * (rnorm + st.y_norm + st.S_fold + vx);
  double gap;
  if (in.dual_mode == kZero) {
    gap = 0.5 * (rnorm + E_r) * (rnorm + E_r);
  } else {
    const double d = E_r + eps * in.t_norm;
    gap = va + eta * vc + 0.5 * d * d;
  }
  gap *= (1.0 + 1e-12);
  const double radius = sqrt(2.0 * gap);
  const bool stop = gap < b.tol || st.k >= b.max_iter;
  // sphere test and stable compaction (a coordinate is fixed once x_k and x_{k+1} sit at the
  // bound the rule names)
  const bool test = b.screening && in.dual_mode != kZero;
  const double rr = radius * (1.0 + 1e-12) + eta;
  if (threadIdx.x == 0) {
    s_nfold = 0;
    s_keep = 0;
  }
  __syncthreads();
  int npins = 0;
  for (int q0 = 0; q0 < n_act; q0 += kRThreads) {
    const int q = q0 + threadIdx.x;
    int j = -1, pin = 0;
    if (q < n_act) {
      j = b.idx[in.c_off + q];
      const long long c = in.c_off + j;
      const double nr = b.nrm[c];
      if (test && nr > 0.0) {
        const double gt = df2_to_double(gc[c]) + (trans ? eps * b.w[c] : 0.0);
        const double thr = rr * nr * (1.0 + 1e-12);
        float2 bnd = make_float2(0.f, 0.f);
        if (gt < -thr) {
          pin = 1;
          bnd = b.l2[c];
        } else if (!b.jinf[c] && gt > thr) {
          pin = 2;
          bnd = b.u2[c];
        }
        if (pin && !(df2_eq(xc[c], bnd) && df2_eq(xn[c], bnd))) pin = 0;
      }
    }
    int tot = 0;
    const int pos = bscan(q < n_act && !pin ? 1 : 0, shi, &tot);
    if (q < n_act && !pin) b.idx_tmp[in.c_off + s_keep + pos] = j;
    if (pin) {
      const long long c = in.c_off + j;
      b.flags[c] = (uint8_t)pin;
      ++npins;
      const float2 bnd = pin == 1 ? b.l2[c] : b.u2[c];
      if (bnd.x != 0.f || bnd.y != 0.f) {
        const int f = atomicAdd(&s_nfold, 1);
        if (f < kRThreads) s_fold[f] = j;
      }
    }
    __syncthreads();
    if (threadIdx.x == 0) s_keep += tot;
    __syncthreads();
    // fold the fixed columns with nonzero bounds into y' (a few at a time)
    const int nf = min(s_nfold, kRThreads);
    if (nf > 0) {
      double sf = 0.0;
      for (int f = 0; f < nf; ++f) {
        const long long c = in.c_off + s_fold[f];
        sf += fabs(df2_to_double(b.flags[c] == 1 ? b.l2[c] : b.u2[c])) * b.nrm[c];
      }
      for (int i = threadIdx.x; i < in.m; i += kRThreads) {
        float yh = b.yh[in.r_off + i], yl = b.yl[in.r_off + i];
        float s = 0.f, e = 0.f;
        for (int f = 0; f < nf; ++f) {
          const long long c = in.c_off + s_fold[f];
          const float2 bv = b.flags[c] == 1 ? b.l2[c] : b.u2[c];
          df_fma(s, e, b.A[in.a_off + (long long)s_fold[f] * in.lda + i], bv.x, bv.y);
        }
        float dh, de;
        two_sum(yh, -s, dh, de);
        de += yl - e;
        two_sum(dh, de, yh, yl);
        b.yh[in.r_off + i] = yh;
        b.yl[in.r_off + i] = yl;
      }
      __syncthreads();
      if (threadIdx.x == 0) {
        st.S_fold += sf;
        st.E_fold += (in.Cf + in.Csub) * sf;
        s_nfold = 0;
      }
      __syncthreads();
    }
  }
  // the compacted list replaces the old one
  const int keep = s_keep;
  for (int q = threadIdx.x; q < keep; q += kRThreads) b.idx[in.c_off + q] = b.idx_tmp[in.c_off + q];
  npins = (int)bsum((double)npins, sh);
  if (threadIdx.x == 0) {
    st.gap = gap;
    st.radius = radius;
    st.eta = eta;
    st.gap_evals += 1;
    st.n_active = keep;
    st.n_pins += npins;
    if (stop) {
      st.converged = gap < b.tol ? 1 : 0;
      st.out_slot = slot;
      st.done = 1;
    }
  }
}

cudaError_t launch_rgap(const RBuf& b, int slot, cudaStream_t s) {
  k_rgap<<<b.B, kRThreads, 0, s>>>(b, slot);
  return cudaGetLastError();
}

__global__ void k_rloop_ctl(RBuf b, cudaGraphConditionalHandle h, int max_chunks) {
  if (threadIdx.x == 0 && blockIdx.x == 0) {
    const int c = ++*b.chunks;
    if (*b.n_act_inst == 0 || *b.err || c >= max_chunks) cudaGraphSetConditional(h, 0);
  }
}

cudaError_t launch_rloop_ctl(const RBuf& b, cudaGraphConditionalHandle h, int max_chunks, cudaStream_t s) {
  k_rloop_ctl<<<1, 32, 0, s>>>(b, h, max_chunks);
  return cudaGetLastError();
}

// x_out per column from the returned iterate, fixed coordinates at their bounds.
__global__ void k_rexport(RBuf b) {
  const int k = blockIdx.x;
  const RInst in = b.inst[k];
  const int slot = b.st[k].out_slot;
  for (int j = threadIdx.x; j < in.n; j += blockDim.x) {
    const long long c = in.c_off + j;
    const uint8_t f = b.flags[c];
    b.xout[c] = f == 1 ? b.l[c] : f == 2 ? b.u[c] : fmin(fmax(df2_to_double(b.x[slot][c]), b.l[c]), b.u[c]);
  }
}

cudaError_t launch_rexport(const RBuf& b, cudaStream_t s) {
  k_rexport<<<b.B, 256, 0, s>>>(b);
  return cudaGetLastError();
}

}  // namespace bvls
