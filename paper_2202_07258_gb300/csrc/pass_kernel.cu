// One streaming pass over the preserved columns per iteration (A read once from HBM).
//
// For iteration k the pass computes, column by column,
//   g_k,j     = a_j^T r_k                       (correlation; -grad P(x_k), Eq. (grad))
//   x_{k+1,j} = clip(v_j + g_v,j / L, l_j, u_j) (FISTA step; g_v = (1+b) g_k - b g_{k-1})
// and, while column a_j is still in shared memory, accumulates q_{k+1} = A_S x_{k+1}
// (Eq. (decmposition_fwd)), so the next residual r_{k+1} = y' - q_{k+1} needs no second
// pass over A.  The per-column step depends on g_k,j alone, so both products of an
// iteration share one read of the column.
//
// Warp roles in each CTA (one CTA per SM, columns split into contiguous ranges):
//   producer  lane 0 streams columns into a ring of shared-memory stages with bulk copies
//             (cp.async.bulk, completion on a `full` mbarrier per stage);
//   dot       kPassDot warps, one column each: a_j^T r from shared memory in double-float,
//             then the FP64 step; x_{k+1,j} is handed to the q warps through shared memory
//             and an `xready` mbarrier;
//   q         QW warps, each owning a fixed slice of rows: q_slice += a_j x_{k+1,j} in
//             double-float registers over every column of the CTA; columns with
//             x_{k+1,j} = 0 are skipped.  At the end the CTA writes its row partials
//             (double-float) to a per-CTA slice of a global buffer.
// A stage is released (`empty` mbarrier) when its dot warp and all q warps are done.
// k_resid then sums the partials and forms r_{k+1} = y' - q and P_{k+1} = 1/2 ||r_{k+1}||^2.
// The per-column step runs in double-float float32 arithmetic: float64 instructions are
// slow on this part and would sit on the path from a column's dot product to its x_{k+1,j}.
#include <algorithm>

#include "common.cuh"
#include "f32x2.cuh"
#include "tma.cuh"

namespace bvls {

// Dynamic shared memory of the pass: the stages, r (hi, lo), x per stage slot, the
// full / xready / empty barriers, the issue counters and the CTA's column indices.
__host__ __device__ inline size_t pass_smem_bytes(int lda, int m4, int nstages, int cps, int idx_cap) {
  const size_t st = (size_t)nstages;
  return st * (size_t)cps * lda * 4 + (size_t)m4 * 8 + st * cps * 8 + 3 * st * 8 + st * 4 +
         (size_t)idx_cap * 4 + 64;
}

// The persistent form adds, 16-byte aligned, x (two slots), g (two slots), l and u of the
// CTA's columns.
__host__ __device__ inline size_t iters_smem_bytes(int lda, int m4, int nstages, int cps, int idx_cap) {
  return pass_smem_bytes(lda, m4, nstages, cps, idx_cap) + 16 + (size_t)idx_cap * 6 * sizeof(float2);
}

namespace {

// Four rows (one float4 as two packed pairs) of one product term: double-float (kX2) or
// float32 accumulation.
template <int PREC>
__device__ __forceinline__ void pacc4x2(f32x2 (&s)[2], f32x2 (&c)[2], const ulonglong2 a, f32x2 h0, f32x2 h1,
                                        f32x2 l0, f32x2 l1) {
  if (PREC == kX2) {
    df_fma_x2(s[0], c[0], a.x, h0, l0);
    df_fma_x2(s[1], c[1], a.y, h1, l1);
  } else {
    s[0] = x2_fma(a.x, h0, s[0]);
    s[1] = x2_fma(a.y, h1, s[1]);
  }
}

template <int PREC>
__device__ __forceinline__ void pmerge(float& s, float& c, float s2, float c2) {
  if (PREC == kX2) df_add(s, c, s2, c2);
  else s += s2;
}

// a_j^T r for the two columns of a work unit (colB == colA for a lone last column: measured
// faster than a one-column loop),
// r staged in shared memory as (hi, lo) float4 rows; double-float (DP == kX2) or float32
// accumulation.  Every lane returns both sums.
template <int DP>
__device__ __forceinline__ void dot_pair(const float4* colA, const float4* colB, const float4* srh,
                                         const float4* srl, int m4q, int lane, float2& ga, float2& gb) {
  const ulonglong2* A2 = reinterpret_cast<const ulonglong2*>(colA);
  const ulonglong2* B2 = reinterpret_cast<const ulonglong2*>(colB);
  const ulonglong2* H2 = reinterpret_cast<const ulonglong2*>(srh);
  const ulonglong2* L2 = reinterpret_cast<const ulonglong2*>(srl);
  f32x2 sa2[2] = {0ull, 0ull}, ca2[2] = {0ull, 0ull}, sb2[2] = {0ull, 0ull}, cb2[2] = {0ull, 0ull};
#pragma unroll 2
  for (int i = lane; i < m4q; i += 32) {
    const ulonglong2 h = H2[i];
    const ulonglong2 l = DP == kX2 ? L2[i] : make_ulonglong2(0ull, 0ull);
    pacc4x2<DP>(sa2, ca2, A2[i], h.x, h.y, l.x, l.y);
    pacc4x2<DP>(sb2, cb2, B2[i], h.x, h.y, l.x, l.y);
  }
  float sa[4], ca[4], sb[4], cb[4];
  x2_unpack(sa2[0], sa[0], sa[1]);
  x2_unpack(sa2[1], sa[2], sa[3]);
  x2_unpack(ca2[0], ca[0], ca[1]);
  x2_unpack(ca2[1], ca[2], ca[3]);
  x2_unpack(sb2[0], sb[0], sb[1]);
  x2_unpack(sb2[1], sb[2], sb[3]);
  x2_unpack(cb2[0], cb[0], cb[1]);
  x2_unpack(cb2[1], cb[2], cb[3]);
  pmerge<DP>(sa[0], ca[0], sa[1], ca[1]);
  pmerge<DP>(sa[2], ca[2], sa[3], ca[3]);
  pmerge<DP>(sa[0], ca[0], sa[2], ca[2]);
  pmerge<DP>(sb[0], cb[0], sb[1], cb[1]);
  pmerge<DP>(sb[2], cb[2], sb[3], cb[3]);
  pmerge<DP>(sb[0], cb[0], sb[2], cb[2]);
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const float os = __shfl_xor_sync(0xffffffffu, sa[0], o);
    const float oc = __shfl_xor_sync(0xffffffffu, ca[0], o);
    const float ps = __shfl_xor_sync(0xffffffffu, sb[0], o);
    const float pc = __shfl_xor_sync(0xffffffffu, cb[0], o);
    pmerge<DP>(sa[0], ca[0], os, oc);
    pmerge<DP>(sb[0], cb[0], ps, pc);
  }
  ga = df2_norm(sa[0], DP == kX2 ? ca[0] : 0.0f);
  gb = df2_norm(sb[0], DP == kX2 ? cb[0] : 0.0f);
}

// As dot_pair<kF32> over at most RTOT float4 chunks per lane, with the lane's first RT chunks
// of r (rows lane + 32 t) held in registers for the whole iteration instead of read from
// shared memory for every pair; the same accumulation order, so the same sums bit for bit.
template <int RT, int RTOT>
__device__ __forceinline__ void dot_pair_reg(const float4* colA, const float4* colB, const float4 (&rr)[RT],
                                             const float4* srh, int m4q, int lane, float2& ga, float2& gb) {
  const ulonglong2* A2 = reinterpret_cast<const ulonglong2*>(colA);
  const ulonglong2* B2 = reinterpret_cast<const ulonglong2*>(colB);
  f32x2 sa2[2] = {0ull, 0ull}, sb2[2] = {0ull, 0ull};
#pragma unroll
  for (int t = 0; t < RTOT; ++t) {
    const int i = lane + 32 * t;
    if (i < m4q) {
      const ulonglong2 a = A2[i], b = B2[i];
      const float4 r4 = t < RT ? rr[t < RT ? t : 0] : srh[i];
      const f32x2 h0 = x2_pack(r4.x, r4.y), h1 = x2_pack(r4.z, r4.w);
      sa2[0] = x2_fma(a.x, h0, sa2[0]);
      sa2[1] = x2_fma(a.y, h1, sa2[1]);
      sb2[0] = x2_fma(b.x, h0, sb2[0]);
      sb2[1] = x2_fma(b.y, h1, sb2[1]);
    }
  }
  float sa[4], sb[4];
  x2_unpack(sa2[0], sa[0], sa[1]);
  x2_unpack(sa2[1], sa[2], sa[3]);
  x2_unpack(sb2[0], sb[0], sb[1]);
  x2_unpack(sb2[1], sb[2], sb[3]);
  sa[0] += sa[1];
  sa[2] += sa[3];
  sa[0] += sa[2];
  sb[0] += sb[1];
  sb[2] += sb[3];
  sb[0] += sb[2];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    sa[0] += __shfl_xor_sync(0xffffffffu, sa[0], o);
    sb[0] += __shfl_xor_sync(0xffffffffu, sb[0], o);
  }
  ga = df2_norm(sa[0], 0.0f);
  gb = df2_norm(sb[0], 0.0f);
}

// q_slice += sum over one stage's columns of a_j x_j on the lane's rows (QT float4 chunks,
// as packed pairs), columns with x_j = 0 skipped (the test is uniform across the warp).  A
// stage holds at most 8 columns and their x values are read together.  With few row chunks
// per lane the column loop is unrolled with a per-column test; with QT = 4 the warp walks
// the stage's nonzero columns two at a time, both columns' loads issued first (measured on
// 4000-row columns: 104 against 114 us per iteration; no gain at QT = 2, and at QT = 8 the
// two columns' registers spill).
//
// QP == kMix (mode MIXED): the stage's columns are summed in float32 with the high part of
// x_j (one packed FMA per element), and that stage sum enters the double-float accumulator
// with one TwoSum.  The stage sum is off by at most gamma_cps sum |a_ij xh_j| plus the dropped
// sum |a_ij xl_j| <= u sum |a_ij x_j|, so the forward product is good to about (cps + 1) u
// relative to sum_j |a_ij x_j| instead of the full double-float accuracy, at a sixth of its
// arithmetic (the double-float forward product was the pass's bottleneck).
template <int QP, int QT, int QW>
__device__ __forceinline__ void q_stage(f32x2 (&qs)[QT][2], f32x2 (&qc)[QT][2], const float* sbase,
                                        const float2* sxs, int nc, int lda, int qw, int lane, int m4q) {
  float2 xs[8];
#pragma unroll
  for (int c = 0; c < 8; ++c) xs[c] = c < nc ? sxs[c] : make_float2(0.f, 0.f);
  if (QP == kMix) {
    f32x2 gs[QT][2];
#pragma unroll
    for (int t = 0; t < QT; ++t) gs[t][0] = gs[t][1] = 0ull;
#pragma unroll
    for (int c = 0; c < 8; ++c) {
      if (xs[c].x != 0.0f) {
        const ulonglong2* col = reinterpret_cast<const ulonglong2*>(sbase + (size_t)c * lda);
        const f32x2 xh = x2_pack(xs[c].x, xs[c].x);
#pragma unroll
        for (int t = 0; t < QT; ++t) {
          const int c4 = qw * 32 + lane + t * 32 * QW;
          if (c4 < m4q) {
            const ulonglong2 a = col[c4];
            gs[t][0] = x2_fma(a.x, xh, gs[t][0]);
            gs[t][1] = x2_fma(a.y, xh, gs[t][1]);
          }
        }
      }
    }
#pragma unroll
    for (int t = 0; t < QT; ++t) {
      df_add_x2(qs[t][0], qc[t][0], gs[t][0], 0ull);
      df_add_x2(qs[t][1], qc[t][1], gs[t][1], 0ull);
    }
    return;
  }
  if (QT != 4) {
#pragma unroll
    for (int c = 0; c < 8; ++c) {
      if (xs[c].x != 0.0f || xs[c].y != 0.0f) {
        const ulonglong2* col = reinterpret_cast<const ulonglong2*>(sbase + (size_t)c * lda);
        const f32x2 xh = x2_pack(xs[c].x, xs[c].x), xl = x2_pack(xs[c].y, xs[c].y);
#pragma unroll
        for (int t = 0; t < QT; ++t) {
          const int c4 = qw * 32 + lane + t * 32 * QW;
          if (c4 < m4q) pacc4x2<QP>(qs[t], qc[t], col[c4], xh, xh, xl, xl);
        }
      }
    }
    return;
  }
  unsigned mask = 0;
#pragma unroll
  for (int c = 0; c < 8; ++c)
    if (xs[c].x != 0.0f || xs[c].y != 0.0f) mask |= 1u << c;
  while (mask) {
    const int c0 = __ffs(mask) - 1;
    mask &= mask - 1;
    int c1 = -1;
    if (mask) {
      c1 = __ffs(mask) - 1;
      mask &= mask - 1;
    }
    const ulonglong2* col0 = reinterpret_cast<const ulonglong2*>(sbase + (size_t)c0 * lda);
    const ulonglong2* col1 = reinterpret_cast<const ulonglong2*>(sbase + (size_t)(c1 >= 0 ? c1 : c0) * lda);
    ulonglong2 a0[QT], a1[QT];
#pragma unroll
    for (int t = 0; t < QT; ++t) {
      const int c4 = qw * 32 + lane + t * 32 * QW;
      if (c4 < m4q) {
        a0[t] = col0[c4];
        a1[t] = col1[c4];
      }
    }
    float2 x0 = xs[0], x1 = xs[0];
#pragma unroll
    for (int c = 0; c < 8; ++c) {
      if (c == c0) x0 = xs[c];
      if (c == c1) x1 = xs[c];
    }
    const f32x2 xh0 = x2_pack(x0.x, x0.x), xl0 = x2_pack(x0.y, x0.y);
    const f32x2 xh1 = x2_pack(x1.x, x1.x), xl1 = x2_pack(x1.y, x1.y);
#pragma unroll
    for (int t = 0; t < QT; ++t) {
      const int c4 = qw * 32 + lane + t * 32 * QW;
      if (c4 < m4q) {
        pacc4x2<QP>(qs[t], qc[t], a0[t], xh0, xh0, xl0, xl0);
        if (c1 >= 0) pacc4x2<QP>(qs[t], qc[t], a1[t], xh1, xh1, xl1, xl1);
      }
    }
  }
}

// The lane's q partials (row chunk c4 of t) as float4 pairs (hi, lo) of four rows.
template <int QP>
__device__ __forceinline__ void q_store(float2* part, int c4, const f32x2 (&s)[2], const f32x2 (&c)[2]) {
  float s0, s1, s2, s3, c0 = 0.f, c1 = 0.f, c2 = 0.f, c3 = 0.f;
  x2_unpack(s[0], s0, s1);
  x2_unpack(s[1], s2, s3);
  if (QP != kF32) {
    x2_unpack(c[0], c0, c1);
    x2_unpack(c[1], c2, c3);
  }
  float4* dst = reinterpret_cast<float4*>(part + 4 * c4);
  dst[0] = make_float4(s0, c0, s1, c1);
  dst[1] = make_float4(s2, c2, s3, c3);
}

__device__ __forceinline__ float2 clip2(float2 x, float2 lj, float2 uj) {
  if (df2_lt(x, lj)) x = lj;
  if (df2_lt(uj, x)) x = uj;
  return x;
}

// One coordinate's step from g2 = a_j^T r_k, in double-float arithmetic (no float64 on this
// path).  FISTA: x_{k+1} = clip(v + g_v / L), v = x_k + beta (x_k - x_{k-1}),
// g_v = (1 + beta) g_k - beta g_{k-1} = a_j^T (y' - A v_k); the forward product takes x_{k+1}
// and *dotc is the restart-test term g_v (x_{k+1} - x_k).  Primal-dual: x_{k+1} =
// clip(x_k - tau a_j^T z) and the forward product takes xbar = 2 x_{k+1} - x_k.
__device__ __forceinline__ float2 coord_step(const Params& p, float2 g2, float2 xk, float2 xp, float2 gpv,
                                             float2 lj, float2 uj, float2 bb, float2 onepb, float2& xfwd,
                                             float2& dotc) {
  if (p.alg == kChambollePock) {
    const float2 xnew = clip2(df2_sub(xk, df2_mul(g2, p.tau2)), lj, uj);
    xfwd = df2_sub(df2_add(xnew, xnew), xk);
    dotc = make_float2(0.f, 0.f);
    return xnew;
  }
  const float2 gv = df2_sub(df2_mul(onepb, g2), df2_mul(bb, gpv));
  const float2 v = df2_add(xk, df2_mul(bb, df2_sub(xk, xp)));
  const float2 xnew = clip2(df2_add(v, df2_mul(gv, p.invL2)), lj, uj);
  xfwd = xnew;
  dotc = df2_mul(gv, df2_sub(xnew, xk));
  return xnew;
}

}  // namespace

template <int PREC, int QW, int QT>
__global__ void __launch_bounds__(32 * (1 + kPassDot + QW), 1)
    k_pass(Params p, Buffers b, int slot, int gap_iter, int nstages, int cps) {
  // arithmetic of the two products: correlations a_j^T r_k (DP) and A_S x_{k+1} (QP)
  constexpr int DP = PREC == kX2 ? kX2 : kF32;
  constexpr int QP = PREC;   // kMix: float32 stage sums merged in double-float
  DevState* st = b.st;
  if (st->done) return;
  extern __shared__ __align__(128) unsigned char smem[];
  const int m4q = p.m4 >> 2;
  const uint32_t col_bytes = (uint32_t)p.lda * 4u;
  const size_t stage_floats = (size_t)cps * p.lda;           // a stage holds cps columns
  float* stages = reinterpret_cast<float*>(smem);
  float4* srh = reinterpret_cast<float4*>(smem + (size_t)nstages * stage_floats * 4);
  float4* srl = srh + m4q;
  float2* sx = reinterpret_cast<float2*>(srl + m4q);            // x_{k+1} per stage slot
  uint64_t* full = reinterpret_cast<uint64_t*>(sx + (size_t)nstages * cps);
  uint64_t* xready = full + nstages;
  uint64_t* empty = xready + nstages;
  // Uses of each stage issued so far.  mbarrier waits only see the parity of a phase, so a
  // dot warp (which takes every kPassDot-th column) first waits until the producer has
  // issued the use it needs: by then the previous use of that stage has landed and been
  // consumed, and the parity wait on `full` is exact.
  volatile int* s_issued = reinterpret_cast<volatile int*>(empty + nstages);
  int* sidx = const_cast<int*>(s_issued) + nstages;   // this CTA's column indices
  __shared__ float2 s_dot[kPassDot];
  __shared__ double s_eps[kPassDot];
  __shared__ double s_scal[3];   // beta, t_{k+1} (no restart), eta_g: computed once per CTA
  __shared__ float2 s_beta2[2];  // beta and 1 + beta as double-float pairs
  __shared__ int s_err;
  __shared__ double s_th[32];

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int n_act = st->n_active;
  const int per = (n_act + gridDim.x - 1) / gridDim.x;
  const int p0 = min(n_act, (int)blockIdx.x * per);
  const int nq = min(n_act, p0 + per) - p0;
  const int ngroups = (nq + cps - 1) / cps;

  // P_k = 1/2 ||r_k||^2: from the residual kernel's block partials after the first
  // iteration (one L2 round trip by warp 0); CTA 0 records it for the gap kernel.
  double Pk = 0.0;
  if (threadIdx.x < 32) {
    Pk = st->k > 0 ? warp_load_sum(b.tileR, (p.m4 + 31) / 32) : st->P[slot];
    if (threadIdx.x == 0 && blockIdx.x == 0) st->P[slot] = Pk;
  }
  if (threadIdx.x == 0) {
    for (int s = 0; s < nstages; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&xready[s], cps);        // one arrival per column of the stage
      mbar_init(&empty[s], cps + QW);    // each column's dot warp and every q warp
      s_issued[s] = 0;
    }
    fence_barrier_init();
    s_err = 0;
    // float64 runs at a small fraction of the float32 rate: scalars once per CTA
    const double tk = st->t;
    const double tn = 0.5 * (1.0 + sqrt(1.0 + 4.0 * tk * tk));
    const double beta = (tk - 1.0) / tn;
    s_scal[0] = beta;
    s_scal[1] = tn;
    s_scal[2] = p.Cg * sqrt(2.0 * Pk) * (1.0 + 1e-6);
    s_beta2[0] = df2_from_double(beta);
    s_beta2[1] = df2_from_double(1.0 + beta);
  }
  if (threadIdx.x < kPassDot) {
    s_dot[threadIdx.x] = make_float2(0.f, 0.f);
    s_eps[threadIdx.x] = 0.0;
  }
  for (int i = threadIdx.x; i < m4q; i += blockDim.x) {
    srh[i] = __ldcg(reinterpret_cast<const float4*>(b.rh) + i);
    srl[i] = __ldcg(reinterpret_cast<const float4*>(b.rl) + i);
  }
  // one coalesced read of the index range instead of a dependent load per column
  for (int q = threadIdx.x; q < nq; q += blockDim.x) sidx[q] = b.idx[p0 + q];
  __syncthreads();
  if (gap_iter && p.wstar && blockIdx.x == 0) {
    // fixed dual point theta = theta_fixed + eps_star t: ||theta - r_k||^2 for the gap
    const float* rh = reinterpret_cast<const float*>(srh);
    const float* rl = reinterpret_cast<const float*>(srl);
    double acc = 0.0;
    for (int i = threadIdx.x; i < p.m; i += blockDim.x) {
      const double d = p.theta[i] + p.eps_star * p.tvec[i] - ((double)rh[i] + (double)rl[i]);
      acc += d * d;
    }
    acc = warp_sum_d(acc);
    if ((threadIdx.x & 31) == 0) s_th[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
      double t2 = 0.0;
      for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t2 += s_th[w];
      st->theta_r2 = t2;
    }
  }

  const double tn = s_scal[1];

  if (warp == 0) {
    // ---------------------------------------------------------------- producer
    // Group g = columns [g*cps, min(nq, (g+1)*cps)) goes to stage g % nstages; columns that
    // are adjacent in A (runs of the preserved list) travel in one bulk copy.
    if (lane == 0) {
      int issued = 0;
      for (int g = 0; g < ngroups; ++g) {
        const int s = g % nstages;
        const int u = g / nstages;
        if (u > 0 && !mbar_wait(&empty[s], (u - 1) & 1)) {
          s_err = 1;
          break;
        }
        const int q0 = g * cps;
        const int nc = min(cps, nq - q0);
        mbar_arrive_expect_tx(&full[s], (uint32_t)nc * col_bytes);
        float* dst = stages + (size_t)s * stage_floats;
        int c = 0;
        while (c < nc) {
          int len = 1;
          while (c + len < nc && sidx[q0 + c + len] == sidx[q0 + c] + len) ++len;
          bulk_g2s(dst + (size_t)c * p.lda, p.A + (size_t)sidx[q0 + c] * p.lda, (uint32_t)len * col_bytes,
                   &full[s]);
          c += len;
        }
        // a short last group: stand in for the missing columns' dot warps
        for (int k = nc; k < cps; ++k) {
          mbar_arrive(&xready[s]);
          mbar_arrive(&empty[s]);
        }
        s_issued[s] = u + 1;
        issued = g + 1;
      }
      // The most recent copy into each stage must land before the CTA may exit.
      for (int g = max(0, issued - nstages); g < issued; ++g)
        if (!mbar_wait(&full[g % nstages], (g / nstages) & 1)) s_err = 1;
    }
  } else if (warp <= kPassDot) {
    // ---------------------------------------------------------------- dot warps
    const int dw = warp - 1;
    const double eta_g = s_scal[2];
    const float2 bb = s_beta2[0], onepb = s_beta2[1];
    const bool want_eps = gap_iter && p.dual_mode == kTranslation && !p.wstar;
    const float2* __restrict__ xc = b.x[slot];
    float2* xn = b.x[slot ^ 1];
    const float2* __restrict__ gp = b.g[slot ^ 1];
    float2* gc = b.g[slot];
    float2 dot = make_float2(0.f, 0.f);
    double epsm = 0.0;
    // Work unit: two adjacent columns of one stage (they share the loads of r and give 8
    // independent accumulation chains); single columns when a stage holds an odd count.
    const int U = (cps % 2 == 0) ? 2 : 1;
    for (int w = dw; w * U < nq; w += kPassDot) {
      const int q0 = w * U;
      const int ncol = min(U, nq - q0);
      const int g = q0 / cps;
      const int s = g % nstages;
      const int u = g / nstages;
      const int c0 = q0 - g * cps;
      // lane e (< ncol) runs the step of column q0 + e: its data does not depend on the
      // column values, so it is loaded before the wait
      const int e = lane < ncol ? lane : 0;
      const int j = sidx[q0 + e];
      float2 xk = make_float2(0.f, 0.f), xp = xk, gpv = xk, lj = xk, uj = xk;
      double nr = 0.0, wj = 0.0;
      int inf_j = 0;
      if (lane < ncol) {
        xk = xc[j];
        xp = xn[j];
        gpv = gp[j];
        lj = p.l2[j];
        uj = p.u2[j];
        if (want_eps) {
          nr = p.nrm[j];
          wj = p.w[j];
          inf_j = p.jinf[j];
        }
      }
      if (!warp_all(smem_wait_geq(&s_issued[s], u + 1) && mbar_wait(&full[s], u & 1))) {
        s_err = 1;
        break;
      }
      const float* sbase = stages + (size_t)s * stage_floats + (size_t)c0 * p.lda;
      const float4* colA = reinterpret_cast<const float4*>(sbase);
      const float4* colB = reinterpret_cast<const float4*>(sbase + (ncol > 1 ? p.lda : 0));
      float2 ga, gb;
      dot_pair<DP>(colA, colB, srh, srl, m4q, lane, ga, gb);
      __syncwarp();
      if (lane < ncol) {
        const int c = c0 + lane;
        mbar_arrive(&empty[s]);  // this column's dot is done with the stage
        const float2 g2 = lane == 0 ? ga : gb;
        float2 xf, dc;
        const float2 xnew = coord_step(p, g2, xk, xp, gpv, lj, uj, bb, onepb, xf, dc);
        sx[(size_t)s * cps + c] = QP != kF32 ? xf : make_float2(xf.x, 0.0f);
        mbar_arrive(&xready[s]);
        xn[j] = xnew;
        gc[j] = g2;
        if (p.alg == kChambollePock) continue;
        dot = df2_add(dot, dc);
        if (want_eps && inf_j && nr > 0.0) {
          const double den = -wj - p.gamma_w * nr * p.t_norm;
          epsm = fmax(epsm, fmax(df2_to_double(g2) + eta_g * nr, 0.0) / den);
        }
      }
    }
    // lanes 0 and 1 carry partial sums
    {
      const float2 o = make_float2(__shfl_down_sync(0xffffffffu, dot.x, 1), __shfl_down_sync(0xffffffffu, dot.y, 1));
      const double oe = __shfl_down_sync(0xffffffffu, epsm, 1);
      if (lane == 0) {
        dot = df2_add(dot, o);
        epsm = fmax(epsm, oe);
      }
    }
    if (lane == 0) {
      s_dot[dw] = dot;
      s_eps[dw] = epsm;
    }
  } else {
    // ---------------------------------------------------------------- q warps
    const int qw = warp - 1 - kPassDot;
    f32x2 qs[QT][2], qc[QT][2];   // QT float4 row chunks per lane
#pragma unroll
    for (int t = 0; t < QT; ++t)
#pragma unroll
      for (int c = 0; c < 2; ++c) qs[t][c] = qc[t][c] = 0ull;
    for (int g = 0; g < ngroups; ++g) {
      const int s = g % nstages;
      const int u = g / nstages;
      if (!warp_all(mbar_wait(&xready[s], u & 1) && mbar_wait(&full[s], u & 1))) {
        s_err = 1;
        break;
      }
      q_stage<QP, QT, QW>(qs, qc, stages + (size_t)s * stage_floats, sx + (size_t)s * cps, min(cps, nq - g * cps),
                          p.lda, qw, lane, m4q);
      __syncwarp();
      if (lane == 0) mbar_arrive(&empty[s]);
    }
    // per-CTA partials of A_S x_{k+1} (every row written, zeros included)
    float2* part = b.qpart + (size_t)blockIdx.x * p.m4;
#pragma unroll
    for (int t = 0; t < QT; ++t) {
      const int c4 = qw * 32 + lane + t * 32 * QW;
      if (c4 < m4q) q_store<QP>(part, c4, qs[t], qc[t]);
    }
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    float2 d = make_float2(0.f, 0.f);
    double e = 0.0;
    for (int w = 0; w < kPassDot; ++w) {
      d = df2_add(d, s_dot[w]);
      e = fmax(e, s_eps[w]);
    }
    b.blk[4 * blockIdx.x + 0] = df2_to_double(d);
    b.blk[4 * blockIdx.x + 1] = e;
    if (s_err) atomicOr(&st->error, 1);
  }
  // last CTA: restart test, momentum parameter, translation step, iteration count
  __shared__ int s_last;
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) {
    const unsigned prev = atomicAdd(&st->cnt_tr, 1u);
    s_last = prev == gridDim.x - 1;
    if (s_last) st->cnt_tr = 0u;
  }
  __syncthreads();
  if (!s_last) return;
  __threadfence();
  if (threadIdx.x < 32) {
    double d = 0.0, e = 0.0;
    for (int t0 = 0; t0 < (int)gridDim.x; t0 += 256) {
      double dv[8], ev[8];
#pragma unroll
      for (int k = 0; k < 8; ++k) {   // loads first: one L2 round trip per 256 CTAs
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

// r_{k+1} = y' - q_{k+1} and P_{k+1} = 1/2 ||r_{k+1}||^2 from the per-CTA partials of the
// pass, in double-float arithmetic.  Block: 32 rows (one per lane) x 8 warps over the
// partials; the summation order is fixed, so r is reproducible run to run.
__global__ void __launch_bounds__(256) k_resid(Params p, Buffers b, int slot, int nparts) {
  DevState* st = b.st;
  if (st->done) return;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int row = blockIdx.x * 32 + lane;
  float s = 0.f, c = 0.f;
  if (row < p.m4) {
    // batches of loads in flight, then the (dependent) double-float additions
    for (int t0 = warp; t0 < nparts; t0 += 8 * 8) {
      float2 v[8];
#pragma unroll
      for (int k = 0; k < 8; ++k) {
        const int t = t0 + 8 * k;
        v[k] = t < nparts ? __ldcg(&b.qpart[(size_t)t * p.m4 + row]) : make_float2(0.f, 0.f);
      }
#pragma unroll
      for (int k = 0; k < 8; ++k) df_add(s, c, v[k].x, v[k].y);
    }
  }
  __shared__ float2 sh[8][32];
  sh[warp][lane] = make_float2(s, c);
  __syncthreads();
  if (warp == 0 && p.alg == kChambollePock) {
    // primal-dual: z_{k+2} = (z_{k+1} + sigma (A xbar - y')) / (1 + sigma) and
    // r(x_{k+1}) = (r(x_k) + y' - A xbar) / 2; partials of 1/2 ||r||^2, ||z_{k+1} + r||^2, ||z_{k+1}||^2
    for (int w = 1; w < 8; ++w) df_add(s, c, sh[w][lane].x, sh[w][lane].y);
    double pv = 0.0, dv = 0.0, zv = 0.0;
    if (row < p.m) {
      const float2 q = df2_norm(s, c);
      const float2 yv = make_float2(b.yh[row], b.yl[row]);
      const float2 z = make_float2(b.rh[row], b.rl[row]);
      const float2 r = make_float2(b.crh[row], b.crl[row]);
      const float2 zn = df2_mul(df2_add(z, df2_mul(df2_sub(q, yv), p.sigma2)), p.inv1ps2);
      const float2 rn = df2_mul(df2_add(r, df2_sub(yv, q)), make_float2(0.5f, 0.f));
      b.rh[row] = zn.x;
      b.rl[row] = zn.y;
      b.crh[row] = rn.x;
      b.crl[row] = rn.y;
      const double rd = df2_to_double(rn), zd = df2_to_double(z);
      pv = 0.5 * rd * rd;
      dv = (zd + rd) * (zd + rd);
      zv = zd * zd;
    }
    for (int o = 16; o > 0; o >>= 1) {
      pv += __shfl_xor_sync(0xffffffffu, pv, o);
      dv += __shfl_xor_sync(0xffffffffu, dv, o);
      zv += __shfl_xor_sync(0xffffffffu, zv, o);
    }
    if (lane == 0) {
      b.tileR[blockIdx.x] = pv;
      b.tileD[blockIdx.x] = dv;
      b.tileZ[blockIdx.x] = zv;
    }
  } else if (warp == 0) {
    for (int w = 1; w < 8; ++w) df_add(s, c, sh[w][lane].x, sh[w][lane].y);
    float ps = 0.f, pc = 0.f;
    if (row < p.m) {
      float dh, de;
      two_sum(b.yh[row], -s, dh, de);
      de += b.yl[row] - c;
      float rh, rl;
      two_sum(dh, de, rh, rl);
      b.rh[row] = rh;
      b.rl[row] = rl;
      const float sq = rh * rh;           // 1/2 r^2 as a double-float
      ps = 0.5f * sq;
      pc = 0.5f * (fmaf(rh, rh, -sq) + 2.0f * rh * rl);
    }
    for (int o = 16; o > 0; o >>= 1) {
      const float os = __shfl_xor_sync(0xffffffffu, ps, o);
      const float oc = __shfl_xor_sync(0xffffffffu, pc, o);
      df_add(ps, pc, os, oc);
    }
    if (lane == 0) b.tileR[blockIdx.x] = df_to_double(ps, pc);   // summed by the next pass
  }
}

// ------------------------------------------------------------------ persistent form
// k_iters runs `niter` consecutive iterations (those between two gap evaluations) in one
// cooperative launch: one CTA per SM, every CTA co-resident.  Each iteration is
//   pass       as k_pass: the CTA's preserved columns stream through the stage ring once,
//              giving a_j^T r_k, the step, and the CTA's partial of A_S x_{k+1};
//   barrier    grid-wide;
//   residual   as k_resid, the rows split into 32-row slices over the CTAs: r_{k+1} and
//              the slice partials of P_{k+1}; one warp per CTA also reduces the per-CTA
//              restart terms (same order everywhere, so all CTAs hold the same t_{k+1})
//              and prepares the next momentum scalars;
//   barrier    grid-wide.
// The CTA's columns keep their x, g and bounds in shared memory for the whole launch
// (written back at the end).  The producer warp takes no part in the barriers: it walks
// the column groups of all `niter` iterations, so the first stages of iteration k+1 load
// while the grid finishes iteration k.  P_k and the margin eta_g are formed only at the
// gap iteration, the one whose values the gap kernel reads.  The outputs after the last
// iteration are those of k_pass + k_resid.

namespace {

// Named barrier 1 over the CTA's consumer warps (all warps but the producer).
template <int NCONS>
__device__ __forceinline__ void consumer_sync() {
  asm volatile("bar.sync 1, %0;" ::"r"(NCONS) : "memory");
}

// Scalars of the step that starts from t_k = T[ti]: t_{k+1} without restart and beta as
// double-float pairs (float64 arithmetic only past the table's end).
__device__ __forceinline__ void momentum(const MomEntry* mom, int ti, double tk, double* s_tn, float2* s_beta2) {
  if (ti < kMomTable) {
    const MomEntry e = mom[ti];
    *s_tn = e.tn;
    s_beta2[0] = e.beta2;
    s_beta2[1] = e.onepb2;
    return;
  }
  const double tn = 0.5 * (1.0 + sqrt(1.0 + 4.0 * tk * tk));
  const double beta = (tk - 1.0) / tn;
  *s_tn = tn;
  s_beta2[0] = df2_from_double(beta);
  s_beta2[1] = df2_from_double(1.0 + beta);
}

}  // namespace


template <int PREC, int DW, int QW, int QT>
__global__ void __launch_bounds__(32 * (1 + DW + QW), 1)
    k_iters(Params p, Buffers b, int slot0, int niter, int gap_last, int nstages, int cps, int idx_cap) {
  constexpr int DP = PREC == kX2 ? kX2 : kF32;
  constexpr int QP = PREC;   // kMix: float32 stage sums merged in double-float
  constexpr int NW = DW + QW;          // consumer warps
  constexpr int NCONS = 32 * NW;
  DevState* st = b.st;
  if (st->done || st->error) return;         // fixed for the whole launch
  extern __shared__ __align__(128) unsigned char smem[];
  const int m4q = p.m4 >> 2;
  const uint32_t col_bytes = (uint32_t)p.lda * 4u;
  const size_t stage_floats = (size_t)cps * p.lda;
  float* stages = reinterpret_cast<float*>(smem);
  float4* srh = reinterpret_cast<float4*>(smem + (size_t)nstages * stage_floats * 4);
  float4* srl = srh + m4q;
  float2* sx = reinterpret_cast<float2*>(srl + m4q);
  uint64_t* full = reinterpret_cast<uint64_t*>(sx + (size_t)nstages * cps);
  uint64_t* xready = full + nstages;
  uint64_t* empty = xready + nstages;
  volatile int* s_issued = reinterpret_cast<volatile int*>(empty + nstages);
  int* sidx = const_cast<int*>(s_issued) + nstages;
  float2* sv = reinterpret_cast<float2*>(smem + ((pass_smem_bytes(p.lda, p.m4, nstages, cps, idx_cap) + 15) & ~(size_t)15));
  float2* sX0 = sv;                    // x by slot (0, 1), this CTA's columns
  float2* sX1 = sv + idx_cap;
  float2* sG0 = sv + 2 * idx_cap;      // g by slot
  float2* sG1 = sv + 3 * idx_cap;
  float2* sL = sv + 4 * idx_cap;
  float2* sU = sv + 5 * idx_cap;
  __shared__ float2 s_dot[DW];
  __shared__ double s_eps[DW];
  __shared__ double s_tn, s_tk, s_etag;   // t_{k+1} without restart, t_k, margin eta_g
  __shared__ float2 s_beta2[2];
  __shared__ int s_ti, s_err, s_ok;
  __shared__ volatile int s_stop;      // the consumers left the iteration loop early
  __shared__ double s_th[NW];
  __shared__ float2 s_red[NW][32];

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int n_act = st->n_active;
  const int k0 = st->k;
  // the CTAs that take part: at least kItersColsMin preserved columns each (the preserved set
  // is fixed for the launch, so every CTA computes the same count)
  const int G = iters_active_ctas(n_act, gridDim.x);
  if ((int)blockIdx.x >= G) return;
  const int per = (n_act + G - 1) / G;
  const int p0 = min(n_act, (int)blockIdx.x * per);
  const int nq = min(n_act, p0 + per) - p0;
  const int ngroups = (nq + cps - 1) / cps;
  const int nslices = (p.m4 + 31) / 32;
  const int nparts = G;
  // grid barriers: a monotonic arrival count, zeroed at the start of the solve; this launch
  // starts from the count st->gbase that earlier launches left, and its barrier number nb
  // (from 1) completes when the count reaches gbase + G * nb
  unsigned long long* gcount = reinterpret_cast<unsigned long long*>(b.gbar);
  const unsigned long long gbase = st->gbase;
  unsigned long long nbar = 0ull;

  if (threadIdx.x == 0) {
    for (int s = 0; s < nstages; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&xready[s], cps);
      mbar_init(&empty[s], cps + QW);
      s_issued[s] = 0;
    }
    fence_barrier_init();
    s_err = 0;
    s_ok = 1;
    s_stop = 0;
    s_ti = st->ti;
    s_tk = st->t;
    momentum(p.mom, s_ti, s_tk, &s_tn, s_beta2);
  }
  for (int q = threadIdx.x; q < nq; q += blockDim.x) {
    const int j = b.idx[p0 + q];
    sidx[q] = j;
    sX0[q] = b.x[0][j];
    sX1[q] = b.x[1][j];
    sG0[q] = b.g[0][j];
    sG1[q] = b.g[1][j];
    sL[q] = p.l2[j];
    sU[q] = p.u2[j];
  }
  __syncthreads();

  if (warp == 0) {
    // ---------------------------------------------------------------- producer
    // Global group gg = it * ngroups + g goes to stage gg % nstages (use gg / nstages).
    if (lane == 0) {
      const int total = niter * ngroups;
      int issued = 0;
      for (int gg = 0; gg < total; ++gg) {
        const int g = gg - (gg / ngroups) * ngroups;
        const int s = gg % nstages;
        const int u = gg / nstages;
        if (u > 0 && !mbar_wait_unless(&empty[s], (u - 1) & 1, &s_stop)) {
          s_err = 1;
          break;
        }
        const int q0 = g * cps;
        const int nc = min(cps, nq - q0);
        mbar_arrive_expect_tx(&full[s], (uint32_t)nc * col_bytes);
        float* dst = stages + (size_t)s * stage_floats;
        int c = 0;
        while (c < nc) {
          int len = 1;
          while (c + len < nc && sidx[q0 + c + len] == sidx[q0 + c] + len) ++len;
          bulk_g2s(dst + (size_t)c * p.lda, p.A + (size_t)sidx[q0 + c] * p.lda, (uint32_t)len * col_bytes,
                   &full[s]);
          c += len;
        }
        for (int k = nc; k < cps; ++k) {
          mbar_arrive(&xready[s]);
          mbar_arrive(&empty[s]);
        }
        s_issued[s] = u + 1;
        issued = gg + 1;
      }
      for (int gg = max(0, issued - nstages); gg < issued; ++gg)
        if (!mbar_wait(&full[gg % nstages], (gg / nstages) & 1)) s_err = 1;
      if (s_err) atomicOr(&st->error, 1);
    }
    return;
  }

  // -------------------------------------------------------------------- consumers
  const int wi = warp - 1;
  const int ct = threadIdx.x - 32;
  for (int it = 0; it < niter; ++it) {
    const int slot = (slot0 + it) & 1;
    const int gap_iter = gap_last && it == niter - 1;
    const int k = k0 + it;
    // prologue: r_k in shared memory; at the gap iteration also P_k and the margin eta_g
    if (gap_iter && warp == 1) {
      const double Pk = k > 0 ? warp_load_sum(b.tileR, nslices) : st->P[slot];
      if (lane == 0) {
        if (blockIdx.x == 0) st->P[slot] = Pk;
        s_etag = p.Cg * sqrt(2.0 * Pk) * (1.0 + 1e-6);
      }
    }
    for (int i = ct; i < m4q; i += NCONS) {
      srh[i] = __ldcg(reinterpret_cast<const float4*>(b.rh) + i);
      if (DP == kX2) srl[i] = __ldcg(reinterpret_cast<const float4*>(b.rl) + i);   // float32 dots use r's high part
    }
    if (gap_iter && p.wstar && blockIdx.x == 0) {
      double acc = 0.0;
      for (int i = ct; i < p.m; i += NCONS) {
        const double d = p.theta[i] + p.eps_star * p.tvec[i] - ((double)__ldcg(b.rh + i) + (double)__ldcg(b.rl + i));
        acc += d * d;
      }
      acc = warp_sum_d(acc);
      if (lane == 0) s_th[wi] = acc;
      consumer_sync<NCONS>();
      if (ct == 0) {
        double t2 = 0.0;
        for (int w = 0; w < NW; ++w) t2 += s_th[w];
        st->theta_r2 = t2;
      }
    }
    consumer_sync<NCONS>();
    const double tn = s_tn;

    if (warp <= DW) {
      // ------------------------------------------------------------ dot warps
      const int dw = warp - 1;
      // mode MIXED with at most 16 float4 row chunks per lane: r_k (high part) in registers
      constexpr bool kRReg = PREC == kMix && QT <= 2;
      constexpr int RT = kRReg ? 8 : 1;   // 16 chunks in registers spilled at 120 registers
      float4 rr[RT];
#pragma unroll
      for (int t = 0; t < RT; ++t) {
        const int i = lane + 32 * t;
        rr[t] = (kRReg && i < m4q) ? srh[i] : make_float4(0.f, 0.f, 0.f, 0.f);
      }
      const double eta_g = gap_iter ? s_etag : 0.0;
      const float2 bb = s_beta2[0], onepb = s_beta2[1];
      const bool want_eps = gap_iter && p.dual_mode == kTranslation && !p.wstar;
      const float2* xc = slot ? sX1 : sX0;
      float2* xn = slot ? sX0 : sX1;
      const float2* gp = slot ? sG0 : sG1;
      float2* gc = slot ? sG1 : sG0;
      float2 dot = make_float2(0.f, 0.f);
      double epsm = 0.0;
      const int U = (cps % 2 == 0) ? 2 : 1;
      for (int w = dw; w * U < nq; w += DW) {
        const int q0 = w * U;
        const int ncol = min(U, nq - q0);
        const int g = q0 / cps;
        const int gg = it * ngroups + g;
        const int s = gg % nstages;
        const int u = gg / nstages;
        const int c0 = q0 - g * cps;
        const int e = lane < ncol ? lane : 0;
        const int qj = q0 + e;                 // the lane's column, local index
        float2 xk = make_float2(0.f, 0.f), xp = xk, gpv = xk, lj = xk, uj = xk;
        double nr = 0.0, wj = 0.0;
        int inf_j = 0;
        if (lane < ncol) {
          xk = xc[qj];
          xp = xn[qj];
          gpv = gp[qj];
          lj = sL[qj];
          uj = sU[qj];
          if (want_eps) {
            const int j = sidx[qj];
            nr = p.nrm[j];
            wj = p.w[j];
            inf_j = p.jinf[j];
          }
        }
        if (!warp_all(smem_wait_geq(&s_issued[s], u + 1) && mbar_wait(&full[s], u & 1))) {
          s_err = 1;
          break;
        }
        const float* sbase = stages + (size_t)s * stage_floats + (size_t)c0 * p.lda;
        const float4* colA = reinterpret_cast<const float4*>(sbase);
        const float4* colB = reinterpret_cast<const float4*>(sbase + (ncol > 1 ? p.lda : 0));
        float2 ga, gb2;
        if constexpr (kRReg) dot_pair_reg<RT, 16>(colA, colB, rr, srh, m4q, lane, ga, gb2);
        else dot_pair<DP>(colA, colB, srh, srl, m4q, lane, ga, gb2);
        __syncwarp();
        if (lane < ncol) {
          const int c = c0 + lane;
          mbar_arrive(&empty[s]);
          const float2 g2 = lane == 0 ? ga : gb2;
          float2 xf, dc;
          const float2 xnew = coord_step(p, g2, xk, xp, gpv, lj, uj, bb, onepb, xf, dc);
          sx[(size_t)s * cps + c] = QP != kF32 ? xf : make_float2(xf.x, 0.0f);
          mbar_arrive(&xready[s]);
          xn[qj] = xnew;
          gc[qj] = g2;
          if (p.alg == kChambollePock) continue;
          dot = df2_add(dot, dc);
          if (want_eps && inf_j && nr > 0.0) {
            const double den = -wj - p.gamma_w * nr * p.t_norm;
            epsm = fmax(epsm, fmax(df2_to_double(g2) + eta_g * nr, 0.0) / den);
          }
        }
      }
      {
        const float2 o = make_float2(__shfl_down_sync(0xffffffffu, dot.x, 1), __shfl_down_sync(0xffffffffu, dot.y, 1));
        const double oe = __shfl_down_sync(0xffffffffu, epsm, 1);
        if (lane == 0) {
          dot = df2_add(dot, o);
          epsm = fmax(epsm, oe);
        }
      }
      if (lane == 0) {
        s_dot[dw] = dot;
        s_eps[dw] = epsm;
      }
    } else {
      // ------------------------------------------------------------ q warps
      const int qw = warp - 1 - DW;
      f32x2 qs[QT][2], qc[QT][2];
#pragma unroll
      for (int t = 0; t < QT; ++t)
#pragma unroll
        for (int c = 0; c < 2; ++c) qs[t][c] = qc[t][c] = 0ull;
      for (int g = 0; g < ngroups; ++g) {
        const int gg = it * ngroups + g;
        const int s = gg % nstages;
        const int u = gg / nstages;
        if (!warp_all(mbar_wait(&xready[s], u & 1) && mbar_wait(&full[s], u & 1))) {
          s_err = 1;
          break;
        }
        q_stage<QP, QT, QW>(qs, qc, stages + (size_t)s * stage_floats, sx + (size_t)s * cps,
                            min(cps, nq - g * cps), p.lda, qw, lane, m4q);
        __syncwarp();
        if (lane == 0) mbar_arrive(&empty[s]);
      }
      float2* part = b.qpart + (size_t)blockIdx.x * p.m4;
#pragma unroll
      for (int t = 0; t < QT; ++t) {
        const int c4 = qw * 32 + lane + t * 32 * QW;
        if (c4 < m4q) q_store<QP>(part, c4, qs[t], qc[t]);
      }
    }

    // ---- grid barrier 1: every CTA's q partials and restart terms are written
    consumer_sync<NCONS>();
    if (ct == 0) {
      float2 d = make_float2(0.f, 0.f);
      double e = 0.0;
      for (int w = 0; w < DW; ++w) {
        d = df2_add(d, s_dot[w]);
        if (gap_iter) e = fmax(e, s_eps[w]);
      }
      *reinterpret_cast<float2*>(&b.blk[4 * blockIdx.x + 0]) = d;   // restart term (double-float)
      b.blk[4 * blockIdx.x + 1] = e;                                 // translation step candidate
      if (s_err) atomicOr(&st->error, 1);
      bool ok = grid_count_sync(gcount, gbase + (unsigned long long)G * ++nbar, p.grid_wait);
      if (ok && *(volatile int*)&st->error) ok = false;
      s_ok = ok ? 1 : 0;
      if (!ok) atomicOr(&st->error, 1);
    }
    consumer_sync<NCONS>();
    if (!s_ok) break;

    // ---- residual slices r_{k+1} = y' - sum of the CTAs' partials (as k_resid); the last
    // warp meanwhile reduces the restart terms and prepares the next step's scalars
    bool scalars_done = false;
    auto scalars = [&]() {
      // the two possible next momentum entries (no restart / restart), loaded before the
      // reduction so their latency overlaps it
      const int ti_keep = s_ti + 1;
      MomEntry e_keep{}, e_rst{};
      if (lane == 0) {
        if (ti_keep < kMomTable) e_keep = p.mom[ti_keep];
        e_rst = p.mom[0];
      }
      // restart test: sign of sum_j g_v,j (x_{k+1,j} - x_{k,j}) over all CTAs, double-float
      float2 d = make_float2(0.f, 0.f);
      double e = 0.0;
      for (int t0 = 0; t0 < nparts; t0 += 256) {
        float2 dv[8];
        double ev[8];
#pragma unroll
        for (int kk = 0; kk < 8; ++kk) {
          const int t = t0 + lane + 32 * kk;
          dv[kk] = t < nparts ? __ldcg(reinterpret_cast<const float2*>(&b.blk[4 * t + 0])) : make_float2(0.f, 0.f);
          ev[kk] = (gap_iter && t < nparts) ? __ldcg(&b.blk[4 * t + 1]) : 0.0;
        }
#pragma unroll
        for (int kk = 0; kk < 8; ++kk) d = df2_add(d, dv[kk]);
        if (gap_iter)
          for (int kk = 0; kk < 8; ++kk) e = fmax(e, ev[kk]);
      }
#pragma unroll
      for (int o = 16; o > 0; o >>= 1)
        d = df2_add(d, make_float2(__shfl_xor_sync(0xffffffffu, d.x, o), __shfl_xor_sync(0xffffffffu, d.y, o)));
      if (gap_iter) e = warp_max_d(e);
      if (lane == 0) {
        const bool restart = p.restart && (d.x < 0.f || (d.x == 0.f && d.y < 0.f));
        const int ti = restart ? 0 : s_ti + 1;
        const double tnext = restart ? 1.0 : tn;
        s_ti = ti;
        s_tk = tnext;
        if (restart || ti_keep < kMomTable) {
          const MomEntry& me = restart ? e_rst : e_keep;
          s_tn = me.tn;
          s_beta2[0] = me.beta2;
          s_beta2[1] = me.onepb2;
        } else {
          momentum(p.mom, ti, tnext, &s_tn, s_beta2);   // past the table's end
        }
        if (blockIdx.x == 0) {
          st->t = tnext;
          st->ti = ti;
          if (gap_iter) st->eps = e;
          st->k = k + 1;
          st->sum_active += (double)n_act;
        }
      }
      scalars_done = true;
    };
    for (int sl = blockIdx.x; sl < nslices; sl += G) {
      const int row = sl * 32 + lane;
      float s = 0.f, c = 0.f;
      if (row < p.m4) {
        for (int t0 = wi; t0 < nparts; t0 += NW * 10) {
          float2 v[10];
#pragma unroll
          for (int kk = 0; kk < 10; ++kk) {
            const int t = t0 + NW * kk;
            v[kk] = t < nparts ? __ldcg(&b.qpart[(size_t)t * p.m4 + row]) : make_float2(0.f, 0.f);
          }
#pragma unroll
          for (int kk = 0; kk < 10; ++kk) df_add(s, c, v[kk].x, v[kk].y);
        }
      }
      s_red[wi][lane] = make_float2(s, c);
      consumer_sync<NCONS>();
      if (wi == 0) {
        for (int w = 1; w < NW; ++w) df_add(s, c, s_red[w][lane].x, s_red[w][lane].y);
        if (p.alg == kChambollePock) {
          double pv = 0.0, dv = 0.0, zv = 0.0;
          if (row < p.m) {
            const float2 q = df2_norm(s, c);
            const float2 yv = make_float2(b.yh[row], b.yl[row]);
            const float2 z = make_float2(__ldcg(b.rh + row), __ldcg(b.rl + row));
            const float2 r = make_float2(__ldcg(b.crh + row), __ldcg(b.crl + row));
            const float2 zn = df2_mul(df2_add(z, df2_mul(df2_sub(q, yv), p.sigma2)), p.inv1ps2);
            const float2 rn = df2_mul(df2_add(r, df2_sub(yv, q)), make_float2(0.5f, 0.f));
            b.rh[row] = zn.x;
            b.rl[row] = zn.y;
            b.crh[row] = rn.x;
            b.crl[row] = rn.y;
            const double rd = df2_to_double(rn), zd = df2_to_double(z);
            pv = 0.5 * rd * rd;
            dv = (zd + rd) * (zd + rd);
            zv = zd * zd;
          }
          pv = warp_sum_d(pv);
          dv = warp_sum_d(dv);
          zv = warp_sum_d(zv);
          if (lane == 0) {
            b.tileR[sl] = pv;
            b.tileD[sl] = dv;
            b.tileZ[sl] = zv;
          }
        } else {
          float ps = 0.f, pc = 0.f;
          if (row < p.m) {
            float dh, de;
            two_sum(b.yh[row], -s, dh, de);
            de += b.yl[row] - c;
            float rh, rl;
            two_sum(dh, de, rh, rl);
            b.rh[row] = rh;
            b.rl[row] = rl;
            const float sq = rh * rh;
            ps = 0.5f * sq;
            pc = 0.5f * (fmaf(rh, rh, -sq) + 2.0f * rh * rl);
          }
          for (int o = 16; o > 0; o >>= 1) {
            const float os = __shfl_xor_sync(0xffffffffu, ps, o);
            const float oc = __shfl_xor_sync(0xffffffffu, pc, o);
            df_add(ps, pc, os, oc);
          }
          if (lane == 0) b.tileR[sl] = df_to_double(ps, pc);
        }
      } else if (wi == NW - 1 && !scalars_done) {
        scalars();
      }
      consumer_sync<NCONS>();
    }
    if (wi == NW - 1 && !scalars_done) scalars();

    // ---- grid barrier 2: r_{k+1} and the P partials are written
    consumer_sync<NCONS>();
    if (ct == 0) {
      bool ok = grid_count_sync(gcount, gbase + (unsigned long long)G * ++nbar, p.grid_wait);
      if (ok && *(volatile int*)&st->error) ok = false;
      s_ok = ok ? 1 : 0;
      if (!ok) atomicOr(&st->error, 1);
    }
    consumer_sync<NCONS>();
    if (!s_ok) break;
  }
  // on an early exit the producer may be waiting for a stage no consumer will free: it stops
  // issuing and waits (bounded) for the copies it already issued before the CTA ends
  if (ct == 0 && !s_ok) s_stop = 1;
  // the count the next launch starts from (every CTA has read gbase before its first barrier)
  if (blockIdx.x == 0 && ct == 0 && s_ok) st->gbase = gbase + (unsigned long long)G * nbar;

  // the CTA's columns back to global memory (both slots of x and g)
  for (int q = ct; q < nq; q += NCONS) {
    const int j = sidx[q];
    b.x[0][j] = sX0[q];
    b.x[1][j] = sX1[q];
    b.g[0][j] = sG0[q];
    b.g[1][j] = sG1[q];
  }
}

__global__ void k_cp_init(Params p, Buffers b) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < p.m4; i += gridDim.x * blockDim.x) {
    const float rh = b.rh[i], rl = b.rl[i];
    b.crh[i] = rh;
    b.crl[i] = rl;
    b.rh[i] = -rh;
    b.rl[i] = -rl;
  }
}

cudaError_t launch_cp_init(const Params& p, const Buffers& b, cudaStream_t s) {
  k_cp_init<<<(p.m4 + 255) / 256, 256, 0, s>>>(p, b);
  return cudaGetLastError();
}

// x_out (float64) from the double-float iterate of the given slot.
__global__ void k_export(Params p, Buffers b, int slot) {
  for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < p.n; j += gridDim.x * blockDim.x)
    b.xout[j] = df2_to_double(b.x[slot][j]);
}

// Stage layout for the fused pass: up to 64 KB and 8 columns per stage (bulk copies much
// smaller than that are dominated by their fixed cost; measured on 2000-row columns, 8
// columns per stage beat 4, 2 and 1) and as many stages as fit.
// Returns the stage count (0 when the fused pass cannot be used) and the columns per stage.
// Float4 row chunks per q-warp lane for m4 rows (1, 2, 4 or 8; 0 if too many rows).
static int pass_qt(int m4) {
  const int m4q = m4 / 4;
  for (int qt = 1; qt <= kPassTmax; qt *= 2)
    if (m4q <= 32 * 8 * qt) return qt;
  return 0;
}

template <int PREC>
static cudaError_t pass_set_smem(int qt, int bytes) {
  switch (qt) {
    case 1: return cudaFuncSetAttribute(k_pass<PREC, 8, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
    case 2: return cudaFuncSetAttribute(k_pass<PREC, 8, 2>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
    case 4: return cudaFuncSetAttribute(k_pass<PREC, 8, 4>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
    default: return cudaFuncSetAttribute(k_pass<PREC, 8, 8>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
  }
}

int pass_configure(int lda, int m4, int idx_cap, int smem_optin, int* qwarps, int* cps_out) {
  const int qt = pass_qt(m4);
  if (qt == 0) return 0;
  const int col_bytes = lda * 4;
  // an even column count splits a stage into column pairs for the dot warps (measured on
  // 4000-row columns: 2 columns per stage 106 us, 3 columns 130-171 us per iteration)
  for (int cps = std::max(1, std::min(8, 65536 / col_bytes)); cps >= 1; --cps) {
    if (cps > 1 && cps % 2 != 0) continue;
    int ns = kPassMaxStages;
    // room for the kernels' static shared memory (the persistent form's is about 5 KB)
    while (ns >= 3 && pass_smem_bytes(lda, m4, ns, cps, idx_cap) + 8192 > (size_t)smem_optin) --ns;
    if (ns < 3) continue;
    const int bytes = (int)pass_smem_bytes(lda, m4, ns, cps, idx_cap);
    cudaError_t e = pass_set_smem<kX2>(qt, bytes);
    if (e == cudaSuccess) e = pass_set_smem<kF32>(qt, bytes);
    if (e == cudaSuccess) e = pass_set_smem<kMix>(qt, bytes);
    if (e != cudaSuccess) return 0;
    *qwarps = 8;
    *cps_out = cps;
    return ns;
  }
  return 0;
}

template <int PREC, int QT>
static void pass_launch_t(const Params& p, const Buffers& b, int slot, int g, int grid, int nstages, int cps,
                          size_t sm, cudaStream_t s) {
  k_pass<PREC, 8, QT><<<grid, 32 * (1 + kPassDot + 8), sm, s>>>(p, b, slot, g, nstages, cps);
}

template <int PREC>
static void pass_launch_p(int qt, const Params& p, const Buffers& b, int slot, int g, int grid, int nstages, int cps,
                          size_t sm, cudaStream_t s) {
  switch (qt) {
    case 1: pass_launch_t<PREC, 1>(p, b, slot, g, grid, nstages, cps, sm, s); break;
    case 2: pass_launch_t<PREC, 2>(p, b, slot, g, grid, nstages, cps, sm, s); break;
    case 4: pass_launch_t<PREC, 4>(p, b, slot, g, grid, nstages, cps, sm, s); break;
    default: pass_launch_t<PREC, 8>(p, b, slot, g, grid, nstages, cps, sm, s); break;
  }
}

cudaError_t launch_pass(const Params& p, const Buffers& b, int slot, int precision, bool gap_iter,
                        int grid, int nstages, int cps, int qwarps, cudaStream_t s) {
  const size_t sm = pass_smem_bytes(p.lda, p.m4, nstages, cps, (p.n + grid - 1) / grid);
  const int g = gap_iter ? 1 : 0;
  const int qt = pass_qt(p.m4);
  if (qwarps != 8 || qt == 0) return cudaErrorInvalidValue;
  switch (precision) {
    case kX2: pass_launch_p<kX2>(qt, p, b, slot, g, grid, nstages, cps, sm, s); break;
    case kF32: pass_launch_p<kF32>(qt, p, b, slot, g, grid, nstages, cps, sm, s); break;
    case kMix: pass_launch_p<kMix>(qt, p, b, slot, g, grid, nstages, cps, sm, s); break;
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

// Warp split of the persistent pass: DW dot warps (column pairs) and QW q warps (row
// slices of the forward product, QT float4 chunks per lane).
struct ItersShape {
  int dw, qw, qt;
};

static int iters_qt(int m4, int qw) {
  const int m4q = m4 / 4;
  for (int qt = 1; qt <= kPassTmax; qt *= 2)
    if (m4q <= 32 * qw * qt) return qt;
  return 0;
}

// 8 dot warps and 8 q warps in every mode.  (Mode MIXED used 4 + 16 while its forward
// product was double-float; with the float32 stage sums of q_stage the dot warps are the
// slower half, and 8 + 8 measured faster than 4 + 16, 8 + 16 and 12 + 8: 0.703 against
// 0.824 ms per solve of the 2000 x 10000 workload, 19.4 against 24.5 us per iteration of the
// 2000 x 10000 |N| one, 67.7 against 69.6 us on 4000 x 20000.)
static ItersShape iters_shape(int precision, int m4) {
  (void)precision;
  ItersShape sh{8, 8, 0};
  sh.qt = iters_qt(m4, sh.qw);
  return sh;
}

template <int PREC, int DW, int QW, int QT>
static const void* iters_fn() {
  return reinterpret_cast<const void*>(k_iters<PREC, DW, QW, QT>);
}

// The kernel of a shape, or null for a shape without an instantiation.
template <int PREC>
static const void* iters_kernel(const ItersShape& sh) {
  if (sh.dw == 8 && sh.qw == 8) {
    switch (sh.qt) {
      case 1: return iters_fn<PREC, 8, 8, 1>();
      case 2: return iters_fn<PREC, 8, 8, 2>();
      case 4: return iters_fn<PREC, 8, 8, 4>();
      case 8: return iters_fn<PREC, 8, 8, 8>();
    }
  }
  return nullptr;
}

static const void* iters_kernel_p(int precision, const ItersShape& sh) {
  switch (precision) {
    case kX2: return iters_kernel<kX2>(sh);
    case kF32: return iters_kernel<kF32>(sh);
    case kMix: return iters_kernel<kMix>(sh);
    default: return nullptr;
  }
}

cudaError_t launch_iters(const Params& p, const Buffers& b, int slot0, int niter, bool gap_last, int precision,
                         int grid, int nstages, int cps, int qwarps, cudaStream_t s) {
  const int idx_cap = iters_idx_cap(p.n, grid);
  const size_t sm = iters_smem_bytes(p.lda, p.m4, nstages, cps, idx_cap);
  const ItersShape sh = iters_shape(precision, p.m4);
  const void* fn = iters_kernel_p(precision, sh);
  if (qwarps != 8 || !fn || niter < 1 || b.gbar == nullptr || grid > kMaxGridFlags) return cudaErrorInvalidValue;
  int g = gap_last ? 1 : 0;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(grid);
  cfg.blockDim = dim3(32 * (1 + sh.dw + sh.qw));
  cfg.dynamicSmemBytes = sm;
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeCooperative;   // all CTAs co-resident (grid barriers)
  attr[0].val.cooperative = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  Params pp = p;
  Buffers bb = b;
  void* args[] = {&pp, &bb, &slot0, &niter, &g, &nstages, &cps, const_cast<int*>(&idx_cap)};
  return cudaLaunchKernelExC(&cfg, fn, args);
}

static bool iters_fits(int precision, int bytes, int grid, int m4) {
  const ItersShape sh = iters_shape(precision, m4);
  const void* fn = iters_kernel_p(precision, sh);
  if (!fn) return false;
  if (cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes) != cudaSuccess) return false;
  int per_sm = 0, dev = 0, sms = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, 32 * (1 + sh.dw + sh.qw), bytes) != cudaSuccess)
    return false;
  if (cudaGetDevice(&dev) != cudaSuccess) return false;
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return false;
  return per_sm >= 1 && grid <= per_sm * sms;
}

bool iters_configure(int lda, int m4, int nstages, int cps, int idx_cap, int grid) {
  if (nstages < 3 || grid > kMaxGridFlags) return false;
  const int bytes = (int)iters_smem_bytes(lda, m4, nstages, cps, idx_cap);
  return iters_fits(kX2, bytes, grid, m4) && iters_fits(kF32, bytes, grid, m4) && iters_fits(kMix, bytes, grid, m4);
}

cudaError_t launch_resid(const Params& p, const Buffers& b, int slot, int nparts, cudaStream_t s) {
  k_resid<<<(p.m4 + 31) / 32, 256, 0, s>>>(p, b, slot, nparts);
  return cudaGetLastError();
}

cudaError_t launch_export(const Params& p, const Buffers& b, int slot, cudaStream_t s) {
  k_export<<<std::min(1024, (p.n + 255) / 256), 256, 0, s>>>(p, b, slot);
  return cudaGetLastError();
}

}  // namespace bvls
