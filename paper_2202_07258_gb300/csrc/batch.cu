// Batched solver kernels: one shared A, B right-hand sides (see batch.cuh for the scheme).
//
//   k_bgram     H~ = bf16(A^T A), once per handle.
//   k_binit     x_0 = clip(x0, l, u) per instance, empty screened sets, t_0 = 1.
//   k_bstep     tcgen05 GEMM  G_tile = H~[coords, :] * D[instances, :]^T  (BF16 x BF16 -> FP32
//               in TMEM), then the FISTA step of Section 5 (accelerated) in the epilogue:
//               g_k = g_{k-1} - acc, g_v = (1 + b) g_k - b g_{k-1}, x_{k+1} = clip(v + g_v / L).
//   k_beval     per instance: r = y - A x_k (double-float), g = A^T r over the preserved
//               coordinates, the dual point (Eq. (BVLR_dual_up) / (BVLR_dual_up2)), the gap in
//               its nonnegative-sum form, the Gap safe radius (Eq. (GAP_Safe_sph)), the sphere
//               test (Eq. (safe_rule)), the stop test, and the step to x_{k+1} from the exact g.
//   k_bsteps    the K - 1 tensor-core steps between two evaluations in one launch of
//               clusters that keep x, g and the GEMM operand d on chip (npad <= 512).
//   k_bcompact  retires finished instances from the active list (stable).
#include <cuda_bf16.h>

#include "batch.cuh"
#include "common.cuh"
#include "f32x2.cuh"
#include "umma.cuh"

namespace bvls {

namespace {

constexpr unsigned kFull = 0xffffffffu;
constexpr int kStageBytes = 2 * kBTile * kBChunk * 2;  // A and B tiles of one K chunk (bf16)
constexpr int kBEvalList = 256;  // columns per chunk of the evaluation's nonzero lists
constexpr int kBEvalRows = 8;    // rows per lane and pass (256 rows) in the evaluation's A x
static_assert(kBEvalThreads / 32 == kBEvalInst, "one list-building warp per instance");

__device__ __forceinline__ double warp_sum_dd(double v) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(kFull, v, o);
  return v;
}

__device__ __forceinline__ double warp_max_dd(double v) {
  for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(kFull, v, o));
  return v;
}

// 4-byte asynchronous copy global -> shared (cp.async.ca)
// Dynamic shared memory of the evaluation, rows rounded up to 8 (mr), zero past m:
//   srh  [mr][kBEvalInst] residual, high parts   srl  [mr][kBEvalInst] low parts
//   s_fl [kBEvalInst][npad] flags                s_item [kBEvalInst][npad] coordinate lists
//   then, 16-byte aligned, phase 1's nonzero lists, which phase 2's copy ring reuses.
__host__ __device__ __forceinline__ size_t beval_lists_offset(int m, int npad) {
  const size_t mr = (size_t)((m + 7) & ~7);
  const size_t base = mr * kBEvalInst * 2 * sizeof(float) + (size_t)kBEvalInst * npad * (1 + sizeof(uint16_t));
  return (base + 15) & ~(size_t)15;
}

constexpr float kUf = 6.0e-8f;  // a little above 2^-24, the unit roundoff of float32

__device__ __forceinline__ float warp_sum_f(float v) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(kFull, v, o);
  return v;
}

// float32 value >= x
__device__ __forceinline__ float f32_up(double x) {
  float f = (float)x;
  if ((double)f < x) f = nextafterf(f, INFINITY);
  return f;
}

// Inputs of one gap term in float32: the distances to the bounds du = u_j - x_j (0 when
// u_j = +inf) and dl = x_j - l_j rounded up, gt = a_j^T theta = g_j + eps w_j, and the
// half-width E of an interval around gt that holds the exact value: the correlation's own
// error bound e plus the rounding of forming gt.
__device__ __forceinline__ void term_inputs_v(float2 xk, float2 g2, float2 l2, float2 u2, bool jinf, float wf,
                                              int dual_mode, float eps, float e, float& du, float& dl, float& gt,
                                              float& E) {
  const float2 a = df2_sub(xk, l2);
  dl = fmaxf(a.x + a.y, 0.f) * (1.f + 2.f * kUf);
  du = 0.f;
  if (!jinf) {
    const float2 c = df2_sub(u2, xk);
    du = fmaxf(c.x + c.y, 0.f) * (1.f + 2.f * kUf);
  }
  const float ew = dual_mode == kTranslation ? eps * wf : 0.f;
  gt = (g2.x + ew) + g2.y;
  E = e * (1.f + 2.f * kUf) + 8.f * kUf * (fabsf(g2.x) + fabsf(ew)) + fabsf(g2.y);
}

__device__ __forceinline__ void term_inputs(float2 xk, float2 g2, int j, const BParams& p, float eps, float e,
                                            float& du, float& dl, float& gt, float& E) {
  term_inputs_v(xk, g2, p.l2[j], p.u2[j], p.jinf[j] != 0, p.wf[j], p.dual_mode, eps, e, du, dl, gt, E);
}

// Upper bound of h(g') = du (g')^+ + dl (-g')^+ over |g' - gt| <= E, computed in float32:
// E is widened so that the rounded ends still enclose the interval, and the result is
// rounded up by the bound of the few operations that form it.
__device__ __forceinline__ float gap_term_up(float du, float dl, float gt, float E) {
  const float E2 = fmaf(4.f * kUf, fabsf(gt) + E, E) + 1e-30f;
  const float hi = gt + E2, lo = gt - E2;
  const float h_hi = du * fmaxf(hi, 0.f) + dl * fmaxf(-hi, 0.f);
  const float h_lo = du * fmaxf(lo, 0.f) + dl * fmaxf(-lo, 0.f);
  return fmaxf(h_hi, h_lo) * (1.f + 4.f * kUf) + 1e-30f;
}

// x_{k+1} = clip(x_k + b dk + g_v / L, l, u) with double-float iterates, dk = x_k - x_{k-1}
// (the evaluation passes it exactly; the tensor-core step passes bf16(x_k - x_{k-1}), the
// operand its Gram product already used).
__device__ __forceinline__ float2 fista_step(float2 xk, float2 dk, float gv, float be, float2 invL2, float2 l2,
                                             float2 u2) {
  const float2 v = df2_add(xk, df2_mul(dk, make_float2(be, 0.f)));
  float2 xn = df2_add(v, df2_mul(make_float2(gv, 0.f), invL2));
  if (df2_lt(xn, l2)) xn = l2;
  if (df2_lt(u2, xn)) xn = u2;
  return xn;
}

// Momentum of iteration k for one instance (Section 5, FISTA with gradient restart): T = t_k
// from tp = t_{k-1} and the restart-test sum of iteration k - 1; returns b = (t_k - 1) / t_{k+1}.
__device__ __forceinline__ float bstep_momentum(float tp, float dsum, int restart, float& T) {
  T = (restart && dsum < 0.f) ? 1.f : 0.5f * (1.f + sqrtf(1.f + 4.f * tp * tp));
  const float tn = 0.5f * (1.f + sqrtf(1.f + 4.f * T * T));
  return (T - 1.f) / tn;
}

// One (coordinate, instance) element of the tensor-core step: g_k = g_{k-1} - acc; for a
// preserved coordinate x_{k+1} = clip(x_k + delta, l, u) with g_v = (1 + b) g_k - b g_{k-1}
// and the increment delta = b d_k + g_v / L formed in float32 (its rounding error is
// relative to the increment, so it vanishes with it) and added to the double-float iterate
// by two TwoSums; d = x_{k+1} - x_k in float32 (delta, or the distance to the bound that
// clipped it).  A fixed coordinate keeps x_{k+1} = x_k, d = 0.  Returns the restart-test
// term g_v d.
__device__ __forceinline__ float bstep_elem(float gp, float acc, float2 xk, float dk, bool fixed, float be,
                                            float invLf, float2 lj, float2 uj, float& gk, float2& xn, float& dx) {
  gk = gp - acc;
  xn = xk;
  dx = 0.f;
  if (fixed) return 0.f;
  const float gv = fmaf(be, gk - gp, gk);
  const float delta = fmaf(gv, invLf, be * dk);
  float s, e, h, l;
  two_sum(xk.x, delta, s, e);
  two_sum(s, e + xk.y, h, l);
  xn = make_float2(h, l);
  dx = delta;
  if (df2_lt(xn, lj)) {
    xn = lj;
    dx = (lj.x - xk.x) + (lj.y - xk.y);
  } else if (df2_lt(uj, xn)) {
    xn = uj;
    dx = (uj.x - xk.x) + (uj.y - xk.y);
  }
  return gv * dx;
}

// bstep_elem for two instance columns of one coordinate, the float32 operations of both on
// packed f32x2 instructions (each lane rounds as the scalar instruction; the products are
// formed as fma(a, b, -0), which rounds as a*b and keeps its sign) and the clip per lane.
// Inputs are bit patterns (TMEM words): g_{k-1}, acc, x high and x low of columns 0 and 1.
// The fixed and inactive cases are left to the caller.
__device__ __forceinline__ void bstep_pair(uint32_t gp0, uint32_t gp1, uint32_t ac0, uint32_t ac1, uint32_t xh0,
                                           uint32_t xh1, uint32_t xl0, uint32_t xl1, float dk0, float dk1,
                                           float be0, float be1, float invLf, float2 lj, float2 uj, float (&gk)[2],
                                           float2 (&xn)[2], float (&dx)[2], float (&dv)[2]) {
  constexpr f32x2 kNegZero = 0x8000000080000000ull;
  const f32x2 gp = x2_pack(__uint_as_float(gp0), __uint_as_float(gp1));
  const f32x2 ac = x2_pack(__uint_as_float(ac0), __uint_as_float(ac1));
  const f32x2 xh = x2_pack(__uint_as_float(xh0), __uint_as_float(xh1));
  const f32x2 xl = x2_pack(__uint_as_float(xl0), __uint_as_float(xl1));
  const f32x2 be = x2_pack(be0, be1);
  const f32x2 gk2 = x2_sub(gp, ac);
  const f32x2 gv = x2_fma(be, x2_sub(gk2, gp), gk2);
  const f32x2 delta = x2_fma(gv, x2_pack(invLf, invLf), x2_fma(be, x2_pack(dk0, dk1), kNegZero));
  // two TwoSums: (s, e) = xh + delta, (h, l) = s + (e + xl)
  const f32x2 s = x2_add(xh, delta);
  f32x2 bb = x2_sub(s, xh);
  const f32x2 e = x2_add(x2_sub(xh, x2_sub(s, bb)), x2_sub(delta, bb));
  const f32x2 e2 = x2_add(e, xl);
  const f32x2 h = x2_add(s, e2);
  bb = x2_sub(h, s);
  const f32x2 l = x2_add(x2_sub(s, x2_sub(h, bb)), x2_sub(e2, bb));
  float hv[2], lv[2], dl[2];
  x2_unpack(h, hv[0], hv[1]);
  x2_unpack(l, lv[0], lv[1]);
  x2_unpack(delta, dl[0], dl[1]);
  x2_unpack(gk2, gk[0], gk[1]);
  const float2 xk[2] = {make_float2(__uint_as_float(xh0), __uint_as_float(xl0)),
                        make_float2(__uint_as_float(xh1), __uint_as_float(xl1))};
#pragma unroll
  for (int t = 0; t < 2; ++t) {
    xn[t] = make_float2(hv[t], lv[t]);
    dx[t] = dl[t];
    if (df2_lt(xn[t], lj)) {
      xn[t] = lj;
      dx[t] = (lj.x - xk[t].x) + (lj.y - xk[t].y);
    } else if (df2_lt(uj, xn[t])) {
      xn[t] = uj;
      dx[t] = (uj.x - xk[t].x) + (uj.y - xk[t].y);
    }
  }
  const f32x2 d = x2_fma(gv, x2_pack(dx[0], dx[1]), kNegZero);
  x2_unpack(d, dv[0], dv[1]);
}

// Column sums over the 32 lanes of v[0..15] (v is overwritten): lanes c and c + 16 return the
// sum of column c (a transposed butterfly, 16 shuffles).
__device__ __forceinline__ float lane_sums16(float (&v)[16], int lane) {
#pragma unroll
  for (int o = 8; o >= 1; o >>= 1) {
    const bool up = (lane & o) != 0;
#pragma unroll
    for (int t = 0; t < o; ++t) {
      const float send = up ? v[t] : v[t + o];
      const float keep = up ? v[t + o] : v[t];
      v[t] = keep + __shfl_xor_sync(kFull, send, o);
    }
  }
  return v[0] + __shfl_xor_sync(kFull, v[0], 16);
}

}  // namespace

// ------------------------------------------------------------------ Gram matrix
// H[i][j] = sum_r A[r][i] A[r][j] in float32 (32 x 32 output tile per block), stored as
// bf16, row-major with pitch npad, zero outside n x n.
__global__ void __launch_bounds__(256) k_bgram(const float* __restrict__ A, int lda, int m, int n, int npad,
                                               __nv_bfloat16* __restrict__ H) {
  __shared__ float si[32][33];
  __shared__ float sj[32][33];
  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
  const int i0 = blockIdx.y * 32, j0 = blockIdx.x * 32;
  float acc[4] = {0.f, 0.f, 0.f, 0.f};
  for (int r0 = 0; r0 < m; r0 += 32) {
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int c = ty + 8 * q;
      const int r = r0 + tx;
      si[c][tx] = (i0 + c < n && r < m) ? A[(size_t)(i0 + c) * lda + r] : 0.f;
      sj[c][tx] = (j0 + c < n && r < m) ? A[(size_t)(j0 + c) * lda + r] : 0.f;
    }
    __syncthreads();
#pragma unroll 8
    for (int rr = 0; rr < 32; ++rr) {
      const float bj = sj[tx][rr];
#pragma unroll
      for (int q = 0; q < 4; ++q) acc[q] = fmaf(si[ty + 8 * q][rr], bj, acc[q]);
    }
    __syncthreads();
  }
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    const int i = i0 + ty + 8 * q, j = j0 + tx;
    if (i < npad && j < npad) H[(size_t)i * npad + j] = __float2bfloat16_rn((i < n && j < n) ? acc[q] : 0.f);
  }
}

cudaError_t launch_bgram(const float* A, int lda, int m, int n, int npad, __nv_bfloat16* H, cudaStream_t s) {
  dim3 grid(npad / 32, npad / 32);
  k_bgram<<<grid, 256, 0, s>>>(A, lda, m, n, npad, H);
  return cudaGetLastError();
}

// ------------------------------------------------------------------ initial state
__global__ void k_binit(BParams p, BBuffers b) {
  const size_t total = (size_t)p.B * p.npad;
  const int MT = p.npad / kBTile;
  int bad = 0;
  for (size_t idx = (size_t)blockIdx.x * blockDim.x + threadIdx.x; idx < total;
       idx += (size_t)gridDim.x * blockDim.x) {
    const int inst = (int)(idx / p.npad), j = (int)(idx % p.npad);
    float2 xf = make_float2(0.f, 0.f);
    if (j < p.n) {
      double x = 0.0;
      if (b.X0) {
        x = b.X0[(size_t)inst * p.n + j];
        if (!isfinite(x)) {
          bad = 1;
          x = 0.0;
        }
      }
      x = fmin(fmax(x, p.l[j]), p.u[j]);   // x_0 = clip(x0, l, u)
      xf = df2_from_double(x);
      if (df2_lt(xf, p.l2[j])) xf = p.l2[j];
      if (df2_lt(p.u2[j], xf)) xf = p.u2[j];
    }
    b.X[0][idx] = xf;
    b.X[1][idx] = xf;
    b.G[0][idx] = 0.f;
    b.G[1][idx] = 0.f;
    b.D[0][idx] = __float2bfloat16_rn(0.f);
    b.D[1][idx] = __float2bfloat16_rn(0.f);
    b.flags[idx] = 0;
  }
  for (size_t idx = (size_t)blockIdx.x * blockDim.x + threadIdx.x; idx < (size_t)p.B * p.m;
       idx += (size_t)gridDim.x * blockDim.x) {
    const int inst = (int)(idx / p.m), i = (int)(idx % p.m);
    if (!isfinite(b.Y[(size_t)inst * p.lda + i])) bad = 1;
  }
  for (int q = blockIdx.x * blockDim.x + threadIdx.x; q < p.npad; q += gridDim.x * blockDim.x) {
    b.D[0][(size_t)p.B * p.npad + q] = __float2bfloat16_rn(0.f);
    b.D[1][(size_t)p.B * p.npad + q] = __float2bfloat16_rn(0.f);
  }
  for (int q = blockIdx.x * blockDim.x + threadIdx.x; q < p.B; q += gridDim.x * blockDim.x) {
    b.tval[0][q] = 1.f;
    b.tval[1][q] = 1.f;
    b.act[q] = q;
    b.fin[q] = 0;
    for (int t = 0; t < MT; ++t) {
      b.dotp[0][(size_t)t * p.B + q] = 0.f;
      b.dotp[1][(size_t)t * p.B + q] = 0.f;
    }
  }
  if (bad) atomicOr(&b.st->nonfinite, 1);
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    b.st->n_act = p.B;
    if (b.st->nonfinite) b.st->done = 1;
  }
}

cudaError_t launch_binit(const BParams& p, const BBuffers& b, cudaStream_t s) {
  const size_t total = (size_t)p.B * p.npad;
  const int blocks = (int)std::min<size_t>((total + 255) / 256, 4096);
  k_binit<<<blocks, 256, 0, s>>>(p, b);
  return cudaGetLastError();
}

// ------------------------------------------------------------------ tensor-core step
// Grid (npad / 128 coordinate tiles, ceil(B / 128) instance tiles), 512 threads, one CTA per
// SM (128 KB of stages).  Operand K chunks of 64 stream through kBStages shared-memory
// stages in the 128-byte swizzled K-major layout, synchronised by mbarriers only.  Into a
// free stage thread 0 issues one tensor copy of the 64 x 128 box of H~ (16 KB of
// transaction bytes on the stage's full barrier) and warps 0-3 copy the D rows of the tile's
// 128 instances (gathered by the active list) with 16-byte cp.async into their swizzled
// places, wait for their own copies, fence them to the async proxy and arrive on the full
// barrier; lane 0 of warp 4 waits for it, issues four 128x128x16 MMAs and commits them to
// the stage's empty barrier, which frees the stage for the chunk kBStages later, and after
// the last chunk to the done barrier.  Meanwhile the other warps load their first epilogue
// operands; then all 16 read the accumulator rows of their 32 coordinates from TMEM.
// (Measured on the 4096 x (224 x 512) batch: cp.async moved each operand at ~17 bytes per
// clock per SM; D as 32 four-row tensor gathers per chunk from one thread was slower still.)
__global__ void __launch_bounds__(kBStepThreads, 1) k_bstep(const __grid_constant__ BParams p, BBuffers b, int jrel) {
  BState* st = b.st;
  if (st->done) return;
  const int n_act = st->n_act;
  const int mt = blockIdx.x, nt = blockIdx.y;
  if (nt * kBTile >= n_act) return;
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  // the swizzle atoms must start on 1024-byte boundaries (the launch adds 1 KB of slack)
  unsigned char* smem = smem_raw + ((1024u - (smem_u32(smem_raw) & 1023u)) & 1023u);
  __shared__ __align__(8) uint64_t full[kBStages], empty[kBStages], done;
  __shared__ uint32_t s_tmem;
  __shared__ int s_inst[kBTile];
  __shared__ float s_beta[kBTile];
  __shared__ float2 s_l[kBTile], s_u[kBTile];
  __shared__ float s_dot[4][kBTile];   // [TMEM lane quarter][instance column]

  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int k = st->kbase + jrel;
  const int s = k & 1;
  const int MT = p.npad / kBTile;
  if (tid < kBTile) {
    // momentum parameter of this iteration for instance column tid (Section 5, FISTA with
    // gradient restart): t_k from t_{k-1} and the restart test of iteration k-1
    const int q = nt * kBTile + tid;
    const int inst = q < n_act ? b.act[q] : -1;
    s_inst[tid] = inst;
    float beta = 0.f;
    if (inst >= 0) {
      const float tp = b.tval[s ^ 1][inst];
      float dsum = 0.f;
      for (int t = 0; t < MT; ++t) dsum += b.dotp[s ^ 1][(size_t)t * p.B + inst];
      float T;
      beta = bstep_momentum(tp, dsum, p.restart, T);
      if (mt == 0) b.tval[s][inst] = T;
    }
    s_beta[tid] = beta;
    const int jj = mt * kBTile + tid;
    s_l[tid] = jj < p.n ? p.l2[jj] : make_float2(0.f, 0.f);
    s_u[tid] = jj < p.n ? p.u2[jj] : make_float2(0.f, 0.f);
  }
  if (warp == 0) tmem_alloc(&s_tmem, kBTile);
  if (tid == 0) {
    for (int q = 0; q < kBStages; ++q) {
      mbar_init(&full[q], kBCopyWarps * 32 + 1);  // the copy threads and the tensor copy's expect-tx
      mbar_init(&empty[q], 1);
    }
    mbar_init(&done, 1);
    fence_barrier_init();
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = s_tmem;

  const int nch = p.npad / kBChunk;
  bool ok = true;
  if (warp < kBCopyWarps) {
    // producers: chunk c into stage c % kBStages once the MMAs of chunk c - kBStages are done
    const __nv_bfloat16* Dsrc = b.D[s];
    constexpr int NPT = kBCopyWarps * 32;
    auto load_chunk = [&](int c) {
      const int st_ = c % kBStages;
      unsigned char* sa = smem + (size_t)st_ * kStageBytes;
      unsigned char* sb = sa + kStageBytes / 2;
      const int kofs = c * kBChunk;
      if (tid == 0) {
        mbar_arrive_expect_tx(&full[st_], (uint32_t)(kStageBytes / 2));
        tma_load_2d(sa, &p.tmH, kofs, mt * kBTile, &full[st_]);
      }
#pragma unroll
      for (int t = 0; t < (kBTile * 8) / NPT; ++t) {
        const int q = tid + t * NPT;
        const int r = q >> 3, kc = q & 7;   // row r, 16-byte chunk kc of its 128-byte K segment
        const int inst = s_inst[r];
        const int row = inst >= 0 ? inst : p.B;  // row B of D is zero
        cp_async16(sb + r * 128 + ((kc ^ (r & 7)) << 4), Dsrc + (size_t)row * p.npad + kofs + kc * 8);
      }
      cp_async_commit();
    };
    static_assert(kBStages == 4, "the drain below waits on up to kBStages - 2 newer groups");
    for (int c = 0; c < nch; ++c) {
      if (c >= kBStages && !mbar_wait(&empty[c % kBStages], ((c / kBStages) - 1) & 1)) ok = false;
      load_chunk(c);
      if (c >= kBStages - 1) {  // chunk c - kBStages + 1 has landed: announce it
        cp_async_wait<kBStages - 1>();
        fence_proxy_async_smem();
        mbar_arrive(&full[(c - kBStages + 1) % kBStages]);
      }
    }
    for (int c = nch - kBStages + 1 > 0 ? nch - kBStages + 1 : 0; c < nch; ++c) {
      const int newer = nch - 1 - c;
      if (newer >= 2) cp_async_wait<2>();
      else if (newer == 1) cp_async_wait<1>();
      else cp_async_wait<0>();
      fence_proxy_async_smem();
      mbar_arrive(&full[c % kBStages]);
    }
  } else if (warp == kBCopyWarps) {
    // MMA issuer: the warp waits for each stage, lane 0 issues and commits
    const uint32_t idesc = umma_idesc_bf16(kBTile, kBTile);
    for (int c = 0; c < nch; ++c) {
      if (!mbar_wait(&full[c % kBStages], (c / kBStages) & 1)) ok = false;
      tc_fence_after();
      if (lane == 0) {
        const uint32_t sa = smem_u32(smem + (size_t)(c % kBStages) * kStageBytes);
        const uint32_t sb = sa + kStageBytes / 2;
#pragma unroll
        for (int kk = 0; kk < kBChunk / 16; ++kk)
          umma_bf16(tmem, umma_smem_desc_sw128(sa + kk * 32), umma_smem_desc_sw128(sb + kk * 32), idesc,
                    c > 0 || kk > 0);
        umma_commit(&empty[c % kBStages]);
      }
      __syncwarp();
    }
    if (lane == 0) umma_commit(&done);
    __syncwarp();
  }

  // epilogue: warp w reads TMEM lane quarter w % 4 (coordinates) and instance columns
  // [32 (w / 4), 32 (w / 4) + 32); thread = coordinate jg
  const int quarter = warp & 3;
  const int i = quarter * 32 + lane;
  const int jg = mt * kBTile + i;
  const bool jv = jg < p.n;
  const float2 lj = s_l[i], uj = s_u[i];
  const float invLf = p.invL2.x;
  const float* __restrict__ Gp = b.G[s ^ 1];
  float* Gc = b.G[s];
  const float2* __restrict__ Xc = b.X[s];
  const __nv_bfloat16* __restrict__ Dk = b.D[s];   // bf16(x_k - x_{k-1}): the momentum's difference
  float2* Xn = b.X[s ^ 1];                         // x_{k+1} replaces x_{k-1}, which is not read
  __nv_bfloat16* Dn = b.D[s ^ 1];
  static_assert(kBTile / (kBStepThreads / 128) == 32, "one 32-column group of instances per warp");
  const int c0 = (warp >> 2) * 32;
  const bool have = s_inst[c0] >= 0;  // active instances are packed at the front of the tile
  float gp[8];
  float2 xk[8];
  __nv_bfloat16 dk[8];
  uint8_t fl[8];
  auto load8 = [&](int c8) {  // eight instances' operands in flight
#pragma unroll
    for (int cc = 0; cc < 8; ++cc) {
      const int inst = s_inst[c0 + c8 + cc];
      gp[cc] = 0.f;
      xk[cc] = make_float2(0.f, 0.f);
      dk[cc] = __float2bfloat16_rn(0.f);
      fl[cc] = 1;
      if (inst >= 0 && jv) {
        const size_t o = (size_t)inst * p.npad + jg;
        gp[cc] = Gp[o];
        xk[cc] = Xc[o];
        dk[cc] = Dk[o];
        fl[cc] = b.flags[o];
      }
    }
  };
  if (have) load8(0);  // while the MMAs run
  if (!mbar_wait(&done, 0)) ok = false;
  __syncwarp();
  tc_fence_after();
  if (have) {
    float acc[32];
    tmem_ld32(tmem + ((uint32_t)(quarter * 32) << 16) + (uint32_t)c0, acc);
#pragma unroll
    for (int h = 0; h < 32; h += 16) {
      float dv[16];
#pragma unroll
      for (int c8 = 0; c8 < 16; c8 += 8) {
        if (h + c8 > 0) load8(h + c8);
#pragma unroll
        for (int cc = 0; cc < 8; ++cc) {
          const int inst = s_inst[c0 + h + c8 + cc];
          dv[c8 + cc] = 0.f;
          if (inst >= 0 && jv) {
            const size_t o = (size_t)inst * p.npad + jg;
            float gk, dx;
            float2 xn;
            dv[c8 + cc] = bstep_elem(gp[cc], acc[h + c8 + cc], xk[cc], __bfloat162float(dk[cc]), fl[cc] != 0,
                                     s_beta[c0 + h + c8 + cc], invLf, lj, uj, gk, xn, dx);
            Gc[o] = gk;
            Xn[o] = xn;
            Dn[o] = __float2bfloat16_rn(dx);
          }
        }
      }
      // restart-test partials of the warp's 32 coordinates for instance columns c0 + h + (0..15)
      const float sum = lane_sums16(dv, lane);
      if (lane < 16) s_dot[quarter][c0 + h + lane] = sum;
    }
  }
  tc_fence_before();
  __syncthreads();
  if (tid < kBTile) {
    const int inst = s_inst[tid];
    if (inst >= 0) b.dotp[s][(size_t)mt * p.B + inst] = s_dot[0][tid] + s_dot[1][tid] + s_dot[2][tid] + s_dot[3][tid];
  }
  if (warp == 0) tmem_dealloc(tmem, kBTile);
  if (!ok) atomicOr(&st->error, 1);
  if (tid == 0 && mt == 0 && nt == 0) st->sum_step += (double)n_act;
}

size_t bstep_smem_bytes() { return (size_t)kBStages * kStageBytes + 1024; }

cudaError_t launch_bstep(const BParams& p, const BBuffers& b, int j, cudaStream_t s) {
  dim3 grid(p.npad / kBTile, (p.B + kBTile - 1) / kBTile);
  k_bstep<<<grid, kBStepThreads, bstep_smem_bytes(), s>>>(p, b, j);
  return cudaGetLastError();
}

// ------------------------------------------------------------------ persistent tensor-core steps
// The run of tensor-core steps between two evaluations in one launch, with the iteration
// state on chip.  A cluster of MT = npad / 128 CTAs (MT <= 4) covers one tile of 128
// instances: CTA mt owns coordinates [128 mt, 128 mt + 128) of them.  Per CTA:
//   TMEM    512 columns: the accumulator [0, 128), x_k as high and low float32 parts
//           [128, 384), g_{k-1} [384, 512); lane = coordinate, column = instance.
//   shared  the whole B operand d_k = bf16(x_k - x_{k-1}) of the tile's instances (npad / 64
//           swizzled K chunks of 16 KB) and a ring of kBPStages 16 KB chunks of H~ (tensor
//           copies, as in k_bstep).
// A step k: the MMA lane waits for the peers' slices of d_k (one dfull phase per step),
// issues the products over all K chunks in k_bstep's order and commits; the 16 warps run
// k_bstep's element arithmetic on TMEM (bstep_pair: the same operations, two instance
// columns per packed instruction), park the new d in the accumulator's columns and send
// their restart-test partials into every CTA's shared memory; a cluster barrier (every
// CTA has finished the products that read d_k, so also every copy of d_k, and the partials
// have landed); each CTA writes d_{k+1} into its own slice of the B operand, sums the
// partials into the next momentum and pushes the 32 KB slice into each peer with one bulk
// copy, completing on the peer's dfull barrier.  Every copy is issued unconditionally and
// awaited by its receiver before the receiver's next cluster barrier, so no CTA leaves while
// a peer may still write to it; every wait is bounded.  The last step leaves g, x, dotp and
// tval in global memory and the one before it x: everything the evaluation that follows
// reads (it rewrites d itself).
constexpr int kBPStages = 4;
constexpr int kBPMaxTiles = 4;
constexpr int kChunkBytes = kBTile * 128;        // one K chunk of 64 bf16 for 128 rows
constexpr int kSliceBytes = 2 * kChunkBytes;     // a CTA's 128 coordinates of d: two K chunks
constexpr uint32_t kTmX = 128, kTmXl = 256, kTmG = 384;

__global__ void __launch_bounds__(kBStepThreads, 1)
    k_bsteps(const __grid_constant__ BParams p, BBuffers b, int j0, int nsteps) {
  BState* st = b.st;
  if (st->done) return;
  const int n_act = st->n_act;
  const int mt = blockIdx.x, nt = blockIdx.y;  // the cluster spans blockIdx.x
  if (nt * kBTile >= n_act) return;            // uniform over the cluster
  const int MT = p.npad / kBTile;
  const int nch = p.npad / kBChunk;
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  unsigned char* smem = smem_raw + ((1024u - (smem_u32(smem_raw) & 1023u)) & 1023u);
  unsigned char* sD = smem;                                // nch chunks: the B operand
  unsigned char* sH = smem + (size_t)nch * kChunkBytes;    // kBPStages chunks of H~
  __shared__ __align__(8) uint64_t full[kBPStages], empty[kBPStages], done, dfull;
  __shared__ uint32_t s_tmem;
  __shared__ int s_inst[kBTile];
  __shared__ __align__(16) float s_beta[kBTile];
  __shared__ float s_tval[kBTile];
  __shared__ float2 s_l[kBTile], s_u[kBTile];
  __shared__ float s_dot[4][kBTile];
  __shared__ float s_part[2][kBPMaxTiles][kBTile];     // [step parity][coordinate tile][instance column]
  __shared__ __align__(16) uint32_t s_fix[4][kBTile];  // bit `lane` of [quarter][column]: fixed coordinate

  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int kb = st->kbase + j0;  // iteration of the first step
  if (tid < kBTile) {
    const int q = nt * kBTile + tid;
    const int inst = q < n_act ? b.act[q] : -1;
    s_inst[tid] = inst;
    float beta = 0.f, T = 1.f;
    if (inst >= 0) {
      const int s = kb & 1;
      const float tp = b.tval[s ^ 1][inst];
      float dsum = 0.f;
      for (int t = 0; t < MT; ++t) dsum += b.dotp[s ^ 1][(size_t)t * p.B + inst];
      beta = bstep_momentum(tp, dsum, p.restart, T);
      if (mt == 0 && nsteps == 1) b.tval[s][inst] = T;
    }
    s_beta[tid] = beta;
    s_tval[tid] = T;
    const int jj = mt * kBTile + tid;
    s_l[tid] = jj < p.n ? p.l2[jj] : make_float2(0.f, 0.f);
    s_u[tid] = jj < p.n ? p.u2[jj] : make_float2(0.f, 0.f);
  }
  if (warp == 0) tmem_alloc(&s_tmem, 512);
  if (tid == 0) {
    for (int q = 0; q < kBPStages; ++q) {
      mbar_init(&full[q], 1);
      mbar_init(&empty[q], 1);
    }
    mbar_init(&done, 1);
    mbar_init(&dfull, 1);
    fence_barrier_init();
  }
  __syncthreads();  // s_inst
  {
    // d_k of the tile's instances (row B of D is zero) into the swizzled B operand
    const __nv_bfloat16* Dsrc = b.D[kb & 1];
    const int units = kBTile * 8 * nch;
    for (int q = tid; q < units; q += kBStepThreads) {
      const int c = q >> 10, rem = q & 1023;
      const int r = rem >> 3, kc = rem & 7;
      const int inst = s_inst[r];
      const int row = inst >= 0 ? inst : p.B;
      cp_async16(sD + (size_t)c * kChunkBytes + r * 128 + ((kc ^ (r & 7)) << 4),
                 Dsrc + (size_t)row * p.npad + c * kBChunk + kc * 8);
    }
    cp_async_commit();
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = s_tmem;
  const int quarter = warp & 3;
  const int i = quarter * 32 + lane;
  const int jg = mt * kBTile + i;
  const bool jv = jg < p.n;
  const int c0 = (warp >> 2) * 32;
  const bool have = s_inst[c0] >= 0;  // active instances are packed at the front of the tile
  const uint32_t tl = tmem + ((uint32_t)(quarter * 32) << 16);
  // this thread's coordinate in row c0 + cc of the B operand (c0 is a multiple of 8, so the
  // swizzle term depends on cc only)
  const int kin = i & 63;
  unsigned char* const drow = sD + (size_t)(2 * mt + (i >> 6)) * kChunkBytes + (size_t)c0 * 128 + (kin & 7) * 2;
  auto dptr = [&](int cc) {
    return reinterpret_cast<__nv_bfloat16*>(drow + cc * 128 + ((((kin >> 3) ^ (cc & 7))) << 4));
  };
  const int nat = min(kBTile, n_act - nt * kBTile);  // active instance columns of the tile
  if (have) {
    // x_k and g_{k-1} into TMEM, fixed flags into bits
    const float2* __restrict__ X0 = b.X[kb & 1];
    const float* __restrict__ G0 = b.G[(kb & 1) ^ 1];
#pragma unroll
    for (int h = 0; h < 32; h += 16) {
      float xh[16], xl[16], gg[16];
#pragma unroll
      for (int cc = 0; cc < 16; ++cc) {
        const int inst = s_inst[c0 + h + cc];
        float2 x = make_float2(0.f, 0.f);
        float g = 0.f;
        uint8_t f = 1;
        if (inst >= 0 && jv) {
          const size_t o = (size_t)inst * p.npad + jg;
          x = X0[o];
          g = G0[o];
          f = b.flags[o];
        }
        xh[cc] = x.x;
        xl[cc] = x.y;
        gg[cc] = g;
        const uint32_t w = __ballot_sync(kFull, f != 0);
        if (lane == 0) s_fix[quarter][c0 + h + cc] = w;
      }
      tmem_st16(tl + kTmX + (uint32_t)(c0 + h), xh);
      tmem_st16(tl + kTmXl + (uint32_t)(c0 + h), xl);
      tmem_st16(tl + kTmG + (uint32_t)(c0 + h), gg);
    }
    tmem_wait_st();
  }
  cp_async_wait<0>();
  fence_proxy_async_smem();
  tc_fence_before();
  __syncthreads();
  cluster_sync_all();  // every CTA of the cluster runs and has initialised its barriers
  tc_fence_after();

  const float2 lj = s_l[i], uj = s_u[i];
  const float invLf = p.invL2.x;
  const int total = nsteps * nch;  // H~ chunks over the launch
  int issued = 0;
  bool ok = true;
  auto produce = [&](int lim) {  // thread 0: H~ chunks into the ring up to chunk lim - 1
    for (; issued < lim; ++issued) {
      const int stg = issued % kBPStages;
      if (issued >= kBPStages && !mbar_wait(&empty[stg], ((issued / kBPStages) - 1) & 1)) ok = false;
      mbar_arrive_expect_tx(&full[stg], (uint32_t)kChunkBytes);
      tma_load_2d(sH + (size_t)stg * kChunkBytes, &p.tmH, (issued % nch) * kBChunk, mt * kBTile, &full[stg]);
    }
  };
  if (tid == 0) produce(total < kBPStages ? total : kBPStages);
  const uint32_t idesc = umma_idesc_bf16(kBTile, kBTile);
  const size_t own = (size_t)mt * kSliceBytes;

  for (int q = 0; q < nsteps; ++q) {
    const int k = kb + q, s = k & 1;
    const bool wr = q >= nsteps - 2;
    const bool last = q == nsteps - 1;
    if (warp == kBCopyWarps) {
      if (lane == 0) {
        if (q > 0 && MT > 1) {
          // the peers' slices of d_k
          mbar_arrive_expect_tx(&dfull, (uint32_t)((MT - 1) * kSliceBytes));
          if (!mbar_wait_cluster(&dfull, (q - 1) & 1)) ok = false;
        }
        for (int c = 0; c < nch; ++c) {
          const int g = q * nch + c, stg = g % kBPStages;
          if (!mbar_wait(&full[stg], (g / kBPStages) & 1)) ok = false;
          tc_fence_after();
          const uint32_t sa = smem_u32(sH + (size_t)stg * kChunkBytes);
          const uint32_t sb = smem_u32(sD + (size_t)c * kChunkBytes);
#pragma unroll
          for (int kk = 0; kk < kBChunk / 16; ++kk)
            umma_bf16(tmem, umma_smem_desc_sw128(sa + kk * 32), umma_smem_desc_sw128(sb + kk * 32), idesc,
                      c > 0 || kk > 0);
          umma_commit(&empty[stg]);
        }
        umma_commit(&done);
      }
      __syncwarp();
    } else if (warp == 0) {
      if (lane == 0) {
        const int lim = (q + 1) * nch + kBPStages;
        produce(lim < total ? lim : total);
      }
      __syncwarp();
    }

    // epilogue (bstep_elem's arithmetic, two instance columns per packed instruction):
    // thread = coordinate jg, instance columns c0 .. c0 + 31 in four groups of eight; the TMEM
    // loads of group g + 1 are in flight while group g is computed
    if (!mbar_wait(&done, q & 1)) ok = false;
    __syncwarp();
    tc_fence_after();
    if (have) {
      float* __restrict__ Gc = b.G[s];
      float2* __restrict__ Xn = b.X[s ^ 1];
      uint32_t R[2][4][8];  // [group parity][accumulator, g, x high, x low][column]
      auto load_group = [&](int g, uint32_t (&r)[4][8]) {
        const uint32_t cb = (uint32_t)(c0 + 8 * g);
        tmem_ld8_nw(tl + cb, r[0]);
        tmem_ld8_nw(tl + kTmG + cb, r[1]);
        tmem_ld8_nw(tl + kTmX + cb, r[2]);
        tmem_ld8_nw(tl + kTmXl + cb, r[3]);
      };
      load_group(0, R[0]);
      float dv[16];
#pragma unroll
      for (int g = 0; g < 4; ++g) {
        uint32_t (&r)[4][8] = R[g & 1];
        tmem_wait_ld8(r[0]);
        tmem_wait_ld8(r[1]);
        tmem_wait_ld8(r[2]);
        tmem_wait_ld8(r[3]);
        if (g < 3) load_group(g + 1, R[(g + 1) & 1]);
        const int cb = c0 + 8 * g;
#pragma unroll
        for (int c4 = 0; c4 < 8; c4 += 4) {
          const float4 b4 = *reinterpret_cast<const float4*>(&s_beta[cb + c4]);
          const uint4 f4 = *reinterpret_cast<const uint4*>(&s_fix[quarter][cb + c4]);
          const float bev[4] = {b4.x, b4.y, b4.z, b4.w};
          const uint32_t fw[4] = {f4.x, f4.y, f4.z, f4.w};
#pragma unroll
          for (int u = 0; u < 4; u += 2) {
            const int cc = c4 + u;  // columns cb + cc, cb + cc + 1
            const __nv_bfloat162 d2 = __halves2bfloat162(*dptr(8 * g + cc), *dptr(8 * g + cc + 1));
            float gk[2], dx[2], dvp[2];
            float2 xn[2];
            bstep_pair(r[1][cc], r[1][cc + 1], r[0][cc], r[0][cc + 1], r[2][cc], r[2][cc + 1], r[3][cc],
                       r[3][cc + 1], __low2float(d2), __high2float(d2), bev[u], bev[u + 1], invLf, lj, uj, gk, xn,
                       dx, dvp);
#pragma unroll
            for (int e = 0; e < 2; ++e) {
              const int c = cb + cc + e;
              const bool act = c < nat && jv;
              const bool fixed = ((fw[u + e] >> lane) & 1u) != 0;
              if (fixed || !act) {
                xn[e] = make_float2(__uint_as_float(r[2][cc + e]), __uint_as_float(r[3][cc + e]));
                dx[e] = 0.f;
                dvp[e] = 0.f;
              }
              dv[(8 * g + cc + e) & 15] = dvp[e];
              if (wr && act) {
                const size_t o = (size_t)s_inst[c] * p.npad + jg;
                Xn[o] = xn[e];
                if (last) Gc[o] = gk[e];
              }
              r[1][cc + e] = __float_as_uint(gk[e]);
              r[2][cc + e] = __float_as_uint(xn[e].x);
              r[3][cc + e] = __float_as_uint(xn[e].y);
              r[0][cc + e] = __float_as_uint(dx[e]);  // the new d waits in the accumulator's own columns
            }
          }
        }
        const uint32_t cbu = (uint32_t)cb;
        tmem_st8(tl + kTmG + cbu, r[1]);
        tmem_st8(tl + kTmX + cbu, r[2]);
        tmem_st8(tl + kTmXl + cbu, r[3]);
        tmem_st8(tl + cbu, r[0]);
        if (g & 1) {
          // restart-test partials of the warp's 32 coordinates for columns c0 + 16 (g / 2) + (0..15)
          const float sum = lane_sums16(dv, lane);
          if (lane < 16) s_dot[quarter][c0 + 16 * (g >> 1) + lane] = sum;
        }
      }
      tmem_wait_st();
    }
    tc_fence_before();
    __syncthreads();
    if (tid < kBTile) {
      const float part = s_dot[0][tid] + s_dot[1][tid] + s_dot[2][tid] + s_dot[3][tid];
      const int inst = s_inst[tid];
      if (last && inst >= 0) b.dotp[s][(size_t)mt * p.B + inst] = part;
      const uint32_t a = smem_u32(&s_part[q & 1][mt][tid]);
      for (int r = 0; r < MT; ++r) st_cluster_f32(map_to_rank(a, (uint32_t)r), part);
    }
    // every CTA of the cluster has finished the products that read d_k and sent its partials
    cluster_sync_all();
    tc_fence_after();
    if (!last) {
      if (have) {
        float dn[32];
        tmem_ld32(tl + (uint32_t)c0, dn);
#pragma unroll
        for (int cc = 0; cc < 32; ++cc) *dptr(cc) = __float2bfloat16_rn(dn[cc]);
        fence_proxy_async_smem();
      }
      if (tid < kBTile) {
        const int inst = s_inst[tid];
        if (inst >= 0) {
          float dsum = 0.f;
          for (int t = 0; t < MT; ++t) dsum += s_part[q & 1][t][tid];
          float T;
          s_beta[tid] = bstep_momentum(s_tval[tid], dsum, p.restart, T);
          s_tval[tid] = T;
          if (mt == 0 && q + 1 == nsteps - 1) b.tval[(k + 1) & 1][inst] = T;
        }
      }
      tc_fence_before();
      __syncthreads();
      if (tid == 0) {
        for (int d = 1; d < MT; ++d) {
          const uint32_t r = (uint32_t)((mt + d) % MT);
          bulk_s2s(map_to_rank(smem_u32(sD + own), r), sD + own, (uint32_t)kSliceBytes,
                   map_to_rank(smem_u32(&dfull), r));
        }
      }
    }
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 0) tmem_dealloc(tmem, 512);
  if (!ok) atomicOr(&st->error, 1);
  if (tid == 0 && mt == 0 && nt == 0) st->sum_step += (double)n_act * nsteps;
}

size_t bsteps_smem_bytes(int npad) {
  return (size_t)(npad / kBChunk) * kChunkBytes + (size_t)kBPStages * kChunkBytes + 1024;
}

// dynamic shared memory within the 227 KB a CTA may hold, the kernel's 12 KB of static
// shared memory aside
bool bsteps_supported(int npad) { return npad / kBTile <= kBPMaxTiles && bsteps_smem_bytes(npad) <= 215 * 1024; }

cudaError_t launch_bsteps(const BParams& p, const BBuffers& b, int j0, int nsteps, cudaStream_t s) {
  const int MT = p.npad / kBTile;
  if (!bsteps_supported(p.npad) || nsteps < 1) return cudaErrorInvalidValue;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(MT, (p.B + kBTile - 1) / kBTile);
  cfg.blockDim = dim3(kBStepThreads);
  cfg.dynamicSmemBytes = bsteps_smem_bytes(p.npad);
  cfg.stream = s;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeClusterDimension;
  at[0].val.clusterDim.x = MT;
  at[0].val.clusterDim.y = 1;
  at[0].val.clusterDim.z = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, k_bsteps, p, b, j0, nsteps);
}

// ------------------------------------------------------------------ evaluation
// kBEvalInst instances per CTA (A is read once for all of them), 256 threads.
//   phase 1  r = y - A x_k (warp = instance, lanes over rows), double-float, nonzero x_j only;
//   phase 2  g_j = a_j^T r for the columns some instance preserves (thread = two columns,
//            all rows), PREC products;
//   phase 3  gap sums and the step (warp = instance, lanes over coordinates);
//   phase 4  sphere test; phase 5  outputs of the instances that stop (warp = instance).
// Bytes of phase 2's copy ring: per warp RING steps of 8 rows of its 32 BC columns.
__host__ __device__ constexpr size_t beval_ring_bytes(int prec, int ring) {
  return (size_t)ring * (kBEvalThreads / 32) * (prec == kX2 ? 1 : 2) * 2 * 32 * 16;
}

template <int PREC, int RING>
__global__ void __launch_bounds__(kBEvalThreads, 2) k_beval(BParams p, BBuffers b, int jrel) {
  BState* st = b.st;
  if (st->done) return;
  const int n_act = st->n_act;
  const int i0 = blockIdx.x * kBEvalInst;
  if (i0 >= n_act) return;
  // dynamic shared memory (beval_lists_offset): the residuals, the screened flags (bit 2
  // marks a correlation recomputed in double-float), the coordinate lists of phases 2 and 2b,
  // and phase 1's nonzero lists
  const int mr = (p.m + 7) & ~7;
  extern __shared__ float4 smem_ev[];
  float* srh = reinterpret_cast<float*>(smem_ev);
  float* srl = srh + (size_t)mr * kBEvalInst;
  uint8_t* s_fl = reinterpret_cast<uint8_t*>(srl + (size_t)mr * kBEvalInst);
  uint16_t* s_item = reinterpret_cast<uint16_t*>(s_fl + (size_t)kBEvalInst * p.npad);
  __shared__ int s_inst[kBEvalInst];
  __shared__ float s_beta[kBEvalInst];
  __shared__ int s_goff[kBMaxCols / 32 + 1];
  int* s_lj = reinterpret_cast<int*>(reinterpret_cast<unsigned char*>(smem_ev) + beval_lists_offset(p.m, p.npad));
  float2* s_lx = reinterpret_cast<float2*>(s_lj + kBEvalInst * kBEvalList);
  __shared__ double s_red[kBEvalThreads / 32][kBEvalInst][5];
  __shared__ int s_ref[kBEvalInst];
  __shared__ float s_qf[kBEvalInst][4];   // eps, eta, eta of refined correlations (rounded up)
  __shared__ double s_sum_infl;           // bound of the relative rounding of the float32 sums
  __shared__ double s_q[kBEvalInst][10];  // P, ||y||^2, eta_g, eps, radius + eta, eta, gap, preserved,
                                          // eta of the recomputed correlations
  __shared__ int s_stop[kBEvalInst];
  __shared__ int s_pins[kBEvalInst];

  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int k = st->kbase + jrel;
  const int s = k & 1;
  const int MT = p.npad / kBTile;
  const bool trans = p.dual_mode == kTranslation;
  if (tid < kBEvalInst) {
    const int q = i0 + tid;
    const int inst = q < n_act ? b.act[q] : -1;
    s_inst[tid] = inst;
    float beta = 0.f;
    if (inst >= 0) {
      float T = 1.f;
      if (k > 0) {
        const float tp = b.tval[s ^ 1][inst];
        float dsum = 0.f;
        for (int t = 0; t < MT; ++t) dsum += b.dotp[s ^ 1][(size_t)t * p.B + inst];
        T = (p.restart && dsum < 0.f) ? 1.f : 0.5f * (1.f + sqrtf(1.f + 4.f * tp * tp));
      }
      const float tn = 0.5f * (1.f + sqrtf(1.f + 4.f * T * T));
      beta = (T - 1.f) / tn;
      b.tval[s][inst] = T;
    }
    s_beta[tid] = beta;
    s_pins[tid] = 0;
  }
  __syncthreads();
  // the screened flags of the CTA's instances, one coalesced pass in 4-byte words (1 = fixed,
  // or no instance)
  {
    const int w4 = p.npad / 4;
#pragma unroll 4
    for (int q = tid; q < kBEvalInst * w4; q += kBEvalThreads) {
      const int bb = q / w4, j4 = q - bb * w4;
      const int inst = s_inst[bb];
      reinterpret_cast<uint32_t*>(s_fl)[q] =
          inst >= 0 ? reinterpret_cast<const uint32_t*>(b.flags + (size_t)inst * p.npad)[j4] : 0x01010101u;
    }
  }

  // ---- phase 1: r = y - A x_k.  Warp bb owns instance bb: for each block of 256 rows it
  // lists the nonzero x_j of a chunk of kBEvalList columns, then its lanes (row pairs
  // 2 lane + 64 t, t < 4) accumulate the listed columns four at a time in packed
  // double-float pairs, so each lane keeps 16 loads of 8 bytes in flight.
  const float2* __restrict__ Xc = b.X[s];
  {
    constexpr int NP = kBEvalRows / 2;  // row pairs per lane and block
    const int bb = warp;  // kBEvalThreads / 32 == kBEvalInst
    const int inst = s_inst[bb];
    double pv = 0.0, yv = 0.0;
    for (int r0 = 0; r0 < p.m; r0 += 32 * kBEvalRows) {
    f32x2 qs[NP], qc[NP];
#pragma unroll
    for (int r = 0; r < NP; ++r) qs[r] = qc[r] = 0ull;
    for (int jc = 0; jc < p.n && inst >= 0; jc += kBEvalList) {
      int cnt = 0;
      float2 xs[kBEvalList / 32];
#pragma unroll
      for (int t = 0; t < kBEvalList / 32; ++t) {  // loads first
        const int j = jc + t * 32 + lane;
        xs[t] = j < p.n ? Xc[(size_t)inst * p.npad + j] : make_float2(0.f, 0.f);
      }
#pragma unroll
      for (int t = 0; t < kBEvalList / 32; ++t) {
        const bool nz = df2_nonzero(xs[t]);
        const unsigned msk = __ballot_sync(kFull, nz);
        if (nz) {
          const int pos = cnt + __popc(msk & ((1u << lane) - 1u));
          s_lj[bb * kBEvalList + pos] = jc + t * 32 + lane;
          s_lx[bb * kBEvalList + pos] = xs[t];
        }
        cnt += __popc(msk);
      }
      __syncwarp();
      for (int e = 0; e < cnt; e += 4) {
        f32x2 a[4][NP];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          const float* col = p.A + (size_t)s_lj[bb * kBEvalList + (e + u < cnt ? e + u : e)] * p.lda;
#pragma unroll
          for (int r = 0; r < NP; ++r) {
            // rows i, i + 1 (i even, i < m <= lda, so i + 1 < lda: in the column)
            const int i = r0 + 2 * lane + 64 * r;
            a[u][r] = (e + u < cnt && i < p.m) ? __ldg(reinterpret_cast<const unsigned long long*>(col + i)) : 0ull;
          }
        }
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          const float2 x = e + u < cnt ? s_lx[bb * kBEvalList + e + u] : make_float2(0.f, 0.f);
          const f32x2 xh = x2_pack(x.x, x.x), xl = x2_pack(x.y, x.y);
#pragma unroll
          for (int r = 0; r < NP; ++r) df_fma_x2(qs[r], qc[r], a[u][r], xh, xl);
        }
      }
      __syncwarp();
    }
#pragma unroll
    for (int r = 0; r < NP; ++r) {
      float q2s[2], q2c[2];
      x2_unpack(qs[r], q2s[0], q2s[1]);
      x2_unpack(qc[r], q2c[0], q2c[1]);
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        const int i = r0 + 2 * lane + 64 * r + h;
        if (i < mr) {
          float rh = 0.f, rl = 0.f;
          if (inst >= 0 && i < p.m) {
            const float y = b.Y[(size_t)inst * p.lda + i];
            float dh, de;
            two_sum(y, -q2s[h], dh, de);
            de -= q2c[h];
            two_sum(dh, de, rh, rl);
            const double rv = (double)rh + (double)rl;
            pv += 0.5 * rv * rv;
            yv += (double)y * (double)y;
          }
          srh[(size_t)i * kBEvalInst + bb] = rh;
          srl[(size_t)i * kBEvalInst + bb] = rl;
        }
      }
    }
    }
    pv = warp_sum_dd(pv);
    yv = warp_sum_dd(yv);
    if (lane == 0) {
      s_q[bb][0] = pv;
      s_q[bb][1] = yv;
      s_q[bb][2] = p.Cg * sqrt(2.0 * pv) * (1.0 + 1e-6);  // eta_g: rounding of a_j^T r per unit norm
    }
  }
  __syncthreads();

  // ---- phase 2: correlations g_j = a_j^T r for the CTA's instances over the columns that
  // some instance preserves.  Those columns are listed in order; thread (warp w, lane c)
  // owns list entries 32 (BC w + u) + c (u < BC, then strides of 256 BC) and walks all
  // rows of its columns for the 8 instances: A in 32-byte pieces (8 rows) that the thread
  // copies from L2 into its own slots of a RING-step shared-memory ring (16-byte cp.async,
  // RING - 1 steps in flight), the residuals broadcast from shared memory.  Summation
  // order: beval_chain (the Cg of make_bparams).
  {
    constexpr int NW = kBEvalThreads / 32;
    constexpr int NI = kBEvalInst;
    constexpr int BC = PREC == kX2 ? 1 : 2;                 // columns per thread
    constexpr int ILV = PREC == kX2 ? kBEvalIlvX2 : kBEvalIlvF32;
    const int NG = p.npad / 32;
    // the list: group counts, an exclusive scan by warp 0, then the entries
    for (int g = warp; g < NG; g += NW) {
      const int j = g * 32 + lane;
      bool need = false;
      if (j < p.n)
#pragma unroll
        for (int bb = 0; bb < NI; ++bb) need |= (s_fl[bb * p.npad + j] & 3) == 0;
      const unsigned msk = __ballot_sync(kFull, need);
      if (lane == 0) s_goff[g] = __popc(msk);
    }
    __syncthreads();
    if (warp == 0) {
      const int per = (NG + 31) / 32;
      int loc = 0;
      for (int q = 0; q < per; ++q) {
        const int g = lane * per + q;
        if (g < NG) loc += s_goff[g];
      }
      int inc = loc;
      for (int o = 1; o < 32; o <<= 1) {
        const int v = __shfl_up_sync(kFull, inc, o);
        if (lane >= o) inc += v;
      }
      int run = inc - loc;
      for (int q = 0; q < per; ++q) {
        const int g = lane * per + q;
        if (g < NG) {
          const int c = s_goff[g];
          s_goff[g] = run;
          run += c;
        }
      }
      if (lane == 31) s_goff[NG] = inc;
    }
    __syncthreads();
    for (int g = warp; g < NG; g += NW) {
      const int j = g * 32 + lane;
      bool need = false;
      if (j < p.n)
#pragma unroll
        for (int bb = 0; bb < NI; ++bb) need |= (s_fl[bb * p.npad + j] & 3) == 0;
      const unsigned msk = __ballot_sync(kFull, need);
      if (need) s_item[s_goff[g] + __popc(msk & ((1u << lane) - 1u))] = (uint16_t)j;
    }
    __syncthreads();
    const int ncol = s_goff[NG];
    const int R = p.erb;
    float4* ring = reinterpret_cast<float4*>(s_lj);  // phase 1's lists are dead
    // s_red[w][bb][3]: warp w's running max of the translation step candidates of instance bb
    if (lane < NI) s_red[warp][lane][3] = 0.0;
    __syncwarp();
    for (int t0 = warp * 32 * BC; t0 < ncol; t0 += kBEvalThreads * BC) {
      int jc[BC];
      bool cv[BC];
      const float* colp[BC];
#pragma unroll
      for (int u = 0; u < BC; ++u) {
        const int t = t0 + u * 32 + lane;
        cv[u] = t < ncol;
        jc[u] = s_item[cv[u] ? t : t0];
        colp[u] = p.A + (size_t)jc[u] * p.lda;
      }
      // instance pairs (2 h, 2 h + 1) in packed registers
      constexpr int NH = NI / 2;
      f32x2 tot[BC][NH], totc[BC][NH], acc[BC][NH][ILV], accc[BC][NH][ILV];
#pragma unroll
      for (int u = 0; u < BC; ++u)
#pragma unroll
        for (int h = 0; h < NH; ++h) {
          tot[u][h] = totc[u][h] = 0ull;
#pragma unroll
          for (int q = 0; q < ILV; ++q) acc[u][h][q] = accc[u][h][q] = 0ull;
        }
      // ring slot (step t, column u, half h) of this thread: ring + ((t % RING) * 2 BC + 2 u + h) * 32 + lane
      float4* ringw = ring + (size_t)warp * RING * 2 * BC * 32 + lane;
      auto issue = [&](int i) {  // rows i..i+7 of the thread's columns
        float4* d = ringw + (size_t)((i >> 3) % RING) * 2 * BC * 32;
#pragma unroll
        for (int u = 0; u < BC; ++u) {
          cp_async16(d + (2 * u) * 32, colp[u] + i);
          cp_async16(d + (2 * u + 1) * 32, colp[u] + i + 4);
        }
      };
#pragma unroll
      for (int t = 0; t < RING - 1; ++t) {
        if (8 * t < mr) issue(8 * t);
        cp_async_commit();
      }
      float a[BC][8];
      int rin = 0;  // rows of the running block done
      for (int i = 0; i < mr; i += 8) {
        if (i + 8 * (RING - 1) < mr) issue(i + 8 * (RING - 1));
        cp_async_commit();
        cp_async_wait<RING - 1>();  // this thread's copy of rows i..i+7 has landed
        {
          const float4* sl = ringw + (size_t)((i >> 3) % RING) * 2 * BC * 32;
#pragma unroll
          for (int u = 0; u < BC; ++u) {
            const float4 v0 = sl[(2 * u) * 32], v1 = sl[(2 * u + 1) * 32];
            a[u][0] = v0.x; a[u][1] = v0.y; a[u][2] = v0.z; a[u][3] = v0.w;
            a[u][4] = v1.x; a[u][5] = v1.y; a[u][6] = v1.z; a[u][7] = v1.w;
          }
        }
#pragma unroll
        for (int q = 0; q < 8; ++q) {
          f32x2 ad[BC];
#pragma unroll
          for (int u = 0; u < BC; ++u) ad[u] = x2_pack(a[u][q], a[u][q]);
          const ulonglong2* rh = reinterpret_cast<const ulonglong2*>(srh + (size_t)(i + q) * NI);
          const ulonglong2* rl = reinterpret_cast<const ulonglong2*>(srl + (size_t)(i + q) * NI);
#pragma unroll
          for (int h2 = 0; h2 < NI / 4; ++h2) {
            const ulonglong2 vh = rh[h2];
            if (PREC == kX2) {
              const ulonglong2 vl = rl[h2];
#pragma unroll
              for (int u = 0; u < BC; ++u) {
                df_fma_x2(acc[u][2 * h2][q % ILV], accc[u][2 * h2][q % ILV], ad[u], vh.x, vl.x);
                df_fma_x2(acc[u][2 * h2 + 1][q % ILV], accc[u][2 * h2 + 1][q % ILV], ad[u], vh.y, vl.y);
              }
            } else {
#pragma unroll
              for (int u = 0; u < BC; ++u) {
                acc[u][2 * h2][q % ILV] = x2_fma(ad[u], vh.x, acc[u][2 * h2][q % ILV]);
                acc[u][2 * h2 + 1][q % ILV] = x2_fma(ad[u], vh.y, acc[u][2 * h2 + 1][q % ILV]);
              }
            }
          }
        }
        rin += 8;
        if (rin == R || i + 8 >= mr) {  // end of a block: merge its sums into the total
#pragma unroll
          for (int u = 0; u < BC; ++u)
#pragma unroll
            for (int h = 0; h < NH; ++h) {
#pragma unroll
              for (int w2 = 1; w2 < ILV; w2 <<= 1)
#pragma unroll
                for (int q = 0; q < ILV; q += 2 * w2) {
                  if (PREC == kX2) df_add_x2(acc[u][h][q], accc[u][h][q], acc[u][h][q + w2], accc[u][h][q + w2]);
                  else acc[u][h][q] = x2_add(acc[u][h][q], acc[u][h][q + w2]);
                }
              if (PREC == kX2) df_add_x2(tot[u][h], totc[u][h], acc[u][h][0], accc[u][h][0]);
              else tot[u][h] = x2_add(tot[u][h], acc[u][h][0]);
#pragma unroll
              for (int q = 0; q < ILV; ++q) acc[u][h][q] = accc[u][h][q] = 0ull;
            }
          rin = 0;
        }
      }
      cp_async_wait<0>();
      float ts[BC][NI], tcs[BC][NI];
#pragma unroll
      for (int u = 0; u < BC; ++u)
#pragma unroll
        for (int h = 0; h < NH; ++h) {
          x2_unpack(tot[u][h], ts[u][2 * h], ts[u][2 * h + 1]);
          x2_unpack(totc[u][h], tcs[u][2 * h], tcs[u][2 * h + 1]);
        }
#pragma unroll
      for (int bb = 0; bb < NI; ++bb) {
        const int inst = s_inst[bb];
        double em = 0.0;
#pragma unroll
        for (int u = 0; u < BC; ++u) {
          const int j = jc[u];
          if (!cv[u] || inst < 0 || s_fl[bb * p.npad + j] != 0) continue;
          const float2 g2 = df2_norm(ts[u][bb], PREC == kX2 ? tcs[u][bb] : 0.f);
          b.Ge[(size_t)inst * p.npad + j] = g2;
          if (trans && p.jinf[j]) {
            const double nr = p.nrm[j];
            if (nr > 0.0) {
              const double den = -p.w[j] - p.gamma_w * nr * p.t_norm;
              em = fmax(em, fmax(df2_to_double(g2) + s_q[bb][2] * nr, 0.0) / den);
            }
          }
        }
        if (trans) {
          em = warp_max_dd(em);
          if (lane == 0) s_red[warp][bb][3] = fmax(s_red[warp][bb][3], em);
        }
      }
    }
  }
  __syncthreads();
  if (tid < kBEvalInst) {
    double e = 0.0;
    for (int w = 0; w < kBEvalThreads / 32; ++w) e = fmax(e, s_red[w][tid][3]);
    const double eps = trans ? (double)f32_up(e) : 0.0;  // theta = r + eps t with the float32 eps
    s_q[tid][3] = eps;
    const double rnorm = sqrt(2.0 * s_q[tid][0]) * (1.0 + 1e-6);
    const double et = trans ? eps * p.gamma_w * p.t_norm : 0.0;
    s_q[tid][5] = p.Cg * rnorm + et;    // eta of the correlations of this precision
    s_q[tid][8] = p.Cg2 * rnorm + et;   // eta of double-float correlations
    s_qf[tid][0] = f32_up(eps);
    s_qf[tid][1] = f32_up(s_q[tid][5]);
    s_qf[tid][2] = f32_up(s_q[tid][8]);
    if (tid == 0) {
      const int T = (p.n + 31) / 32;  // terms per lane in phase 3
      s_sum_infl = 1.0 + 2.0 * (T + 8) * 6.0e-8;
    }
  }
  __syncthreads();

  // ---- phase 3: gap terms and the step, in float32 with every rounding bounded.  Each term
  // of the nonnegative-sum form of P - D is a convex piecewise-linear function of
  // gt_j = a_j^T theta; with the computed gt_j within E_j of the exact one, the term is
  // bounded by its larger value at the two ends of [gt_j - E_j, gt_j + E_j] (gap_term_up).
  {
    const float* __restrict__ Gp = b.G[s ^ 1];
    float* Gc = b.G[s];
    float2* Xn = b.X[s ^ 1];
    __nv_bfloat16* Dn = b.D[s ^ 1];
    const float2 invL2 = p.invL2;
    {
      const int bb = warp;  // warp bb owns instance bb, lanes over coordinates
      const int inst = s_inst[bb];
      const float be = s_beta[bb];
      const float eps = s_qf[bb][0], eta = s_qf[bb][1], eta_ref = s_qf[bb][2];
      float va = 0.f, vx = 0.f, vd = 0.f, vs = 0.f;
      int vp = 0;
      // four coordinates per lane and round, every load of the round issued before its stores
      // (the stores into x_{k+1} could alias the loads of a later coordinate otherwise)
      constexpr int NB = 4;
      for (int jb = lane; jb < p.n && inst >= 0; jb += 32 * NB) {
        float2 xk[NB], xp[NB], g2[NB], l2[NB], u2[NB];
        float gp[NB], nr[NB], wf[NB];
        uint8_t fl[NB], jf[NB];
#pragma unroll
        for (int u = 0; u < NB; ++u) {
          const int j = jb + 32 * u;
          if (j < p.n) {
            const size_t o = (size_t)inst * p.npad + j;
            xk[u] = Xc[o];
            xp[u] = Xn[o];
            g2[u] = b.Ge[o];
            gp[u] = Gp[o];
            nr[u] = p.nrmf[j];
            l2[u] = p.l2[j];
            u2[u] = p.u2[j];
            jf[u] = p.jinf[j];
            wf[u] = p.wf[j];
            fl[u] = s_fl[bb * p.npad + j];
          }
        }
#pragma unroll
        for (int u = 0; u < NB; ++u) {
          const int j = jb + 32 * u;
          if (j >= p.n) break;
          const size_t o = (size_t)inst * p.npad + j;
          vx += fabsf(xk[u].x) * nr[u];
          if (fl[u] & 3) {
            Xn[o] = xk[u];
            Dn[o] = __float2bfloat16_rn(0.f);
            continue;
          }
          ++vp;
          if (p.dual_mode != kZero) {
            float du, dl, gt, E;
            term_inputs_v(xk[u], g2[u], l2[u], u2[u], jf[u] != 0, wf[u], p.dual_mode, eps,
                          ((fl[u] & 4) ? eta_ref : eta) * nr[u], du, dl, gt, E);
            const float hup = gap_term_up(du, dl, gt, E);
            va += hup;
            vs += hup - (du * fmaxf(gt, 0.f) + dl * fmaxf(-gt, 0.f));  // what exact correlations could remove
          }
          const float gk = g2[u].x;
          const float gv = fmaf(be, gk - gp[u], gk);
          const float2 xn = fista_step(xk[u], df2_sub(xk[u], xp[u]), gv, be, invL2, l2[u], u2[u]);
          const float2 d = df2_sub(xn, xk[u]);
          const float dx = d.x + d.y;
          Gc[o] = gk;
          Xn[o] = xn;
          Dn[o] = __float2bfloat16_rn(dx);
          vd = fmaf(gv, dx, vd);
        }
      }
      va = warp_sum_f(va);
      vx = warp_sum_f(vx);
      vd = warp_sum_f(vd);
      vs = warp_sum_f(vs);
      for (int o2 = 16; o2 > 0; o2 >>= 1) vp += __shfl_xor_sync(kFull, vp, o2);
      if (lane == 0) {
        s_red[bb][bb][0] = va;
        s_red[bb][bb][1] = vx;
        s_red[bb][bb][2] = vd;
        s_red[bb][bb][3] = vp;
        s_red[bb][bb][4] = vs;
      }
    }
  }
  __syncthreads();
  if (tid < kBEvalInst) {
    double a = s_red[tid][tid][0], x1 = s_red[tid][tid][1], d = s_red[tid][tid][2], np = s_red[tid][tid][3],
           sl = s_red[tid][tid][4];
    a *= s_sum_infl;   // float32 sums of nonnegative terms: per-lane runs and 5 shuffle levels
    x1 *= s_sum_infl;
    const int inst = s_inst[tid];
    int ref = 0;
    if (inst >= 0) {
      const double P = s_q[tid][0];
      const double rnorm = sqrt(2.0 * P) * (1.0 + 1e-6);
      const double E_r = p.Cf * x1 + p.Csub * (rnorm + sqrt(s_q[tid][1]) + x1);
      // the part of the bound that does not depend on the correlations' rounding
      const double dd = p.dual_mode == kZero ? rnorm + E_r : E_r + (double)s_qf[tid][0] * p.t_norm;
      s_q[tid][9] = 0.5 * dd * dd;
      const double gap = (p.dual_mode == kZero ? s_q[tid][9] : a + s_q[tid][9]) * (1.0 + 1e-12);
      s_q[tid][6] = gap;
      // recompute the sensitive correlations in double-float when that could decide the stop
      ref = PREC == kF32 && p.dual_mode != kZero && gap >= p.tol && (gap - sl < p.tol || k >= p.max_iter);
      b.dotp[s][inst] = (float)d;
      for (int t = 1; t < MT; ++t) b.dotp[s][(size_t)t * p.B + inst] = 0.f;
      atomicAdd(&st->sum_pres, np);
    }
    s_ref[tid] = ref;
    s_q[tid][7] = np;
  }
  __syncthreads();

  if (PREC == kF32 && __syncthreads_or(tid < kBEvalInst && s_ref[tid])) {
    // ---- phase 2b: a gap term depends on the rounding of its correlation only when the
    // coordinate is free or its correlation is within the margin of zero; those
    // correlations are recomputed in double-float.
    const int bb = warp;
    const int inst = s_ref[bb] ? s_inst[bb] : -1;
    int cnt = 0;
    if (inst >= 0) {
      const double eps = s_q[bb][3], eF = s_q[bb][5];
      for (int jc = 0; jc < p.n; jc += 32) {
        const int j = jc + lane;
        bool ref = false;
        if (j < p.n && (s_fl[bb * p.npad + j] & 3) == 0) {
          const size_t o = (size_t)inst * p.npad + j;
          const double nr = p.nrm[j];
          if (nr > 0.0) {
            const float2 xk = Xc[o];
            const double gt = (double)b.Ge[o].x + (trans ? eps * p.w[j] : 0.0);
            const double e = eF * nr;
            const bool at_l = df2_eq(xk, p.l2[j]);
            const bool at_u = !p.jinf[j] && df2_eq(xk, p.u2[j]);
            // at l_j with u_j = +inf the term (x_j - l_j)(-gt)^+ is zero whatever gt is
            ref = at_l ? (!p.jinf[j] && gt + e > 0.0) : at_u ? (gt - e < 0.0) : true;
          }
        }
        const unsigned msk = __ballot_sync(kFull, ref);
        if (ref) s_item[bb * p.npad + cnt + __popc(msk & ((1u << lane) - 1u))] = (uint16_t)j;
        cnt += __popc(msk);
      }
      __syncwarp();
      // four listed coordinates at a time; lanes over rows, then a shuffle reduction, so the
      // double-float chains are as short as in the main correlation
      for (int t0 = 0; t0 < cnt; t0 += 4) {
        int jj[4];
        const float* col[4];
#pragma unroll
        for (int c = 0; c < 4; ++c) {
          jj[c] = s_item[bb * p.npad + (t0 + c < cnt ? t0 + c : t0)];
          col[c] = p.A + (size_t)jj[c] * p.lda;
        }
        float sh[4] = {0.f, 0.f, 0.f, 0.f}, sc[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll 2
        for (int i = lane; i < p.m; i += 32) {
          const float rh = srh[(size_t)i * kBEvalInst + bb], rl = srl[(size_t)i * kBEvalInst + bb];
#pragma unroll
          for (int c = 0; c < 4; ++c) df_fma(sh[c], sc[c], __ldg(col[c] + i), rh, rl);
        }
#pragma unroll
        for (int c = 0; c < 4; ++c) {
#pragma unroll
          for (int o = 16; o > 0; o >>= 1) {
            const float ox = __shfl_xor_sync(kFull, sh[c], o);
            const float oc = __shfl_xor_sync(kFull, sc[c], o);
            df_add(sh[c], sc[c], ox, oc);
          }
        }
        if (lane < 4 && t0 + lane < cnt) {
          float h = sh[0], l = sc[0];
#pragma unroll
          for (int c = 1; c < 4; ++c)
            if (lane == c) {
              h = sh[c];
              l = sc[c];
            }
          b.Ge[(size_t)inst * p.npad + jj[lane]] = df2_norm(h, l);
          s_fl[bb * p.npad + jj[lane]] |= 4;
        }
        __syncwarp();
      }
    }
    __syncthreads();
    // ---- phase 3b: the gap terms of the refined instances again (warp = instance)
    {
      const int bb2 = warp;
      const int inst2 = s_ref[bb2] ? s_inst[bb2] : -1;
      const float eps = s_qf[bb2][0], eta = s_qf[bb2][1], eta_ref = s_qf[bb2][2];
      float va = 0.f;
#pragma unroll 4
      for (int j = lane; j < p.n && inst2 >= 0; j += 32) {
        const uint8_t fl = s_fl[bb2 * p.npad + j];
        if (fl & 3) continue;
        const size_t o = (size_t)inst2 * p.npad + j;
        float du, dl, gt, E;
        term_inputs(Xc[o], b.Ge[o], j, p, eps, ((fl & 4) ? eta_ref : eta) * p.nrmf[j], du, dl, gt, E);
        va += gap_term_up(du, dl, gt, E);
      }
      va = warp_sum_f(va);
      if (lane == 0) s_red[bb2][bb2][0] = va;
    }
    __syncthreads();
    if (tid < kBEvalInst && s_ref[tid]) {
      const double a = s_red[tid][tid][0];
      s_q[tid][6] = fmin(s_q[tid][6], (a * s_sum_infl + s_q[tid][9]) * (1.0 + 1e-12));
    }
    __syncthreads();
  }
  if (tid < kBEvalInst) {
    const int inst = s_inst[tid];
    int stop = 0;
    if (inst >= 0) {
      const double gap = s_q[tid][6];
      s_q[tid][4] = sqrt(2.0 * gap) * (1.0 + 1e-12) + s_q[tid][5];  // radius + margin, per unit ||a_j||
      stop = (gap < p.tol || k >= p.max_iter) ? 1 : 0;
    }
    s_stop[tid] = stop;
  }
  __syncthreads();

  // ---- phase 4: sphere test (Eq. (safe_rule)) in float32: the computed gt_j, widened by its
  // own rounding, must clear (radius + eta) ||a_j|| rounded up.  A coordinate is fixed once
  // x_k and x_{k+1} both sit at the bound the test gives.
  if (p.screening && p.dual_mode != kZero) {
    const float2* __restrict__ Xn = b.X[s ^ 1];
    {
      const int bb = warp;  // warp = instance
      const int inst = s_inst[bb];
      const float eps = s_qf[bb][0];
      const float rr = f32_up(s_q[bb][4]);
      int pins = 0;
      // four coordinates per lane and round, their loads issued before any flag store
      constexpr int NB = 4;
      for (int jb = lane; jb < p.n && inst >= 0; jb += 32 * NB) {
        float2 g2[NB], l2[NB], u2[NB];
        float nr[NB], wf[NB];
        uint8_t fl[NB], jf[NB];
#pragma unroll
        for (int u = 0; u < NB; ++u) {
          const int j = jb + 32 * u;
          fl[u] = 1;
          if (j < p.n) {
            fl[u] = s_fl[bb * p.npad + j];
            nr[u] = p.nrmf[j];
            g2[u] = b.Ge[(size_t)inst * p.npad + j];
            wf[u] = p.wf[j];
            jf[u] = p.jinf[j];
            l2[u] = p.l2[j];
            u2[u] = p.u2[j];
          }
        }
#pragma unroll
        for (int u = 0; u < NB; ++u) {
          const int j = jb + 32 * u;
          if ((fl[u] & 3) || !(nr[u] > 0.f)) continue;
          const size_t o = (size_t)inst * p.npad + j;
          const float ew = trans ? eps * wf[u] : 0.f;
          const float gt = (g2[u].x + ew) + g2[u].y;
          const float dl = 8.f * kUf * (fabsf(g2[u].x) + fabsf(ew)) + fabsf(g2[u].y);
          const float thr = rr * nr[u] * (1.f + 4.f * kUf);
          int pin = 0;
          float2 bnd = make_float2(0.f, 0.f);
          if (gt + dl < -thr) {
            pin = 1;
            bnd = l2[u];
          } else if (!jf[u] && gt - dl > thr) {
            pin = 2;
            bnd = u2[u];
          }
          if (pin && df2_eq(Xc[o], bnd) && df2_eq(Xn[o], bnd)) {
            b.flags[o] = (uint8_t)pin;
            s_fl[bb * p.npad + j] = (uint8_t)pin;
            ++pins;
          }
        }
      }
      for (int o2 = 16; o2 > 0; o2 >>= 1) pins += __shfl_xor_sync(kFull, pins, o2);
      if (lane == 0) s_pins[bb] = pins;
    }
    __syncthreads();
  }

  // ---- phase 5: outputs of the instances that stop at this evaluation
  {
    const int bb = warp;  // warp = instance
    const int inst = s_stop[bb] ? s_inst[bb] : -1;
#pragma unroll 4
    for (int j = lane; j < p.n && inst >= 0; j += 32) {
      const uint8_t f = s_fl[bb * p.npad + j] & 3;
      const size_t o = (size_t)inst * p.npad + j;
      const double x = f == 1 ? p.l[j] : f == 2 ? p.u[j] : fmin(fmax(df2_to_double(Xc[o]), p.l[j]), p.u[j]);
      b.xout[(size_t)inst * p.n + j] = x;
    }
  }
  if (tid < kBEvalInst) {
    const int inst = s_inst[tid];
    if (inst >= 0 && s_stop[tid]) {
      const double gap = s_q[tid][6];
      b.gap[inst] = gap;
      b.primal[inst] = s_q[tid][0];
      b.iters[inst] = k;
      b.status[inst] = gap < p.tol ? 0 : 4;
      b.npres[inst] = (int)s_q[tid][7] - s_pins[tid];
      b.fin[inst] = 1;
    }
  }
  if (blockIdx.x == 0 && tid == 0) st->sum_eval += (double)n_act;
}

size_t beval_smem_bytes(int m, int npad, int prec, int ring) {
  const size_t lists = (size_t)kBEvalInst * kBEvalList * (sizeof(int) + sizeof(float2));
  const size_t rb = beval_ring_bytes(prec, ring);
  return beval_lists_offset(m, npad) + (lists > rb ? lists : rb);
}

namespace {
// The deep ring when the kernel's shared memory fits the opt-in limit, else a single slot.
template <int PREC>
int beval_ring(int m, int npad) {
  static const int optin = [] {
    int dev = 0, v = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&v, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) != cudaSuccess) return 0;
    return v;
  }();
  cudaFuncAttributes fa;
  if (cudaFuncGetAttributes(&fa, k_beval<PREC, kBEvalRing>) != cudaSuccess) return 1;
  return beval_smem_bytes(m, npad, PREC, kBEvalRing) + fa.sharedSizeBytes <= (size_t)optin ? kBEvalRing : 1;
}

template <int PREC>
cudaError_t beval_configure(int m, int npad) {
  if (beval_ring<PREC>(m, npad) == kBEvalRing)
    return cudaFuncSetAttribute(k_beval<PREC, kBEvalRing>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)beval_smem_bytes(m, npad, PREC, kBEvalRing));
  return cudaFuncSetAttribute(k_beval<PREC, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              (int)beval_smem_bytes(m, npad, PREC, 1));
}

template <int PREC>
cudaError_t beval_launch(const BParams& p, const BBuffers& b, int j, cudaStream_t s) {
  const int grid = (p.B + kBEvalInst - 1) / kBEvalInst;
  if (beval_ring<PREC>(p.m, p.npad) == kBEvalRing)
    k_beval<PREC, kBEvalRing><<<grid, kBEvalThreads, beval_smem_bytes(p.m, p.npad, PREC, kBEvalRing), s>>>(p, b, j);
  else
    k_beval<PREC, 1><<<grid, kBEvalThreads, beval_smem_bytes(p.m, p.npad, PREC, 1), s>>>(p, b, j);
  return cudaGetLastError();
}
}  // namespace


cudaError_t launch_beval(const BParams& p, const BBuffers& b, int j, int precision, cudaStream_t s) {
  return precision == kX2 ? beval_launch<kX2>(p, b, j, s) : beval_launch<kF32>(p, b, j, s);
}

// ------------------------------------------------------------------ retirement
// One block: the active list keeps its order (stable), so every later launch sees the same
// instance-to-tile assignment for the same inputs.
__global__ void __launch_bounds__(1024) k_bcompact(BParams p, BBuffers b) {
  BState* st = b.st;
  if (st->done) return;
  __shared__ int sh[32];
  __shared__ int s_total;
  const int n = st->n_act;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  for (int q = tid; q < n; q += blockDim.x) b.act_tmp[q] = b.act[q];
  __syncthreads();
  int out = 0;
  for (int base = 0; base < n; base += blockDim.x) {
    const int q = base + tid;
    const int inst = q < n ? b.act_tmp[q] : -1;
    const int keep = (inst >= 0 && !b.fin[inst]) ? 1 : 0;
    int x = keep;
    for (int o = 1; o < 32; o <<= 1) {
      const int y = __shfl_up_sync(kFull, x, o);
      if (lane >= o) x += y;
    }
    if (lane == 31) sh[warp] = x;
    __syncthreads();
    if (warp == 0) {
      int w = lane < (int)(blockDim.x >> 5) ? sh[lane] : 0;
      for (int o = 1; o < 32; o <<= 1) {
        const int y = __shfl_up_sync(kFull, w, o);
        if (lane >= o) w += y;
      }
      sh[lane] = w;  // inclusive prefix over warps
      if (lane == 31) s_total = w;
    }
    __syncthreads();
    const int pos = out + (warp > 0 ? sh[warp - 1] : 0) + x - keep;
    if (keep) b.act[pos] = inst;
    out += s_total;
    __syncthreads();
  }
  if (tid == 0) {
    st->n_act = out;
    st->gap_evals += 1;
    if (out == 0) st->done = 1;
  }
}

cudaError_t batch_configure(int m, int npad) {
  cudaError_t e = cudaFuncSetAttribute(k_bstep, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bstep_smem_bytes());
  if (e == cudaSuccess && bsteps_supported(npad))
    e = cudaFuncSetAttribute(k_bsteps, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bsteps_smem_bytes(npad));
  if (e != cudaSuccess) return e;
  e = beval_configure<kX2>(m, npad);
  if (e != cudaSuccess) return e;
  return beval_configure<kF32>(m, npad);
}

cudaError_t launch_bcompact(const BParams& p, const BBuffers& b, cudaStream_t s) {
  k_bcompact<<<1, 1024, 0, s>>>(p, b);
  return cudaGetLastError();
}

__global__ void k_bchunk_end(BBuffers b, int chunk_len) {
  if (threadIdx.x == 0 && blockIdx.x == 0) b.st->kbase += chunk_len;
}

__global__ void k_bloop_ctl(BState* st, cudaGraphConditionalHandle h, int max_chunks) {
  if (threadIdx.x == 0 && blockIdx.x == 0) {
    const int c = ++st->chunks;
    if (st->done || st->error || c >= max_chunks) cudaGraphSetConditional(h, 0);
  }
}

cudaError_t launch_bloop_ctl(const BBuffers& b, cudaGraphConditionalHandle h, int max_chunks, cudaStream_t s) {
  k_bloop_ctl<<<1, 32, 0, s>>>(b.st, h, max_chunks);
  return cudaGetLastError();
}

cudaError_t launch_bchunk_end(const BBuffers& b, int chunk_len, cudaStream_t s) {
  k_bchunk_end<<<1, 32, 0, s>>>(b, chunk_len);
  return cudaGetLastError();
}

}  // namespace bvls
