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
//   k_bcompact  retires finished instances from the active list (stable).
#include <cuda_bf16.h>

#include "batch.cuh"
#include "common.cuh"
#include "umma.cuh"

namespace bvls {

namespace {

constexpr unsigned kFull = 0xffffffffu;
constexpr int kStageBytes = 2 * kBTile * kBChunk * 2;  // A and B tiles of one K chunk (bf16)

__device__ __forceinline__ double warp_sum_dd(double v) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(kFull, v, o);
  return v;
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
    float xf = 0.f;
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
      xf = (float)x;
      xf = fminf(fmaxf(xf, p.lf[j]), p.uf[j]);
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
// Grid (npad / 128 coordinate tiles, ceil(B / 128) instance tiles), 128 threads, one CTA per
// SM (128 KB of stages).  Operand K chunks of 64 stream through kBStages shared-memory
// stages with 16-byte asynchronous copies; thread 0 issues four 128x128x16 MMAs per chunk and
// commits them to the stage's mbarrier, which releases the stage for the chunk kBStages
// later.  The epilogue warps read the accumulator rows of their 32 coordinates from TMEM.
__global__ void __launch_bounds__(kBStepThreads, 1) k_bstep(BParams p, BBuffers b, int jrel) {
  BState* st = b.st;
  if (st->done) return;
  const int n_act = st->n_act;
  const int mt = blockIdx.x, nt = blockIdx.y;
  if (nt * kBTile >= n_act) return;
  extern __shared__ __align__(1024) unsigned char smem[];
  __shared__ __align__(8) uint64_t mbar[kBStages];
  __shared__ uint32_t s_tmem;
  __shared__ int s_inst[kBTile];
  __shared__ float s_beta[kBTile];
  __shared__ float s_l[kBTile], s_u[kBTile];
  __shared__ float s_dot[kBStepThreads / 32][kBTile];

  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int k = st->kbase + jrel;
  const int s = k & 1;
  const int MT = p.npad / kBTile;
  {
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
      const float T = (p.restart && dsum < 0.f) ? 1.f : 0.5f * (1.f + sqrtf(1.f + 4.f * tp * tp));
      const float tn = 0.5f * (1.f + sqrtf(1.f + 4.f * T * T));
      beta = (T - 1.f) / tn;
      if (mt == 0) b.tval[s][inst] = T;
    }
    s_beta[tid] = beta;
    const int jj = mt * kBTile + tid;
    s_l[tid] = jj < p.n ? p.lf[jj] : 0.f;
    s_u[tid] = jj < p.n ? p.uf[jj] : 0.f;
  }
  if (warp == 0) tmem_alloc(&s_tmem, kBTile);
  if (tid == 0) {
    for (int q = 0; q < kBStages; ++q) mbar_init(&mbar[q], 1);
    fence_barrier_init();
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = s_tmem;

  const int nch = p.npad / kBChunk;
  const __nv_bfloat16* Hrow = p.H + (size_t)mt * kBTile * p.npad;
  const __nv_bfloat16* Dsrc = b.D[s];
  auto load_chunk = [&](int c) {
    unsigned char* sa = smem + (size_t)(c % kBStages) * kStageBytes;
    unsigned char* sb = sa + kStageBytes / 2;
    const int kofs = c * kBChunk;
#pragma unroll
    for (int t = 0; t < (kBTile * 8) / kBStepThreads; ++t) {
      const int q = tid + t * kBStepThreads;
      const int r = ((q >> 6) << 3) | (q & 7);
      const int kc = (q >> 3) & 7;
      const uint32_t off = core_offset(r, kc);
      cp_async16(sa + off, Hrow + (size_t)r * p.npad + kofs + kc * 8);
      const int inst = s_inst[r];
      const int row = inst >= 0 ? inst : p.B;  // row B of D is zero
      cp_async16(sb + off, Dsrc + (size_t)row * p.npad + kofs + kc * 8);
    }
    cp_async_commit();
  };
  const int npro = nch < kBStages ? nch : kBStages;
  for (int c = 0; c < npro; ++c) load_chunk(c);
  const uint32_t idesc = umma_idesc_bf16(kBTile, kBTile);
  bool ok = true;
  for (int c = 0; c < nch; ++c) {
    const int ahead = min(kBStages - 1, nch - 1 - c);
    if (ahead >= 3) cp_async_wait<3>();
    else if (ahead == 2) cp_async_wait<2>();
    else if (ahead == 1) cp_async_wait<1>();
    else cp_async_wait<0>();
    fence_proxy_async_smem();
    __syncthreads();
    if (tid == 0) {
      tc_fence_after();
      const uint32_t sa = smem_u32(smem + (size_t)(c % kBStages) * kStageBytes);
      const uint32_t sb = sa + kStageBytes / 2;
#pragma unroll
      for (int kk = 0; kk < kBChunk / 16; ++kk)
        umma_bf16(tmem, umma_smem_desc(sa + kk * 256), umma_smem_desc(sb + kk * 256), idesc, c > 0 || kk > 0);
      umma_commit(&mbar[c % kBStages]);
    }
    if (c + kBStages < nch) {
      if (!mbar_wait(&mbar[c % kBStages], (c / kBStages) & 1)) ok = false;
      load_chunk(c + kBStages);
    }
  }
  {
    const int cl = nch - 1;
    if (!mbar_wait(&mbar[cl % kBStages], (cl / kBStages) & 1)) ok = false;
  }
  tc_fence_after();

  // epilogue: thread = coordinate jg of this tile, 32 instance columns per TMEM load
  const int i = warp * 32 + lane;
  const int jg = mt * kBTile + i;
  const bool jv = jg < p.n;
  const float lj = s_l[i], uj = s_u[i];
  const float invL = p.invLf;
  const float* __restrict__ Gp = b.G[s ^ 1];
  float* Gc = b.G[s];
  const float* __restrict__ Xc = b.X[s];
  float* Xn = b.X[s ^ 1];
  __nv_bfloat16* Dn = b.D[s ^ 1];
  for (int c0 = 0; c0 < kBTile; c0 += 32) {
    if (s_inst[c0] < 0) break;  // active instances are packed at the front of the tile
    float acc[32];
    tmem_ld32(tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)c0, acc);
    float dv[32];
#pragma unroll
    for (int c8 = 0; c8 < 32; c8 += 8) {
      float gp[8], xk[8], xp[8];
      uint8_t fl[8];
#pragma unroll
      for (int cc = 0; cc < 8; ++cc) {  // loads first: eight instances in flight
        const int inst = s_inst[c0 + c8 + cc];
        gp[cc] = 0.f;
        xk[cc] = 0.f;
        xp[cc] = 0.f;
        fl[cc] = 1;
        if (inst >= 0 && jv) {
          const size_t o = (size_t)inst * p.npad + jg;
          gp[cc] = Gp[o];
          xk[cc] = Xc[o];
          xp[cc] = Xn[o];
          fl[cc] = b.flags[o];
        }
      }
#pragma unroll
      for (int cc = 0; cc < 8; ++cc) {
        const int inst = s_inst[c0 + c8 + cc];
        dv[c8 + cc] = 0.f;
        if (inst >= 0 && jv) {
          const size_t o = (size_t)inst * p.npad + jg;
          const float gk = gp[cc] - acc[c8 + cc];
          float xn = xk[cc];
          if (!fl[cc]) {
            const float be = s_beta[c0 + c8 + cc];
            const float gv = fmaf(be, gk - gp[cc], gk);            // (1 + b) g_k - b g_{k-1}
            const float v = fmaf(be, xk[cc] - xp[cc], xk[cc]);     // x_k + b (x_k - x_{k-1})
            xn = fminf(fmaxf(fmaf(gv, invL, v), lj), uj);
            dv[c8 + cc] = gv * (xn - xk[cc]);
          }
          Gc[o] = gk;
          Xn[o] = xn;
          Dn[o] = __float2bfloat16_rn(xn - xk[cc]);
        }
      }
    }
    // restart-test partials: transpose-reduce 32 values over the 32 lanes; lane L ends with
    // the warp's sum for instance column c0 + L
#pragma unroll
    for (int o = 16; o >= 1; o >>= 1) {
      const bool up = (lane & o) != 0;
#pragma unroll
      for (int t = 0; t < o; ++t) {
        const float send = up ? dv[t] : dv[t + o];
        const float keep = up ? dv[t + o] : dv[t];
        dv[t] = keep + __shfl_xor_sync(kFull, send, o);
      }
    }
    s_dot[warp][c0 + lane] = dv[0];
  }
  tc_fence_before();
  __syncthreads();
  {
    const int inst = s_inst[tid];
    if (inst >= 0) {
      float d = 0.f;
#pragma unroll
      for (int w = 0; w < kBStepThreads / 32; ++w) d += s_dot[w][tid];
      b.dotp[s][(size_t)mt * p.B + inst] = d;
    }
  }
  if (warp == 0) tmem_dealloc(tmem, kBTile);
  if (!ok && tid == 0) atomicOr(&st->error, 1);
  if (tid == 0 && mt == 0 && nt == 0) st->sum_step += (double)n_act;
}

size_t bstep_smem_bytes() { return (size_t)kBStages * kStageBytes; }

cudaError_t launch_bstep(const BParams& p, const BBuffers& b, int j, cudaStream_t s) {
  dim3 grid(p.npad / kBTile, (p.B + kBTile - 1) / kBTile);
  k_bstep<<<grid, kBStepThreads, bstep_smem_bytes(), s>>>(p, b, j);
  return cudaGetLastError();
}

// ------------------------------------------------------------------ evaluation
// kBEvalInst instances per CTA (A is read once for all of them), 256 threads.
//   phase 1  r = y - A x_k per row (thread = row), double-float, skipping zero x_j;
//   phase 2  g_j = a_j^T r for preserved j (warp = column, lanes over rows), PREC products;
//   phase 3  gap sums and the step (thread = coordinate);
//   phase 4  sphere test; phase 5  outputs of the instances that stop.
template <int PREC>
__global__ void __launch_bounds__(kBEvalThreads) k_beval(BParams p, BBuffers b, int jrel) {
  BState* st = b.st;
  if (st->done) return;
  const int n_act = st->n_act;
  const int i0 = blockIdx.x * kBEvalInst;
  if (i0 >= n_act) return;
  extern __shared__ float2 sr[];  // [m][kBEvalInst] residual (hi, lo)
  __shared__ int s_inst[kBEvalInst];
  __shared__ float s_beta[kBEvalInst];
  __shared__ float sx[kBEvalInst][33];
  __shared__ double s_red[kBEvalThreads / 32][kBEvalInst][5];
  __shared__ double s_q[kBEvalInst][8];  // P, ||y||^2, eta_g, eps, rr, eta, gap, X1
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

  // ---- phase 1: r = y - A x_k, one block of kBEvalThreads rows at a time
  const float* __restrict__ Xc = b.X[s];
  double pv[kBEvalInst], yv[kBEvalInst];
#pragma unroll
  for (int bb = 0; bb < kBEvalInst; ++bb) {
    pv[bb] = 0.0;
    yv[bb] = 0.0;
  }
  for (int r0 = 0; r0 < p.m; r0 += kBEvalThreads) {
    const int i = r0 + tid;
    float qs[kBEvalInst], qc[kBEvalInst];
#pragma unroll
    for (int bb = 0; bb < kBEvalInst; ++bb) {
      qs[bb] = 0.f;
      qc[bb] = 0.f;
    }
    for (int jc = 0; jc < p.n; jc += 32) {
      {
        const int bb = tid >> 5, jj = tid & 31;
        const int inst = s_inst[bb];
        sx[bb][jj] = (inst >= 0 && jc + jj < p.n) ? Xc[(size_t)inst * p.npad + jc + jj] : 0.f;
      }
      __syncthreads();
      const int jn = min(32, p.n - jc);
      for (int jj = 0; jj < jn; ++jj) {
        float xv[kBEvalInst];
        bool any = false;
#pragma unroll
        for (int bb = 0; bb < kBEvalInst; ++bb) {
          xv[bb] = sx[bb][jj];
          any |= xv[bb] != 0.f;
        }
        if (!any || i >= p.m) continue;
        const float a = p.A[(size_t)(jc + jj) * p.lda + i];
#pragma unroll
        for (int bb = 0; bb < kBEvalInst; ++bb)
          if (xv[bb] != 0.f) df_fma(qs[bb], qc[bb], a, xv[bb], 0.f);
      }
      __syncthreads();
    }
    if (i < p.m) {
#pragma unroll
      for (int bb = 0; bb < kBEvalInst; ++bb) {
        const int inst = s_inst[bb];
        float rh = 0.f, rl = 0.f;
        if (inst >= 0) {
          const float y = b.Y[(size_t)inst * p.lda + i];
          float dh, de;
          two_sum(y, -qs[bb], dh, de);
          de -= qc[bb];
          two_sum(dh, de, rh, rl);
          const double rv = (double)rh + (double)rl;
          pv[bb] += 0.5 * rv * rv;
          yv[bb] += (double)y * (double)y;
        }
        sr[(size_t)i * kBEvalInst + bb] = make_float2(rh, rl);
      }
    }
  }
#pragma unroll
  for (int bb = 0; bb < kBEvalInst; ++bb) {
    pv[bb] = warp_sum_dd(pv[bb]);
    yv[bb] = warp_sum_dd(yv[bb]);
  }
  if (lane == 0) {
#pragma unroll
    for (int bb = 0; bb < kBEvalInst; ++bb) {
      s_red[warp][bb][0] = pv[bb];
      s_red[warp][bb][1] = yv[bb];
    }
  }
  __syncthreads();
  if (tid < kBEvalInst) {
    double P = 0.0, Y2 = 0.0;
    for (int w = 0; w < kBEvalThreads / 32; ++w) {
      P += s_red[w][tid][0];
      Y2 += s_red[w][tid][1];
    }
    s_q[tid][0] = P;
    s_q[tid][1] = Y2;
    s_q[tid][2] = p.Cg * sqrt(2.0 * P) * (1.0 + 1e-6);  // eta_g: rounding of a_j^T r per unit norm
  }
  __syncthreads();

  // ---- phase 2: correlations of the preserved coordinates
  double epsm = 0.0;  // lane bb < kBEvalInst: translation step candidate of instance bb
  {
    const double eta_g = lane < kBEvalInst ? s_q[lane][2] : 0.0;
    const int inst_l = lane < kBEvalInst ? s_inst[lane] : -1;
    for (int j = warp; j < p.n; j += kBEvalThreads / 32) {
      const bool need_l = inst_l >= 0 && b.flags[(size_t)inst_l * p.npad + j] == 0;
      const unsigned need = __ballot_sync(kFull, need_l);
      if (!need) continue;
      const float* __restrict__ col = p.A + (size_t)j * p.lda;
      float sa[kBEvalInst], ca[kBEvalInst];
#pragma unroll
      for (int bb = 0; bb < kBEvalInst; ++bb) {
        sa[bb] = 0.f;
        ca[bb] = 0.f;
      }
      for (int i = lane; i < p.m; i += 32) {
        const float a = col[i];
        const float4* rr = reinterpret_cast<const float4*>(sr + (size_t)i * kBEvalInst);
#pragma unroll
        for (int h = 0; h < kBEvalInst / 2; ++h) {
          const float4 v = rr[h];
          if (PREC == kX2) {
            df_fma(sa[2 * h], ca[2 * h], a, v.x, v.y);
            df_fma(sa[2 * h + 1], ca[2 * h + 1], a, v.z, v.w);
          } else {
            sa[2 * h] = fmaf(a, v.x, sa[2 * h]);
            sa[2 * h + 1] = fmaf(a, v.z, sa[2 * h + 1]);
          }
        }
      }
      float gs = 0.f, gc = 0.f;
#pragma unroll
      for (int bb = 0; bb < kBEvalInst; ++bb) {
        float x = sa[bb], c = ca[bb];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
          const float ox = __shfl_xor_sync(kFull, x, o);
          if (PREC == kX2) {
            const float oc = __shfl_xor_sync(kFull, c, o);
            df_add(x, c, ox, oc);
          } else {
            x += ox;
          }
        }
        if (lane == bb) {
          gs = x;
          gc = PREC == kX2 ? c : 0.f;
        }
      }
      if (need_l) {
        const float2 g2 = df2_norm(gs, gc);
        b.Ge[(size_t)inst_l * p.npad + j] = g2;
        if (trans && p.jinf[j]) {
          const double nr = p.nrm[j];
          if (nr > 0.0) {
            const double den = -p.w[j] - p.gamma_w * nr * p.t_norm;
            epsm = fmax(epsm, fmax(df2_to_double(g2) + eta_g * nr, 0.0) / den);
          }
        }
      }
    }
  }
  if (lane < kBEvalInst) s_red[warp][lane][4] = epsm;
  __syncthreads();
  if (tid < kBEvalInst) {
    double e = 0.0;
    for (int w = 0; w < kBEvalThreads / 32; ++w) e = fmax(e, s_red[w][tid][4]);
    s_q[tid][3] = trans ? e : 0.0;
  }
  __syncthreads();

  // ---- phase 3: gap sums (nonnegative-sum form of P - D) and the step
  {
    const float* __restrict__ Gp = b.G[s ^ 1];
    float* Gc = b.G[s];
    float* Xn = b.X[s ^ 1];
    __nv_bfloat16* Dn = b.D[s ^ 1];
    const float invL = p.invLf;
    for (int bb = 0; bb < kBEvalInst; ++bb) {
      const int inst = s_inst[bb];
      if (inst < 0) break;  // active instances are packed at the front
      const float be = s_beta[bb];
      const double eps = s_q[bb][3];
      double va = 0.0, vc = 0.0, vx = 0.0, vd = 0.0, vp = 0.0;
      for (int j = tid; j < p.n; j += kBEvalThreads) {
        const size_t o = (size_t)inst * p.npad + j;
        const double nr = p.nrm[j];
        const float xk = Xc[o];
        vx += fabs((double)xk) * nr;
        if (b.flags[o]) {
          Xn[o] = xk;
          Dn[o] = __float2bfloat16_rn(0.f);
          continue;
        }
        vp += 1.0;
        const float2 g2 = b.Ge[o];
        if (p.dual_mode != kZero) {
          const double x = (double)xk, lj = p.l[j];
          const double gt = df2_to_double(g2) + (trans ? eps * p.w[j] : 0.0);
          if (p.jinf[j]) {
            va += (x - lj) * fmax(-gt, 0.0);
            vc += (x - lj) * nr;
          } else {
            const double uj = p.u[j];
            va += (uj - x) * fmax(gt, 0.0) + (x - lj) * fmax(-gt, 0.0);
            vc += fmax(uj - x, x - lj) * nr;
          }
        }
        const float gk = g2.x;
        const float gp = Gp[o], xp = Xn[o];
        const float gv = fmaf(be, gk - gp, gk);
        const float v = fmaf(be, xk - xp, xk);
        const float xn = fminf(fmaxf(fmaf(gv, invL, v), p.lf[j]), p.uf[j]);
        Gc[o] = gk;
        Xn[o] = xn;
        Dn[o] = __float2bfloat16_rn(xn - xk);
        vd += (double)gv * (double)(xn - xk);
      }
      va = warp_sum_dd(va);
      vc = warp_sum_dd(vc);
      vx = warp_sum_dd(vx);
      vd = warp_sum_dd(vd);
      vp = warp_sum_dd(vp);
      if (lane == 0) {
        s_red[warp][bb][0] = va;
        s_red[warp][bb][1] = vc;
        s_red[warp][bb][2] = vx;
        s_red[warp][bb][3] = vd;
        s_red[warp][bb][4] = vp;
      }
    }
  }
  __syncthreads();
  if (tid < kBEvalInst) {
    double a = 0.0, c = 0.0, x1 = 0.0, d = 0.0, np = 0.0;
    for (int w = 0; w < kBEvalThreads / 32; ++w) {
      a += s_red[w][tid][0];
      c += s_red[w][tid][1];
      x1 += s_red[w][tid][2];
      d += s_red[w][tid][3];
      np += s_red[w][tid][4];
    }
    const int inst = s_inst[tid];
    int stop = 0;
    if (inst >= 0) {
      const double P = s_q[tid][0];
      const double eps = s_q[tid][3];
      const double rnorm = sqrt(2.0 * P) * (1.0 + 1e-6);
      const double eta = p.Cg * rnorm + (trans ? eps * p.gamma_w * p.t_norm : 0.0);
      const double E_r = p.Cf * x1 + p.Csub * (rnorm + sqrt(s_q[tid][1]) + x1);
      double gap;
      if (p.dual_mode == kZero) {
        gap = 0.5 * (rnorm + E_r) * (rnorm + E_r);
      } else {
        const double dd = E_r + eps * p.t_norm;
        gap = a + eta * c + 0.5 * dd * dd;
      }
      gap *= (1.0 + 1e-12);
      s_q[tid][4] = sqrt(2.0 * gap) * (1.0 + 1e-12) + eta;  // radius + margin, per unit ||a_j||
      s_q[tid][6] = gap;
      stop = (gap < p.tol || k >= p.max_iter) ? 1 : 0;
      b.dotp[s][inst] = (float)d;
      for (int t = 1; t < MT; ++t) b.dotp[s][(size_t)t * p.B + inst] = 0.f;
      atomicAdd(&st->sum_pres, np);
    }
    s_stop[tid] = stop;
    s_q[tid][7] = np;
  }
  __syncthreads();

  // ---- phase 4: sphere test (Eq. (safe_rule)); a coordinate is fixed once x_k and x_{k+1}
  // both sit at the bound the test gives
  if (p.screening && p.dual_mode != kZero) {
    const float* __restrict__ Xn = b.X[s ^ 1];
    for (int j = tid; j < p.n; j += kBEvalThreads) {
      const double nr = p.nrm[j];
      if (!(nr > 0.0)) continue;
      const double wj = trans ? p.w[j] : 0.0;
      const int ji = p.jinf[j];
      const float ljf = p.lf[j], ujf = p.uf[j];
#pragma unroll
      for (int bb = 0; bb < kBEvalInst; ++bb) {
        const int inst = s_inst[bb];
        if (inst < 0) continue;
        const size_t o = (size_t)inst * p.npad + j;
        if (b.flags[o]) continue;
        const double gt = df2_to_double(b.Ge[o]) + s_q[bb][3] * wj;
        const double thr = s_q[bb][4] * nr * (1.0 + 1e-12);
        int pin = 0;
        float bnd = 0.f;
        if (gt < -thr) {
          pin = 1;
          bnd = ljf;
        } else if (!ji && gt > thr) {
          pin = 2;
          bnd = ujf;
        }
        if (pin && Xc[o] == bnd && Xn[o] == bnd) {
          b.flags[o] = (uint8_t)pin;
          atomicAdd(&s_pins[bb], 1);
        }
      }
    }
    __syncthreads();
  }

  // ---- phase 5: outputs of the instances that stop at this evaluation
  for (int j = tid; j < p.n; j += kBEvalThreads) {
#pragma unroll
    for (int bb = 0; bb < kBEvalInst; ++bb) {
      const int inst = s_inst[bb];
      if (inst < 0 || !s_stop[bb]) continue;
      const size_t o = (size_t)inst * p.npad + j;
      const uint8_t f = b.flags[o];
      double x = f == 1 ? p.l[j] : f == 2 ? p.u[j] : fmin(fmax((double)Xc[o], p.l[j]), p.u[j]);
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

size_t beval_smem_bytes(int m) { return (size_t)m * kBEvalInst * sizeof(float2); }

cudaError_t launch_beval(const BParams& p, const BBuffers& b, int j, int precision, cudaStream_t s) {
  const int grid = (p.B + kBEvalInst - 1) / kBEvalInst;
  const size_t sm = beval_smem_bytes(p.m);
  if (precision == kX2) k_beval<kX2><<<grid, kBEvalThreads, sm, s>>>(p, b, j);
  else k_beval<kF32><<<grid, kBEvalThreads, sm, s>>>(p, b, j);
  return cudaGetLastError();
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

cudaError_t batch_configure(int m) {
  cudaError_t e = cudaFuncSetAttribute(k_bstep, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bstep_smem_bytes());
  if (e != cudaSuccess) return e;
  e = cudaFuncSetAttribute(k_beval<kX2>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)beval_smem_bytes(m));
  if (e != cudaSuccess) return e;
  return cudaFuncSetAttribute(k_beval<kF32>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)beval_smem_bytes(m));
}

cudaError_t launch_bcompact(const BParams& p, const BBuffers& b, cudaStream_t s) {
  k_bcompact<<<1, 1024, 0, s>>>(p, b);
  return cudaGetLastError();
}

__global__ void k_bchunk_end(BBuffers b, int chunk_len) {
  if (threadIdx.x == 0 && blockIdx.x == 0) b.st->kbase += chunk_len;
}

cudaError_t launch_bchunk_end(const BBuffers& b, int chunk_len, cudaStream_t s) {
  k_bchunk_end<<<1, 32, 0, s>>>(b, chunk_len);
  return cudaGetLastError();
}

}  // namespace bvls
