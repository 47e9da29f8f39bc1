// Least-squares solve of min ||M a - h|| (paper Eq. multilevel_ls).
//
// The paper's solver is LSQR (§3 last paragraph; §4.1 "Optimisation and
// solvers": SciPy LSQR, up to 15000 iterations).  This file runs LSQR
// (Paige & Saunders, ACM TOMS 8(1), 1982, the bidiagonalisation recurrences
// and the stopping estimates of its §5-6) on the GPU with an optional
// right preconditioner that the paper does not use: block-Jacobi over
// subdomains, P = blockdiag(R_j^{-1}) with R_j^T R_j = G_jj + eps tr(G_jj)/K I
// the shifted Cholesky factor of the diagonal Gram block G_jj = M_j^T M_j.
// LSQR then runs on A = M P and returns a = P y.
//
// Data flow of one iteration (all scalars stay on the device), fused path:
//   k_fused_pipe    u' = M t - (alpha/beta) u, the per-unit partials of M^T u'
//                   and the ||u'||^2 partials, in one read of the panels
//                   (k_fused_pipe_df for DF32 panels, k_fused without a ring)
//   k_panel_chunks  fixed slices of each panel's partials; block 0 commits the
//                   staged scalars and forms beta^2
//   FP32 / DF32 panels: k_lsqr_tail_tri -- the previous iteration's deferred
//                   w / x update, v' = X z / beta - beta v, t' = X^T v' (the
//                   next pass scales M t' by 1/alpha), the recurrence in the
//                   last block to finish; k_lsqr_finish after the loop
//   FP64 panels:    k_panel_T2 (v'), then k_update_precond (recurrence, v, w,
//                   x, t = X^T v)
// Without the fused plan (more than 32 covering panels or K > 128) an
// iteration is k_precond, k_gather, k_entry_T, k_panel_T, k_update.
// Every reduction is a fixed-order sum, so results are bitwise reproducible
// from run to run.
#include <algorithm>
#include <cmath>
#include <cstdlib>
#include <map>
#include <mutex>
#include <tuple>
#include <type_traits>

#include "elmfb_internal.cuh"
#include "sm100_ptx.cuh"

namespace {

constexpr int kGatherBlocks = 1216;   // 152 SMs x 8
constexpr int kGatherThreads = 256;
constexpr int kScal = 48;             // device scalar slots

// scalar slots in d_scal: [0, 24) committed values read by the kernels of an
// iteration, [24, 48) staged values written by the kernel that runs the
// recurrence; the next iteration's first reader of committed values
// (k_panel_chunks, or k_precond without the fused plan) commits staged ->
// committed.
constexpr int kStage = 24;
enum {
  S_ALPHA = 0, S_BETA, S_RHOBAR, S_PHIBAR, S_ANORM2, S_RNORM, S_ARNORM, S_ITER, S_BNORM,
  S_XNORM2, S_BAD, S_PHI_RHO, S_THETA_RHO,
  S_BSQ,     // staged: sum of the fused pass's ||u'||^2 partials (beta^2), formed once
  S_TSCALE,  // 1/alpha: the fused pass's factor on M t' (mode 2, t' = P v' unnormalised)
  S_GKCAP,   // capacity (entries) of the Golub-Kahan record after the 2 kScal slots
  // the stopping tests on the device (LSQR with the pair tail, S_STOP_ON):
  S_DONE,    // set by the recurrence once a test is met; the next iterations' kernels return
  S_ARN0,    // ||(M P)^T h|| = alpha_1 beta_1, staged at the start
  S_STOP_ON, S_NTOL, S_BTOL, S_ATOL   // set by the host, both copies
};
static_assert(S_ATOL < kStage, "scalar slots");

// Record alpha_{i+1}, beta_{i+1} of LSQR step i (i = the new iteration count;
// 0 = the start: alpha_1, beta_1) after the scalar slots, while it fits: the
// lower bidiagonal B_k of Golub-Kahan (Paige & Saunders 1982, §3), whose
// extreme singular values estimate those of the operator.
__device__ __forceinline__ void record_bidiagonal(double* __restrict__ scal, double iter,
                                                  double alpha, double beta) {
  const int cap = (int)scal[kStage + S_GKCAP];
  const int it = (int)iter;
  if (it >= 0 && it < cap) {
    double* gk = scal + 2 * kScal;
    gk[2 * it] = alpha;
    gk[2 * it + 1] = beta;
  }
}

template <class T>
__device__ __forceinline__ double warp_sum(double v) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}
__device__ __forceinline__ float warp_sumf(float v) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// block-wide fixed-order sum; every thread gets the result.  Warp 0 alone
// reduces the per-warp sums (FP64 work in every thread is costly on GB300,
// whose FP64 rate is 1/64 of FP32).
__device__ double block_sum(double v, double* sh) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
  v = warp_sum<double>(v);
  __syncthreads();
  if (lane == 0) sh[wid] = v;
  __syncthreads();
  if (wid == 0) {
    double s = lane < nw ? sh[lane] : 0.0;
    s = warp_sum<double>(s);
    if (lane == 0) sh[32] = s;
  }
  __syncthreads();
  const double r = sh[32];
  __syncthreads();
  return r;
}

// sum of n partials by warp 0 of the block in a fixed order (lane-strided
// sums, then a fixed xor tree); the result is broadcast through shared memory
// so that every block of a grid computes the identical value.
__device__ double block_partial_sum(const double* __restrict__ part, int n, double* sh) {
  if (threadIdx.x < 32) {
    double v = 0.0;
    for (int i = threadIdx.x; i < n; i += 32) v += part[i];
    v = warp_sum<double>(v);
    if (threadIdx.x == 0) *sh = v;
  }
  __syncthreads();
  const double r = *sh;
  __syncthreads();
  return r;
}

// (s, c) += hi - lo in float-float arithmetic (TwoSum, then a fast
// renormalisation; Dekker 1971 / Knuth TAOCP 4.2.2): FP32 pipes only, about
// 2^-44 relative, used to sum compensated FP32 partials without FP64 work.
__device__ __forceinline__ void ff_add(float& s, float& c, float hi, float lo) {
  const float t = s + hi;
  const float bp = t - s;
  const float e = (s - (t - bp)) + (hi - bp);
  c += e - lo;
  s = t + c;
  c = c - (s - t);
}
// FP32 (hi, lo) pair stored in the 8 bytes of partial idx
__device__ __forceinline__ float2 partial_pair(const double* part, int64_t idx) {
  return reinterpret_cast<const float2*>(part)[idx];
}
// FP32 copy of an FP64 vector (the fused pass's operand for FP32 panels)
__global__ void k_to_float(const double* __restrict__ x, float* __restrict__ y, int64_t n) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    y[i] = (float)x[i];
}

// FP32-pair copy of an FP64 vector (the fused pass's operand for DF32 panels)
__global__ void k_to_df(const double* __restrict__ x, float2* __restrict__ y, int64_t n) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const float hi = __double2float_rn(x[i]);
    y[i] = make_float2(hi, __double2float_rn(x[i] - (double)hi));
  }
}

// ------------------------------------------------------ float-float (DF32) ---
// Error-free transformations on the FP32 pipes (Dekker 1971; Knuth TAOCP
// 4.2.2; the FMA form of the exact product): a value is a pair hi + lo.
// __fmul_rn / __fadd_rn keep the compiler from contracting a product into a
// following add, which would break the exactness of the transformations.

// (S, C) += (xh + xl) (yh + yl), renormalised (|C| <= ulp(S) / 2); the
// xl yl term (below 2^-48 relative) is dropped.
__device__ __forceinline__ void df_acc(float& S, float& C, float xh, float xl, float yh,
                                       float yl) {
  const float p = __fmul_rn(xh, yh);
  float e = fmaf(xh, yh, -p);
  e = fmaf(xh, yl, fmaf(xl, yh, e));
  const float s = __fadd_rn(S, p);
  const float bp = __fadd_rn(s, -S);
  const float t = __fadd_rn(__fadd_rn(S, -__fadd_rn(s, -bp)), __fadd_rn(p, -bp));
  C = __fadd_rn(C, __fadd_rn(t, e));
  S = __fadd_rn(s, C);
  C = __fadd_rn(C, -__fadd_rn(S, -s));
}

// (ah + al) + (bh + bl), renormalised
__device__ __forceinline__ float2 df_add(float2 a, float2 b) {
  const float s = __fadd_rn(a.x, b.x);
  const float bp = __fadd_rn(s, -a.x);
  float t = __fadd_rn(__fadd_rn(a.x, -__fadd_rn(s, -bp)), __fadd_rn(b.x, -bp));
  t = __fadd_rn(t, __fadd_rn(a.y, b.y));
  const float hi = __fadd_rn(s, t);
  return make_float2(hi, __fadd_rn(t, -__fadd_rn(hi, -s)));
}

__device__ __forceinline__ float2 df_shfl_xor(float2 v, int m) {
  return make_float2(__shfl_xor_sync(0xffffffffu, v.x, m), __shfl_xor_sync(0xffffffffu, v.y, m));
}

// FP64 value split into an FP32 pair
__device__ __forceinline__ float2 df_split(double v) {
  const float hi = __double2float_rn(v);
  return make_float2(hi, __double2float_rn(v - (double)hi));
}

// X_j as FP32 pairs (FP32 and DF32 panels), packed lower triangle: row m of
// panel j holds X_mi, i = 0..m, from pair m (m + 1) / 2 on.  Panels are
// tri_pairs(K) pairs apart (an even count, so that each one starts on a
// 16-byte boundary and moves into shared memory as one bulk copy).
__host__ __device__ __forceinline__ int64_t tri_pairs(int K) {
  return ((int64_t)K * (K + 1) / 2 + 1) & ~int64_t(1);
}

// sum of 4 per-lane pairs over the warp; lane 8r holds the total of pair r
__device__ __forceinline__ float2 warp_sum4_df(float2 v0, float2 v1, float2 v2, float2 v3,
                                               int lane) {
  const bool b4 = lane & 16, b3 = lane & 8;
  const float2 k0 = df_add(b4 ? v2 : v0, df_shfl_xor(b4 ? v0 : v2, 16));
  const float2 k1 = df_add(b4 ? v3 : v1, df_shfl_xor(b4 ? v1 : v3, 16));
  float2 k = df_add(b3 ? k1 : k0, df_shfl_xor(b3 ? k0 : k1, 8));
  k = df_add(k, df_shfl_xor(k, 4));
  k = df_add(k, df_shfl_xor(k, 2));
  k = df_add(k, df_shfl_xor(k, 1));
  return k;
}

// FPL consecutive pairs p[0..FPL) (vector loads when whole; zeros past rem)
template <int FPL>
__device__ __forceinline__ void load_slice_df(const float2* p, float2 (&x)[FPL], bool whole,
                                              int rem) {
  if (whole) {
    if constexpr (FPL % 2 == 0) {
#pragma unroll
      for (int j = 0; j < FPL; j += 2) {
        const float4 v = reinterpret_cast<const float4*>(p)[j / 2];
        x[j] = make_float2(v.x, v.y);
        x[j + 1] = make_float2(v.z, v.w);
      }
    } else {
#pragma unroll
      for (int j = 0; j < FPL; ++j) x[j] = p[j];
    }
  } else {
#pragma unroll
    for (int j = 0; j < FPL; ++j) x[j] = j < rem ? p[j] : make_float2(0.f, 0.f);
  }
}


// ------------------------------------------------------------ Gram diag -----
// Partial sums of the upper triangle of P^T P over one chunk of panel rows.
// Thread t owns the 4x4 tile (ti, tj), ti <= tj, of the Gram block: per row it
// reads two float4 from shared memory and does 16 FMAs.  Products are summed
// in FP32 over 16 rows, those sums Kahan-compensated in FP32 over the chunk,
// and the result stored in FP64 (upper triangle, row-major, K(K+1)/2 values).
// A diagonal-Gram chunk is a run of 16-row steps of one panel; step (e, p0)
// covers rows p0 .. p0+15 of entry e (cell c, covering panel w), which sit at
// element rows entry_base[e] + p m_c in the cell-interleaved storage.
struct DiagStepRows {
  int64_t row0;   // element row of the step's first row
  int64_t mK;     // element stride between its rows (m_c K)
};
__device__ __forceinline__ DiagStepRows diag_step(const int2* __restrict__ steps,
                                                  const int64_t* __restrict__ entry_base,
                                                  const int* __restrict__ entry_cell,
                                                  const int* __restrict__ cover_off, int q,
                                                  int K) {
  const int2 st = steps[q];
  const int c = entry_cell[st.x];
  const int64_t m = cover_off[c + 1] - cover_off[c];
  return {entry_base[st.x] + (int64_t)st.y * m, m * K};
}

// Four consecutive elements from shared memory (16-byte aligned) as vector
// loads: a lane's four scalars at a 16-byte lane stride would meet 4-way bank
// conflicts, one 16-byte load per lane meets none.
__device__ __forceinline__ void lds4(const float* p, float (&x)[4]) {
  const float4 v = *reinterpret_cast<const float4*>(p);
  x[0] = v.x, x[1] = v.y, x[2] = v.z, x[3] = v.w;
}
__device__ __forceinline__ void lds4(const double* p, double (&x)[4]) {
  const double2 v0 = reinterpret_cast<const double2*>(p)[0];
  const double2 v1 = reinterpret_cast<const double2*>(p)[1];
  x[0] = v0.x, x[1] = v0.y, x[2] = v1.x, x[3] = v1.y;
}
__device__ __forceinline__ void lds4(const float2* p, float2 (&x)[4]) {
  const float4 v0 = reinterpret_cast<const float4*>(p)[0];
  const float4 v1 = reinterpret_cast<const float4*>(p)[1];
  x[0] = make_float2(v0.x, v0.y), x[1] = make_float2(v0.z, v0.w);
  x[2] = make_float2(v1.x, v1.y), x[3] = make_float2(v1.z, v1.w);
}

template <class T>
__global__ void __launch_bounds__(544) k_gram_diag_partial(const T* __restrict__ panels, int K,
                                                            const int4* __restrict__ chunks,
                                                            const int2* __restrict__ steps,
                                                            const int64_t* __restrict__ entry_base,
                                                            const int* __restrict__ entry_cell,
                                                            const int* __restrict__ cover_off,
                                                            double* __restrict__ partial) {
  extern __shared__ __align__(128) unsigned char smraw[];
  T* sm = reinterpret_cast<T*>(smraw);   // [16][Kp]
  const int4 ch = chunks[blockIdx.x];     // (panel, first step, steps, -)
  const int Kp = (K + 3) & ~3;
  const int TT = Kp / 4;
  const int ntiles = TT * (TT + 1) / 2;
  int ti = -1, tj = -1;
  if ((int)threadIdx.x < ntiles) {
    int rem = threadIdx.x;
    ti = 0;
    while (rem >= TT - ti) {
      rem -= TT - ti;
      ++ti;
    }
    tj = ti + rem;
  }
  T acc[4][4], hi[4][4], lo[4][4];
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int b = 0; b < 4; ++b) hi[a][b] = lo[a][b] = T(0);
  for (int q = 0; q < ch.z; ++q) {
    const DiagStepRows sr = diag_step(steps, entry_base, entry_cell, cover_off, ch.y + q, K);
    const T* base = panels + sr.row0 * K;
    __syncthreads();
    for (int t = threadIdx.x; t < 16 * Kp; t += blockDim.x) {
      const int r = t / Kp, k = t - r * Kp;
      sm[t] = k < K ? base[(int64_t)r * sr.mK + k] : T(0);
    }
    __syncthreads();
    if (ti < 0) continue;
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
      for (int b = 0; b < 4; ++b) acc[a][b] = T(0);
#pragma unroll 4
    for (int r = 0; r < 16; ++r) {
      T x[4], y[4];
      lds4(sm + r * Kp + 4 * ti, x);
      lds4(sm + r * Kp + 4 * tj, y);
#pragma unroll
      for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int b = 0; b < 4; ++b) acc[a][b] += x[a] * y[b];
    }
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
      for (int b = 0; b < 4; ++b) {
        if (sizeof(T) == 8) {
          hi[a][b] += acc[a][b];
        } else {
          const T yv = acc[a][b] - lo[a][b];
          const T tv = hi[a][b] + yv;
          lo[a][b] = (tv - hi[a][b]) - yv;
          hi[a][b] = tv;
        }
      }
  }
  if (ti < 0) return;
  const int KT = K * (K + 1) / 2;
  double* out = partial + (int64_t)blockIdx.x * KT;
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int b = 0; b < 4; ++b) {
      const int i = 4 * ti + a, j = 4 * tj + b;
      if (i < K && j < K && j >= i) {
        // row-major upper-triangle index of (i, j)
        const int idx = i * K - i * (i - 1) / 2 + (j - i);
        out[idx] = (double)hi[a][b] - (double)lo[a][b];
      }
    }
}

// Same partial sums with the rows staged by bulk copies: every chunk is a
// whole number of 16-row groups of one panel (cells are padded to 16 rows),
// so step q copies rows [16q, 16q + 16) of the chunk, contiguous in HBM, into
// stage q % S of a ring (thread 0 issues; one mbarrier per stage), and the
// stage is refilled after the barrier that ends its step.  Requires K
// sizeof(T) to be a multiple of 16 bytes (rows stay 16-byte aligned) and
// K % 4 == 0.  A wait that times out raises flags[3].
constexpr int kDiagStages = 6;

template <class T>
__global__ void __launch_bounds__(544) k_gram_diag_pipe(const T* __restrict__ panels, int K,
                                                         const int4* __restrict__ chunks,
                                                         const int2* __restrict__ steps,
                                                         const int64_t* __restrict__ entry_base,
                                                         const int* __restrict__ entry_cell,
                                                         const int* __restrict__ cover_off,
                                                         double* __restrict__ partial,
                                                         int* __restrict__ flags) {
  extern __shared__ __align__(128) unsigned char smraw[];
  T* ring = reinterpret_cast<T*>(smraw);   // [kDiagStages][16][K]
  __shared__ __align__(8) uint64_t full[kDiagStages];
  const int4 ch = chunks[blockIdx.x];   // (panel, first step, steps, -)
  const int TT = K / 4;
  const int ntiles = TT * (TT + 1) / 2;
  int ti = -1, tj = -1;
  if ((int)threadIdx.x < ntiles) {
    int rem = threadIdx.x;
    ti = 0;
    while (rem >= TT - ti) {
      rem -= TT - ti;
      ++ti;
    }
    tj = ti + rem;
  }
  const int nsteps = ch.z;
  const uint32_t step_bytes = (uint32_t)(16 * K * sizeof(T));
  // warp 0: lane i copies row i of a step (rows are m_c K elements apart)
  auto issue = [&](int q, int st) {
    const DiagStepRows sr = diag_step(steps, entry_base, entry_cell, cover_off, ch.y + q, K);
    if (threadIdx.x == 0) sm100::mbar_arrive_expect_tx(&full[st], step_bytes);
    __syncwarp();
    if (threadIdx.x < 16)
      sm100::bulk_load(ring + ((int64_t)st * 16 + threadIdx.x) * K,
                       panels + (sr.row0 * K + (int64_t)threadIdx.x * sr.mK),
                       (uint32_t)(K * sizeof(T)), &full[st]);
  };
  if (threadIdx.x == 0) {
    for (int q = 0; q < kDiagStages; ++q) sm100::mbar_init(&full[q], 1);
    sm100::fence_mbar_init();
  }
  __syncwarp();
  if (threadIdx.x < 32)
    for (int q = 0; q < kDiagStages && q < nsteps; ++q) issue(q, q);
  __syncthreads();
  T hi[4][4], lo[4][4];
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int b = 0; b < 4; ++b) hi[a][b] = lo[a][b] = T(0);
  bool ok = true;
  for (int q = 0; q < nsteps; ++q) {
    const int st = q % kDiagStages;
    if (!sm100::mbar_wait(&full[st], (q / kDiagStages) & 1, ok ? sm100::kSpinLimit : 4u)) ok = false;
    const T* sm = ring + (int64_t)st * 16 * K;
    if (ti >= 0) {
      T acc[4][4];
#pragma unroll
      for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int b = 0; b < 4; ++b) acc[a][b] = T(0);
#pragma unroll 8
      for (int r = 0; r < 16; ++r) {
        T x[4], y[4];
        lds4(sm + r * K + 4 * ti, x);
        lds4(sm + r * K + 4 * tj, y);
#pragma unroll
        for (int a = 0; a < 4; ++a)
#pragma unroll
          for (int b = 0; b < 4; ++b) acc[a][b] += x[a] * y[b];
      }
#pragma unroll
      for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int b = 0; b < 4; ++b) {
          if (sizeof(T) == 8) {
            hi[a][b] += acc[a][b];
          } else {
            const T yv = acc[a][b] - lo[a][b];
            const T tv = hi[a][b] + yv;
            lo[a][b] = (tv - hi[a][b]) - yv;
            hi[a][b] = tv;
          }
        }
    }
    __syncthreads();
    if (threadIdx.x < 32 && q + kDiagStages < nsteps) {
      sm100::fence_proxy_async_smem();
      issue(q + kDiagStages, st);
    }
  }
  if (!ok) atomicOr(&flags[3], 1);
  if (ti < 0) return;
  const int KT = K * (K + 1) / 2;
  double* out = partial + (int64_t)blockIdx.x * KT;
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int b = 0; b < 4; ++b) {
      const int i = 4 * ti + a, j = 4 * tj + b;
      if (j >= i) {
        const int idx = i * K - i * (i - 1) / 2 + (j - i);
        out[idx] = (double)hi[a][b] - (double)lo[a][b];
      }
    }
}

// Diagonal Gram partials of DF32 panels: k_gram_diag_pipe's pipeline, every
// product and sum in float-float arithmetic (4x4 tile of pair accumulators
// per thread), FP64 result.  Requires K % 4 == 0.
__global__ void __launch_bounds__(544) k_gram_diag_pipe_df(const float2* __restrict__ panels,
                                                            int K, const int4* __restrict__ chunks,
                                                                   const int2* __restrict__ steps,
                                                                   const int64_t* __restrict__ entry_base,
                                                                   const int* __restrict__ entry_cell,
                                                                   const int* __restrict__ cover_off,
                                                            double* __restrict__ partial,
                                                            int* __restrict__ flags) {
  extern __shared__ __align__(128) unsigned char smraw[];
  float2* ring = reinterpret_cast<float2*>(smraw);   // [kDiagStages][16][K]
  __shared__ __align__(8) uint64_t full[kDiagStages];
  const int4 ch = chunks[blockIdx.x];   // (panel, first step, steps, -)
  const int TT = K / 4;
  const int ntiles = TT * (TT + 1) / 2;
  int ti = -1, tj = -1;
  if ((int)threadIdx.x < ntiles) {
    int rem = threadIdx.x;
    ti = 0;
    while (rem >= TT - ti) {
      rem -= TT - ti;
      ++ti;
    }
    tj = ti + rem;
  }
  const int nsteps = ch.z;
  const uint32_t step_bytes = (uint32_t)(16 * K * sizeof(float2));
  // warp 0: lane i copies row i of a step (rows are m_c K elements apart)
  auto issue = [&](int q, int st) {
    const DiagStepRows sr = diag_step(steps, entry_base, entry_cell, cover_off, ch.y + q, K);
    if (threadIdx.x == 0) sm100::mbar_arrive_expect_tx(&full[st], step_bytes);
    __syncwarp();
    if (threadIdx.x < 16)
      sm100::bulk_load(ring + ((int64_t)st * 16 + threadIdx.x) * K,
                       panels + (sr.row0 * K + (int64_t)threadIdx.x * sr.mK),
                       (uint32_t)(K * sizeof(float2)), &full[st]);
  };
  if (threadIdx.x == 0) {
    for (int q = 0; q < kDiagStages; ++q) sm100::mbar_init(&full[q], 1);
    sm100::fence_mbar_init();
  }
  __syncwarp();
  if (threadIdx.x < 32)
    for (int q = 0; q < kDiagStages && q < nsteps; ++q) issue(q, q);
  __syncthreads();
  float S[4][4], C[4][4];
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int b = 0; b < 4; ++b) S[a][b] = C[a][b] = 0.f;
  bool ok = true;
  int st = 0, ph = 0;
  for (int q = 0; q < nsteps; ++q) {
    if (!sm100::mbar_wait(&full[st], ph, ok ? sm100::kSpinLimit : 4u)) ok = false;
    const float2* sm = ring + (int64_t)st * 16 * K;
    if (ti >= 0) {
#pragma unroll 2
      for (int r = 0; r < 16; ++r) {
        float2 x[4], y[4];
        lds4(sm + r * K + 4 * ti, x);
        lds4(sm + r * K + 4 * tj, y);
#pragma unroll
        for (int a = 0; a < 4; ++a)
#pragma unroll
          for (int b = 0; b < 4; ++b) df_acc(S[a][b], C[a][b], x[a].x, x[a].y, y[b].x, y[b].y);
      }
    }
    __syncthreads();
    if (threadIdx.x < 32 && q + kDiagStages < nsteps) {
      sm100::fence_proxy_async_smem();
      issue(q + kDiagStages, st);
    }
    if (++st == kDiagStages) {
      st = 0;
      ph ^= 1;
    }
  }
  if (!ok) atomicOr(&flags[3], 1);
  if (ti < 0) return;
  const int KT = K * (K + 1) / 2;
  double* out = partial + (int64_t)blockIdx.x * KT;
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int b = 0; b < 4; ++b) {
      const int i = 4 * ti + a, j = 4 * tj + b;
      if (j >= i) out[i * K - i * (i - 1) / 2 + (j - i)] = (double)S[a][b] + (double)C[a][b];
    }
}

// Sum of each panel's diagonal-Gram chunk partials (upper-triangle order,
// FP64) into its packed lower triangle G_s (row i from i (i + 1) / 2 on;
// tri_pairs(K) doubles per panel, so that each panel starts 16-byte aligned):
// one thread per entry, the chunks added in order.  grid = (entry blocks, panels).
__global__ void k_gram_reduce(const double* __restrict__ partial, const int* __restrict__ chunk_off,
                              int K, double* __restrict__ Gp) {
  const int s = blockIdx.y;
  const int KT = K * (K + 1) / 2;
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= KT) return;
  const int c0 = chunk_off[s], c1 = chunk_off[s + 1];
  double v = 0.0;
#pragma unroll 8
  for (int c = c0; c < c1; ++c) v += partial[(int64_t)c * KT + e];
  int i = 0, r = e;   // e = i K - i (i - 1) / 2 + (j - i), i <= j
  while (r >= K - i) {
    r -= K - i;
    ++i;
  }
  const int j = i + r;
  Gp[(int64_t)s * tri_pairs(K) + j * (j + 1) / 2 + i] = v;
}

constexpr int kCholThreads = 512;   // 4 slices x 128 columns in the inverse
static_assert(kCholThreads == 4 * 128, "k_block_chol's inverse maps 512 threads");

// Shared memory of k_block_chol: the packed triangle, then the copy's mbarrier
// (about 66 KB at K = 128: three blocks per SM, so that a few hundred
// subdomains are one wave).
static size_t chol_smem_bytes(int K) { return (size_t)tri_pairs(K) * sizeof(double) + 16; }

__device__ __forceinline__ int trirow(int i) { return i * (i + 1) / 2; }

// One block per subdomain: G_s (packed lower triangle, from k_gram_reduce)
// by one bulk copy; shift; Cholesky (lower L with L L^T = G + eps tr/K I);
// X = L^{-1} in place; X stored row- and column-major (and, given xtri, as
// the packed pair triangle).  R_j = L^T, so R_j^{-1} = X^T and R_j^{-T} = X.
// Right-looking factorisation: column k, once scaled, is also copied to a
// contiguous vector; the trailing update is spread over all threads pair by
// pair (no idle lanes on the short rows: the FP64 pipe is the limit), and the
// thread that finishes G_{k+1,k+1} takes pivot k + 1 at once, so a step has
// two barriers.  The inverse is formed in place row by
// row (row i of X needs row i of L and rows < i of X): lanes over columns j,
// four warp-uniform slices of the sum over m, the slice sums added in a fixed
// order.  A non-positive pivot starts again from a fresh copy of G_s with the
// shift raised 100-fold (at most 8 times; each retry counted in flags[4]),
// then raises flags[1].  With drop > 0 a column whose pivot (its Schur
// complement) is at most drop times its shifted diagonal is numerically
// dependent on the columns before it: it is dropped (its row and column of X
// are zero, so its coefficient stays 0), counted in flags[5], and never
// triggers a retry.  On FP32 panels the Gram carries rounding of about 1e-7
// of its entries, so directions below that are noise that the factors would
// otherwise amplify by 1 / shift.
// The factorisation is FP64 (the blocks are as ill-conditioned as the shift
// allows); with three blocks per SM it keeps GB300's FP64 pipe (1/64 of the
// FP32 FMA rate) about 80% busy.  kDfInv (FP32 and DF32 panels, whose solvers
// apply X as FP32 pairs anyway): the inverse runs in float-float arithmetic
// on the FP32 pipes instead, each finished row of X stored as pairs over the
// row of L it replaces.
template <bool kDfInv>
__global__ void __launch_bounds__(kCholThreads, 3) k_block_chol(const double* __restrict__ Gp,
                                                                 int K, double shift,
                                                                 double abs_shift, double drop,
                                                                 double* __restrict__ Xr,
                                                                 double* __restrict__ Xc,
                                                                 int* __restrict__ flags,
                                                                 float2* __restrict__ xtri) {
  extern __shared__ __align__(16) unsigned char chsm[];
  __shared__ double red[33];
  __shared__ double rpiv[128];       // 1 / L_kk
  __shared__ double colk[128];       // scaled column k of L
  __shared__ double xpart[4][128];   // slice sums of a row of the inverse (pairs with kDfInv)
  __shared__ float2 lrow2[128];      // kDfInv: row i of L as pairs
  __shared__ double gdiag[128];      // the shifted diagonal (drop test)
  __shared__ int fail, ndrop;
  const int64_t PT = tri_pairs(K);
  double* P = reinterpret_cast<double*>(chsm);   // packed lower triangle
  float2* X2 = reinterpret_cast<float2*>(chsm);  // kDfInv: rows of X as pairs
  uint64_t* bar = reinterpret_cast<uint64_t*>(P + PT);
  const int s = blockIdx.x;
  const int tid = threadIdx.x, nt = blockDim.x;
  const uint32_t bytes = (uint32_t)(PT * sizeof(double));
  if (tid == 0) {
    sm100::mbar_init(bar, 1);
    sm100::fence_mbar_init();
  }
  __syncthreads();
  uint32_t phase = 0;
  auto fetch = [&]() {
    sm100::fence_proxy_async_smem();   // earlier writes to P before the copy
    __syncthreads();
    if (tid == 0) {
      sm100::mbar_arrive_expect_tx(bar, bytes);
      sm100::bulk_load(P, Gp + (int64_t)s * PT, bytes, bar);
    }
    if (!sm100::mbar_wait(bar, phase)) {   // bounded; the host reports ELMFB_ERR_TIMEOUT
      atomicOr(&flags[3], 1);
      sm100::mbar_wait(bar, phase);
    }
    phase ^= 1;
  };
  fetch();
  double tr = 0.0;
  {
    double v = 0.0;
    for (int i = tid; i < K; i += nt) v += P[trirow(i) + i];
    tr = block_sum(v, red);
  }
  // pivot k: L_kk = sqrt(G_kk), 1 / L_kk (one thread: FP64 sqrt / division are costly)
  auto pivot = [&](int k) {
    const double d = P[trirow(k) + k];
    if (drop > 0.0 && !(d > drop * gdiag[k])) {   // dependent column: dropped
      P[trirow(k) + k] = 1.0;
      rpiv[k] = 0.0;
      ++ndrop;
      return;
    }
    if (!(d > 0.0)) fail = 1;
    const double l = sqrt(d > 0.0 ? d : 1.0);
    P[trirow(k) + k] = l;
    rpiv[k] = 1.0 / l;
  };
  double eps = shift;
  for (int attempt = 0; attempt < 8; ++attempt) {
    if (attempt > 0) {
      if (tid == 0) atomicAdd(&flags[4], 1);   // retries, reported to the caller
      fetch();
      eps = eps > 0.0 ? eps * 100.0 : 1e-14;
    }
    const double add = eps * tr / K + abs_shift + (tr == 0.0 && abs_shift == 0.0 ? 1.0 : 0.0);
    if (tid == 0) {
      fail = 0;
      ndrop = 0;
    }
    for (int i = tid; i < K; i += nt) {
      P[trirow(i) + i] += add;
      gdiag[i] = P[trirow(i) + i];
    }
    __syncthreads();
    if (tid == 0) pivot(0);
    __syncthreads();
    for (int k = 0; k < K; ++k) {
      if (fail) break;
      const double rp = rpiv[k];
      for (int i = k + 1 + tid; i < K; i += nt) {
        const double l = P[trirow(i) + k] * rp;
        P[trirow(i) + k] = l;
        colk[i] = l;
      }
      __syncthreads();
      // pairs q of the trailing triangle k < c <= i < K (q = a (a + 1) / 2 + b:
      // row i = k + 1 + a, column c = k + 1 + b), every thread busy; the thread
      // with q = 0 finishes G_{k+1,k+1} and takes pivot k + 1 at once
      const int n = K - 1 - k;
      const int T = n * (n + 1) / 2;
      for (int q = tid; q < T; q += nt) {
        int a = (int)((__fsqrt_rn(8.f * (float)q + 1.f) - 1.f) * 0.5f);
        if ((a + 1) * (a + 2) / 2 <= q) ++a;
        else if (a * (a + 1) / 2 > q) --a;
        const int i = k + 1 + a, c = k + 1 + (q - a * (a + 1) / 2);
        P[trirow(i) + c] -= colk[i] * colk[c];
        if (q == 0) pivot(k + 1);
      }
      __syncthreads();
    }
    __syncthreads();
    if (!fail) break;
  }
  if (fail) {
    if (tid == 0) atomicOr(&flags[1], 1);
    return;
  }
  if (tid == 0 && ndrop) atomicAdd(&flags[5], ndrop);
  // X = L^{-1} in place: X_ii = 1/L_ii; X_ij = -(sum_{m=j}^{i-1} L_im X_mj) / L_ii.
  // Row i of L is read while row i of X is formed, then overwritten.
  // Thread (p, j): column j, slice p of [0, i); rows m < j hold no X_mj.
  const int j = tid & 127, p = tid >> 7;
  for (int i = 0; i < K; ++i) {
    const int step = (i + 3) >> 2;
    const int m0 = p * step, m1 = min(i, m0 + step);
    const double* Li = P + trirow(i);
    if (kDfInv) {
      for (int m = tid; m < i; m += nt) lrow2[m] = df_split(Li[m]);
      __syncthreads();
      float S = 0.f, C = 0.f;
      if (j < i)
        for (int m = m0; m < m1; ++m)
          if (m >= j) {
            const float2 x = X2[trirow(m) + j];
            df_acc(S, C, lrow2[m].x, lrow2[m].y, x.x, x.y);
          }
      float2* xp = reinterpret_cast<float2*>(&xpart[0][0]);
      xp[p * 128 + j] = make_float2(S, C);
      __syncthreads();   // row i of L has been read: its place takes row i of X
      if (tid <= i) {
        const float2 rp = df_split(rpiv[i]);
        float2 v = rp;
        if (tid < i) {
          const float2 a =
              df_add(df_add(df_add(xp[tid], xp[128 + tid]), xp[256 + tid]), xp[384 + tid]);
          float Sv = 0.f, Cv = 0.f;
          df_acc(Sv, Cv, a.x, a.y, rp.x, rp.y);
          v = make_float2(-Sv, -Cv);
        }
        X2[trirow(i) + tid] = v;
      }
      __syncthreads();
      continue;
    }
    double acc = 0.0;
    if (j < i)
      for (int m = m0; m < m1; ++m)
        if (m >= j) acc += Li[m] * P[trirow(m) + j];
    xpart[p][j] = acc;
    __syncthreads();   // row i of L has been read: its place takes row i of X
    if (tid < i)
      P[trirow(i) + tid] =
          -(((xpart[0][tid] + xpart[1][tid]) + xpart[2][tid]) + xpart[3][tid]) * rpiv[i];
    else if (tid == i)
      P[trirow(i) + i] = rpiv[i];
    __syncthreads();
  }
  double* xr = Xr + (int64_t)s * K * K;
  double* xc = Xc + (int64_t)s * K * K;
  auto xval = [&](int i, int jj) -> double {
    if (jj > i) return 0.0;
    const int q = trirow(i) + jj;
    return kDfInv ? (double)X2[q].x + (double)X2[q].y : P[q];
  };
  for (int o = tid; o < K * K; o += nt) {
    const int i = o / K, jj = o - i * K;
    xr[o] = xval(i, jj);   // X_ij row-major
  }
  for (int o = tid; o < K * K; o += nt) {
    const int jj = o / K, i = o - jj * K;
    xc[o] = xval(i, jj);   // X_ij column-major
  }
  if (xtri) {   // the triangle again, as packed FP32 pairs
    const int KT = K * (K + 1) / 2;
    for (int q = tid; q < KT; q += nt) xtri[(int64_t)s * PT + q] = kDfInv ? X2[q] : df_split(P[q]);
  }
}

// low-precision copy of an FP64 value: kind 1 FP32, kind 2 FP32 pair (hi, lo)
__device__ __forceinline__ void store_low(void* dst, int kind, int64_t i, double v) {
  if (kind == 1) {
    static_cast<float*>(dst)[i] = (float)v;
  } else if (kind == 2) {
    const float hi = __double2float_rn(v);
    static_cast<float2*>(dst)[i] = make_float2(hi, __double2float_rn(v - (double)hi));
  }
}

// t_j = R_j^{-1} v_j = X_j^T v_j per subdomain (t_i = sum_{m>=i} X_mi v_m; X_j lower
// triangular, row-major; identity without a preconditioner); tlow receives a
// low-precision copy of t (store_low kind; 0 = none).  The G
// thread groups of the block split the inner sum into fixed slices, then one
// pass adds the group sums in order (deterministic).  Block 0 commits the
// staged LSQR scalars.
__global__ void __launch_bounds__(1024) k_precond(const double* __restrict__ Xr,
                                                  const double* __restrict__ v, int K,
                                                  double* __restrict__ t, int identity,
                                                  double* __restrict__ scal,
                                                  void* __restrict__ tlow, int low_kind) {
  extern __shared__ double psh[];   // vs[K] then part[G][K]
  const int s = blockIdx.x;
  if (s == 0 && threadIdx.x < kStage) scal[threadIdx.x] = scal[kStage + threadIdx.x];
  const double* vv = v + (int64_t)s * K;
  if (identity) {
    for (int i = threadIdx.x; i < K; i += blockDim.x) {
      t[(int64_t)s * K + i] = vv[i];
      store_low(tlow, low_kind, (int64_t)s * K + i, vv[i]);
    }
    return;
  }
  double* vs = psh;
  double* part = psh + K;
  for (int i = threadIdx.x; i < K; i += blockDim.x) vs[i] = vv[i];
  __syncthreads();
  const int Kp = (K + 31) & ~31;
  const int G = blockDim.x / Kp;
  const int g = threadIdx.x / Kp, i = threadIdx.x - g * Kp;
  const int chunk = (K + G - 1) / G;
  const double* X = Xr + (int64_t)s * K * K;
  if (g < G && i < K) {
    double acc = 0.0;
    const int m1 = min(K, (g + 1) * chunk);
    for (int m = max(i, g * chunk); m < m1; ++m) acc += X[m * K + i] * vs[m];
    part[g * K + i] = acc;
  }
  __syncthreads();
  for (int j = threadIdx.x; j < K; j += blockDim.x) {
    double acc = 0.0;
    for (int q = 0; q < G; ++q) acc += part[q * K + j];
    t[(int64_t)s * K + j] = acc;
    store_low(tlow, low_kind, (int64_t)s * K + j, acc);
  }
}

// u'_R = sum over covering panels of P[rho] . t_s  - alpha * u_R / beta_prev
// (u is stored unnormalised; u_norm = u / beta_prev).  mode 1: u' = h - M t.
template <class T>
__global__ void __launch_bounds__(kGatherThreads) k_gather(
    const T* __restrict__ panels, const double* __restrict__ tvec, int K, int64_t NR,
    const int* __restrict__ grow_cell, const int* __restrict__ cell_pstart,
    const int* __restrict__ cell_count, const int* __restrict__ cover_off,
    const int* __restrict__ cover_sub, const int* __restrict__ cover_start,
    const int64_t* __restrict__ entry_base, const double* __restrict__ scal,
    double* __restrict__ u, const double* __restrict__ hvec, int mode,
    double* __restrict__ norm_partial) {
  __shared__ double red[33];
  const int lane = threadIdx.x & 31;
  const int warps = (gridDim.x * blockDim.x) >> 5;
  const int wg = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  double coef = 0.0;
  if (mode == 0) {
    const double beta = scal[S_BETA];
    coef = beta > 0.0 ? scal[S_ALPHA] / beta : 0.0;
  }
  double nrm = 0.0;
  for (int64_t R = wg; R < NR; R += warps) {
    const int c = grow_cell[R];
    const int p = (int)(R - cell_pstart[c]);
    double y = 0.0;
    if (p < cell_count[c]) {
      for (int e = cover_off[c]; e < cover_off[c + 1]; ++e) {
        const int s = cover_sub[e];
        const T* row =
            panels + (entry_base[e] + (int64_t)p * (cover_off[c + 1] - cover_off[c])) * (int64_t)K;
        const double* tv = tvec + (int64_t)s * K;
        T part = 0;
        for (int k = lane; k < K; k += 32) part += row[k] * (T)tv[k];
        if (sizeof(T) == 8) y += warp_sum<double>((double)part);
        else y += (double)warp_sumf((float)part);
      }
      double out;
      if (mode == 0) out = y - coef * u[R];
      else out = hvec[R] - y;
      if (lane == 0) u[R] = out;
      nrm += out * out;
    }
  }
  // lane 0 holds the warp's sum
  nrm = __shfl_sync(0xffffffffu, nrm, 0);
  double tot = block_sum(lane == 0 ? nrm : 0.0, red);
  if (threadIdx.x == 0) norm_partial[blockIdx.x] = tot;
}

// partial_e[k] = sum_p P[rho(e,p)][k] u[R(e,p)]  (one block per (cell, panel) entry)
template <class T>
__global__ void __launch_bounds__(128) k_entry_T(const T* __restrict__ panels,
                                                 const double* __restrict__ u, int K,
                                                 const int* __restrict__ entry_cell,
                                                 const int* __restrict__ cover_sub,
                                                 const int* __restrict__ cover_off,
                                                 const int* __restrict__ cell_pstart,
                                                 const int* __restrict__ cell_count,
                                                 const int64_t* __restrict__ entry_base,
                                                 double* __restrict__ partial) {
  const int e = blockIdx.x;
  const int c = entry_cell[e];
  const int cnt = cell_count[c];
  const int64_t R0 = cell_pstart[c];
  const T* base = panels + entry_base[e] * (int64_t)K;
  const int64_t rs = (int64_t)(cover_off[c + 1] - cover_off[c]) * K;   // row stride
  double* out = partial + (int64_t)e * K;
  if (cnt == 0) {
    for (int k = threadIdx.x; k < K; k += blockDim.x) out[k] = 0.0;
    return;
  }
  const double* us = u + R0;   // broadcast reads, cached
  for (int k = threadIdx.x; k < K; k += blockDim.x) {
    double acc = 0.0;
    if (sizeof(T) == 8) {
      for (int p = 0; p < cnt; ++p) acc += (double)base[(int64_t)p * rs + k] * us[p];
    } else {
      float a32 = 0.f;
      int p = 0;
      for (; p < cnt; ++p) {
        a32 += (float)base[(int64_t)p * rs + k] * (float)us[p];
        if ((p & 31) == 31) {
          acc += a32;
          a32 = 0.f;
        }
      }
      acc += a32;
    }
    out[k] = acc;
  }
}

// One pass over the panels per LSQR iteration.  A CTA takes one unit (a row
// range of one cell); warp w owns the w-th covering panel of the cell.  For
// each 8-row chunk the warps load their panel rows into registers and form
// d_w(r) = P_w[r] . t_w; the row values u'(r) = sum_w d_w(r) - coef u(r)
// (mode 0; mode 2: sum_w d_w(r) / alpha - coef u(r), t = P v' not yet
// normalised) or h(r) - sum_w d_w(r) (mode 1) are formed in FP64 in a fixed
// order; then every warp adds P_w[r] u'(r) into its running partial of
// M^T u' (Kahan-compensated in FP32 panels).  The unit's partials and its
// ||u'||^2 are written once: M t and M^T u' read each panel entry once.
constexpr int kFusedRows = 8;

template <class T, int FPL, int MAXT>
__global__ void __launch_bounds__(MAXT, 1) k_fused(
    const T* __restrict__ panels, const T* __restrict__ tvec, int K,
    const int4* __restrict__ units, const int* __restrict__ cell_pstart,
    const int* __restrict__ cell_count, const int* __restrict__ cover_off,
    const int* __restrict__ cover_sub, const int* __restrict__ cover_start,
    const int64_t* __restrict__ entry_base, const double* __restrict__ scal,
    double* __restrict__ u, const double* __restrict__ hvec, int mode,
    double* __restrict__ partial, double* __restrict__ norm_partial) {
  __shared__ double sd[32][kFusedRows];
  __shared__ double su[kFusedRows];
  if (mode == 2 && scal[kStage + S_DONE] != 0.0) return;   // LSQR stopped on the device
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int4 un = units[blockIdx.x];   // (cell, first row, end row, first partial)
  const int c = un.x;
  const int m = cover_off[c + 1] - cover_off[c];
  const int cnt = cell_count[c];
  const int64_t R0 = cell_pstart[c];
  const bool active = w < m;
  const int e = cover_off[c] + (active ? w : 0);
  const int s = cover_sub[e];
  const T* base = panels + entry_base[e] * (int64_t)K;   // row r at base + r m K
  const int64_t rs = (int64_t)m * K;
  T tv[FPL];
#pragma unroll
  for (int j = 0; j < FPL; ++j) {
    const int k = lane + 32 * j;
    tv[j] = (active && k < K) ? tvec[(int64_t)s * K + k] : T(0);
  }
  double coef = 0.0, ts = 1.0;   // used by warp 0 only (an FP64 division is costly)
  if (mode != 1 && threadIdx.x < 32) {
    const double beta = scal[kStage + S_BETA];   // staged by the previous LSQR update
    coef = beta > 0.0 ? scal[kStage + S_ALPHA] / beta : 0.0;
    if (mode == 2) ts = scal[kStage + S_TSCALE];
  }
  T ahi[FPL], alo[FPL];
#pragma unroll
  for (int j = 0; j < FPL; ++j) ahi[j] = alo[j] = T(0);
  double nrm = 0.0;
  // register double buffer: rows (and u values) of the next chunk are loaded
  // while the current chunk is reduced
  T pv[kFusedRows][FPL], pn[kFusedRows][FPL];
  double uold = 0.0, unext = 0.0;
  auto load_chunk = [&](int r0, T (&dst)[kFusedRows][FPL], double& uo) {
    const int nr = min(kFusedRows, un.z - r0);
#pragma unroll
    for (int r = 0; r < kFusedRows; ++r)
#pragma unroll
      for (int j = 0; j < FPL; ++j) {
        const int k = lane + 32 * j;
        dst[r][j] = (active && r < nr && k < K) ? base[(int64_t)(r0 + r) * rs + k] : T(0);
      }
    const int p = r0 + (int)threadIdx.x;
    uo = 0.0;
    if (threadIdx.x < (unsigned)nr && p < cnt)
      uo = mode != 1 ? u[R0 + p] : hvec[R0 + p];
  };
  if (un.y < un.z) load_chunk(un.y, pv, uold);
  for (int r0 = un.y; r0 < un.z; r0 += kFusedRows) {
    const int nr = min(kFusedRows, un.z - r0);
    if (r0 + kFusedRows < un.z) load_chunk(r0 + kFusedRows, pn, unext);
#pragma unroll
    for (int r = 0; r < kFusedRows; ++r) {
      T d = 0;
#pragma unroll
      for (int j = 0; j < FPL; ++j) d += pv[r][j] * tv[j];
      for (int o = 16; o > 0; o >>= 1) d += __shfl_xor_sync(0xffffffffu, d, o);
      if (lane == 0) sd[w][r] = (double)d;
    }
    __syncthreads();
    if (threadIdx.x < nr) {
      const int r = threadIdx.x;
      const int p = r0 + r;
      double y = 0.0;
      for (int q = 0; q < m; ++q) y += sd[q][r];
      double out = 0.0;
      if (p < cnt) {
        out = mode != 1 ? y * ts - coef * uold : uold - y;
        u[R0 + p] = out;
        nrm += out * out;
      }
      su[r] = out;
    }
    __syncthreads();
#pragma unroll
    for (int r = 0; r < kFusedRows; ++r) {
      const T ur = r < nr ? (T)su[r] : T(0);
#pragma unroll
      for (int j = 0; j < FPL; ++j) {
        if (sizeof(T) == 8) {
          ahi[j] += pv[r][j] * ur;
        } else {
          const T y = pv[r][j] * ur - alo[j];
          const T t = ahi[j] + y;
          alo[j] = (t - ahi[j]) - y;
          ahi[j] = t;
        }
      }
    }
#pragma unroll
    for (int r = 0; r < kFusedRows; ++r)
#pragma unroll
      for (int j = 0; j < FPL; ++j) pv[r][j] = pn[r][j];
    uold = unext;
  }
  if (active) {
    const int64_t base_idx = (int64_t)(un.w + w) * K;
#pragma unroll
    for (int j = 0; j < FPL; ++j) {
      const int k = lane + 32 * j;
      if (k >= K) continue;
      if (sizeof(T) == 8)
        partial[base_idx + k] = (double)ahi[j];
      else
        reinterpret_cast<float2*>(partial)[base_idx + k] =
            make_float2((float)ahi[j], (float)alo[j]);
    }
  }
  // threads 0..7 of warp 0 hold the row norms
  if (threadIdx.x < 32) {   // the row norms live in warp 0
    const double tot = warp_sum<double>(nrm);
    if (threadIdx.x == 0) norm_partial[blockIdx.x] = tot;
  }
}

// Same pass, pipelined through shared memory by bulk copies and specialised
// warps.  Warp w < m owns covering panel w of the unit; one extra producer
// warp issues the copies and one control warp forms u'.  Chunks of kPipeRows
// rows of every covering panel land in a ring of S stages.
// There is no block-wide barrier in the loop; mbarriers carry every
// dependency:
//   full[st]   chunk copied in (transaction bytes)
//   dots[b]    every panel warp has written its dots of the chunk (slot b)
//   u[b]       the control warp has written u' of the chunk (slot b)
//   empty[st]  every panel warp has finished its update with the stage
// Panel warp, chunk i: wait full, form the dots of chunk i, then wait u of
// chunk i-1 and add P_w[r,:]^T u'_r of chunk i-1, then free its stage.
// Control warp, chunk j: wait dots, sum them over the panels, form
// u'_r = y_r - (alpha/beta) u_r in FP64 (written to u).  Producer warp,
// chunk c >= S: wait empty for chunk c-S and refill that stage with chunk c,
// so that a refill never waits behind the control warp's FP64 chain (which
// had shortened the time a copy has to land).  A warp cannot run two
// phases ahead on any barrier: each wait is ordered behind the arrivals it
// depends on (a panel warp's dots of chunk i+2 follow its wait for u' of
// chunk i, which needs every dots arrival of chunk i).  The unit's u (or h)
// values come in by one bulk copy, so no global load sits inside the loop.
// FP64 work is confined to the control warp (GB300's FP64 rate is 1/64 of
// FP32).  Lane l holds features k = l FPL + j, read from shared memory as one
// vector.  Every wait is bounded; a timeout raises flags[3].
constexpr int kPipeRows = 4;
// k_fused_pipe takes 4 or 8 rows a chunk: both divide every unit (units are
// multiples of kFusedRows rows, cells multiples of kCellPad)
static_assert(kFusedRows % 8 == 0 && kCellPad % 8 == 0, "fused chunks must divide the units");
constexpr int kPipeMaxStages = 12;
constexpr int kMaxUnitRows = 1024;   // rows of one unit (its u values are staged in smem)

// sum of 4 per-lane values over the warp; lane 8r holds the total of value r
template <class T>
__device__ __forceinline__ T warp_sum4(T v0, T v1, T v2, T v3, int lane) {
  const bool b4 = lane & 16, b3 = lane & 8;
  const T k0 = (b4 ? v2 : v0) + __shfl_xor_sync(0xffffffffu, b4 ? v0 : v2, 16);
  const T k1 = (b4 ? v3 : v1) + __shfl_xor_sync(0xffffffffu, b4 ? v1 : v3, 16);
  T k = (b3 ? k1 : k0) + __shfl_xor_sync(0xffffffffu, b3 ? k0 : k1, 8);
  k += __shfl_xor_sync(0xffffffffu, k, 4);
  k += __shfl_xor_sync(0xffffffffu, k, 2);
  k += __shfl_xor_sync(0xffffffffu, k, 1);
  return k;
}

// FPL consecutive elements p[0..FPL) into x (vector loads when the slice is
// whole; zeros past rem elements otherwise).  p is aligned to the slice width.
template <class T, int FPL>
__device__ __forceinline__ void load_slice(const T* p, T (&x)[FPL], bool whole, int rem) {
  if (whole) {
    if constexpr (sizeof(T) * FPL == 16) {
      const float4 v = *reinterpret_cast<const float4*>(p);
      const T* e = reinterpret_cast<const T*>(&v);
#pragma unroll
      for (int j = 0; j < FPL; ++j) x[j] = e[j];
    } else if constexpr (sizeof(T) * FPL == 32) {
      const float4 v0 = reinterpret_cast<const float4*>(p)[0];
      const float4 v1 = reinterpret_cast<const float4*>(p)[1];
      const T* e0 = reinterpret_cast<const T*>(&v0);
      const T* e1 = reinterpret_cast<const T*>(&v1);
#pragma unroll
      for (int j = 0; j < FPL / 2; ++j) {
        x[j] = e0[j];
        x[j + FPL / 2] = e1[j];
      }
    } else if constexpr (sizeof(T) * FPL == 8) {
      const float2 v = *reinterpret_cast<const float2*>(p);
      const T* e = reinterpret_cast<const T*>(&v);
#pragma unroll
      for (int j = 0; j < FPL; ++j) x[j] = e[j];
    } else {
#pragma unroll
      for (int j = 0; j < FPL; ++j) x[j] = p[j];
    }
  } else {
#pragma unroll
    for (int j = 0; j < FPL; ++j) x[j] = j < rem ? p[j] : T(0);
  }
}

template <class T, int FPL, int kRows, bool kBatch = false>
__global__ void __launch_bounds__(1024, 1) k_fused_pipe(
    const T* __restrict__ panels, const T* __restrict__ tvec, int K,
    const int4* __restrict__ units, const int* __restrict__ cell_pstart,
    const int* __restrict__ cell_count, const int* __restrict__ cover_off,
    const int* __restrict__ cover_sub, const int* __restrict__ cover_start,
    const int64_t* __restrict__ entry_base, const double* __restrict__ scal,
    double* __restrict__ u, const double* __restrict__ hvec, int mode,
    double* __restrict__ partial, double* __restrict__ norm_partial, int S, int mmax,
    int* __restrict__ flags, const BatchInst* __restrict__ bi, const int2* __restrict__ bmap) {
  int ub = blockIdx.x;   // this CTA's unit
  if constexpr (kBatch) {
    // a multi-instance launch: the unit's instance supplies every array
    const int2 bm = bmap[blockIdx.x];
    const BatchInst& I = bi[bm.x];
    panels = reinterpret_cast<const T*>(I.panels);
    tvec = reinterpret_cast<const T*>(I.tlow);
    units = I.units;
    cell_pstart = I.cell_pstart;
    cell_count = I.cell_count;
    cover_off = I.cover_off;
    cover_sub = I.cover_sub;
    entry_base = I.entry_base;
    scal = I.scal;
    u = I.u;
    hvec = I.hvec;
    partial = I.part;
    norm_partial = I.gpart;
    flags = I.flags;
    ub = bm.y;
  }
  if (mode == 2 && scal[kStage + S_DONE] != 0.0) return;   // LSQR stopped on the device
  extern __shared__ __align__(128) unsigned char ring_raw[];
  __shared__ __align__(8) uint64_t full[kPipeMaxStages];    // chunk copied in
  __shared__ __align__(8) uint64_t empty[kPipeMaxStages];   // stage free again
  __shared__ __align__(8) uint64_t dots_bar[2];             // dots of a chunk written
  __shared__ __align__(8) uint64_t u_bar[2];                // u' of a chunk written
  __shared__ __align__(8) uint64_t ubar;                    // the unit's u / h values in
  __shared__ T sd[2][32][kRows];
  __shared__ T su[2][kRows];
  T* ring = reinterpret_cast<T*>(ring_raw);
  const int64_t stage_elems = (int64_t)mmax * kRows * K;
  double* us = reinterpret_cast<double*>(ring_raw + (size_t)S * stage_elems * sizeof(T));
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int cw = (blockDim.x >> 5) - 1;   // control warp: u', norms
  const int pw = cw - 1;                  // producer warp: the ring's copies
  const int4 un = units[ub];              // (cell, first row, end row, first partial)
  const int c = un.x;
  const int m = cover_off[c + 1] - cover_off[c];
  const int cnt = cell_count[c];
  const int64_t R0 = cell_pstart[c];
  const bool active = w < m;
  const int s = cover_sub[cover_off[c] + (active ? w : 0)];
  const uint32_t copy_bytes = (uint32_t)(kRows * K * sizeof(T));
  const int nrows = un.z - un.y;
  const int nchunks = nrows / kRows;
  // the unit's rows of all m covering panels form one contiguous block
  // (cell-interleaved storage): chunk q = element rows base_row + q kRows m ...
  const int64_t base_row = entry_base[cover_off[c]] + (int64_t)un.y * m;
  if (threadIdx.x == 0) {
    for (int q = 0; q < S; ++q) {
      sm100::mbar_init(&full[q], 1);
      sm100::mbar_init(&empty[q], (uint32_t)m);
    }
    for (int b = 0; b < 2; ++b) {
      sm100::mbar_init(&dots_bar[b], (uint32_t)(kRows * m));   // one arrival per row and warp
      sm100::mbar_init(&u_bar[b], (uint32_t)kRows);
    }
    sm100::mbar_init(&ubar, 1);
    sm100::fence_mbar_init();
  }
  __syncthreads();   // the only block-wide barrier
  bool ok = true;
  // control warp: kYG lanes (panel groups) per row of a chunk
  constexpr int kYG = 32 / kRows;
  const int yr = lane / kYG, yg = lane % kYG;

  if (w == pw) {
    // --------------------------------------------------------- producer warp
    // chunk c goes to stage c mod S once chunk c - S has left it (release
    // number (c - S) / S of that stage's empty barrier)
    if (lane == 0) {
      // the panels stream through once per pass: evict them first, so that
      // the data the rest of the iteration reuses (the triangles X_j, the
      // partials, the vectors: tens of MB) stays in L2
      const uint64_t pol = sm100::l2_evict_first_policy();
      auto issue = [&](int chunk, int stage) {
        sm100::mbar_arrive_expect_tx(&full[stage], copy_bytes * (uint32_t)m);
        sm100::bulk_load_hint(ring + stage * stage_elems,
                              panels + (base_row + (int64_t)chunk * kRows * m) * K,
                              copy_bytes * (uint32_t)m, &full[stage], pol);
      };
      for (int q = 0; q < S && q < nchunks; ++q) issue(q, q);
      int st_r = 0, ph_r = 0;   // stage / empty parity of chunk c - S
      for (int c = S; c < nchunks; ++c) {
        if (!sm100::mbar_wait(&empty[st_r], ph_r, ok ? sm100::kSpinLimit : 4u)) ok = false;
        sm100::fence_proxy_async_smem();
        issue(c, st_r);
        if (++st_r == S) {
          st_r = 0;
          ph_r ^= 1;
        }
      }
      if (!ok) atomicOr(&flags[3], 1);
    }
    return;
  }
  if (w == cw) {
    // ---------------------------------------------------------- control warp
    if (lane == 0) {
      const uint32_t ub = (uint32_t)(nrows * sizeof(double));
      sm100::mbar_arrive_expect_tx(&ubar, ub);
      sm100::bulk_load(us, (mode != 1 ? u : hvec) + R0 + un.y, ub, &ubar);
    }
    double coef = 0.0, ts = 1.0;
    if (mode != 1) {
      const double beta = scal[kStage + S_BETA];   // staged by the previous LSQR update
      coef = beta > 0.0 ? scal[kStage + S_ALPHA] / beta : 0.0;
      if (mode == 2) ts = scal[kStage + S_TSCALE];
    }
    if (!sm100::mbar_wait(&ubar, 0, ok ? sm100::kSpinLimit : 4u)) ok = false;
    double nrm = 0.0;
    for (int j = 0; j < nchunks; ++j) {
      const int b = j & 1;
      if (!sm100::mbar_wait(&dots_bar[b], (j >> 1) & 1, ok ? sm100::kSpinLimit : 4u)) ok = false;
      T part = T(0);
      for (int q = yg; q < m; q += kYG) part += sd[b][q][yr];
#pragma unroll
      for (int o = kYG / 2; o > 0; o >>= 1) part += __shfl_xor_sync(0xffffffffu, part, o);
      if (yg == 0) {
        const int pr = j * kRows + yr;   // row within the unit
        double out = 0.0;
        if (un.y + pr < cnt) {
          const double uo = us[pr];
          out = mode != 1 ? (double)part * ts - coef * uo : uo - (double)part;
          u[R0 + un.y + pr] = out;
          nrm += out * out;
        }
        su[b][yr] = (T)out;
        sm100::mbar_arrive(&u_bar[b]);
      }
    }
    if (!ok && lane == 0) atomicOr(&flags[3], 1);
    const double tot = warp_sum<double>(nrm);
    if (lane == 0) norm_partial[ub] = tot;
    return;
  }
  if (!active) return;

  // ------------------------------------------------------------ panel warps
  const int k0 = lane * FPL;   // lane slice of the features: k = lane * FPL + j
  const bool whole = k0 + FPL <= K;
  const int rem = K - k0;
  T tv[FPL];
#pragma unroll
  for (int j = 0; j < FPL; ++j) {
    const int k = k0 + j;
    tv[j] = k < K ? tvec[(int64_t)s * K + k] : T(0);
  }
  T ahi[FPL], alo[FPL];
#pragma unroll
  for (int j = 0; j < FPL; ++j) ahi[j] = alo[j] = T(0);
  // update with chunk i (rows of stage st, u' slot i & 1), then free the stage
  auto update = [&](int i, int st) {
    const int b = i & 1;
    if (!sm100::mbar_wait(&u_bar[b], (i >> 1) & 1, ok ? sm100::kSpinLimit : 4u)) ok = false;
    const T* sp = ring + st * stage_elems + (int64_t)w * K + k0;   // row r at + r m K
    T acc[FPL];
#pragma unroll
    for (int j = 0; j < FPL; ++j) acc[j] = T(0);
#pragma unroll
    for (int r = 0; r < kRows; ++r) {
      const T ur = su[b][r];
      T x[FPL];
      load_slice<T, FPL>(sp + (int64_t)r * m * K, x, whole, rem);
#pragma unroll
      for (int j = 0; j < FPL; ++j) acc[j] += x[j] * ur;
    }
    // chunk sums added with compensation (FP32 panels)
#pragma unroll
    for (int j = 0; j < FPL; ++j) {
      if (sizeof(T) == 8) {
        ahi[j] += acc[j];
      } else {
        const T y = acc[j] - alo[j];
        const T t = ahi[j] + y;
        alo[j] = (t - ahi[j]) - y;
        ahi[j] = t;
      }
    }
    __syncwarp();
    if (lane == 0) sm100::mbar_arrive(&empty[st]);
  };
  int st_i = 0, ph_i = 0, st_prev = 0;
  for (int i = 0; i < nchunks; ++i) {
    if (!sm100::mbar_wait(&full[st_i], ph_i, ok ? sm100::kSpinLimit : 4u)) ok = false;
    const T* sp = ring + st_i * stage_elems + (int64_t)w * K + k0;   // row r at + r m K
    T d[kRows];
#pragma unroll
    for (int r = 0; r < kRows; ++r) {
      T x[FPL];
      load_slice<T, FPL>(sp + (int64_t)r * m * K, x, whole, rem);
      d[r] = T(0);
#pragma unroll
      for (int j = 0; j < FPL; ++j) d[r] += x[j] * tv[j];
    }
    // butterflies of 4 rows: lane 8r holds row 4h + r of group h
#pragma unroll
    for (int h4 = 0; h4 < kRows / 4; ++h4) {
      const T tot = warp_sum4(d[4 * h4], d[4 * h4 + 1], d[4 * h4 + 2], d[4 * h4 + 3], lane);
      if ((lane & 7) == 0) {
        sd[i & 1][w][4 * h4 + (lane >> 3)] = tot;
        sm100::mbar_arrive(&dots_bar[i & 1]);
      }
    }
    if (i >= 1) update(i - 1, st_prev);
    st_prev = st_i;
    if (++st_i == S) {
      st_i = 0;
      ph_i ^= 1;
    }
  }
  if (nchunks >= 1) update(nchunks - 1, st_prev);
  if (!ok && lane == 0) atomicOr(&flags[3], 1);
  const int64_t base_idx = (int64_t)(un.w + w) * K;
#pragma unroll
  for (int j = 0; j < FPL; ++j) {
    const int k = k0 + j;
    if (k >= K) continue;
    if (sizeof(T) == 8)
      partial[base_idx + k] = (double)ahi[j];
    else
      reinterpret_cast<float2*>(partial)[base_idx + k] =
          make_float2((float)ahi[j], (float)alo[j]);
  }
}

// The fused LSQR pass of k_fused_pipe for DF32 panels: identical warp roles
// and barriers, with every product and sum of panel entries in float-float
// arithmetic (about 15 FP32 operations per entry and product, against one
// FP64 FMA that GB300 issues at 1/64 of the FP32 rate).  Partials are stored as pairs in
// the hi - lo convention of the FP32 path.
template <int FPL>
__global__ void __launch_bounds__(1024, 1) k_fused_pipe_df(
    const float2* __restrict__ panels, const float2* __restrict__ tvec, int K,
    const int4* __restrict__ units, const int* __restrict__ cell_pstart,
    const int* __restrict__ cell_count, const int* __restrict__ cover_off,
    const int* __restrict__ cover_sub, const int* __restrict__ cover_start,
    const int64_t* __restrict__ entry_base, const double* __restrict__ scal,
    double* __restrict__ u, const double* __restrict__ hvec, int mode,
    double* __restrict__ partial, double* __restrict__ norm_partial, int S, int mmax,
    int* __restrict__ flags) {
  if (mode == 2 && scal[kStage + S_DONE] != 0.0) return;   // LSQR stopped on the device
  extern __shared__ __align__(128) unsigned char ring_raw[];
  __shared__ __align__(8) uint64_t full[kPipeMaxStages];    // chunk copied in
  __shared__ __align__(8) uint64_t empty[kPipeMaxStages];   // stage free again
  __shared__ __align__(8) uint64_t dots_bar[2];             // dots of a chunk written
  __shared__ __align__(8) uint64_t u_bar[2];                // u' of a chunk written
  __shared__ __align__(8) uint64_t ubar;                    // the unit's u / h values in
  __shared__ float2 sd[2][32][kPipeRows];
  __shared__ float2 su[2][kPipeRows];
  float2* ring = reinterpret_cast<float2*>(ring_raw);
  const int64_t stage_elems = (int64_t)mmax * kPipeRows * K;
  double* us = reinterpret_cast<double*>(ring_raw + (size_t)S * stage_elems * sizeof(float2));
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int cw = (blockDim.x >> 5) - 1;   // control warp: u', norms
  const int pw = cw - 1;                  // producer warp: the ring's copies
  const int4 un = units[blockIdx.x];      // (cell, first row, end row, first partial)
  const int c = un.x;
  const int m = cover_off[c + 1] - cover_off[c];
  const int cnt = cell_count[c];
  const int64_t R0 = cell_pstart[c];
  const bool active = w < m;
  const int s = cover_sub[cover_off[c] + (active ? w : 0)];
  const uint32_t copy_bytes = (uint32_t)(kPipeRows * K * sizeof(float2));
  const int nrows = un.z - un.y;
  const int nchunks = nrows / kPipeRows;
  // the unit's rows of all m covering panels form one contiguous block
  // (cell-interleaved storage): chunk q = element rows base_row + q kPipeRows m ...
  const int64_t base_row = entry_base[cover_off[c]] + (int64_t)un.y * m;
  if (threadIdx.x == 0) {
    for (int q = 0; q < S; ++q) {
      sm100::mbar_init(&full[q], 1);
      sm100::mbar_init(&empty[q], (uint32_t)m);
    }
    for (int b = 0; b < 2; ++b) {
      sm100::mbar_init(&dots_bar[b], 4u * (uint32_t)m);   // lanes 0, 8, 16, 24 of each warp
      sm100::mbar_init(&u_bar[b], 4u);
    }
    sm100::mbar_init(&ubar, 1);
    sm100::fence_mbar_init();
  }
  __syncthreads();   // the only block-wide barrier
  bool ok = true;
  const int yr = lane >> 3, yg = lane & 7;

  if (w == pw) {
    // --------------------------------------------------------- producer warp
    // chunk c goes to stage c mod S once chunk c - S has left it (release
    // number (c - S) / S of that stage's empty barrier)
    if (lane == 0) {
      // the panels stream through once per pass: evict them first, so that
      // the data the rest of the iteration reuses (the triangles X_j, the
      // partials, the vectors: tens of MB) stays in L2
      const uint64_t pol = sm100::l2_evict_first_policy();
      auto issue = [&](int chunk, int stage) {
        sm100::mbar_arrive_expect_tx(&full[stage], copy_bytes * (uint32_t)m);
        sm100::bulk_load_hint(ring + stage * stage_elems,
                              panels + (base_row + (int64_t)chunk * kPipeRows * m) * K,
                              copy_bytes * (uint32_t)m, &full[stage], pol);
      };
      for (int q = 0; q < S && q < nchunks; ++q) issue(q, q);
      int st_r = 0, ph_r = 0;   // stage / empty parity of chunk c - S
      for (int c = S; c < nchunks; ++c) {
        if (!sm100::mbar_wait(&empty[st_r], ph_r, ok ? sm100::kSpinLimit : 4u)) ok = false;
        sm100::fence_proxy_async_smem();
        issue(c, st_r);
        if (++st_r == S) {
          st_r = 0;
          ph_r ^= 1;
        }
      }
      if (!ok) atomicOr(&flags[3], 1);
    }
    return;
  }
  if (w == cw) {
    // ---------------------------------------------------------- control warp
    if (lane == 0) {
      const uint32_t ub = (uint32_t)(nrows * sizeof(double));
      sm100::mbar_arrive_expect_tx(&ubar, ub);
      sm100::bulk_load(us, (mode != 1 ? u : hvec) + R0 + un.y, ub, &ubar);
    }
    double coef = 0.0, ts = 1.0;
    if (mode != 1) {
      const double beta = scal[kStage + S_BETA];   // staged by the previous LSQR update
      coef = beta > 0.0 ? scal[kStage + S_ALPHA] / beta : 0.0;
      if (mode == 2) ts = scal[kStage + S_TSCALE];
    }
    if (!sm100::mbar_wait(&ubar, 0, ok ? sm100::kSpinLimit : 4u)) ok = false;
    double nrm = 0.0;
    for (int j = 0; j < nchunks; ++j) {
      const int b = j & 1;
      if (!sm100::mbar_wait(&dots_bar[b], (j >> 1) & 1, ok ? sm100::kSpinLimit : 4u)) ok = false;
      float2 part = make_float2(0.f, 0.f);
      for (int q = yg; q < m; q += 8) part = df_add(part, sd[b][q][yr]);
      part = df_add(part, df_shfl_xor(part, 4));
      part = df_add(part, df_shfl_xor(part, 2));
      part = df_add(part, df_shfl_xor(part, 1));
      if (yg == 0) {
        const int pr = j * kPipeRows + yr;   // row within the unit
        double out = 0.0;
        if (un.y + pr < cnt) {
          const double y = (double)part.x + (double)part.y;
          const double uo = us[pr];
          out = mode != 1 ? y * ts - coef * uo : uo - y;
          u[R0 + un.y + pr] = out;
          nrm += out * out;
        }
        su[b][yr] = df_split(out);
        sm100::mbar_arrive(&u_bar[b]);
      }
    }
    if (!ok && lane == 0) atomicOr(&flags[3], 1);
    const double tot = warp_sum<double>(nrm);
    if (lane == 0) norm_partial[blockIdx.x] = tot;
    return;
  }
  if (!active) return;

  // ------------------------------------------------------------ panel warps
  const int k0 = lane * FPL;   // lane slice of the features: k = lane * FPL + j
  const bool whole = k0 + FPL <= K;
  const int rem = K - k0;
  float2 tv[FPL];
#pragma unroll
  for (int j = 0; j < FPL; ++j) {
    const int k = k0 + j;
    tv[j] = k < K ? tvec[(int64_t)s * K + k] : make_float2(0.f, 0.f);
  }
  float ah[FPL], al[FPL];
#pragma unroll
  for (int j = 0; j < FPL; ++j) ah[j] = al[j] = 0.f;
  // update with chunk i (rows of stage st, u' slot i & 1), then free the stage
  auto update = [&](int i, int st) {
    const int b = i & 1;
    if (!sm100::mbar_wait(&u_bar[b], (i >> 1) & 1, ok ? sm100::kSpinLimit : 4u)) ok = false;
    const float2* sp = ring + st * stage_elems + (int64_t)w * K + k0;   // row r at + r m K
#pragma unroll
    for (int r = 0; r < kPipeRows; ++r) {
      const float2 ur = su[b][r];
      float2 x[FPL];
      load_slice_df<FPL>(sp + (int64_t)r * m * K, x, whole, rem);
#pragma unroll
      for (int j = 0; j < FPL; ++j) df_acc(ah[j], al[j], x[j].x, x[j].y, ur.x, ur.y);
    }
    __syncwarp();
    if (lane == 0) sm100::mbar_arrive(&empty[st]);
  };
  int st_i = 0, ph_i = 0, st_prev = 0;
  for (int i = 0; i < nchunks; ++i) {
    if (!sm100::mbar_wait(&full[st_i], ph_i, ok ? sm100::kSpinLimit : 4u)) ok = false;
    const float2* sp = ring + st_i * stage_elems + (int64_t)w * K + k0;   // row r at + r m K
    float2 d[kPipeRows];
#pragma unroll
    for (int r = 0; r < kPipeRows; ++r) {
      float2 x[FPL];
      load_slice_df<FPL>(sp + (int64_t)r * m * K, x, whole, rem);
      float Sx = 0.f, Cx = 0.f;
#pragma unroll
      for (int j = 0; j < FPL; ++j) df_acc(Sx, Cx, x[j].x, x[j].y, tv[j].x, tv[j].y);
      d[r] = make_float2(Sx, Cx);
    }
    const float2 tot = warp_sum4_df(d[0], d[1], d[2], d[3], lane);
    if (yg == 0) {
      sd[i & 1][w][yr] = tot;
      sm100::mbar_arrive(&dots_bar[i & 1]);
    }
    if (i >= 1) update(i - 1, st_prev);
    st_prev = st_i;
    if (++st_i == S) {
      st_i = 0;
      ph_i ^= 1;
    }
  }
  if (nchunks >= 1) update(nchunks - 1, st_prev);
  if (!ok && lane == 0) atomicOr(&flags[3], 1);
  const int64_t base_idx = (int64_t)(un.w + w) * K;
#pragma unroll
  for (int j = 0; j < FPL; ++j) {
    const int k = k0 + j;
    if (k < K) reinterpret_cast<float2*>(partial)[base_idx + k] = make_float2(ah[j], -al[j]);
  }
}

// Sum of one fixed slice of a panel's partials (at most kPanelChunk entries of
// the panel's entry list), one thread per feature k.  FP32 (hi, lo) pairs are
// summed in float-float arithmetic and stored as a pair in the same
// convention (value hi - lo); FP64 partials are summed in FP64.
constexpr int kPanelChunk = 32;

__global__ void k_panel_chunks(const double* __restrict__ partial, const int* __restrict__ fe,
                               const int2* __restrict__ pch, int K, double* __restrict__ csum,
                               int pairs, const double* __restrict__ beta_partial, int n_beta,
                               double* __restrict__ scal, const BatchInst* __restrict__ bi,
                               const int2* __restrict__ bmap) {
  __shared__ int ent[kPanelChunk];
  int cb = blockIdx.x;   // this block's slice
  if (bi) {   // a multi-instance launch: the slice's instance supplies every array
    const int2 bm = bmap[blockIdx.x];
    const BatchInst& I = bi[bm.x];
    partial = I.part;
    fe = I.fe;
    pch = I.pch;
    csum = I.csum;
    beta_partial = I.gpart;
    n_beta = I.n_units;
    scal = I.scal;
    cb = bm.y;
  }
  if (beta_partial && scal[kStage + S_DONE] != 0.0) return;   // LSQR stopped on the device
  // block 0, LSQR: commit the scalars staged by the previous update (no kernel
  // of the iteration reads the committed slots before this point), then
  // warp 0 forms beta^2 = sum of the norm partials, once for every panel block
  // of the next kernel (a fixed order)
  if (beta_partial && cb == 0 && threadIdx.x < kStage && threadIdx.x != S_BSQ)
    scal[threadIdx.x] = scal[kStage + threadIdx.x];
  if (beta_partial && cb == 0 && threadIdx.x < 32) {
    double v = 0.0;
    for (int i = threadIdx.x; i < n_beta; i += 32) v += beta_partial[i];
    v = warp_sum<double>(v);
    if (threadIdx.x == 0) scal[kStage + S_BSQ] = v;
  }
  const int2 ch = pch[cb];
  const int n = ch.y - ch.x;
  if ((int)threadIdx.x < n) ent[threadIdx.x] = fe[ch.x + threadIdx.x];
  __syncthreads();
  // every load of the slice is issued before the first add (one round of L2
  // latency instead of one per few partials); the adds keep the slice order
  for (int k = threadIdx.x; k < K; k += blockDim.x) {
    const int64_t out = (int64_t)cb * K + k;
    if (pairs) {
      float2 pr[kPanelChunk];
#pragma unroll
      for (int q = 0; q < kPanelChunk; ++q)
        pr[q] = q < n ? partial_pair(partial, (int64_t)ent[q] * K + k) : make_float2(0.f, 0.f);
      float hi = 0.f, lo = 0.f;
#pragma unroll
      for (int q = 0; q < kPanelChunk; ++q)
        if (q < n) ff_add(hi, lo, pr[q].x, pr[q].y);
      reinterpret_cast<float2*>(csum)[out] = make_float2(hi, -lo);
    } else {
      double pv[kPanelChunk];
#pragma unroll
      for (int q = 0; q < kPanelChunk; ++q)
        pv[q] = q < n ? partial[(int64_t)ent[q] * K + k] : 0.0;
      double acc = 0.0;
#pragma unroll
      for (int q = 0; q < kPanelChunk; ++q)
        if (q < n) acc += pv[q];
      csum[out] = acc;
    }
  }
}

// v'_j = X_j z_j / beta - beta v_j with z_j = sum of the slice sums of panel j
// (X_j = R_j^{-T}); several thread groups split the slice list of a panel.
__global__ void __launch_bounds__(1024) k_panel_T2(
    const double* __restrict__ csum, const int* __restrict__ pco, const double* __restrict__ Xc,
    int K, double* __restrict__ v, double* __restrict__ scal, int identity, int init,
    double* __restrict__ norm_partial, int pairs) {
  extern __shared__ double zsh[];   // [groups][K] then z[K]
  __shared__ double red[33];
  const int s = blockIdx.x;
  const int Kp = (K + 31) & ~31;
  const int G = blockDim.x / Kp;
  const int g = threadIdx.x / Kp, k = threadIdx.x - g * Kp;
  __shared__ double sh_beta, sh_ib;
  if (threadIdx.x == 0) {   // one thread: FP64 sqrt / division are costly
    const double bt = sqrt(scal[kStage + S_BSQ]);   // k_panel_chunks formed beta^2
    sh_beta = bt;
    sh_ib = bt > 0.0 ? 1.0 / bt : 0.0;
  }
  __syncthreads();
  const double beta = sh_beta, ib = sh_ib;
  if (g < G && k < K) {
    double z = 0.0;
    if (pairs) {
      float zs_hi = 0.f, zs_lo = 0.f;
      for (int q = pco[s] + g; q < pco[s + 1]; q += G) {
        const float2 pr = partial_pair(csum, (int64_t)q * K + k);
        ff_add(zs_hi, zs_lo, pr.x, pr.y);
      }
      z = (double)zs_hi + (double)zs_lo;
    } else {
      for (int q = pco[s] + g; q < pco[s + 1]; q += G) z += csum[(int64_t)q * K + k];
    }
    zsh[g * K + k] = z;
  }
  __syncthreads();
  double* zs = zsh + G * K;
  for (int i = threadIdx.x; i < K; i += blockDim.x) {
    double z = 0.0;
    for (int q = 0; q < G; ++q) z += zsh[q * K + i];
    zs[i] = z * ib;
  }
  __syncthreads();
  const double* X = Xc + (int64_t)s * K * K;
  if (!identity) {
    // the groups split the sum over mm <= i into fixed slices
    const int chunk = (K + G - 1) / G;
    if (g < G && k < K) {
      double acc = 0.0;
      const int m1 = min(k + 1, (g + 1) * chunk);
      for (int mm = g * chunk; mm < m1; ++mm) acc += X[mm * K + k] * zs[mm];
      zsh[g * K + k] = acc;
    }
    __syncthreads();
  }
  double nrm = 0.0;
  for (int i = threadIdx.x; i < K; i += blockDim.x) {
    double acc = 0.0;
    if (identity) {
      acc = zs[i];
    } else {
      for (int q = 0; q < G; ++q) acc += zsh[q * K + i];
    }
    const double vold = init ? 0.0 : v[(int64_t)s * K + i];
    const double vn = acc - beta * vold;
    v[(int64_t)s * K + i] = vn;
    nrm += vn * vn;
  }
  double tot = block_sum(nrm, red);
  if (threadIdx.x == 0) norm_partial[blockIdx.x] = tot;
  if (s == 0 && threadIdx.x == 0) scal[kStage + S_BETA] = beta;
}

// k_precond with X_j held as the packed pair triangle (FP32 and DF32 panels):
// the products and sums of t_j = X_j^T v_j run in float-float arithmetic on
// the FP32 pipes (about 2^-48 relative), so that the only FP64 work left is
// splitting v_j and forming t_j.  Same group split and fixed summation order
// as k_precond.
__global__ void __launch_bounds__(1024) k_precond_df(const float2* __restrict__ Xt,
                                                     const double* __restrict__ v, int K,
                                                     double* __restrict__ t, int identity,
                                                     double* __restrict__ scal,
                                                     void* __restrict__ tlow, int low_kind) {
  extern __shared__ double psh[];   // vs[K] then part[G][K], here as FP32 pairs
  const int s = blockIdx.x;
  if (s == 0 && threadIdx.x < kStage) scal[threadIdx.x] = scal[kStage + threadIdx.x];
  const double* vv = v + (int64_t)s * K;
  if (identity) {
    for (int i = threadIdx.x; i < K; i += blockDim.x) {
      t[(int64_t)s * K + i] = vv[i];
      store_low(tlow, low_kind, (int64_t)s * K + i, vv[i]);
    }
    return;
  }
  float2* vs = reinterpret_cast<float2*>(psh);
  float2* part = vs + K;
  for (int i = threadIdx.x; i < K; i += blockDim.x) vs[i] = df_split(vv[i]);
  __syncthreads();
  const int Kp = (K + 31) & ~31;
  const int G = blockDim.x / Kp;
  const int g = threadIdx.x / Kp, i = threadIdx.x - g * Kp;
  const int chunk = (K + G - 1) / G;
  const float2* X = Xt + (int64_t)s * tri_pairs(K);
  if (g < G && i < K) {
    float S = 0.f, C = 0.f;
    const int m1 = min(K, (g + 1) * chunk);
    for (int m = max(i, g * chunk); m < m1; ++m) {
      const float2 x = X[m * (m + 1) / 2 + i];
      df_acc(S, C, x.x, x.y, vs[m].x, vs[m].y);
    }
    part[g * K + i] = make_float2(S, C);
  }
  __syncthreads();
  for (int j = threadIdx.x; j < K; j += blockDim.x) {
    float2 a = part[j];
    for (int q = 1; q < G; ++q) a = df_add(a, part[q * K + j]);
    const double acc = (double)a.x + (double)a.y;
    t[(int64_t)s * K + j] = acc;
    store_low(tlow, low_kind, (int64_t)s * K + j, acc);
  }
}

// Block size of the kernels that apply the packed pair triangle: four groups
// of K (rounded up to 32) threads, 128 to 512 -- at K = 128, 512 threads and
// about 70 KB of shared memory, three blocks per SM, so that every panel of
// the 2-D workloads (a few hundred) runs in one wave; at K = 64, 256 threads,
// so that the thousands of small panels of the large 2-D workload run with
// more blocks per SM rather than more idle threads per block.  Without a
// preconditioner (X = I, no triangle) the tail's products vanish and one
// group of at least 128 threads does the rest, with no triangle in shared
// memory, so that many blocks share an SM.
constexpr int kTriThreads = 512;
static int tri_threads(int K, bool ident = false) {
  const int Kp = (K + 31) & ~31;
  if (ident) return std::max(128, Kp);
  return std::min(kTriThreads, std::max(128, 4 * Kp));
}

// Shared memory of those kernels: the triangle (none for X = I), a K-vector of
// pairs, G x K group partials and the copy's mbarrier.
static size_t tri_smem_bytes(int K, bool ident = false) {
  const int Kp = (K + 31) & ~31;
  const int G = tri_threads(K, ident) / Kp;
  return (size_t)((ident ? 0 : tri_pairs(K)) + K + (int64_t)G * K) * sizeof(float2) + 16;
}

// One bulk copy of panel s's triangle into shared memory (thread 0 issues it;
// the caller's next __syncthreads publishes the mbarrier's initialisation).
__device__ __forceinline__ void tri_fetch(float2* Xs, const float2* __restrict__ Xt, int s, int K,
                                          uint64_t* bar) {
  if (threadIdx.x == 0) {
    const int64_t P = tri_pairs(K);
    sm100::mbar_init(bar, 1);
    sm100::fence_mbar_init();
    sm100::mbar_arrive_expect_tx(bar, (uint32_t)(P * sizeof(float2)));
    sm100::bulk_load(Xs, Xt + (int64_t)s * P, (uint32_t)(P * sizeof(float2)), bar);
  }
}

// Bounded wait for tri_fetch's copy.  On a timeout flags[3] is raised and the
// block waits once more (bounded) for the copy still in flight, then goes on
// with whatever arrived; the host turns the flag into ELMFB_ERR_TIMEOUT.
__device__ __forceinline__ void tri_wait(uint64_t* bar, int* __restrict__ flags) {
  if (!sm100::mbar_wait(bar, 0)) {
    if (threadIdx.x == 0) atomicOr(&flags[3], 1);
    sm100::mbar_wait(bar, 0);
  }
}

// First half of the LSQR tail for FP32-pair partials with X_j as the packed
// pair triangle (Xs, fetched by tri_fetch): beta (from beta^2 formed by
// k_panel_chunks), z_j =
// the sum of panel j's slice sums, scaled by 1/beta, y = X_j z_j, v' = y -
// beta v_j (written to v), in float-float arithmetic except beta, v' and its
// norm.  y_k = sum_{m<=k} X_km z_m: each warp takes rows k = w, w + nw, ...
// four at a time, its lanes the terms m = l, l + 32, ..., one warp_sum4_df per
// four rows (a fixed order).  Returns ||v'||^2 of the panel in every thread
// and leaves v' as pairs in zs; block 0 stages beta.
__device__ double tail_v_tri(const double* __restrict__ csum, const int* __restrict__ pco,
                             int K, double* __restrict__ v, double* __restrict__ scal, int init,
                             const float2* Xs, float2* zs, float2* part, uint64_t* bar,
                             int* __restrict__ flags, int s, bool ident) {
  __shared__ double red[33];
  __shared__ double sh_beta;
  __shared__ float2 sh_ib;
  const int Kp = (K + 31) & ~31;
  const int G = blockDim.x / Kp;
  const int g = threadIdx.x / Kp, k = threadIdx.x - g * Kp;
  if (threadIdx.x == 0) {   // one thread: FP64 sqrt / division are costly
    const double bt = sqrt(scal[kStage + S_BSQ]);
    sh_beta = bt;
    sh_ib = df_split(bt > 0.0 ? 1.0 / bt : 0.0);
  }
  if (g < G && k < K) {
    float hi = 0.f, lo = 0.f;
#pragma unroll 8
    for (int q = pco[s] + g; q < pco[s + 1]; q += G) {
      const float2 pr = partial_pair(csum, (int64_t)q * K + k);
      ff_add(hi, lo, pr.x, pr.y);
    }
    part[g * K + k] = make_float2(hi, lo);
  }
  __syncthreads();
  const double beta = sh_beta;
  const float2 ib = sh_ib;
  for (int i = threadIdx.x; i < K; i += blockDim.x) {
    float2 z = part[i];
    for (int q = 1; q < G; ++q) z = df_add(z, part[q * K + i]);
    float S = 0.f, C = 0.f;
    df_acc(S, C, z.x, z.y, ib.x, ib.y);
    zs[i] = make_float2(S, C);
  }
  __syncthreads();
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
  float2* ys = ident ? zs : part;   // the group partials are consumed
  if (!ident) tri_wait(bar, flags);
  for (int k0 = wid; k0 < K && !ident; k0 += 4 * nw) {
    float2 acc[4];
#pragma unroll
    for (int r = 0; r < 4; ++r) {
      const int kr = k0 + r * nw;
      float S = 0.f, C = 0.f;
      if (kr < K) {
        const float2* row = Xs + kr * (kr + 1) / 2;
        for (int m = lane; m <= kr; m += 32) df_acc(S, C, row[m].x, row[m].y, zs[m].x, zs[m].y);
      }
      acc[r] = make_float2(S, C);
    }
    const float2 tot = warp_sum4_df(acc[0], acc[1], acc[2], acc[3], lane);
    const int kr = k0 + (lane >> 3) * nw;
    if ((lane & 7) == 0 && kr < K) ys[kr] = tot;
  }
  __syncthreads();
  double nrm = 0.0;
  for (int i = threadIdx.x; i < K; i += blockDim.x) {
    const double acc = (double)ys[i].x + (double)ys[i].y;
    const double vold = init ? 0.0 : v[(int64_t)s * K + i];
    const double vn = acc - beta * vold;
    v[(int64_t)s * K + i] = vn;
    zs[i] = df_split(vn);   // z is consumed: v' as pairs for X^T v'
    nrm += vn * vn;
  }
  if (s == 0 && threadIdx.x == 0) scal[kStage + S_BETA] = beta;
  return block_sum(nrm, red);
}

// Second half's product for the packed pair triangle: t_s = X_s^T v_s (v_s as
// pairs in vs) in float-float arithmetic, with t's low-precision copy.
// t_i = sum_{m>=i} X_mi v_m: G groups of Kp threads take fixed slices of the
// rows m, lane i column i; all lanes of a warp walk the same rows (contiguous
// in shared memory), those with i > m idle; then one pass adds the group sums
// in order.
__device__ void tail_t_tri(int K, const float2* Xs, const float2* vs, float2* part,
                           double* __restrict__ t, void* __restrict__ tlow, int low_kind, int s) {
  const int Kp = (K + 31) & ~31;
  const int G = blockDim.x / Kp;
  const int g = threadIdx.x / Kp, i = threadIdx.x - g * Kp;
  const int chunk = (K + G - 1) / G;
  const int m0 = g * chunk, m1 = min(K, m0 + chunk);
  if (g < G && i < K) {
    float S = 0.f, C = 0.f;
    const int wlo = (i & ~31);   // rows below the warp's first column hold nothing for it
#pragma unroll 4
    for (int m = max(m0, wlo); m < m1; ++m) {
      const float2 xv = Xs[m * (m + 1) / 2 + i];
      if (m >= i) df_acc(S, C, xv.x, xv.y, vs[m].x, vs[m].y);
    }
    part[g * K + i] = make_float2(S, C);
  }
  __syncthreads();
  const int64_t o = (int64_t)s * K;
  for (int j = threadIdx.x; j < K; j += blockDim.x) {
    float2 a = part[j];
    for (int q = 1; q < G; ++q) a = df_add(a, part[q * K + j]);
    const double acc = (double)a.x + (double)a.y;
    t[o + j] = acc;
    store_low(tlow, low_kind, o + j, acc);
  }
}

// Shared-memory layout of the packed-triangle kernels: X, a K-vector of
// pairs, part[G][K], the mbarrier.
struct TriSmem {
  float2* Xs;
  float2* vec;
  float2* part;
  uint64_t* bar;
  __device__ TriSmem(unsigned char* raw, int K, bool ident = false) {
    const int G = blockDim.x / ((K + 31) & ~31);
    Xs = reinterpret_cast<float2*>(raw);
    vec = Xs + (ident ? 0 : tri_pairs(K));
    part = vec + K;
    bar = reinterpret_cast<uint64_t*>(part + (int64_t)G * K);
  }
};

// v'_j = X_j z_j / beta - beta v_j with z_j = sum of the entry partials of panel j
// (X_j = R_j^{-T}); writes v' (unnormalised) and ||v'||^2 per block.
__global__ void k_panel_T(const double* __restrict__ partial, const int* __restrict__ pent_off,
                          const int* __restrict__ pent, const double* __restrict__ Xc, int K,
                          const double* __restrict__ beta_partial, int n_beta_partial,
                          double* __restrict__ v, double* __restrict__ scal, int identity,
                          int init, double* __restrict__ norm_partial) {
  extern __shared__ double zs[];
  __shared__ double red[33];
  const int s = blockIdx.x;
  // beta = sqrt(sum of gather partials), same fixed order in every block
  double b2 = 0.0;
  for (int i = 0; i < n_beta_partial; ++i) b2 += beta_partial[i];
  const double beta = sqrt(b2);
  const double ib = beta > 0.0 ? 1.0 / beta : 0.0;
  for (int k = threadIdx.x; k < K; k += blockDim.x) {
    double z = 0.0;
    for (int q = pent_off[s]; q < pent_off[s + 1]; ++q) z += partial[(int64_t)pent[q] * K + k];
    zs[k] = z * ib;
  }
  __syncthreads();
  const double* X = Xc + (int64_t)s * K * K;
  double nrm = 0.0;
  for (int i = threadIdx.x; i < K; i += blockDim.x) {
    double acc;
    if (identity) {
      acc = zs[i];
    } else {
      acc = 0.0;
      for (int m = 0; m <= i; ++m) acc += X[m * K + i] * zs[m];   // X_im, column-major
    }
    double vold = init ? 0.0 : v[(int64_t)s * K + i];
    double vn = acc - beta * vold;
    v[(int64_t)s * K + i] = vn;
    nrm += vn * vn;
  }
  double tot = block_sum(nrm, red);
  if (threadIdx.x == 0) norm_partial[blockIdx.x] = tot;
  if (s == 0 && threadIdx.x == 0) scal[kStage + S_BETA] = beta;   // staged beta_{i+1}
}

// LSQR scalar recurrence + vector updates.  Every block recomputes the scalars
// (identical fixed-order sums); block 0 commits them.
__global__ void k_update(double* __restrict__ scal, const double* __restrict__ alpha_partial,
                         int n_alpha_partial, double* __restrict__ v, double* __restrict__ w,
                         double* __restrict__ x, int64_t N, int init) {
  __shared__ double shs;
  __shared__ double shv[4];   // ia, phi_rho, theta_rho (scalars formed by one thread)
  const double a2 = block_partial_sum(alpha_partial, n_alpha_partial, &shs);
  const double beta = scal[kStage + S_BETA];   // beta_{i+1}
  double alpha = 0.0, ia = 0.0, phi_rho = 0.0, theta_rho = 0.0;
  double rhobar_new = 0.0, phibar_new = 0.0, anorm2 = scal[S_ANORM2], arnorm = 0.0;
  if (threadIdx.x == 0) {   // one thread: the recurrence needs FP64 sqrt / divisions
    alpha = sqrt(a2);
    ia = alpha > 0.0 ? 1.0 / alpha : 0.0;
    if (init) {
      // beta_1 u_1 = b, alpha_1 v_1 = A^T u_1, w_1 = v_1, phibar_1 = beta_1, rhobar_1 = alpha_1
      rhobar_new = alpha;
      phibar_new = beta;
      anorm2 = alpha * alpha;
      arnorm = alpha * beta;
    } else {
      const double rhobar = scal[S_RHOBAR], phibar = scal[S_PHIBAR];
      const double rho = sqrt(rhobar * rhobar + beta * beta);
      const double c = rho > 0.0 ? rhobar / rho : 1.0;
      const double sn = rho > 0.0 ? beta / rho : 0.0;
      const double theta = sn * alpha;
      rhobar_new = -c * alpha;
      const double phi = c * phibar;
      phibar_new = sn * phibar;
      phi_rho = rho > 0.0 ? phi / rho : 0.0;
      theta_rho = rho > 0.0 ? theta / rho : 0.0;
      anorm2 += alpha * alpha + beta * beta;
      arnorm = phibar_new * alpha * fabs(c);
    }
    shv[0] = ia;
    shv[1] = phi_rho;
    shv[2] = theta_rho;
  }
  __syncthreads();
  ia = shv[0];
  phi_rho = shv[1];
  theta_rho = shv[2];
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < N;
       i += (int64_t)gridDim.x * blockDim.x) {
    const double vn = v[i] * ia;   // v_{i+1}
    if (init) {
      w[i] = vn;
      x[i] = 0.0;
    } else {
      const double wi = w[i];
      x[i] += phi_rho * wi;
      w[i] = vn - theta_rho * wi;
    }
    v[i] = vn;
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    double* sg = scal + kStage;
    sg[S_ALPHA] = alpha;
    sg[S_BETA] = beta;
    sg[S_RHOBAR] = rhobar_new;
    sg[S_PHIBAR] = phibar_new;
    sg[S_ANORM2] = anorm2;
    sg[S_RNORM] = phibar_new;
    sg[S_ARNORM] = arnorm;
    sg[S_BNORM] = init ? beta : scal[S_BNORM];
    sg[S_ITER] = scal[S_ITER] + (init ? 0.0 : 1.0);
    sg[S_BAD] = (scal[S_BAD] != 0.0 || !(alpha == alpha) || !(beta == beta)) ? 1.0 : 0.0;
    record_bidiagonal(scal, sg[S_ITER], alpha, beta);
  }
}

// One step of the LSQR recurrence (Paige & Saunders 1982, the plane rotation
// from rhobar, beta and alpha) from alpha^2, beta_{i+1} and the committed
// scalars; with `stage`, all scalars go to the staged slots (S_TSCALE = 1/alpha
// included).  Returns 1/alpha, phi/rho and theta/rho (0 and 0 at the start).
struct LsqrStep {
  double ia, phi_rho, theta_rho;
};
__device__ LsqrStep lsqr_recurrence(double* __restrict__ scal, double a2, double beta, int init,
                                    bool stage) {
  const double alpha = sqrt(a2);
  LsqrStep r{alpha > 0.0 ? 1.0 / alpha : 0.0, 0.0, 0.0};
  double rhobar_new, phibar_new, anorm2, arnorm;
  if (init) {
    rhobar_new = alpha;
    phibar_new = beta;
    anorm2 = alpha * alpha;
    arnorm = alpha * beta;
  } else {
    const double rhobar = scal[S_RHOBAR], phibar = scal[S_PHIBAR];
    const double rho = sqrt(rhobar * rhobar + beta * beta);
    const double irho = rho > 0.0 ? 1.0 / rho : 0.0;   // one FP64 division, then products
    const double c = rho > 0.0 ? rhobar * irho : 1.0;
    const double sn = beta * irho;
    const double theta = sn * alpha;
    rhobar_new = -c * alpha;
    const double phi = c * phibar;
    phibar_new = sn * phibar;
    r.phi_rho = phi * irho;
    r.theta_rho = theta * irho;
    anorm2 = scal[S_ANORM2] + alpha * alpha + beta * beta;
    arnorm = phibar_new * alpha * fabs(c);
  }
  if (stage) {
    double* sg = scal + kStage;
    sg[S_ALPHA] = alpha;
    sg[S_BETA] = beta;
    sg[S_RHOBAR] = rhobar_new;
    sg[S_PHIBAR] = phibar_new;
    sg[S_ANORM2] = anorm2;
    sg[S_RNORM] = phibar_new;
    sg[S_ARNORM] = arnorm;
    sg[S_BNORM] = init ? beta : scal[S_BNORM];
    sg[S_ITER] = scal[S_ITER] + (init ? 0.0 : 1.0);
    sg[S_BAD] = (scal[S_BAD] != 0.0 || !(alpha == alpha) || !(beta == beta)) ? 1.0 : 0.0;
    sg[S_PHI_RHO] = r.phi_rho;
    sg[S_THETA_RHO] = r.theta_rho;
    sg[S_TSCALE] = r.ia;
    record_bidiagonal(scal, sg[S_ITER], alpha, beta);
    // the host's stopping tests (Paige & Saunders' btol / atol, and ntol on
    // the normal residual relative to its start), taken here after every
    // iteration: once one is met the next iterations' kernels return at once,
    // so the solve stops at this iteration whatever the host's check interval
    if (scal[kStage + S_STOP_ON] != 0.0) {
      bool done = !(alpha > 0.0) || !(beta > 0.0) || sg[S_BAD] != 0.0;
      if (init) {
        sg[S_ARN0] = arnorm;
      } else {
        const double anorm = sqrt(anorm2), rn = phibar_new;
        const double btol = scal[kStage + S_BTOL], atol = scal[kStage + S_ATOL];
        const double ntol = scal[kStage + S_NTOL];
        done = done || (btol > 0.0 && rn <= btol * sg[S_BNORM]) ||
               (atol > 0.0 && anorm > 0.0 && rn > 0.0 && arnorm <= atol * anorm * rn) ||
               (ntol > 0.0 && arnorm <= ntol * scal[kStage + S_ARN0]);
      }
      sg[S_DONE] = done ? 1.0 : 0.0;
    }
  }
  return r;
}

// One LSQR step on panel s's K entries (Paige & Saunders 1982: the plane
// rotation from rhobar, beta and alpha, then the v, w, x updates): alpha =
// ||v'|| (every block sums the norm partials in the same fixed order, with all
// its threads; thread 0 runs the recurrence, block 0 stages the scalars, as
// k_update).  sink(i, v_i)
// receives each normalised v entry.  The committed scalars are read here and
// committed later by k_panel_chunks, so no block overwrites what another
// block reads.  Ends with a __syncthreads.
template <class Sink>
__device__ __forceinline__ void lsqr_step_panel(double* __restrict__ scal,
                                                const double* __restrict__ alpha_partial,
                                                int n_alpha_partial, double* __restrict__ v,
                                                double* __restrict__ w, double* __restrict__ x,
                                                int K, int init, Sink sink) {
  __shared__ double red[33];
  __shared__ double shv[4];
  const int s = blockIdx.x;
  // alpha^2: thread-strided sums of the partials, then block_sum (a fixed
  // order, the same in every block)
  double a2 = 0.0;
  for (int i = threadIdx.x; i < n_alpha_partial; i += blockDim.x) a2 += alpha_partial[i];
  a2 = block_sum(a2, red);
  const double beta = scal[kStage + S_BETA];   // beta_{i+1}
  if (threadIdx.x == 0) {   // one thread: the recurrence needs FP64 sqrt / divisions
    const LsqrStep st = lsqr_recurrence(scal, a2, beta, init, s == 0);
    shv[0] = st.ia;
    shv[1] = st.phi_rho;
    shv[2] = st.theta_rho;
  }
  __syncthreads();
  const double ia = shv[0];
  const double phi_rho = shv[1];
  const double theta_rho = shv[2];
  const int64_t o = (int64_t)s * K;
  for (int i = threadIdx.x; i < K; i += blockDim.x) {
    const double vn = v[o + i] * ia;   // v_{i+1}
    if (init) {
      w[o + i] = vn;
      x[o + i] = 0.0;
    } else {
      const double wi = w[o + i];
      x[o + i] += phi_rho * wi;
      w[o + i] = vn - theta_rho * wi;
    }
    v[o + i] = vn;
    sink(i, vn);
  }
  __syncthreads();
}

// The fused path's k_update merged with the next iteration's k_precond, one
// block per subdomain, FP64 X (FP64 panels) or no preconditioner: the LSQR
// step, then t_s = X_s^T v_s for the next fused pass, with t's low-precision
// copy.
__global__ void __launch_bounds__(1024) k_update_precond(
    double* __restrict__ scal, const double* __restrict__ alpha_partial, int n_alpha_partial,
    double* __restrict__ v, double* __restrict__ w, double* __restrict__ x, int K, int init,
    int identity, const double* __restrict__ Xr, double* __restrict__ t,
    void* __restrict__ tlow, int low_kind) {
  extern __shared__ double psh[];   // vs[K] then part[G][K]
  const int64_t o = (int64_t)blockIdx.x * K;
  double* vs = psh;
  lsqr_step_panel(scal, alpha_partial, n_alpha_partial, v, w, x, K, init,
                  [&](int i, double vn) {
                    if (identity) {
                      t[o + i] = vn;
                      store_low(tlow, low_kind, o + i, vn);
                    } else {
                      vs[i] = vn;
                    }
                  });
  if (identity) return;
  // t_s = X_s^T v_s: G groups split each sum into fixed slices (as k_precond)
  const int Kp = (K + 31) & ~31;
  const int G = blockDim.x / Kp;
  const int g = threadIdx.x / Kp, i = threadIdx.x - g * Kp;
  const int chunk = (K + G - 1) / G;
  const int m1 = min(K, (g + 1) * chunk);
  double* part = vs + K;
  const double* X = Xr + (int64_t)blockIdx.x * K * K;
  if (g < G && i < K) {
    double acc = 0.0;
    for (int m = max(i, g * chunk); m < m1; ++m) acc += X[m * K + i] * vs[m];
    part[g * K + i] = acc;
  }
  __syncthreads();
  for (int j = threadIdx.x; j < K; j += blockDim.x) {
    double acc = 0.0;
    for (int q = 0; q < G; ++q) acc += part[q * K + j];
    t[o + j] = acc;
    store_low(tlow, low_kind, o + j, acc);
  }
}

// The LSQR iteration's tail for FP32 and DF32 panels in one kernel, one block
// per panel, with the update of the previous iteration deferred into it:
//  1. x += (phi/rho) w, w = v - (theta/rho) w with v = v' / alpha (v' as the
//     previous call left it; 1/alpha and the ratios from the committed
//     scalars); not at the start of a solve, where w and x are zero and the
//     ratios are staged as 0 (so the next call sets w = v_1);
//  2. v'' = X z / beta - beta v, stored unnormalised, its norm partial
//     (tail_v_tri; the triangle's bulk copy is issued first);
//  3. t' = X^T v'' (tail_t_tri) for the next fused pass, which multiplies
//     M t' by the staged 1/alpha (mode 2);
//  4. the last block to finish (a counter, reset by that block) adds all
//     norm partials with the whole block in a fixed order, runs the
//     recurrence and stages every scalar.
// The solve's end applies the last deferred x update (k_lsqr_finish).
__global__ void __launch_bounds__(kTriThreads, 3) k_lsqr_tail_tri(
    const double* __restrict__ csum, const int* __restrict__ pco, const float2* __restrict__ Xt,
    int K, double* __restrict__ v, double* __restrict__ w, double* __restrict__ x,
    double* __restrict__ scal, int init, double* __restrict__ norm_partial,
    double* __restrict__ t, void* __restrict__ tlow, int low_kind,
    unsigned int* __restrict__ counter, int* __restrict__ flags, const BatchInst* __restrict__ bi,
    const int2* __restrict__ bmap) {
  extern __shared__ __align__(16) unsigned char trsm[];
  __shared__ double red[33];
  __shared__ int last;
  int s = blockIdx.x, nblk = gridDim.x;   // this block's panel, the instance's panels
  if (bi) {   // a multi-instance launch: the panel's instance supplies every array
    const int2 bm = bmap[blockIdx.x];
    const BatchInst& I = bi[bm.x];
    csum = I.csum;
    pco = I.pco;
    Xt = I.Xt;
    v = I.v;
    w = I.w;
    x = I.x;
    scal = I.scal;
    norm_partial = I.vpart;
    t = I.t;
    tlow = const_cast<float*>(I.tlow);
    counter = I.counter;
    flags = I.flags;
    s = bm.y;
    nblk = I.n_sub;
  }
  if (scal[kStage + S_DONE] != 0.0) return;   // LSQR stopped on the device
  const bool ident = Xt == nullptr;   // no preconditioner: X = I
  TriSmem sm(trsm, K, ident);
  if (!ident) tri_fetch(sm.Xs, Xt, s, K, sm.bar);
  const int64_t o = (int64_t)s * K;
  if (!init) {
    const double ia = scal[S_TSCALE], pr = scal[S_PHI_RHO], tr = scal[S_THETA_RHO];
    for (int i = threadIdx.x; i < K; i += blockDim.x) {
      const double vn = v[o + i] * ia;
      const double wi = w[o + i];
      x[o + i] += pr * wi;
      w[o + i] = vn - tr * wi;
      v[o + i] = vn;
    }
  }
  const double nrm = tail_v_tri(csum, pco, K, v, scal, init, sm.Xs, sm.vec, sm.part, sm.bar,
                                flags, s, ident);
  if (threadIdx.x == 0) norm_partial[s] = nrm;
  __syncthreads();
  if (ident) {   // t' = v'
    for (int j = threadIdx.x; j < K; j += blockDim.x) {
      const double vn = v[o + j];
      t[o + j] = vn;
      store_low(tlow, low_kind, o + j, vn);
    }
  } else {
    tail_t_tri(K, sm.Xs, sm.vec, sm.part, t, tlow, low_kind, s);
  }
  // the last block: alpha, the recurrence, the staged scalars
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) last = atomicAdd(counter, 1u) == (unsigned)nblk - 1;
  __syncthreads();
  if (!last) return;
  __threadfence();
  double a2 = 0.0;
  for (int i = threadIdx.x; i < nblk; i += blockDim.x) a2 += __ldcg(norm_partial + i);
  a2 = block_sum(a2, red);
  if (threadIdx.x == 0) {
    lsqr_recurrence(scal, a2, sqrt(scal[kStage + S_BSQ]), init, true);
    *counter = 0u;
  }
}

// The last deferred update of k_lsqr_tail_tri: x += (phi/rho) w, ratio staged.
__global__ void k_lsqr_finish(const double* __restrict__ scal, const double* __restrict__ w,
                              double* __restrict__ x, int64_t N) {
  const double pr = scal[kStage + S_PHI_RHO];
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < N;
       i += (int64_t)gridDim.x * blockDim.x)
    x[i] += pr * w[i];
}

__global__ void k_add_to(double* __restrict__ a, const double* __restrict__ d, int64_t N) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < N;
       i += (int64_t)gridDim.x * blockDim.x)
    a[i] += d[i];
}

}  // namespace

// ----------------------------------------------------------------------------
namespace {

struct SolveLayout {
  int n_chunks = 0;
  std::vector<int4> chunks;
  std::vector<int> chunk_off;
  std::vector<int> pent_off, pent;
};

}  // namespace

// Heuristic rows per fused-pass work unit (see build_fused_plan).
int64_t fused_unit_target(const elmfb_ctx* h) {
  const double row_bytes =
      (double)h->NPR / (double)std::max<int64_t>(h->NR, 1) * h->K * (double)h->panel_elem();
  const int64_t by_bytes = (int64_t)((2.0 * 1024 * 1024) / std::max(row_bytes, 1.0));
  return std::min<int64_t>(
      kMaxUnitRows, std::max<int64_t>(8, std::max(h->NR / 608, by_bytes) & ~int64_t(7)));
}

bool build_fused_plan(elmfb_ctx* h, FusedPlan& fp, int unit_rows) {
  const int K = h->K;
  if (h->max_cover > 32 || K > 128) return false;
  cudaStream_t st = h->stream;
  fp.threads = 32 * std::max(1, h->max_cover);
  // rows per work unit: about NR / 608 (4 waves of one-CTA-per-SM units), but
  // at least the rows of about 2 MB of covering panels, so that a unit's
  // start-up (barrier set-up, the first copies in flight) stays small next to
  // its stream.  2-D workload (17 panels of 128 FP32): 264 rows either way;
  // DHO (13 panels of 96 DF32): 200 rather than 32 rows, one wave of whole
  // cells, fused pass 75 -> 68 us.  ELMFB_FUSED_UNIT_ROWS overrides it (a
  // tuning knob: units change the timing and the grouping of the Mᵀu partial
  // sums, not the order of the terms within a row)
  const double row_bytes =
      (double)h->NPR / (double)std::max<int64_t>(h->NR, 1) * K * (double)h->panel_elem();
  const int64_t by_bytes = (int64_t)((2.0 * 1024 * 1024) / std::max(row_bytes, 1.0));
  int64_t target = std::min<int64_t>(
      kMaxUnitRows, std::max<int64_t>(8, std::max(h->NR / 608, by_bytes) & ~int64_t(7)));
  if (const char* e = getenv("ELMFB_FUSED_UNIT_ROWS")) {
    const long v = atol(e);
    if (v >= 8 && v <= kMaxUnitRows) target = v & ~7L;
  }
  if (unit_rows >= 8) target = std::min<int64_t>(kMaxUnitRows, unit_rows & ~7);
  std::vector<int4> units;
  std::vector<std::vector<int>> plist(h->n_sub);
  int pbase = 0;
  for (int c = 0; c < h->n_cells; ++c) {
    const int pad = h->cell_pstart[c + 1] - h->cell_pstart[c];
    const int m = h->cover_off[c + 1] - h->cover_off[c];
    if (pad == 0) continue;
    const int nunit = (int)ceil_div(pad, target);
    const int per = (int)(ceil_div(ceil_div(pad, nunit), kFusedRows) * kFusedRows);
    for (int r = 0; r < pad; r += per) {
      units.push_back(make_int4(c, r, std::min(pad, r + per), pbase));
      for (int w = 0; w < m; ++w) plist[h->cover_sub[h->cover_off[c] + w]].push_back(pbase + w);
      pbase += m;
    }
  }
  fp.n_units = (int)units.size();
  fp.max_unit_rows = 0;
  for (const int4& u4 : units) fp.max_unit_rows = std::max(fp.max_unit_rows, u4.z - u4.y);
  std::vector<int> fo(h->n_sub + 1, 0), fe;
  fe.reserve(pbase);
  for (int s2 = 0; s2 < h->n_sub; ++s2) {
    fo[s2] = (int)fe.size();
    fe.insert(fe.end(), plist[s2].begin(), plist[s2].end());
  }
  fo[h->n_sub] = (int)fe.size();
  fp.units.alloc(std::max<size_t>(units.size(), 1) * sizeof(int4), st);
  fp.fo.alloc(fo.size() * sizeof(int), st);
  fp.fe.alloc(std::max<size_t>(fe.size(), 1) * sizeof(int), st);
  fp.part.alloc(std::max<int64_t>(pbase, 1) * K * sizeof(double), st);
  fp.pairs = !h->fp64();
  // fixed slices of at most kPanelChunk partials per panel: the big panels of
  // the coarse levels (one partial per unit of every cell) are summed by many
  // blocks, then each panel adds its few slice sums in order
  {
    std::vector<int2> pch;
    std::vector<int> pco(h->n_sub + 1, 0);
    for (int s2 = 0; s2 < h->n_sub; ++s2) {
      pco[s2] = (int)pch.size();
      for (int e0 = fo[s2]; e0 < fo[s2 + 1]; e0 += kPanelChunk)
        pch.push_back(make_int2(e0, std::min(e0 + kPanelChunk, fo[s2 + 1])));
    }
    pco[h->n_sub] = (int)pch.size();
    fp.n_pchunks = (int)pch.size();
    fp.pch.alloc(std::max<size_t>(pch.size(), 1) * sizeof(int2), st);
    fp.pco.alloc(pco.size() * sizeof(int), st);
    fp.csum.alloc(std::max<size_t>(pch.size(), 1) * K * sizeof(double), st);
    if (!pch.empty())
      CUDA_CHECK(cudaMemcpyAsync(fp.pch.p, pch.data(), pch.size() * sizeof(int2),
                                 cudaMemcpyHostToDevice, st));
    CUDA_CHECK(cudaMemcpyAsync(fp.pco.p, pco.data(), pco.size() * sizeof(int),
                               cudaMemcpyHostToDevice, st));
  }
  if (fp.pairs)
    fp.tf.alloc(std::max<int64_t>(h->NPhi, 1) * (h->df32() ? sizeof(float2) : sizeof(float)), st);
  CUDA_CHECK(cudaMemcpyAsync(fp.units.p, units.data(), units.size() * sizeof(int4),
                             cudaMemcpyHostToDevice, st));
  CUDA_CHECK(cudaMemcpyAsync(fp.fo.p, fo.data(), fo.size() * sizeof(int), cudaMemcpyHostToDevice,
                             st));
  CUDA_CHECK(cudaMemcpyAsync(fp.fe.p, fe.data(), fe.size() * sizeof(int), cudaMemcpyHostToDevice,
                             st));
  return true;
}

// Shared memory for the fused pass's ring and staged u values, per CTA (one
// CTA per SM): 220 KB, or ELMFB_FUSED_SMEM_KB (a tuning knob; the stage count
// changes timing only, but a budget without room for three 8-row stages makes
// the pass take 4-row chunks, which group the compensated sums differently).
static size_t fused_ring_budget() {
  static const size_t kb = [] {
    const char* e = getenv("ELMFB_FUSED_SMEM_KB");
    const long v = e ? atol(e) : 0;
    return (size_t)(v >= 64 && v <= 220 ? v : 220);
  }();
  return kb * 1024;
}

// Shared memory per CTA of k_fused_pipe when several CTAs share an SM.  A
// CTA's chunk chain (copy in, the per-row dots, u', the M^T u' update) is
// latency-bound and one chunk carries the rows of all m covering panels, so a
// CTA streams about m times faster with m panels: with few panels per cell,
// several CTAs per SM, each keeping four 8-row stages (2-D single-level cells,
// 4 panels of K = 128 FP32: 2.98 TB/s at one CTA per SM, 5.3 TB/s at three);
// the multilevel workloads' 17 panels stay at one.  ELMFB_FUSED_SMEM_KB fixes
// the one-CTA budget instead, ELMFB_FUSED_CTAS the number of CTAs (tuning
// knobs: both change timing only).
constexpr size_t kSmemPerSM = 228 * 1024;
constexpr size_t kCtaSmemReserve = 4096;   // the kernel's static arrays and the per-CTA reserve
static size_t fused_pipe_budget(int mmax, int K, size_t elem, size_t u_bytes, int threads) {
  if (getenv("ELMFB_FUSED_SMEM_KB")) return fused_ring_budget();
  const char* e = getenv("ELMFB_FUSED_CTAS");
  const int force = e ? atoi(e) : 0;
  if (force == 1) return fused_ring_budget();
  const size_t stage8 = std::max<size_t>((size_t)mmax * 8 * K * elem, 1);
  for (int n = 4; n >= 2; --n) {
    if ((force && n != force) || threads * n > 2048) continue;
    const size_t b = kSmemPerSM / n - kCtaSmemReserve;
    if (b > u_bytes && (b - u_bytes) / stage8 >= 4) return b;
  }
  return fused_ring_budget();
}

// The launch shape of k_fused_pipe for T panels: rows per chunk, ring stages,
// dynamic shared memory, threads.  False when the pass takes the register
// kernel k_fused instead.
template <class T>
static bool fused_pipe_shape(const elmfb_ctx* h, const FusedPlan& fp, int& rows, int& S,
                             size_t& smem, int& pthreads) {
  const int K = h->K;
  // bulk-copy ring: S stages of (covering panels x rows x K) elements
  const int mmax = std::max(1, h->max_cover);
  // the unit's u values, staged after the ring (16-byte aligned for the copy)
  const size_t u_bytes =
      ((size_t)std::max(8, std::min(fp.max_unit_rows, kMaxUnitRows)) * sizeof(double) + 15) &
      ~size_t(15);
  pthreads = fp.threads + 64;   // covering-panel warps + producer + control
  const size_t budget = fused_pipe_budget(mmax, K, sizeof(T), u_bytes, pthreads);
  auto stages_for = [&](int r) {
    const size_t sb = std::max<size_t>((size_t)mmax * r * K * sizeof(T), 1);
    return (int)std::min<size_t>(kPipeMaxStages, (budget - u_bytes) / sb);
  };
  // rows per chunk: 8 while the ring still holds three such stages (fewer,
  // larger copies and half the per-chunk synchronisation; on the 2-D
  // workload's 17 covering panels a pass drops from 0.26 to 0.20 ms), else 4.
  // ELMFB_FUSED_ROWS=4 forces 4 (it changes the grouping of the compensated
  // sums, not the order of the terms within a row).
  const char* erows = getenv("ELMFB_FUSED_ROWS");
  rows = ((erows && atoi(erows) == 4) || stages_for(8) < 3) ? 4 : 8;
  S = stages_for(rows);
  smem = (size_t)S * mmax * rows * K * sizeof(T) + u_bytes;
  const char* force_regs = getenv("ELMFB_FUSED_REGISTERS");
  // bulk copies need 16-byte aligned rows (K sizeof(T) a multiple of 16); the
  // ring needs the two stages in use plus at least one in flight
  return S >= 3 && pthreads <= 1024 && (K * sizeof(T)) % 16 == 0 &&
         !(force_regs && force_regs[0] == '1');
}

template <class T>
void launch_fused(elmfb_ctx* h, FusedPlan& fp, const double* t64, int mode, double* scal,
                  double* gpart, const void* tlow) {
  const int K = h->K;
  const int fpl = (K + 31) / 32;
  const int fthreads = fp.threads;
  cudaStream_t st = h->stream;
  if constexpr (std::is_same<T, df2>::value) {
    // DF32 panels: the pass reads t as FP32 pairs
    if (!tlow) {
      k_to_df<<<(unsigned)std::min<int64_t>(ceil_div(h->NPhi, 256), 1216), 256, 0, st>>>(
          t64, fp.tf.as<float2>(), h->NPhi);
      count_launch(h);
      tlow = fp.tf.p;
    }
    const int mmax = std::max(1, h->max_cover);
    const size_t stage_bytes = (size_t)mmax * kPipeRows * K * sizeof(float2);
    const size_t u_bytes = kMaxUnitRows * sizeof(double);
    const int S = (int)std::min<size_t>(kPipeMaxStages,
                                        (fused_ring_budget() - u_bytes) / std::max<size_t>(stage_bytes, 1));
    const int pthreads = fthreads + 64;   // covering-panel warps + producer + control
    if (S < 4 || pthreads > 1024 || K % 2 != 0 || fpl > 4)
      ELMFB_THROW(ELMFB_ERR_UNSUPPORTED,
                  "DF32 needs K even, K <= 128, at most 30 covering panels per cell and "
                  "(covering panels per cell) x K <= 1696 (four ring stages of 4 rows)");
    const size_t smem = (size_t)S * stage_bytes + u_bytes;
    prof_begin(h, KID_FUSED, (double)h->NPR * K * 8.0 + 16.0 * h->NR + 8.0 * h->NPhi);
#define ELMFB_FD(F)                                                                             \
  if (fpl == F) {                                                                               \
    ensure_dyn_smem((const void*)k_fused_pipe_df<F>, smem);                                     \
    k_fused_pipe_df<F><<<fp.n_units, pthreads, smem, st>>>(                                     \
        h->d_panels.as<float2>(), (const float2*)tlow, K, fp.units.as<int4>(),                  \
        h->d_cell_pstart.as<int>(), h->d_cell_count.as<int>(), h->d_cover_off.as<int>(),        \
        h->d_cover_sub.as<int>(), h->d_cover_start.as<int>(), h->d_entry_base.as<int64_t>(),    \
        scal, h->d_u.as<double>(), h->d_h.as<double>(), mode, fp.part.as<double>(), gpart, S,   \
        mmax, h->d_flags.as<int>());                                                            \
  }
    ELMFB_FD(1) ELMFB_FD(2) ELMFB_FD(3) ELMFB_FD(4)
#undef ELMFB_FD
    prof_end(h, KID_FUSED);
    count_launch(h);
    return;
  } else {
  const T* P = (const T*)h->d_panels.p;
  const float* tf = (const float*)tlow;
  // the pass reads t in the panels' precision
  const T* t = reinterpret_cast<const T*>(t64);
  if (sizeof(T) == 4) {
    if (!tf) {
      k_to_float<<<(unsigned)std::min<int64_t>(ceil_div(h->NPhi, 256), 1216), 256, 0, st>>>(
          t64, fp.tf.as<float>(), h->NPhi);
      count_launch(h);
      tf = fp.tf.as<float>();
    }
    t = reinterpret_cast<const T*>(tf);
  }
  prof_begin(h, KID_FUSED, (double)h->NPR * K * sizeof(T) + 16.0 * h->NR + 8.0 * h->NPhi);
  const int mmax = std::max(1, h->max_cover);
  int rows = 8, S = 0, pthreads = 0;
  size_t smem = 0;
  if (fused_pipe_shape<T>(h, fp, rows, S, smem, pthreads)) {
#define ELMFB_FTR(F, R)                                                                        \
  if (fpl == F && rows == R) {                                                                 \
    ensure_dyn_smem((const void*)k_fused_pipe<T, F, R>, smem, true);                          \
    k_fused_pipe<T, F, R><<<fp.n_units, pthreads, smem, st>>>(                                 \
        P, t, K, fp.units.as<int4>(), h->d_cell_pstart.as<int>(), h->d_cell_count.as<int>(),   \
        h->d_cover_off.as<int>(), h->d_cover_sub.as<int>(), h->d_cover_start.as<int>(),        \
        h->d_entry_base.as<int64_t>(), scal, h->d_u.as<double>(), h->d_h.as<double>(), mode,    \
        fp.part.as<double>(), gpart, S, mmax, h->d_flags.as<int>(), nullptr, nullptr);          \
  } else
#define ELMFB_FT(F) ELMFB_FTR(F, 4) ELMFB_FTR(F, 8)
    ELMFB_FT(1) ELMFB_FT(2) ELMFB_FT(3) ELMFB_FT(4)
    ELMFB_THROW(ELMFB_ERR_UNSUPPORTED, "fused path needs K <= 128");
#undef ELMFB_FT
#undef ELMFB_FTR
  } else {
#define ELMFB_FU(F, MT)                                                                      \
  if (fpl == F && fthreads <= MT) {                                                          \
    k_fused<T, F, MT><<<fp.n_units, fthreads, 0, st>>>(                                      \
        P, t, K, fp.units.as<int4>(), h->d_cell_pstart.as<int>(), h->d_cell_count.as<int>(), \
        h->d_cover_off.as<int>(), h->d_cover_sub.as<int>(), h->d_cover_start.as<int>(),      \
        h->d_entry_base.as<int64_t>(), scal, h->d_u.as<double>(), h->d_h.as<double>(), mode,  \
        fp.part.as<double>(), gpart);                                                        \
  } else
#define ELMFB_FU4(F) ELMFB_FU(F, 256) ELMFB_FU(F, 512) ELMFB_FU(F, 640) ELMFB_FU(F, 1024)
  ELMFB_FU4(1) ELMFB_FU4(2) ELMFB_FU4(3) ELMFB_FU4(4)
  ELMFB_THROW(ELMFB_ERR_UNSUPPORTED, "fused path needs K <= 128 and <= 32 covering panels");
#undef ELMFB_FU4
#undef ELMFB_FU
  }
  prof_end(h, KID_FUSED);
  count_launch(h);
  }
}

// rows per diagonal-Gram chunk: fewer, larger chunks keep the triangular
// partials (K(K+1)/2 doubles per chunk) small next to the panel reads
constexpr int kDiagChunk = 2048;

template <class T>
void block_jacobi_setup(elmfb_ctx* h, double shift, bool identity, double abs_shift,
                        double drop) {
  cudaStream_t st = h->stream;
  const int K = h->K;
  const int64_t KK = (int64_t)K * K;
  h->d_R.alloc(2 * h->n_sub * KK * sizeof(double), st);
  h->bj_retries = 0;
  h->bj_dropped = 0;
  if (identity) return;
  if (K > 128) ELMFB_THROW(ELMFB_ERR_UNSUPPORTED, "block-Jacobi set-up supports K <= 128");
  // chunks of at most 2048 rows of one panel, as 16-row steps (entry, first
  // row) taken cell by cell in the cell-interleaved storage
  const int ne = (int)h->cover_sub.size();
  // entries panel by panel (each panel's in cell order), with the global
  // index of each entry's first step; the steps themselves are written on
  // the device (k_expand_steps), the chunks here from the step counts
  std::vector<int> pent_off(h->n_sub + 1, 0), pent(ne);
  for (int e = 0; e < ne; ++e) pent_off[h->cover_sub[e] + 1]++;
  for (int s2 = 0; s2 < h->n_sub; ++s2) pent_off[s2 + 1] += pent_off[s2];
  {
    std::vector<int> fill(pent_off.begin(), pent_off.end() - 1);
    for (int e = 0; e < ne; ++e) pent[fill[h->cover_sub[e]]++] = e;
  }
  std::vector<int64_t> step_off(ne + 1, 0);
  for (int q = 0; q < ne; ++q) {
    const int c = h->entry_cell[pent[q]];
    step_off[q + 1] = step_off[q] + ceil_div(h->cell_pstart[c + 1] - h->cell_pstart[c], 16);
  }
  if (step_off[ne] >= ((int64_t)1 << 31))
    ELMFB_THROW(ELMFB_ERR_UNSUPPORTED, "block-Jacobi set-up: more than 2^31 row steps");
  std::vector<int4> chunks;
  std::vector<int> chunk_off(h->n_sub + 1, 0);
  constexpr int kStepsPerChunk = kDiagChunk / 16;
  for (int s2 = 0; s2 < h->n_sub; ++s2) {
    chunk_off[s2] = (int)chunks.size();
    const int64_t f0 = step_off[pent_off[s2]], f1 = step_off[pent_off[s2 + 1]];
    for (int64_t f = f0; f < f1; f += kStepsPerChunk)
      chunks.push_back(make_int4(s2, (int)f, (int)std::min<int64_t>(kStepsPerChunk, f1 - f), 0));
  }
  chunk_off[h->n_sub] = (int)chunks.size();
  const int KT = K * (K + 1) / 2;
  DevBuf dch, dcoff, dsteps;
  dch.alloc(std::max<size_t>(chunks.size(), 1) * sizeof(int4), st);
  dcoff.alloc(chunk_off.size() * sizeof(int), st);
  CUDA_CHECK(cudaMemcpyAsync(dch.p, chunks.data(), chunks.size() * sizeof(int4),
                             cudaMemcpyHostToDevice, st));
  expand_entry_steps(h, pent, step_off, 16, dsteps);
  CUDA_CHECK(cudaMemcpyAsync(dcoff.p, chunk_off.data(), chunk_off.size() * sizeof(int),
                             cudaMemcpyHostToDevice, st));
  h->d_gpart.alloc(std::max<size_t>(chunks.size(), 1) * KT * sizeof(double), st);
  const int Kp4 = (K + 3) & ~3;
  const int ntiles = (Kp4 / 4) * (Kp4 / 4 + 1) / 2;
  const int gthreads = std::max(32, ((ntiles + 31) / 32) * 32);
  const size_t smem = 16 * Kp4 * sizeof(T);
  CUDA_CHECK(cudaMemsetAsync(h->d_flags.p, 0, 16 * sizeof(int), st));
  if (!chunks.empty()) {
    prof_begin(h, KID_GRAM_DIAG,
               (double)h->NPR * K * sizeof(T) + (double)chunks.size() * KT * sizeof(double));
    if constexpr (std::is_same<T, df2>::value) {
      if (K % 4 != 0) ELMFB_THROW(ELMFB_ERR_UNSUPPORTED, "DF32 block-Jacobi set-up needs K % 4 == 0");
      const size_t psmem = (size_t)kDiagStages * 16 * K * sizeof(float2);
      ensure_dyn_smem((const void*)k_gram_diag_pipe_df, psmem);
      k_gram_diag_pipe_df<<<(unsigned)chunks.size(), gthreads, psmem, st>>>(
          h->d_panels.as<float2>(), K, dch.as<int4>(), dsteps.as<int2>(),
          h->d_entry_base.as<int64_t>(), h->d_entry_cell.as<int>(), h->d_cover_off.as<int>(),
          h->d_gpart.as<double>(), h->d_flags.as<int>());
    } else if (K % 4 == 0 && (K * sizeof(T)) % 16 == 0) {
      const size_t psmem = (size_t)kDiagStages * 16 * K * sizeof(T);
      ensure_dyn_smem((const void*)k_gram_diag_pipe<T>, psmem);
      k_gram_diag_pipe<T><<<(unsigned)chunks.size(), gthreads, psmem, st>>>(
          (const T*)h->d_panels.p, K, dch.as<int4>(), dsteps.as<int2>(),
          h->d_entry_base.as<int64_t>(), h->d_entry_cell.as<int>(), h->d_cover_off.as<int>(),
          h->d_gpart.as<double>(), h->d_flags.as<int>());
    } else {
      k_gram_diag_partial<T><<<(unsigned)chunks.size(), gthreads, smem, st>>>(
          (const T*)h->d_panels.p, K, dch.as<int4>(), dsteps.as<int2>(),
          h->d_entry_base.as<int64_t>(), h->d_entry_cell.as<int>(), h->d_cover_off.as<int>(),
          h->d_gpart.as<double>());
    }
    prof_end(h, KID_GRAM_DIAG);
    check_launch("k_gram_diag_partial");
    count_launch(h);
  }
  // the chunk partials summed into one packed triangle per panel, then the
  // factorisation and inverse from a bulk copy of it
  if (h->n_sub > 65535)
    ELMFB_THROW(ELMFB_ERR_UNSUPPORTED, "block-Jacobi set-up: too many subdomains");
  DevBuf dG;
  dG.alloc((size_t)h->n_sub * tri_pairs(K) * sizeof(double), st);
  prof_begin(h, KID_BLOCK_CHOL,
             (double)chunks.size() * KT * sizeof(double) + 2.0 * h->n_sub * KK * sizeof(double));
  k_gram_reduce<<<dim3((unsigned)ceil_div(KT, 256), (unsigned)h->n_sub), 256, 0, st>>>(
      h->d_gpart.as<double>(), dcoff.as<int>(), K, dG.as<double>());
  count_launch(h);
  const size_t csm = chol_smem_bytes(K);
  ensure_dyn_smem((const void*)k_block_chol<false>, csm);
  ensure_dyn_smem((const void*)k_block_chol<true>, csm);
  // FP32 and DF32 panels apply X_j in float-float arithmetic: keep a pair copy
  const bool pairs_x = !std::is_same<T, double>::value;
  if (pairs_x) h->d_R2.alloc(h->n_sub * tri_pairs(K) * sizeof(float2), st);
  if (pairs_x)
    k_block_chol<true><<<h->n_sub, kCholThreads, csm, st>>>(
        dG.as<double>(), K, shift, abs_shift, drop, h->d_R.as<double>(),
        h->d_R.as<double>() + h->n_sub * KK, h->d_flags.as<int>(), h->d_R2.as<float2>());
  else
    k_block_chol<false><<<h->n_sub, kCholThreads, csm, st>>>(
        dG.as<double>(), K, shift, abs_shift, drop, h->d_R.as<double>(),
        h->d_R.as<double>() + h->n_sub * KK, h->d_flags.as<int>(), nullptr);
  prof_end(h, KID_BLOCK_CHOL);
  check_launch("k_block_chol");
  count_launch(h);
  int flags[6];
  CUDA_CHECK(cudaMemcpyAsync(flags, h->d_flags.p, 6 * sizeof(int), cudaMemcpyDeviceToHost, st));
  stream_sync(h);
  h->bj_retries = flags[4];
  h->bj_dropped = flags[5];
  if (flags[3]) ELMFB_THROW(ELMFB_ERR_TIMEOUT, "block-Jacobi set-up: a copy wait timed out");
  if (flags[1]) ELMFB_THROW(ELMFB_ERR_BREAKDOWN, "block Cholesky failed after shift increases");
}

namespace {

// Number of eigenvalues below lam of the Golub-Kahan tridiagonal of B_k: the
// (2k+1) x (2k+1) symmetric matrix with zero diagonal and off-diagonal
// alpha_1, beta_2, alpha_2, beta_3, ..., alpha_k, beta_{k+1}, whose eigenvalues
// are +-sigma_i(B_k) and 0 (Golub & Kahan 1965).  Sturm sequence of the LDL^T
// factorisation of T - lam I, tiny pivots replaced by -pivmin.
__device__ int gk_sturm_count(const double* __restrict__ gk, int k, double lam, double pivmin) {
  double d = -lam;
  int cnt = d < 0.0;
  for (int i = 0; i < 2 * k; ++i) {
    const int j = i >> 1;
    const double e = (i & 1) ? gk[2 * (j + 1) + 1] : gk[2 * j];   // beta_{j+2} : alpha_{j+1}
    if (fabs(d) < pivmin) d = -pivmin;
    d = -lam - e * e / d;
    cnt += d < 0.0;
  }
  return cnt;
}

// Extreme singular values of B_k by multisection of the Sturm count (one
// block: 256 trial points per round for each extreme, the two searched side
// by side; geometric spacing once the interval is off 0; to 1e-10 relative):
// out[0] = sigma_max (the point where the count reaches 2k+1), out[1] =
// sigma_min (where it reaches k+2).  k = 0: zeros.
__global__ void __launch_bounds__(512) k_bidiag_extremes(const double* __restrict__ gk, int k,
                                                        double* __restrict__ out) {
  // two groups of 256 threads, one per extreme: each round every thread
  // counts at one of 256 points spread geometrically over the group's
  // interval, and the interval shrinks to the pair of points where the count
  // crosses the target
  constexpr int kPts = 256;
  __shared__ double lam_s[2][kPts];
  __shared__ int nb_w[16];
  __shared__ double lo_s[2], hi_s[2];
  __shared__ int done_s[2];
  const int g = threadIdx.x / kPts, i = threadIdx.x % kPts;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (k <= 0) {
    if (threadIdx.x < 2) out[threadIdx.x] = 0.0;
    return;
  }
  double bound = 0.0, emax2 = 0.0, eprev = 0.0;
  for (int q = 0; q < 2 * k; ++q) {
    const int j = q >> 1;
    const double e = fabs((q & 1) ? gk[2 * (j + 1) + 1] : gk[2 * j]);
    bound = fmax(bound, eprev + e);
    eprev = e;
    emax2 = fmax(emax2, e * e);
  }
  bound = fmax(bound, eprev) * (1.0 + 1e-12) + 1e-300;
  const double pivmin = 2.2250738585072014e-308 * fmax(1.0, emax2);
  const int target = g == 0 ? 2 * k + 1 : k + 2;   // sigma_max, sigma_min
  if (threadIdx.x < 2) {
    lo_s[threadIdx.x] = 0.0;
    hi_s[threadIdx.x] = bound;
    done_s[threadIdx.x] = 0;
  }
  __syncthreads();
  for (int round = 0; round < 200 && !(done_s[0] && done_s[1]); ++round) {
    const double lo = lo_s[g], hi = hi_s[g];
    const double f = (double)(i + 1) / (kPts + 1);
    const double lam = lo > 0.0 ? lo * pow(hi / lo, f) : hi * f;
    lam_s[g][i] = lam;
    const bool below = !done_s[g] && gk_sturm_count(gk, k, lam, pivmin) < target;
    const unsigned m = __ballot_sync(0xffffffffu, below);
    if (lane == 0) nb_w[warp] = __popc(m);
    __syncthreads();
    if (i == 0 && !done_s[g]) {
      // points 0..nb-1 lie below the crossing; the new interval is [lam_{nb-1}, lam_nb]
      int nb = 0;
      for (int w = 0; w < kPts / 32; ++w) nb += nb_w[g * (kPts / 32) + w];
      double nlo = lo, nhi = hi;
      if (nb > 0) nlo = lam_s[g][nb - 1];
      if (nb < kPts) nhi = lam_s[g][nb];
      lo_s[g] = nlo;
      hi_s[g] = nhi;
      done_s[g] = !(nhi > nlo * (1.0 + 1e-10));
    }
    __syncthreads();
  }
  if (threadIdx.x < 2) out[threadIdx.x] = 0.5 * (lo_s[threadIdx.x] + hi_s[threadIdx.x]);
}

}  // namespace

void bidiag_extremes(elmfb_ctx* h, const double* gk, int k, double* out2) {
  k_bidiag_extremes<<<1, 512, 0, h->stream>>>(gk, k, out2);
  check_launch("k_bidiag_extremes");
  count_launch(h);
}

namespace {

// ---- autotuner of the fused pass's work-unit size --------------------------
// Shape class: panel precision, K, covering panels per cell, log2 of the
// padded rows.  The first solve of a class with `autotune` times the fused
// pass (mode 1, t = 0, CUDA events on the handle's stream, one warm-up and
// three timed launches each) at the heuristic unit size and at half and twice
// it (half and a quarter where twice would pass the 1024-row cap), keeps the
// fastest for the class for the life of the process, and records the
// candidates and their times (elmfb_tuning_table).  Handles of a batch of
// several workers only look the choices up (tune_lookup_only).
struct TuneKey {
  int prec, K, cover, rows_log2;
  bool operator<(const TuneKey& o) const {
    return std::tie(prec, K, cover, rows_log2) < std::tie(o.prec, o.K, o.cover, o.rows_log2);
  }
};
std::mutex g_tune_mu;
std::map<TuneKey, elmfb_tuning_entry> g_tune;

template <class T>
int autotune_unit_rows(elmfb_ctx* h) {
  int lg = 0;
  while ((int64_t(1) << (lg + 1)) <= h->NR) ++lg;
  const TuneKey key{h->cfg.precision, h->K, h->max_cover, lg};
  {
    std::lock_guard<std::mutex> lock(g_tune_mu);
    auto it = g_tune.find(key);
    if (it != g_tune.end()) return it->second.unit_rows;
  }
  // beside other instances on the GPU a timing measures them too: keep the
  // heuristic for classes not tuned before
  if (h->tune_lookup_only) return 0;
  cudaStream_t st = h->stream;
  // half the heuristic, the heuristic, twice it; at the cap a quarter instead of twice
  const int64_t t0 = fused_unit_target(h);
  const int64_t t_hi = 2 * t0 <= kMaxUnitRows ? 2 * t0 : t0;
  const int64_t t_lo = 2 * t0 <= kMaxUnitRows ? t0 / 2 : t0 / 4;
  int cand[3] = {(int)std::max<int64_t>(8, t_lo & ~7), (int)std::max<int64_t>(8, (t0 / 2) & ~7),
                 (int)t_hi};
  if (2 * t0 <= kMaxUnitRows) cand[1] = (int)t0;
  std::sort(cand, cand + 3);
  DevBuf zero, sc, gp;
  zero.alloc(std::max<int64_t>(h->NPhi, 1) * sizeof(double), st);
  sc.alloc(2 * kScal * sizeof(double), st);
  CUDA_CHECK(cudaMemsetAsync(zero.p, 0, h->NPhi * sizeof(double), st));
  CUDA_CHECK(cudaMemsetAsync(sc.p, 0, 2 * kScal * sizeof(double), st));
  h->d_u.alloc(h->NR * sizeof(double), st);
  cudaEvent_t a, b;
  CUDA_CHECK(cudaEventCreate(&a));
  CUDA_CHECK(cudaEventCreate(&b));
  elmfb_tuning_entry e{};
  e.precision = key.prec;
  e.features = key.K;
  e.covering_panels = key.cover;
  e.rows_log2 = key.rows_log2;
  double best = 1e300;
  try {
    for (int c = 0; c < 3; ++c) {
      e.candidates[c] = cand[c];
      if (c > 0 && cand[c] == cand[c - 1]) {
        e.ms[c] = e.ms[c - 1];
        continue;
      }
      FusedPlan fp;
      if (!build_fused_plan(h, fp, cand[c])) ELMFB_THROW(ELMFB_ERR_UNSUPPORTED, "no fused plan");
      gp.alloc((size_t)(std::max(kGatherBlocks, fp.n_units) + h->n_sub + 8) * sizeof(double), st);
      launch_fused<T>(h, fp, zero.as<double>(), 1, sc.as<double>(), gp.as<double>());
      CUDA_CHECK(cudaEventRecord(a, st));
      for (int r = 0; r < 3; ++r)
        launch_fused<T>(h, fp, zero.as<double>(), 1, sc.as<double>(), gp.as<double>());
      CUDA_CHECK(cudaEventRecord(b, st));
      CUDA_CHECK(cudaEventSynchronize(b));
      float ms = 0.f;
      CUDA_CHECK(cudaEventElapsedTime(&ms, a, b));
      e.ms[c] = ms / 3.0;
      if (e.ms[c] < best) {
        best = e.ms[c];
        e.unit_rows = cand[c];
      }
    }
  } catch (...) {
    cudaEventDestroy(a);
    cudaEventDestroy(b);
    throw;
  }
  cudaEventDestroy(a);
  cudaEventDestroy(b);
  check_launch("autotune");
  std::lock_guard<std::mutex> lock(g_tune_mu);
  g_tune.emplace(key, e);
  return g_tune.at(key).unit_rows;
}

template <class T>
void lsqr(elmfb_ctx* h, const elmfb_solve_opts* o, elmfb_solve_info* info) {
  cudaStream_t st = h->stream;
  const int K = h->K;
  const int64_t N = h->NPhi;
  const int64_t KK = (int64_t)K * K;
  const bool identity = o->preconditioner == ELMFB_PREC_NONE;

  stage_begin(h, 4);
  if (!h->bj_reuse) block_jacobi_setup<T>(h, o->shift, identity, 0.0, o->drop_tol);
  stage_end(h, 4);
  info->setup_ms = h->stage_ms[4];
  info->precond_retries = h->bj_retries;
  info->precond_dropped = h->bj_dropped;

  // panel -> entries (cell order)
  const int ne = (int)h->cover_sub.size();
  std::vector<int> pent_off(h->n_sub + 1, 0), pent(ne);
  for (int e = 0; e < ne; ++e) pent_off[h->cover_sub[e] + 1]++;
  for (int s = 0; s < h->n_sub; ++s) pent_off[s + 1] += pent_off[s];
  {
    std::vector<int> fill(pent_off.begin(), pent_off.end() - 1);
    for (int e = 0; e < ne; ++e) pent[fill[h->cover_sub[e]]++] = e;
  }
  DevBuf dpo, dpe;
  dpo.alloc(pent_off.size() * sizeof(int), st);
  dpe.alloc(std::max(ne, 1) * sizeof(int), st);
  CUDA_CHECK(cudaMemcpyAsync(dpo.p, pent_off.data(), pent_off.size() * sizeof(int),
                             cudaMemcpyHostToDevice, st));
  CUDA_CHECK(cudaMemcpyAsync(dpe.p, pent.data(), ne * sizeof(int), cudaMemcpyHostToDevice, st));

  h->d_u.alloc(h->NR * sizeof(double), st);
  h->d_v.alloc(N * sizeof(double), st);
  h->d_w.alloc(N * sizeof(double), st);
  h->d_x_sol.alloc(N * sizeof(double), st);
  h->d_tmp.alloc(std::max<int64_t>(N, h->NR) * sizeof(double), st);
  h->d_partial.alloc((int64_t)ne * K * sizeof(double), st);
  // scalar slots, then the Golub-Kahan record (alpha, beta) of steps 0..max_iter
  const int gk_cap = o->max_iter + 1;
  h->d_scal.alloc((2 * kScal + 2 * (size_t)gk_cap) * sizeof(double), st);
  h->d_ptile.alloc((kGatherBlocks + h->n_sub + 8) * sizeof(double), st);
  double* gpart = h->d_ptile.as<double>();
  double* vpart = gpart + kGatherBlocks;
  const double panel_bytes = (double)h->NPR * K * sizeof(T);
  CUDA_CHECK(cudaMemsetAsync(h->d_scal.p, 0, 2 * kScal * sizeof(double), st));
  {
    const double cap_d = (double)gk_cap;   // pageable: staged before the call returns
    CUDA_CHECK(cudaMemcpyAsync(h->d_scal.as<double>() + S_GKCAP, &cap_d, sizeof(double),
                               cudaMemcpyHostToDevice, st));
    CUDA_CHECK(cudaMemcpyAsync(h->d_scal.as<double>() + kStage + S_GKCAP, &cap_d, sizeof(double),
                               cudaMemcpyHostToDevice, st));
  }

  const T* P = (const T*)h->d_panels.p;
  double* scal = h->d_scal.as<double>();
  const double* Xr = h->d_R.as<double>();
  const double* Xc = h->d_R.as<double>() + h->n_sub * KK;
  int pblock = std::min(std::max(32, ((K + 31) / 32) * 32), 256);
  const int upd_blocks = (int)std::min<int64_t>(ceil_div(N, 256), 1216);
  // k_precond: G groups of Kp threads split each X_j^T v_j sum
  const int pc_Kp = (K + 31) & ~31;
  const int pc_G = std::max(1, std::min(8, std::min(1024 / pc_Kp, K / 8)));
  const int pc_threads = pc_G * pc_Kp;
  const size_t pc_smem = (size_t)(K + pc_G * K) * sizeof(double);

  auto gather = [&](const double* t, int mode) {
    if constexpr (std::is_same<T, df2>::value) {
      ELMFB_THROW(ELMFB_ERR_UNSUPPORTED, "DF32 runs the fused pass only");
    } else {
      prof_begin(h, KID_GATHER, panel_bytes + 16.0 * h->NR + 8.0 * N);
      k_gather<T><<<kGatherBlocks, kGatherThreads, 0, st>>>(
          P, t, K, h->NR, h->d_grow_cell.as<int>(), h->d_cell_pstart.as<int>(),
          h->d_cell_count.as<int>(), h->d_cover_off.as<int>(), h->d_cover_sub.as<int>(),
          h->d_cover_start.as<int>(), h->d_entry_base.as<int64_t>(), scal, h->d_u.as<double>(),
          h->d_h.as<double>(), mode, gpart);
      prof_end(h, KID_GATHER);
    }
  };
  auto transpose_step = [&](int init) {
    if constexpr (!std::is_same<T, df2>::value) {
      prof_begin(h, KID_ENTRY_T, panel_bytes + 8.0 * h->NR + 8.0 * ne * K);
      k_entry_T<T><<<ne, 128, 0, st>>>(P, h->d_u.as<double>(), K, h->d_entry_cell.as<int>(),
                                          h->d_cover_sub.as<int>(), h->d_cover_off.as<int>(),
                                          h->d_cell_pstart.as<int>(), h->d_cell_count.as<int>(),
                                          h->d_entry_base.as<int64_t>(), h->d_partial.as<double>());
      prof_end(h, KID_ENTRY_T);
    }
    prof_begin(h, KID_PANEL_T, 8.0 * ne * K + (identity ? 0.0 : 8.0 * h->n_sub * KK) + 16.0 * N);
    k_panel_T<<<h->n_sub, pblock, K * sizeof(double), st>>>(
        h->d_partial.as<double>(), dpo.as<int>(), dpe.as<int>(), Xc, K, gpart, kGatherBlocks,
        h->d_v.as<double>(), scal, identity ? 1 : 0, init, vpart);
    prof_end(h, KID_PANEL_T);
    prof_begin(h, KID_UPDATE, 48.0 * N);
    k_update<<<upd_blocks, 256, 0, st>>>(scal, vpart, h->n_sub, h->d_v.as<double>(),
                                         h->d_w.as<double>(), h->d_x_sol.as<double>(), N, init);
    prof_end(h, KID_UPDATE);
  };

  // fused single-pass iteration (M t and M^T u' in one read of the panels)
  FusedPlan fp;
  const int tuned_rows = o->autotune && h->max_cover <= 32 && K <= 128
                             ? autotune_unit_rows<T>(h) : 0;
  const bool fused = build_fused_plan(h, fp, tuned_rows);
  DevBuf& dfpart = fp.part;
  const int n_units = fp.n_units;
  if (fused) {
    h->d_ptile.alloc((std::max(kGatherBlocks, n_units) + h->n_sub + 8) * sizeof(double), st);
    gpart = h->d_ptile.as<double>();
    vpart = gpart + std::max(kGatherBlocks, n_units);
  }
  const int KpT = (K + 31) & ~31;
  const int tgroups = std::max(1, 1024 / KpT);
  const size_t p2smem = (size_t)(tgroups + 1) * K * sizeof(double);
  auto fused_step = [&](const double* t, int mode, const void* tf = nullptr) {
    launch_fused<T>(h, fp, t, mode, scal, gpart, tf);
  };
  // FP32 and DF32 panels apply X_j as FP32 pairs (block_jacobi_setup keeps a
  // pair copy), or no X at all without a preconditioner (the tail's identity
  // form); the fused path's partials are then pairs too
  const bool xpairs = !std::is_same<T, double>::value && fused && fp.pairs;
  const float2* Xt = xpairs && !identity ? h->d_R2.as<float2>() : nullptr;
  const size_t tsmem = tri_smem_bytes(K, identity);
  const int tthreads = tri_threads(K, identity);
  const double tri_bytes = identity ? 0.0 : 8.0 * h->n_sub * ((double)K * (K + 1) / 2);
  // k_precond also writes the fused pass's low-precision copy of t
  const int low_kind = !fused ? 0 : (std::is_same<T, df2>::value ? 2 : (fp.pairs ? 1 : 0));
  // FP32 / DF32 panels: the whole tail in k_lsqr_tail_tri (the update deferred
  // into the next call, t unnormalised, the fused pass in mode 2); w and x start
  // at zero, the tail's block counter too
  DevBuf dcount;
  if (xpairs) {
    ensure_dyn_smem((const void*)k_lsqr_tail_tri, tsmem);
    dcount.alloc(sizeof(unsigned int), st);
    CUDA_CHECK(cudaMemsetAsync(dcount.p, 0, sizeof(unsigned int), st));
    CUDA_CHECK(cudaMemsetAsync(h->d_w.p, 0, N * sizeof(double), st));
    CUDA_CHECK(cudaMemsetAsync(h->d_x_sol.p, 0, N * sizeof(double), st));
  }
  const int fmode = xpairs ? 2 : 0;              // the loop's fused-pass mode
  if (xpairs) {   // the stopping tests run on the device too (lsqr_recurrence)
    const double sp[4] = {1.0, o->ntol, o->btol, o->atol};   // S_STOP_ON .. S_ATOL
    CUDA_CHECK(cudaMemcpyAsync(scal + S_STOP_ON, sp, sizeof(sp), cudaMemcpyHostToDevice, st));
    CUDA_CHECK(cudaMemcpyAsync(scal + kStage + S_STOP_ON, sp, sizeof(sp), cudaMemcpyHostToDevice,
                               st));
  }
  const int tail_launches = xpairs ? 1 : 2;      // besides the slice sums (counted by themselves)
  auto fused_tail = [&](int init) {
    if (xpairs) {
      // panel_MTu: the slice sums; lsqr_update: the rest (slice sums, X's
      // triangle, v, w, x, t read or written once)
      const double csum_bytes = 8.0 * fp.n_pchunks * K;
      prof_begin(h, KID_PANEL_T, (double)dfpart.bytes + csum_bytes);
      panel_chunk_sums(h, fp, gpart, n_units, scal);
      prof_end(h, KID_PANEL_T);
      prof_begin(h, KID_UPDATE, csum_bytes + tri_bytes + 72.0 * N);
      k_lsqr_tail_tri<<<h->n_sub, tthreads, tsmem, st>>>(
          fp.csum.as<double>(), fp.pco.as<int>(), Xt, K, h->d_v.as<double>(),
          h->d_w.as<double>(), h->d_x_sol.as<double>(), scal, init, vpart,
          h->d_tmp.as<double>(), fp.tf.p, low_kind, dcount.as<unsigned int>(),
          h->d_flags.as<int>(), nullptr, nullptr);
      prof_end(h, KID_UPDATE);
      return;
    }
    // algorithmic bytes: the partials, X's triangle (8 bytes a value), v read and written
    prof_begin(h, KID_PANEL_T, (double)dfpart.bytes + (identity ? 0.0 : tri_bytes) + 16.0 * N);
    panel_chunk_sums(h, fp, gpart, n_units, scal);
    k_panel_T2<<<h->n_sub, tgroups * KpT, p2smem, st>>>(
        fp.csum.as<double>(), fp.pco.as<int>(), Xc, K, h->d_v.as<double>(), scal,
        identity ? 1 : 0, init, vpart, fp.pairs ? 1 : 0);
    prof_end(h, KID_PANEL_T);
    prof_begin(h, KID_UPDATE, 48.0 * N + (identity ? 0.0 : tri_bytes));
    k_update_precond<<<h->n_sub, pc_threads, pc_smem, st>>>(
        scal, vpart, h->n_sub, h->d_v.as<double>(), h->d_w.as<double>(),
        h->d_x_sol.as<double>(), K, init, identity ? 1 : 0, Xr, h->d_tmp.as<double>(), fp.tf.p,
        low_kind);
    prof_end(h, KID_UPDATE);
  };
  if (fused && p2smem > 48 * 1024)
    ensure_dyn_smem((const void*)k_panel_T2, p2smem);

  stage_begin(h, 5);
  // start: b = h (cold) or h - M a0 (warm start)
  if (fused) {
    if (o->warm_start) {
      fused_step(h->d_a.as<double>(), 1);
    } else {
      CUDA_CHECK(cudaMemsetAsync(h->d_tmp.p, 0, N * sizeof(double), st));
      fused_step(h->d_tmp.as<double>(), 1);
    }
    fused_tail(1);
    count_launch(h, tail_launches);
  } else {
    if (o->warm_start) {
      gather(h->d_a.as<double>(), 1);
    } else {
      // u' = h: gather with t = 0 in mode 1 gives h - 0
      CUDA_CHECK(cudaMemsetAsync(h->d_tmp.p, 0, N * sizeof(double), st));
      gather(h->d_tmp.as<double>(), 1);
    }
    transpose_step(1);
    count_launch(h, 4);
  }
  check_launch("lsqr init");
  // ||(M P)^T h|| = alpha_1 beta_1, the start of the normal-residual estimate
  double arnorm0 = 0.0;
  if (o->ntol > 0.0) {
    double s0[kStage];
    CUDA_CHECK(cudaMemcpyAsync(s0, scal + kStage, kStage * sizeof(double), cudaMemcpyDeviceToHost,
                               st));
    stream_sync(h);
    arnorm0 = s0[S_ARNORM];
  }

  int it = 0;
  int status = ELMFB_ERR_NOT_CONVERGED;
  double sc[kScal];
  const int max_it = o->max_iter;
  // Graph mode: the kernels of one check interval (all device-resident, no
  // host values between them) are captured once as a CUDA graph and replayed,
  // one launch per interval.  Needs a stream other than the legacy default
  // stream and profiling off.
  const bool use_graph = o->graph && fused && st != nullptr && !h->prof;
  struct GraphExec {
    cudaGraphExec_t e = nullptr;
    ~GraphExec() {
      if (e) cudaGraphExecDestroy(e);
    }
  } gx;
  int g_batch = 0;
  int64_t g_launches = 0;
  auto capture_interval = [&](int batch_len) {
    const int64_t l0 = h->launches;
    cudaGraph_t g = nullptr;
    CUDA_CHECK(cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal));
    try {
      for (int b = 0; b < batch_len; ++b) {
        fused_step(h->d_tmp.as<double>(), fmode, low_kind ? fp.tf.p : nullptr);
        fused_tail(0);
      }
    } catch (...) {
      cudaStreamEndCapture(st, &g);
      if (g) cudaGraphDestroy(g);
      throw;
    }
    CUDA_CHECK(cudaStreamEndCapture(st, &g));
    g_launches = h->launches - l0;   // kernels that count themselves, per replay
    h->launches = l0;
    return g;
  };
  // true: converged; rec = the staged scalars and the first four flags as
  // the batch's coordinator gathered them, else read here
  auto check_scalars = [&](const double* rec = nullptr) -> bool {
    int dflags[4];
    if (rec) {
      for (int i = 0; i < kStage; ++i) sc[i] = rec[i];
      for (int i = 0; i < 4; ++i) dflags[i] = (int)rec[kStage + i];
    } else {
      // with blocking waits, sleep until the interval is done: the copies
      // into pageable memory below would otherwise wait for it in a spin
      if (h->blocking_sync) stream_sync(h);
      CUDA_CHECK(cudaMemcpyAsync(sc, scal + kStage, kStage * sizeof(double),
                                 cudaMemcpyDeviceToHost, st));
      CUDA_CHECK(cudaMemcpyAsync(dflags, h->d_flags.p, 4 * sizeof(int), cudaMemcpyDeviceToHost,
                                 st));
      stream_sync(h);
    }
    if (dflags[3])
      ELMFB_THROW(ELMFB_ERR_TIMEOUT,
                  "LSQR iteration: an on-device wait (bulk copy) timed out");
    if (sc[S_BAD] != 0.0) ELMFB_THROW(ELMFB_ERR_NONFINITE, "non-finite LSQR scalar");
    const double anorm = std::sqrt(sc[S_ANORM2]);
    const double rn = sc[S_RNORM], arn = sc[S_ARNORM];
    const bool t1 = o->btol > 0.0 && rn <= o->btol * sc[S_BNORM];
    const bool t2 = o->atol > 0.0 && anorm > 0.0 && rn > 0.0 && arn <= o->atol * anorm * rn;
    const bool t3 = o->ntol > 0.0 && arn <= o->ntol * arnorm0;
    return t1 || t2 || t3 || sc[S_ALPHA] == 0.0 || sc[S_BETA] == 0.0 || sc[S_DONE] != 0.0;
  };
  // Multi-instance launches: full check intervals in the batch's shared
  // rounds, then leave and finish any remainder below.  FP32 panels with the
  // FP32-pair tail and the bulk-copy fused pass only.
  bool in_rounds = false;
  BatchShape bsh;
  if constexpr (std::is_same<T, float>::value) {
    if (h->round && round_interval(h->round) == o->check_every && xpairs && fused &&
        fp.n_pchunks > 0 && o->check_every <= max_it)
      in_rounds = fused_pipe_shape<T>(h, fp, bsh.rows, bsh.S, bsh.smem, bsh.pthreads);
  }
  if (in_rounds) {
    bsh.K = K;
    bsh.fpl = (K + 31) / 32;
    bsh.mmax = std::max(1, h->max_cover);
    bsh.chunk_threads = std::min(std::max(32, ((K + 31) / 32) * 32), 128);   // as panel_chunk_sums
    bsh.low_kind = low_kind;
    bsh.mode = fmode;
    bsh.tsmem = tsmem;
    bsh.tthreads = tthreads;
    BatchInst bi{};
    bi.panels = reinterpret_cast<const float*>(P);
    bi.tlow = fp.tf.as<float>();
    bi.units = fp.units.as<int4>();
    bi.cell_pstart = h->d_cell_pstart.as<int>();
    bi.cell_count = h->d_cell_count.as<int>();
    bi.cover_off = h->d_cover_off.as<int>();
    bi.cover_sub = h->d_cover_sub.as<int>();
    bi.entry_base = h->d_entry_base.as<int64_t>();
    bi.scal = scal;
    bi.u = h->d_u.as<double>();
    bi.hvec = h->d_h.as<double>();
    bi.part = fp.part.as<double>();
    bi.gpart = gpart;
    bi.flags = h->d_flags.as<int>();
    bi.fe = fp.fe.as<int>();
    bi.pch = fp.pch.as<int2>();
    bi.csum = fp.csum.as<double>();
    bi.pco = fp.pco.as<int>();
    bi.Xt = Xt;
    bi.v = h->d_v.as<double>();
    bi.w = h->d_w.as<double>();
    bi.x = h->d_x_sol.as<double>();
    bi.vpart = vpart;
    bi.t = h->d_tmp.as<double>();
    bi.counter = dcount.as<unsigned int>();
    bi.n_units = n_units;
    bi.n_pchunks = fp.n_pchunks;
    bi.n_sub = h->n_sub;
    // the rounds run on the batch's own streams: the start-up work on st first
    stream_sync(h);
    struct Leave {   // leave the rounds on every exit, errors included
      elmfb_ctx* h;
      bool joined = false;
      ~Leave() {
        if (joined) round_leave(h->round, h->round_slot);
      }
    } lv{h};
    round_join(h->round, h->round_slot, bi, bsh);
    lv.joined = true;
    double rec[kRoundRecord];
    while (it + o->check_every <= max_it) {
      h->launches += round_step(h->round, h->round_slot, rec);
      it += o->check_every;
      if (check_scalars(rec)) {
        status = ELMFB_OK;
        break;
      }
    }
  }
  while (it < max_it && status != ELMFB_OK) {
    int batch = std::min(o->check_every, max_it - it);
    if (use_graph && !in_rounds) {
      if (!gx.e || batch != g_batch) {
        if (gx.e) CUDA_CHECK(cudaGraphExecDestroy(gx.e));
        gx.e = nullptr;
        cudaGraph_t g = capture_interval(batch);
        const cudaError_t ie = cudaGraphInstantiate(&gx.e, g, 0);
        cudaGraphDestroy(g);
        CUDA_CHECK(ie);
        g_batch = batch;
      }
      CUDA_CHECK(cudaGraphLaunch(gx.e, st));
      h->launches += g_launches;
    }
    const bool graphed = use_graph && !in_rounds;
    for (int b = 0; b < batch && !graphed; ++b) {
      if (fused) {
        // t (and its low-precision copy) come from the previous iteration's tail
        fused_step(h->d_tmp.as<double>(), fmode, low_kind ? fp.tf.p : nullptr);
        fused_tail(0);
      } else {
        prof_begin(h, KID_PRECOND, (identity ? 0.0 : 8.0 * h->n_sub * KK) + 16.0 * N);
        k_precond<<<h->n_sub, pc_threads, pc_smem, st>>>(
            Xr, h->d_v.as<double>(), K, h->d_tmp.as<double>(), identity, scal, nullptr, 0);
        prof_end(h, KID_PRECOND);
        gather(h->d_tmp.as<double>(), 0);
        transpose_step(0);
      }
    }
    // fused: the tail kernels (the fused pass and the slice sums count
    // themselves); else k_precond, k_gather, k_entry_T, k_panel_T, k_update
    count_launch(h, (fused ? tail_launches : 5) * batch);
    it += batch;
    check_launch("lsqr iteration");
    if (check_scalars()) {
      status = ELMFB_OK;
      break;
    }
  }
  // a = (a0 +) P y, after the last deferred update of y (x here)
  if (xpairs) {
    k_lsqr_finish<<<upd_blocks, 256, 0, st>>>(scal, h->d_w.as<double>(), h->d_x_sol.as<double>(),
                                               N);
    count_launch(h);
  }
  if (xpairs)
    k_precond_df<<<h->n_sub, pc_threads, pc_smem, st>>>(Xt, h->d_x_sol.as<double>(), K,
                                                         h->d_tmp.as<double>(), identity, scal,
                                                         nullptr, 0);
  else
    k_precond<<<h->n_sub, pc_threads, pc_smem, st>>>(Xr, h->d_x_sol.as<double>(), K,
                                                      h->d_tmp.as<double>(), identity, scal,
                                                      nullptr, 0);
  if (o->warm_start)
    k_add_to<<<upd_blocks, 256, 0, st>>>(h->d_a.as<double>(), h->d_tmp.as<double>(), N);
  else
    CUDA_CHECK(cudaMemcpyAsync(h->d_a.p, h->d_tmp.p, N * sizeof(double), cudaMemcpyDeviceToDevice,
                               st));
  count_launch(h, 2);
  check_launch("lsqr finish");
  CUDA_CHECK(cudaMemcpyAsync(sc, scal, kStage * sizeof(double), cudaMemcpyDeviceToHost, st));
  stage_end(h, 5);
  // with the tests on the device the iterations stop where a test was met;
  // the launches after it returned at once and are no part of the kernels'
  // timings
  if (xpairs) {
    const int ran = (int)sc[S_ITER];
    if (ran < it && h->prof)
      for (int kid : {(int)KID_FUSED, (int)KID_PANEL_T, (int)KID_UPDATE})
        prof_drop_from(h, kid, h->prof_seen[kid] - (it - ran));
    it = ran;
  }
  // the Golub-Kahan record and its extreme singular values (B_k, k = it)
  const int gk_k = std::min(it, gk_cap - 1);
  h->gk_alpha.assign(gk_k + 1, 0.0);
  h->gk_beta.assign(gk_k + 1, 0.0);
  {
    std::vector<double> rec(2 * (size_t)(gk_k + 1));
    DevBuf dsv;
    dsv.alloc(2 * sizeof(double), st);
    bidiag_extremes(h, scal + 2 * kScal, gk_k, dsv.as<double>());
    double sv[2];
    CUDA_CHECK(cudaMemcpyAsync(rec.data(), scal + 2 * kScal, rec.size() * sizeof(double),
                               cudaMemcpyDeviceToHost, st));
    CUDA_CHECK(cudaMemcpyAsync(sv, dsv.p, sizeof(sv), cudaMemcpyDeviceToHost, st));
    stream_sync(h);
    for (int i = 0; i <= gk_k; ++i) {
      h->gk_alpha[i] = rec[2 * i];
      h->gk_beta[i] = rec[2 * i + 1];
    }
    info->sigma_max = sv[0];
    info->sigma_min = sv[1];
  }
  info->status = status;
  info->iterations = it;
  info->residual_norm = sc[S_RNORM];
  info->normal_residual_norm = sc[S_ARNORM];
  info->solve_ms = h->stage_ms[5];
}


// ------------------------------------------------------------------ PCG -----
// Normal equations (G + mu I) a = g with G the tensor-core Gram (BF16 products,
// FP32 blocks), block-Jacobi preconditioned; outer refinement steps recompute
// g = M^T (h - M a) exactly from the panels with the fused pass.

// per pair: y_i part = G_ij x_j, y_j part = G_ij^T x_i (FP32 products summed in
// FP32 per row, stored FP64); one block per pair
__global__ void __launch_bounds__(128) k_gspmv_pairs(const float* __restrict__ G,
                                                     const int2* __restrict__ pij, int K,
                                                     const double* __restrict__ x,
                                                     double* __restrict__ part) {
  __shared__ float xi[128], xj[128];
  const int p = blockIdx.x;
  const int2 ij = pij[p];
  for (int k = threadIdx.x; k < K; k += blockDim.x) {
    xi[k] = (float)x[(int64_t)ij.x * K + k];
    xj[k] = (float)x[(int64_t)ij.y * K + k];
  }
  __syncthreads();
  const float* B = G + (int64_t)p * K * K;
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
  double* yi = part + (int64_t)p * 2 * K;
  double* yj = yi + K;
  // rows: warp per row, lanes along the row (coalesced)
  for (int m = w; m < K; m += nw) {
    float acc = 0.f;
    for (int n = lane; n < K; n += 32) acc += B[(int64_t)m * K + n] * xj[n];
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if (lane == 0) yi[m] = (double)acc;
  }
  if (ij.x != ij.y) {
    // columns: thread per column, loop over rows (coalesced across threads)
    for (int n = threadIdx.x; n < K; n += blockDim.x) {
      float acc = 0.f;
      for (int m = 0; m < K; ++m) acc += B[(int64_t)m * K + n] * xi[m];
      yj[n] = (double)acc;
    }
  }
}

// y_s = sum of its incident pair parts (fixed order) + mu x_s; partial x.y per block
__global__ void k_gspmv_reduce(const double* __restrict__ part, const int* __restrict__ inc_off,
                               const int* __restrict__ inc, int K, const double* __restrict__ x,
                               double mu, double* __restrict__ y, double* __restrict__ dot_part) {
  __shared__ double red[33];
  const int s = blockIdx.x;
  double d = 0.0;
  for (int k = threadIdx.x; k < K; k += blockDim.x) {
    double acc = 0.0;
    for (int q = inc_off[s]; q < inc_off[s + 1]; ++q) acc += part[(int64_t)inc[q] * K + k];
    const double xv = x[(int64_t)s * K + k];
    acc += mu * xv;
    y[(int64_t)s * K + k] = acc;
    d += xv * acc;
  }
  const double tot = block_sum(d, red);
  if (threadIdx.x == 0) dot_part[s] = tot;
}

// z_s = X_s^T X_s r_s (= (G_ss + eps tr/K I)^{-1} r_s); partial r.z per block
__global__ void k_bj_apply(const double* __restrict__ Xr, const double* __restrict__ Xc, int K,
                           const double* __restrict__ r, double* __restrict__ z,
                           double* __restrict__ dot_part) {
  extern __shared__ double sh[];   // r[K], w[K]
  __shared__ double red[33];
  const int s = blockIdx.x;
  double* rs = sh;
  double* ws = sh + K;
  for (int i = threadIdx.x; i < K; i += blockDim.x) rs[i] = r[(int64_t)s * K + i];
  __syncthreads();
  const double* XC = Xc + (int64_t)s * K * K;   // XC[m*K + i] = X_im
  const double* XR = Xr + (int64_t)s * K * K;   // XR[m*K + i] = X_mi
  for (int i = threadIdx.x; i < K; i += blockDim.x) {
    double acc = 0.0;
    for (int m = 0; m <= i; ++m) acc += XC[m * K + i] * rs[m];
    ws[i] = acc;
  }
  __syncthreads();
  double d = 0.0;
  for (int i = threadIdx.x; i < K; i += blockDim.x) {
    double acc = 0.0;
    for (int m = i; m < K; ++m) acc += XR[m * K + i] * ws[m];
    z[(int64_t)s * K + i] = acc;
    d += acc * rs[i];
  }
  const double tot = block_sum(d, red);
  if (threadIdx.x == 0) dot_part[s] = tot;
}

// g_s = sum of the fused pass partials of panel s (M^T u' unscaled)
__global__ void k_panel_sum(const double* __restrict__ csum, const int* __restrict__ pco, int K,
                            double* __restrict__ g, int pairs) {
  const int s = blockIdx.x;
  for (int k = threadIdx.x; k < K; k += blockDim.x) {
    double acc = 0.0;
    if (pairs) {
      float hi = 0.f, lo = 0.f;
      for (int q = pco[s]; q < pco[s + 1]; ++q) {
        const float2 pr = partial_pair(csum, (int64_t)q * K + k);
        ff_add(hi, lo, pr.x, pr.y);
      }
      acc = (double)hi + (double)lo;
    } else {
      for (int q = pco[s]; q < pco[s + 1]; ++q) acc += csum[(int64_t)q * K + k];
    }
    g[(int64_t)s * K + k] = acc;
  }
}


// alpha = rz / p.q;  x += alpha p;  r -= alpha q   (rz in sc[slot])
__global__ void k_pcg_axpy(const double* __restrict__ sc, int slot,
                           const double* __restrict__ pq_part, int npart,
                           const double* __restrict__ p, const double* __restrict__ q,
                           double* __restrict__ x, double* __restrict__ r, int64_t N) {
  __shared__ double shs, sha;
  const double pq = block_partial_sum(pq_part, npart, &shs);
  if (threadIdx.x == 0) sha = pq > 0.0 ? sc[slot] / pq : 0.0;   // one FP64 division
  __syncthreads();
  const double alpha = sha;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < N;
       i += (int64_t)gridDim.x * blockDim.x) {
    x[i] += alpha * p[i];
    r[i] -= alpha * q[i];
  }
}

// beta = rz_new / rz;  p = z + beta p;  sc[slot ^ 1] = rz_new  (init: p = z)
__global__ void k_pcg_pupdate(double* __restrict__ sc, int slot, const double* __restrict__ rz_part,
                              int npart, const double* __restrict__ z, double* __restrict__ p,
                              int64_t N, int init) {
  __shared__ double shs, shb;
  const double rzn = block_partial_sum(rz_part, npart, &shs);
  if (threadIdx.x == 0) {   // one FP64 division
    const double rz = sc[slot];
    shb = (!init && rz > 0.0) ? rzn / rz : 0.0;
  }
  __syncthreads();
  const double beta = shb;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < N;
       i += (int64_t)gridDim.x * blockDim.x)
    p[i] = z[i] + beta * p[i];
  if (blockIdx.x == 0 && threadIdx.x == 0) sc[init ? slot : (slot ^ 1)] = rzn;
}

template <class T>
void pcg_solve(elmfb_ctx* h, const elmfb_solve_opts* o, elmfb_solve_info* info) {
  if (h->cfg.precision != ELMFB_MIXED)
    ELMFB_THROW(ELMFB_ERR_UNSUPPORTED, "PCG on the tensor-core Gram needs ELMFB_MIXED precision");
  cudaStream_t st = h->stream;
  const int K = h->K;
  const int64_t N = h->NPhi;
  const int64_t KK = (int64_t)K * K;
  if (!h->have_gram) gram_compute(h);
  const int64_t np_ = h->n_gram_pairs;
  // mu as a fraction of the mean Gram diagonal (host estimate from the diagonal blocks)
  double mu = 0.0;
  if (o->gram_shift > 0.0) {
    std::vector<float> blk(K * K);
    double tr = 0.0;
    for (int64_t p = 0; p < np_; ++p)
      if (h->gram_pair_ij[p].first == h->gram_pair_ij[p].second) {
        CUDA_CHECK(cudaMemcpy(blk.data(), h->d_gram.as<float>() + p * KK, KK * sizeof(float),
                              cudaMemcpyDeviceToHost));
        for (int k = 0; k < K; ++k) tr += blk[k * K + k];
      }
    mu = o->gram_shift * tr / (double)N;
  }
  stage_begin(h, 4);
  block_jacobi_setup<T>(h, o->shift, false, mu);
  stage_end(h, 4);
  info->setup_ms = h->stage_ms[4] + h->stage_ms[3];
  info->precond_retries = h->bj_retries;
  FusedPlan fp;
  if (!build_fused_plan(h, fp))
    ELMFB_THROW(ELMFB_ERR_UNSUPPORTED, "PCG needs K <= 128 and <= 32 covering panels per cell");
  // per-subdomain incident pair parts, in pair order
  const int64_t np = h->n_gram_pairs;
  std::vector<int2> pij(np);
  std::vector<std::vector<int>> inc(h->n_sub);
  for (int64_t p = 0; p < np; ++p) {
    const auto ij = h->gram_pair_ij[p];
    pij[p] = make_int2(ij.first, ij.second);
    inc[ij.first].push_back((int)(2 * p));
    if (ij.first != ij.second) inc[ij.second].push_back((int)(2 * p + 1));
  }
  std::vector<int> ioff(h->n_sub + 1, 0), ilist;
  for (int s2 = 0; s2 < h->n_sub; ++s2) {
    ioff[s2] = (int)ilist.size();
    ilist.insert(ilist.end(), inc[s2].begin(), inc[s2].end());
  }
  ioff[h->n_sub] = (int)ilist.size();
  // panel -> fused partial rows (for g)
  DevBuf dpij, dioff, dilist, dpart2, dvec, dpartial, dsc;
  auto up = [&](DevBuf& d, const void* src, size_t bytes) {
    d.alloc(std::max<size_t>(bytes, 8), st);
    if (bytes) CUDA_CHECK(cudaMemcpyAsync(d.p, src, bytes, cudaMemcpyHostToDevice, st));
  };
  up(dpij, pij.data(), np * sizeof(int2));
  up(dioff, ioff.data(), ioff.size() * sizeof(int));
  up(dilist, ilist.data(), ilist.size() * sizeof(int));
  dpart2.alloc(std::max<int64_t>(np, 1) * 2 * K * sizeof(double), st);
  dvec.alloc(6 * N * sizeof(double), st);
  double* x = dvec.as<double>();
  double* r = x + N;
  double* z = r + N;
  double* pv = z + N;
  double* q = pv + N;
  double* g = q + N;
  h->d_u.alloc(h->NR * sizeof(double), st);
  h->d_tmp.alloc(std::max<int64_t>(N, h->NR) * sizeof(double), st);
  const int nparts = std::max(fp.n_units, h->n_sub);
  dpartial.alloc((size_t)(nparts + 2 * h->n_sub + 8) * sizeof(double), st);
  double* gpart = dpartial.as<double>();
  double* dot1 = gpart + nparts;
  double* dot2 = dot1 + h->n_sub;
  dsc.alloc(kScal * sizeof(double), st);
  CUDA_CHECK(cudaMemsetAsync(dsc.p, 0, kScal * sizeof(double), st));
  double* sc = dsc.as<double>();
  const double* Xr = h->d_R.as<double>();
  const double* Xc = h->d_R.as<double>() + h->n_sub * KK;
  const int vb = (int)std::min<int64_t>(ceil_div(N, 256), 1216);
  const int pb = std::min(std::max(32, ((K + 31) / 32) * 32), 256);
  const size_t fsz = 16;   // unused scalar slots of the fused kernel (mode 1 reads none)

  stage_begin(h, 5);
  if (!o->warm_start) CUDA_CHECK(cudaMemsetAsync(h->d_a.p, 0, N * sizeof(double), st));
  int its = 0;
  for (int ref = 0; ref < o->refine; ++ref) {
    // g = M^T (h - M a), exact from the panels
    launch_fused<T>(h, fp, h->d_a.as<double>(), 1, sc + fsz, gpart);
    panel_chunk_sums(h, fp);
    k_panel_sum<<<h->n_sub, pb, 0, st>>>(fp.csum.as<double>(), fp.pco.as<int>(), K, g,
                                         fp.pairs ? 1 : 0);
    // PCG from x = 0: r = g, z = P r, p = z
    CUDA_CHECK(cudaMemsetAsync(x, 0, N * sizeof(double), st));
    CUDA_CHECK(cudaMemcpyAsync(r, g, N * sizeof(double), cudaMemcpyDeviceToDevice, st));
    k_bj_apply<<<h->n_sub, pb, 2 * K * sizeof(double), st>>>(Xr, Xc, K, r, z, dot2);
    k_pcg_pupdate<<<vb, 256, 0, st>>>(sc, 0, dot2, h->n_sub, z, pv, N, 1);
    count_launch(h, 3);
    for (int k = 0; k < o->max_iter; ++k) {
      const int slot = k & 1;
      prof_begin(h, KID_GSPMV, (double)np * KK * 4.0 + 16.0 * N);
      k_gspmv_pairs<<<(unsigned)std::max<int64_t>(np, 1), 128, 0, st>>>(
          h->d_gram.as<float>(), dpij.as<int2>(), K, pv, dpart2.as<double>());
      k_gspmv_reduce<<<h->n_sub, pb, 0, st>>>(dpart2.as<double>(), dioff.as<int>(),
                                              dilist.as<int>(), K, pv, mu, q, dot1);
      prof_end(h, KID_GSPMV);
      k_pcg_axpy<<<vb, 256, 0, st>>>(sc, slot, dot1, h->n_sub, pv, q, x, r, N);
      k_bj_apply<<<h->n_sub, pb, 2 * K * sizeof(double), st>>>(Xr, Xc, K, r, z, dot2);
      k_pcg_pupdate<<<vb, 256, 0, st>>>(sc, slot, dot2, h->n_sub, z, pv, N, 0);
      count_launch(h, 5);
      ++its;
    }
    k_add_to<<<vb, 256, 0, st>>>(h->d_a.as<double>(), x, N);
    count_launch(h);
    check_launch("pcg");
  }
  // final residual norm ||h - M a|| from the fused pass partials
  launch_fused<T>(h, fp, h->d_a.as<double>(), 1, sc + fsz, gpart);
  std::vector<double> gp(fp.n_units);
  CUDA_CHECK(cudaMemcpyAsync(gp.data(), gpart, fp.n_units * sizeof(double),
                             cudaMemcpyDeviceToHost, st));
  stream_sync(h);
  stage_end(h, 5);
  double rn = 0.0;
  for (double v : gp) rn += v;
  info->status = ELMFB_OK;
  info->iterations = its;
  info->residual_norm = std::sqrt(rn);
  info->normal_residual_norm = NAN;
  info->solve_ms = h->stage_ms[5];
}

}  // namespace

namespace {

// r = h - M a from the FP32-pair panels of ELMFB_FP32_DF32 (the fused pass in
// mode 1 on the pair panels: float-float products and sums, FP64-accurate),
// into h->d_u (padded sorted rows).
void residual_pairs(elmfb_ctx* h, const double* a) {
  struct Swap {   // the pair panels and ELMFB_DF32 for the duration of the pass
    elmfb_ctx* h;
    explicit Swap(elmfb_ctx* hh) : h(hh) {
      std::swap(h->d_panels.p, h->d_panels_df.p);
      std::swap(h->d_panels.bytes, h->d_panels_df.bytes);
      h->cfg.precision = ELMFB_DF32;
    }
    ~Swap() {
      std::swap(h->d_panels.p, h->d_panels_df.p);
      std::swap(h->d_panels.bytes, h->d_panels_df.bytes);
      h->cfg.precision = ELMFB_FP32_DF32;
    }
  } swap(h);
  cudaStream_t st = h->stream;
  FusedPlan fp;
  if (!build_fused_plan(h, fp))
    ELMFB_THROW(ELMFB_ERR_UNSUPPORTED, "refinement: the pair panels need the fused pass");
  DevBuf sc, gp;
  sc.alloc(2 * kScal * sizeof(double), st);
  gp.alloc((size_t)(std::max(kGatherBlocks, fp.n_units) + h->n_sub + 8) * sizeof(double), st);
  CUDA_CHECK(cudaMemsetAsync(sc.p, 0, 2 * kScal * sizeof(double), st));
  h->d_u.alloc(h->NR * sizeof(double), st);
  launch_fused<df2>(h, fp, a, 1, sc.as<double>(), gp.as<double>());
  check_launch("refinement residual");
  stream_sync(h);   // fp's buffers are released on return
}

// Mixed-precision LSQR with refinement (ELMFB_FP32_DF32): `refine` outer
// steps; step 0 solves min ||M a - h|| on the FP32 panels, every later step
// forms r = h - M a from the pair panels and solves min ||M d - r|| on the FP32
// panels (LSQR from zero, the block-Jacobi factors of step 0 reused), a += d.
void lsqr_refine(elmfb_ctx* h, const elmfb_solve_opts* o, elmfb_solve_info* info) {
  cudaStream_t st = h->stream;
  const int64_t N = h->NPhi;
  elmfb_solve_opts oi = *o;
  DevBuf acc, rbuf;
  acc.alloc(N * sizeof(double), st);
  int total = 0;
  double solve_ms = 0.0;
  int status = ELMFB_OK;
  struct Reset {   // the next solve sets up its own preconditioner again
    elmfb_ctx* h;
    ~Reset() { h->bj_reuse = false; }
  } reset{h};
  for (int k = 0; k < o->refine; ++k) {
    elmfb_solve_info ii{};
    if (k == 0) {
      lsqr<float>(h, &oi, &ii);
      CUDA_CHECK(cudaMemcpyAsync(acc.p, h->d_a.p, N * sizeof(double), cudaMemcpyDeviceToDevice,
                                 st));
      info->setup_ms = ii.setup_ms;
      info->precond_retries = ii.precond_retries;
    } else {
      residual_pairs(h, acc.as<double>());
      // the residual becomes the right-hand side of the correction solve
      rbuf.alloc(h->NR * sizeof(double), st);
      CUDA_CHECK(cudaMemcpyAsync(rbuf.p, h->d_u.p, h->NR * sizeof(double),
                                 cudaMemcpyDeviceToDevice, st));
      std::swap(h->d_h.p, rbuf.p);
      std::swap(h->d_h.bytes, rbuf.bytes);
      h->bj_reuse = true;
      oi.warm_start = 0;
      try {
        lsqr<float>(h, &oi, &ii);
      } catch (...) {
        std::swap(h->d_h.p, rbuf.p);
        std::swap(h->d_h.bytes, rbuf.bytes);
        throw;
      }
      std::swap(h->d_h.p, rbuf.p);
      std::swap(h->d_h.bytes, rbuf.bytes);
      const int ub = (int)std::min<int64_t>(ceil_div(N, 256), 1216);
      k_add_to<<<ub, 256, 0, st>>>(acc.as<double>(), h->d_a.as<double>(), N);
      count_launch(h);
      check_launch("refinement update");
    }
    total += ii.iterations;
    solve_ms += ii.solve_ms;
    if (ii.status != ELMFB_OK) status = ii.status;
    info->residual_norm = ii.residual_norm;
    info->normal_residual_norm = ii.normal_residual_norm;
    info->sigma_max = ii.sigma_max;
    info->sigma_min = ii.sigma_min;
  }
  CUDA_CHECK(cudaMemcpyAsync(h->d_a.p, acc.p, N * sizeof(double), cudaMemcpyDeviceToDevice, st));
  stream_sync(h);
  info->status = status;
  info->iterations = total;
  info->solve_ms = solve_ms;
}

}  // namespace

void solve_system(elmfb_ctx* h, const elmfb_solve_opts* o, elmfb_solve_info* info) {
  if (o->method == ELMFB_SOLVE_PCG) {
    pcg_solve<float>(h, o, info);
    return;
  }
  if (o->method == ELMFB_SOLVE_FCG_GNN) {
    fcg_solve(h, o, info);
    return;
  }
  if (o->method == ELMFB_SOLVE_QR) {
    qr_solve(h, o, info);
    return;
  }
  if (o->method != ELMFB_SOLVE_LSQR)
    ELMFB_THROW(ELMFB_ERR_UNSUPPORTED, "solver method not available in this build");
  if (o->preconditioner != ELMFB_PREC_NONE && o->preconditioner != ELMFB_PREC_BLOCK_JACOBI)
    ELMFB_THROW(ELMFB_ERR_INVALID_ARG, "LSQR takes no or block-Jacobi preconditioning");
  if (h->dual()) {
    if (o->warm_start) ELMFB_THROW(ELMFB_ERR_INVALID_ARG, "refinement starts from a = 0");
    lsqr_refine(h, o, info);
  } else if (h->df32()) lsqr<df2>(h, o, info);
  else if (h->fp64()) lsqr<double>(h, o, info);
  else lsqr<float>(h, o, info);
}

template void launch_fused<float>(elmfb_ctx*, FusedPlan&, const double*, int, double*, double*,
                                  const void*);
template void launch_fused<double>(elmfb_ctx*, FusedPlan&, const double*, int, double*, double*,
                                   const void*);
template void launch_fused<df2>(elmfb_ctx*, FusedPlan&, const double*, int, double*, double*,
                                const void*);

namespace {
__global__ void k_gather_records(const BatchInst* __restrict__ inst, int n,
                                 double* __restrict__ out) {
  const int j = blockIdx.x;
  if (j >= n) return;
  const BatchInst& I = inst[j];
  const int t = threadIdx.x;
  if (t < kStage) out[(int64_t)j * kRoundRecord + t] = I.scal[kStage + t];
  else if (t < kRoundRecord) out[(int64_t)j * kRoundRecord + t] = (double)I.flags[t - kStage];
}
}  // namespace

void launch_gather_records(const BatchInst* d_inst, int n, double* out, cudaStream_t st) {
  static_assert(kRoundRecord == kStage + 4, "a record is the staged scalars and four flags");
  if (n <= 0) return;
  k_gather_records<<<n, 32, 0, st>>>(d_inst, n, out);
  check_launch("k_gather_records");
}

void launch_batch_iteration(const BatchShape& sh, const BatchInst* d_inst, const int2* d_fmap,
                            int n_f, const int2* d_cmap, int n_c, const int2* d_tmap, int n_t,
                            cudaStream_t st) {
  if (n_f <= 0 || n_c <= 0 || n_t <= 0) return;
  // the fused pass: every array from the unit's instance
#define ELMFB_FB(F, R)                                                                         \
  if (sh.fpl == F && sh.rows == R) {                                                           \
    ensure_dyn_smem((const void*)k_fused_pipe<float, F, R, true>, sh.smem, true);             \
    k_fused_pipe<float, F, R, true><<<n_f, sh.pthreads, sh.smem, st>>>(                        \
        nullptr, nullptr, sh.K, nullptr, nullptr, nullptr, nullptr, nullptr, nullptr, nullptr, \
        nullptr, nullptr, nullptr, sh.mode, nullptr, nullptr, sh.S, sh.mmax, nullptr, d_inst,  \
        d_fmap);                                                                               \
  } else
  ELMFB_FB(1, 4) ELMFB_FB(1, 8) ELMFB_FB(2, 4) ELMFB_FB(2, 8) ELMFB_FB(3, 4) ELMFB_FB(3, 8)
  ELMFB_FB(4, 4) ELMFB_FB(4, 8)
  ELMFB_THROW(ELMFB_ERR_UNSUPPORTED, "multi-instance fused pass needs K <= 128");
#undef ELMFB_FB
  // the slice sums (the first slice of each instance commits its scalars)
  k_panel_chunks<<<n_c, sh.chunk_threads, 0, st>>>(nullptr, nullptr, nullptr, sh.K, nullptr, 1,
                                                   nullptr, 0, nullptr, d_inst, d_cmap);
  // the tail (the last block of each instance runs its recurrence)
  ensure_dyn_smem((const void*)k_lsqr_tail_tri, sh.tsmem);
  k_lsqr_tail_tri<<<n_t, sh.tthreads, sh.tsmem, st>>>(
      nullptr, nullptr, nullptr, sh.K, nullptr, nullptr, nullptr, nullptr, 0, nullptr, nullptr,
      nullptr, sh.low_kind, nullptr, nullptr, d_inst, d_tmap);
  check_launch("multi-instance LSQR iteration");
}
template void block_jacobi_setup<float>(elmfb_ctx*, double, bool, double, double);
template void block_jacobi_setup<double>(elmfb_ctx*, double, bool, double, double);
template void block_jacobi_setup<df2>(elmfb_ctx*, double, bool, double, double);

void panel_chunk_sums(elmfb_ctx* h, FusedPlan& fp, const double* beta_partial, int n_beta,
                      double* scal) {
  if (fp.n_pchunks == 0) return;
  const int tb = std::min(std::max(32, ((h->K + 31) / 32) * 32), 128);
  k_panel_chunks<<<fp.n_pchunks, tb, 0, h->stream>>>(
      fp.part.as<double>(), fp.fe.as<int>(), fp.pch.as<int2>(), h->K, fp.csum.as<double>(),
      fp.pairs ? 1 : 0, beta_partial, n_beta, scal, nullptr, nullptr);
  check_launch("k_panel_chunks");
  count_launch(h);
}

void panel_sum(elmfb_ctx* h, FusedPlan& fp, double* g) {
  const int pb = std::min(std::max(32, ((h->K + 31) / 32) * 32), 256);
  panel_chunk_sums(h, fp);
  k_panel_sum<<<h->n_sub, pb, 0, h->stream>>>(fp.csum.as<double>(), fp.pco.as<int>(), h->K, g,
                                               fp.pairs ? 1 : 0);
  check_launch("k_panel_sum");
  count_launch(h);
}

void bj_apply(elmfb_ctx* h, const double* r, double* z, double* dot_part) {
  const int K = h->K;
  const int64_t KK = (int64_t)K * K;
  const int pb = std::min(std::max(32, ((K + 31) / 32) * 32), 256);
  k_bj_apply<<<h->n_sub, pb, 2 * K * sizeof(double), h->stream>>>(
      h->d_R.as<double>(), h->d_R.as<double>() + h->n_sub * KK, K, r, z, dot_part);
  check_launch("k_bj_apply");
  count_launch(h);
}

extern "C" int elmfb_tuning_table(int max, elmfb_tuning_entry* out) {
  if (max < 0 || (max > 0 && !out)) return -ELMFB_ERR_INVALID_ARG;
  std::lock_guard<std::mutex> lock(g_tune_mu);
  int n = 0;
  for (const auto& kv : g_tune) {
    if (n < max) out[n] = kv.second;
    ++n;
  }
  return n;
}
