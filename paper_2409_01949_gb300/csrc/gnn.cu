// Learned preconditioner and flexible CG on the normal equations (not in the
// paper).
//
// FCG solves M^T M a = M^T h with the operator applied exactly through the
// panels (one fused pass per iteration, the same cost as an LSQR iteration)
// and a preconditioner that may change between iterations:
//     z = B r + sigma * N(B r / sigma),   sigma = ||B r||,
// B the block-Jacobi factor (X^T X per subdomain) and N a message-passing
// network on the subdomain graph (nodes = subdomains, edges = subdomain pairs
// sharing collocation points): an input layer K -> H, three layers
//     A_l[s] = relu(W_self_l A_{l-1}[s] + W_nb_l mean_{t in N(s)} A_{l-1}[t] + b_l)
// and an output layer H -> K (H = 64).  FCG keeps one previous direction
// (beta = -z.q / p.q, Notay's flexible CG with truncation 1).
//
// The network is trained on (residual, error) pairs produced by FCG solves
// of the same matrix with other right-hand sides: e_k = a_final - a_k, input
// X = B r_k / sigma_k, target T = e_k / sigma_k - X, loss weight
// sigma_k^2 / ||e_k||^2 (so the loss is the relative error of the corrected
// preconditioner), with Adam.  Forward and backward passes are hand-written
// FP32 kernels below; the FP64 definition lives in the oracle's gnn module.
#include <algorithm>
#include <cmath>

#include <new>
#include <stdexcept>

#include <cuda_bf16.h>

#include "elmfb_internal.cuh"
#include "sm100_ptx.cuh"

namespace {

constexpr int kH = 64;
constexpr int kLayers = 3;

__device__ __forceinline__ float relu(float x) { return x > 0.f ? x : 0.f; }

// out[r][o] (+)= sum_i W[o][i] in[r][i] + bias[o]; optional relu.  One block per
// 8 rows, thread per output channel.
__global__ void k_dense_fwd(const float* __restrict__ in, int R, int Din,
                            const float* __restrict__ W, const float* __restrict__ bias,
                            int Dout, float* __restrict__ out, int accumulate, int act) {
  extern __shared__ float xs[];   // [8][Din]
  const int r0 = blockIdx.x * 8;
  for (int t = threadIdx.x; t < 8 * Din; t += blockDim.x) {
    const int r = r0 + t / Din;
    xs[t] = r < R ? in[(int64_t)r * Din + t % Din] : 0.f;
  }
  __syncthreads();
  for (int o = threadIdx.x; o < Dout; o += blockDim.x) {
    const float* w = W + (int64_t)o * Din;
    for (int rr = 0; rr < 8; ++rr) {
      const int r = r0 + rr;
      if (r >= R) break;
      float acc = 0.f;
      for (int i = 0; i < Din; ++i) acc += w[i] * xs[rr * Din + i];
      float* dst = out + (int64_t)r * Dout + o;
      float v = acc + (accumulate ? *dst : (bias ? bias[o] : 0.f));
      *dst = act ? relu(v) : v;
    }
  }
}

// dIn[r][i] (+)= sum_o W[o][i] dOut[r][o]
__global__ void k_dense_bwd_in(const float* __restrict__ dout, int R, int Dout,
                               const float* __restrict__ W, int Din, float* __restrict__ din,
                               int accumulate) {
  extern __shared__ float gs[];   // [8][Dout]
  const int r0 = blockIdx.x * 8;
  for (int t = threadIdx.x; t < 8 * Dout; t += blockDim.x) {
    const int r = r0 + t / Dout;
    gs[t] = r < R ? dout[(int64_t)r * Dout + t % Dout] : 0.f;
  }
  __syncthreads();
  for (int i = threadIdx.x; i < Din; i += blockDim.x) {
    for (int rr = 0; rr < 8; ++rr) {
      const int r = r0 + rr;
      if (r >= R) break;
      float acc = 0.f;
      for (int o = 0; o < Dout; ++o) acc += W[(int64_t)o * Din + i] * gs[rr * Dout + o];
      float* dst = din + (int64_t)r * Din + i;
      *dst = acc + (accumulate ? *dst : 0.f);
    }
  }
}

// dW[o][i] += sum_r dOut[r][o] in[r][i];  db[o] += sum_r dOut[r][o]  (fixed order)
__global__ void k_wgrad(const float* __restrict__ dout, const float* __restrict__ in, int R,
                        int Dout, int Din, float* __restrict__ dW, float* __restrict__ db) {
  const int idx = blockIdx.x * blockDim.x + threadIdx.x;
  if (idx < Dout * Din) {
    const int o = idx / Din, i = idx - o * Din;
    float acc = 0.f;
    for (int r = 0; r < R; ++r) acc += dout[(int64_t)r * Dout + o] * in[(int64_t)r * Din + i];
    dW[idx] += acc;
  }
  if (db && idx < Dout) {
    float acc = 0.f;
    for (int r = 0; r < R; ++r) acc += dout[(int64_t)r * Dout + idx];
    db[idx] += acc;
  }
}

// agg[(b,s)][h] = mean_{t in N(s)} A[(b,t)][h]
__global__ void k_agg(const float* __restrict__ A, int nb_nodes, int B,
                      const int* __restrict__ off, const int* __restrict__ nb,
                      float* __restrict__ agg) {
  const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= (int64_t)B * nb_nodes * kH) return;
  const int h = idx % kH;
  const int64_t rs = idx / kH;
  const int s = rs % nb_nodes, b = rs / nb_nodes;
  const int e0 = off[s], e1 = off[s + 1];
  float acc = 0.f;
  for (int e = e0; e < e1; ++e) acc += A[((int64_t)b * nb_nodes + nb[e]) * kH + h];
  agg[idx] = e1 > e0 ? acc / (float)(e1 - e0) : 0.f;
}

// dA[(b,s)][h] += sum_{t in N(s)} G[(b,t)][h] / |N(t)|   (transpose of the mean)
__global__ void k_aggT(const float* __restrict__ G, int nb_nodes, int B,
                       const int* __restrict__ off, const int* __restrict__ nb,
                       float* __restrict__ dA) {
  const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= (int64_t)B * nb_nodes * kH) return;
  const int h = idx % kH;
  const int64_t rs = idx / kH;
  const int s = rs % nb_nodes, b = rs / nb_nodes;
  float acc = 0.f;
  for (int e = off[s]; e < off[s + 1]; ++e) {
    const int t = nb[e];
    acc += G[((int64_t)b * nb_nodes + t) * kH + h] / (float)(off[t + 1] - off[t]);
  }
  dA[idx] += acc;
}

// dZ = dA * (A > 0)
__global__ void k_relu_mask(const float* __restrict__ A, float* __restrict__ dA, int64_t n) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n && !(A[i] > 0.f)) dA[i] = 0.f;
}

// dY = 2 w_b (Y - T) / B;  loss partial per block
__global__ void k_loss_grad(const float* __restrict__ Y, const float* __restrict__ T,
                            const float* __restrict__ wb, int64_t per_sample, int B,
                            float* __restrict__ dY, double* __restrict__ loss_part) {
  __shared__ double red[32];
  const int64_t n = per_sample * B;
  double acc = 0.0;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int b = (int)(i / per_sample);
    const float d = Y[i] - T[i];
    acc += (double)wb[b] * d * d / B;
    if (dY) dY[i] = 2.f * wb[b] * d / (float)B;
  }
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += red[w];
    loss_part[blockIdx.x] = t;
  }
}

__global__ void k_adam(float* __restrict__ w, const float* __restrict__ g, float* __restrict__ m,
                       float* __restrict__ v, int64_t n, float lr, float b1t, float b2t) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const float gi = g[i];
  m[i] = 0.9f * m[i] + 0.1f * gi;
  v[i] = 0.999f * v[i] + 0.001f * gi * gi;
  const float mh = m[i] / (1.f - b1t), vh = v[i] / (1.f - b2t);
  w[i] -= lr * mh / (sqrtf(vh) + 1e-8f);
}

// x_in[s][k] = (B r)[s][k] / sigma (float) ; sigma = ||B r||
__global__ void k_scale_to_float(const double* __restrict__ z, double inv, float* __restrict__ out,
                                 int64_t n) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) out[i] = (float)(z[i] * inv);
}

// z += sigma * y
__global__ void k_add_scaled_float(double* __restrict__ z, const float* __restrict__ y,
                                   double sigma, int64_t n) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) z[i] += sigma * (double)y[i];
}

__global__ void k_dot_part(const double* __restrict__ a, const double* __restrict__ b, int64_t n,
                           double* __restrict__ part) {
  __shared__ double red[32];
  double acc = 0.0;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    acc += a[i] * b[i];
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += red[w];
    part[blockIdx.x] = t;
  }
}

__global__ void k_axpby(double* __restrict__ y, const double* __restrict__ x, double a, double b,
                        int64_t n) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) y[i] = a * x[i] + b * y[i];
}

// h_sorted[R] = rhs_user[sorted[R]] * hscale(class)
__global__ void k_permute_rhs(const int* __restrict__ sorted, const int* __restrict__ rcls,
                              const double* __restrict__ hscale, const double* __restrict__ rhs,
                              int64_t NR, double* __restrict__ out) {
  const int64_t R = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (R >= NR) return;
  const int r = sorted[R];
  out[R] = r < 0 ? 0.0 : rhs[r] * hscale[rcls[R]];
}

// ---- the network on the tensor cores (inference in FCG's preconditioner) ---
//
// One dense layer, 128 rows r = (sample b, node s) per CTA:
//   out[r][o] = act(sum_c in[r][c] W[o][c] + bias[o])
// with the contraction c over the D1 channels of in1 (weights W1 [Dout][D1])
// and, for the message-passing layers, the H channels of the neighbour mean of
// in2 (weights W2 [Dout][H]): mean over t in N(s) of row (b, t), FP32 sums in
// the neighbour list's order, then one FP32 division by the degree.  Every
// operand is rounded to bfloat16 (to nearest, ties to even) as the threads
// write it into shared memory, in the K-major layout with 128-byte swizzle
// that a TMA SWIZZLE_128B load produces: 64 channels (128 B) per row and
// block, element c of row m at block c / 64, byte
//   m * 128 + ((((c % 64) / 8) ^ (m % 8)) * 16) + (c % 8) * 2.
// One thread issues (D1 + D2) / 16 tcgen05.mma (kind::f16, BF16 x BF16, FP32
// accumulation, M = 128, N = Dout) into TMEM; the four warps read the
// accumulator back (warp w: TMEM lanes = rows 32w .. 32w + 31), add the bias,
// apply the ReLU and store FP32.  Limits: D1 + D2 <= 128 and Dout <= 128, all
// multiples of 16.  The completion wait is bounded: on a timeout flags[6] is
// raised and the block waits once more (bounded) before freeing TMEM.
constexpr int kTcRows = 128;
constexpr int kTcBlock = 128 * 128;                    // bytes: 128 rows x 64 BF16
constexpr size_t kTcSmem = 4 * (size_t)kTcBlock + 1024;   // A and B, 2 blocks each; alignment

// 8 consecutive channels c .. c + 7 (c % 8 == 0) of row m, rounded to bfloat16
__device__ __forceinline__ void tc_store8(uint8_t* tile, int m, int c, const float (&v)[8]) {
  uint32_t p[4];
#pragma unroll
  for (int j = 0; j < 4; ++j) {
    const __nv_bfloat162 b2 = __floats2bfloat162_rn(v[2 * j], v[2 * j + 1]);
    p[j] = *reinterpret_cast<const uint32_t*>(&b2);
  }
  const int chunk = ((c & 63) >> 3) ^ (m & 7);
  *reinterpret_cast<uint4*>(tile + (size_t)(c >> 6) * kTcBlock + (size_t)m * 128 + chunk * 16) =
      make_uint4(p[0], p[1], p[2], p[3]);
}

__global__ void __launch_bounds__(128, 1)
    k_gnn_layer_tc(const float* __restrict__ in1, int D1, const float* __restrict__ W1,
                   const float* __restrict__ in2, const float* __restrict__ W2,
                   const int* __restrict__ off, const int* __restrict__ nb, int n_nodes,
                   const float* __restrict__ bias, int Dout, int64_t R, int act,
                   float* __restrict__ out, int* __restrict__ flags) {
  extern __shared__ uint8_t smraw[];
  __shared__ __align__(8) uint64_t done;
  __shared__ uint32_t tmem_slot;
  uint8_t* At = reinterpret_cast<uint8_t*>(
      (reinterpret_cast<uintptr_t>(smraw) + 1023) & ~uintptr_t(1023));
  uint8_t* Bt = At + 2 * kTcBlock;
  const int D2 = W2 ? kH : 0;
  const int Dk = D1 + D2;
  const int warp = threadIdx.x >> 5;
  const int m = threadIdx.x;   // this thread's row of B and of the output
  const int64_t r = (int64_t)blockIdx.x * kTcRows + m;
  if (threadIdx.x == 0) {
    sm100::mbar_init(&done, 1);
    sm100::fence_mbar_init();
  }
  if (warp == 0) sm100::tmem_alloc(&tmem_slot, 128);
  // A: the tile's rows of in1, then the neighbour means of in2 (zeros past R),
  // as tasks (row, 8-channel chunk) spread over all threads.  A coarse node's
  // long neighbour list is shared by the 8 threads of its chunks; each chunk
  // sums its neighbours in list order.
  const int64_t tile0 = (int64_t)blockIdx.x * kTcRows;
  const int n1 = D1 / 8;
  for (int task = threadIdx.x; task < kTcRows * n1; task += blockDim.x) {
    const int mt = task / n1, c = (task - mt * n1) * 8;
    float v[8];
#pragma unroll
    for (int j = 0; j < 8; ++j) v[j] = 0.f;
    if (tile0 + mt < R) {
      const float4* p = reinterpret_cast<const float4*>(in1 + (tile0 + mt) * D1 + c);
      const float4 a = p[0], b = p[1];
      v[0] = a.x, v[1] = a.y, v[2] = a.z, v[3] = a.w;
      v[4] = b.x, v[5] = b.y, v[6] = b.z, v[7] = b.w;
    }
    tc_store8(At, mt, c, v);
  }
  if (D2 > 0) {
    for (int task = threadIdx.x; task < kTcRows * (kH / 8); task += blockDim.x) {
      const int mt = task >> 3, c = (task & 7) * 8;
      const int64_t rt = tile0 + mt;
      float v[8];
#pragma unroll
      for (int j = 0; j < 8; ++j) v[j] = 0.f;
      if (rt < R) {
        const int s = (int)(rt % n_nodes);
        const int64_t row0 = rt - s;   // node 0 of this sample
        const int e0 = off[s], e1 = off[s + 1];
#pragma unroll 4
        for (int e = e0; e < e1; ++e) {
          const float4* p = reinterpret_cast<const float4*>(in2 + (row0 + nb[e]) * kH + c);
          const float4 a = p[0], b = p[1];
          v[0] += a.x, v[1] += a.y, v[2] += a.z, v[3] += a.w;
          v[4] += b.x, v[5] += b.y, v[6] += b.z, v[7] += b.w;
        }
        if (e1 > e0) {
          const float deg = (float)(e1 - e0);
#pragma unroll
          for (int j = 0; j < 8; ++j) v[j] = v[j] / deg;
        }
      }
      tc_store8(At, mt, D1 + c, v);
    }
  }
  // B: row m of [W1 | W2]
  if (m < Dout) {
    for (int c = 0; c < Dk; c += 8) {
      const float* w = c < D1 ? W1 + (int64_t)m * D1 + c : W2 + (int64_t)m * kH + (c - D1);
      float v[8];
#pragma unroll
      for (int j = 0; j < 8; ++j) v[j] = w[j];
      tc_store8(Bt, m, c, v);
    }
  }
  sm100::fence_proxy_async_smem();   // generic-proxy writes -> the tensor core's reads
  sm100::tc_fence_before();
  __syncthreads();
  sm100::tc_fence_after();
  const uint32_t tmem = tmem_slot;
  if (threadIdx.x == 0) {
    const uint32_t idesc = sm100::idesc_bf16_f32(128, (uint32_t)Dout);
    for (int k = 0; k < Dk / 16; ++k) {
      // 16 channels (32 B) per instruction, inside block k / 4
      const uint32_t blk = (uint32_t)(k >> 2) * kTcBlock;
      const uint64_t ad = sm100::sdesc_k_sw128(sm100::smem_u32(At + blk)) + 2 * (k & 3);
      const uint64_t bd = sm100::sdesc_k_sw128(sm100::smem_u32(Bt + blk)) + 2 * (k & 3);
      sm100::mma_bf16(tmem, ad, bd, idesc, k > 0 ? 1u : 0u);
    }
    sm100::mma_commit(&done);
  }
  __syncwarp();
  const bool got = sm100::mbar_wait(&done, 0);
  if (!got) {
    if (threadIdx.x == 0) atomicOr(&flags[6], 1);
    sm100::mbar_wait(&done, 0);   // let the MMAs finish before TMEM is read or freed
  }
  sm100::tc_fence_after();
  for (int c0 = 0; c0 < Dout; c0 += 16) {
    uint32_t v[16];
    sm100::tmem_ld16(tmem + ((uint32_t)(32 * warp) << 16) + (uint32_t)c0, v);
    sm100::tmem_ld_wait();
    if (r < R && got) {
      float* o = out + r * Dout + c0;
#pragma unroll
      for (int j = 0; j < 16; ++j) {
        const float x = __uint_as_float(v[j]) + bias[c0 + j];
        o[j] = act ? relu(x) : x;
      }
    }
  }
  sm100::tc_fence_before();
  __syncthreads();
  if (warp == 0) sm100::tmem_dealloc(tmem, 128);
}

}  // namespace

// ------------------------------------------------------------------ host ----
namespace {

constexpr int kDotBlocks = 256;

struct Gnn {
  elmfb_ctx* h;
  int K;
  int n;   // nodes
  int64_t nw;
  float *W_in, *b_in, *W_self[kLayers], *W_nb[kLayers], *b_l[kLayers], *W_out, *b_out;
  void bind(float* w) {
    float* p = w;
    W_in = p;
    p += kH * K;
    b_in = p;
    p += kH;
    for (int l = 0; l < kLayers; ++l) {
      W_self[l] = p;
      p += kH * kH;
      W_nb[l] = p;
      p += kH * kH;
      b_l[l] = p;
      p += kH;
    }
    W_out = p;
    p += K * kH;
    b_out = p;
    p += K;
  }
};

int64_t gnn_weight_count(int K) { return (int64_t)kH * K + kH + kLayers * (2 * kH * kH + kH) + K * kH + K; }

void gnn_graph(elmfb_ctx* h) {
  if (!h->gnn_off.empty()) return;
  if (h->gram_pair_ij.empty()) gram_build_pairs(h);
  std::vector<std::vector<int>> nb(h->n_sub);
  for (auto& ij : h->gram_pair_ij)
    if (ij.first != ij.second) {
      nb[ij.first].push_back(ij.second);
      nb[ij.second].push_back(ij.first);
    }
  h->gnn_off.assign(h->n_sub + 1, 0);
  h->gnn_nb.clear();
  for (int s = 0; s < h->n_sub; ++s) {
    std::sort(nb[s].begin(), nb[s].end());
    h->gnn_off[s] = (int)h->gnn_nb.size();
    h->gnn_nb.insert(h->gnn_nb.end(), nb[s].begin(), nb[s].end());
  }
  h->gnn_off[h->n_sub] = (int)h->gnn_nb.size();
  h->d_gnn_off.alloc(h->gnn_off.size() * sizeof(int), h->stream);
  h->d_gnn_nb.alloc(std::max<size_t>(h->gnn_nb.size(), 1) * sizeof(int), h->stream);
  CUDA_CHECK(cudaMemcpyAsync(h->d_gnn_off.p, h->gnn_off.data(), h->gnn_off.size() * sizeof(int),
                             cudaMemcpyHostToDevice, h->stream));
  if (!h->gnn_nb.empty())
    CUDA_CHECK(cudaMemcpyAsync(h->d_gnn_nb.p, h->gnn_nb.data(), h->gnn_nb.size() * sizeof(int),
                               cudaMemcpyHostToDevice, h->stream));
}

void gnn_alloc(elmfb_ctx* h) {
  gnn_graph(h);
  const int64_t nw = gnn_weight_count(h->K);
  if (h->d_gnn_w.bytes < (size_t)nw * sizeof(float)) {
    h->d_gnn_w.alloc(nw * sizeof(float), h->stream);
    CUDA_CHECK(cudaMemsetAsync(h->d_gnn_w.p, 0, nw * sizeof(float), h->stream));
  }
}

// Forward (and backward when dW != nullptr) for a batch of B samples.
// X, T: [B][n][K] float; wb: [B]; Y out: [B][n][K].  Returns the loss.
double gnn_pass(elmfb_ctx* h, int B, const float* X, const float* T, const float* wb, float* Y,
                float* dW) {
  cudaStream_t st = h->stream;
  const int K = h->K, n = h->n_sub;
  const int64_t R = (int64_t)B * n;
  Gnn g{h, K, n, gnn_weight_count(K)};
  g.bind(h->d_gnn_w.as<float>());
  // activations: A0..A3, AGG1..3 [R][H]; scratch dA, tmp [R][H]
  h->d_gnn_act.alloc((size_t)R * kH * (2 * kLayers + 3) * sizeof(float), st);
  float* A[kLayers + 1];
  float* AG[kLayers];
  float* base = h->d_gnn_act.as<float>();
  for (int l = 0; l <= kLayers; ++l) A[l] = base + (int64_t)l * R * kH;
  for (int l = 0; l < kLayers; ++l) AG[l] = base + (int64_t)(kLayers + 1 + l) * R * kH;
  float* dA = base + (int64_t)(2 * kLayers + 1) * R * kH;
  float* tmp = dA + R * kH;
  const unsigned rb = (unsigned)ceil_div(R, 8);
  const unsigned eb = (unsigned)ceil_div(R * kH, 256);
  const int* off = h->d_gnn_off.as<int>();
  const int* nb = h->d_gnn_nb.as<int>();
  k_dense_fwd<<<rb, 128, 8 * K * sizeof(float), st>>>(X, (int)R, K, g.W_in, g.b_in, kH, A[0], 0, 1);
  for (int l = 0; l < kLayers; ++l) {
    k_agg<<<eb, 256, 0, st>>>(A[l], n, B, off, nb, AG[l]);
    k_dense_fwd<<<rb, 128, 8 * kH * sizeof(float), st>>>(A[l], (int)R, kH, g.W_self[l], g.b_l[l],
                                                          kH, A[l + 1], 0, 0);
    k_dense_fwd<<<rb, 128, 8 * kH * sizeof(float), st>>>(AG[l], (int)R, kH, g.W_nb[l], nullptr,
                                                          kH, A[l + 1], 1, 1);
  }
  k_dense_fwd<<<rb, 128, 8 * kH * sizeof(float), st>>>(A[kLayers], (int)R, kH, g.W_out, g.b_out,
                                                        K, Y, 0, 0);
  count_launch(h, 2 + 3 * kLayers);
  double loss = 0.0;
  if (T) {
    h->d_gnn_lp.alloc(kDotBlocks * sizeof(double), st);
    h->d_gnn_dy.alloc((size_t)R * K * sizeof(float), st);
    float* dY = h->d_gnn_dy.as<float>();
    k_loss_grad<<<kDotBlocks, 256, 0, st>>>(Y, T, wb, (int64_t)n * K, B, dW ? dY : nullptr,
                                            h->d_gnn_lp.as<double>());
    count_launch(h);
    if (dW) {
      Gnn gd{h, K, n, g.nw};
      gd.bind(dW);
      CUDA_CHECK(cudaMemsetAsync(dW, 0, g.nw * sizeof(float), st));
      // output layer
      k_wgrad<<<(unsigned)ceil_div((int64_t)K * kH, 256), 256, 0, st>>>(dY, A[kLayers], (int)R, K,
                                                                         kH, gd.W_out, gd.b_out);
      k_dense_bwd_in<<<rb, 128, 8 * K * sizeof(float), st>>>(dY, (int)R, K, g.W_out, kH, dA, 0);
      for (int l = kLayers - 1; l >= 0; --l) {
        k_relu_mask<<<eb, 256, 0, st>>>(A[l + 1], dA, R * kH);   // dA now holds dZ_l
        k_wgrad<<<(unsigned)ceil_div(kH * kH, 256), 256, 0, st>>>(dA, A[l], (int)R, kH, kH,
                                                                  gd.W_self[l], gd.b_l[l]);
        k_wgrad<<<(unsigned)ceil_div(kH * kH, 256), 256, 0, st>>>(dA, AG[l], (int)R, kH, kH,
                                                                  gd.W_nb[l], nullptr);
        k_dense_bwd_in<<<rb, 128, 8 * kH * sizeof(float), st>>>(dA, (int)R, kH, g.W_nb[l], kH,
                                                                 tmp, 0);
        // dA_{l-1} = dZ W_self + aggT(dZ W_nb): write into the tmp2 region (reuse A? no)
        float* dprev = AG[l];   // AG[l] no longer needed once its gradient is taken
        k_dense_bwd_in<<<rb, 128, 8 * kH * sizeof(float), st>>>(dA, (int)R, kH, g.W_self[l],
                                                                 kH, dprev, 0);
        k_aggT<<<eb, 256, 0, st>>>(tmp, n, B, off, nb, dprev);
        CUDA_CHECK(cudaMemcpyAsync(dA, dprev, R * kH * sizeof(float), cudaMemcpyDeviceToDevice,
                                   st));
        count_launch(h, 6);
      }
      k_relu_mask<<<eb, 256, 0, st>>>(A[0], dA, R * kH);
      k_wgrad<<<(unsigned)ceil_div((int64_t)kH * K, 256), 256, 0, st>>>(dA, X, (int)R, kH, K,
                                                                         gd.W_in, gd.b_in);
      count_launch(h, 4);
    }
    std::vector<double> lp(kDotBlocks);
    CUDA_CHECK(cudaMemcpyAsync(lp.data(), h->d_gnn_lp.p, kDotBlocks * sizeof(double),
                               cudaMemcpyDeviceToHost, st));
    stream_sync(h);
    for (double v : lp) loss += v;
  }
  check_launch("gnn pass");
  return loss;
}

// The forward pass as FCG applies it: bfloat16 operands on the tensor cores,
// one k_gnn_layer_tc launch per layer (the neighbour means formed inside the
// message-passing layers).  X, Y: [B][n][K] float on the device.  K must be a
// multiple of 16 up to 128; other K take gnn_pass's FP32 forward.  A timed-out
// completion wait raises flags[6] (cleared by the caller).
bool gnn_tc_supported(int K) { return K >= 16 && K <= 128 && K % 16 == 0; }

void gnn_infer(elmfb_ctx* h, int B, const float* X, float* Y) {
  const int K = h->K, n = h->n_sub;
  if (!gnn_tc_supported(K)) {
    gnn_pass(h, B, X, nullptr, nullptr, Y, nullptr);
    return;
  }
  cudaStream_t st = h->stream;
  const int64_t R = (int64_t)B * n;
  Gnn g{h, K, n, gnn_weight_count(K)};
  g.bind(h->d_gnn_w.as<float>());
  h->d_gnn_act.alloc((size_t)R * kH * 2 * sizeof(float), st);
  float* cur = h->d_gnn_act.as<float>();
  float* nxt = cur + R * kH;
  ensure_dyn_smem((const void*)k_gnn_layer_tc, kTcSmem);
  const unsigned grid = (unsigned)ceil_div(R, kTcRows);
  const int* off = h->d_gnn_off.as<int>();
  const int* nb = h->d_gnn_nb.as<int>();
  int* flags = h->d_flags.as<int>();
  k_gnn_layer_tc<<<grid, 128, kTcSmem, st>>>(X, K, g.W_in, nullptr, nullptr, off, nb, n, g.b_in,
                                              kH, R, 1, cur, flags);
  for (int l = 0; l < kLayers; ++l) {
    k_gnn_layer_tc<<<grid, 128, kTcSmem, st>>>(cur, kH, g.W_self[l], cur, g.W_nb[l], off, nb, n,
                                                g.b_l[l], kH, R, 1, nxt, flags);
    std::swap(cur, nxt);
  }
  k_gnn_layer_tc<<<grid, 128, kTcSmem, st>>>(cur, kH, g.W_out, nullptr, nullptr, off, nb, n,
                                              g.b_out, K, R, 0, Y, flags);
  count_launch(h, kLayers + 2);
  check_launch("gnn inference");
}

double dot(elmfb_ctx* h, const double* a, const double* b, int64_t n, DevBuf& part) {
  part.alloc(kDotBlocks * sizeof(double), h->stream);
  k_dot_part<<<kDotBlocks, 256, 0, h->stream>>>(a, b, n, part.as<double>());
  count_launch(h);
  std::vector<double> p(kDotBlocks);
  CUDA_CHECK(cudaMemcpyAsync(p.data(), part.p, kDotBlocks * sizeof(double), cudaMemcpyDeviceToHost,
                             h->stream));
  stream_sync(h);
  double s = 0.0;
  for (double v : p) s += v;
  return s;
}

// state of one FCG run on M^T M a = g
struct Fcg {
  elmfb_ctx* h;
  FusedPlan fp;
  DevBuf vec, part, sc, xin, yout, gpart;
  DevBuf Xc, ctmp;   // coarse-level correction: X_c = L_c^{-1} of the joint coarse block
  int nc = 0;        // its columns (0: plain block-Jacobi)
  double *x, *r, *z, *p, *q, *g;
  int64_t N;
  void init() {
    N = h->NPhi;
    if (!build_fused_plan(h, fp))
      ELMFB_THROW(ELMFB_ERR_UNSUPPORTED, "FCG needs K <= 128 and <= 32 covering panels per cell");
    vec.alloc(6 * N * sizeof(double), h->stream);
    x = vec.as<double>();
    r = x + N;
    z = r + N;
    p = z + N;
    q = p + N;
    g = q + N;
    sc.alloc(32 * sizeof(double), h->stream);
    CUDA_CHECK(cudaMemsetAsync(sc.p, 0, 32 * sizeof(double), h->stream));   // alpha = 0
    gpart.alloc((size_t)std::max(fp.n_units, 1) * sizeof(double), h->stream);
    h->d_u.alloc(h->NR * sizeof(double), h->stream);
    // the fused pass reads u with coefficient 0 in normal_op: keep it finite
    CUDA_CHECK(cudaMemsetAsync(h->d_u.p, 0, h->NR * sizeof(double), h->stream));
  }
  // y = M^T M v   (fused pass with coef 0: u' = M v, then the panel sums)
  void normal_op(const double* v, double* y) {
    if (h->df32()) launch_fused<df2>(h, fp, v, 0, sc.as<double>(), gpart.as<double>());
    else if (h->fp64()) launch_fused<double>(h, fp, v, 0, sc.as<double>(), gpart.as<double>());
    else launch_fused<float>(h, fp, v, 0, sc.as<double>(), gpart.as<double>());
    panel_sum(h, fp, y);
  }
  // g = M^T h(sorted) for the handle's current h vector
  void rhs() {
    if (h->df32()) launch_fused<df2>(h, fp, x, 1, sc.as<double>(), gpart.as<double>());
    else if (h->fp64()) launch_fused<double>(h, fp, x, 1, sc.as<double>(), gpart.as<double>());
    else launch_fused<float>(h, fp, x, 1, sc.as<double>(), gpart.as<double>());
    panel_sum(h, fp, g);
  }
  // z = B r (+ sigma N(B r / sigma))
  void precond(bool use_gnn) {
    bj_apply(h, r, z, part.as<double>());
    if (nc > 0) coarse_apply(h, Xc, nc, r, z, ctmp);
    if (!use_gnn) return;
    const double s2 = dot(h, z, z, N, part);
    const double sigma = std::sqrt(s2);
    if (!(sigma > 0.0)) return;
    xin.alloc(N * sizeof(float), h->stream);
    yout.alloc(N * sizeof(float), h->stream);
    const unsigned nb = (unsigned)ceil_div(N, 256);
    k_scale_to_float<<<nb, 256, 0, h->stream>>>(z, 1.0 / sigma, xin.as<float>(), N);
    gnn_infer(h, 1, xin.as<float>(), yout.as<float>());
    k_add_scaled_float<<<nb, 256, 0, h->stream>>>(z, yout.as<float>(), sigma, N);
    count_launch(h, 2);
  }
  // run `iters` FCG iterations from x (zero unless warm), recording (r_k, x_k) if asked
  int run(int iters, bool use_gnn, double rtol, std::vector<float>* rec_r,
          std::vector<float>* rec_x, double* final_rel) {
    part.alloc(std::max<int64_t>(kDotBlocks, h->n_sub) * sizeof(double), h->stream);
    const unsigned nb = (unsigned)ceil_div(N, 256);
    normal_op(x, q);
    CUDA_CHECK(cudaMemcpyAsync(r, g, N * sizeof(double), cudaMemcpyDeviceToDevice, h->stream));
    k_axpby<<<nb, 256, 0, h->stream>>>(r, q, -1.0, 1.0, N);   // r = g - A x
    const double g0 = std::sqrt(dot(h, g, g, N, part));
    precond(use_gnn);
    CUDA_CHECK(cudaMemcpyAsync(p, z, N * sizeof(double), cudaMemcpyDeviceToDevice, h->stream));
    int it = 0;
    double rel = 1.0;
    for (; it < iters; ++it) {
      if (rec_r) {
        std::vector<double> hr(N), hx(N);
        CUDA_CHECK(cudaMemcpyAsync(hr.data(), r, N * sizeof(double), cudaMemcpyDeviceToHost,
                                   h->stream));
        CUDA_CHECK(cudaMemcpyAsync(hx.data(), x, N * sizeof(double), cudaMemcpyDeviceToHost,
                                   h->stream));
        stream_sync(h);
        rec_r->insert(rec_r->end(), hr.begin(), hr.end());
        rec_x->insert(rec_x->end(), hx.begin(), hx.end());
      }
      normal_op(p, q);
      const double pq = dot(h, p, q, N, part);
      const double rz = dot(h, r, z, N, part);
      if (!(pq > 0.0)) break;
      const double alpha = rz / pq;
      k_axpby<<<nb, 256, 0, h->stream>>>(x, p, alpha, 1.0, N);
      k_axpby<<<nb, 256, 0, h->stream>>>(r, q, -alpha, 1.0, N);
      count_launch(h, 3);
      rel = std::sqrt(dot(h, r, r, N, part)) / (g0 > 0 ? g0 : 1.0);
      if (rel <= rtol) {
        ++it;
        break;
      }
      precond(use_gnn);
      const double zq = dot(h, z, q, N, part);
      const double beta = -zq / pq;
      k_axpby<<<nb, 256, 0, h->stream>>>(p, z, 1.0, beta, N);   // p = z + beta p
      count_launch(h);
    }
    check_launch("fcg");
    if (final_rel) *final_rel = rel;
    return it;
  }
};

}  // namespace

// FCG on the normal equations (method ELMFB_SOLVE_FCG_GNN)
void fcg_solve(elmfb_ctx* h, const elmfb_solve_opts* o, elmfb_solve_info* info) {
  const bool use_gnn = o->preconditioner == ELMFB_PREC_BJ_GNN;
  if (use_gnn && !h->gnn_trained)
    ELMFB_THROW(ELMFB_ERR_STATE, "learned preconditioner requested before elmfb_gnn_train / "
                                 "elmfb_gnn_set_weights");
  stage_begin(h, 4);
  if (h->df32()) block_jacobi_setup<df2>(h, o->shift, false);
  else if (h->fp64()) block_jacobi_setup<double>(h, o->shift, false);
  else block_jacobi_setup<float>(h, o->shift, false);
  stage_end(h, 4);
  info->setup_ms = h->stage_ms[4];
  info->precond_retries = h->bj_retries;
  if (use_gnn) gnn_alloc(h);
  Fcg f{h};
  f.init();
  if (o->preconditioner == ELMFB_PREC_BJ_COARSE) {
    // the coarse block from the same normal operator the iteration applies
    stage_begin(h, 4);
    int cr = 0;
    coarse_setup(h, o->coarse_levels, o->shift,
                 [&](const double* v, double* y) { f.normal_op(v, y); }, f.Xc, &cr);
    f.nc = coarse_columns(h, o->coarse_levels);
    stage_end(h, 4);
    info->setup_ms += h->stage_ms[4];
    info->precond_retries += cr;
  }
  stage_begin(h, 5);
  CUDA_CHECK(cudaMemsetAsync(f.x, 0, f.N * sizeof(double), h->stream));
  f.rhs();
  if (o->warm_start)
    CUDA_CHECK(cudaMemcpyAsync(f.x, h->d_a.p, f.N * sizeof(double), cudaMemcpyDeviceToDevice,
                               h->stream));
  double rel = 1.0;
  const int its = f.run(o->max_iter, use_gnn, o->btol, nullptr, nullptr, &rel);
  CUDA_CHECK(cudaMemcpyAsync(h->d_a.p, f.x, f.N * sizeof(double), cudaMemcpyDeviceToDevice,
                             h->stream));
  stage_end(h, 5);
  if (use_gnn && gnn_tc_supported(h->K)) {
    int timed_out = 0;
    CUDA_CHECK(cudaMemcpyAsync(&timed_out, h->d_flags.as<int>() + 6, sizeof(int),
                               cudaMemcpyDeviceToHost, h->stream));
    stream_sync(h);
    if (timed_out)
      ELMFB_THROW(ELMFB_ERR_TIMEOUT, "learned preconditioner: a tensor-core wait timed out");
  }
  info->status = rel <= o->btol ? ELMFB_OK : ELMFB_ERR_NOT_CONVERGED;
  info->iterations = its;
  info->residual_norm = NAN;
  info->normal_residual_norm = rel;   // ||g - M^T M a|| / ||g||
  info->solve_ms = h->stage_ms[5];
}

extern "C" {

int64_t elmfb_gnn_num_weights(elmfb_t h) { return h ? gnn_weight_count(h->K) : -1; }

int elmfb_gnn_graph(elmfb_t h, int* off, int* nb, int64_t* n_edges) {
  if (!h) return ELMFB_ERR_INVALID_ARG;
  try {
    CUDA_CHECK(cudaSetDevice(h->device));
    if (!h->assembled) ELMFB_THROW(ELMFB_ERR_STATE, "graph before assemble");
    gnn_graph(h);
    if (n_edges) *n_edges = (int64_t)h->gnn_nb.size();
    if (off) std::copy(h->gnn_off.begin(), h->gnn_off.end(), off);
    if (nb) std::copy(h->gnn_nb.begin(), h->gnn_nb.end(), nb);
    return ELMFB_OK;
  } catch (const elmfb_error& e) {
    h->err = e.msg;
    return e.code;
  } catch (const std::bad_alloc&) {
    h->err = "host allocation failed";
    return ELMFB_ERR_OOM;
  } catch (const std::exception& e) {
    h->err = e.what();
    return ELMFB_ERR_CUDA;
  }
}

int elmfb_gnn_set_weights(elmfb_t h, const float* w) {
  if (!h || !w) return ELMFB_ERR_INVALID_ARG;
  try {
    CUDA_CHECK(cudaSetDevice(h->device));
    if (!h->assembled) ELMFB_THROW(ELMFB_ERR_STATE, "set_weights before assemble");
    gnn_alloc(h);
    CUDA_CHECK(cudaMemcpy(h->d_gnn_w.p, w, gnn_weight_count(h->K) * sizeof(float),
                          cudaMemcpyDefault));
    h->gnn_trained = true;
    return ELMFB_OK;
  } catch (const elmfb_error& e) {
    h->err = e.msg;
    return e.code;
  } catch (const std::bad_alloc&) {
    h->err = "host allocation failed";
    return ELMFB_ERR_OOM;
  } catch (const std::exception& e) {
    h->err = e.what();
    return ELMFB_ERR_CUDA;
  }
}

int elmfb_gnn_get_weights(elmfb_t h, float* w) {
  if (!h || !w) return ELMFB_ERR_INVALID_ARG;
  try {
    CUDA_CHECK(cudaSetDevice(h->device));
    if (!h->d_gnn_w.p) ELMFB_THROW(ELMFB_ERR_STATE, "no network weights yet");
    CUDA_CHECK(cudaMemcpy(w, h->d_gnn_w.p, gnn_weight_count(h->K) * sizeof(float),
                          cudaMemcpyDefault));
    return ELMFB_OK;
  } catch (const elmfb_error& e) {
    h->err = e.msg;
    return e.code;
  } catch (const std::bad_alloc&) {
    h->err = "host allocation failed";
    return ELMFB_ERR_OOM;
  } catch (const std::exception& e) {
    h->err = e.what();
    return ELMFB_ERR_CUDA;
  }
}

int elmfb_gnn_infer(elmfb_t h, int batch, const float* x, float* y) {
  if (!h || batch < 1 || !x || !y) return ELMFB_ERR_INVALID_ARG;
  try {
    CUDA_CHECK(cudaSetDevice(h->device));
    if (!h->d_gnn_w.p) ELMFB_THROW(ELMFB_ERR_STATE, "no network weights yet");
    if (!gnn_tc_supported(h->K))
      ELMFB_THROW(ELMFB_ERR_UNSUPPORTED,
                  "tensor-core inference needs K a multiple of 16, at most 128");
    cudaStream_t st = h->stream;
    const int64_t n = (int64_t)batch * h->n_sub * h->K;
    DevBuf dx, dy;
    dx.alloc(n * sizeof(float), st);
    dy.alloc(n * sizeof(float), st);
    CUDA_CHECK(cudaMemcpyAsync(dx.p, x, n * sizeof(float), cudaMemcpyDefault, st));
    CUDA_CHECK(cudaMemsetAsync(h->d_flags.as<int>() + 6, 0, sizeof(int), st));
    gnn_infer(h, batch, dx.as<float>(), dy.as<float>());
    int timed_out = 0;
    CUDA_CHECK(cudaMemcpyAsync(&timed_out, h->d_flags.as<int>() + 6, sizeof(int),
                               cudaMemcpyDeviceToHost, st));
    CUDA_CHECK(cudaMemcpyAsync(y, dy.p, n * sizeof(float), cudaMemcpyDefault, st));
    stream_sync(h);
    if (timed_out) ELMFB_THROW(ELMFB_ERR_TIMEOUT, "network inference: a tensor-core wait timed out");
    return ELMFB_OK;
  } catch (const elmfb_error& e) {
    h->err = e.msg;
    return e.code;
  } catch (const std::bad_alloc&) {
    h->err = "host allocation failed";
    return ELMFB_ERR_OOM;
  } catch (const std::exception& e) {
    h->err = e.what();
    return ELMFB_ERR_CUDA;
  }
}

int elmfb_gnn_eval(elmfb_t h, int batch, const float* x, const float* t, const float* wb,
                   float* y, float* grad, double* loss) {
  if (!h || batch < 1 || !x || !y) return ELMFB_ERR_INVALID_ARG;
  try {
    CUDA_CHECK(cudaSetDevice(h->device));
    if (!h->d_gnn_w.p) ELMFB_THROW(ELMFB_ERR_STATE, "no network weights yet");
    cudaStream_t st = h->stream;
    const int64_t n = (int64_t)batch * h->n_sub * h->K;
    DevBuf dx, dt, dw, dy, dg;
    dx.alloc(n * sizeof(float), st);
    dy.alloc(n * sizeof(float), st);
    CUDA_CHECK(cudaMemcpyAsync(dx.p, x, n * sizeof(float), cudaMemcpyDefault, st));
    if (t) {
      dt.alloc(n * sizeof(float), st);
      dw.alloc(batch * sizeof(float), st);
      CUDA_CHECK(cudaMemcpyAsync(dt.p, t, n * sizeof(float), cudaMemcpyDefault, st));
      CUDA_CHECK(cudaMemcpyAsync(dw.p, wb, batch * sizeof(float), cudaMemcpyDefault, st));
    }
    if (grad) dg.alloc(gnn_weight_count(h->K) * sizeof(float), st);
    const double L = gnn_pass(h, batch, dx.as<float>(), t ? dt.as<float>() : nullptr,
                              t ? dw.as<float>() : nullptr, dy.as<float>(),
                              (t && grad) ? dg.as<float>() : nullptr);
    CUDA_CHECK(cudaMemcpyAsync(y, dy.p, n * sizeof(float), cudaMemcpyDefault, st));
    if (t && grad)
      CUDA_CHECK(cudaMemcpyAsync(grad, dg.p, gnn_weight_count(h->K) * sizeof(float),
                                 cudaMemcpyDefault, st));
    stream_sync(h);
    if (loss) *loss = L;
    return ELMFB_OK;
  } catch (const elmfb_error& e) {
    h->err = e.msg;
    return e.code;
  } catch (const std::bad_alloc&) {
    h->err = "host allocation failed";
    return ELMFB_ERR_OOM;
  } catch (const std::exception& e) {
    h->err = e.what();
    return ELMFB_ERR_CUDA;
  }
}

int elmfb_gnn_train(elmfb_t h, int n_rhs, const double* rhs, int solve_iters, int epochs,
                    double lr, uint64_t seed, double* loss2) {
  if (!h || n_rhs < 1 || !rhs || solve_iters < 2 || epochs < 1 || !(lr > 0.0))
    return ELMFB_ERR_INVALID_ARG;
  try {
    CUDA_CHECK(cudaSetDevice(h->device));
    if (!h->assembled) ELMFB_THROW(ELMFB_ERR_STATE, "train before assemble");
    cudaStream_t st = h->stream;
    const int K = h->K;
    const int64_t N = h->NPhi;
    if (h->df32()) block_jacobi_setup<df2>(h, 1e-12, false);
    else if (h->fp64()) block_jacobi_setup<double>(h, 1e-12, false);
    else block_jacobi_setup<float>(h, 1e-10, false);
    gnn_alloc(h);
    // initial weights: He-uniform from SplitMix64 (seeded), biases zero; output layer zero so
    // the untrained preconditioner equals block-Jacobi
    {
      const int64_t nw = gnn_weight_count(K);
      std::vector<float> w(nw, 0.f);
      auto rnd = [&](uint64_t i) {
        uint64_t z = seed + (i + 1) * 0x9E3779B97F4A7C15ULL;
        z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
        z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
        z ^= z >> 31;
        return (float)((double)(z >> 40) * (1.0 / 16777216.0) * 2.0 - 1.0);
      };
      int64_t o = 0;
      auto fill = [&](int64_t count, float a) {
        for (int64_t i = 0; i < count; ++i) w[o + i] = a * rnd(o + i);
        o += count;
      };
      fill((int64_t)kH * K, std::sqrt(6.f / K));
      o += kH;
      for (int l = 0; l < kLayers; ++l) {
        fill((int64_t)kH * kH, std::sqrt(3.f / kH));
        fill((int64_t)kH * kH, std::sqrt(3.f / kH));
        o += kH;
      }
      CUDA_CHECK(cudaMemcpy(h->d_gnn_w.p, w.data(), nw * sizeof(float), cudaMemcpyHostToDevice));
    }
    // training pairs from FCG solves with block-Jacobi, one per right-hand side
    std::vector<float> X, T, WB;
    DevBuf drhs, dhs, dsave;
    drhs.alloc(h->n_rows * sizeof(double), st);
    dhs.alloc(h->NR * sizeof(double), st);
    dsave.alloc(h->NR * sizeof(double), st);
    CUDA_CHECK(cudaMemcpyAsync(dsave.p, h->d_h.p, h->NR * sizeof(double),
                               cudaMemcpyDeviceToDevice, st));
    std::vector<double> hsc(kMaxClasses);
    for (int c = 0; c < h->n_classes; ++c) hsc[c] = h->cls[c].hscale;
    DevBuf dhsc;
    dhsc.alloc(kMaxClasses * sizeof(double), st);
    CUDA_CHECK(cudaMemcpyAsync(dhsc.p, hsc.data(), kMaxClasses * sizeof(double),
                               cudaMemcpyHostToDevice, st));
    Fcg f{h};
    f.init();
    DevBuf part;
    part.alloc(std::max<int64_t>(kDotBlocks, h->n_sub) * sizeof(double), st);
    std::vector<double> zr(N);
    for (int i = 0; i < n_rhs; ++i) {
      CUDA_CHECK(cudaMemcpyAsync(drhs.p, rhs + (int64_t)i * h->n_rows,
                                 h->n_rows * sizeof(double), cudaMemcpyDefault, st));
      k_permute_rhs<<<(unsigned)ceil_div(h->NR, 256), 256, 0, st>>>(
          h->d_sorted.as<int>(), h->d_rcls.as<int>(), dhsc.as<double>(), drhs.as<double>(),
          h->NR, h->d_h.as<double>());
      count_launch(h);
      CUDA_CHECK(cudaMemsetAsync(f.x, 0, N * sizeof(double), st));
      f.rhs();
      std::vector<float> rr, xx;
      f.run(2 * solve_iters, false, 0.0, &rr, &xx, nullptr);
      // final iterate = reference solution for the recorded errors
      std::vector<double> xf(N);
      CUDA_CHECK(cudaMemcpy(xf.data(), f.x, N * sizeof(double), cudaMemcpyDeviceToHost));
      for (int k = 0; k < solve_iters; ++k) {
        // z = B r_k on the device
        std::vector<double> rk(rr.begin() + (int64_t)k * N, rr.begin() + (int64_t)(k + 1) * N);
        CUDA_CHECK(cudaMemcpy(f.r, rk.data(), N * sizeof(double), cudaMemcpyHostToDevice));
        bj_apply(h, f.r, f.z, part.as<double>());
        CUDA_CHECK(cudaMemcpy(zr.data(), f.z, N * sizeof(double), cudaMemcpyDeviceToHost));
        double s2 = 0.0, e2 = 0.0;
        for (int64_t j = 0; j < N; ++j) s2 += zr[j] * zr[j];
        for (int64_t j = 0; j < N; ++j) {
          const double e = xf[j] - xx[(int64_t)k * N + j];
          e2 += e * e;
        }
        const double sigma = std::sqrt(s2);
        if (!(sigma > 0.0) || !(e2 > 0.0)) continue;
        for (int64_t j = 0; j < N; ++j) {
          const double xin = zr[j] / sigma;
          const double e = xf[j] - xx[(int64_t)k * N + j];
          X.push_back((float)xin);
          T.push_back((float)(e / sigma - xin));
        }
        WB.push_back((float)(s2 / e2));
      }
    }
    CUDA_CHECK(cudaMemcpyAsync(h->d_h.p, dsave.p, h->NR * sizeof(double),
                               cudaMemcpyDeviceToDevice, st));
    const int S = (int)WB.size();
    if (S == 0) ELMFB_THROW(ELMFB_ERR_BREAKDOWN, "no training pairs");
    // Adam over mini-batches of 8 samples, fixed order
    const int64_t nw = gnn_weight_count(K);
    DevBuf dX, dT, dWB, dY, dG;
    dX.alloc(X.size() * sizeof(float), st);
    dT.alloc(T.size() * sizeof(float), st);
    dWB.alloc(WB.size() * sizeof(float), st);
    dY.alloc((size_t)8 * N * sizeof(float), st);
    dG.alloc(nw * sizeof(float), st);
    CUDA_CHECK(cudaMemcpyAsync(dX.p, X.data(), X.size() * sizeof(float), cudaMemcpyHostToDevice, st));
    CUDA_CHECK(cudaMemcpyAsync(dT.p, T.data(), T.size() * sizeof(float), cudaMemcpyHostToDevice, st));
    CUDA_CHECK(cudaMemcpyAsync(dWB.p, WB.data(), WB.size() * sizeof(float), cudaMemcpyHostToDevice, st));
    h->d_gnn_m.alloc(nw * sizeof(float), st);
    h->d_gnn_v.alloc(nw * sizeof(float), st);
    CUDA_CHECK(cudaMemsetAsync(h->d_gnn_m.p, 0, nw * sizeof(float), st));
    CUDA_CHECK(cudaMemsetAsync(h->d_gnn_v.p, 0, nw * sizeof(float), st));
    double first = -1.0, last = 0.0;
    int step = 0;
    for (int ep = 0; ep < epochs; ++ep) {
      double ep_loss = 0.0;
      for (int b0 = 0; b0 < S; b0 += 8) {
        const int B = std::min(8, S - b0);
        const double L = gnn_pass(h, B, dX.as<float>() + (int64_t)b0 * N,
                                  dT.as<float>() + (int64_t)b0 * N, dWB.as<float>() + b0,
                                  dY.as<float>(), dG.as<float>());
        ++step;
        k_adam<<<(unsigned)ceil_div(nw, 256), 256, 0, st>>>(
            h->d_gnn_w.as<float>(), dG.as<float>(), h->d_gnn_m.as<float>(),
            h->d_gnn_v.as<float>(), nw, (float)lr, powf(0.9f, (float)step),
            powf(0.999f, (float)step));
        count_launch(h);
        ep_loss += L * B;
      }
      ep_loss /= S;
      if (first < 0) first = ep_loss;
      last = ep_loss;
    }
    check_launch("gnn train");
    if (loss2) {
      loss2[0] = first;
      loss2[1] = last;
    }
    h->gnn_trained = true;
    return ELMFB_OK;
  } catch (const elmfb_error& e) {
    h->err = e.msg;
    return e.code;
  } catch (const std::bad_alloc&) {
    h->err = "host allocation failed";
    return ELMFB_ERR_OOM;
  } catch (const std::exception& e) {
    h->err = e.what();
    return ELMFB_ERR_CUDA;
  }
}

}  // extern "C"
