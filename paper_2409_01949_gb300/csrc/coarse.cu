// Coarse-level correction of the block-Jacobi preconditioner (not in the
// paper; its multilevel structure, §3, motivates it).
//
// The columns of the coarse levels 1..l_c (the first N_c = K sum_{l<=l_c} J_l
// columns) form one block: G_c = M_c^T M_c, their joint Gram, couples every
// pair of coarse subdomains, where block-Jacobi keeps only each subdomain's own
// K x K block.  The preconditioner of FCG on M^T M a = M^T h then applies, to
// the coarse part of the residual, the inverse of the shifted joint block,
//     z_c = X_c^T X_c r_c,   X_c = L_c^{-1},  L_c L_c^T = G_c + eps tr(G_c)/N_c I,
// and block-Jacobi (X_j^T X_j r_j) to every finer subdomain.
//
// Set-up (once per solve): column q of G_c is the coarse part of M^T M e_q,
// from the same fused pass that applies the normal operator in FCG, so the
// joint block is exactly the operator the iteration sees; then a right-looking
// FP64 Cholesky with the shift (raised 100-fold on a non-positive pivot, up to
// six times) and the explicit lower inverse X_c, both in one block (N_c is a
// few hundred).  Application: two FP64 triangular products, a warp per output
// entry.
#include <algorithm>
#include <cmath>

#include "elmfb_internal.cuh"

namespace {

__global__ void k_unit(double* __restrict__ v, int64_t n, int64_t q) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    v[i] = i == q ? 1.0 : 0.0;
}

// column q of G (n x n, column-major = row-major by symmetry) from y[0:n]
__global__ void k_copy_col(const double* __restrict__ y, int n, int q, double* __restrict__ G) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
    G[(int64_t)q * n + i] = y[i];
}

__device__ double block_sum_c(double v, double* sh) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  __syncthreads();
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = v;
  __syncthreads();
  if (threadIdx.x < 32) {
    double s = threadIdx.x < (blockDim.x >> 5) ? sh[threadIdx.x] : 0.0;
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (threadIdx.x == 0) sh[32] = s;
  }
  __syncthreads();
  const double r = sh[32];
  __syncthreads();
  return r;
}

// Shifted Cholesky of the symmetric G (n x n) into W (lower, row-major), then
// X = W^{-1} (lower, row-major).  One block.  flags[0] = failed after all
// retries, flags[1] = retries taken.
__global__ void __launch_bounds__(1024) k_coarse_chol_inv(const double* __restrict__ G, int n,
                                                         double shift, double* __restrict__ W,
                                                         double* __restrict__ X,
                                                         int* __restrict__ flags) {
  __shared__ double red[33];
  __shared__ int bad;
  // symmetrise (the two triangles of M^T M e_q agree to rounding) and trace
  double tr = 0.0;
  for (int i = threadIdx.x; i < n; i += blockDim.x) tr += G[(int64_t)i * n + i];
  tr = block_sum_c(tr, red);
  double eps = shift * tr / n;
  int retries = 0;
  for (int attempt = 0; attempt < 7; ++attempt) {
    for (int64_t idx = threadIdx.x; idx < (int64_t)n * n; idx += blockDim.x) {
      const int i = (int)(idx / n), j = (int)(idx % n);
      W[idx] = j <= i ? 0.5 * (G[(int64_t)i * n + j] + G[(int64_t)j * n + i]) + (i == j ? eps : 0.0)
                      : 0.0;
    }
    if (threadIdx.x == 0) bad = 0;
    __syncthreads();
    for (int k = 0; k < n && !bad; ++k) {
      __shared__ double lkk;
      if (threadIdx.x == 0) {
        const double d = W[(int64_t)k * n + k];
        if (!(d > 0.0)) bad = 1;
        lkk = d > 0.0 ? sqrt(d) : 1.0;
        W[(int64_t)k * n + k] = lkk;
      }
      __syncthreads();
      if (bad) break;
      const double il = 1.0 / lkk;
      for (int i = k + 1 + threadIdx.x; i < n; i += blockDim.x) W[(int64_t)i * n + k] *= il;
      __syncthreads();
      // trailing update of the lower triangle, rows and columns > k
      const int m = n - k - 1;
      for (int64_t t = threadIdx.x; t < (int64_t)m * m; t += blockDim.x) {
        const int i = k + 1 + (int)(t / m), j = k + 1 + (int)(t % m);
        if (j <= i) W[(int64_t)i * n + j] -= W[(int64_t)i * n + k] * W[(int64_t)j * n + k];
      }
      __syncthreads();
    }
    if (!bad) break;
    ++retries;
    eps = eps > 0.0 ? eps * 100.0 : 1e-14 * tr / n;
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    flags[0] = bad;
    flags[1] = retries;
  }
  if (bad) return;
  // X = L^{-1}: column j by one thread, rows in order (X[i][j] needs X[k][j], k < i)
  for (int j = threadIdx.x; j < n; j += blockDim.x) {
    for (int i = 0; i < j; ++i) X[(int64_t)i * n + j] = 0.0;
    X[(int64_t)j * n + j] = 1.0 / W[(int64_t)j * n + j];
    for (int i = j + 1; i < n; ++i) {
      double s = 0.0;
      for (int k = j; k < i; ++k) s = fma(W[(int64_t)i * n + k], X[(int64_t)k * n + j], s);
      X[(int64_t)i * n + j] = -s / W[(int64_t)i * n + i];
    }
  }
}

// y = X r (trans = 0) or y = X^T r (trans = 1), X lower triangular row-major
// n x n; a warp per output entry, fixed-order lane sums.
__global__ void k_tri_mv(const double* __restrict__ X, int n, const double* __restrict__ r,
                         double* __restrict__ y, int trans) {
  const int lane = threadIdx.x & 31;
  const int w = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int nw = (gridDim.x * blockDim.x) >> 5;
  for (int i = w; i < n; i += nw) {
    double s = 0.0;
    if (!trans) {
      for (int k = lane; k <= i; k += 32) s = fma(X[(int64_t)i * n + k], r[k], s);
    } else {
      for (int k = i + lane; k < n; k += 32) s = fma(X[(int64_t)k * n + i], r[k], s);
    }
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (lane == 0) y[i] = s;
  }
}

}  // namespace

int coarse_columns(const elmfb_ctx* h, int levels) {
  if (levels < 1 || levels > h->L) ELMFB_THROW(ELMFB_ERR_INVALID_ARG, "coarse_levels out of range");
  return h->lev_sub_off[levels] * h->K;
}

// Joint coarse block: G_c from `normal_op` on unit vectors, then X_c.
void coarse_setup(elmfb_ctx* h, int levels, double shift,
                  const std::function<void(const double*, double*)>& normal_op,
                  DevBuf& X, int* retries) {
  cudaStream_t st = h->stream;
  const int n = coarse_columns(h, levels);
  if (n > 4096) ELMFB_THROW(ELMFB_ERR_UNSUPPORTED, "coarse block above 4096 columns");
  const int64_t N = h->NPhi;
  DevBuf e, y, G, W, fl;
  e.alloc(N * sizeof(double), st);
  y.alloc(N * sizeof(double), st);
  G.alloc((size_t)n * n * sizeof(double), st);
  W.alloc((size_t)n * n * sizeof(double), st);
  X.alloc((size_t)n * n * sizeof(double), st);
  fl.alloc(2 * sizeof(int), st);
  const unsigned nb = (unsigned)std::min<int64_t>(ceil_div(N, 256), 1216);
  for (int q = 0; q < n; ++q) {
    k_unit<<<nb, 256, 0, st>>>(e.as<double>(), N, q);
    normal_op(e.as<double>(), y.as<double>());
    k_copy_col<<<(unsigned)ceil_div(n, 256), 256, 0, st>>>(y.as<double>(), n, q, G.as<double>());
    count_launch(h, 2);
  }
  check_launch("coarse Gram");
  k_coarse_chol_inv<<<1, 1024, 0, st>>>(G.as<double>(), n, shift, W.as<double>(), X.as<double>(),
                                        fl.as<int>());
  count_launch(h);
  check_launch("k_coarse_chol_inv");
  int flags[2];
  CUDA_CHECK(cudaMemcpyAsync(flags, fl.p, sizeof(flags), cudaMemcpyDeviceToHost, st));
  stream_sync(h);
  if (flags[0]) ELMFB_THROW(ELMFB_ERR_BREAKDOWN, "coarse block Cholesky failed after shift increases");
  if (retries) *retries = flags[1];
}

// z[0:n] = X^T X r[0:n]  (the block-Jacobi part of the coarse columns replaced)
void coarse_apply(elmfb_ctx* h, const DevBuf& X, int n, const double* r, double* z, DevBuf& tmp) {
  cudaStream_t st = h->stream;
  tmp.alloc((size_t)n * sizeof(double), st);
  const unsigned blocks = (unsigned)std::min(ceil_div((int64_t)n * 32, 256), (int64_t)608);
  k_tri_mv<<<blocks, 256, 0, st>>>(X.as<double>(), n, r, tmp.as<double>(), 0);
  k_tri_mv<<<blocks, 256, 0, st>>>(X.as<double>(), n, tmp.as<double>(), z, 1);
  count_launch(h, 2);
  check_launch("coarse apply");
}
