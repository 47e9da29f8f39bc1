// Model evaluation and error norms.
//
// u_hat(x) = (1/L) sum_l sum_j w_j(x) sum_k a_ljk phi_ljk(x)   (paper Eq.
// multilevel_solution), evaluated in FP64: one warp per point.  Lane j forms
// the window of covering subdomain j, the lanes then share the features of
// each covering subdomain.  The covering subdomains of a point are
// those of its cell (the common refinement of all supports).
//
// Error norms (paper Eq. l1_error): e_L1 = sum |u_hat - u| / (M std(u)) with
// the population standard deviation, plus the relative L2 error and the max
// error; fixed-order two-stage reductions in FP64.
#include <algorithm>
#include <cmath>

#include "elmfb_internal.cuh"

namespace {

__device__ __forceinline__ double warp_sum_d(double v) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// 1-D window factor [1 + cos(pi dx / sigma)]^2 = 4 cos^4(pi dx / (2 sigma)) on the
// open support |dx| < sigma; near the edge cos(theta/2) = sin(pi u / 2) with
// u = (sigma - |dx|) / sigma.
__device__ __forceinline__ double factor(double dx, double sigma, double inv_sigma) {
  const double adx = fabs(dx);
  if (!(adx < sigma)) return 0.0;
  const double u = (sigma - adx) * inv_sigma;
  const double c = u < 0.5 ? sinpi(0.5 * u) : cospi(0.5 * dx * inv_sigma);
  const double c2 = c * c;
  return 4.0 * c2 * c2;
}

// the hard-constraint factor A(x) of paper §4.3 (1 without the ansatz)
__device__ __forceinline__ double ansatz_value(const Ansatz& an, const double* x, int dim) {
  if (!(an.w > 0.0)) return 1.0;
  double A, dA[2], ddA[2];
  ansatz_at(an, x, dim, A, dA, ddA);
  return A;
}

__global__ void __launch_bounds__(256) k_eval(const double* __restrict__ xs, int64_t n, int dim,
                                              int K, int L, const double* __restrict__ bnd,
                                              int nc0, int nc1, const SubGeom* __restrict__ sub,
                                              const int* __restrict__ cell_level_off,
                                              const int* __restrict__ cover_sub,
                                              const double* __restrict__ W,
                                              const double* __restrict__ B,
                                              const double* __restrict__ a,
                                              double* __restrict__ out, const Ansatz an) {
  const int lane = threadIdx.x & 31;
  const int64_t pt = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  if (pt >= n) return;
  double x[2] = {xs[pt * dim], dim == 2 ? xs[pt * dim + 1] : 0.0};
  // cell of the point
  int c[2] = {0, 0};
  const int ncs[2] = {nc0, nc1};
  const double* bb = bnd;
  for (int i = 0; i < dim; ++i) {
    int lo = 0, hi = ncs[i];
    while (hi - lo > 1) {
      int mid = (lo + hi) >> 1;
      if (bb[mid] <= x[i]) lo = mid;
      else hi = mid;
    }
    c[i] = lo;
    bb += ncs[i] + 1;
  }
  const int cell = c[1] * nc0 + c[0];
  const int e0 = cell_level_off[(int64_t)cell * (L + 1)];
  const int m = cell_level_off[(int64_t)cell * (L + 1) + L] - e0;
  if (m <= 32) {
    // lane j takes covering entry e0 + j: its window factor (FP64 sin/cos, so
    // once per entry instead of once per lane and entry) and scaled input
    double wj = 0.0, xj[2] = {0.0, 0.0};
    int lvl = -1, sj = 0;
    if (lane < m) {
      sj = cover_sub[e0 + lane];
      const SubGeom g = sub[sj];
      lvl = g.level;
      wj = 1.0;
      for (int i = 0; i < dim; ++i) {
        xj[i] = (x[i] - g.mu[i]) * g.inv_sigma_d[i];
        wj *= factor(x[i] - g.mu[i], g.sigma_d[i], g.inv_sigma_d[i]);
      }
    }
    // partition of unity per level: S_l = sum of the level's factors
    double Sj = 0.0;
    for (int l = 0; l < L; ++l) {
      const double S = warp_sum_d(lvl == l ? wj : 0.0);
      if (lvl == l) Sj = S;
    }
    const double cj = (Sj > 0.0 && wj != 0.0) ? wj / Sj : 0.0;
    // each lane sums its features over the entries; one reduction at the end
    double acc = 0.0;
    for (int j = 0; j < m; ++j) {
      const double cw = __shfl_sync(0xffffffffu, cj, j);
      if (cw == 0.0) continue;   // warp-uniform
      const int s = __shfl_sync(0xffffffffu, sj, j);
      const double x0 = __shfl_sync(0xffffffffu, xj[0], j);
      const double x1 = __shfl_sync(0xffffffffu, xj[1], j);
      for (int f = lane; f < K; f += 32) {
        const int64_t q = (int64_t)s * K + f;
        const double arg = W[q * dim] * x0 + (dim == 2 ? W[q * dim + 1] * x1 : 0.0) + B[q];
        acc += cw * (a[q] * tanh(arg));
      }
    }
    const double total = warp_sum_d(acc);
    if (lane == 0) out[pt] = total / L * ansatz_value(an, x, dim);
    return;
  }
  double total = 0.0;   // more than 32 covering subdomains: entry by entry
  for (int l = 0; l < L; ++l) {
    const int b = cell_level_off[(int64_t)cell * (L + 1) + l];
    const int e = cell_level_off[(int64_t)cell * (L + 1) + l + 1];
    double S = 0.0;
    for (int k = b; k < e; ++k) {
      const SubGeom g = sub[cover_sub[k]];
      double w = 1.0;
      for (int i = 0; i < dim; ++i) w *= factor(x[i] - g.mu[i], g.sigma_d[i], g.inv_sigma_d[i]);
      S += w;
    }
    if (!(S > 0.0)) continue;
    for (int k = b; k < e; ++k) {
      const int s = cover_sub[k];
      const SubGeom g = sub[s];
      double w = 1.0, xt[2] = {0.0, 0.0};
      for (int i = 0; i < dim; ++i) {
        xt[i] = (x[i] - g.mu[i]) * g.inv_sigma_d[i];
        w *= factor(x[i] - g.mu[i], g.sigma_d[i], g.inv_sigma_d[i]);
      }
      if (w == 0.0) continue;
      double part = 0.0;
      for (int f = lane; f < K; f += 32) {
        const int64_t q = (int64_t)s * K + f;
        double arg = W[q * dim] * xt[0] + (dim == 2 ? W[q * dim + 1] * xt[1] : 0.0) + B[q];
        part += a[q] * tanh(arg);
      }
      part = warp_sum_d(part);
      total += (w / S) * part;
    }
  }
  if (lane == 0) out[pt] = total / L * ansatz_value(an, x, dim);
}

// pass 1: sum u, sum |d|, sum d^2, sum u^2, max |d|  (per block)
__global__ void k_err_pass1(const double* __restrict__ uh, const double* __restrict__ ur,
                            int64_t n, double* __restrict__ part) {
  __shared__ double sh[5][32];
  double su = 0, sad = 0, sd2 = 0, su2 = 0, mx = 0;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    double d = uh[i] - ur[i];
    su += ur[i];
    sad += fabs(d);
    sd2 += d * d;
    su2 += ur[i] * ur[i];
    mx = fmax(mx, fabs(d));
  }
  double v[5] = {su, sad, sd2, su2, mx};
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  for (int k = 0; k < 5; ++k) {
    double t = v[k];
    for (int o = 16; o > 0; o >>= 1) {
      double y = __shfl_xor_sync(0xffffffffu, t, o);
      t = k == 4 ? fmax(t, y) : t + y;
    }
    if (lane == 0) sh[k][wid] = t;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int k = 0; k < 5; ++k) {
      double t = 0.0;
      for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t = k == 4 ? fmax(t, sh[k][w]) : t + sh[k][w];
      part[blockIdx.x * 5 + k] = t;
    }
  }
}

// pass 2: sum (u - mean)^2 per block
__global__ void k_err_pass2(const double* __restrict__ ur, int64_t n,
                            const double* __restrict__ part1, int nb, double* __restrict__ part2) {
  __shared__ double sh[32];
  double su = 0.0;
  for (int b = 0; b < nb; ++b) su += part1[b * 5 + 0];
  const double mean = su / (double)n;
  double acc = 0.0;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    double d = ur[i] - mean;
    acc += d * d;
  }
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += sh[w];
    part2[blockIdx.x] = t;
  }
}

}  // namespace

void eval_model(elmfb_ctx* h, const double* xs, int64_t n, double* out) {
  if (n == 0) return;
  cudaStream_t st = h->stream;
  stage_begin(h, 6);
  DevBuf dx, dout;
  dx.alloc(n * h->dim * sizeof(double), st);
  dout.alloc(n * sizeof(double), st);
  CUDA_CHECK(cudaMemcpyAsync(dx.p, xs, n * h->dim * sizeof(double), cudaMemcpyDefault, st));
  const int64_t threads = n * 32;
  k_eval<<<(unsigned)ceil_div(threads, 256), 256, 0, st>>>(
      dx.as<double>(), n, h->dim, h->K, h->L, h->d_bnd.as<double>(), h->nc[0], h->nc[1],
      h->d_sub.as<SubGeom>(), h->d_cell_level_off.as<int>(), h->d_cover_sub.as<int>(),
      h->d_W64.as<double>(), h->d_b64.as<double>(), h->d_a.as<double>(), dout.as<double>(),
      make_ansatz(h->cfg));
  check_launch("k_eval");
  count_launch(h);
  CUDA_CHECK(cudaMemcpyAsync(out, dout.p, n * sizeof(double), cudaMemcpyDefault, st));
  stage_end(h, 6);
}

void error_norms(elmfb_ctx* h, const double* uh, const double* ur, int64_t n, double* out3) {
  cudaStream_t st = h->stream;
  const int nb = (int)std::min<int64_t>(ceil_div(n, 256), 256);
  DevBuf du, dr, p1, p2;
  du.alloc(n * sizeof(double), st);
  dr.alloc(n * sizeof(double), st);
  p1.alloc(nb * 5 * sizeof(double), st);
  p2.alloc(nb * sizeof(double), st);
  CUDA_CHECK(cudaMemcpyAsync(du.p, uh, n * sizeof(double), cudaMemcpyDefault, st));
  CUDA_CHECK(cudaMemcpyAsync(dr.p, ur, n * sizeof(double), cudaMemcpyDefault, st));
  k_err_pass1<<<nb, 256, 0, st>>>(du.as<double>(), dr.as<double>(), n, p1.as<double>());
  k_err_pass2<<<nb, 256, 0, st>>>(dr.as<double>(), n, p1.as<double>(), nb, p2.as<double>());
  check_launch("k_err");
  count_launch(h, 2);
  std::vector<double> a(nb * 5), b(nb);
  CUDA_CHECK(cudaMemcpyAsync(a.data(), p1.p, nb * 5 * sizeof(double), cudaMemcpyDeviceToHost, st));
  CUDA_CHECK(cudaMemcpyAsync(b.data(), p2.p, nb * sizeof(double), cudaMemcpyDeviceToHost, st));
  stream_sync(h);
  double sad = 0, sd2 = 0, su2 = 0, mx = 0, var = 0;
  for (int i = 0; i < nb; ++i) {
    sad += a[i * 5 + 1];
    sd2 += a[i * 5 + 2];
    su2 += a[i * 5 + 3];
    mx = std::max(mx, a[i * 5 + 4]);
    var += b[i];
  }
  const double sd = std::sqrt(var / (double)n);
  out3[0] = su2 > 0.0 ? std::sqrt(sd2 / su2) : NAN;
  out3[1] = sd > 0.0 ? sad / ((double)n * sd) : NAN;
  out3[2] = mx;
}
