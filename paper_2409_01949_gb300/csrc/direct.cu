// Dense least-squares solve of min ||M a - h|| (paper Eq. multilevel_ls) by
// Householder QR with column pivoting (Businger & Golub 1965), for systems
// whose dense M fits in device memory.
//
// The paper reaches the least-squares minimiser with LSQR (§3, §4.1); M is
// numerically rank deficient (the paper's tables report condition numbers up
// to ~1e20), and the accurate minimisers use singular directions far below
// what an iterative solve resolves in a few thousand iterations.  This path
// computes the basic solution of the rank-revealing factorisation instead:
//   step k: take the remaining column of largest norm over rows k..; stop once
//   that norm is <= rcond |R_11| (rank = k); else swap it into place, form the
//   reflector H = I - 2 v v^T / (v^T v), v = x - beta e_1, beta = -sign(x_1)||x||
//   (so R_kk = beta), apply it to every later column and to h, and recompute
//   the later columns' norms over rows k+1.. exactly (no downdating).
// Then R z = (Q^T h)[0:rank] by back substitution and a[perm[i]] = z[i].
// ||(Q^T h)[rank:]|| is the least-squares residual norm.
//
// Layout: A is column-major FP64 [ld x (n+1)], ld >= m = the padded sorted
// rows (padding rows are zero rows and change nothing), column n = h.  One
// step is two kernels: k_qr_house (one block: pivot swap, reflector) and
// k_qr_apply (a warp per column: v^T A_j, the update, the new norm, and the
// arg-max of the norms for the next step, finished by the last block).  The
// update is FP64-bound: three FP64 FMAs per trailing entry and step.
#include <algorithm>
#include <cmath>

#include "elmfb_internal.cuh"

namespace {

constexpr int kApplyThreads = 256;   // 8 warps, a warp per column
constexpr int kHouseThreads = 1024;
constexpr int kQrBatch = 32;         // steps launched between host checks of the stop flag

struct QrState {
  int piv;       // pivot column of the next step
  int stop;      // the rank cut was met
  int rank;      // steps taken
  int pad_;
  double cmax;   // squared norm of the pivot column over the remaining rows
  double r11;    // |R_11|
  double c;      // 2 / v^T v of the current reflector
  double bad;    // non-finite norm seen
};

__device__ __forceinline__ double warp_sum_d(double v) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// larger norm wins; equal norms: the smaller column index (the first maximum)
__device__ __forceinline__ bool better(double v, int i, double bv, int bi) {
  return v > bv || (v == bv && bi >= 0 && i < bi) || (bi < 0 && i >= 0);
}

__device__ double block_sum_d(double v, double* sh) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
  v = warp_sum_d(v);
  __syncthreads();
  if (lane == 0) sh[wid] = v;
  __syncthreads();
  if (wid == 0) {
    double s = lane < nw ? sh[lane] : 0.0;
    s = warp_sum_d(s);
    if (lane == 0) sh[32] = s;
  }
  __syncthreads();
  const double r = sh[32];
  __syncthreads();
  return r;
}

__device__ __forceinline__ double value_of(float v) { return (double)v; }
__device__ __forceinline__ double value_of(double v) { return v; }
__device__ __forceinline__ double value_of(df2 v) { return (double)v.hi + (double)v.lo; }

// Panels (cell-interleaved: row p of entry e at element row entry_base[e] +
// p m_c) -> dense column-major A.  A warp per assembly tile (entry, 32 rows):
// rows are read K-contiguous, staged in shared memory, written column-wise.
template <class T>
__global__ void __launch_bounds__(128) k_qr_densify(
    const int2* __restrict__ tiles, int64_t n_tiles, int K, const int* __restrict__ entry_cell,
    const int* __restrict__ cover_sub, const int* __restrict__ cover_off,
    const int* __restrict__ cell_pstart, const int64_t* __restrict__ entry_base,
    const T* __restrict__ panels, double* __restrict__ A, int64_t ld) {
  __shared__ double sh[4][32][33];
  const int lane = threadIdx.x & 31, wq = threadIdx.x >> 5;
  const int64_t t = (int64_t)blockIdx.x * 4 + wq;
  if (t >= n_tiles) return;
  const int2 tile = tiles[t];
  const int e = tile.x, p0 = tile.y;
  const int c = entry_cell[e];
  const int s = cover_sub[e];
  const int pad = cell_pstart[c + 1] - cell_pstart[c];
  const int nrows = min(32, pad - p0);
  const int64_t R0 = cell_pstart[c] + p0;
  const int64_t rstride = (int64_t)(cover_off[c + 1] - cover_off[c]) * K;
  const T* src = panels + entry_base[e] * (int64_t)K + (int64_t)p0 * rstride;
  for (int kc = 0; kc < K; kc += 32) {
    for (int r = 0; r < nrows; ++r)
      sh[wq][r][lane] = kc + lane < K ? value_of(src[(int64_t)r * rstride + kc + lane]) : 0.0;
    __syncwarp();
    const int kn = min(32, K - kc);
    for (int kk = 0; kk < kn; ++kk)
      if (lane < nrows) A[((int64_t)s * K + kc + kk) * ld + R0 + lane] = sh[wq][lane][kk];
    __syncwarp();
  }
}

__global__ void k_qr_copy_h(const double* __restrict__ hv, int64_t m, double* __restrict__ col) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < m;
       i += (int64_t)gridDim.x * blockDim.x)
    col[i] = hv[i];
}

// The block's best (norm, column) into part[blockIdx]; the last block to
// finish reduces all partials (the order does not matter: "better" is a total
// order) into the state.  `lo` is the first candidate column.
__device__ void argmax_finish(double bv, int bi, double* __restrict__ part_v,
                              int* __restrict__ part_i, unsigned int* __restrict__ counter,
                              QrState* st, int lo) {
  __shared__ double sv[32];
  __shared__ int si[32];
  __shared__ bool last;
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
  if (lane == 0) {
    sv[wid] = bv;
    si[wid] = bi;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double v = -1.0;
    int i = -1;
    for (int w = 0; w < nw; ++w)
      if (better(sv[w], si[w], v, i)) {
        v = sv[w];
        i = si[w];
      }
    part_v[blockIdx.x] = v;
    part_i[blockIdx.x] = i;
    __threadfence();
    last = atomicAdd(counter, 1u) == gridDim.x - 1;
  }
  __syncthreads();
  if (!last) return;
  if (wid == 0) {
    double v = -1.0;
    int i = -1;
    for (int b = lane; b < (int)gridDim.x; b += 32) {
      const double pv = __ldcg(part_v + b);
      const int pi = __ldcg(part_i + b);
      if (better(pv, pi, v, i)) {
        v = pv;
        i = pi;
      }
    }
    for (int o = 16; o > 0; o >>= 1) {
      const double ov = __shfl_xor_sync(0xffffffffu, v, o);
      const int oi = __shfl_xor_sync(0xffffffffu, i, o);
      if (better(ov, oi, v, i)) {
        v = ov;
        i = oi;
      }
    }
    if (lane == 0) {
      st->piv = i >= 0 ? i : lo;
      st->cmax = i >= 0 ? v : 0.0;
      if (!(v == v) || isinf(v)) st->bad = 1.0;
      *counter = 0u;
    }
  }
}

// squared column norms over all rows, and their arg-max (the first pivot)
__global__ void __launch_bounds__(kApplyThreads) k_qr_colnorms(
    const double* __restrict__ A, int64_t ld, int64_t m, int n, double* __restrict__ cn,
    double* __restrict__ part_v, int* __restrict__ part_i, unsigned int* __restrict__ counter,
    QrState* st) {
  const int lane = threadIdx.x & 31;
  const int gw = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  const int nwarps = gridDim.x * (blockDim.x >> 5);
  double bv = -1.0;
  int bi = -1;
  for (int j = gw; j < n; j += nwarps) {
    const double* col = A + (int64_t)j * ld;
    double s = 0.0;
    for (int64_t i = lane; i < m; i += 32) s = fma(col[i], col[i], s);
    s = warp_sum_d(s);
    if (lane == 0) cn[j] = s;
    if (better(s, j, bv, bi)) {
      bv = s;
      bi = j;
    }
  }
  argmax_finish(bv, bi, part_v, part_i, counter, st, 0);
}

// Step k, part 1: pivot swap and the Householder reflector of column k.
__global__ void __launch_bounds__(kHouseThreads) k_qr_house(
    double* __restrict__ A, int64_t ld, int64_t m, int k, double* __restrict__ cn,
    int* __restrict__ perm, double* __restrict__ vbuf, QrState* __restrict__ st, double rcond) {
  __shared__ double red[33];
  __shared__ int s_go, s_j;
  if (threadIdx.x == 0) {
    int go = !st->stop;
    if (go) {
      const int j = st->piv;
      const double cj = st->cmax;
      if (k == 0) st->r11 = sqrt(cj);
      if (st->bad != 0.0 || !(cj > 0.0) || sqrt(cj) <= rcond * st->r11) {
        st->stop = 1;
        st->rank = k;
        go = 0;
      } else {
        s_j = j;
        if (j != k) {
          cn[j] = cn[k];
          const int t = perm[j];
          perm[j] = perm[k];
          perm[k] = t;
        }
      }
    }
    s_go = go;
  }
  __syncthreads();
  if (!s_go) return;
  const int j = s_j;
  double* ck = A + (int64_t)k * ld;
  if (j != k) {
    double* cj = A + (int64_t)j * ld;
    for (int64_t i = threadIdx.x; i < m; i += blockDim.x) {
      const double t = ck[i];
      ck[i] = cj[i];
      cj[i] = t;
    }
    __syncthreads();
  }
  double s1 = 0.0;
  for (int64_t i = k + 1 + threadIdx.x; i < m; i += blockDim.x) {
    const double x = ck[i];
    s1 = fma(x, x, s1);
    vbuf[i] = x;
  }
  s1 = block_sum_d(s1, red);
  if (threadIdx.x == 0) {
    const double alpha = ck[k];
    const double beta = -copysign(sqrt(fma(alpha, alpha, s1)), alpha);
    const double v0 = alpha - beta;
    vbuf[k] = v0;
    ck[k] = beta;
    st->c = 2.0 / fma(v0, v0, s1);
    st->rank = k + 1;
    if (!(beta == beta) || isinf(beta)) st->bad = 1.0;
  }
}

// Step k, part 2: A_j -= c (v^T A_j) v for every later column j (h included),
// the new squared norms over rows k+1.., and their arg-max.
__global__ void __launch_bounds__(kApplyThreads) k_qr_apply(
    double* __restrict__ A, int64_t ld, int64_t m, int n, int k, const double* __restrict__ vbuf,
    QrState* st, double* __restrict__ cn, double* __restrict__ part_v, int* __restrict__ part_i,
    unsigned int* __restrict__ counter) {
  if (st->stop) return;
  const double c = st->c;
  const int lane = threadIdx.x & 31;
  const int gw = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  const int nwarps = gridDim.x * (blockDim.x >> 5);
  double bv = -1.0;
  int bi = -1;
  for (int j = k + 1 + gw; j <= n; j += nwarps) {
    double* col = A + (int64_t)j * ld;
    double s0 = 0.0, s1 = 0.0;
    int64_t i = k + lane;
    for (; i + 32 < m; i += 64) {
      s0 = fma(vbuf[i], col[i], s0);
      s1 = fma(vbuf[i + 32], col[i + 32], s1);
    }
    if (i < m) s0 = fma(vbuf[i], col[i], s0);
    const double s = warp_sum_d(s0 + s1) * c;
    double n0 = 0.0, n1 = 0.0;
    i = k + lane;
    for (; i + 32 < m; i += 64) {
      const double a0 = fma(-s, vbuf[i], col[i]);
      const double a1 = fma(-s, vbuf[i + 32], col[i + 32]);
      col[i] = a0;
      col[i + 32] = a1;
      if (i > k) n0 = fma(a0, a0, n0);
      n1 = fma(a1, a1, n1);
    }
    if (i < m) {
      const double a0 = fma(-s, vbuf[i], col[i]);
      col[i] = a0;
      if (i > k) n0 = fma(a0, a0, n0);
    }
    if (j < n) {
      const double nr = warp_sum_d(n0 + n1);
      if (lane == 0) {
        cn[j] = nr;
        if (!(nr == nr)) st->bad = 1.0;
      }
      if (better(nr, j, bv, bi)) {
        bv = nr;
        bi = j;
      }
    }
  }
  argmax_finish(bv, bi, part_v, part_i, counter, st, k + 1);
}

// R z = (Q^T h)[0:r] by back substitution, column by column (R's columns are
// contiguous); res2 = ||(Q^T h)[r:m]||^2, the squared least-squares residual.
__global__ void __launch_bounds__(1024) k_qr_backsub(const double* __restrict__ A, int64_t ld,
                                                     int64_t m, int n, const QrState* __restrict__ st,
                                                     double* __restrict__ y, double* __restrict__ z,
                                                     double* __restrict__ res2) {
  __shared__ double red[33];
  __shared__ double zj;
  const int r = st->rank;
  const double* hc = A + (int64_t)n * ld;
  double s = 0.0;
  for (int64_t i = r + threadIdx.x; i < m; i += blockDim.x) s = fma(hc[i], hc[i], s);
  s = block_sum_d(s, red);
  if (threadIdx.x == 0) *res2 = s;
  for (int i = threadIdx.x; i < r; i += blockDim.x) y[i] = hc[i];
  __syncthreads();
  for (int j = r - 1; j >= 0; --j) {
    const double* cj = A + (int64_t)j * ld;
    if (threadIdx.x == 0) {
      zj = y[j] / cj[j];
      z[j] = zj;
    }
    __syncthreads();
    const double zz = zj;
    for (int i = threadIdx.x; i < j; i += blockDim.x) y[i] = fma(-cj[i], zz, y[i]);
    __syncthreads();
  }
}

__global__ void k_qr_scatter(const double* __restrict__ z, const int* __restrict__ perm,
                             const QrState* __restrict__ st, double* __restrict__ a) {
  const int r = st->rank;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < r; i += gridDim.x * blockDim.x)
    a[perm[i]] = z[i];
}

__global__ void k_qr_iota(int* __restrict__ perm, int n) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
    perm[i] = i;
}

template <class T>
void densify(elmfb_ctx* h, const void* panels, double* A, int64_t ld) {
  ensure_qr_tiles(h);
  const int64_t blocks = ceil_div(h->n_tiles, 4);
  if (blocks > 0)
    k_qr_densify<T><<<(unsigned)blocks, 128, 0, h->stream>>>(
        h->d_tiles.as<int2>(), h->n_tiles, h->K, h->d_entry_cell.as<int>(),
        h->d_cover_sub.as<int>(), h->d_cover_off.as<int>(), h->d_cell_pstart.as<int>(),
        h->d_entry_base.as<int64_t>(), (const T*)panels, A, ld);
  check_launch("k_qr_densify");
  count_launch(h);
}

}  // namespace

void qr_solve(elmfb_ctx* h, const elmfb_solve_opts* o, elmfb_solve_info* info) {
  cudaStream_t st = h->stream;
  const int64_t m = h->NR;
  const int64_t N = h->NPhi;
  if (N + 1 > (int64_t)1 << 30) ELMFB_THROW(ELMFB_ERR_UNSUPPORTED, "QR: too many columns");
  const int n = (int)N;
  const int64_t ld = (m + 3) & ~int64_t(3);
  const double bytes = 8.0 * (double)ld * (double)(n + 1);
  size_t free_b = 0, total_b = 0;
  CUDA_CHECK(cudaMemGetInfo(&free_b, &total_b));
  if (bytes > 0.8 * (double)free_b)
    ELMFB_THROW(ELMFB_ERR_UNSUPPORTED,
                "QR: the dense matrix (" + std::to_string(bytes / 1e9) +
                    " GB) does not fit in free device memory; use LSQR");
  if (!(o->rcond >= 0.0)) ELMFB_THROW(ELMFB_ERR_INVALID_ARG, "QR: rcond must be >= 0");

  stage_begin(h, 5);
  DevBuf dA, dcn, dperm, dv, dstate, dpv, dpi, dcnt, dy, dz, dres;
  dA.alloc((size_t)bytes, st);
  double* A = dA.as<double>();
  CUDA_CHECK(cudaMemsetAsync(A, 0, (size_t)bytes, st));
  if (h->df32()) densify<df2>(h, h->d_panels.p, A, ld);
  else if (h->dual()) densify<df2>(h, h->d_panels_df.p, A, ld);   // the pair panels
  else if (h->fp64()) densify<double>(h, h->d_panels.p, A, ld);
  else densify<float>(h, h->d_panels.p, A, ld);
  k_qr_copy_h<<<(unsigned)std::min<int64_t>(ceil_div(m, 256), 1024), 256, 0, st>>>(
      h->d_h.as<double>(), m, A + (int64_t)n * ld);
  count_launch(h);

  const int warps_per_block = kApplyThreads / 32;
  const int max_blocks = 152 * 8;
  const int nb0 = (int)std::max<int64_t>(1, std::min<int64_t>(ceil_div(n, warps_per_block),
                                                               max_blocks));
  dcn.alloc((size_t)n * sizeof(double), st);
  dperm.alloc((size_t)n * sizeof(int), st);
  dv.alloc((size_t)m * sizeof(double), st);
  dstate.alloc(sizeof(QrState), st);
  dpv.alloc((size_t)max_blocks * sizeof(double), st);
  dpi.alloc((size_t)max_blocks * sizeof(int), st);
  dcnt.alloc(sizeof(unsigned int), st);
  CUDA_CHECK(cudaMemsetAsync(dstate.p, 0, sizeof(QrState), st));
  CUDA_CHECK(cudaMemsetAsync(dcnt.p, 0, sizeof(unsigned int), st));
  QrState* S = dstate.as<QrState>();
  k_qr_iota<<<(unsigned)std::max<int64_t>(1, std::min<int64_t>(ceil_div(n, 256), 1024)), 256, 0,
              st>>>(dperm.as<int>(), n);
  k_qr_colnorms<<<nb0, kApplyThreads, 0, st>>>(A, ld, m, n, dcn.as<double>(), dpv.as<double>(),
                                               dpi.as<int>(), dcnt.as<unsigned int>(), S);
  count_launch(h, 2);
  check_launch("qr set-up");

  const int steps = (int)std::min<int64_t>(m, n);
  QrState hs{};
  int k = 0;
  while (k < steps) {
    const int batch = std::min(kQrBatch, steps - k);
    for (int b = 0; b < batch; ++b, ++k) {
      k_qr_house<<<1, kHouseThreads, 0, st>>>(A, ld, m, k, dcn.as<double>(), dperm.as<int>(),
                                              dv.as<double>(), S, o->rcond);
      const int nb = (int)std::max<int64_t>(
          1, std::min<int64_t>(ceil_div(n - k, warps_per_block), max_blocks));
      k_qr_apply<<<nb, kApplyThreads, 0, st>>>(A, ld, m, n, k, dv.as<double>(), S,
                                               dcn.as<double>(), dpv.as<double>(), dpi.as<int>(),
                                               dcnt.as<unsigned int>());
    }
    count_launch(h, 2 * batch);
    check_launch("qr step");
    CUDA_CHECK(cudaMemcpyAsync(&hs, S, sizeof(QrState), cudaMemcpyDeviceToHost, st));
    stream_sync(h);
    if (hs.bad != 0.0) ELMFB_THROW(ELMFB_ERR_NONFINITE, "QR: non-finite column norm");
    if (hs.stop) break;
  }
  const int rank = hs.rank;
  dy.alloc((size_t)std::max(rank, 1) * sizeof(double), st);
  dz.alloc((size_t)std::max(rank, 1) * sizeof(double), st);
  dres.alloc(sizeof(double), st);
  k_qr_backsub<<<1, 1024, 0, st>>>(A, ld, m, n, S, dy.as<double>(), dz.as<double>(),
                                   dres.as<double>());
  CUDA_CHECK(cudaMemsetAsync(h->d_a.p, 0, (size_t)N * sizeof(double), st));
  k_qr_scatter<<<(unsigned)std::max(1, std::min((rank + 255) / 256, 1024)), 256, 0, st>>>(
      dz.as<double>(), dperm.as<int>(), S, h->d_a.as<double>());
  count_launch(h, 2);
  check_launch("qr back substitution");
  double res2 = 0.0, rrr = 0.0;
  CUDA_CHECK(cudaMemcpyAsync(&res2, dres.p, sizeof(double), cudaMemcpyDeviceToHost, st));
  if (rank > 0)
    CUDA_CHECK(cudaMemcpyAsync(&rrr, A + (int64_t)(rank - 1) * ld + (rank - 1), sizeof(double),
                               cudaMemcpyDeviceToHost, st));
  stream_sync(h);
  stage_end(h, 5);
  info->status = ELMFB_OK;
  info->iterations = rank;
  info->rank = rank;
  info->residual_norm = std::sqrt(res2);
  info->normal_residual_norm = NAN;
  info->sigma_max = hs.r11;
  info->sigma_min = std::fabs(rrr);
  info->setup_ms = 0.0;
  info->solve_ms = h->stage_ms[5];
}
