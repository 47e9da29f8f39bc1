// System assembly: cell sort of the collocation rows (K0) and the fused panel
// assembly kernel (K1).
//
// The paper defines every entry of M (§3 "Definition of the system matrices")
//     M[r, q] = s_r / L * Op_r[w_j phi_jk](x_r)
// with s_r = 1/sqrt(N_I) for interior rows and sqrt(lambda_b / N_B^(b)) for
// boundary rows, w_j the normalised cos^2 window (§4.1 Eq. window_func) and
// phi_jk = tanh(w . (x - mu_j)/sigma_j + b) (§3 shallow network, h = 1).  M is
// nonzero only on I_j x K_j (Eq. multilevel_domain_decomp), so it is stored as
// one dense row-major panel |I_j| x K per subdomain j.
//
// Panel rows are ordered cell-major: the rows of each cell of the common
// refinement of all supports are contiguous and padded with zero rows to a
// multiple of 16, in every panel that covers the cell.  A point's covering
// subdomains, and its row offset inside each of their panels, then follow from
// its cell alone.
//
// K1 evaluates the operator analytically.  With t = 1 - phi^2 and
// d_i = w_i / sigma_i (= d s / d x_i),
//     d_i phi = t d_i,    d_ii phi = -2 phi t d_i^2,
// and the product rule of Op[w phi] collects into
//     Op[w phi] = phi A + t sum_i beta_i d_i - 2 phi t sum_i gamma_i d_i^2
// with per-(row, subdomain) A = c0 w + sum c1_i d_i w + sum c2_i d_ii w,
// beta_i = c1_i w + 2 c2_i d_i w, gamma_i = c2_i w.  A warp computes these for
// 32 rows (one row per lane), then broadcasts them while every lane evaluates
// its own features of each row, so stores of a row are contiguous.
//
// Window factors use the half-angle form 1 + cos(theta) = 2 cos^2(theta/2):
//     f = 4 c^4,  f' = -8 c^3 s g,  f'' = 4 c^2 (3 s^2 - c^2) g^2
// with (s, c) = sincos(theta/2), g = pi/sigma, which keeps full relative
// accuracy near the support edge (theta -> +-pi) where 1 + cos(theta) cancels;
// there c = sin(pi u / 2) with the edge distance u = (sigma - |x - mu|)/sigma
// formed in FP64.  The support test is |x - mu| < sigma in FP64, as in the
// paper's open support.
// tanh is formed from expm1: e = expm1(2|s|), phi = sign(s) e/(e+2) and
// 1 - phi^2 = 4 (e+1)/(e+2)^2, free of cancellation for every s.
#include <algorithm>
#include <cmath>
#include <numeric>

#include <cuda_bf16.h>

#include "elmfb_internal.cuh"

namespace {

constexpr float kPiF = 3.14159265358979323846f;
constexpr double kPiD = 3.14159265358979323846;


// ------------------------------------------------------------------ K0 ------
__global__ void k_cell_of_rows(const double* __restrict__ pts, int64_t n, int dim,
                               const double* __restrict__ bnd, int nc0, int nc1,
                               double lo0, double hi0, double lo1, double hi1,
                               int* __restrict__ row_cell, int* __restrict__ count,
                               int* __restrict__ flags) {
  int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= n) return;
  int c[2] = {0, 0};
  const int ncs[2] = {nc0, nc1};
  const double los[2] = {lo0, lo1}, his[2] = {hi0, hi1};
  const double* b = bnd;
  for (int i = 0; i < dim; ++i) {
    double x = pts[r * dim + i];
    if (!(x >= los[i] && x <= his[i])) atomicOr(&flags[0], 1);  // outside the box / NaN
    // last boundary <= x
    int lo = 0, hi = ncs[i];  // search in b[0..nc]
    while (hi - lo > 1) {
      int mid = (lo + hi) >> 1;
      if (b[mid] <= x) lo = mid;
      else hi = mid;
    }
    c[i] = lo;
    b += ncs[i] + 1;
  }
  int cell = c[1] * nc0 + c[0];
  row_cell[r] = cell;
  atomicAdd(&count[cell], 1);
}

// Stable LSD radix sort of the rows by cell id (8-bit digits), so rows of a
// cell are ordered by their user index whatever the launch schedule; then
// k_place_rows writes them into the padded cell layout.  A tile of kSortTile
// rows is handled by one CTA: k_radix_hist counts its digits, k_radix_scan
// turns the digit-major table into output offsets, k_radix_scatter moves the
// tile 256 rows at a time, ranking equal digits by warp match and per-warp
// counts so equal keys keep their order.
constexpr int kSortTile = 4096;
constexpr int kSortThreads = 256;

__global__ void __launch_bounds__(kSortThreads) k_radix_hist(const int* __restrict__ keys,
                                                             int64_t n, int shift,
                                                             int* __restrict__ hist,
                                                             int n_tiles) {
  __shared__ int cnt[256];
  cnt[threadIdx.x] = 0;
  __syncthreads();
  const int64_t t0 = (int64_t)blockIdx.x * kSortTile;
  const int64_t t1 = t0 + kSortTile < n ? t0 + kSortTile : n;
  for (int64_t i = t0 + threadIdx.x; i < t1; i += kSortThreads)
    atomicAdd(&cnt[(keys[i] >> shift) & 255], 1);
  __syncthreads();
  hist[(int64_t)threadIdx.x * n_tiles + blockIdx.x] = cnt[threadIdx.x];
}

// exclusive scan of m ints in place, one CTA of 1024 threads
__global__ void __launch_bounds__(1024) k_radix_scan(int* __restrict__ a, int64_t m) {
  __shared__ int part[1024];
  const int64_t per = (m + 1023) / 1024;
  const int64_t b0 = threadIdx.x * per;
  const int64_t b1 = b0 + per < m ? b0 + per : m;
  int sum = 0;
  for (int64_t i = b0; i < b1; ++i) sum += a[i];
  part[threadIdx.x] = sum;
  __syncthreads();
  for (int o = 1; o < 1024; o <<= 1) {
    int v = threadIdx.x >= o ? part[threadIdx.x - o] : 0;
    __syncthreads();
    part[threadIdx.x] += v;
    __syncthreads();
  }
  int run = part[threadIdx.x] - sum;
  for (int64_t i = b0; i < b1; ++i) {
    int v = a[i];
    a[i] = run;
    run += v;
  }
}

__global__ void __launch_bounds__(kSortThreads) k_radix_scatter(
    const int* __restrict__ keys_in, const int* __restrict__ vals_in, int64_t n, int shift,
    const int* __restrict__ offs, int n_tiles, int* __restrict__ keys_out,
    int* __restrict__ vals_out) {
  constexpr int W = kSortThreads / 32;
  __shared__ int running[256];
  __shared__ int wcount[W][256];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  running[threadIdx.x] = offs[(int64_t)threadIdx.x * n_tiles + blockIdx.x];
  const int64_t t0 = (int64_t)blockIdx.x * kSortTile;
  const int64_t t1 = t0 + kSortTile < n ? t0 + kSortTile : n;
  const unsigned lt = (1u << lane) - 1u;
  for (int64_t c0 = t0; c0 < t1; c0 += kSortThreads) {
#pragma unroll
    for (int q = 0; q < W; ++q) wcount[q][threadIdx.x] = 0;
    __syncthreads();
    const int64_t i = c0 + threadIdx.x;
    const bool valid = i < t1;
    const int key = valid ? keys_in[i] : 0;
    const int val = valid ? (vals_in ? vals_in[i] : (int)i) : 0;
    const int d = valid ? (key >> shift) & 255 : 256 + lane;
    const unsigned peers = __match_any_sync(0xffffffffu, d);
    const int rank = __popc(peers & lt);
    if (valid && rank == 0) wcount[w][d] = __popc(peers);
    __syncthreads();
    if (valid) {
      int pos = running[d] + rank;
      for (int q = 0; q < w; ++q) pos += wcount[q][d];
      keys_out[pos] = key;
      vals_out[pos] = val;
    }
    __syncthreads();
    int add = 0;
#pragma unroll
    for (int q = 0; q < W; ++q) add += wcount[q][threadIdx.x];
    running[threadIdx.x] += add;
  }
}

// sorted[cell_pstart[c] + j] = j-th row of cell c (keys sorted, ustart = unpadded starts)
__global__ void k_place_rows(const int* __restrict__ keys, const int* __restrict__ vals,
                             int64_t n, const int* __restrict__ ustart,
                             const int* __restrict__ cell_pstart, int* __restrict__ sorted) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const int c = keys[i];
  sorted[cell_pstart[c] + (i - ustart[c])] = vals[i];
}

__global__ void k_gather_rows(const RowClass* __restrict__ c_cls, const int* __restrict__ sorted,
                              int64_t NR, int dim,
                              const double* __restrict__ pts, const double* __restrict__ rhs,
                              const int* __restrict__ cls_user, const int* __restrict__ row_cell,
                              double* __restrict__ x, int* __restrict__ rcls,
                              double* __restrict__ hvec, int* __restrict__ grow_cell,
                              int* __restrict__ user_to_sorted, const int* __restrict__ cell_of_R) {
  int64_t R = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (R >= NR) return;
  int r = sorted[R];
  grow_cell[R] = cell_of_R[R];
  if (r < 0) {
    for (int i = 0; i < dim; ++i) x[R * dim + i] = 0.0;
    rcls[R] = -1;
    hvec[R] = 0.0;
    return;
  }
  for (int i = 0; i < dim; ++i) x[R * dim + i] = pts[(int64_t)r * dim + i];
  int k = cls_user[r];
  rcls[R] = k;
  // scaled right-hand side (§3 "Definition of vectors")
  hvec[R] = rhs[r] * c_cls[k].hscale;
  user_to_sorted[r] = (int)R;
}

__global__ void k_fill_cell_of_R(const int* __restrict__ cell_pstart, int n_cells,
                                 int* __restrict__ cell_of_R) {
  int c = blockIdx.x;
  if (c >= n_cells) return;
  for (int p = cell_pstart[c] + threadIdx.x; p < cell_pstart[c + 1]; p += blockDim.x)
    cell_of_R[p] = c;
}

// Work lists written on the device from one record per group (a group's
// items are consecutive in the output, off[g] .. off[g + 1]).
// Entry steps: item t of group g is (ent[g], rows t).
__global__ void k_expand_steps(const int* __restrict__ ent, const int64_t* __restrict__ off,
                               int n_groups, int rows, int2* __restrict__ out) {
  const int g = blockIdx.x;
  if (g >= n_groups) return;
  const int64_t o = off[g], n = off[g + 1] - o;
  const int e = ent[g];
  for (int64_t t = threadIdx.x; t < n; t += blockDim.x) out[o + t] = make_int2(e, (int)(rows * t));
}

// Assembly tiles: item t of group g = (first entry, entries, 32 t, 0).
__global__ void k_expand_ltiles(const int2* __restrict__ grp, const int64_t* __restrict__ off,
                                int n_groups, int4* __restrict__ out) {
  const int g = blockIdx.x;
  if (g >= n_groups) return;
  const int64_t o = off[g], n = off[g + 1] - o;
  const int2 b = grp[g];
  for (int64_t t = threadIdx.x; t < n; t += blockDim.x)
    out[o + t] = make_int4(b.x, b.y, (int)(32 * t), 0);
}

__global__ void k_fill_int(int* __restrict__ p, int64_t n, int v) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    p[i] = v;
}

// ------------------------------------------------------------------ K1 ------
template <class T> struct Math;
template <> struct Math<float> {
  static __device__ __forceinline__ void sincospi(float x, float* s, float* c) { sincospif(x, s, c); }
  static __device__ __forceinline__ float expm1(float x) { return expm1f(x); }
  static __device__ __forceinline__ float rcp(float x) { return __frcp_rn(x); }
  static __device__ __forceinline__ float pi() { return kPiF; }
};
template <> struct Math<double> {
  static __device__ __forceinline__ void sincospi(double x, double* s, double* c) { ::sincospi(x, s, c); }
  static __device__ __forceinline__ double expm1(double x) { return ::expm1(x); }
  static __device__ __forceinline__ double rcp(double x) { return 1.0 / x; }
  static __device__ __forceinline__ double pi() { return kPiD; }
};

// tanh(s) and 1 - tanh(s)^2 from one expm1 (see file header)
template <class T>
__device__ __forceinline__ void tanh_pair(T s, T* phi, T* t) {
  T as = fabs(s);
  as = as < T(15) ? as : T(15);
  T e = Math<T>::expm1(T(2) * as);
  T r = Math<T>::rcp(e + T(2));
  T p = e * r;
  *phi = copysign(p, s);
  *t = T(4) * (e + T(1)) * r * r;
}
// FP32 panels: with r = 1 / (e^{2s} + 1), tanh s = 1 - 2 r and 1 - tanh^2 s =
// 4 r (1 - r), from the hardware exp2 and reciprocal (relative errors below
// 2^-22).  Their absolute errors in phi and t stay near 1e-7, which the FP32
// entries' tolerance (1e-6 of the largest term magnitude of their K-feature
// block) absorbs; e = inf (s > 44) gives r = 0, phi = 1, t = 0, and e = 0
// gives r = 1, phi = -1, t = 0.
__device__ __forceinline__ void tanh_pair_fast(float s, float* phi, float* t) {
  float e, r;
  asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(e) : "f"(s * 2.8853900817779268f));   // 2 log2(e)
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(e + 1.0f));
  *phi = fmaf(-2.0f, r, 1.0f);
  *t = 4.0f * r * (1.0f - r);
}

// Window factor of one subdomain at one point: w = prod_i f_i(x_i) with
// f = 4 c^4 (half-angle form, see the file header), its first and second
// derivative along each axis, and the scaled coordinate xt = (x - mu)/sigma.
// The support test |x - mu| < sigma and the edge distance are FP64.
template <class T>
__device__ __forceinline__ void window_factor(const double* x, int dim, const SubGeom& g, T& w,
                                              T dw[2], T ddw[2], T xt[2]) {
  T f[2] = {1, 1}, fp[2] = {0, 0}, fpp[2] = {0, 0};
  xt[0] = xt[1] = 0;
  for (int i = 0; i < dim; ++i) {
    const double dx = x[i] - g.mu[i];
    const double adx = fabs(dx);
    const T inv_s = sizeof(T) == 8 ? (T)g.inv_sigma_d[i] : (T)g.inv_sigma[i];
    xt[i] = (T)dx * inv_s;
    if (adx < g.sigma_d[i]) {
      // half angle theta/2 = pi xt / 2: (sh, ch) = (sin, cos)(theta/2).  Near the
      // edge use u = 1 - |xt| = (sigma - |dx|)/sigma formed in FP64, so
      // ch = sin(pi u / 2) keeps its relative accuracy as ch -> 0.
      T sh, ch;
      const double ud = (g.sigma_d[i] - adx) * g.inv_sigma_d[i];
      if (ud < 0.5) {
        T su, cu;
        Math<T>::sincospi(T(0.5) * (T)ud, &su, &cu);
        ch = su;
        sh = dx < 0.0 ? -cu : cu;
      } else {
        Math<T>::sincospi(T(0.5) * xt[i], &sh, &ch);
      }
      const T gg = Math<T>::pi() * inv_s;
      const T c2 = ch * ch;
      f[i] = T(4) * c2 * c2;
      fp[i] = T(-8) * c2 * ch * sh * gg;
      fpp[i] = T(4) * c2 * (T(3) * sh * sh - c2) * gg * gg;
    } else {
      f[i] = 0;
      fp[i] = 0;
      fpp[i] = 0;
    }
  }
  w = f[0] * f[1];
  dw[0] = fp[0] * f[1];
  ddw[0] = fpp[0] * f[1];
  dw[1] = f[0] * fp[1];
  ddw[1] = f[0] * fpp[1];
}

constexpr int kFacVals = 7;   // w, dw[2], ddw[2], xt[2] per (row, covering subdomain)

// K1: one warp per tile (first covering entry e0 of one level's group in one
// cell, nl entries, 32 rows from p0).  Phase 1: lane = row; the window factors
// of the level's nl covering subdomains are formed once (kept in the warp's
// shared memory, each lane reading back only its own column) together with
// their level sums S, dS, ddS.  Then per covering panel: the normalised window
// by the quotient rule (and the ansatz factor), the per-row terms A, beta_i,
// gamma_i, and phase 2, which broadcasts one row at a time while every lane
// evaluates its own features, so that the K entries of a row are stored
// contiguously.  SPLIT (T = double): entries stored as FP32 pairs (ELMFB_DF32).
template <class T, int FPL, bool WRITE_T, bool SPLIT, bool kVec>
__global__ void __launch_bounds__(128) k_assemble(
    const int4* __restrict__ tiles, int64_t n_tiles, int dim, int K, int nl_max,
    const SubGeom* __restrict__ sub, const int* __restrict__ cover_sub,
    const int* __restrict__ cover_start, const int* __restrict__ entry_cell,
    const int* __restrict__ cell_count, const int* __restrict__ cell_pstart,
    const int64_t* __restrict__ panel_off, const int64_t* __restrict__ entry_base,
    const int* __restrict__ cover_off, const double* __restrict__ xs, const int* __restrict__ rcls,
    const RowClass* __restrict__ c_cls, const T* __restrict__ W, const T* __restrict__ Bias,
    T* __restrict__ panels, __nv_bfloat16* __restrict__ pt, int64_t NPR, const Ansatz an,
    float* __restrict__ panels32) {
  extern __shared__ __align__(16) unsigned char k1_smem[];
  const int lane = threadIdx.x & 31, wq = threadIdx.x >> 5;
  const int64_t t = (int64_t)blockIdx.x * (blockDim.x >> 5) + wq;
  if (t >= n_tiles) return;
  T* fac = reinterpret_cast<T*>(k1_smem) + (size_t)wq * nl_max * kFacVals * 32;
  __nv_bfloat16* tsm =
      reinterpret_cast<__nv_bfloat16*>(k1_smem + (size_t)(blockDim.x >> 5) * nl_max * kFacVals *
                                                     32 * sizeof(T)) +
      (size_t)wq * K * 32;
  T* rowt = reinterpret_cast<T*>(k1_smem + (size_t)(blockDim.x >> 5) * nl_max * kFacVals * 32 *
                                                 sizeof(T) +
                                 (WRITE_T ? (size_t)(blockDim.x >> 5) * K * 32 *
                                                sizeof(__nv_bfloat16)
                                          : 0)) +
            (size_t)wq * 32 * 8;
  // lanes own consecutive features where a row leaves as vector stores;
  // elsewhere f = lane + 32 i keeps every scalar store coalesced
  constexpr bool kConsec = kVec;
  const int4 tile = tiles[t];
  const int e0 = tile.x, nl = tile.y, p0 = tile.z;
  const int c = entry_cell[e0];
  const int cnt = cell_count[c];
  const int pad = cell_pstart[c + 1] - cell_pstart[c];
  const int nrows = min(32, pad - p0);
  const int64_t R0 = cell_pstart[c] + p0;
  // cell-interleaved storage: row p of entry e at element row entry_base[e] + p m_c
  const int64_t rstride = (int64_t)(cover_off[c + 1] - cover_off[c]) * K;
  const int p = p0 + lane;
  const bool valid = lane < nrows && p < cnt;
  const int64_t R = R0 + lane;
  double x[2] = {0.0, 0.0};
  if (valid) {
    x[0] = xs[R * dim];
    if (dim == 2) x[1] = xs[R * dim + 1];
  }

  // phase 1a: the level's window factors and their sums
  T S = 0, dS[2] = {0, 0}, ddS[2] = {0, 0};
  for (int k = 0; k < nl; ++k) {
    T w = 0, dw[2] = {0, 0}, ddw[2] = {0, 0}, xt[2] = {0, 0};
    if (valid) window_factor<T>(x, dim, sub[cover_sub[e0 + k]], w, dw, ddw, xt);
    S += w;
    for (int i = 0; i < 2; ++i) {
      dS[i] += dw[i];
      ddS[i] += ddw[i];
    }
    T* fk = fac + (size_t)k * kFacVals * 32 + lane;
    fk[0] = w;
    fk[32] = dw[0];
    fk[64] = dw[1];
    fk[96] = ddw[0];
    fk[128] = ddw[1];
    fk[160] = xt[0];
    fk[192] = xt[1];
  }
  const T iS = S > T(0) ? T(1) / S : T(0);
  RowClass rc{};
  double Aa = 1.0, dA[2] = {0.0, 0.0}, ddA[2] = {0.0, 0.0};
  if (valid) {
    rc = c_cls[rcls[R]];
    if (an.w > 0.0) ansatz_at(an, x, dim, Aa, dA, ddA);
  }

  for (int k = 0; k < nl; ++k) {
    const int e = e0 + k;
    const int s = cover_sub[e];
    const SubGeom gs = sub[s];
    // phase 1b: this panel's normalised window (quotient rule over the level)
    const T* fk = fac + (size_t)k * kFacVals * 32 + lane;
    const T wo = fk[0], dwo[2] = {fk[32], fk[64]}, ddwo[2] = {fk[96], fk[128]};
    T om = wo * iS, dom[2], ddom[2];
    for (int i = 0; i < 2; ++i) {
      const T a = dS[i] * iS;
      dom[i] = (dwo[i] - wo * a) * iS;
      ddom[i] = (ddwo[i] - T(2) * dwo[i] * a - wo * ddS[i] * iS + T(2) * wo * a * a) * iS;
    }
    if (an.w > 0.0) {
      // hard-constraint ansatz (paper §4.3): the window factor becomes
      // g = A w, with g' = A' w + A w' and g'' = A'' w + 2 A' w' + A w''
      for (int i = 0; i < 2; ++i) {
        ddom[i] = (T)ddA[i] * om + T(2) * (T)dA[i] * dom[i] + (T)Aa * ddom[i];
        dom[i] = (T)dA[i] * om + (T)Aa * dom[i];
      }
      om = (T)Aa * om;
    }
    T A = 0, be0 = 0, be1 = 0, ga0 = 0, ga1 = 0;
    const T xt0 = fk[160], xt1 = fk[192];
    if (valid) {
      const T sc = (T)rc.scale;
      A = sc * ((T)rc.c0 * om + (T)rc.c1[0] * dom[0] + (T)rc.c2[0] * ddom[0] +
                (T)rc.c1[1] * dom[1] + (T)rc.c2[1] * ddom[1]);
      be0 = sc * ((T)rc.c1[0] * om + T(2) * (T)rc.c2[0] * dom[0]);
      be1 = sc * ((T)rc.c1[1] * om + T(2) * (T)rc.c2[1] * dom[1]);
      ga0 = sc * (T)rc.c2[0] * om;
      ga1 = sc * (T)rc.c2[1] * om;
    }

    // per-lane feature constants: with vector stores lanes own FPL
    // consecutive features (f = lane FPL + i), else f = lane + 32 i
    T w0[FPL], w1[FPL], bb[FPL], d0[FPL], d1[FPL], e0[FPL], e1[FPL];
    const T is0 = sizeof(T) == 8 ? (T)gs.inv_sigma_d[0] : (T)gs.inv_sigma[0];
    const T is1 = sizeof(T) == 8 ? (T)gs.inv_sigma_d[1] : (T)gs.inv_sigma[1];
#pragma unroll
    for (int i = 0; i < FPL; ++i) {
      const int f = kConsec ? lane * FPL + i : lane + 32 * i;
      if (f < K) {
        const int64_t q = (int64_t)s * K + f;
        w0[i] = W[q * dim];
        w1[i] = dim == 2 ? W[q * dim + 1] : T(0);
        bb[i] = Bias[q];
      } else {
        w0[i] = w1[i] = bb[i] = 0;
      }
      d0[i] = w0[i] * is0;
      d1[i] = w1[i] * is1;
      e0[i] = d0[i] * d0[i];
      e1[i] = d1[i] * d1[i];
    }

    // phase 2: the per-row terms go to shared memory, then each row's are
    // read back by every lane (broadcast) while the lanes form its features:
    // Op[w phi] = phi A + t (B - 2 phi C), B = sum_i beta_i d_i,
    // C = sum_i gamma_i d_i^2
    T* out = panels + entry_base[e] * (int64_t)K + (int64_t)p0 * rstride;
    __syncwarp();   // the previous panel's row terms (and BF16 staging) have been read
    {
      T* rt = rowt + lane * 8;
      rt[0] = A;
      rt[1] = be0;
      rt[2] = be1;
      rt[3] = ga0;
      rt[4] = ga1;
      rt[5] = xt0;
      rt[6] = xt1;
    }
    __syncwarp();
    for (int r = 0; r < nrows; ++r) {
      const T* rt = rowt + r * 8;
      const T rA = rt[0], rb0 = rt[1], rb1 = rt[2], rg0 = rt[3], rg1 = rt[4], rx0 = rt[5],
              rx1 = rt[6];
      T* orow = out + (int64_t)r * rstride;
      T vals[FPL];
#pragma unroll
      for (int i = 0; i < FPL; ++i) {
        const T sarg = w0[i] * rx0 + w1[i] * rx1 + bb[i];
        T phi, tt;
        if constexpr (sizeof(T) == 4) tanh_pair_fast(sarg, &phi, &tt);
        else tanh_pair<T>(sarg, &phi, &tt);
        const T B = rb0 * d0[i] + rb1 * d1[i];
        const T Cc = rg0 * e0[i] + rg1 * e1[i];
        vals[i] = tt * (B - T(2) * phi * Cc) + phi * rA;
      }
      if constexpr (kVec) {
        // K = 32 FPL and FP32 entries: one 8- or 16-byte store per lane
        if constexpr (FPL == 4)
          reinterpret_cast<float4*>(orow)[lane] = make_float4(vals[0], vals[1], vals[2], vals[3]);
        else
          reinterpret_cast<float2*>(orow)[lane] = make_float2(vals[0], vals[1]);
      } else {
#pragma unroll
        for (int i = 0; i < FPL; ++i) {
          const int f = kConsec ? lane * FPL + i : lane + 32 * i;
          if (f < K) {
            const T v = vals[i];
            if (SPLIT) {
              const float hi = __double2float_rn((double)v);
              reinterpret_cast<float2*>(orow)[f] =
                  make_float2(hi, __double2float_rn((double)v - (double)hi));
              // ELMFB_FP32_DF32: the FP32 panels hold the rounded entries
              if (panels32) panels32[(orow - panels) + f] = hi;
            } else {
              orow[f] = v;
            }
            if (WRITE_T) tsm[(size_t)f * 32 + r] = __float2bfloat16_rn((float)v);
          }
        }
      }
    }
    if (WRITE_T) {
      // feature-major BF16 copy: feature f, rows rho0 .. rho0+nrows in 16-byte pieces
      __syncwarp();
      const int64_t rho0 = panel_off[s] + cover_start[e] + p0;
      const int pieces = nrows / 8;   // nrows is 16 or 32
      for (int idx = lane; idx < K * pieces; idx += 32) {
        const int f = idx / pieces, q = idx - f * pieces;
        const uint4 val = *reinterpret_cast<const uint4*>(tsm + (size_t)f * 32 + q * 8);
        *reinterpret_cast<uint4*>(pt + (int64_t)f * NPR + rho0 + q * 8) = val;
      }
    }
  }
}

template <class T>
void launch_assemble(elmfb_ctx* h) {
  const int K = h->K;
  const int fpl = (K + 31) / 32;
  const int warps = 4;
  const int64_t blocks = ceil_div(h->n_ltiles, warps);
  if (blocks == 0) return;
  const T* W = sizeof(T) == 8 ? (const T*)h->d_W64.p : (const T*)h->d_W32.p;
  const T* B = sizeof(T) == 8 ? (const T*)h->d_b64.p : (const T*)h->d_b32.p;
  const bool wt = h->cfg.precision == ELMFB_MIXED && sizeof(T) == 4;
  const bool split = (h->df32() || h->dual()) && sizeof(T) == 8;
  // ELMFB_FP32_DF32: pairs into d_panels_df, their FP32 rounding into d_panels
  T* const pout = h->dual() ? (T*)h->d_panels_df.p : (T*)h->d_panels.p;
  float* const p32 = h->dual() && sizeof(T) == 8 ? (float*)h->d_panels.p : nullptr;
  const size_t smem = (size_t)warps * h->nl_max * kFacVals * 32 * sizeof(T) +
                      (wt ? (size_t)warps * K * 32 * sizeof(__nv_bfloat16) : 0) +
                      (size_t)warps * 32 * 8 * sizeof(T);
  // FP32 entries with K = 64 or 128: vector stores of a lane's features
  const bool vec = !wt && !split && sizeof(T) == 4 && (K == 64 || K == 128);
  if (wt && K > 128) ELMFB_THROW(ELMFB_ERR_UNSUPPORTED, "mixed precision supports K <= 128");
  if (smem > 220 * 1024)
    ELMFB_THROW(ELMFB_ERR_UNSUPPORTED, "assembly: too many covering subdomains per level");
  const Ansatz an = make_ansatz(h->cfg);
#define ELMFB_K1_ARGS                                                                        \
  h->d_ltiles.as<int4>(), h->n_ltiles, h->dim, K, h->nl_max, h->d_sub.as<SubGeom>(),         \
      h->d_cover_sub.as<int>(), h->d_cover_start.as<int>(), h->d_entry_cell.as<int>(),       \
      h->d_cell_count.as<int>(), h->d_cell_pstart.as<int>(), h->d_panel_off.as<int64_t>(),   \
      h->d_entry_base.as<int64_t>(), h->d_cover_off.as<int>(), h->d_x.as<double>(),          \
      h->d_rcls.as<int>(), h->d_cls.as<RowClass>(), W, B, pout
#define ELMFB_K1_LAUNCH(F, WT, SP, VEC, PT, P32)                                                \
  do {                                                                                       \
    ensure_dyn_smem((const void*)k_assemble<T, F, WT, SP, VEC>, smem);                       \
    k_assemble<T, F, WT, SP, VEC><<<(unsigned)blocks, warps * 32, smem, h->stream>>>(        \
        ELMFB_K1_ARGS, PT, h->NPR, an, P32);                                                 \
  } while (0)
#define ELMFB_K1(F)                                                                          \
  case F:                                                                                    \
    if (wt) ELMFB_K1_LAUNCH(F, true, false, false, h->d_pt.as<__nv_bfloat16>(), nullptr);    \
    else if (split) ELMFB_K1_LAUNCH(F, false, true, false, nullptr, p32);                    \
    else if (vec) ELMFB_K1_LAUNCH(F, false, false, (F == 2 || F == 4), nullptr, nullptr);    \
    else ELMFB_K1_LAUNCH(F, false, false, false, nullptr, nullptr);                          \
    break;
  // algorithmic bytes: every panel entry written once (twice in mixed precision:
  // FP32 row-major and BF16 feature-major), point data read once
  prof_begin(h, KID_ASSEMBLE,
             (double)h->NPR * K * (sizeof(T) + (wt ? 2.0 : 0.0) + (p32 ? 4.0 : 0.0)) +
                 (double)h->NR * (h->dim * 8.0 + 4.0));
  switch (fpl) {
    ELMFB_K1(1) ELMFB_K1(2) ELMFB_K1(3) ELMFB_K1(4) ELMFB_K1(5) ELMFB_K1(6) ELMFB_K1(7) ELMFB_K1(8)
    default: ELMFB_THROW(ELMFB_ERR_UNSUPPORTED, "features > 256");
  }
#undef ELMFB_K1
#undef ELMFB_K1_LAUNCH
#undef ELMFB_K1_ARGS
  prof_end(h, KID_ASSEMBLE);
  check_launch("k_assemble");
  count_launch(h);
}

// --------------------------------------------------------------- export -----
__device__ __forceinline__ double value_of(float v) { return (double)v; }
__device__ __forceinline__ double value_of(double v) { return v; }
__device__ __forceinline__ double value_of(df2 v) { return (double)v.hi + (double)v.lo; }

template <class T>
__global__ void k_export_rows(const int64_t* __restrict__ rows, int64_t n,
                              const int* __restrict__ user_to_sorted,
                              const int* __restrict__ grow_cell, const int* __restrict__ cell_pstart,
                              const int* __restrict__ cover_off, const int* __restrict__ cover_sub,
                              const int* __restrict__ cover_start,
                              const int64_t* __restrict__ entry_base, const T* __restrict__ panels,
                              int K, int64_t NPhi, const double* __restrict__ hvec,
                              double* __restrict__ out, double* __restrict__ hout) {
  int64_t i = blockIdx.x;
  if (i >= n) return;
  int R = user_to_sorted[rows[i]];
  int c = grow_cell[R];
  int p = R - cell_pstart[c];
  if (threadIdx.x == 0 && hout) hout[i] = hvec[R];
  for (int e = cover_off[c]; e < cover_off[c + 1]; ++e) {
    int s = cover_sub[e];
    const int64_t mc = cover_off[c + 1] - cover_off[c];
    const T* src = panels + (entry_base[e] + (int64_t)p * mc) * (int64_t)K;
    for (int k = threadIdx.x; k < K; k += blockDim.x)
      out[i * NPhi + (int64_t)s * K + k] = value_of(src[k]);
  }
}

}  // namespace

// ----------------------------------------------------------------------------
void assemble_system(elmfb_ctx* h, int n_sets, const elmfb_rowset* sets) {
  cudaStream_t st = h->stream;
  h->assembled = false;
  h->have_coeffs = false;
  const int dim = h->dim;
  int64_t n = 0;
  for (int b = 0; b < n_sets; ++b) {
    if (sets[b].n < 0 || (sets[b].n > 0 && (!sets[b].points || !sets[b].rhs)))
      ELMFB_THROW(ELMFB_ERR_INVALID_ARG, "row set " + std::to_string(b) + ": bad pointers");
    if (b > 0 && !(sets[b].weight > 0.0))
      ELMFB_THROW(ELMFB_ERR_INVALID_ARG, "boundary weight must be > 0");
    n += sets[b].n;
  }
  if (sets[0].n < 1) ELMFB_THROW(ELMFB_ERR_INVALID_ARG, "empty interior set");
  if (n >= (int64_t)1 << 31) ELMFB_THROW(ELMFB_ERR_UNSUPPORTED, "more than 2^31 rows");
  h->n_rows = n;

  // row classes (§3: interior scale 1/sqrt(N_I), boundary sqrt(lambda_b / N_B^(b)); 1/L folded in)
  h->n_classes = n_sets;
  for (int b = 0; b < n_sets; ++b) {
    RowClass rc{};
    rc.c0 = sets[b].c0;
    for (int i = 0; i < 2; ++i) {
      rc.c1[i] = i < dim ? sets[b].c1[i] : 0.0;
      rc.c2[i] = i < dim ? sets[b].c2[i] : 0.0;
    }
    double s = b == 0 ? 1.0 / std::sqrt((double)sets[0].n)
                      : (sets[b].n > 0 ? std::sqrt(sets[b].weight / (double)sets[b].n) : 0.0);
    rc.scale = s / h->L;
    rc.hscale = s;
    h->cls[b] = rc;
  }
  h->d_cls.alloc(sizeof(RowClass) * kMaxClasses, st);
  CUDA_CHECK(cudaMemcpyAsync(h->d_cls.p, h->cls, sizeof(RowClass) * n_sets,
                             cudaMemcpyHostToDevice, st));

  stage_begin(h, 7);
  stage_begin(h, 1);
  // user-order inputs
  h->d_pts_user.alloc(n * dim * sizeof(double), st);
  h->d_rhs_user.alloc(n * sizeof(double), st);
  h->d_cls_user.alloc(n * sizeof(int), st);
  {
    int64_t off = 0;
    for (int b = 0; b < n_sets; ++b) {
      int64_t m = sets[b].n;
      if (m == 0) continue;
      CUDA_CHECK(cudaMemcpyAsync(h->d_pts_user.as<double>() + off * dim, sets[b].points,
                                 m * dim * sizeof(double), cudaMemcpyDefault, st));
      CUDA_CHECK(cudaMemcpyAsync(h->d_rhs_user.as<double>() + off, sets[b].rhs, m * sizeof(double),
                                 cudaMemcpyDefault, st));
      k_fill_int<<<(unsigned)std::min<int64_t>(ceil_div(m, 256), 1216), 256, 0, st>>>(
          h->d_cls_user.as<int>() + off, m, b);
      count_launch(h);
      off += m;
    }
    check_launch("k_fill_int");
  }

  // K0: cells
  const int nc = h->n_cells;
  h->d_row_cell.alloc(n * sizeof(int), st);
  h->d_cell_count.alloc(nc * sizeof(int), st);
  CUDA_CHECK(cudaMemsetAsync(h->d_cell_count.p, 0, nc * sizeof(int), st));
  CUDA_CHECK(cudaMemsetAsync(h->d_flags.p, 0, 16 * sizeof(int), st));
  k_cell_of_rows<<<(unsigned)ceil_div(n, 256), 256, 0, st>>>(
      h->d_pts_user.as<double>(), n, dim, h->d_bnd.as<double>(), h->nc[0], h->nc[1], h->cfg.lo[0],
      h->cfg.hi[0], dim == 2 ? h->cfg.lo[1] : 0.0, dim == 2 ? h->cfg.hi[1] : 1.0,
      h->d_row_cell.as<int>(), h->d_cell_count.as<int>(), h->d_flags.as<int>());
  check_launch("k_cell_of_rows");
  count_launch(h);
  h->cell_count.resize(nc);
  int flags[4];
  CUDA_CHECK(cudaMemcpyAsync(h->cell_count.data(), h->d_cell_count.p, nc * sizeof(int),
                             cudaMemcpyDeviceToHost, st));
  CUDA_CHECK(cudaMemcpyAsync(flags, h->d_flags.p, 4 * sizeof(int), cudaMemcpyDeviceToHost, st));
  stream_sync(h);
  if (flags[0]) ELMFB_THROW(ELMFB_ERR_INVALID_ARG, "a collocation point lies outside the domain box");

  // host: padded cell layout, panel offsets, tiles
  h->cell_pstart.assign(nc + 1, 0);
  for (int c = 0; c < nc; ++c) {
    int cnt = h->cell_count[c];
    h->cell_pstart[c + 1] = h->cell_pstart[c] + (int)ceil_div(cnt, kCellPad) * kCellPad;
  }
  h->NR = h->cell_pstart[nc];
  const int ne = (int)h->cover_sub.size();
  h->cover_start.assign(ne, 0);
  h->panel_off.assign(h->n_sub + 1, 0);
  std::vector<int64_t> panel_len(h->n_sub, 0);
  // cells are visited in increasing id (y-major), so each panel's rows are cell-major
  for (int c = 0; c < nc; ++c) {
    int pad = h->cell_pstart[c + 1] - h->cell_pstart[c];
    for (int e = h->cover_off[c]; e < h->cover_off[c + 1]; ++e) {
      int s = h->cover_sub[e];
      h->cover_start[e] = (int)panel_len[s];
      panel_len[s] += pad;
    }
  }
  for (int s = 0; s < h->n_sub; ++s) h->panel_off[s + 1] = h->panel_off[s] + panel_len[s];
  h->NPR = h->panel_off[h->n_sub];
  // cell-interleaved element rows (see elmfb_ctx::cell_eoff)
  h->cell_eoff.assign(nc + 1, 0);
  for (int c = 0; c < nc; ++c)
    h->cell_eoff[c + 1] = h->cell_eoff[c] + (int64_t)(h->cell_pstart[c + 1] - h->cell_pstart[c]) *
                                                (h->cover_off[c + 1] - h->cover_off[c]);
  h->entry_base.assign(ne, 0);
  for (int e = 0; e < ne; ++e) {
    const int c = h->entry_cell[e];
    h->entry_base[e] = h->cell_eoff[c] + (e - h->cover_off[c]);
  }
  if (h->NPR >= (int64_t)1 << 31) ELMFB_THROW(ELMFB_ERR_UNSUPPORTED, "more than 2^31 panel rows");
  h->nnz = 0;
  for (int e = 0; e < ne; ++e) h->nnz += (int64_t)h->cell_count[h->entry_cell[e]] * h->K;
  h->n_tiles = -1;   // the QR's tiles, made when it runs (ensure_qr_tiles)
  // assembly tiles: one per (cell, level group of covering entries, 32 rows),
  // written on the device from one record per group
  std::vector<int2> lgrp;
  std::vector<int64_t> lgoff(1, 0);
  h->nl_max = 1;
  for (int c = 0; c < nc; ++c) {
    const int pad = h->cell_pstart[c + 1] - h->cell_pstart[c];
    for (int l = 0; l < h->L; ++l) {
      const int b = h->cell_level_off[(size_t)c * (h->L + 1) + l];
      const int en = h->cell_level_off[(size_t)c * (h->L + 1) + l + 1];
      if (en <= b) continue;
      h->nl_max = std::max(h->nl_max, en - b);
      if (pad == 0) continue;
      lgrp.push_back(make_int2(b, en - b));
      lgoff.push_back(lgoff.back() + ceil_div(pad, 32));
    }
  }
  h->n_ltiles = lgoff.back();
  // Gram pair count: subdomain pairs (i <= j) that share a cell with points,
  // and the algorithmic Gram flops 2 K^2 per shared row and pair
  h->gram_flops = 0.0;
  for (int c = 0; c < nc; ++c) {
    const double m = h->cover_off[c + 1] - h->cover_off[c];
    h->gram_flops += 0.5 * m * (m + 1) * 2.0 * h->K * h->K * h->cell_count[c];
  }
  h->n_gram_pairs = -1;   // counted when asked for (count_gram_pairs)

  auto up = [&](DevBuf& b, const void* src, size_t bytes) {
    b.alloc(std::max<size_t>(bytes, 4), st);
    if (bytes) CUDA_CHECK(cudaMemcpyAsync(b.p, src, bytes, cudaMemcpyHostToDevice, st));
  };
  up(h->d_cell_pstart, h->cell_pstart.data(), (nc + 1) * sizeof(int));
  up(h->d_cover_start, h->cover_start.data(), ne * sizeof(int));
  up(h->d_panel_off, h->panel_off.data(), (h->n_sub + 1) * sizeof(int64_t));
  up(h->d_cell_eoff, h->cell_eoff.data(), (nc + 1) * sizeof(int64_t));
  up(h->d_entry_base, h->entry_base.data(), ne * sizeof(int64_t));
  {
    DevBuf dg, dgo;
    up(dg, lgrp.data(), lgrp.size() * sizeof(int2));
    up(dgo, lgoff.data(), lgoff.size() * sizeof(int64_t));
    h->d_ltiles.alloc(std::max<int64_t>(h->n_ltiles, 1) * sizeof(int4), st);
    if (!lgrp.empty()) {
      k_expand_ltiles<<<(unsigned)lgrp.size(), 128, 0, st>>>(dg.as<int2>(), dgo.as<int64_t>(),
                                                             (int)lgrp.size(), h->d_ltiles.as<int4>());
      check_launch("k_expand_ltiles");
      count_launch(h);
    }
  }

  // K0: scatter into cells, deterministic order inside each cell, gather row data
  const int64_t NR = h->NR;
  h->d_sorted.alloc(NR * sizeof(int), st);
  CUDA_CHECK(cudaMemsetAsync(h->d_sorted.p, 0xff, NR * sizeof(int), st));
  {
    int bits = 1;
    while (bits < 31 && ((int64_t)1 << bits) < nc) ++bits;
    const int passes = (bits + 7) / 8;
    const int n_tiles = (int)ceil_div(n, kSortTile);
    std::vector<int> ustart(nc + 1, 0);
    for (int c = 0; c < nc; ++c) ustart[c + 1] = ustart[c] + h->cell_count[c];
    DevBuf ka, kb, va, vb, hist, dus;
    ka.alloc(n * sizeof(int), st);
    kb.alloc(n * sizeof(int), st);
    va.alloc(n * sizeof(int), st);
    vb.alloc(n * sizeof(int), st);
    hist.alloc((size_t)n_tiles * 256 * sizeof(int), st);
    up(dus, ustart.data(), (nc + 1) * sizeof(int));
    prof_begin(h, KID_CELL_SORT, (16.0 * passes + 12.0) * (double)n + 4.0 * (double)NR);
    const int* kin = h->d_row_cell.as<int>();
    const int* vin = nullptr;
    int* kout = ka.as<int>();
    int* vout = va.as<int>();
    for (int ps = 0; ps < passes; ++ps) {
      k_radix_hist<<<n_tiles, kSortThreads, 0, st>>>(kin, n, 8 * ps, hist.as<int>(), n_tiles);
      k_radix_scan<<<1, 1024, 0, st>>>(hist.as<int>(), (int64_t)n_tiles * 256);
      k_radix_scatter<<<n_tiles, kSortThreads, 0, st>>>(kin, vin, n, 8 * ps, hist.as<int>(),
                                                         n_tiles, kout, vout);
      check_launch("k_radix_scatter");
      kin = kout;
      vin = vout;
      kout = kout == ka.as<int>() ? kb.as<int>() : ka.as<int>();
      vout = vout == va.as<int>() ? vb.as<int>() : va.as<int>();
    }
    k_place_rows<<<(unsigned)ceil_div(n, 256), 256, 0, st>>>(
        kin, vin, n, dus.as<int>(), h->d_cell_pstart.as<int>(), h->d_sorted.as<int>());
    check_launch("k_place_rows");
    prof_end(h, KID_CELL_SORT);
    count_launch(h, 3 * passes + 1);
  }
  h->d_grow_cell.alloc(NR * sizeof(int), st);
  h->d_x.alloc(NR * dim * sizeof(double), st);
  h->d_rcls.alloc(NR * sizeof(int), st);
  h->d_h.alloc(NR * sizeof(double), st);
  h->d_u2s.alloc(n * sizeof(int), st);
  h->d_tmp.alloc(NR * sizeof(int), st);
  int* user_to_sorted = h->d_u2s.as<int>();
  int* cell_of_R = h->d_tmp.as<int>();
  k_fill_cell_of_R<<<nc, 128, 0, st>>>(h->d_cell_pstart.as<int>(), nc, cell_of_R);
  check_launch("k_fill_cell_of_R");
  k_gather_rows<<<(unsigned)ceil_div(NR, 256), 256, 0, st>>>(
      h->d_cls.as<RowClass>(), h->d_sorted.as<int>(), NR, dim, h->d_pts_user.as<double>(), h->d_rhs_user.as<double>(),
      h->d_cls_user.as<int>(), h->d_row_cell.as<int>(), h->d_x.as<double>(), h->d_rcls.as<int>(),
      h->d_h.as<double>(), h->d_grow_cell.as<int>(), user_to_sorted, cell_of_R);
  check_launch("k_gather_rows");
  count_launch(h, 2);
  stage_end(h, 1);

  // K1: panels
  stage_begin(h, 2);
  h->d_panels.alloc(h->NPR * h->K * h->panel_elem(), st);
  if (h->dual()) h->d_panels_df.alloc(h->NPR * h->K * sizeof(df2), st);
  h->bj_reuse = false;
  h->gram_pair_ij.clear();
  h->have_gram = false;
  h->gnn_off.clear();
  h->gnn_nb.clear();
  h->gnn_trained = false;
  if (h->cfg.precision == ELMFB_MIXED) {
    h->d_pt.alloc(h->NPR * h->K * 2, st);
    // padding tail of 16-row tiles is written by the kernel; clear once for safety
    CUDA_CHECK(cudaMemsetAsync(h->d_pt.p, 0, h->NPR * h->K * 2, st));
  }
  if (h->eval64() || h->dual()) launch_assemble<double>(h);
  else launch_assemble<float>(h);
  stage_end(h, 2);
  stage_end(h, 7);
  h->assembled = true;
}

// subdomain pairs (i <= j) that share a cell with points
int64_t count_gram_pairs(const elmfb_ctx* h) {
  std::vector<std::vector<int>> nb(h->n_sub);
  for (int c = 0; c < h->n_cells; ++c) {
    if (h->cell_count[c] == 0) continue;
    for (int e = h->cover_off[c]; e < h->cover_off[c + 1]; ++e)
      for (int f = e; f < h->cover_off[c + 1]; ++f) nb[h->cover_sub[e]].push_back(h->cover_sub[f]);
  }
  int64_t n = 0;
  for (auto& v : nb) {
    std::sort(v.begin(), v.end());
    n += std::unique(v.begin(), v.end()) - v.begin();
  }
  return n;
}

void export_rows(elmfb_ctx* h, const int64_t* rows, int64_t n, double* out, double* h_out) {
  if (n == 0) return;
  cudaStream_t st = h->stream;
  DevBuf drows, dout, dh;
  drows.alloc(n * sizeof(int64_t), st);
  CUDA_CHECK(cudaMemcpyAsync(drows.p, rows, n * sizeof(int64_t), cudaMemcpyDefault, st));
  {
    std::vector<int64_t> hr(n);
    CUDA_CHECK(cudaMemcpyAsync(hr.data(), drows.p, n * sizeof(int64_t), cudaMemcpyDeviceToHost, st));
    stream_sync(h);
    for (int64_t v : hr)
      if (v < 0 || v >= h->n_rows) ELMFB_THROW(ELMFB_ERR_INVALID_ARG, "row index out of range");
  }
  dout.alloc(n * h->NPhi * sizeof(double), st);
  dh.alloc(n * sizeof(double), st);
  CUDA_CHECK(cudaMemsetAsync(dout.p, 0, n * h->NPhi * sizeof(double), st));
  if (h->df32())
    k_export_rows<df2><<<(unsigned)n, 128, 0, st>>>(
        drows.as<int64_t>(), n, h->d_u2s.as<int>(), h->d_grow_cell.as<int>(),
        h->d_cell_pstart.as<int>(), h->d_cover_off.as<int>(), h->d_cover_sub.as<int>(),
        h->d_cover_start.as<int>(), h->d_entry_base.as<int64_t>(), h->d_panels.as<df2>(), h->K,
        h->NPhi, h->d_h.as<double>(), dout.as<double>(), dh.as<double>());
  else if (h->fp64())
    k_export_rows<double><<<(unsigned)n, 128, 0, st>>>(
        drows.as<int64_t>(), n, h->d_u2s.as<int>(), h->d_grow_cell.as<int>(),
        h->d_cell_pstart.as<int>(), h->d_cover_off.as<int>(), h->d_cover_sub.as<int>(),
        h->d_cover_start.as<int>(), h->d_entry_base.as<int64_t>(), h->d_panels.as<double>(), h->K,
        h->NPhi, h->d_h.as<double>(), dout.as<double>(), dh.as<double>());
  else
    k_export_rows<float><<<(unsigned)n, 128, 0, st>>>(
        drows.as<int64_t>(), n, h->d_u2s.as<int>(), h->d_grow_cell.as<int>(),
        h->d_cell_pstart.as<int>(), h->d_cover_off.as<int>(), h->d_cover_sub.as<int>(),
        h->d_cover_start.as<int>(), h->d_entry_base.as<int64_t>(), h->d_panels.as<float>(), h->K,
        h->NPhi, h->d_h.as<double>(), dout.as<double>(), dh.as<double>());
  check_launch("k_export_rows");
  count_launch(h);
  CUDA_CHECK(cudaMemcpyAsync(out, dout.p, n * h->NPhi * sizeof(double), cudaMemcpyDefault, st));
  if (h_out) CUDA_CHECK(cudaMemcpyAsync(h_out, dh.p, n * sizeof(double), cudaMemcpyDefault, st));
  stream_sync(h);
}

// Per-entry 32-row tiles of the panels, (entry, first row), for the QR's
// densification: made on the first call after an assembly.
void ensure_qr_tiles(elmfb_ctx* h) {
  if (h->n_tiles >= 0) return;
  const int ne = (int)h->cover_sub.size();
  std::vector<int> ent(ne);
  std::vector<int64_t> off(ne + 1, 0);
  for (int e = 0; e < ne; ++e) {
    const int c = h->entry_cell[e];
    ent[e] = e;
    off[e + 1] = off[e] + ceil_div(h->cell_pstart[c + 1] - h->cell_pstart[c], 32);
  }
  expand_entry_steps(h, ent, off, 32, h->d_tiles);
  h->n_tiles = off[ne];
}

void expand_entry_steps(elmfb_ctx* h, const std::vector<int>& ent, const std::vector<int64_t>& off,
                        int rows, DevBuf& out) {
  cudaStream_t st = h->stream;
  const int ng = (int)ent.size();
  out.alloc(std::max<int64_t>(off.back(), 1) * sizeof(int2), st);
  if (ng == 0) return;
  DevBuf de, doff;
  de.alloc(ng * sizeof(int), st);
  doff.alloc((ng + 1) * sizeof(int64_t), st);
  CUDA_CHECK(cudaMemcpyAsync(de.p, ent.data(), ng * sizeof(int), cudaMemcpyHostToDevice, st));
  CUDA_CHECK(cudaMemcpyAsync(doff.p, off.data(), (ng + 1) * sizeof(int64_t),
                             cudaMemcpyHostToDevice, st));
  k_expand_steps<<<(unsigned)ng, 128, 0, st>>>(de.as<int>(), doff.as<int64_t>(), ng, rows,
                                               out.as<int2>());
  check_launch("k_expand_steps");
  count_launch(h);
}
