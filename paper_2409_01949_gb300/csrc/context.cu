// Handle lifetime, geometry, random parameters and the thin ABI wrappers.
//
// Geometry follows the paper's §4.1 "Domain decomposition": per level a
// uniform tensor grid of n^d subdomains with centres mu and half-width
// sigma = delta * spacing / 2.  The random hidden parameters follow §4.1
// "weight initialisation" (U(-a, a)), drawn from SplitMix64 (Steele, Lea &
// Flood 2014) by the counter stream documented in elmfb.h.
//
// Besides the paper's quantities this file builds the "cells": the common
// refinement of every subdomain support along each dimension.  Every cell lies
// entirely inside or outside each support, so all points of a cell share one
// set of covering subdomains; the row layout of the panels and the Gram pair
// structure are built on it.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <map>
#include <mutex>
#include <new>
#include <utility>

#include "elmfb_internal.cuh"

namespace {

__host__ __device__ inline uint64_t splitmix64_mix(uint64_t z) {
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
  return z ^ (z >> 31);
}
__host__ __device__ inline uint64_t splitmix64_at(uint64_t seed, uint64_t i) {
  return splitmix64_mix(seed + (i + 1) * 0x9E3779B97F4A7C15ULL);
}

// The random parameters of every column, on the device: column q (of kept
// subdomain q / K) takes the draws of its full-grid column qf, outputs
// qf (d + 1) + p of the stream, u = the top 24 bits / 2^24, value a (2u - 1);
// W and b in FP64 and FP32.
__global__ void k_params(uint64_t seed, double a, int d, int K, int64_t n_cols,
                         const int* __restrict__ param_sub, double* __restrict__ W64,
                         double* __restrict__ b64, float* __restrict__ W32,
                         float* __restrict__ b32) {
  for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < n_cols;
       q += (int64_t)gridDim.x * blockDim.x) {
    const int64_t qf = (int64_t)param_sub[q / K] * K + q % K;
    for (int p = 0; p <= d; ++p) {
      const uint64_t z = splitmix64_at(seed, (uint64_t)qf * (d + 1) + p);
      const double u = (double)(z >> 40) * (1.0 / 16777216.0);
      const double v = a * (2.0 * u - 1.0);
      if (p < d) {
        W64[q * d + p] = v;
        W32[q * d + p] = (float)v;
      } else {
        b64[q] = v;
        b32[q] = (float)v;
      }
    }
  }
}

template <class F>
int guarded(elmfb_ctx* h, F&& f) {
  if (!h) return ELMFB_ERR_INVALID_ARG;
  try {
    CUDA_CHECK(cudaSetDevice(h->device));
    h->err.clear();
    f();
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

// Drop every subdomain whose centre lies inside a hole box (strictly between
// its faces, a face on the domain box's boundary counting as part of the
// hole; paper §4.1, the L-shaped domain of §4.4) and renumber the rest in
// order: the geometry, the parameter sources (the full-grid subdomain whose
// draws a kept one keeps), the cell ranges and the covering lists are
// compacted.
void discard_in_holes(elmfb_ctx* h) {
  const elmfb_config& c = h->cfg;
  const int nfull = h->n_sub;
  std::vector<int> map(nfull, -1);
  int kept = 0;
  for (int s = 0; s < nfull; ++s) {
    bool in_hole = false;
    for (int k = 0; k < c.n_holes && !in_hole; ++k) {
      bool inside = true;
      for (int i = 0; i < h->dim; ++i) {
        // strictly between the hole's faces; a face on the domain box's
        // boundary belongs to the hole
        const double m = h->sub[s].mu[i], hl = c.holes[k][i], hh = c.holes[k][2 + i];
        const bool above = m > hl || (hl == c.lo[i] && m == c.lo[i]);
        const bool below = m < hh || (hh == c.hi[i] && m == c.hi[i]);
        inside = inside && above && below;
      }
      in_hole = inside;
    }
    if (!in_hole) map[s] = kept++;
  }
  if (kept == 0) ELMFB_THROW(ELMFB_ERR_INVALID_ARG, "every subdomain lies inside a hole");
  const int K = h->K;
  std::vector<SubGeom> sub(kept);
  std::vector<int> psub(kept);
  std::vector<int> c0[2], c1[2];
  for (int i = 0; i < 2; ++i) {
    c0[i].resize(kept);
    c1[i].resize(kept);
  }
  std::vector<int> lev_off(h->L + 1, 0);
  for (int s = 0; s < nfull; ++s) {
    const int t = map[s];
    if (t < 0) continue;
    sub[t] = h->sub[s];
    psub[t] = h->param_sub[s];
    lev_off[h->sub[s].level + 1]++;
    for (int i = 0; i < 2; ++i) {
      c0[i][t] = h->sub_c0[i][s];
      c1[i][t] = h->sub_c1[i][s];
    }
  }
  for (int l = 0; l < h->L; ++l) lev_off[l + 1] += lev_off[l];
  std::vector<int> cover_off(h->n_cells + 1, 0), cover_sub;
  std::vector<int> cell_level_off((size_t)h->n_cells * (h->L + 1), 0);
  int max_cover = 0;
  for (int cell = 0; cell < h->n_cells; ++cell) {
    cover_off[cell] = (int)cover_sub.size();
    for (int l = 0; l <= h->L; ++l) {
      const size_t li = (size_t)cell * (h->L + 1) + l;
      cell_level_off[li] = (int)cover_sub.size();
      if (l == h->L) break;
      for (int e = h->cell_level_off[li]; e < h->cell_level_off[li + 1]; ++e)
        if (map[h->cover_sub[e]] >= 0) cover_sub.push_back(map[h->cover_sub[e]]);
    }
    max_cover = std::max(max_cover, (int)cover_sub.size() - cover_off[cell]);
  }
  cover_off[h->n_cells] = (int)cover_sub.size();
  h->sub.swap(sub);
  h->param_sub.swap(psub);
  for (int i = 0; i < 2; ++i) {
    h->sub_c0[i].swap(c0[i]);
    h->sub_c1[i].swap(c1[i]);
  }
  h->lev_sub_off.swap(lev_off);
  h->cover_off.swap(cover_off);
  h->cover_sub.swap(cover_sub);
  h->cell_level_off.swap(cell_level_off);
  h->max_cover = max_cover;
  h->n_sub = kept;
  h->NPhi = (int64_t)kept * K;
}

void build_geometry(elmfb_ctx* h) {
  const elmfb_config& c = h->cfg;
  h->dim = c.dim;
  h->L = c.n_levels;
  h->K = c.features;
  h->lev_n.assign(c.levels, c.levels + c.n_levels);
  h->lev_sub_off.assign(h->L + 1, 0);
  for (int l = 0; l < h->L; ++l) {
    int J = 1;
    for (int i = 0; i < h->dim; ++i) J *= h->lev_n[l];
    h->lev_sub_off[l + 1] = h->lev_sub_off[l] + J;
  }
  h->n_sub = h->lev_sub_off[h->L];
  h->NPhi = (int64_t)h->n_sub * h->K;

  // centres and half-widths per level and dimension
  std::vector<std::vector<double>> mu(h->L * 2);
  std::vector<double> sig(h->L * 2, 0.0);
  for (int l = 0; l < h->L; ++l) {
    int n = h->lev_n[l];
    for (int i = 0; i < h->dim; ++i) {
      double lo = c.lo[i], hi = c.hi[i], D;
      std::vector<double>& m = mu[l * 2 + i];
      m.resize(n);
      if (c.placement == ELMFB_PLACE_CELL) {
        D = (hi - lo) / n;
        for (int j = 0; j < n; ++j) m[j] = lo + (j + 0.5) * D;
      } else {
        if (n == 1) {
          D = hi - lo;
          m[0] = 0.5 * (lo + hi);
        } else {
          D = (hi - lo) / (n - 1);
          for (int j = 0; j < n; ++j) m[j] = lo + j * D;
        }
      }
      sig[l * 2 + i] = c.delta * D / 2.0;
    }
  }
  h->sub.resize(h->n_sub);
  for (int l = 0; l < h->L; ++l) {
    int n = h->lev_n[l];
    for (int j = h->lev_sub_off[l]; j < h->lev_sub_off[l + 1]; ++j) {
      int loc = j - h->lev_sub_off[l];
      int ji[2] = {loc % n, h->dim == 2 ? loc / n : 0};
      SubGeom g{};
      for (int i = 0; i < 2; ++i) {
        if (i < h->dim) {
          g.mu[i] = mu[l * 2 + i][ji[i]];
          g.sigma_d[i] = sig[l * 2 + i];
          g.inv_sigma_d[i] = 1.0 / sig[l * 2 + i];
          g.inv_sigma[i] = (float)g.inv_sigma_d[i];
        } else {
          g.mu[i] = 0.0;
          g.sigma_d[i] = 1.0;
          g.inv_sigma_d[i] = 0.0;
          g.inv_sigma[i] = 0.f;
        }
      }
      g.level = l;
      h->sub[j] = g;
    }
  }

  // random parameters (drawn on the device, k_params): column q draws
  // outputs q*(d+1)+p of the stream; each subdomain is its own source until
  // subdomains in holes are discarded
  h->param_sub.resize(h->n_sub);
  for (int s = 0; s < h->n_sub; ++s) h->param_sub[s] = s;

  // cells: common refinement of all supports, per dimension
  for (int i = 0; i < 2; ++i) {
    h->bnd[i].clear();
    h->sub_c0[i].assign(h->n_sub, 0);
    h->sub_c1[i].assign(h->n_sub, 1);
    if (i >= h->dim) {
      h->bnd[i] = {0.0, 1.0};
      h->nc[i] = 1;
      continue;
    }
    double lo = c.lo[i], hi = c.hi[i];
    double tol = 1e-12 * (hi - lo);
    std::vector<double> b = {lo, hi};
    for (int l = 0; l < h->L; ++l)
      for (double m : mu[l * 2 + i]) {
        double e0 = m - sig[l * 2 + i], e1 = m + sig[l * 2 + i];
        if (e0 > lo + tol && e0 < hi - tol) b.push_back(e0);
        if (e1 > lo + tol && e1 < hi - tol) b.push_back(e1);
      }
    std::sort(b.begin(), b.end());
    std::vector<double> u;
    for (double v : b)
      if (u.empty() || v > u.back() + tol) u.push_back(v);
    u.back() = hi;
    h->bnd[i] = u;
    h->nc[i] = (int)u.size() - 1;
    // cell range of each subdomain along this dimension
    for (int s = 0; s < h->n_sub; ++s) {
      int l = h->sub[s].level;
      double e0 = h->sub[s].mu[i] - sig[l * 2 + i], e1 = h->sub[s].mu[i] + sig[l * 2 + i];
      int c0 = h->nc[i], c1 = 0;
      for (int cc = 0; cc < h->nc[i]; ++cc) {
        if (u[cc] >= e0 - tol && u[cc + 1] <= e1 + tol) {
          c0 = std::min(c0, cc);
          c1 = std::max(c1, cc + 1);
        }
      }
      if (c1 <= c0) c0 = c1 = 0;  // support misses the box entirely
      h->sub_c0[i][s] = c0;
      h->sub_c1[i][s] = c1;
    }
  }
  h->n_cells = h->nc[0] * h->nc[1];

  // covering index range per level, dimension and cell coordinate
  std::vector<int> jlo((size_t)h->L * 2 * std::max(h->nc[0], h->nc[1])),
      jhi(jlo.size());
  auto rix = [&](int l, int i, int cc) { return ((size_t)l * 2 + i) * std::max(h->nc[0], h->nc[1]) + cc; };
  for (int l = 0; l < h->L; ++l) {
    int n = h->lev_n[l];
    for (int i = 0; i < 2; ++i)
      for (int cc = 0; cc < h->nc[i]; ++cc) {
        int lo_j = n, hi_j = 0;
        if (i >= h->dim) {
          lo_j = 0;
          hi_j = 1;
        } else {
          for (int j = 0; j < n; ++j) {
            int s = h->lev_sub_off[l] + (i == 0 ? j : j * n);
            if (cc >= h->sub_c0[i][s] && cc < h->sub_c1[i][s]) {
              lo_j = std::min(lo_j, j);
              hi_j = std::max(hi_j, j + 1);
            }
          }
        }
        if (hi_j <= lo_j)
          ELMFB_THROW(ELMFB_ERR_INVALID_ARG,
                      "level " + std::to_string(l) +
                          " leaves part of the domain uncovered (width ratio too small)");
        jlo[rix(l, i, cc)] = lo_j;
        jhi[rix(l, i, cc)] = hi_j;
      }
  }
  // covering subdomains per cell, grouped by level, increasing subdomain id
  h->cover_off.assign(h->n_cells + 1, 0);
  h->cell_level_off.assign((size_t)h->n_cells * (h->L + 1), 0);
  h->cover_sub.clear();
  h->max_cover = 0;
  for (int cy = 0; cy < h->nc[1]; ++cy)
    for (int cx = 0; cx < h->nc[0]; ++cx) {
      int cell = cy * h->nc[0] + cx;
      h->cover_off[cell] = (int)h->cover_sub.size();
      for (int l = 0; l < h->L; ++l) {
        h->cell_level_off[(size_t)cell * (h->L + 1) + l] = (int)h->cover_sub.size();
        int n = h->lev_n[l];
        for (int jy = jlo[rix(l, 1, cy)]; jy < jhi[rix(l, 1, cy)]; ++jy)
          for (int jx = jlo[rix(l, 0, cx)]; jx < jhi[rix(l, 0, cx)]; ++jx)
            h->cover_sub.push_back(h->lev_sub_off[l] + jy * n + jx);
      }
      h->cell_level_off[(size_t)cell * (h->L + 1) + h->L] = (int)h->cover_sub.size();
      h->max_cover = std::max(h->max_cover, (int)h->cover_sub.size() - h->cover_off[cell]);
    }
  h->cover_off[h->n_cells] = (int)h->cover_sub.size();
  if (c.n_holes > 0) discard_in_holes(h);
  h->entry_cell.resize(h->cover_sub.size());
  for (int cell = 0; cell < h->n_cells; ++cell)
    for (int e = h->cover_off[cell]; e < h->cover_off[cell + 1]; ++e) h->entry_cell[e] = cell;
}

template <class T>
void upload(elmfb_ctx* h, DevBuf& b, const std::vector<T>& v) {
  b.alloc(std::max<size_t>(v.size(), 1) * sizeof(T), h->stream);
  if (!v.empty())
    CUDA_CHECK(cudaMemcpyAsync(b.p, v.data(), v.size() * sizeof(T), cudaMemcpyHostToDevice,
                               h->stream));
}

}  // namespace

cudaMemPool_t library_pool() {
  static std::mutex mu;
  static std::map<int, cudaMemPool_t> pools;
  int dev = 0;
  CUDA_CHECK(cudaGetDevice(&dev));
  std::lock_guard<std::mutex> lock(mu);
  auto it = pools.find(dev);
  if (it != pools.end()) return it->second;
  cudaMemPoolProps props{};
  props.allocType = cudaMemAllocationTypePinned;
  props.location.type = cudaMemLocationTypeDevice;
  props.location.id = dev;
  cudaMemPool_t pool = nullptr;
  CUDA_CHECK(cudaMemPoolCreate(&pool, &props));
  uint64_t keep = UINT64_MAX;
  CUDA_CHECK(cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &keep));
  pools[dev] = pool;
  return pool;
}

void ensure_dyn_smem(const void* func, size_t bytes, bool max_carveout) {
  static std::mutex mu;
  static std::map<std::pair<int, const void*>, size_t> limit;
  int dev = 0;
  CUDA_CHECK(cudaGetDevice(&dev));
  std::lock_guard<std::mutex> lock(mu);
  // the default limit covers static plus dynamic memory, so opt in to at
  // least 48 KB of dynamic memory whenever a kernel asks
  const size_t want = std::max<size_t>(bytes, 48 * 1024);
  size_t& cur = limit[{dev, func}];
  if (cur == 0 && max_carveout)   // several CTAs of it share an SM's shared memory
    CUDA_CHECK(cudaFuncSetAttribute(func, cudaFuncAttributePreferredSharedMemoryCarveout,
                                    (int)cudaSharedmemCarveoutMaxShared));
  if (want <= cur) return;
  CUDA_CHECK(cudaFuncSetAttribute(func, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)want));
  cur = want;
}

void stream_sync(elmfb_ctx* h) {
  if (!h->blocking_sync) {
    CUDA_CHECK(cudaStreamSynchronize(h->stream));
    return;
  }
  if (!h->sync_ev)
    CUDA_CHECK(cudaEventCreateWithFlags(&h->sync_ev,
                                        cudaEventBlockingSync | cudaEventDisableTiming));
  CUDA_CHECK(cudaEventRecord(h->sync_ev, h->stream));
  CUDA_CHECK(cudaEventSynchronize(h->sync_ev));
}

void check_launch(const char* what) {
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess)
    ELMFB_THROW(ELMFB_ERR_CUDA, std::string(what) + ": " + cudaGetErrorString(e));
}

void stage_begin(elmfb_ctx* h, int s) { CUDA_CHECK(cudaEventRecord(h->st[s].a, h->stream)); }
void stage_end(elmfb_ctx* h, int s) {
  CUDA_CHECK(cudaEventRecord(h->st[s].b, h->stream));
  stream_sync(h);
  float ms = 0.f;
  CUDA_CHECK(cudaEventElapsedTime(&ms, h->st[s].a, h->st[s].b));
  h->stage_ms[s] = ms;
}

namespace {
cudaEvent_t prof_event(elmfb_ctx* h) {
  if (!h->prof_pool.empty()) {
    cudaEvent_t e = h->prof_pool.back();
    h->prof_pool.pop_back();
    return e;
  }
  cudaEvent_t e;
  CUDA_CHECK(cudaEventCreate(&e));
  return e;
}
const char* kKernelNames[KID_COUNT] = {"assemble_panels", "gather_Mv",    "entry_MTu",
                                       "panel_MTu",       "precond_apply", "lsqr_update",
                                       "gram_diag",       "block_chol",   "gram_tc",
                                       "cell_sort",       "fused_Mt_MTu",  "gram_spmv"};
}  // namespace

void prof_begin(elmfb_ctx* h, int kid, double bytes) {
  if (!h->prof || !((h->prof_mask >> kid) & 1)) return;
  const int64_t seq = h->prof_seen[kid]++;
  h->prof_now[kid] = seq % h->prof_stride == 0;
  if (!h->prof_now[kid]) return;
  ProfRec r{kid, prof_event(h), prof_event(h), seq};
  CUDA_CHECK(cudaEventRecord(r.a, h->stream));
  h->prof_live.push_back(r);
  h->prof_bytes[kid] = bytes;
}

void prof_end(elmfb_ctx* h, int kid) {
  if (!h->prof || !((h->prof_mask >> kid) & 1) || !h->prof_now[kid]) return;
  for (auto it = h->prof_live.rbegin(); it != h->prof_live.rend(); ++it)
    if (it->kid == kid) {
      CUDA_CHECK(cudaEventRecord(it->b, h->stream));
      break;
    }
  // the most recent records stay live: a solve may still drop them
  if (h->prof_live.size() > 4096) prof_harvest(h, 256);
}

void prof_harvest(elmfb_ctx* h, size_t keep) {
  if (h->prof_live.size() <= keep) return;
  const size_t n = h->prof_live.size() - keep;
  stream_sync(h);
  for (size_t i = 0; i < n; ++i) {
    const ProfRec& r = h->prof_live[i];
    float ms = 0.f;
    CUDA_CHECK(cudaEventElapsedTime(&ms, r.a, r.b));
    h->prof_ms[r.kid] += ms;
    h->prof_n[r.kid] += 1;
    h->prof_pool.push_back(r.a);
    h->prof_pool.push_back(r.b);
  }
  h->prof_live.erase(h->prof_live.begin(), h->prof_live.begin() + n);
}

void prof_drop_from(elmfb_ctx* h, int kid, int64_t from) {
  auto& v = h->prof_live;
  size_t w = 0;
  for (size_t i = 0; i < v.size(); ++i) {
    if (v[i].kid == kid && v[i].seq >= from) {
      h->prof_pool.push_back(v[i].a);
      h->prof_pool.push_back(v[i].b);
    } else {
      v[w++] = v[i];
    }
  }
  v.resize(w);
}

void upload_geometry(elmfb_ctx* h) {
  upload(h, h->d_sub, h->sub);
  {
    cudaStream_t st = h->stream;
    const int d = h->dim;
    DevBuf dps;
    upload(h, dps, h->param_sub);
    h->d_W64.alloc(std::max<int64_t>(h->NPhi * d, 1) * sizeof(double), st);
    h->d_b64.alloc(std::max<int64_t>(h->NPhi, 1) * sizeof(double), st);
    h->d_W32.alloc(std::max<int64_t>(h->NPhi * d, 1) * sizeof(float), st);
    h->d_b32.alloc(std::max<int64_t>(h->NPhi, 1) * sizeof(float), st);
    k_params<<<(unsigned)std::min<int64_t>(ceil_div(h->NPhi, 256), 1216), 256, 0, st>>>(
        h->cfg.seed, h->cfg.weight_scale, d, h->K, h->NPhi, dps.as<int>(), h->d_W64.as<double>(),
        h->d_b64.as<double>(), h->d_W32.as<float>(), h->d_b32.as<float>());
    check_launch("k_params");
    count_launch(h);
  }
  std::vector<double> bnd(h->bnd[0]);
  bnd.insert(bnd.end(), h->bnd[1].begin(), h->bnd[1].end());
  upload(h, h->d_bnd, bnd);
  upload(h, h->d_cover_off, h->cover_off);
  upload(h, h->d_cover_sub, h->cover_sub);
  upload(h, h->d_cell_level_off, h->cell_level_off);
  upload(h, h->d_entry_cell, h->entry_cell);
  h->d_a.alloc(h->NPhi * sizeof(double), h->stream);
  CUDA_CHECK(cudaMemsetAsync(h->d_a.p, 0, h->NPhi * sizeof(double), h->stream));
  h->d_flags.alloc(16 * sizeof(int), h->stream);
  CUDA_CHECK(cudaMemsetAsync(h->d_flags.p, 0, 16 * sizeof(int), h->stream));
}

extern "C" {

int elmfb_create(elmfb_t* out, const elmfb_config* cfg, void* cuda_stream) {
  if (!out || !cfg) return ELMFB_ERR_INVALID_ARG;
  *out = nullptr;
  const elmfb_config& c = *cfg;
  if (c.dim < 1 || c.dim > 2 || c.n_levels < 1 || c.n_levels > ELMFB_MAX_LEVELS ||
      c.features < 1 || c.features > ELMFB_MAX_FEATURES || !(c.delta > 1.0) ||
      (c.placement != ELMFB_PLACE_CELL && c.placement != ELMFB_PLACE_ENDPOINT) ||
      c.precision < ELMFB_FP64 || c.precision > ELMFB_FP32_DF32 || !(c.weight_scale >= 0.0))
    return ELMFB_ERR_INVALID_ARG;
  for (int i = 0; i < c.dim; ++i)
    if (!(c.hi[i] > c.lo[i])) return ELMFB_ERR_INVALID_ARG;
  if (c.n_holes < 0 || c.n_holes > ELMFB_MAX_HOLES || !(c.ansatz_omega >= 0.0))
    return ELMFB_ERR_INVALID_ARG;
  int64_t nsub = 0;
  for (int l = 0; l < c.n_levels; ++l) {
    if (c.levels[l] < 1 || c.levels[l] > 4096) return ELMFB_ERR_INVALID_ARG;
    nsub += c.dim == 2 ? (int64_t)c.levels[l] * c.levels[l] : c.levels[l];
  }
  if (nsub * c.features > (int64_t)1 << 30) return ELMFB_ERR_UNSUPPORTED;
  elmfb_ctx* h = new (std::nothrow) elmfb_ctx();   // no exception crosses the C ABI
  if (!h) return ELMFB_ERR_OOM;
  h->cfg = c;
  h->stream = (cudaStream_t)cuda_stream;
  cudaGetDevice(&h->device);
  int rc = guarded(h, [&] {
    for (auto& s : h->st) {
      CUDA_CHECK(cudaEventCreate(&s.a));
      CUDA_CHECK(cudaEventCreate(&s.b));
    }
    stage_begin(h, 0);
    build_geometry(h);
    upload_geometry(h);
    stage_end(h, 0);
  });
  if (rc != ELMFB_OK) {
    elmfb_destroy(h);
    return rc;
  }
  *out = h;
  return ELMFB_OK;
}

void elmfb_destroy(elmfb_t h) {
  if (!h) return;
  cudaSetDevice(h->device);
  cudaStream_t st = h->stream;
  cudaStreamSynchronize(st);
  for (auto& s : h->st) {
    if (s.a) cudaEventDestroy(s.a);
    if (s.b) cudaEventDestroy(s.b);
  }
  for (auto& r : h->prof_live) {
    cudaEventDestroy(r.a);
    cudaEventDestroy(r.b);
  }
  for (auto e : h->prof_pool) cudaEventDestroy(e);
  if (h->sync_ev) cudaEventDestroy(h->sync_ev);
  delete h;  // DevBuf destructors free device memory, ordered on the handle's stream
  cudaStreamSynchronize(st);
}

const char* elmfb_last_error(elmfb_t h) { return h ? h->err.c_str() : "null handle"; }

int elmfb_assemble(elmfb_t h, int n_sets, const elmfb_rowset* sets) {
  return guarded(h, [&] {
    if (n_sets < 1 || n_sets > ELMFB_MAX_ROWSETS || !sets)
      ELMFB_THROW(ELMFB_ERR_INVALID_ARG, "n_sets must be in 1..16");
    assemble_system(h, n_sets, sets);
  });
}

int elmfb_get_sizes(elmfb_t h, elmfb_sizes* o) {
  return guarded(h, [&] {
    if (!o) ELMFB_THROW(ELMFB_ERR_INVALID_ARG, "null output");
    o->n_columns = h->NPhi;
    o->n_rows = h->assembled ? h->n_rows : 0;
    o->n_subdomains = h->n_sub;
    o->nnz = h->assembled ? h->nnz : 0;
    o->panel_rows = h->assembled ? h->NPR : 0;
    o->n_cells = h->n_cells;
    if (h->assembled && h->n_gram_pairs < 0) h->n_gram_pairs = count_gram_pairs(h);
    o->n_gram_pairs = h->assembled ? h->n_gram_pairs : 0;
    o->gram_flops = h->gram_flops;
    o->features = h->K;
    o->n_levels = h->L;
    o->dim = h->dim;
    o->precision = h->cfg.precision;
  });
}

int elmfb_get_params(elmfb_t h, double* W, double* b) {
  return guarded(h, [&] {
    if (W)
      CUDA_CHECK(cudaMemcpyAsync(W, h->d_W64.p, h->NPhi * h->dim * sizeof(double),
                                 cudaMemcpyDefault, h->stream));
    if (b)
      CUDA_CHECK(cudaMemcpyAsync(b, h->d_b64.p, h->NPhi * sizeof(double), cudaMemcpyDefault,
                                 h->stream));
    stream_sync(h);
  });
}

int elmfb_get_rows(elmfb_t h, const int64_t* rows, int64_t n, double* out, double* h_out) {
  return guarded(h, [&] {
    if (!h->assembled) ELMFB_THROW(ELMFB_ERR_STATE, "get_rows before assemble");
    if (n < 0 || (n > 0 && (!rows || !out))) ELMFB_THROW(ELMFB_ERR_INVALID_ARG, "bad arguments");
    export_rows(h, rows, n, out, h_out);
  });
}

void elmfb_default_solve_opts(elmfb_solve_opts* o) {
  if (!o) return;
  o->method = ELMFB_SOLVE_LSQR;
  o->preconditioner = ELMFB_PREC_BLOCK_JACOBI;
  o->max_iter = 15000;
  o->atol = 1e-10;
  o->btol = 1e-10;
  o->shift = 1e-12;
  o->check_every = 50;
  o->warm_start = 0;
  o->refine = 1;
  o->gram_shift = 0.0;
  o->rcond = 1e-13;
  o->ntol = 0.0;
  o->coarse_levels = 2;
  o->autotune = 0;
  o->graph = 0;
  o->batch_shared = 1;
  o->drop_tol = 0.0;
}

int elmfb_solve(elmfb_t h, const elmfb_solve_opts* opts, elmfb_solve_info* info) {
  int nc_status = ELMFB_OK;
  int rc = guarded(h, [&] {
    if (!h->assembled) ELMFB_THROW(ELMFB_ERR_STATE, "solve before assemble");
    elmfb_solve_opts o;
    elmfb_default_solve_opts(&o);
    if (opts) o = *opts;
    if (o.max_iter < 0 || o.check_every < 1 || !(o.shift >= 0.0) || o.refine < 1 ||
        !(o.gram_shift >= 0.0) || !(o.rcond >= 0.0) || !(o.ntol >= 0.0) ||
        !(o.drop_tol >= 0.0 && o.drop_tol < 1.0))
      ELMFB_THROW(ELMFB_ERR_INVALID_ARG, "bad solver options");
    elmfb_solve_info inf{};
    h->gk_alpha.clear();
    h->gk_beta.clear();
    solve_system(h, &o, &inf);
    h->have_coeffs = true;
    nc_status = inf.status;
    if (info) *info = inf;
  });
  if (rc != ELMFB_OK) return rc;
  return nc_status;
}

int elmfb_get_bidiagonal(elmfb_t h, int64_t max, double* alpha, double* beta, int64_t* k_out) {
  return guarded(h, [&] {
    if (max < 0) ELMFB_THROW(ELMFB_ERR_INVALID_ARG, "negative max");
    const int64_t n = (int64_t)h->gk_alpha.size();
    if (k_out) *k_out = n > 0 ? n - 1 : 0;
    const int64_t c = std::min<int64_t>(n, max);
    if (alpha && c > 0)
      CUDA_CHECK(cudaMemcpy(alpha, h->gk_alpha.data(), c * sizeof(double), cudaMemcpyDefault));
    if (beta && c > 0)
      CUDA_CHECK(cudaMemcpy(beta, h->gk_beta.data(), c * sizeof(double), cudaMemcpyDefault));
  });
}

int elmfb_get_coeffs(elmfb_t h, double* a) {
  return guarded(h, [&] {
    if (!a) ELMFB_THROW(ELMFB_ERR_INVALID_ARG, "null output");
    CUDA_CHECK(cudaMemcpyAsync(a, h->d_a.p, h->NPhi * sizeof(double), cudaMemcpyDefault,
                               h->stream));
    stream_sync(h);
  });
}

int elmfb_set_coeffs(elmfb_t h, const double* a) {
  return guarded(h, [&] {
    if (!a) ELMFB_THROW(ELMFB_ERR_INVALID_ARG, "null input");
    CUDA_CHECK(cudaMemcpyAsync(h->d_a.p, a, h->NPhi * sizeof(double), cudaMemcpyDefault,
                               h->stream));
    stream_sync(h);
    h->have_coeffs = true;
  });
}

int elmfb_eval(elmfb_t h, const double* xs, int64_t n, double* out) {
  return guarded(h, [&] {
    if (n < 0 || (n > 0 && (!xs || !out))) ELMFB_THROW(ELMFB_ERR_INVALID_ARG, "bad arguments");
    eval_model(h, xs, n, out);
  });
}

int elmfb_error_norms(elmfb_t h, const double* uh, const double* ur, int64_t n, double* out3) {
  return guarded(h, [&] {
    if (n <= 0 || !uh || !ur || !out3) ELMFB_THROW(ELMFB_ERR_INVALID_ARG, "bad arguments");
    error_norms(h, uh, ur, n, out3);
  });
}

int elmfb_stage_times(elmfb_t h, double* ms) {
  return guarded(h, [&] {
    if (!ms) ELMFB_THROW(ELMFB_ERR_INVALID_ARG, "null output");
    for (int i = 0; i < ELMFB_N_STAGES; ++i) ms[i] = h->stage_ms[i];
  });
}

int64_t elmfb_kernel_launches(elmfb_t h) { return h ? h->launches : -1; }

int elmfb_trim_memory(int device) {
  int cur = 0;
  if (cudaGetDevice(&cur) != cudaSuccess) return ELMFB_ERR_CUDA;
  if (device < 0) device = cur;
  if (cudaSetDevice(device) != cudaSuccess) return ELMFB_ERR_INVALID_ARG;
  int rc = ELMFB_OK;
  try {
    if (cudaDeviceSynchronize() != cudaSuccess ||
        cudaMemPoolTrimTo(library_pool(), 0) != cudaSuccess)
      rc = ELMFB_ERR_CUDA;
  } catch (...) {
    rc = ELMFB_ERR_CUDA;
  }
  cudaSetDevice(cur);
  return rc;
}

int elmfb_set_profiling_only(elmfb_t h, const char* kernel) {
  return guarded(h, [&] {
    if (!kernel) ELMFB_THROW(ELMFB_ERR_INVALID_ARG, "null kernel name");
    int kid = -1;
    for (int k = 0; k < KID_COUNT; ++k)
      if (std::strcmp(kernel, kKernelNames[k]) == 0) kid = k;
    if (kid < 0) ELMFB_THROW(ELMFB_ERR_INVALID_ARG, "unknown kernel name");
    prof_harvest(h);
    h->prof = true;
    h->prof_mask = uint64_t(1) << kid;
    for (int k = 0; k < KID_COUNT; ++k) {
      h->prof_ms[k] = 0.0;
      h->prof_n[k] = 0;
    }
  });
}

int elmfb_set_profiling_stride(elmfb_t h, int stride) {
  return guarded(h, [&] {
    if (stride < 1) ELMFB_THROW(ELMFB_ERR_INVALID_ARG, "profiling stride must be >= 1");
    h->prof_stride = stride;
    for (int k = 0; k < KID_COUNT; ++k) h->prof_seen[k] = 0;
  });
}

int elmfb_set_profiling(elmfb_t h, int on) {
  return guarded(h, [&] {
    prof_harvest(h);
    h->prof = on != 0;
    h->prof_mask = ~uint64_t(0);
    for (int k = 0; k < KID_COUNT; ++k) {
      h->prof_ms[k] = 0.0;
      h->prof_n[k] = 0;
    }
  });
}

int elmfb_kernel_stats(elmfb_t h, int max, const char** names, double* total_ms, int64_t* launches,
                       double* bytes_per_launch) {
  int count = 0;
  int rc = guarded(h, [&] {
    prof_harvest(h);
    for (int k = 0; k < KID_COUNT && count < max; ++k) {
      if (h->prof_n[k] == 0) continue;
      if (names) names[count] = kKernelNames[k];
      if (total_ms) total_ms[count] = h->prof_ms[k];
      if (launches) launches[count] = h->prof_n[k];
      if (bytes_per_launch) bytes_per_launch[count] = h->prof_bytes[k];
      ++count;
    }
  });
  return rc == ELMFB_OK ? count : -rc;
}

}  // extern "C"
