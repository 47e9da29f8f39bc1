// Gram blocks G_ij = M_i^T M_j on the tcgen05 tensor cores (BF16 in, FP32
// accumulation in TMEM).
//
// The Gram matrix of the least-squares system (normal equations of Eq.
// multilevel_ls) inherits the block structure of Eq. multilevel_domain_decomp:
// G_ij is nonzero only when the supports of subdomains i and j share
// collocation points, and then it is a dense K x K contraction over those
// rows.  With rows sorted by cells, the shared rows of a pair are a list of
// runs (one per shared cell, merged where both panels continue contiguously),
// each a multiple of 16 rows.
//
// Operands come from the BF16 feature-major copy of the panels written by the
// assembly kernel in mixed precision: PT[k][rho] (rho = panel row).  For one
// pair, A = P_i^T (features x rows) and B = P_j^T are both K-major along the
// contraction, loaded by 2-D TMA boxes of 64 rows x K features with 128-byte
// swizzle into a 4-stage shared-memory ring.  One thread issues
// tcgen05.mma (M = 128, N = K rounded up to 16, 16 rows per instruction) into
// a TMEM accumulator, releasing each stage with tcgen05.commit; all four warps
// then read the accumulator with tcgen05.ld and store the FP32 block.  Rows of
// a box beyond its run are skipped by issuing only the valid 16-row steps.
// Every mbarrier wait is bounded; a timeout raises flags[2].
#include <algorithm>
#include <map>
#include <cstring>

#include <cudaTypedefs.h>

#include <new>
#include <stdexcept>

#include "elmfb_internal.cuh"
#include "sm100_ptx.cuh"

namespace {

constexpr int kStages = 4;
constexpr int kBoxRows = 64;                 // contraction rows per box (128 B of BF16)
constexpr int kTileBytes = 128 * 128;        // 128 feature rows x 128 B
constexpr int kGramThreads = 128;
constexpr size_t kGramSmem = 2 * kStages * kTileBytes + 1024;

__global__ void __launch_bounds__(kGramThreads, 1)
    k_gram_tc(const __grid_constant__ CUtensorMap tmap, const int4* __restrict__ pairs,
              const int4* __restrict__ runs, int K, int N, float* __restrict__ G,
              int* __restrict__ flags) {
  extern __shared__ uint8_t smraw[];
  __shared__ __align__(8) uint64_t full[kStages];
  __shared__ __align__(8) uint64_t empty[kStages];
  __shared__ __align__(8) uint64_t done;
  __shared__ uint32_t tmem_slot;
  uint8_t* sm = reinterpret_cast<uint8_t*>(
      (reinterpret_cast<uintptr_t>(smraw) + 1023) & ~uintptr_t(1023));
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int4 task = pairs[blockIdx.x];   // (first run, end run, diagonal, -)
  const bool diag = task.z != 0;

  if (threadIdx.x == 0) {
    for (int s = 0; s < kStages; ++s) {
      sm100::mbar_init(&full[s], 1);
      sm100::mbar_init(&empty[s], 1);
    }
    sm100::mbar_init(&done, 1);
    sm100::fence_mbar_init();
    sm100::prefetch_tensormap(&tmap);
  }
  if (warp == 2) sm100::tmem_alloc(&tmem_slot, 128);
  // zero the tiles once: feature rows >= K are never written by TMA
  for (int i = threadIdx.x; i < 2 * kStages * kTileBytes / 16; i += blockDim.x)
    reinterpret_cast<uint4*>(sm)[i] = make_uint4(0, 0, 0, 0);
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  sm100::tc_fence_before();
  __syncthreads();
  sm100::tc_fence_after();
  const uint32_t tmem = tmem_slot;
  const uint32_t idesc = sm100::idesc_bf16_f32(128, N);
  const uint32_t box_bytes = (uint32_t)K * 128u;
  int nboxes = 0;
  for (int r = task.x; r < task.y; ++r) nboxes += (runs[r].z + kBoxRows - 1) / kBoxRows;

  if (warp == 0 && lane == 0) {
    // TMA producer
    int b = 0;
    bool ok = true;
    for (int r = task.x; r < task.y && ok; ++r) {
      const int4 run = runs[r];
      for (int off = 0; off < run.z; off += kBoxRows, ++b) {
        const int stage = b % kStages, round = b / kStages;
        if (round > 0 && !sm100::mbar_wait(&empty[stage], (round - 1) & 1)) {
          atomicOr(&flags[2], 1);
          ok = false;
          break;
        }
        uint8_t* a = sm + stage * 2 * kTileBytes;
        sm100::mbar_arrive_expect_tx(&full[stage], diag ? box_bytes : 2 * box_bytes);
        sm100::tma_load_2d(a, &tmap, run.x + off, 0, &full[stage]);
        if (!diag) sm100::tma_load_2d(a + kTileBytes, &tmap, run.y + off, 0, &full[stage]);
      }
    }
  } else if (warp == 1 && lane == 0) {
    // MMA issuer
    int b = 0;
    uint32_t acc = 0;
    bool ok = true;
    for (int r = task.x; r < task.y && ok; ++r) {
      const int4 run = runs[r];
      for (int off = 0; off < run.z; off += kBoxRows, ++b) {
        const int stage = b % kStages, round = b / kStages;
        if (!sm100::mbar_wait(&full[stage], round & 1)) {
          atomicOr(&flags[2], 1);
          ok = false;
          break;
        }
        sm100::tc_fence_after();
        const uint8_t* a = sm + stage * 2 * kTileBytes;
        const uint64_t ad = sm100::sdesc_k_sw128(sm100::smem_u32(a));
        const uint64_t bd = sm100::sdesc_k_sw128(sm100::smem_u32(diag ? a : a + kTileBytes));
        const int ksteps = min(kBoxRows, run.z - off) / 16;
        for (int ks = 0; ks < ksteps; ++ks) {
          // advance 16 BF16 (32 B) along the contraction inside the swizzle atom
          sm100::mma_bf16(tmem, ad + 2 * ks, bd + 2 * ks, idesc, acc);
          acc = 1;
        }
        sm100::mma_commit(&empty[stage]);
      }
    }
    sm100::mma_commit(&done);
  }
  __syncwarp();
  // epilogue: warp w reads TMEM lanes 32w .. 32w+31 (= rows of G_ij)
  const bool got = sm100::mbar_wait(&done, 0);
  sm100::tc_fence_after();
  if (!got && threadIdx.x == 0) atomicOr(&flags[2], 1);
  const int m = 32 * warp + lane;
  float* Gp = G + (int64_t)blockIdx.x * K * K;
  for (int c0 = 0; c0 < N; c0 += 16) {
    uint32_t v[16];
    sm100::tmem_ld16(tmem + ((uint32_t)(32 * warp) << 16) + (uint32_t)c0, v);
    sm100::tmem_ld_wait();
    if (m < K) {
#pragma unroll
      for (int j = 0; j < 16; ++j)
        if (c0 + j < K) Gp[(int64_t)m * K + c0 + j] = nboxes > 0 && got ? __uint_as_float(v[j]) : 0.f;
    }
  }
  sm100::tc_fence_before();
  __syncthreads();
  if (warp == 2) sm100::tmem_dealloc(tmem, 128);
}

// cuTensorMapEncodeTiled from the driver, resolved at run time through the
// runtime's entry-point query (the library does not link libcuda directly).
PFN_cuTensorMapEncodeTiled_v12000 encode_tiled() {
  // thread-safe one-time lookup (function-local static initialisation)
  static PFN_cuTensorMapEncodeTiled_v12000 fn = []() -> PFN_cuTensorMapEncodeTiled_v12000 {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault,
                                         &q) != cudaSuccess ||
        q != cudaDriverEntryPointSuccess)
      return nullptr;
    return reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
  }();
  if (!fn) ELMFB_THROW(ELMFB_ERR_CUDA, "cuTensorMapEncodeTiled is not available from the driver");
  return fn;
}

}  // namespace

// Build the pair / run lists (host) for the assembled system.
void gram_build_pairs(elmfb_ctx* h) {
  struct RunL {
    int a, b, len;
  };
  std::map<std::pair<int, int>, std::vector<RunL>> pr;
  for (int c = 0; c < h->n_cells; ++c) {
    if (h->cell_count[c] == 0) continue;
    const int pad = h->cell_pstart[c + 1] - h->cell_pstart[c];
    for (int e1 = h->cover_off[c]; e1 < h->cover_off[c + 1]; ++e1)
      for (int e2 = e1; e2 < h->cover_off[c + 1]; ++e2) {
        const int s1 = h->cover_sub[e1], s2 = h->cover_sub[e2];
        const int a = (int)(h->panel_off[s1] + h->cover_start[e1]);
        const int b = (int)(h->panel_off[s2] + h->cover_start[e2]);
        auto& v = pr[{s1, s2}];
        if (!v.empty() && v.back().a + v.back().len == a && v.back().b + v.back().len == b)
          v.back().len += pad;
        else
          v.push_back({a, b, pad});
      }
  }
  h->gram_pair_ij.clear();
  std::vector<int4> pairs, runs;
  for (auto& kv : pr) {
    pairs.push_back(make_int4((int)runs.size(), (int)(runs.size() + kv.second.size()),
                              kv.first.first == kv.first.second ? 1 : 0, 0));
    for (auto& r : kv.second) runs.push_back(make_int4(r.a, r.b, r.len, 0));
    h->gram_pair_ij.push_back(kv.first);
  }
  h->n_gram_pairs = (int64_t)pairs.size();
  h->gram_runs = (int64_t)runs.size();
  auto up = [&](DevBuf& d, const std::vector<int4>& v) {
    d.alloc(std::max<size_t>(v.size(), 1) * sizeof(int4), h->stream);
    if (!v.empty())
      CUDA_CHECK(cudaMemcpyAsync(d.p, v.data(), v.size() * sizeof(int4), cudaMemcpyHostToDevice,
                                 h->stream));
  };
  up(h->d_gram_pairs, pairs);
  up(h->d_gram_runs, runs);
}

void gram_compute(elmfb_ctx* h) {
  if (h->cfg.precision != ELMFB_MIXED)
    ELMFB_THROW(ELMFB_ERR_UNSUPPORTED, "tensor-core Gram blocks need ELMFB_MIXED precision");
  if (h->K > 128) ELMFB_THROW(ELMFB_ERR_UNSUPPORTED, "tensor-core Gram blocks need K <= 128");
  cudaStream_t st = h->stream;
  if (h->gram_pair_ij.empty()) gram_build_pairs(h);
  const int K = h->K;
  const int N = (K + 15) & ~15;
  h->d_gram.alloc(std::max<int64_t>(h->n_gram_pairs, 1) * K * K * sizeof(float), st);
  // tensor map over PT[K][NPR] (BF16, rows innermost)
  CUtensorMap tm;
  cuuint64_t gdim[2] = {(cuuint64_t)h->NPR, (cuuint64_t)K};
  cuuint64_t gstride[1] = {(cuuint64_t)h->NPR * 2};
  cuuint32_t box[2] = {(cuuint32_t)kBoxRows, (cuuint32_t)K};
  cuuint32_t estr[2] = {1, 1};
  CUresult r = encode_tiled()(&tm, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, h->d_pt.p, gdim,
                                      gstride, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                                      CU_TENSOR_MAP_SWIZZLE_128B,
                                      CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                                      CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS)
    ELMFB_THROW(ELMFB_ERR_CUDA, "cuTensorMapEncodeTiled failed: " + std::to_string((int)r));
  ensure_dyn_smem((const void*)k_gram_tc, kGramSmem);
  CUDA_CHECK(cudaMemsetAsync(h->d_flags.p, 0, 16 * sizeof(int), st));
  stage_begin(h, 3);
  // algorithmic work: 2 K^2 flops per shared row per pair; bytes: BF16 rows read once
  prof_begin(h, KID_GRAM_TC, (double)h->NPR * K * 2.0 + (double)h->n_gram_pairs * K * K * 4.0);
  if (h->n_gram_pairs > 0)
    k_gram_tc<<<(unsigned)h->n_gram_pairs, kGramThreads, kGramSmem, st>>>(
        tm, h->d_gram_pairs.as<int4>(), h->d_gram_runs.as<int4>(), K, N, h->d_gram.as<float>(),
        h->d_flags.as<int>());
  prof_end(h, KID_GRAM_TC);
  check_launch("k_gram_tc");
  count_launch(h);
  stage_end(h, 3);
  int flags[4];
  CUDA_CHECK(cudaMemcpyAsync(flags, h->d_flags.p, 4 * sizeof(int), cudaMemcpyDeviceToHost, st));
  stream_sync(h);
  if (flags[2]) ELMFB_THROW(ELMFB_ERR_TIMEOUT, "tensor-core Gram: a pipeline wait timed out");
  h->have_gram = true;
}

extern "C" {

int elmfb_compute_gram(elmfb_t h) {
  if (!h) return ELMFB_ERR_INVALID_ARG;
  try {
    CUDA_CHECK(cudaSetDevice(h->device));
    if (!h->assembled) ELMFB_THROW(ELMFB_ERR_STATE, "compute_gram before assemble");
    gram_compute(h);
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

int elmfb_get_gram(elmfb_t h, int64_t n, const int* ij, double* out) {
  if (!h) return ELMFB_ERR_INVALID_ARG;
  try {
    CUDA_CHECK(cudaSetDevice(h->device));
    if (!h->have_gram) ELMFB_THROW(ELMFB_ERR_STATE, "get_gram before compute_gram");
    if (n < 0 || (n > 0 && (!ij || !out))) ELMFB_THROW(ELMFB_ERR_INVALID_ARG, "bad arguments");
    const int K = h->K;
    std::vector<int> hij(2 * n);
    CUDA_CHECK(cudaMemcpy(hij.data(), ij, 2 * n * sizeof(int), cudaMemcpyDefault));
    std::vector<float> blk((size_t)K * K);
    std::vector<double> res((size_t)n * K * K, 0.0);
    for (int64_t q = 0; q < n; ++q) {
      int i = hij[2 * q], j = hij[2 * q + 1];
      bool tr = i > j;
      if (tr) std::swap(i, j);
      auto it = std::lower_bound(h->gram_pair_ij.begin(), h->gram_pair_ij.end(),
                                 std::make_pair(i, j));
      if (it == h->gram_pair_ij.end() || *it != std::make_pair(i, j)) continue;   // zero block
      const int64_t p = it - h->gram_pair_ij.begin();
      CUDA_CHECK(cudaMemcpy(blk.data(), h->d_gram.as<float>() + p * K * K, K * K * sizeof(float),
                            cudaMemcpyDeviceToHost));
      for (int a = 0; a < K; ++a)
        for (int b = 0; b < K; ++b)
          res[(size_t)q * K * K + a * K + b] = tr ? blk[b * K + a] : blk[a * K + b];
    }
    CUDA_CHECK(cudaMemcpy(out, res.data(), res.size() * sizeof(double), cudaMemcpyDefault));
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
