// Batched solves of many independent instances (not in the paper).
//
// Each instance runs the full path (create -> assemble -> solve -> eval ->
// error norms) through its own handle.  A pool of host worker threads, each
// owning a non-blocking CUDA stream, takes instances from a shared counter in
// decreasing order of estimated work (rows x covering panels x K), so the
// GPU is kept busy by several instances at once and the long instances start
// first.  Results are independent of the schedule: every instance's kernels
// are deterministic and touch only that instance's buffers.
#include <algorithm>
#include <atomic>
#include <chrono>
#include <cstdio>
#include <thread>

#include "elmfb_internal.cuh"

extern "C" int elmfb_batch_solve(int n, const elmfb_batch_item* items,
                                 const elmfb_solve_opts* opts, int n_workers,
                                 elmfb_batch_result* results) {
  if (n < 0 || (n > 0 && (!items || !results)) || n_workers < 1 || n_workers > 64)
    return ELMFB_ERR_INVALID_ARG;
  if (n == 0) return ELMFB_OK;
  int device = 0;
  if (cudaGetDevice(&device) != cudaSuccess) return ELMFB_ERR_CUDA;
  // largest estimated work first
  std::vector<int> order(n);
  std::vector<double> work(n, 0.0);
  for (int i = 0; i < n; ++i) {
    order[i] = i;
    int64_t rows = 0;
    for (int b = 0; b < items[i].n_sets; ++b) rows += items[i].sets ? items[i].sets[b].n : 0;
    const double cover = (double)items[i].cfg.n_levels * (items[i].cfg.dim == 2 ? 4.0 : 2.0);
    work[i] = (double)rows * cover * items[i].cfg.features;
  }
  std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return work[a] > work[b]; });
  std::atomic<int> next{0};
  auto worker = [&]() {
    cudaSetDevice(device);
    cudaStream_t st = nullptr;
    if (cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) != cudaSuccess) return;
    for (;;) {
      const int k = next.fetch_add(1);
      if (k >= n) break;
      const int i = order[k];
      const elmfb_batch_item& it = items[i];
      elmfb_batch_result& res = results[i];
      res = elmfb_batch_result{};
      res.rel_l2 = res.e_l1 = res.max_abs = NAN;
      const auto t0 = std::chrono::steady_clock::now();
      elmfb_t h = nullptr;
      int rc = elmfb_create(&h, &it.cfg, st);
      if (rc != ELMFB_OK) std::snprintf(res.message, sizeof(res.message), "create failed");
      if (rc == ELMFB_OK) rc = elmfb_assemble(h, it.n_sets, it.sets);
      elmfb_solve_info info{};
      if (rc == ELMFB_OK) {
        rc = elmfb_solve(h, opts, &info);
        if (rc == ELMFB_ERR_NOT_CONVERGED) rc = ELMFB_OK;
        res.iterations = info.iterations;
      }
      if (rc == ELMFB_OK && it.coeffs_out) rc = elmfb_get_coeffs(h, it.coeffs_out);
      if (rc == ELMFB_OK && it.n_eval > 0 && it.eval_points && it.eval_out) {
        rc = elmfb_eval(h, it.eval_points, it.n_eval, it.eval_out);
        if (rc == ELMFB_OK && it.eval_ref) {
          double out3[3];
          rc = elmfb_error_norms(h, it.eval_out, it.eval_ref, it.n_eval, out3);
          if (rc == ELMFB_OK) {
            res.rel_l2 = out3[0];
            res.e_l1 = out3[1];
            res.max_abs = out3[2];
          }
        }
      }
      if (h) {
        if (rc != ELMFB_OK) {
          std::snprintf(res.message, sizeof(res.message), "%s", elmfb_last_error(h));
        }
        res.launches = elmfb_kernel_launches(h);
        elmfb_destroy(h);
      }
      res.status = rc;
      res.total_ms =
          std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
    }
    cudaStreamSynchronize(st);
    cudaStreamDestroy(st);
  };
  std::vector<std::thread> pool;
  const int w = std::min(n_workers, n);
  for (int t = 0; t < w; ++t) pool.emplace_back(worker);
  for (auto& t : pool) t.join();
  for (int i = 0; i < n; ++i)
    if (results[i].status != ELMFB_OK) return results[i].status;
  return ELMFB_OK;
}
