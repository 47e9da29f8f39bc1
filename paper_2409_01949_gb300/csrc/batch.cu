// Batched solves of many independent instances (not in the paper).
//
// Each instance runs the full path (create -> assemble -> solve -> eval ->
// error norms) through its own handle.  A pool of host worker threads, each
// owning a non-blocking CUDA stream, takes instances from a shared counter in
// decreasing order of estimated work (rows x covering panels x K), so the
// GPU is kept busy by several instances at once and the long instances start
// first.  Results are independent of the schedule: every instance's kernels
// are deterministic and touch only that instance's buffers.
//
// Graph mode (opts->graph): besides capturing its check intervals, every
// instance in its LSQR loop joins shared rounds.  Each round is ONE launch of
// a parent graph whose independent child nodes are the current members'
// captured intervals, so the GPU runs the members' small kernels side by
// side instead of one instance's launches at a time.  A member reads its
// scalars after every round and leaves on convergence, at its iteration cap
// or on an error; its device skip flag then turns its nodes into no-ops (every
// kernel of the interval reads the flag first), so the parent is rebuilt only
// when a new member joins.  A rebuild keeps only the members' nodes, so a
// slot is reused by the next instance of the same worker only after the old
// nodes are gone.
#include <algorithm>
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <cstdio>
#include <mutex>
#include <thread>

#include "elmfb_internal.cuh"

struct GraphRound {
  std::mutex m;
  std::condition_variable cv;
  int n_slots = 0;
  cudaStream_t stream = nullptr;
  int* d_skip = nullptr;              // one flag per slot, on the device
  std::vector<cudaGraph_t> child;     // slot -> its member's interval (owned)
  std::vector<char> member;           // slot joined and not yet left
  std::vector<char> in_exec;          // slot's nodes are in the instantiated parent
  bool dirty = false;                 // membership grew since the last build
  int members = 0, arrived = 0;
  uint64_t gen = 0;                   // rounds completed
  cudaGraphExec_t exec = nullptr;
  cudaError_t err = cudaSuccess;
  int64_t rounds = 0, builds = 0;

  // Rebuild if needed, launch, wait; then release the waiting members.
  // Called with the lock held by the last member to arrive.
  void run_locked() {
    if (err == cudaSuccess) {
      cudaError_t e = cudaSuccess;
      if (dirty) {
        if (exec) cudaGraphExecDestroy(exec);
        exec = nullptr;
        cudaGraph_t parent = nullptr;
        e = cudaGraphCreate(&parent, 0);
        for (int s = 0; s < n_slots && e == cudaSuccess; ++s) {
          if (!member[s]) continue;
          cudaGraphNode_t nd;
          e = cudaGraphAddChildGraphNode(&nd, parent, nullptr, 0, child[s]);
        }
        if (e == cudaSuccess) e = cudaGraphInstantiate(&exec, parent, 0);
        if (parent) cudaGraphDestroy(parent);
        std::vector<int> flags(n_slots);
        for (int s = 0; s < n_slots; ++s) {
          in_exec[s] = member[s] && e == cudaSuccess;
          flags[s] = member[s] ? 0 : 1;
        }
        if (e == cudaSuccess)
          e = cudaMemcpyAsync(d_skip, flags.data(), n_slots * sizeof(int), cudaMemcpyHostToDevice,
                              stream);
        dirty = false;
        ++builds;
      }
      if (e == cudaSuccess) e = cudaGraphLaunch(exec, stream);
      if (e == cudaSuccess) e = cudaStreamSynchronize(stream);
      err = e;
      ++rounds;
    }
    arrived = 0;
    ++gen;
    cv.notify_all();
  }
};

void round_join(GraphRound* r, int slot, cudaGraph_t g) {
  std::lock_guard<std::mutex> lk(r->m);
  if (r->child[slot]) cudaGraphDestroy(r->child[slot]);
  r->child[slot] = g;
  r->member[slot] = 1;
  ++r->members;
  r->dirty = true;
}

void round_step(GraphRound* r, int slot) {
  (void)slot;
  std::unique_lock<std::mutex> lk(r->m);
  if (r->err != cudaSuccess)
    ELMFB_THROW(ELMFB_ERR_CUDA, std::string("batched graph round: ") + cudaGetErrorString(r->err));
  ++r->arrived;
  if (r->arrived == r->members) {
    r->run_locked();
  } else {
    const uint64_t g0 = r->gen;
    // every member either arrives or leaves, and the last of them runs the
    // round; the bound only turns a host-side fault into an error
    if (!r->cv.wait_for(lk, std::chrono::seconds(600), [&] { return r->gen != g0; })) {
      --r->arrived;
      ELMFB_THROW(ELMFB_ERR_TIMEOUT, "batched graph round: the other members did not arrive");
    }
  }
  if (r->err != cudaSuccess)
    ELMFB_THROW(ELMFB_ERR_CUDA, std::string("batched graph round: ") + cudaGetErrorString(r->err));
}

void round_leave(GraphRound* r, int slot) {
  std::lock_guard<std::mutex> lk(r->m);
  if (!r->member[slot]) return;
  r->member[slot] = 0;
  --r->members;
  if (r->child[slot]) cudaGraphDestroy(r->child[slot]);   // the parent holds its own copy
  r->child[slot] = nullptr;
  if (r->in_exec[slot] && r->err == cudaSuccess) {
    // no round runs while the lock is held: the flag is set before the next one
    static const int one = 1;
    cudaError_t e = cudaMemcpyAsync(r->d_skip + slot, &one, sizeof(int), cudaMemcpyHostToDevice,
                                    r->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(r->stream);
    if (e != cudaSuccess) r->err = e;
  }
  if (r->members > 0 && r->arrived == r->members) r->run_locked();
}

const int* round_skip_flag(GraphRound* r, int slot) { return r->d_skip + slot; }

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
  const int w = std::min(n_workers, n);
  // graph mode: the shared rounds, one slot per worker
  GraphRound round;
  const bool rounds = opts && opts->graph;
  if (rounds) {
    round.n_slots = w;
    round.child.assign(w, nullptr);
    round.member.assign(w, 0);
    round.in_exec.assign(w, 0);
    if (cudaStreamCreateWithFlags(&round.stream, cudaStreamNonBlocking) != cudaSuccess)
      return ELMFB_ERR_CUDA;
    if (cudaMalloc(&round.d_skip, w * sizeof(int)) != cudaSuccess) {
      cudaStreamDestroy(round.stream);
      return ELMFB_ERR_CUDA;
    }
  }
  auto worker = [&](int slot) {
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
        if (rounds) {
          h->round = &round;
          h->round_slot = slot;
        }
        rc = elmfb_solve(h, opts, &info);
        h->round = nullptr;
        h->round_slot = -1;
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
  for (int t = 0; t < w; ++t) pool.emplace_back(worker, t);
  for (auto& t : pool) t.join();
  if (rounds) {
    if (round.exec) cudaGraphExecDestroy(round.exec);
    for (cudaGraph_t g : round.child)
      if (g) cudaGraphDestroy(g);
    cudaStreamSynchronize(round.stream);
    cudaFree(round.d_skip);
    cudaStreamDestroy(round.stream);
  }
  for (int i = 0; i < n; ++i)
    if (results[i].status != ELMFB_OK) return results[i].status;
  return ELMFB_OK;
}
