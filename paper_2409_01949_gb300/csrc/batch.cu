// Batched solves of many independent instances (not in the paper).
//
// Each instance runs the full path (create -> assemble -> solve -> eval ->
// error norms) through its own handle.  A pool of host worker threads, each
// owning a non-blocking CUDA stream, takes instances from a shared counter in
// decreasing order of estimated work (rows x covering panels x K), so the
// GPU is kept busy by several instances at once and the long instances start
// first.
//
// Multi-instance launches: an instance that iterates on FP32 panels with the
// FP32-pair tail joins shared rounds once its start-up step is done.  A
// round runs check_every LSQR iterations of every member, each iteration as
// three launches per launch shape (members of different K run on their own
// streams side by side): the fused pass over all members' units, the slice
// sums over all their slices, the tail over all their panels.  So the many
// small per-instance kernels become a few large ones that fill the GPU.  The
// last member to arrive at a round launches it; each member then reads its
// own scalars and leaves on convergence, at its iteration cap or on an
// error, after which the next round's maps are rebuilt without it.
//
// Results are independent of the schedule: every block of a shared launch
// does what it does in the instance's own launch, on that instance's arrays
// only, and each instance's kernels run in the same order.
#include <algorithm>
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <cstdio>
#include <map>
#include <memory>
#include <mutex>
#include <new>
#include <system_error>
#include <thread>

#include "elmfb_internal.cuh"

struct BatchRound {
  struct Member {
    BatchInst inst{};
    BatchShape shape;
    int64_t launches = 0;   // shared launches attributed to this member, not yet reported
    double rec[kRoundRecord];   // its scalars and flags after the last round
  };
  // one launch shape's members and their block maps
  struct Class {
    BatchShape shape;
    cudaStream_t stream = nullptr;
    cudaEvent_t done = nullptr;   // blocking-sync event: the launcher sleeps while the round runs
    std::vector<BatchInst> h_inst;
    std::vector<int2> h_fmap, h_cmap, h_tmap;
    DevBuf inst, fmap, cmap, tmap;
    int first_slot = -1;
  };
  std::mutex m;
  std::condition_variable cv;
  int check_every = 1;
  std::vector<Member> slot;
  std::vector<char> member;
  std::vector<cudaStream_t> streams;   // one per class in use, kept across rebuilds
  std::vector<cudaEvent_t> events;     // and its blocking-sync event
  // every member's record gathered after a round by one kernel and one copy
  // (rather than a copy and a wait in every member's thread)
  cudaStream_t gstream = nullptr;
  cudaEvent_t gdone = nullptr;
  DevBuf all_inst, d_rec;
  std::vector<BatchInst> h_all;
  std::vector<int> all_slot;
  double* h_rec = nullptr;   // pinned, n_slots records
  std::vector<std::unique_ptr<Class>> classes;
  bool dirty = false;
  bool running = false;   // a round is on the GPU (the lock is free meanwhile)
  int members = 0, arrived = 0;
  uint64_t gen = 0;
  int err = ELMFB_OK;
  std::string msg;
  int64_t rounds = 0, rebuilds = 0;
  // ELMFB_BATCH_TRACE=<file>: one line per round (start and length in ms
  // since the batch began, the wait since the previous round ended, members,
  // fused-pass units), written when the batch ends
  struct Trace {
    double t0, ms, gap;
    int members, units;
  };
  bool trace = false;
  std::vector<Trace> log;
  std::chrono::steady_clock::time_point start = std::chrono::steady_clock::now(),
                                        last_end = start;

  // Device buffers are freed on the streams they were allocated on, before
  // those streams go; every exit of the batch (errors included) passes here.
  ~BatchRound() {
    classes.clear();
    all_inst.release();
    d_rec.release();
    if (gstream) {
      cudaStreamSynchronize(gstream);
      cudaStreamDestroy(gstream);
    }
    if (gdone) cudaEventDestroy(gdone);
    if (h_rec) cudaFreeHost(h_rec);
    for (cudaStream_t st : streams) {
      cudaStreamSynchronize(st);
      cudaStreamDestroy(st);
    }
    for (cudaEvent_t ev : events) cudaEventDestroy(ev);
  }

  void rebuild() {
    h_all.clear();
    all_slot.clear();
    for (int q = 0; q < (int)slot.size(); ++q)
      if (member[q]) {
        h_all.push_back(slot[q].inst);
        all_slot.push_back(q);
      }
    if (!h_all.empty()) {
      all_inst.alloc(h_all.size() * sizeof(BatchInst), gstream);
      CUDA_CHECK(cudaMemcpyAsync(all_inst.p, h_all.data(), h_all.size() * sizeof(BatchInst),
                                 cudaMemcpyHostToDevice, gstream));
    }
    // members by launch shape, each shape's members dealt round-robin to up
    // to kGroups groups on their own streams, so that one group's tail (a
    // latency-bound kernel) overlaps another's fused pass
    constexpr int kGroups = 4;
    std::map<BatchShape, std::vector<int>> by_shape;
    for (int q = 0; q < (int)slot.size(); ++q)
      if (member[q]) by_shape[slot[q].shape].push_back(q);
    std::vector<std::pair<BatchShape, std::vector<int>>> groups;
    for (auto& g : by_shape) {
      const int ng = std::min<int>(kGroups, (int)g.second.size());
      for (int a = 0; a < ng; ++a) {
        std::vector<int> part;
        for (int j = a; j < (int)g.second.size(); j += ng) part.push_back(g.second[j]);
        groups.emplace_back(g.first, std::move(part));
      }
    }
    // drop the old maps only after the streams are idle (they are: rounds
    // end with a synchronisation)
    classes.clear();
    int c = 0;
    for (auto& g : groups) {
      if ((int)streams.size() <= c) {
        cudaStream_t st = nullptr;
        CUDA_CHECK(cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking));
        streams.push_back(st);
        cudaEvent_t ev = nullptr;
        CUDA_CHECK(cudaEventCreateWithFlags(&ev, cudaEventBlockingSync | cudaEventDisableTiming));
        events.push_back(ev);
      }
      classes.push_back(std::make_unique<Class>());
      Class& k = *classes.back();
      k.shape = g.first;
      k.stream = streams[c];
      k.done = events[c];
      k.first_slot = g.second.front();
      for (int j = 0; j < (int)g.second.size(); ++j) {
        const BatchInst& bi = slot[g.second[j]].inst;
        k.h_inst.push_back(bi);
        for (int u = 0; u < bi.n_units; ++u) k.h_fmap.push_back(make_int2(j, u));
        for (int q = 0; q < bi.n_pchunks; ++q) k.h_cmap.push_back(make_int2(j, q));
        for (int p = 0; p < bi.n_sub; ++p) k.h_tmap.push_back(make_int2(j, p));
      }
      auto put = [&](DevBuf& d, const void* src, size_t bytes) {
        d.alloc(bytes, k.stream);
        CUDA_CHECK(cudaMemcpyAsync(d.p, src, bytes, cudaMemcpyHostToDevice, k.stream));
      };
      put(k.inst, k.h_inst.data(), k.h_inst.size() * sizeof(BatchInst));
      put(k.fmap, k.h_fmap.data(), k.h_fmap.size() * sizeof(int2));
      put(k.cmap, k.h_cmap.data(), k.h_cmap.size() * sizeof(int2));
      put(k.tmap, k.h_tmap.data(), k.h_tmap.size() * sizeof(int2));
      ++c;
    }
    dirty = false;
    ++rebuilds;
  }

  // Launch one round and wait for it; then release the waiting members.
  // Called with the lock held (lk) once every member has arrived and no round
  // runs.  The lock is released while the GPU works, so that instances can
  // join (their arrivals count towards the next round) and leave meanwhile;
  // the round's own arrays (classes, all_inst, all_slot) change only in
  // rebuild(), which runs here before the lock is released.
  void run_round(std::unique_lock<std::mutex>& lk) {
    const auto t0 = std::chrono::steady_clock::now();
    running = true;
    arrived = 0;
    const int participants = members;
    int e_code = err;
    std::string e_msg;
    if (e_code == ELMFB_OK) {
      try {
        if (dirty) rebuild();
      } catch (const elmfb_error& e) {
        e_code = e.code;
        e_msg = e.msg;
      }
    }
    const int n = (int)all_slot.size();
    if (e_code == ELMFB_OK) {
      lk.unlock();
      try {
        for (int i = 0; i < check_every; ++i)
          for (auto& k : classes)
            launch_batch_iteration(k->shape, k->inst.as<BatchInst>(), k->fmap.as<int2>(),
                                   (int)k->h_fmap.size(), k->cmap.as<int2>(),
                                   (int)k->h_cmap.size(), k->tmap.as<int2>(),
                                   (int)k->h_tmap.size(), k->stream);
        for (auto& k : classes) {
          CUDA_CHECK(cudaEventRecord(k->done, k->stream));
          CUDA_CHECK(cudaStreamWaitEvent(gstream, k->done, 0));
        }
        launch_gather_records(all_inst.as<BatchInst>(), n, d_rec.as<double>(), gstream);
        CUDA_CHECK(cudaMemcpyAsync(h_rec, d_rec.p, (size_t)n * kRoundRecord * sizeof(double),
                                   cudaMemcpyDeviceToHost, gstream));
        CUDA_CHECK(cudaEventRecord(gdone, gstream));
        CUDA_CHECK(cudaEventSynchronize(gdone));   // sleeps (blocking-sync event)
      } catch (const elmfb_error& e) {
        e_code = e.code;
        e_msg = e.msg;
      } catch (...) {
        e_code = ELMFB_ERR_CUDA;
        e_msg = "unexpected error";
      }
      lk.lock();
    }
    if (e_code == ELMFB_OK) {
      for (auto& k : classes) slot[k->first_slot].launches += 3 * (int64_t)check_every;
      if (n > 0) slot[all_slot[0]].launches += 1;
      for (int j = 0; j < n; ++j)
        std::copy(h_rec + (size_t)j * kRoundRecord, h_rec + (size_t)(j + 1) * kRoundRecord,
                  slot[all_slot[j]].rec);
      ++rounds;
      if (trace) {
        const auto t1 = std::chrono::steady_clock::now();
        using ms = std::chrono::duration<double, std::milli>;
        int units = 0;
        for (auto& k : classes) units += (int)k->h_fmap.size();
        log.push_back({ms(t0 - start).count(), ms(t1 - t0).count(), ms(t0 - last_end).count(),
                       participants, units});
        last_end = t1;
      }
    } else if (err == ELMFB_OK) {
      err = e_code;
      msg = e_msg;
    }
    running = false;
    ++gen;
    cv.notify_all();
  }
};

void round_join(BatchRound* r, int q, const BatchInst& inst, const BatchShape& shape) {
  std::lock_guard<std::mutex> lk(r->m);
  r->slot[q].inst = inst;
  r->slot[q].shape = shape;
  r->slot[q].launches = 0;
  r->member[q] = 1;
  ++r->members;
  r->dirty = true;
}

int64_t round_step(BatchRound* r, int q, double* rec) {
  std::unique_lock<std::mutex> lk(r->m);
  if (r->err != ELMFB_OK) ELMFB_THROW(r->err, "multi-instance round: " + r->msg);
  // the round this arrival takes part in: the next one to start (after the
  // running one, if a round runs now)
  const uint64_t target = r->gen + (r->running ? 2 : 1);
  ++r->arrived;
  if (!r->running && r->arrived == r->members) r->run_round(lk);
  // every member either arrives or leaves, and the last of them runs the
  // round; the bound only turns a host-side fault into an error
  if (!r->cv.wait_for(lk, std::chrono::seconds(600), [&] { return r->gen >= target; })) {
    if (r->gen + 1 == target && !r->running) --r->arrived;
    ELMFB_THROW(ELMFB_ERR_TIMEOUT, "multi-instance round: the other members did not arrive");
  }
  if (r->err != ELMFB_OK) ELMFB_THROW(r->err, "multi-instance round: " + r->msg);
  std::copy(r->slot[q].rec, r->slot[q].rec + kRoundRecord, rec);
  const int64_t n = r->slot[q].launches;
  r->slot[q].launches = 0;
  return n;
}

int round_interval(const BatchRound* r) { return r->check_every; }

void round_leave(BatchRound* r, int q) {
  std::unique_lock<std::mutex> lk(r->m);
  if (!r->member[q]) return;
  r->member[q] = 0;
  --r->members;
  r->dirty = true;
  if (!r->running && r->members > 0 && r->arrived == r->members) r->run_round(lk);
}

static int batch_solve(int n, const elmfb_batch_item* items, const elmfb_solve_opts* opts,
                       int n_workers, elmfb_batch_result* results) {
  if (n < 0 || (n > 0 && (!items || !results)) || n_workers < 1 || n_workers > 256)
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
  // the shared rounds, one slot per worker
  BatchRound round;
  round.check_every = std::max(1, opts ? opts->check_every : 10);
  round.slot.resize(w);
  round.member.assign(w, 0);
  if (cudaStreamCreateWithFlags(&round.gstream, cudaStreamNonBlocking) != cudaSuccess ||
      cudaEventCreateWithFlags(&round.gdone, cudaEventBlockingSync | cudaEventDisableTiming) !=
          cudaSuccess ||
      cudaMallocHost(&round.h_rec, (size_t)w * kRoundRecord * sizeof(double)) != cudaSuccess)
    return ELMFB_ERR_CUDA;
  try {
    round.d_rec.alloc((size_t)w * kRoundRecord * sizeof(double), round.gstream);
  } catch (...) {
    return ELMFB_ERR_CUDA;
  }
  // an item no worker takes (no worker could start) reports that
  for (int i = 0; i < n; ++i) {
    results[i] = elmfb_batch_result{};
    results[i].status = ELMFB_ERR_CUDA;
    results[i].rel_l2 = results[i].e_l1 = results[i].max_abs = NAN;
    std::snprintf(results[i].message, sizeof(results[i].message),
                  "not run: no batch worker could start");
  }
  const char* trace_path = getenv("ELMFB_BATCH_TRACE");
  round.trace = trace_path && trace_path[0];
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
      // more worker threads than host cores: waits sleep instead of spinning;
      // with other instances on the GPU the autotuner cannot time in isolation
      if (h) {
        h->blocking_sync = true;
        h->tune_lookup_only = w > 1;
      }
      if (rc == ELMFB_OK) rc = elmfb_assemble(h, it.n_sets, it.sets);
      elmfb_solve_info info{};
      if (rc == ELMFB_OK) {
        if (opts && opts->batch_shared) {
          h->round = &round;
          h->round_slot = slot;
        }
        rc = elmfb_solve(h, it.opts ? it.opts : opts, &info);
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
  // a thread that cannot be started leaves its share to the others; with none
  // started, this thread does the work
  std::vector<std::thread> pool;
  pool.reserve(w);
  for (int t = 0; t < w; ++t) {
    try {
      pool.emplace_back(worker, t);
    } catch (const std::system_error&) {
      break;
    }
  }
  if (pool.empty()) worker(0);
  for (auto& t : pool) t.join();
  if (round.trace) {
    if (FILE* f = std::fopen(trace_path, "w")) {
      std::fprintf(f, "t0_ms,ms,gap_ms,members,units\n");
      for (const auto& r : round.log)
        std::fprintf(f, "%.3f,%.3f,%.3f,%d,%d\n", r.t0, r.ms, r.gap, r.members, r.units);
      std::fclose(f);
    }
  }
  for (int i = 0; i < n; ++i)
    if (results[i].status != ELMFB_OK) return results[i].status;
  return ELMFB_OK;
}

// no exception crosses the C ABI
extern "C" int elmfb_batch_solve(int n, const elmfb_batch_item* items,
                                 const elmfb_solve_opts* opts, int n_workers,
                                 elmfb_batch_result* results) {
  try {
    return batch_solve(n, items, opts, n_workers, results);
  } catch (const std::bad_alloc&) {
    return ELMFB_ERR_OOM;
  } catch (...) {
    return ELMFB_ERR_CUDA;
  }
}
