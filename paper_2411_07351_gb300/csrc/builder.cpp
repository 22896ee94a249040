// Plan builder pool: fht_plan on native worker threads.
//
// A serving loop that meets a new image size every request cannot afford to
// build the plan on its own thread, and building it on interpreter threads
// makes the builders and the loop queue for the interpreter lock.  The pool
// takes build requests (tagged by the caller), runs fht_plan on its own
// threads, and hands finished plans back through fht_builder_poll.  The paper
// has no counterpart: this is runtime of this library.
#include <algorithm>
#include <condition_variable>
#include <deque>
#include <mutex>
#include <new>
#include <string>
#include <thread>
#include <vector>

#include "../../include/fht.h"

fht_status fht_capi_fail(fht_status st, const std::string& msg);

namespace {

struct BuildJob {
  uint64_t tag;
  int32_t h, w;
  fht_dtype dtype;
  uint32_t quads;
  fht_boundary boundary;
  fht_split split;
  int device;
  bool has_tuning;
  fht_tuning_t tuning;
};

struct BuildResult {
  uint64_t tag;
  fht_plan_t plan;
  fht_status status;
};

}  // namespace

struct fht_builder_s {
  std::mutex mu;
  std::condition_variable cv;
  std::deque<BuildJob> queue;
  std::vector<BuildResult> done;
  bool stop = false;
  std::vector<std::thread> threads;

  void work() {
    for (;;) {
      BuildJob j;
      {
        std::unique_lock<std::mutex> lock(mu);
        cv.wait(lock, [&] { return stop || !queue.empty(); });
        if (queue.empty()) return;  // stopping and drained
        j = queue.front();
        queue.pop_front();
      }
      fht_plan_t plan = nullptr;
      const fht_status st = fht_plan(&plan, j.h, j.w, j.dtype, j.quads, j.boundary, j.split, j.device,
                                     j.has_tuning ? &j.tuning : nullptr);
      std::lock_guard<std::mutex> lock(mu);
      done.push_back(BuildResult{j.tag, st == FHT_OK ? plan : nullptr, st});
    }
  }
};

extern "C" {

fht_status fht_builder_create(fht_builder_t* out, int32_t threads) {
  if (!out) return fht_capi_fail(FHT_ERR_INVALID, "fht_builder_create: out is NULL");
  *out = nullptr;
  if (threads < 1 || threads > 256) return fht_capi_fail(FHT_ERR_INVALID, "fht_builder_create: threads in [1, 256]");
  fht_builder_s* b = new (std::nothrow) fht_builder_s();
  if (!b) return fht_capi_fail(FHT_ERR_NOMEM, "fht_builder_create: host allocation failed");
  try {
    for (int32_t k = 0; k < threads; k++) b->threads.emplace_back([b] { b->work(); });
  } catch (...) {
    {
      std::lock_guard<std::mutex> lock(b->mu);
      b->stop = true;
    }
    b->cv.notify_all();
    for (auto& t : b->threads) t.join();
    delete b;
    return fht_capi_fail(FHT_ERR_NOMEM, "fht_builder_create: could not start the worker threads");
  }
  *out = b;
  return FHT_OK;
}

fht_status fht_builder_submit(fht_builder_t b, uint64_t tag, int32_t h, int32_t w, fht_dtype dtype,
                              uint32_t quadrants, fht_boundary boundary, fht_split split, int device,
                              const fht_tuning_t* tuning) {
  if (!b) return fht_capi_fail(FHT_ERR_INVALID, "fht_builder_submit: builder is NULL");
  BuildJob j{tag, h, w, dtype, quadrants, boundary, split, device, tuning != nullptr, {}};
  if (tuning) j.tuning = *tuning;
  {
    std::lock_guard<std::mutex> lock(b->mu);
    if (b->stop) return fht_capi_fail(FHT_ERR_INVALID, "fht_builder_submit: builder is being destroyed");
    b->queue.push_back(j);
  }
  b->cv.notify_one();
  return FHT_OK;
}

fht_status fht_builder_poll(fht_builder_t b, uint64_t* tags, fht_plan_t* plans, fht_status* status, int32_t cap,
                            int32_t* n) {
  if (!b || !tags || !plans || !status || !n || cap < 0)
    return fht_capi_fail(FHT_ERR_INVALID, "fht_builder_poll: NULL argument or negative capacity");
  std::lock_guard<std::mutex> lock(b->mu);
  const int32_t k = (int32_t)std::min<size_t>((size_t)cap, b->done.size());
  for (int32_t i = 0; i < k; i++) {
    tags[i] = b->done[(size_t)i].tag;
    plans[i] = b->done[(size_t)i].plan;
    status[i] = b->done[(size_t)i].status;
  }
  b->done.erase(b->done.begin(), b->done.begin() + k);
  *n = k;
  return FHT_OK;
}

fht_status fht_builder_pending(fht_builder_t b, int32_t* queued, int32_t* finished) {
  if (!b || !queued || !finished) return fht_capi_fail(FHT_ERR_INVALID, "fht_builder_pending: NULL argument");
  std::lock_guard<std::mutex> lock(b->mu);
  *queued = (int32_t)b->queue.size();
  *finished = (int32_t)b->done.size();
  return FHT_OK;
}

fht_status fht_builder_destroy(fht_builder_t b) {
  if (!b) return FHT_OK;
  {
    std::lock_guard<std::mutex> lock(b->mu);
    b->stop = true;
  }
  b->cv.notify_all();
  for (auto& t : b->threads) t.join();
  for (const BuildResult& r : b->done)
    if (r.plan) fht_plan_destroy(r.plan);  // finished but never claimed
  delete b;
  return FHT_OK;
}

}  // extern "C"
