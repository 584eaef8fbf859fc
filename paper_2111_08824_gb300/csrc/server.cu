// Serving loop: resident learned indexes, probe requests, continuous batching.
//
// Each request is one join (Section 2.A probe of its keys S against one
// resident relation's learned index, Section 2.D).  A scheduler thread owns
// the device work:
//   admission   a pending request is admitted when an in-flight slot is free
//               and the memory it needs (8 bytes per probe for its pairs,
//               4 for its search words) fits the server's HBM budget;
//               requests larger than the whole budget are rejected
//               (LJ_E_BUDGET); admission is first come, first served.
//   batching    all requests admitted together form one dynamic batch (one
//               persistent search launch, one scan, one compaction) on the
//               slot's stream -- a batch of one request takes join_emit's
//               own kernels instead, and so does every request to a
//               relation with gapped or hash arrays (grmi_build,
//               lhash_build, lhash_build_rs), always alone; requests
//               arriving while batches run are
//               admitted into the next free slot, so batches overlap on the
//               device (continuous batching, not a queue in front of a
//               single worker).
//   completion  one waiter thread per slot waits for its batch's event
//               (the runtime polls, so completion is seen within
//               microseconds), releases the batch's scratch, wakes the
//               waiting clients and the scheduler.
// Latency of a request = submit to completion detected (host clock).
#include <algorithm>
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <deque>
#include <mutex>
#include <thread>
#include <unordered_map>
#include <vector>

#include "device_common.cuh"
#include "internal.h"

namespace {

using Clock = std::chrono::steady_clock;

struct Request {
  uint64_t id = 0;
  uint32_t rel = 0;
  const uint64_t* S = nullptr;
  uint64_t m = 0;
  lj_pair* pairs = nullptr;   // server-owned until released
  uint64_t need = 0;          // bytes charged against the budget
  uint64_t count = 0;
  int status = 1;             // 1 pending, 2 running, 0 done, < 0 error
  Clock::time_point t_submit, t_start, t_done;
};

struct Slot {
  cudaStream_t stream = nullptr;
  cudaEvent_t done = nullptr;
  lj::DynBatchBuffers buf;
  char* scratch = nullptr;
  uint64_t* written_dev = nullptr;
  uint64_t* written_host = nullptr;   // page-locked
  std::vector<Request*> reqs;
  bool busy = false;
};

}  // namespace

struct lj_server {
  lj_server_cfg cfg{};
  int device = 0;
  std::vector<const lj_index*> rels;
  std::mutex mu;
  std::condition_variable cv_sched, cv_done;
  std::deque<Request*> pending;
  std::unordered_map<uint64_t, Request*> reqs;
  std::vector<Slot> slots;
  cudaStream_t free_stream = nullptr;
  cudaEvent_t fetch_done = nullptr;  // orders the release of a request's pairs after its fetches
  uint64_t next_id = 1;
  uint64_t resident = 0;             // bytes of the registered relations (R and index)
  uint64_t mem_in_use = 0, mem_peak = 0;
  bool stop = false;
  std::atomic<bool> wake{false};   // set by submissions and completions
  std::thread sched;
  std::condition_variable cv_launch;   // wakes the slot waiters
  std::vector<std::thread> waiters;    // one per slot: waits for its batch on the GPU
  std::vector<char> launched;          // per slot: a batch is in flight, its waiter takes it
  bool stop_waiters = false;
  // statistics
  std::vector<double> lat_us;
  uint64_t submitted = 0, completed = 0, rejected = 0, keys = 0, batches = 0, batched_reqs = 0;
  Clock::time_point t_first, t_last;
  bool any = false;
};

namespace {

void complete_slot(lj_server* sv, Slot& sl) {
  const auto now = Clock::now();
  for (size_t i = 0; i < sl.reqs.size(); ++i) {
    Request* r = sl.reqs[i];
    r->count = sl.written_host[i];
    r->status = r->count > r->m ? LJ_E_CAPACITY : 0;
    r->t_done = now;
    sv->mem_in_use -= r->m * 4;   // the search words are gone; the pairs stay
    sv->lat_us.push_back(std::chrono::duration<double, std::micro>(now - r->t_submit).count());
    sv->completed++;
    sv->keys += r->m;
    sv->t_last = now;
  }
  if (sl.scratch) lj::scratch_free(sl.scratch, sl.stream);
  sl.scratch = nullptr;
  sl.reqs.clear();
  sl.busy = false;
}

// Waiter of slot k: when its batch is launched, waits for the batch's event
// (the runtime's synchronisation polls, so a finished batch is seen within
// microseconds), then completes the requests and frees the slot.
void slot_waiter(lj_server* sv, size_t k) {
  cudaSetDevice(sv->device);
  std::unique_lock<std::mutex> lk(sv->mu);
  while (true) {
    sv->cv_launch.wait(lk, [&] { return sv->launched[k] || sv->stop_waiters; });
    if (!sv->launched[k]) return;   // stopping, nothing in flight
    Slot& sl = sv->slots[k];
    const cudaEvent_t ev = sl.done;
    lk.unlock();
    cudaEventSynchronize(ev);
    lk.lock();
    complete_slot(sv, sl);
    sv->launched[k] = 0;
    sv->cv_done.notify_all();
    sv->wake.store(true);
    sv->cv_sched.notify_one();
  }
}

// Launch the admitted requests `batch` on slot `sl` (called with sv->mu held).
int launch_slot(lj_server* sv, Slot& sl, std::vector<Request*>& batch) {
  std::vector<lj::BatchJob> jobs(batch.size());
  for (size_t i = 0; i < batch.size(); ++i) {
    Request* r = batch[i];
    if (lj::scratch_alloc((void**)&r->pairs, std::max<uint64_t>(r->m, 1) * 8, sl.stream) !=
        cudaSuccess)
      return lj::fail(LJ_E_NOMEM, "server: no room for a request's pairs");
    jobs[i] = lj::BatchJob{sv->rels[r->rel], r->S, r->m, r->pairs, r->m};
    r->status = 2;
    r->t_start = Clock::now();
  }
  if (batch.size() == 1) {
    // a batch of one request: the plain probe's own path (the fused kernel
    // for small batches, else the search-compaction pipeline), so a request
    // alone costs what join_emit costs and the slots add the overlap
    Request* r = batch[0];
    if (r->m == 0) {
      if (cudaMemsetAsync(sl.written_dev, 0, 8, sl.stream) != cudaSuccess)
        return lj::fail(LJ_E_CUDA, "server: cannot enqueue a request");
    } else if (int rc = lj::probe_emit_impl(jobs[0].idx, r->S, r->m, nullptr, r->pairs, r->m,
                                            sl.written_dev, nullptr, 0, sl.stream)) {
      return rc;
    }
  } else {
    const size_t bytes = lj::dyn_batch_scratch_bytes(jobs.data(), (uint32_t)jobs.size());
    if (lj::scratch_alloc((void**)&sl.scratch, bytes, sl.stream) != cudaSuccess)
      return lj::fail(LJ_E_NOMEM, "server: no room for a batch's scratch");
    if (int rc = lj::enqueue_dyn_batch(jobs.data(), (uint32_t)jobs.size(), sl.buf, sl.scratch,
                                       sl.written_dev, sl.stream))
      return rc;
  }
  if (cudaMemcpyAsync(sl.written_host, sl.written_dev, jobs.size() * 8, cudaMemcpyDeviceToHost,
                      sl.stream) != cudaSuccess ||
      cudaEventRecord(sl.done, sl.stream) != cudaSuccess)
    return lj::fail(LJ_E_CUDA, "server: cannot enqueue the completion of a batch");
  sl.reqs = batch;
  sl.busy = true;
  sv->batches++;
  sv->batched_reqs += batch.size();
  return 0;
}

void scheduler(lj_server* sv) {
  cudaSetDevice(sv->device);
  std::unique_lock<std::mutex> lk(sv->mu);
  while (true) {
    bool progressed = false;
    // admission into free slots (first come, first served); completions are
    // taken by the slots' waiters
    for (size_t k = 0; k < sv->slots.size(); ++k) {
      Slot& sl = sv->slots[k];
      if (sl.busy || sv->pending.empty()) continue;
      std::vector<Request*> batch;
      while (!sv->pending.empty() && batch.size() < sv->cfg.max_batch) {
        Request* r = sv->pending.front();
        // a relation with gapped or hash arrays is probed by join_emit's own
        // kernels: its requests run as batches of one
        const bool alone = sv->rels[r->rel]->gkeys != nullptr;
        if (alone && !batch.empty()) break;
        if (sv->mem_in_use + r->need > sv->cfg.hbm_budget_bytes) break;
        sv->pending.pop_front();
        sv->mem_in_use += r->need;
        sv->mem_peak = std::max(sv->mem_peak, sv->mem_in_use);
        batch.push_back(r);
        if (alone) break;
      }
      if (batch.empty()) break;
      if (int rc = launch_slot(sv, sl, batch)) {
        for (Request* r : batch) {
          r->status = rc;
          r->t_done = Clock::now();
          sv->mem_in_use -= r->need;
          if (r->pairs) lj::scratch_free(r->pairs, sl.stream);
          r->pairs = nullptr;
        }
        if (sl.scratch) lj::scratch_free(sl.scratch, sl.stream);
        sl.scratch = nullptr;
        sl.reqs.clear();
        sl.busy = false;
        sv->cv_done.notify_all();
      } else {
        sv->launched[k] = 1;
        sv->cv_launch.notify_all();
      }
      progressed = true;
    }
    if (sv->stop && sv->pending.empty()) {
      bool idle = true;
      for (Slot& sl : sv->slots) idle = idle && !sl.busy;
      if (idle) break;
    }
    // sleep until a submission or a completion (slot waiter) wakes us; the
    // timeout only guards against a wake-up lost between check and wait
    if (!progressed)
      sv->cv_sched.wait_for(lk, std::chrono::microseconds(200),
                            [&] { return sv->wake.exchange(false) || sv->stop; });
  }
}

}  // namespace

extern "C" {

int join_server_create(const lj_server_cfg* cfg, lj_server** out) {
  using namespace lj;
  if (!cfg || !out) return fail(LJ_E_INVAL, "join_server_create: NULL argument");
  *out = nullptr;
  if (cfg->streams < 1 || cfg->streams > 16 || cfg->max_batch < 1 || cfg->max_batch > 65536)
    return fail(LJ_E_INVAL, "join_server_create: streams in [1, 16], max_batch in [1, 65536]");
  lj_server* sv = new lj_server();
  sv->cfg = *cfg;
  sv->device = current_device();
  sv->slots.resize(cfg->streams);
  auto bail = [&](int rc) {
    join_server_destroy(sv);
    return rc;
  };
  if (!device_error_word(sv->device)) return bail(fail(LJ_E_NOMEM, "error word"));
  for (Slot& sl : sv->slots) {
    if (cudaStreamCreateWithFlags(&sl.stream, cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreateWithFlags(&sl.done, cudaEventDisableTiming) != cudaSuccess ||
        cudaMalloc(&sl.written_dev, (size_t)cfg->max_batch * 8) != cudaSuccess ||
        cudaMallocHost(&sl.written_host, (size_t)cfg->max_batch * 8) != cudaSuccess)
      return bail(fail(LJ_E_NOMEM, "join_server_create: slot resources"));
    if (int rc = dyn_batch_alloc(sl.buf, cfg->max_batch)) return bail(rc);
  }
  if (cudaStreamCreateWithFlags(&sv->free_stream, cudaStreamNonBlocking) != cudaSuccess ||
      cudaEventCreateWithFlags(&sv->fetch_done, cudaEventDisableTiming) != cudaSuccess)
    return bail(fail(LJ_E_CUDA, "join_server_create: stream"));
  sv->launched.assign(sv->slots.size(), 0);
  for (size_t k = 0; k < sv->slots.size(); ++k) sv->waiters.emplace_back(slot_waiter, sv, k);
  sv->sched = std::thread(scheduler, sv);
  *out = sv;
  return LJ_OK;
}

int join_server_add_relation(lj_server* sv, const lj_index* index, uint32_t* rel_id) {
  using namespace lj;
  if (!sv || !index || !rel_id) return fail(LJ_E_INVAL, "join_server_add_relation: NULL argument");
  if (!index->unique) return fail(LJ_E_NOTUNIQUE, "served relations need an R without duplicates");
  if (index->device != sv->device) return fail(LJ_E_INVAL, "relation on another device");
  std::lock_guard<std::mutex> lk(sv->mu);
  if (!sv->rels.empty() && sv->rels[0]->precision != index->precision)
    return fail(LJ_E_INVAL, "served relations must share one precision");
  // the resident relation (its keys, its leaf records and any gapped or
  // hash arrays) counts against the budget
  const uint64_t rec = index->precision == LJ_FP64 ? sizeof(lj::LeafF64) : sizeof(lj::LeafF32);
  uint64_t bytes = index->n * 8 + (uint64_t)index->L * rec;
  if (index->gkeys) {
    bytes += (uint64_t)index->gslots * 8;                                   // keys
    bytes += index->gkind == 0 ? ((uint64_t)index->gslots + 1) * 4          // GRMI payloads
                               : (uint64_t)index->gslots * 8 + (index->ndistinct + 1) * 4;
    if (index->gkind == 2)   // RadixSpline: points, reciprocals, radix table
      bytes += (uint64_t)index->rs_S * 20 + ((1ull << index->rs_rbits) + 1) * 4;
  }
  if (sv->mem_in_use + bytes > sv->cfg.hbm_budget_bytes)
    return fail(LJ_E_BUDGET, "join_server_add_relation: %llu resident bytes exceed the HBM budget",
                (unsigned long long)bytes);
  sv->resident += bytes;
  sv->mem_in_use += bytes;
  sv->mem_peak = std::max(sv->mem_peak, sv->mem_in_use);
  *rel_id = (uint32_t)sv->rels.size();
  sv->rels.push_back(index);
  return LJ_OK;
}

int join_submit(lj_server* sv, uint32_t rel_id, const uint64_t* S, uint64_t m, lj_ticket* out) {
  using namespace lj;
  if (!sv || !out) return fail(LJ_E_INVAL, "join_submit: NULL argument");
  if (m >= (1ull << 32) || (m > 0 && !S)) return fail(LJ_E_INVAL, "join_submit: bad S");
  Request* r = new Request();
  r->S = S;
  r->m = m;
  r->need = m * 12 + 256;
  r->t_submit = Clock::now();
  {
    std::lock_guard<std::mutex> lk(sv->mu);
    if (rel_id >= sv->rels.size()) {
      delete r;
      return fail(LJ_E_INVAL, "join_submit: unknown relation %u", rel_id);
    }
    if (sv->stop) {
      delete r;
      return fail(LJ_E_STATE, "join_submit: server is stopping");
    }
    r->rel = rel_id;
    r->id = sv->next_id++;
    sv->submitted++;
    if (!sv->any) {
      sv->t_first = r->t_submit;
      sv->any = true;
    }
    if (r->need + sv->resident > sv->cfg.hbm_budget_bytes) {
      sv->rejected++;
      delete r;
      return fail(LJ_E_BUDGET,
                  "join_submit: %llu probes need more than the HBM budget left by the "
                  "resident relations", (unsigned long long)m);
    }
    sv->reqs[r->id] = r;
    sv->pending.push_back(r);
    *out = r->id;
  }
  sv->wake.store(true);
  sv->cv_sched.notify_one();
  return LJ_OK;
}

int join_wait(lj_server* sv, lj_ticket t, int64_t timeout_us, lj_result* res) {
  using namespace lj;
  if (!sv) return fail(LJ_E_INVAL, "join_wait: NULL server");
  std::unique_lock<std::mutex> lk(sv->mu);
  auto it = sv->reqs.find(t);
  if (it == sv->reqs.end()) return fail(LJ_E_INVAL, "join_wait: unknown ticket");
  Request* r = it->second;
  auto ready = [&] { return r->status <= 0; };
  if (timeout_us < 0)
    sv->cv_done.wait(lk, ready);
  else if (!sv->cv_done.wait_for(lk, std::chrono::microseconds(timeout_us), ready))
    return fail(LJ_E_TIMEOUT, "join_wait: request %llu not done", (unsigned long long)t);
  if (res) {
    res->status = r->status;
    res->pairs = r->count;
    res->pairs_dev = r->pairs;
    res->latency_us = std::chrono::duration<double, std::micro>(r->t_done - r->t_submit).count();
    res->queue_us = std::chrono::duration<double, std::micro>(r->t_start - r->t_submit).count();
  }
  return r->status < 0 ? fail(r->status, "join_wait: request failed") : LJ_OK;
}

int join_fetch(lj_server* sv, lj_ticket t, lj_pair* dst_dev, uint64_t capacity, lj_stream_t stream) {
  using namespace lj;
  if (!sv) return fail(LJ_E_INVAL, "join_fetch: NULL server");
  std::unique_lock<std::mutex> lk(sv->mu);
  auto it = sv->reqs.find(t);
  if (it == sv->reqs.end()) return fail(LJ_E_INVAL, "join_fetch: unknown ticket");
  Request* r = it->second;
  if (r->status != 0) return fail(LJ_E_STATE, "join_fetch: request not completed");
  const uint64_t n = std::min(capacity, r->count);
  if (n) {
    LJ_CUDA(cudaMemcpyAsync(dst_dev, r->pairs, n * 8, cudaMemcpyDeviceToDevice, (cudaStream_t)stream));
    // join_release frees the pairs on free_stream: make that stream wait for
    // this copy, so the memory is not handed out again while it is read
    LJ_CUDA(cudaEventRecord(sv->fetch_done, (cudaStream_t)stream));
    LJ_CUDA(cudaStreamWaitEvent(sv->free_stream, sv->fetch_done, 0));
  }
  if (r->count > capacity) return fail(LJ_E_CAPACITY, "join_fetch: %llu pairs, capacity %llu",
                                       (unsigned long long)r->count, (unsigned long long)capacity);
  return LJ_OK;
}

int join_release(lj_server* sv, lj_ticket t) {
  using namespace lj;
  if (!sv) return fail(LJ_E_INVAL, "join_release: NULL server");
  std::lock_guard<std::mutex> lk(sv->mu);
  auto it = sv->reqs.find(t);
  if (it == sv->reqs.end()) return fail(LJ_E_INVAL, "join_release: unknown ticket");
  Request* r = it->second;
  if (r->status > 0) return fail(LJ_E_STATE, "join_release: request still running");
  if (r->pairs) scratch_free(r->pairs, sv->free_stream);
  if (r->status == 0) sv->mem_in_use -= r->need - r->m * 4;
  sv->reqs.erase(it);
  delete r;
  sv->wake.store(true);
  sv->cv_sched.notify_one();
  return LJ_OK;
}

int join_server_stats(lj_server* sv, lj_server_stats* out, int reset) {
  using namespace lj;
  if (!sv || !out) return fail(LJ_E_INVAL, "join_server_stats: NULL argument");
  std::lock_guard<std::mutex> lk(sv->mu);
  *out = lj_server_stats{};
  out->submitted = sv->submitted;
  out->completed = sv->completed;
  out->rejected = sv->rejected;
  out->keys = sv->keys;
  out->batches = sv->batches;
  out->mean_batch = sv->batches ? (double)sv->batched_reqs / (double)sv->batches : 0.0;
  out->mem_in_use = sv->mem_in_use;
  out->resident = sv->resident;
  out->mem_peak = sv->mem_peak;
  if (!sv->lat_us.empty()) {
    std::vector<double> v = sv->lat_us;
    std::sort(v.begin(), v.end());
    auto q = [&](double f) { return v[std::min(v.size() - 1, (size_t)(f * (v.size() - 1) + 0.5))]; };
    out->p50_us = q(0.50);
    out->p99_us = q(0.99);
    out->max_us = v.back();
    double s = 0;
    for (double x : v) s += x;
    out->mean_us = s / v.size();
  }
  if (sv->any && sv->completed) {
    out->span_s = std::chrono::duration<double>(sv->t_last - sv->t_first).count();
    out->keys_per_s = out->span_s > 0 ? (double)sv->keys / out->span_s : 0.0;
  }
  if (reset) {
    sv->lat_us.clear();
    sv->submitted = sv->completed = sv->rejected = sv->keys = sv->batches = sv->batched_reqs = 0;
    sv->any = false;
    sv->mem_peak = sv->mem_in_use;
  }
  return LJ_OK;
}

void join_server_destroy(lj_server* sv) {
  if (!sv) return;
  {
    std::lock_guard<std::mutex> lk(sv->mu);
    sv->stop = true;
  }
  sv->cv_sched.notify_all();
  if (sv->sched.joinable()) sv->sched.join();   // returns once every slot is idle
  {
    std::lock_guard<std::mutex> lk(sv->mu);
    sv->stop_waiters = true;
  }
  sv->cv_launch.notify_all();
  for (std::thread& t : sv->waiters)
    if (t.joinable()) t.join();
  for (auto& kv : sv->reqs) {
    if (kv.second->pairs) lj::scratch_free(kv.second->pairs, sv->free_stream);
    delete kv.second;
  }
  if (sv->free_stream) cudaStreamSynchronize(sv->free_stream);
  for (Slot& sl : sv->slots) {
    if (sl.stream) cudaStreamSynchronize(sl.stream);
    lj::dyn_batch_release(sl.buf);
    if (sl.written_dev) cudaFree(sl.written_dev);
    if (sl.written_host) cudaFreeHost(sl.written_host);
    if (sl.done) cudaEventDestroy(sl.done);
    if (sl.stream) cudaStreamDestroy(sl.stream);
  }
  if (sv->free_stream) cudaStreamDestroy(sv->free_stream);
  if (sv->fetch_done) cudaEventDestroy(sv->fetch_done);
  delete sv;
}

}  // extern "C"
