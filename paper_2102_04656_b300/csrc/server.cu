// server.cu -- continuous-batching request loop around the search of Section 3.5.
//
// Requests (a few queries each, host memory) are queued by bdg_server_submit.
// A scheduler thread keeps up to n_streams batches in flight: whenever a
// stream is free it packs the oldest queued requests into one batch, as long
// as the batch stays within max_batch queries and the device memory of all
// in-flight batches stays within the memory budget (admission by memory),
// copies the batch to the device, runs search + FP32 re-rank, copies the
// results back and records an event. Finished batches hand their rows back to
// their requests. Requests that arrive while batches run are admitted as soon
// as a stream and memory free up, so their work overlaps on the device with
// the batches already running. Every query is processed by its own warp with
// its own ef, so a query's result does not depend on the batch it rides in.
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <mutex>
#include <thread>
#include <unordered_map>
#include <vector>

#include "common.cuh"

namespace {

using Clock = std::chrono::steady_clock;

struct Request {
  int64_t id;
  int nq;
  std::vector<uint64_t> q;    // [nq][W]
  std::vector<float> qf;      // [nq][D]
  std::vector<int32_t> ef;    // [nq]
  std::vector<int32_t> ids;   // [nq][k] results
  std::vector<float> d2;      // [nq][k]
  Clock::time_point t_arrive, t_done;
  bool done = false;
  bdg_status status = BDG_OK;
};

struct Slot {                 // one stream and its buffers
  cudaStream_t st = nullptr;
  cudaEvent_t ev = nullptr;
  uint64_t* dq = nullptr;  float* dqf = nullptr;  int32_t* def = nullptr;
  int32_t* dcand = nullptr; int32_t* dcdist = nullptr;
  int32_t* dids = nullptr;  float* dd2 = nullptr;
  uint64_t* hq = nullptr;  float* hqf = nullptr;  int32_t* hef = nullptr;  // pinned
  int32_t* hids = nullptr; float* hd2 = nullptr;
  std::vector<std::pair<Request*, int>> batch;  // requests and their first row
  int rows = 0;
  uint64_t bytes = 0;
  bool busy = false;
};

}  // namespace

struct bdg_server {
  const bdg_graph* g;
  const float* feats;
  int D, R, k, ef_max, max_batch, W;
  int64_t N;
  uint64_t budget, in_flight_bytes = 0;
  std::vector<Slot> slots;
  std::deque<Request*> pending;
  std::unordered_map<int64_t, Request*> reqs;
  int64_t next_id = 1;
  std::mutex mu;
  std::condition_variable cv_work, cv_done;
  bool stop = false;
  std::thread worker;
  int64_t batches = 0, queries = 0;
  bdg_status fatal = BDG_OK;
  int device = 0;
};

namespace {

uint64_t row_bytes(const bdg_server* s) {
  return (uint64_t)(8 * s->W + 4 * s->D + 4 + 8 * s->R + 8 * s->k);
}

void launch(bdg_server* s, Slot& sl) {
  const int W = s->W, D = s->D;
  for (auto& br : sl.batch) {
    Request* rq = br.first;
    memcpy(sl.hq + (size_t)br.second * W, rq->q.data(), rq->q.size() * 8);
    memcpy(sl.hqf + (size_t)br.second * D, rq->qf.data(), rq->qf.size() * 4);
    memcpy(sl.hef + br.second, rq->ef.data(), rq->ef.size() * 4);
  }
  const int n = sl.rows;
  cudaMemcpyAsync(sl.dq, sl.hq, (size_t)n * W * 8, cudaMemcpyHostToDevice, sl.st);
  cudaMemcpyAsync(sl.dqf, sl.hqf, (size_t)n * D * 4, cudaMemcpyHostToDevice, sl.st);
  cudaMemcpyAsync(sl.def, sl.hef, (size_t)n * 4, cudaMemcpyHostToDevice, sl.st);
  bdg_status st = bdg_search_rerank(s->g, sl.dq, sl.dqf, s->feats, D, n, sl.def, s->ef_max, s->R,
                                    s->k, sl.dcand, sl.dcdist, sl.dids, sl.dd2, sl.st);
  if (st != BDG_OK) s->fatal = st;
  cudaMemcpyAsync(sl.hids, sl.dids, (size_t)n * s->k * 4, cudaMemcpyDeviceToHost, sl.st);
  cudaMemcpyAsync(sl.hd2, sl.dd2, (size_t)n * s->k * 4, cudaMemcpyDeviceToHost, sl.st);
  cudaEventRecord(sl.ev, sl.st);
  sl.busy = true;
}

void finish(bdg_server* s, Slot& sl) {  // called with s->mu held
  const auto now = Clock::now();
  for (auto& br : sl.batch) {
    Request* rq = br.first;
    memcpy(rq->ids.data(), sl.hids + (size_t)br.second * s->k, (size_t)rq->nq * s->k * 4);
    memcpy(rq->d2.data(), sl.hd2 + (size_t)br.second * s->k, (size_t)rq->nq * s->k * 4);
    rq->t_done = now;
    rq->done = true;
    rq->status = s->fatal;
  }
  s->in_flight_bytes -= sl.bytes;
  s->batches += 1;
  s->queries += sl.rows;
  sl.batch.clear();
  sl.rows = 0;
  sl.bytes = 0;
  sl.busy = false;
}

void worker_loop(bdg_server* s) {
  cudaSetDevice(s->device);
  std::unique_lock<std::mutex> lk(s->mu);
  while (!s->stop) {
    bool progressed = false;
    // completions
    for (auto& sl : s->slots) {
      if (sl.busy && cudaEventQuery(sl.ev) == cudaSuccess) {
        finish(s, sl);
        progressed = true;
      }
    }
    if (progressed) s->cv_done.notify_all();
    // admissions: fill free streams with the oldest requests that fit
    for (auto& sl : s->slots) {
      if (sl.busy || s->pending.empty()) continue;
      while (!s->pending.empty()) {
        Request* rq = s->pending.front();
        const uint64_t b = row_bytes(s) * (uint64_t)rq->nq;
        if (sl.rows + rq->nq > s->max_batch) break;
        // admission by memory: all in-flight batches plus this one within the budget
        if (s->budget != 0 && s->in_flight_bytes + sl.bytes + b > s->budget) break;
        s->pending.pop_front();
        sl.batch.push_back({rq, sl.rows});
        sl.rows += rq->nq;
        sl.bytes += b;
      }
      if (sl.rows > 0) {
        s->in_flight_bytes += sl.bytes;
        launch(s, sl);
        progressed = true;
      }
    }
    bool any_busy = false;
    for (auto& sl : s->slots) any_busy |= sl.busy;
    if (!progressed) {
      // poll completions quickly while work is on the device, else sleep until submit
      if (any_busy) s->cv_work.wait_for(lk, std::chrono::microseconds(20));
      else s->cv_work.wait_for(lk, std::chrono::milliseconds(5));
    }
  }
}

}  // namespace

extern "C" {

bdg_status bdg_server_create(const bdg_graph* g, const float* feats, int32_t D, int32_t R,
                             int32_t k, int32_t ef_max, int32_t max_batch, int32_t n_streams,
                             uint64_t memory_budget, bdg_server** out) {
  if (!out) return bdg_set_error(BDG_EINVAL, "server_create: out is NULL");
  *out = nullptr;
  if (!g || !feats || max_batch < 1 || n_streams < 1 || n_streams > 16 || k < 1 || k > 32 ||
      R < k || R > 2048 || ef_max < 1 || ef_max > 2048)
    return bdg_set_error(BDG_EINVAL, "server_create: bad arguments");
  const int32_t* ids = nullptr;
  int64_t N = 0;
  int32_t kk = 0, bits = 0;
  BDG_TRY(bdg_graph_info(g, &ids, nullptr, &N, &kk, &bits));
  bdg_server* s = new bdg_server();
  s->g = g; s->feats = feats; s->D = D; s->R = R; s->k = k; s->ef_max = ef_max;
  s->max_batch = max_batch; s->W = bits / 64; s->N = N; s->budget = memory_budget;
  s->slots.resize(n_streams);
  cudaGetDevice(&s->device);
  bool ok = true;
  for (auto& sl : s->slots) {
    const size_t mb = (size_t)max_batch;
    ok = ok && cudaStreamCreateWithFlags(&sl.st, cudaStreamNonBlocking) == cudaSuccess;
    ok = ok && cudaEventCreateWithFlags(&sl.ev, cudaEventDisableTiming) == cudaSuccess;
    ok = ok && cudaMalloc(&sl.dq, mb * s->W * 8) == cudaSuccess;
    ok = ok && cudaMalloc(&sl.dqf, mb * D * 4) == cudaSuccess;
    ok = ok && cudaMalloc(&sl.def, mb * 4) == cudaSuccess;
    ok = ok && cudaMalloc(&sl.dcand, mb * R * 4) == cudaSuccess;
    ok = ok && cudaMalloc(&sl.dcdist, mb * R * 4) == cudaSuccess;
    ok = ok && cudaMalloc(&sl.dids, mb * k * 4) == cudaSuccess;
    ok = ok && cudaMalloc(&sl.dd2, mb * k * 4) == cudaSuccess;
    ok = ok && cudaMallocHost(&sl.hq, mb * s->W * 8) == cudaSuccess;
    ok = ok && cudaMallocHost(&sl.hqf, mb * D * 4) == cudaSuccess;
    ok = ok && cudaMallocHost(&sl.hef, mb * 4) == cudaSuccess;
    ok = ok && cudaMallocHost(&sl.hids, mb * k * 4) == cudaSuccess;
    ok = ok && cudaMallocHost(&sl.hd2, mb * k * 4) == cudaSuccess;
  }
  if (!ok) {
    cudaGetLastError();
    bdg_server_free(s);
    return bdg_set_error(BDG_ENOMEM, "server_create: allocating stream buffers failed");
  }
  s->worker = std::thread(worker_loop, s);
  *out = s;
  return BDG_OK;
}

bdg_status bdg_server_submit(bdg_server* s, const uint64_t* queries, const float* qfeats,
                             const int32_t* ef, int32_t nq, int64_t* request_id) {
  if (!s || !queries || !qfeats || !ef || !request_id || nq < 1)
    return bdg_set_error(BDG_EINVAL, "server_submit: bad arguments");
  if (nq > s->max_batch)
    return bdg_set_error(BDG_EINVAL, "server_submit: %d queries > max_batch %d", nq, s->max_batch);
  if (s->budget != 0 && row_bytes(s) * (uint64_t)nq > s->budget)
    return bdg_set_error(BDG_ENOMEM, "server_submit: request needs more than the memory budget");
  Request* rq = new Request();
  rq->nq = nq;
  rq->q.assign(queries, queries + (size_t)nq * s->W);
  rq->qf.assign(qfeats, qfeats + (size_t)nq * s->D);
  rq->ef.assign(ef, ef + nq);
  rq->ids.resize((size_t)nq * s->k);
  rq->d2.resize((size_t)nq * s->k);
  rq->t_arrive = Clock::now();
  {
    std::lock_guard<std::mutex> lk(s->mu);
    rq->id = s->next_id++;
    s->reqs[rq->id] = rq;
    s->pending.push_back(rq);
  }
  s->cv_work.notify_one();
  *request_id = rq->id;
  return BDG_OK;
}

bdg_status bdg_server_wait(bdg_server* s, int64_t request_id, int32_t* out_ids, float* out_d2,
                           double* latency_ms, int32_t timeout_ms) {
  if (!s) return bdg_set_error(BDG_EINVAL, "server_wait: server is NULL");
  std::unique_lock<std::mutex> lk(s->mu);
  auto it = s->reqs.find(request_id);
  if (it == s->reqs.end()) return bdg_set_error(BDG_EINVAL, "server_wait: unknown request");
  Request* rq = it->second;
  if (!s->cv_done.wait_for(lk, std::chrono::milliseconds(timeout_ms), [&] { return rq->done; }))
    return bdg_set_error(BDG_ETIMEOUT, "server_wait: request %lld not done after %d ms",
                         (long long)request_id, timeout_ms);
  if (out_ids) memcpy(out_ids, rq->ids.data(), rq->ids.size() * 4);
  if (out_d2) memcpy(out_d2, rq->d2.data(), rq->d2.size() * 4);
  if (latency_ms)
    *latency_ms = std::chrono::duration<double, std::milli>(rq->t_done - rq->t_arrive).count();
  const bdg_status st = rq->status;
  s->reqs.erase(it);
  delete rq;
  return st == BDG_OK ? BDG_OK : bdg_set_error(st, "server: a batch failed");
}

bdg_status bdg_server_stats(bdg_server* s, int64_t* batches, int64_t* queries, int64_t* pending,
                            uint64_t* in_flight_bytes) {
  if (!s) return bdg_set_error(BDG_EINVAL, "server_stats: server is NULL");
  std::lock_guard<std::mutex> lk(s->mu);
  if (batches) *batches = s->batches;
  if (queries) *queries = s->queries;
  if (pending) *pending = (int64_t)s->pending.size();
  if (in_flight_bytes) *in_flight_bytes = s->in_flight_bytes;
  return BDG_OK;
}

void bdg_server_free(bdg_server* s) {
  if (!s) return;
  {
    std::lock_guard<std::mutex> lk(s->mu);
    s->stop = true;
  }
  s->cv_work.notify_all();
  if (s->worker.joinable()) s->worker.join();
  for (auto& sl : s->slots) {
    if (sl.st) cudaStreamSynchronize(sl.st);
    cudaFree(sl.dq); cudaFree(sl.dqf); cudaFree(sl.def); cudaFree(sl.dcand);
    cudaFree(sl.dcdist); cudaFree(sl.dids); cudaFree(sl.dd2);
    cudaFreeHost(sl.hq); cudaFreeHost(sl.hqf); cudaFreeHost(sl.hef);
    cudaFreeHost(sl.hids); cudaFreeHost(sl.hd2);
    if (sl.ev) cudaEventDestroy(sl.ev);
    if (sl.st) cudaStreamDestroy(sl.st);
  }
  for (auto& kv : s->reqs) delete kv.second;
  delete s;
}

}  // extern "C"
