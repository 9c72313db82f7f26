// server.cu -- serving loop with continuous batching for oblivious scans.
//
// A query is one scan-select (Alg. 2 ProcessQuery over all rows of a table;
// §4.2).  Its per-row netlist is a DAG of circuit levels; the gates of one
// level are independent across rows and across queries.  The server keeps
// every admitted query's descriptors and intermediate wires on the device
// and runs rounds: each round gathers the next level (or the next part of a
// level) of every admitted query into one descriptor list and bootstraps it
// with one blind-rotation + keyswitch launch pair, so queries of different
// sizes, widths and predicates share launches.  A query that arrives while
// others run is admitted at the next round once its scratch fits the memory
// budget, and joins the following launches (continuous batching); a finished
// query frees its scratch at once.  Results are independent of the mix: each
// gate's output depends only on its own inputs and the keys.
//
// Pipelining.  All device work of the server goes to one stream, so a round
// that reads the outputs of an earlier round is ordered after it by the
// stream itself.  The worker therefore enqueues round r + 1 (its descriptor
// gather, its launches, the outputs no gate writes of queries that finish in
// it) while round r runs, and only then waits for round r's completion event
// to time-stamp and release the queries that finished in it; admission
// copies a query's scan program (its netlist and buffer pointers, a few KB)
// asynchronously and generates its descriptors on the device.  The GPU is
// never idle between rounds while there is work, and no round waits for the
// host's bookkeeping.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <mutex>
#include <thread>
#include <vector>

#include "engine.h"

namespace fsql {
namespace {

using Clock = std::chrono::steady_clock;

// First-fit sub-allocator over [0, size) of one device block.
class Pool {
 public:
  explicit Pool(size_t size) : size_(size) { free_[0] = size; }
  bool alloc(size_t bytes, size_t* off) {
    bytes = (bytes + 255) / 256 * 256;
    for (auto it = free_.begin(); it != free_.end(); ++it) {
      if (it->second >= bytes) {
        *off = it->first;
        const size_t rest = it->second - bytes, start = it->first + bytes;
        free_.erase(it);
        if (rest) free_[start] = rest;
        used_ += bytes;
        return true;
      }
    }
    return false;
  }
  void release(size_t off, size_t bytes) {
    bytes = (bytes + 255) / 256 * 256;
    used_ -= bytes;
    auto it = free_.emplace(off, bytes).first;
    auto next = std::next(it);
    if (next != free_.end() && it->first + it->second == next->first) {
      it->second += next->second;
      free_.erase(next);
    }
    if (it != free_.begin()) {
      auto prev = std::prev(it);
      if (prev->first + prev->second == it->first) {
        prev->second += it->second;
        free_.erase(it);
      }
    }
  }
  size_t used() const { return used_; }
  size_t size() const { return size_; }

 private:
  size_t size_, used_ = 0;
  std::map<size_t, size_t> free_;
};

enum { Q_WAITING = 0, Q_RUNNING = 1, Q_DONE = 2, Q_FAILED = 3, Q_CANCELLED = 4 };

struct Query {
  uint64_t id = 0;
  fsql_query q{};
  Netlist nl;
  std::vector<size_t> level_offset;
  size_t total_gates = 0;
  size_t bytes = 0, off = 0;  // pool block: scan program, gate descriptors, output descriptors, wires
  GateDesc* d_desc = nullptr;
  OutDesc* d_lits = nullptr;  // outputs no gate writes (plaintext constants)
  size_t n_lits = 0;
  int level = 0;              // next level to enqueue
  size_t done_in_level = 0;   // gates of that level already enqueued
  bool all_issued = false;    // every gate and the literal outputs enqueued
  int inflight = 0;           // enqueued rounds holding work of this query, not yet seen complete
  int state = Q_WAITING;
  bool cancel = false;
  Clock::time_point t_submit, t_done;
};

size_t round256(size_t b) { return (b + 255) / 256 * 256; }

size_t query_bytes(const Netlist& nl, const fsql_query& q, size_t words) {
  const size_t prog = scan_program_bytes(nl);
  const size_t desc = q.rows * nl.type.size() * sizeof(GateDesc);
  const size_t lits = q.rows * nl.literal_outs.size() * sizeof(OutDesc);
  const size_t wires = q.rows * static_cast<size_t>(scan_internal_wires(nl)) * words * 4;
  return round256(prog) + round256(desc) + round256(lits) + wires;
}

// One enqueued round: its queries and the events around its device work.
struct Round {
  cudaEvent_t start = nullptr, end = nullptr;
  std::vector<Query*> queries;
  size_t gates = 0;
};

constexpr int kPipelineDepth = 2;  // rounds enqueued ahead of the one being waited for

}  // namespace

struct Server {
  Ctx* ctx = nullptr;
  size_t max_batch = 0;
  size_t fill_gates = 0;  // admission stops while the running queries' current levels hold this many gates
  Pool pool{0};
  uint8_t* d_pool = nullptr;
  GateDesc* d_round = nullptr;
  uint32_t* d_big = nullptr;
  cudaStream_t stream = nullptr;
  std::vector<cudaEvent_t> free_events;
  std::mutex mu;
  std::condition_variable cv;
  std::thread worker;
  bool stop = false;
  uint64_t next_id = 1;
  std::deque<Query*> waiting;
  std::vector<Query*> running;
  std::deque<Round> inflight;
  std::map<uint64_t, Query*> all;
  // statistics
  uint64_t rounds = 0, gates = 0, completed = 0;
  double busy_ms = 0.0;
  std::vector<double> latencies_ms;
  std::string error;

  cudaEvent_t get_event() {
    if (!free_events.empty()) {
      cudaEvent_t e = free_events.back();
      free_events.pop_back();
      return e;
    }
    cudaEvent_t e = nullptr;
    if (cudaEventCreate(&e) != cudaSuccess) return nullptr;
    return e;
  }

  // Gates the running queries still have in their current levels: the size
  // of the next round before anything else is admitted.
  size_t pending_gates_locked() const {
    size_t g = 0;
    for (const Query* q : running)
      if (!q->all_issued && !q->cancel && q->state == Q_RUNNING && q->level < q->nl.levels)
        g += q->level_offset[q->level + 1] - q->level_offset[q->level] - q->done_in_level;
    return g;
  }

  // Admit waiting queries in arrival order while their blocks fit and the
  // running queries' current levels do not already fill an efficient round
  // (fill_gates: 64 gates per SM, about 21 waves of the 3-gate kernel, or
  // max_batch if smaller) (caller holds mu): copy the
  // scan program, generate the descriptors on the device, copy the
  // descriptors of the outputs no gate writes (all on the stream).  The
  // round-fill condition keeps early arrivals from being slowed down by
  // later ones once the GPU is busy (queries run closer to arrival order),
  // while every round that can be full still is.
  void admit_locked() {
    size_t pending = pending_gates_locked();
    while (!waiting.empty()) {
      Query* q = waiting.front();
      if (q->cancel) {
        q->state = Q_CANCELLED;
        waiting.pop_front();
        continue;
      }
      if (pending >= fill_gates) break;
      size_t off = 0;
      if (!pool.alloc(q->bytes, &off)) break;
      q->off = off;
      uint8_t* base = d_pool + off;
      const size_t prog_bytes = round256(scan_program_bytes(q->nl));
      const size_t desc_bytes = round256(q->total_gates * sizeof(GateDesc));
      const size_t lit_bytes = round256(q->q.rows * q->nl.literal_outs.size() * sizeof(OutDesc));
      q->d_desc = reinterpret_cast<GateDesc*>(base + prog_bytes);
      q->d_lits = reinterpret_cast<OutDesc*>(base + prog_bytes + desc_bytes);
      ScanIO io;
      io.column = q->q.d_column;
      io.rows = q->q.rows;
      io.width = q->q.width;
      io.pred = q->q.pred;
      io.cst = q->q.d_const;
      io.n_payloads = q->q.n_payloads;
      io.payloads = q->q.d_payloads;
      io.payload_width = q->q.payload_width;
      io.match = q->q.d_match;
      io.outs = q->q.d_out_payloads;
      io.wires = reinterpret_cast<uint32_t*>(base + prog_bytes + desc_bytes + lit_bytes);
      io.words = ctx->p.n + 1;
      std::vector<uint8_t> prog;
      std::vector<OutDesc> hl;
      scan_literals(q->nl, io, &hl);
      q->n_lits = hl.size();
      // pageable sources: each copy is staged before cudaMemcpyAsync returns
      const bool ok = build_scan_program(q->nl, io, &prog, &q->level_offset) &&
                      cudaMemcpyAsync(base, prog.data(), prog.size(), cudaMemcpyHostToDevice, stream) == cudaSuccess &&
                      launch_gen_desc(base, q->d_desc, q->total_gates, stream) == FSQL_OK &&
                      (hl.empty() || cudaMemcpyAsync(q->d_lits, hl.data(), hl.size() * sizeof(OutDesc),
                                                     cudaMemcpyHostToDevice, stream) == cudaSuccess);
      if (!ok) {
        pool.release(q->off, q->bytes);
        q->state = Q_FAILED;
        error = "admission copy failed";
        waiting.pop_front();
        continue;
      }
      q->state = Q_RUNNING;
      running.push_back(q);
      waiting.pop_front();
      if (q->nl.levels > 0) pending += q->level_offset[1] - q->level_offset[0];
    }
  }

  // A query whose last work completed (caller holds mu).
  void complete_locked(Query* q) {
    pool.release(q->off, q->bytes);
    if (q->state == Q_FAILED) return;
    if (q->cancel) {
      q->state = Q_CANCELLED;
      return;
    }
    q->state = Q_DONE;
    q->t_done = Clock::now();
    ++completed;
    latencies_ms.push_back(std::chrono::duration<double, std::milli>(q->t_done - q->t_submit).count());
  }

  // Wait for the oldest enqueued round and retire the queries it finishes
  // (called with lk held; waits without it).
  void retire_oldest(std::unique_lock<std::mutex>& lk) {
    Round r = std::move(inflight.front());
    inflight.pop_front();
    lk.unlock();
    cudaError_t e = cudaEventSynchronize(r.end);
    float ms = 0.f;
    if (e == cudaSuccess && r.start) e = cudaEventElapsedTime(&ms, r.start, r.end);
    lk.lock();
    busy_ms += ms;
    if (e != cudaSuccess) {
      error = std::string("round failed: ") + cudaGetErrorString(e);
      for (Query* q : r.queries) q->state = Q_FAILED;
    }
    for (Query* q : r.queries) {
      if (--q->inflight == 0 && (q->all_issued || q->cancel || q->state == Q_FAILED)) {
        auto it = std::find(running.begin(), running.end(), q);
        if (it != running.end()) {
          complete_locked(q);
          running.erase(it);
        }
      }
    }
    if (r.start) free_events.push_back(r.start);
    free_events.push_back(r.end);
    cv.notify_all();
  }

  void run() {
    cudaSetDevice(ctx->device);
    struct Seg {
      Query* q;
      size_t start, n;
    };
    std::unique_lock<std::mutex> lk(mu);
    while (!stop || !inflight.empty()) {
      if (!stop) admit_locked();
      // cancelled or failed queries with nothing in flight leave now
      for (auto it = running.begin(); it != running.end();) {
        Query* q = *it;
        if ((q->cancel || q->state == Q_FAILED) && q->inflight == 0) {
          complete_locked(q);
          it = running.erase(it);
        } else {
          ++it;
        }
      }
      if (stop) {  // no new round after a stop: wait for the enqueued ones
        if (!inflight.empty()) retire_oldest(lk);
        continue;
      }
      // gather the next level (part) of every running query, oldest first
      std::vector<Seg> segs;
      std::vector<Query*> lit_only;  // queries whose only remaining work is their literal outputs
      size_t total = 0;
      for (Query* q : running) {
        if (q->all_issued || q->cancel || q->state == Q_FAILED) continue;
        if (q->level == q->nl.levels) {
          lit_only.push_back(q);
          continue;
        }
        if (total >= max_batch) continue;
        const size_t lb = q->level_offset[q->level], le = q->level_offset[q->level + 1];
        const size_t start = lb + q->done_in_level;
        const size_t n = std::min(le - start, max_batch - total);
        if (n == 0) continue;
        segs.push_back({q, start, n});
        total += n;
      }
      if (segs.empty() && lit_only.empty()) {
        if (!inflight.empty()) {
          retire_oldest(lk);
        } else if (!stop) {
          cv.wait_for(lk, std::chrono::milliseconds(50));
        }
        continue;
      }
      // advance the bookkeeping as enqueued; a query whose last gates are in
      // this round also gets its literal outputs enqueued after them
      Round r;
      r.gates = total;
      std::vector<Query*> finishing;
      for (const Seg& sg : segs) {
        Query* q = sg.q;
        q->done_in_level += sg.n;
        if (q->level_offset[q->level] + q->done_in_level == q->level_offset[q->level + 1]) {
          ++q->level;
          q->done_in_level = 0;
        }
        if (q->level == q->nl.levels) finishing.push_back(q);
      }
      for (Query* q : lit_only) finishing.push_back(q);
      for (const Seg& sg : segs) r.queries.push_back(sg.q);
      for (Query* q : lit_only) r.queries.push_back(q);
      for (Query* q : finishing) q->all_issued = true;
      for (Query* q : r.queries) ++q->inflight;
      r.start = get_event();
      r.end = get_event();
      lk.unlock();
      bool ok = r.end != nullptr;
      if (ok && r.start) ok = cudaEventRecord(r.start, stream) == cudaSuccess;
      size_t pos = 0;
      for (const Seg& sg : segs) {
        ok = ok && cudaMemcpyAsync(d_round + pos, sg.q->d_desc + sg.start, sg.n * sizeof(GateDesc),
                                   cudaMemcpyDeviceToDevice, stream) == cudaSuccess;
        pos += sg.n;
      }
      if (ok && total) {
        std::lock_guard<std::mutex> ctx_lk(ctx->mu);  // the context's launch bookkeeping is shared
        ok = launch_gates(*ctx, d_round, total, d_big, stream) == FSQL_OK;
      }
      for (Query* q : finishing)
        if (ok && q->n_lits) ok = launch_literals(q->d_lits, q->n_lits, static_cast<int>(ctx->p.n), stream) == FSQL_OK;
      if (ok) ok = cudaEventRecord(r.end, stream) == cudaSuccess;
      lk.lock();
      ++rounds;
      gates += total;
      if (!ok) {
        error = std::string("round launch failed: ") + cudaGetErrorString(cudaGetLastError());
        for (Query* q : r.queries) q->state = Q_FAILED;
        // nothing of this round can be waited for: undo its in-flight marks
        for (Query* q : r.queries) --q->inflight;
        if (r.start) free_events.push_back(r.start);
        if (r.end) free_events.push_back(r.end);
        cv.notify_all();
        continue;
      }
      inflight.push_back(std::move(r));
      while (static_cast<int>(inflight.size()) > kPipelineDepth) retire_oldest(lk);
    }
  }
};

}  // namespace fsql

using fsql::Server;

namespace {
int arg_error(const char* msg) {
  fsql::set_error(msg);
  return FSQL_ERR_ARG;
}
double percentile(std::vector<double> v, double p) {
  if (v.empty()) return 0.0;
  std::sort(v.begin(), v.end());
  const double idx = p * (v.size() - 1);
  const size_t lo = static_cast<size_t>(idx), hi = std::min(lo + 1, v.size() - 1);
  return v[lo] + (v[hi] - v[lo]) * (idx - lo);
}
}  // namespace

extern "C" {

int fsql_server_create(fsql_ctx* ctx, size_t scratch_budget_bytes, size_t max_batch_gates, fsql_server** out) {
  if (!ctx || !out) return arg_error("null argument");
  *out = nullptr;
  auto* c = reinterpret_cast<fsql::Ctx*>(ctx);
  if (c->device < 0 || !c->d_bkhat) return arg_error("context has no device keys");
  if (scratch_budget_bytes < (1u << 20)) return arg_error("scratch budget below 1 MiB");
  if (max_batch_gates == 0) max_batch_gates = size_t(1) << 17;
  if (max_batch_gates > (size_t(1) << 20)) return arg_error("max_batch_gates above 2^20");
  if (cudaSetDevice(c->device) != cudaSuccess) return arg_error("cudaSetDevice failed");
  auto* s = new Server();
  s->ctx = c;
  s->max_batch = max_batch_gates;
  s->fill_gates = std::min<size_t>(max_batch_gates, static_cast<size_t>(64) * std::max(1, c->sm_count));
  s->pool = fsql::Pool(scratch_budget_bytes);
  cudaError_t e = cudaMalloc(&s->d_pool, scratch_budget_bytes);
  if (e == cudaSuccess) e = cudaMalloc(&s->d_round, max_batch_gates * sizeof(fsql::GateDesc));
  if (e == cudaSuccess) e = cudaMalloc(&s->d_big, std::min<size_t>(max_batch_gates, size_t(1) << 18) * (fsql::kN + 1) * 4);
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&s->stream, cudaStreamNonBlocking);
  if (e != cudaSuccess) {
    fsql::set_error(std::string("server allocation: ") + cudaGetErrorString(e));
    cudaFree(s->d_pool);
    cudaFree(s->d_round);
    cudaFree(s->d_big);
    delete s;
    return FSQL_ERR_OOM;
  }
  s->worker = std::thread([s] { s->run(); });
  *out = reinterpret_cast<fsql_server*>(s);
  return FSQL_OK;
}

int fsql_server_submit(fsql_server* server, const fsql_query* q, uint64_t* id) {
  if (!server || !q || !id) return arg_error("null argument");
  auto* s = reinterpret_cast<Server*>(server);
  if (q->rows == 0) return arg_error("empty table");
  if (!q->d_column || (!q->d_const && !q->plain) || !q->d_match)
    return arg_error("null column, constant or match pointer");
  if (q->n_payloads > FSQL_MAX_PAYLOADS) return arg_error("too many payload columns");
  for (uint32_t k = 0; k < q->n_payloads; ++k)
    if (!q->d_payloads[k] || !q->d_out_payloads[k]) return arg_error("null payload pointer");
  auto* qq = new fsql::Query();
  qq->q = *q;
  const bool range = q->pred == FSQL_RANGE || q->pred == FSQL_RANGE_MAJ;
  if (q->plain && q->width < 64 && (q->consts[0] >> q->width || (range && q->consts[1] >> q->width))) {
    delete qq;
    return arg_error("constant wider than the column");
  }
  const bool built = q->plain ? fsql::build_netlist_plain(q->pred, q->width, q->n_payloads, q->payload_width,
                                                          q->consts[0], range ? q->consts[1] : 0, &qq->nl)
                              : fsql::build_netlist(q->pred, q->width, q->n_payloads, q->payload_width, &qq->nl);
  if (!built) {
    delete qq;
    return arg_error("bad predicate shape");
  }
  qq->total_gates = q->rows * qq->nl.type.size();
  qq->bytes = fsql::query_bytes(qq->nl, *q, s->ctx->p.n + 1);
  if (qq->bytes > s->pool.size()) {
    delete qq;
    fsql::set_error("query scratch exceeds the server's whole memory budget");
    return FSQL_ERR_ADMISSION;
  }
  qq->t_submit = fsql::Clock::now();
  {
    std::lock_guard<std::mutex> lk(s->mu);
    qq->id = s->next_id++;
    s->all[qq->id] = qq;
    s->waiting.push_back(qq);
  }
  s->cv.notify_all();
  *id = qq->id;
  return FSQL_OK;
}

int fsql_server_status(fsql_server* server, uint64_t id, int* state, double* latency_ms) {
  if (!server || !state) return arg_error("null argument");
  auto* s = reinterpret_cast<Server*>(server);
  std::lock_guard<std::mutex> lk(s->mu);
  auto it = s->all.find(id);
  if (it == s->all.end()) return arg_error("unknown query id");
  *state = it->second->state;
  if (latency_ms)
    *latency_ms = it->second->state == fsql::Q_DONE
                      ? std::chrono::duration<double, std::milli>(it->second->t_done - it->second->t_submit).count()
                      : -1.0;
  return FSQL_OK;
}

int fsql_server_wait(fsql_server* server, uint64_t id, double timeout_ms) {
  if (!server) return arg_error("null server");
  auto* s = reinterpret_cast<Server*>(server);
  std::unique_lock<std::mutex> lk(s->mu);
  auto it = s->all.find(id);
  if (it == s->all.end()) return arg_error("unknown query id");
  fsql::Query* q = it->second;
  const auto deadline = fsql::Clock::now() + std::chrono::duration<double, std::milli>(timeout_ms);
  while (q->state == fsql::Q_WAITING || q->state == fsql::Q_RUNNING) {
    if (s->cv.wait_until(lk, deadline) == std::cv_status::timeout &&
        (q->state == fsql::Q_WAITING || q->state == fsql::Q_RUNNING)) {
      fsql::set_error("query still running at the timeout");
      return FSQL_ERR_TIMEOUT;
    }
  }
  if (q->state == fsql::Q_FAILED) {
    fsql::set_error(s->error.empty() ? "query failed" : s->error);
    return FSQL_ERR_CUDA;
  }
  return FSQL_OK;
}

int fsql_server_cancel(fsql_server* server, uint64_t id) {
  if (!server) return arg_error("null server");
  auto* s = reinterpret_cast<Server*>(server);
  {
    std::lock_guard<std::mutex> lk(s->mu);
    auto it = s->all.find(id);
    if (it == s->all.end()) return arg_error("unknown query id");
    it->second->cancel = true;
  }
  s->cv.notify_all();
  return FSQL_OK;
}

int fsql_server_get_stats(fsql_server* server, fsql_server_stats* out) {
  if (!server || !out) return arg_error("null argument");
  auto* s = reinterpret_cast<Server*>(server);
  std::lock_guard<std::mutex> lk(s->mu);
  out->completed = s->completed;
  out->rounds = s->rounds;
  out->gates = s->gates;
  out->busy_ms = s->busy_ms;
  out->p50_ms = percentile(s->latencies_ms, 0.50);
  out->p99_ms = percentile(s->latencies_ms, 0.99);
  out->waiting = s->waiting.size();
  out->running = s->running.size();
  out->scratch_used = s->pool.used();
  return FSQL_OK;
}

void fsql_server_destroy(fsql_server* server) {
  if (!server) return;
  auto* s = reinterpret_cast<Server*>(server);
  {
    std::lock_guard<std::mutex> lk(s->mu);
    s->stop = true;
  }
  s->cv.notify_all();
  if (s->worker.joinable()) s->worker.join();
  cudaSetDevice(s->ctx->device);
  cudaStreamSynchronize(s->stream);
  for (cudaEvent_t e : s->free_events) cudaEventDestroy(e);
  cudaStreamDestroy(s->stream);
  cudaFree(s->d_pool);
  cudaFree(s->d_round);
  cudaFree(s->d_big);
  for (auto& kv : s->all) delete kv.second;
  delete s;
}

}  // extern "C"
