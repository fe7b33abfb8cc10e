// Serving: a request loop with continuous batching over the batch pipeline
// of sky_pipeline.cu.
//
// sky_submit queues a query and returns a ticket at once.  Worker threads
// (each with its own Runner: stream, resident workspace, pinned staging)
// take the queued queries in arrival order into a batch as long as the
// batch's device memory fits the worker's share of the serving budget, run
// the batch (every local skyline of the batch in one persistent launch,
// every sequential merge in a second one), and publish each query's result.
// A query that arrives while a batch is on the GPU joins the next batch of
// whichever worker frees up first; with two or more workers, one batch's
// copies and HBM-bound stages run while another's dominance kernel runs.
// The workers' persistent launches are ordered on the GPU by an EngineGate
// so that two cooperative grids never wait on each other for SMs.
#include <chrono>
#include <condition_variable>
#include <deque>
#include <memory>
#include <thread>
#include <unordered_map>
#include "sky_serve.cuh"

namespace sky {

namespace {
using Clock = std::chrono::steady_clock;
double us_between(Clock::time_point a, Clock::time_point b) {
  return std::chrono::duration<double, std::micro>(b - a).count();
}
}  // namespace

struct Server::Ticket {
  u64 id = 0;
  const float* points = nullptr;
  u64 n = 0;
  u32 d = 0;
  sky_params params{};
  bool has_params = false;
  size_t bytes = 0;
  std::vector<u32> result;
  u64 count = 0;
  sky_status status = SKY_OK;
  bool done = false;
  u32 batch_queries = 0;
  sky_stats stats{};
  Clock::time_point t_submit, t_start, t_done;
};

// Statistics of collected tickets kept for sky_get_stats (the most recent).
constexpr size_t KEEP_COLLECTED_STATS = 4096;

struct Server::Impl {
  int device = 0;
  u32 max_batch = 64;
  size_t budget_per_worker = 0;
  std::mutex mu;
  std::condition_variable cv_work, cv_done;
  std::deque<Ticket*> pending;
  std::unordered_map<u64, std::unique_ptr<Ticket>> tickets;
  std::vector<std::unique_ptr<Runner>> runners;
  std::vector<cudaStream_t> streams;
  std::vector<std::thread> workers;
  EngineGate gate;
  bool stop = false;
  u64 next_id = 1;
  u64 batches = 0;
  std::deque<std::pair<u64, sky_stats>> collected;  // (ticket, statistics), oldest first

  void loop(u32 w);
};

Server::Server() : impl_(new Impl) {}

Server::~Server() { shutdown(); }

sky_status Server::start(int device, const sky_serve_config& cfg, int timing, std::string* msg) {
  Impl& I = *impl_;
  I.device = device;
  const u32 nw = cfg.workers ? cfg.workers : 2;
  I.max_batch = cfg.max_batch ? cfg.max_batch : 64;
  if (nw > 16) {
    *msg = "at most 16 serving workers";
    return SKY_EINVAL;
  }
  if (cudaSetDevice(device) != cudaSuccess) return SKY_ECUDA;
  {
    std::lock_guard<std::mutex> g(I.mu);
    I.stop = false;
  }
  size_t budget = cfg.mem_budget_bytes;
  if (!budget) {
    size_t free_b = 0, total_b = 0;
    if (cudaMemGetInfo(&free_b, &total_b) != cudaSuccess) return SKY_ECUDA;
    budget = free_b / 2;
  }
  I.budget_per_worker = budget / nw;
  for (u32 w = 0; w < nw; ++w) {
    cudaStream_t s = nullptr;
    if (cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking) != cudaSuccess) return SKY_ECUDA;
    I.streams.push_back(s);
    std::unique_ptr<Runner> r(new Runner());
    sky_status st = r->init(device, I.budget_per_worker);
    if (st != SKY_OK) return st;
    r->stream = s;
    r->timing = timing;
    r->gate = nw > 1 ? &I.gate : nullptr;
    I.runners.push_back(std::move(r));
  }
  for (u32 w = 0; w < nw; ++w) I.workers.emplace_back([this, w] { impl_->loop(w); });
  return SKY_OK;
}

bool Server::running() const { return !impl_->workers.empty(); }

void Server::shutdown() {
  if (!impl_) return;
  Impl& I = *impl_;
  {
    std::lock_guard<std::mutex> g(I.mu);
    I.stop = true;
  }
  I.cv_work.notify_all();
  for (auto& t : I.workers) t.join();
  I.workers.clear();
  // the gate refers to an event of one of the Runners destroyed below
  {
    std::lock_guard<std::mutex> g(I.gate.mu);
    I.gate.last = nullptr;
  }
  I.runners.clear();
  for (auto s : I.streams) {
    cudaSetDevice(I.device);
    cudaStreamDestroy(s);
  }
  I.streams.clear();
}

void Server::Impl::loop(u32 w) {
  cudaSetDevice(device);
  Runner& R = *runners[w];
  for (;;) {
    std::vector<Ticket*> batch;
    {
      std::unique_lock<std::mutex> lk(mu);
      cv_work.wait(lk, [&] { return stop || !pending.empty(); });
      if (pending.empty()) return;  // stop requested and nothing left
      // admission by device memory: arrival order, up to max_batch queries
      // whose workspaces fit this worker's share of the budget together (a
      // query too large for the share alone runs alone and fails ENOMEM)
      size_t bytes = 0;
      while (!pending.empty() && batch.size() < max_batch) {
        Ticket* t = pending.front();
        if (!batch.empty() && bytes + t->bytes > budget_per_worker) break;
        pending.pop_front();
        batch.push_back(t);
        bytes += t->bytes;
      }
      ++batches;
    }
    const auto t0 = Clock::now();
    std::vector<Runner::Query> qs(batch.size());
    for (size_t i = 0; i < batch.size(); ++i) {
      Ticket* t = batch[i];
      t->t_start = t0;
      t->result.assign(t->n ? t->n : 1, 0u);
      qs[i].points = t->points;
      qs[i].n = t->n;
      qs[i].d = t->d;
      qs[i].params = t->has_params ? &t->params : nullptr;
      qs[i].out_idx = t->result.data();
      qs[i].out_count = &t->count;
    }
    sky_status s = R.run(qs.data(), (u32)qs.size());
    const auto t1 = Clock::now();
    {
      std::lock_guard<std::mutex> g(mu);
      // a failure of the whole batch (memory, CUDA) sets no per-query
      // status: then every query of the batch gets it
      bool any_query_failed = false;
      for (auto& q : qs) any_query_failed |= q.status != SKY_OK;
      for (size_t i = 0; i < batch.size(); ++i) {
        Ticket* t = batch[i];
        t->status = qs[i].status;
        if (s != SKY_OK && !any_query_failed) t->status = s;
        if (t->status != SKY_OK) t->count = 0;
        t->result.resize(t->count);
        t->batch_queries = (u32)batch.size();
        // the query's own sizes and counts; launches and device times are
        // those of its whole batch (the batch shares its engine launches)
        t->stats = qs[i].stats;
        t->stats.launches = R.stats.launches;
        t->stats.ms_total = R.stats.ms_total;
        for (int k = 0; k < 6; ++k) t->stats.ms_phase[k] = R.stats.ms_phase[k];
        t->stats.ms_dom_local = R.stats.ms_dom_local;
        t->stats.ms_dom_merge = R.stats.ms_dom_merge;
        t->t_done = t1;
        t->done = true;
      }
    }
    cv_done.notify_all();
  }
}

sky_status Server::submit(const float* points, u64 n, u32 d, const sky_params* params, u64* ticket,
                          std::string* msg) {
  Impl& I = *impl_;
  sky_status s = validate_query(points, n, d, params, msg);
  if (s != SKY_OK) return s;
  std::unique_ptr<Ticket> t(new Ticket());
  t->points = points;
  t->n = n;
  t->d = d;
  if (params) {
    t->params = *params;
    t->has_params = true;
  }
  t->bytes = Runner::query_bytes(n, d, params);
  t->t_submit = Clock::now();
  Ticket* raw = t.get();
  {
    std::lock_guard<std::mutex> g(I.mu);
    t->id = I.next_id++;
    *ticket = t->id;
    if (n == 0) {
      t->done = true;
      t->t_start = t->t_done = t->t_submit;
    } else {
      I.pending.push_back(raw);
    }
    I.tickets.emplace(t->id, std::move(t));
  }
  I.cv_work.notify_one();
  return SKY_OK;
}

sky_status Server::poll(u64 ticket) {
  Impl& I = *impl_;
  std::lock_guard<std::mutex> g(I.mu);
  auto it = I.tickets.find(ticket);
  if (it == I.tickets.end()) return SKY_ECANCELLED;
  return it->second->done ? SKY_OK : SKY_EBUSY;
}

sky_status Server::wait(u64 ticket, u32* out_idx, u64* out_count, int64_t timeout_us, sky_ticket_info* info,
                        std::string* msg) {
  Impl& I = *impl_;
  std::unique_ptr<Ticket> t;
  {
    std::unique_lock<std::mutex> lk(I.mu);
    auto it = I.tickets.find(ticket);
    if (it == I.tickets.end()) return SKY_ECANCELLED;
    Ticket* raw = it->second.get();
    auto ready = [&] { return raw->done; };
    if (timeout_us < 0) {
      I.cv_done.wait(lk, ready);
    } else if (!I.cv_done.wait_for(lk, std::chrono::microseconds(timeout_us), ready)) {
      return SKY_EBUSY;
    }
    t = std::move(it->second);
    I.tickets.erase(it);
    I.collected.emplace_back(t->id, t->stats);
    if (I.collected.size() > KEEP_COLLECTED_STATS) I.collected.pop_front();
  }
  if (info) {
    info->queue_us = us_between(t->t_submit, t->t_start);
    info->run_us = us_between(t->t_start, t->t_done);
    info->latency_us = us_between(t->t_submit, t->t_done);
    info->batch_queries = t->batch_queries;
  }
  if (out_count) *out_count = t->count;
  if (t->status != SKY_OK) {
    *msg = "query failed";
    return t->status;
  }
  if (t->count && out_idx) {
    cudaSetDevice(I.device);
    if (cudaMemcpy(out_idx, t->result.data(), t->count * sizeof(u32), cudaMemcpyDefault) != cudaSuccess) {
      cudaGetLastError();
      *msg = "copy of the result failed";
      return SKY_ECUDA;
    }
  }
  return SKY_OK;
}

sky_status Server::stats(u64 ticket, sky_stats* out) {
  Impl& I = *impl_;
  std::lock_guard<std::mutex> g(I.mu);
  auto it = I.tickets.find(ticket);
  if (it != I.tickets.end()) {
    if (!it->second->done) return SKY_EBUSY;
    *out = it->second->stats;
    return SKY_OK;
  }
  for (auto c = I.collected.rbegin(); c != I.collected.rend(); ++c) {
    if (c->first == ticket) {
      *out = c->second;
      return SKY_OK;
    }
  }
  return SKY_ECANCELLED;
}

u64 Server::batches() const {
  std::lock_guard<std::mutex> g(impl_->mu);
  return impl_->batches;
}

}  // namespace sky
