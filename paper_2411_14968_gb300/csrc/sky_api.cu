// C ABI of libskyline (include/skyline.h): contexts and the entry points of
// the partitioned skyline method.  The orchestration of Algorithm 2 over one
// query or a batch of queries is the Runner of sky_pipeline.cu; every step
// of it runs in the kernels of sky_prep.cu, sky_prims.cu, sky_dom.cu and
// sky_engine.cu.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <initializer_list>
#include <cstring>
#include <string>
#include <vector>
#include "../../include/skyline.h"
#include "../../include/skyline_diag.h"
#include "sky_internal.cuh"
#include "sky_pipeline.cuh"
#include "sky_serve.cuh"
#include <memory>
#include <mutex>

using namespace sky;

namespace sky {
u64& launch_counter() {
  static thread_local u64 count = 0;
  return count;
}
}  // namespace sky

struct sky_ctx {
  Runner run;                     // synchronous calls
  std::mutex serve_mu;            // guards the creation of the server
  std::unique_ptr<Server> server; // serving loop (sky_submit / sky_wait)
  std::string serve_error;
};

namespace sky {
int ctx_timing(sky_ctx* ctx) { return ctx ? ctx->run.timing : 0; }
}  // namespace sky

namespace {

sky_status run_one(sky_ctx* ctx, const float* points, u64 n, u32 d, const sky_params* pa, u32* out_idx,
                   u64* out_count, u32* out_pid, u8* out_stage) {
  if (!ctx) return SKY_EINVAL;
  Runner::Query q;
  q.points = points;
  q.n = n;
  q.d = d;
  q.params = pa;
  q.out_idx = out_idx;
  q.out_count = out_count;
  q.out_pid = out_pid;
  q.out_stage = out_stage;
  sky_status s = ctx->run.run(&q, 1);
  return s;
}

}  // namespace

extern "C" {

void sky_params_init(sky_params* p) {
  if (!p) return;
  memset(p, 0, sizeof(*p));
  p->struct_size = sizeof(sky_params);
  p->scheme = SKY_NONE;
  p->num_partitions = 1;
  for (int a = 0; a < 8; ++a) p->slices[a] = 1;
  p->grid_filter = 1;
  p->rep = SKY_REP_NONE;
  p->reps_per_partition = 1;
  p->merge = SKY_MERGE_SEQUENTIAL;
  p->exec = SKY_EXEC_PERSISTENT;
  p->images = SKY_IMAGES_VALUES;
}

sky_status sky_create(sky_ctx** ctx, int device, size_t mem_budget_bytes) {
  if (!ctx) return SKY_EINVAL;
  *ctx = nullptr;
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || device < 0 || device >= ndev) {
    cudaGetLastError();
    return SKY_ECUDA;
  }
  if (cudaSetDevice(device) != cudaSuccess) return SKY_ECUDA;
  sky_ctx* c = new sky_ctx();
  sky_status s = c->run.init(device, mem_budget_bytes);
  if (s != SKY_OK) {
    delete c;
    return s;
  }
  device_sm_count();
  *ctx = c;
  return SKY_OK;
}

sky_status sky_set_stream(sky_ctx* ctx, void* cuda_stream) {
  if (!ctx) return SKY_EINVAL;
  ctx->run.stream = reinterpret_cast<cudaStream_t>(cuda_stream);
  return SKY_OK;
}

sky_status sky_set_timing(sky_ctx* ctx, int on) {
  if (!ctx) return SKY_EINVAL;
  ctx->run.timing = on ? 1 : 0;
  return SKY_OK;
}

sky_status sky_skyline(sky_ctx* ctx, const float* points, uint64_t n, uint32_t d, const sky_params* params,
                       uint32_t* out_idx, uint64_t* out_count) {
  return run_one(ctx, points, n, d, params, out_idx, out_count, nullptr, nullptr);
}

sky_status sky_skyline_ex(sky_ctx* ctx, const float* points, uint64_t n, uint32_t d, const sky_params* params,
                          uint32_t* out_idx, uint64_t* out_count, uint32_t* out_pid, uint8_t* out_stage) {
  return run_one(ctx, points, n, d, params, out_idx, out_count, out_pid, out_stage);
}

sky_status sky_skyline_batch(sky_ctx* ctx, sky_query* queries, uint32_t nq) {
  if (!ctx || (nq && !queries)) return SKY_EINVAL;
  std::vector<Runner::Query> qs(nq);
  for (u32 i = 0; i < nq; ++i) {
    qs[i].points = queries[i].points;
    qs[i].n = queries[i].n;
    qs[i].d = queries[i].d;
    qs[i].params = queries[i].params;
    qs[i].out_idx = queries[i].out_idx;
    qs[i].out_count = queries[i].out_count;
  }
  sky_status s = ctx->run.run(qs.data(), nq);
  for (u32 i = 0; i < nq; ++i) queries[i].status = qs[i].status;
  return s;
}

void sky_serve_config_init(sky_serve_config* cfg) {
  if (!cfg) return;
  memset(cfg, 0, sizeof(*cfg));
  cfg->struct_size = sizeof(sky_serve_config);
  cfg->workers = 2;
  cfg->max_batch = 64;
}

sky_status sky_rank_space(sky_ctx* ctx, const float* points, uint64_t n, uint32_t d, uint32_t* out_ranks,
                          uint32_t* out_distinct, uint16_t* out_codes) {
  if (!ctx) return SKY_EINVAL;
  return ctx->run.rank_space(points, n, d, out_ranks, out_distinct, reinterpret_cast<unsigned short*>(out_codes));
}

uint64_t sky_query_bytes(uint64_t n, uint32_t d, const sky_params* params) {
  return Runner::query_bytes(n, d, params);
}

namespace {
sky_status serve_start_locked(sky_ctx* ctx, const sky_serve_config* cfg) {
  sky_serve_config def;
  sky_serve_config_init(&def);
  if (cfg && cfg->struct_size != sizeof(sky_serve_config)) return SKY_EINVAL;
  if (!ctx->server) ctx->server.reset(new Server());
  if (ctx->server->running()) return SKY_EBUSY;
  std::string msg;
  sky_status s = ctx->server->start(ctx->run.device, cfg ? *cfg : def, ctx->run.timing, &msg);
  if (s != SKY_OK) {
    ctx->server->shutdown();
    ctx->serve_error = msg.empty() ? "serving start failed" : msg;
  }
  return s;
}
}  // namespace

sky_status sky_serve_start(sky_ctx* ctx, const sky_serve_config* cfg) {
  if (!ctx) return SKY_EINVAL;
  std::lock_guard<std::mutex> g(ctx->serve_mu);
  return serve_start_locked(ctx, cfg);
}

sky_status sky_submit(sky_ctx* ctx, const float* points, uint64_t n, uint32_t d, const sky_params* params,
                      uint64_t* ticket) {
  if (!ctx || !ticket) return SKY_EINVAL;
  Server* srv = nullptr;
  {
    std::lock_guard<std::mutex> g(ctx->serve_mu);
    if (!ctx->server || !ctx->server->running()) {
      sky_status s = serve_start_locked(ctx, nullptr);
      if (s != SKY_OK) return s;
    }
    srv = ctx->server.get();
  }
  std::string msg;
  sky_status s = srv->submit(points, n, d, params, ticket, &msg);
  if (s != SKY_OK) {
    std::lock_guard<std::mutex> g(ctx->serve_mu);
    ctx->serve_error = msg;
  }
  return s;
}

sky_status sky_poll(sky_ctx* ctx, uint64_t ticket) {
  if (!ctx) return SKY_EINVAL;
  Server* srv = nullptr;
  {
    std::lock_guard<std::mutex> g(ctx->serve_mu);
    srv = ctx->server.get();
  }
  return srv ? srv->poll(ticket) : SKY_ECANCELLED;
}

sky_status sky_wait(sky_ctx* ctx, uint64_t ticket, uint32_t* out_idx, uint64_t* out_count, int64_t timeout_us,
                    sky_ticket_info* info) {
  if (!ctx) return SKY_EINVAL;
  Server* srv = nullptr;
  {
    std::lock_guard<std::mutex> g(ctx->serve_mu);
    srv = ctx->server.get();
  }
  if (!srv) return SKY_ECANCELLED;
  std::string msg;
  sky_status s = srv->wait(ticket, out_idx, out_count, timeout_us, info, &msg);
  if (s != SKY_OK && s != SKY_EBUSY) {
    std::lock_guard<std::mutex> g(ctx->serve_mu);
    ctx->serve_error = msg;
  }
  return s;
}

sky_status sky_serve_stop(sky_ctx* ctx) {
  if (!ctx) return SKY_EINVAL;
  std::lock_guard<std::mutex> g(ctx->serve_mu);
  if (ctx->server) ctx->server->shutdown();
  return SKY_OK;
}

struct sky_graph {
  GraphRun* run = nullptr;
  cudaStream_t after = nullptr;
  u32 nq = 0;
  std::string error;
};

sky_status sky_graph_capture(sky_ctx* ctx, const sky_query* queries, uint32_t nq, sky_graph** graph) {
  if (!graph) return SKY_EINVAL;
  *graph = nullptr;
  if (!ctx || (nq && !queries)) return SKY_EINVAL;
  std::vector<Runner::Query> qs(nq);
  std::vector<u64> dummy(nq);
  for (u32 i = 0; i < nq; ++i) {
    qs[i].points = queries[i].points;
    qs[i].n = queries[i].n;
    qs[i].d = queries[i].d;
    qs[i].params = queries[i].params;
    qs[i].out_idx = queries[i].out_idx;
    qs[i].out_count = &dummy[i];
  }
  GraphRun* g = nullptr;
  std::string msg;
  sky_status s = graph_capture(ctx->run.device, ctx->run.budget, qs.data(), nq, &g, &msg);
  if (s != SKY_OK) {
    ctx->run.last_error = msg;
    return s;
  }
  sky_graph* h = new sky_graph();
  h->run = g;
  h->after = ctx->run.stream;
  h->nq = nq;
  *graph = h;
  return SKY_OK;
}

sky_status sky_graph_launch(sky_graph* graph, uint64_t* out_counts, double* ms) {
  if (!graph) return SKY_EINVAL;
  std::vector<sky_status> st(graph->nq);
  std::vector<u64> counts(graph->nq);
  sky_status s = graph_launch(graph->run, graph->after, counts.data(), st.data(), ms, nullptr, &graph->error);
  if (out_counts)
    for (u32 i = 0; i < graph->nq; ++i) out_counts[i] = counts[i];
  return s;
}

void sky_graph_destroy(sky_graph* graph) {
  if (!graph) return;
  graph_destroy(graph->run);
  delete graph;
}

sky_status sky_get_stats(sky_ctx* ctx, uint64_t ticket_or_0, sky_stats* out) {
  if (!ctx || !out) return SKY_EINVAL;
  if (ticket_or_0 == 0) {
    *out = ctx->run.stats;
    return SKY_OK;
  }
  Server* srv = nullptr;
  {
    std::lock_guard<std::mutex> g(ctx->serve_mu);
    srv = ctx->server.get();
  }
  if (!srv) return SKY_ECANCELLED;
  return srv->stats(ticket_or_0, out);
}

const char* sky_status_str(sky_status s) {
  switch (s) {
    case SKY_OK: return "SKY_OK";
    case SKY_EINVAL: return "SKY_EINVAL: invalid argument";
    case SKY_ENOMEM: return "SKY_ENOMEM: out of memory";
    case SKY_ECUDA: return "SKY_ECUDA: CUDA error";
    case SKY_ETIMEOUT: return "SKY_ETIMEOUT: device wait timed out";
    case SKY_EBUSY: return "SKY_EBUSY: still running";
    case SKY_ECANCELLED: return "SKY_ECANCELLED: unknown ticket";
  }
  return "unknown status";
}

sky_status sky_probe_compare_rate(sky_ctx* ctx, uint32_t iterations, double* compares_per_s,
                                  uint32_t* sm_count) {
  if (!ctx || !compares_per_s || !sm_count || iterations == 0) return SKY_EINVAL;
  if (cudaSetDevice(ctx->run.device) != cudaSuccess) return SKY_ECUDA;
  u32* sink = nullptr;
  if (cudaMalloc(&sink, 256) != cudaSuccess) {
    cudaGetLastError();
    return SKY_ENOMEM;
  }
  cudaError_t e = probe_compare_rate(iterations, ctx->run.stream, compares_per_s, sm_count, sink);
  cudaFree(sink);
  if (e != cudaSuccess) {
    ctx->run.last_error = std::string("compare probe: ") + cudaGetErrorString(e);
    return SKY_ECUDA;
  }
  return SKY_OK;
}

sky_status sky_probe_reject_rate(sky_ctx* ctx, uint32_t iterations, double* dim_compares_per_s,
                                 uint32_t* sm_count) {
  if (!ctx || !dim_compares_per_s || !sm_count || iterations == 0) return SKY_EINVAL;
  if (cudaSetDevice(ctx->run.device) != cudaSuccess) return SKY_ECUDA;
  u32* sink = nullptr;
  if (cudaMalloc(&sink, 256) != cudaSuccess) {
    cudaGetLastError();
    return SKY_ENOMEM;
  }
  cudaError_t e = probe_reject_rate(iterations, ctx->run.stream, dim_compares_per_s, sm_count, sink);
  cudaFree(sink);
  if (e != cudaSuccess) {
    ctx->run.last_error = std::string("reject probe: ") + cudaGetErrorString(e);
    return SKY_ECUDA;
  }
  return SKY_OK;
}

sky_status sky_diag_engine_wait_test(sky_ctx* ctx, uint64_t wait_limit_ns, uint32_t withhold_task) {
  if (!ctx || wait_limit_ns < 1000000ull) return SKY_EINVAL;
  ctx->run.test_wait_ns = wait_limit_ns;
  ctx->run.test_withhold_task = withhold_task;
  return SKY_OK;
}

const char* sky_last_error(sky_ctx* ctx) { return ctx ? ctx->run.last_error.c_str() : "no context"; }

void sky_destroy(sky_ctx* ctx) {
  if (!ctx) return;
  {
    std::lock_guard<std::mutex> g(ctx->serve_mu);
    ctx->server.reset();  // stops the workers after the queued queries
  }
  delete ctx;
}

}  // extern "C"
