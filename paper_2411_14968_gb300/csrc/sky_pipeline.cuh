// Host-side orchestration of Algorithm 2 over a batch of independent
// skyline queries (internal; the C ABI is in sky_api.cu).
#pragma once
#include <mutex>
#include <string>
#include <vector>
#include "../../include/skyline.h"
#include "sky_internal.cuh"

namespace sky {

// Orders the persistent engine launches of several Runners that share a
// device: each launch waits (on the GPU) for the one enqueued before it, so
// two cooperative grids never compete for the SMs, while the other stages
// of the Runners' batches still overlap.
struct EngineGate {
  std::mutex mu;
  cudaEvent_t last = nullptr;  // completion event of the latest gated launch
};

// Checks one query's arguments (Section 3 parameters included); msg
// receives the reason of a failure.
sky_status validate_query(const float* points, u64 n, u32 d, const sky_params* params, std::string* msg);

struct BatchState;

// Execution state that the pipeline needs: a device, a stream, a grow-only
// device workspace, pinned host staging and timing events.  One Runner runs
// one batch at a time.
class Runner {
 public:
  int device = 0;
  size_t budget = 0;            // workspace limit in bytes (0 = none)
  cudaStream_t stream = nullptr;
  int timing = 0;
  std::string last_error;
  sky_stats stats{};
  EngineGate* gate = nullptr;   // set when several Runners share the device
  // Test hooks of the engine's bounded waits for the next run() only
  // (EngineCfg::wait_ns, EngineCfg::withhold_task); zero = off.
  u64 test_wait_ns = 0;
  u32 test_withhold_task = 0;

  ~Runner();
  sky_status init(int dev, size_t mem_budget);
  // Frees the device workspace (kept otherwise between batches).
  void release();
  size_t workspace_bytes() const { return ws_size_; }

  // One query of a batch.  Inputs are caller-owned; out_idx has capacity
  // >= n; out_pid / out_stage may be NULL.  Host or device pointers.
  struct Query {
    const float* points = nullptr;
    u64 n = 0;
    u32 d = 0;
    const sky_params* params = nullptr;
    u32* out_idx = nullptr;
    u64* out_count = nullptr;
    u32* out_pid = nullptr;
    u8* out_stage = nullptr;
    sky_status status = SKY_OK;   // out
    sky_stats stats{};            // out: per-query statistics (no timing)
  };

  // Validates every query, then runs all of them: prep and sort per query,
  // every local skyline of the batch in one persistent engine launch, every
  // sequential final phase in a second one, outputs per query.  Blocks until
  // the results are in the output buffers.  Returns the first failing
  // status (queries[i].status says which).
  sky_status run(Query* queries, u32 nq);

  // run() in three stages, so that the device work of a batch can be
  // captured into a CUDA graph: prepare (validate, size, lay out the
  // workspace; graph = device inputs and outputs only), enqueue (every
  // launch and copy of the batch on `stream`, no host round trip), finish
  // (wait, read the counts, copy host outputs, statistics).
  sky_status prepare(BatchState& B, Query* queries, u32 nq, bool graph);
  sky_status enqueue(BatchState& B);
  sky_status finish(BatchState& B);

  // sky_rank_space: dense ranks, distinct counts and rank codes of every
  // column (each output optional; host or device).  Blocks.
  sky_status rank_space(const float* points, u64 n, u32 d, u32* out_ranks, u32* out_distinct,
                        unsigned short* out_codes);

  // Workspace bytes a query of this shape needs (for admission control).
  static size_t query_bytes(u64 n, u32 d, const sky_params* params);

 private:
  char* ws_ = nullptr;
  size_t ws_size_ = 0;
  u32* pinned_ = nullptr;
  size_t pinned_words_ = 0;
  cudaEvent_t ev_[12] = {};
  cudaEvent_t gate_ev_ = nullptr;
  static constexpr int NAUX = 4;   // streams the per-query work of a batch is spread over
  cudaStream_t aux_[NAUX] = {};
  cudaEvent_t fork_ev_ = nullptr;
  std::vector<cudaEvent_t> copy_ev_;  // one per host input of a batch (grown on demand)
  cudaEvent_t join_ev_[NAUX] = {};
  sky_status ensure_ws(size_t bytes);
  sky_status ensure_pinned(size_t words);
  sky_status fail(sky_status s, const std::string& msg);
  void record(int i, const BatchState& B);
};

// Where a caller's pointer lives: host memory (pageable, pinned or unknown
// to CUDA), device memory of the current device (or managed memory), or
// device memory of another device, which the library's kernels must not be
// given.
enum { PTR_HOST = 0, PTR_DEVICE = 1, PTR_OTHER_DEVICE = 2 };
int pointer_kind(const void* p);
bool is_device_ptr(const void* p);  // pointer_kind(p) == PTR_DEVICE

// A batch captured into a CUDA graph with its own Runner (workspace, pinned
// staging, stream), replayed as one graph launch.  Inputs and outputs must
// be device memory; shapes, parameters and pointers are fixed at capture.
struct GraphRun;
sky_status graph_capture(int device, size_t budget, const Runner::Query* queries, u32 nq, GraphRun** out,
                         std::string* msg);
// Replays after the work queued on `after`, waits, and reports each query's
// |Sky| and status, the device time of the replay and the statistics.
sky_status graph_launch(GraphRun* g, cudaStream_t after, u64* counts, sky_status* statuses, double* ms,
                        sky_stats* stats, std::string* msg);
void graph_destroy(GraphRun* g);

}  // namespace sky
