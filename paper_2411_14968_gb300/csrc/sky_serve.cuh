// Serving loop with continuous batching (internal; the C ABI is in
// sky_api.cu).
#pragma once
#include <memory>
#include <string>
#include "sky_pipeline.cuh"

namespace sky {

class Server {
 public:
  Server();
  ~Server();
  // timing != 0: the workers time their batches with CUDA events (the
  // device times of a ticket's statistics).
  sky_status start(int device, const sky_serve_config& cfg, int timing, std::string* msg);
  // Stops the workers after the queued queries have run; completed tickets
  // stay collectable and start() may be called again.
  void shutdown();
  bool running() const;
  sky_status submit(const float* points, u64 n, u32 d, const sky_params* params, u64* ticket, std::string* msg);
  sky_status poll(u64 ticket);
  sky_status wait(u64 ticket, u32* out_idx, u64* out_count, int64_t timeout_us, sky_ticket_info* info,
                  std::string* msg);
  // Statistics of a completed ticket, collected or not (the most recent
  // 4096 collected ones are kept): SKY_EBUSY while it runs, SKY_ECANCELLED
  // for an unknown ticket.
  sky_status stats(u64 ticket, sky_stats* out);
  u64 batches() const;

 private:
  struct Ticket;
  struct Impl;
  std::unique_ptr<Impl> impl_;
};

}  // namespace sky
