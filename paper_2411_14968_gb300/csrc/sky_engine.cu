// Dispatch of a persistent engine launch to the compiled launch shape that
// its EngineCfg asks for (warps per CTA x candidates per lane; see
// sky_engine_impl.cuh), and the engine's capacity rules, which hold for
// every shape.
#include "sky_internal.cuh"

namespace sky {

u64 engine_tile_capacity(u64 total_points, u32 nseg) {
  // a phase of a segment of n points has at most ceil(n / tile) tiles, with
  // the smallest tile of any shape
  return total_points / ENGINE_MIN_TILE + 2ull * nseg + 1;
}

u64 engine_task_capacity(u64 total_points, u32 nseg, u32 chunk_min) {
  // every round but a segment's last processes at least chunk_min points,
  // and a round publishes at most two tasks
  return 2 * (total_points / (chunk_min ? chunk_min : 1) + 2ull * nseg) + 16;
}

bool engine_shape_ok(u32 warps, u32 cands) {
  return (warps == 0 || warps == 4 || warps == 8) && (cands == 0 || cands == 2 || cands == 4);
}

cudaError_t engine_run(const SegDesc* segs_dev, u32 nseg, const EngineCfg& cfg, const EngineWork& w, u32* err,
                       cudaStream_t st) {
  const u32 wp = cfg.warps ? cfg.warps : DEFAULT_ENGINE_WARPS;
  const u32 r = cfg.cands ? cfg.cands : DEFAULT_ENGINE_CANDS;
  if (wp == 4 && r == 4) return engine_run_variant<4, 4>(segs_dev, nseg, cfg, w, err, st);
  if (wp == 8 && r == 4) return engine_run_variant<8, 4>(segs_dev, nseg, cfg, w, err, st);
  if (wp == 4 && r == 2) return engine_run_variant<4, 2>(segs_dev, nseg, cfg, w, err, st);
  if (wp == 8 && r == 2) return engine_run_variant<8, 2>(segs_dev, nseg, cfg, w, err, st);
  return cudaErrorInvalidValue;
}

}  // namespace sky
