// sky_autotune: picks the dominance engine's tuning knobs for a workload by
// measurement.  The knobs change only how Algorithm 1 is cut into parallel
// work (chunk sizes of the SFS rounds, the dominator block a CTA stages in
// shared memory, the launch shape: warps per CTA and candidates per lane,
// i.e. a work item's tile width), never the result, so any choice is exact;
// the tuner times whole queries (CUDA events around the call on the
// context's stream) and keeps the fastest.
//
// A batch is tuned as a whole (one set of knobs for all of its queries): the
// best knobs for a batch differ from those of its queries alone, because
// the queries share the engine's launches.
//
// Search: from the built-in defaults, a joint search over the chunk growth
// factor and the first chunk length (the two knobs that interact most),
// then every launch shape, then coordinate descent (the launch shape
// counting as one knob): for each knob in turn every candidate value is
// tried with the others held at their best values so far; two sweeps,
// within a trial budget.  Each candidate runs three times and counts its
// median run; the winner is then confirmed against the starting knobs by the
// median of five interleaved runs each.
#include <algorithm>
#include <cfloat>
#include <cstring>
#include <vector>
#include "../../include/skyline.h"
#include "sky_internal.cuh"

namespace sky {
int ctx_timing(sky_ctx* ctx);
}

namespace {

struct Knob {
  uint32_t sky_params::*field;
  std::vector<uint32_t> values;
};

}  // namespace

namespace {

// Tunes the knobs of every query of a batch together.  queries[i].params
// are the method parameters; the trial outputs go to one scratch buffer.
sky_status tune(sky_ctx* ctx, const sky_query* queries, uint32_t nq, uint32_t max_trials, sky_params* knobs,
                double* best_ms) {
  uint64_t total = 0;
  for (uint32_t i = 0; i < nq; ++i) total += queries[i].n;
  if (total == 0) {
    *best_ms = 0;
    return SKY_OK;
  }
  if (max_trials == 0) max_trials = 48;
  uint32_t* out = nullptr;
  if (cudaMalloc(&out, total * sizeof(uint32_t)) != cudaSuccess) {
    cudaGetLastError();
    return SKY_ENOMEM;
  }
  std::vector<sky_params> ps(nq);
  std::vector<sky_query> qs(queries, queries + nq);
  std::vector<uint64_t> counts(nq);
  {
    uint64_t off = 0;
    for (uint32_t i = 0; i < nq; ++i) {
      if (queries[i].params) {
        ps[i] = *queries[i].params;
      } else {
        sky_params_init(&ps[i]);
      }
      qs[i].params = &ps[i];
      qs[i].out_idx = out + off;
      qs[i].out_count = &counts[i];
      off += queries[i].n;
    }
  }
  const int timing_was = sky::ctx_timing(ctx);
  sky_set_timing(ctx, 1);
  sky_params cur = *knobs;
  sky_params start;
  if (!cur.dom_block) cur.dom_block = sky::DEFAULT_DOM_BLOCK;
  if (!cur.chunk_min) cur.chunk_min = sky::DEFAULT_CHUNK_MIN;
  if (!cur.chunk_max) cur.chunk_max = sky::DEFAULT_CHUNK_MAX;
  if (!cur.chunk_alpha_x4) cur.chunk_alpha_x4 = sky::DEFAULT_ALPHA_X4;
  if (!cur.engine_warps) cur.engine_warps = sky::DEFAULT_ENGINE_WARPS;
  if (!cur.engine_cands) cur.engine_cands = sky::DEFAULT_ENGINE_CANDS;
  // the compiled launch shapes (warps per CTA, candidates per lane)
  const uint32_t shapes[][2] = {{4, 4}, {8, 4}, {4, 2}, {8, 2}};
  const Knob knob_set[] = {
      {&sky_params::chunk_alpha_x4, {4, 8, 16, 32, 64}},
      {&sky_params::dom_block, {256, 512, 1024, 2048}},
      {&sky_params::chunk_min, {256, 1024, 4096, 16384}},
      {&sky_params::chunk_max, {16384, 65536, 262144, 1048576}},
  };
  uint32_t trials = 0;
  sky_status status = SKY_OK;
  auto run_once = [&](const sky_params& k, double* ms) -> sky_status {
    for (uint32_t i = 0; i < nq; ++i) {
      ps[i].chunk_min = k.chunk_min;
      ps[i].chunk_max = k.chunk_max;
      ps[i].chunk_alpha_x4 = k.chunk_alpha_x4;
      ps[i].dom_block = k.dom_block;
      ps[i].engine_warps = k.engine_warps;
      ps[i].engine_cands = k.engine_cands;
    }
    sky_status s = sky_skyline_batch(ctx, qs.data(), nq);
    if (s != SKY_OK) return s;
    sky_stats st;
    sky_get_stats(ctx, 0, &st);
    *ms = st.ms_total;
    return SKY_OK;
  };
  auto measure = [&](const sky_params& k, double* ms) -> sky_status {
    double t[3];
    for (int rep = 0; rep < 3; ++rep) {
      sky_status s = run_once(k, &t[rep]);
      if (s != SKY_OK) return s;
    }
    std::sort(t, t + 3);
    *ms = t[1];
    ++trials;
    return SKY_OK;
  };
  start = cur;
  double cur_ms = 0;
  status = measure(cur, &cur_ms);
  // first a joint search over the two knobs that interact most (the chunk
  // growth factor and the first chunk), then coordinate descent on all
  for (uint32_t al : {8u, 16u, 32u})
    for (uint32_t cm : {256u, 1024u, 4096u}) {
      if (trials >= max_trials || status != SKY_OK) break;
      if (cur.chunk_alpha_x4 == al && cur.chunk_min == cm) continue;
      sky_params cand = cur;
      cand.chunk_alpha_x4 = al;
      cand.chunk_min = cm;
      if (cand.chunk_max < cand.chunk_min) continue;
      double ms = 0;
      status = measure(cand, &ms);
      if (status == SKY_OK && ms < cur_ms) {
        cur = cand;
        cur_ms = ms;
      }
    }
  // every launch shape at the knobs found so far
  auto shape_pass = [&]() -> bool {
    bool changed = false;
    for (const auto& sh : shapes) {
      if (trials >= max_trials || status != SKY_OK) break;
      if (cur.engine_warps == sh[0] && cur.engine_cands == sh[1]) continue;
      sky_params cand = cur;
      cand.engine_warps = sh[0];
      cand.engine_cands = sh[1];
      double ms = 0;
      status = measure(cand, &ms);
      if (status == SKY_OK && ms < cur_ms) {
        cur = cand;
        cur_ms = ms;
        changed = true;
      }
    }
    return changed;
  };
  shape_pass();
  for (int sweep = 0; sweep < 2 && status == SKY_OK; ++sweep) {
    bool changed = sweep > 0 && shape_pass();
    for (const Knob& k : knob_set) {
      for (uint32_t v : k.values) {
        if (trials >= max_trials || status != SKY_OK) break;
        if (cur.*(k.field) == v) continue;
        sky_params cand = cur;
        cand.*(k.field) = v;
        if (cand.chunk_max < cand.chunk_min) continue;
        double ms = 0;
        status = measure(cand, &ms);
        if (status == SKY_OK && ms < cur_ms) {
          cur = cand;
          cur_ms = ms;
          changed = true;
        }
      }
    }
    if (!changed) break;
  }
  // A batch's time varies from run to run (the work queue's order changes
  // which dominators meet which candidates first), so even a median of
  // three can favour a worse candidate.  Confirm the winner against the
  // starting knobs with the median of CONFIRM interleaved runs each.
  const bool moved = cur.chunk_min != start.chunk_min || cur.chunk_max != start.chunk_max ||
                     cur.chunk_alpha_x4 != start.chunk_alpha_x4 || cur.dom_block != start.dom_block ||
                     cur.engine_warps != start.engine_warps || cur.engine_cands != start.engine_cands;
  if (status == SKY_OK && moved) {
    constexpr int CONFIRM = 5;
    double a[CONFIRM], b[CONFIRM];
    for (int i = 0; i < CONFIRM && status == SKY_OK; ++i) {
      status = run_once(start, &a[i]);
      if (status == SKY_OK) status = run_once(cur, &b[i]);
    }
    if (status == SKY_OK) {
      std::sort(a, a + CONFIRM);
      std::sort(b, b + CONFIRM);
      if (a[CONFIRM / 2] <= b[CONFIRM / 2]) {
        cur = start;
        cur_ms = a[CONFIRM / 2];
      } else {
        cur_ms = b[CONFIRM / 2];
      }
    }
  }
  cudaFree(out);
  sky_set_timing(ctx, timing_was);
  if (status != SKY_OK) return status;
  knobs->chunk_min = cur.chunk_min;
  knobs->chunk_max = cur.chunk_max;
  knobs->chunk_alpha_x4 = cur.chunk_alpha_x4;
  knobs->dom_block = cur.dom_block;
  knobs->engine_warps = cur.engine_warps;
  knobs->engine_cands = cur.engine_cands;
  *best_ms = cur_ms;
  return SKY_OK;
}

}  // namespace

extern "C" sky_status sky_autotune(sky_ctx* ctx, const float* points, uint64_t n, uint32_t d, sky_params* params,
                                   uint32_t max_trials, double* best_ms) {
  if (!ctx || !params || !best_ms || params->struct_size != sizeof(sky_params)) return SKY_EINVAL;
  sky_query q;
  memset(&q, 0, sizeof(q));
  q.points = points;
  q.n = n;
  q.d = d;
  q.params = params;
  return tune(ctx, &q, 1, max_trials, params, best_ms);
}

extern "C" sky_status sky_autotune_batch(sky_ctx* ctx, const sky_query* queries, uint32_t nq, uint32_t max_trials,
                                         sky_params* knobs, double* best_ms) {
  if (!ctx || !knobs || !best_ms || (nq && !queries) || knobs->struct_size != sizeof(sky_params)) return SKY_EINVAL;
  for (uint32_t i = 0; i < nq; ++i)
    if (queries[i].params && queries[i].params->struct_size != sizeof(sky_params)) return SKY_EINVAL;
  return tune(ctx, queries, nq, max_trials, knobs, best_ms);
}
