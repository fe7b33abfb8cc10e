// C ABI of libskyline (include/skyline.h): contexts, scratch memory and the
// host-side orchestration of Algorithm 2 (Section 3) with the optimisations
// of Sections 3.2 (Grid Filtering), 4.1 (Sorted representatives) and 4.2
// (NoSeq).  Every step runs in the kernels of sky_prep.cu, sky_prims.cu,
// sky_dom.cu and sky_engine.cu; the host only sizes buffers, launches and
// copies results.
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

using namespace sky;

namespace sky {
u64& launch_counter() {
  static thread_local u64 count = 0;
  return count;
}
}  // namespace sky

struct sky_ctx {
  int device = 0;
  size_t budget = 0;
  cudaStream_t stream = nullptr;
  int timing = 0;
  char* ws = nullptr;
  size_t ws_size = 0;
  u32* pinned = nullptr;  // small host staging area (pinned)
  std::string last_error;
  sky_stats stats;
  cudaEvent_t ev[12] = {};
};

namespace {

constexpr size_t PINNED_WORDS = 64;

// Bump allocator over one scratch block; sizes are rounded to 256 bytes.
struct Carve {
  char* base;
  size_t off = 0;
  explicit Carve(char* b) : base(b) {}
  template <class T>
  T* take(size_t count) {
    size_t bytes = (count * sizeof(T) + 255) & ~(size_t)255;
    T* p = base ? reinterpret_cast<T*>(base + off) : nullptr;
    off += bytes ? bytes : 256;
    return p;
  }
};

struct Plan {
  u64 n = 0;
  int d = 0, V = 1;
  int scheme = SCHEME_NONE;
  u32 P = 1;
  u32 slices[8] = {1, 1, 1, 1, 1, 1, 1, 1};
  int normalize = 0, slice_dim = 0;
  u64 seed = 0;
  bool grid_filter = false;
  int rep = 0;
  u32 k = 1;
  int merge = 0;
  int exec = 0;
  EngineCfg cfg{};
  int pid_bits = 0;
  bool x_on_host = false;
};

struct Bufs {
  float* X;
  u64* keys[2];
  u32* vals[2];
  u32* head;
  float* pts;
  uint4* hc;
  float* score;
  u32* orig;
  u32* spid;
  u8* alive;
  u8* stage_s;
  u32* seg_off;
  u32* scan_tmp;
  u32* hist;
  float* win;
  uint4* whc;
  u32* dpos;
  uint4* dhc;
  float* upts;
  uint4* uhc;
  float* uscore;
  u32* upos;
  u32* useg;
  float* mpts;
  uint4* mhc;
  float* mscore;
  u32* mpos;
  u8* malive;
  u8* ualive;
  SegDesc* segs;
  SegState* st;
  u32* done_round;
  u32* tdoneA;
  u32* tdoneB;
  u64 tcap;
  u32* ctl;
  u32* words;  // err, colmax[8], counters
  u8* clos;
  u8* dropped;
  float* rep_pts;
  u8* rep_alive;
  float* kept_pts;
  u32* rep_excl;
  float* ang_table;
  u8* mask;
  u32* excl;
  u32* out_dev;
  u32* gcnt;
  u32* gpre;
};

// word slots of Bufs::words
enum { W_ERR = 0, W_COLMAX = 1, W_GRID_DROPPED = 9, W_KEPT = 10, W_NU = 11, W_SKY = 12, W_MAXROUND_LOCAL = 13,
       W_MAXROUND_MERGE = 14, W_HIST = 16, W_WORDS = 32 };

size_t layout(const Plan& pl, u32 ang_words, char* base, Bufs* b) {
  Carve c(base);
  const u64 n = pl.n ? pl.n : 1;
  const u64 P = pl.P;
  const u64 V = pl.V;
  const u64 nrep = (pl.rep ? P * pl.k : 1);
  b->X = c.take<float>(pl.x_on_host ? n * pl.d : 1);
  b->keys[0] = c.take<u64>(n);
  b->keys[1] = c.take<u64>(n);
  b->vals[0] = c.take<u32>(n);
  b->vals[1] = c.take<u32>(n);
  b->head = c.take<u32>(n);
  b->pts = c.take<float>(n * 4 * V);
  b->hc = c.take<uint4>(n);
  b->score = c.take<float>(n);
  b->orig = c.take<u32>(n);
  b->spid = c.take<u32>(n);
  b->alive = c.take<u8>(n);
  b->stage_s = c.take<u8>(n);
  b->seg_off = c.take<u32>(P + 1);
  size_t scan_words = scan_tmp_words(std::max<u64>({(u64)radix_hist_words(n), n, P + 1, nrep}));
  b->scan_tmp = c.take<u32>(scan_words);
  b->hist = c.take<u32>(radix_hist_words(n));
  b->win = c.take<float>(n * 4 * V);
  b->whc = c.take<uint4>(n);
  b->dpos = c.take<u32>(n);
  b->dhc = c.take<uint4>(n);
  b->upts = c.take<float>(n * 4 * V);
  b->uhc = c.take<uint4>(n);
  b->uscore = c.take<float>(n);
  b->upos = c.take<u32>(n);
  b->useg = c.take<u32>(P + 1);
  b->mpts = c.take<float>(n * 4 * V);
  b->mhc = c.take<uint4>(n);
  b->mscore = c.take<float>(n);
  b->mpos = c.take<u32>(n);
  b->malive = c.take<u8>(n);
  b->ualive = c.take<u8>(n);
  b->segs = c.take<SegDesc>(P);
  b->st = c.take<SegState>(2 * P);
  b->done_round = c.take<u32>(P);
  b->tcap = engine_tile_capacity(n, (u32)P);
  b->tdoneA = c.take<u32>(b->tcap);
  b->tdoneB = c.take<u32>(b->tcap);
  b->ctl = c.take<u32>(ENGINE_CTL_WORDS);
  b->words = c.take<u32>(W_WORDS);
  b->clos = c.take<u8>(P);
  b->dropped = c.take<u8>(P);
  b->rep_pts = c.take<float>(nrep * 4 * V);
  b->rep_alive = c.take<u8>(nrep);
  b->kept_pts = c.take<float>(nrep * 4 * V);
  b->rep_excl = c.take<u32>(nrep);
  b->ang_table = c.take<float>(ang_words ? ang_words : 1);
  b->mask = c.take<u8>(n);
  b->excl = c.take<u32>(n);
  b->out_dev = c.take<u32>(n);
  b->gcnt = c.take<u32>(P + 1);
  b->gpre = c.take<u32>(P + 1);
  return c.off;
}

bool is_device_ptr(const void* p) {
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

sky_status fail(sky_ctx* ctx, sky_status s, const std::string& msg) {
  if (ctx) ctx->last_error = msg;
  return s;
}

#define CK(expr)                                                                          \
  do {                                                                                    \
    cudaError_t e_ = (expr);                                                              \
    if (e_ != cudaSuccess)                                                                \
      return fail(ctx, SKY_ECUDA, std::string(#expr) + ": " + cudaGetErrorString(e_));  \
  } while (0)

int bits_for(u64 v) {  // bits needed to represent values in [0, v)
  int b = 0;
  while (b < 64 && (1ull << b) < v) ++b;
  return b;
}

sky_status validate(sky_ctx* ctx, const float* points, u64 n, u32 d, const sky_params* pa, Plan* pl) {
  if (!ctx) return SKY_EINVAL;
  if (d < 1 || d > 8) return fail(ctx, SKY_EINVAL, "d must be in 1..8");
  if (n >= (1ull << 32) - 1) return fail(ctx, SKY_EINVAL, "N must be below 2^32 - 1");
  if (n > 0 && !points) return fail(ctx, SKY_EINVAL, "points is NULL");
  sky_params def;
  sky_params_init(&def);
  const sky_params& p = pa ? *pa : def;
  if (pa && pa->struct_size != sizeof(sky_params)) return fail(ctx, SKY_EINVAL, "sky_params.struct_size mismatch");
  pl->n = n;
  pl->d = (int)d;
  pl->V = vec_of((int)d);
  pl->scheme = (int)p.scheme;
  pl->normalize = p.normalize ? 1 : 0;
  pl->seed = p.seed;
  pl->rep = p.rep == SKY_REP_SORTED ? 1 : 0;
  if (p.rep != SKY_REP_NONE && p.rep != SKY_REP_SORTED) return fail(ctx, SKY_EINVAL, "unknown rep mode");
  pl->k = p.reps_per_partition ? p.reps_per_partition : 1;
  if (p.merge != SKY_MERGE_SEQUENTIAL && p.merge != SKY_MERGE_NOSEQ) return fail(ctx, SKY_EINVAL, "unknown merge");
  pl->merge = (int)p.merge;
  if (p.exec != SKY_EXEC_PERSISTENT && p.exec != SKY_EXEC_PLAIN) return fail(ctx, SKY_EINVAL, "unknown exec");
  pl->exec = (int)p.exec;
  u64 P = 1;
  switch (p.scheme) {
    case SKY_GRID:
      for (u32 a = 0; a < d; ++a) {
        if (p.slices[a] < 1) return fail(ctx, SKY_EINVAL, "Grid slices must be >= 1");
        P *= p.slices[a];
        if (P > (1u << 20)) return fail(ctx, SKY_EINVAL, "Grid cell count above 2^20");
        pl->slices[a] = p.slices[a];
      }
      pl->grid_filter = p.grid_filter != 0;
      break;
    case SKY_ANGULAR:
      for (u32 a = 0; a + 1 < d; ++a) {
        if (p.slices[a] < 1) return fail(ctx, SKY_EINVAL, "Angular slices must be >= 1");
        P *= p.slices[a];
        if (P > (1u << 20)) return fail(ctx, SKY_EINVAL, "Angular partition count above 2^20");
        pl->slices[a] = p.slices[a];
      }
      break;
    case SKY_RANDOM:
    case SKY_SLICED:
      P = p.num_partitions ? p.num_partitions : 1;
      if (P > (1u << 20)) return fail(ctx, SKY_EINVAL, "partition count above 2^20");
      if (n > 0 && P > n) P = n;
      if (p.scheme == SKY_SLICED) {
        if (p.slice_dim >= d) return fail(ctx, SKY_EINVAL, "slice_dim must be < d");
        pl->slice_dim = (int)p.slice_dim;
      }
      break;
    case SKY_NONE:
      P = 1;
      break;
    default:
      return fail(ctx, SKY_EINVAL, "unknown partitioning scheme");
  }
  pl->P = (u32)P;
  if (pl->rep && (u64)pl->P * pl->k > (1u << 22)) return fail(ctx, SKY_EINVAL, "too many representatives");
  pl->pid_bits = bits_for(P);
  pl->cfg.chunk_min = p.chunk_min ? p.chunk_min : 4096;
  pl->cfg.chunk_max = p.chunk_max ? p.chunk_max : 65536;
  if (pl->cfg.chunk_max < pl->cfg.chunk_min) pl->cfg.chunk_max = pl->cfg.chunk_min;
  pl->cfg.alpha_x4 = p.chunk_alpha_x4 ? p.chunk_alpha_x4 : 8;
  pl->cfg.dom_block = p.dom_block ? p.dom_block : 1024;
  if (pl->cfg.dom_block % 32) return fail(ctx, SKY_EINVAL, "dom_block must be a multiple of 32");
  if (pl->cfg.chunk_min > (1u << 24) || pl->cfg.chunk_max > (1u << 24)) return fail(ctx, SKY_EINVAL, "chunk too large");
  return SKY_OK;
}

sky_status ensure_ws(sky_ctx* ctx, size_t bytes) {
  if (bytes <= ctx->ws_size) return SKY_OK;
  if (ctx->budget && bytes > ctx->budget)
    return fail(ctx, SKY_ENOMEM, "scratch memory of " + std::to_string(bytes) + " bytes exceeds the budget");
  if (ctx->ws) {
    cudaStreamSynchronize(ctx->stream);
    cudaFree(ctx->ws);
    ctx->ws = nullptr;
    ctx->ws_size = 0;
  }
  size_t grow = bytes + bytes / 8;
  if (ctx->budget && grow > ctx->budget) grow = bytes;
  cudaError_t e = cudaMalloc(&ctx->ws, grow);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return fail(ctx, SKY_ENOMEM, std::string("cudaMalloc: ") + cudaGetErrorString(e));
  }
  ctx->ws_size = grow;
  return SKY_OK;
}

// Angular thresholds tan^2(k pi / (2 m)), k = 1..m-1, evaluated in double
// and rounded to FP32 (Section 3.3 evaluated without device transcendentals).
void angular_table(const Plan& pl, std::vector<float>* tab, u32* off) {
  tab->clear();
  const double pi = 3.14159265358979323846;
  for (int a = 0; a + 1 < pl.d; ++a) {
    off[a] = (u32)tab->size();
    u32 m = pl.slices[a];
    for (u32 k = 1; k < m; ++k) {
      double t = tan((double)k * pi / (2.0 * (double)m));
      tab->push_back((float)(t * t));
    }
  }
  if (tab->empty()) tab->push_back(0.0f);
}

void record(sky_ctx* ctx, int i) {
  if (ctx->timing) cudaEventRecord(ctx->ev[i], ctx->stream);
}

sky_status run(sky_ctx* ctx, const float* points, u64 n, u32 d, const sky_params* pa, u32* out_idx,
               u64* out_count, u32* out_pid, u8* out_stage) {
  Plan pl;
  sky_status s = validate(ctx, points, n, d, pa, &pl);
  if (s != SKY_OK) return s;
  const u64 launches0 = launch_counter();
  if (!out_count) return fail(ctx, SKY_EINVAL, "out_count is NULL");
  CK(cudaSetDevice(ctx->device));
  memset(&ctx->stats, 0, sizeof(ctx->stats));
  ctx->stats.n = n;
  ctx->stats.d = d;
  ctx->stats.partitions = pl.P;
  if (n == 0) {
    *out_count = 0;
    return SKY_OK;
  }
  if (n > 0 && !out_idx) return fail(ctx, SKY_EINVAL, "out_idx is NULL");
  cudaStream_t st = ctx->stream;
  pl.x_on_host = !is_device_ptr(points);
  std::vector<float> tab;
  u32 ang_off[8] = {0};
  if (pl.scheme == SCHEME_ANGULAR) angular_table(pl, &tab, ang_off);
  Bufs b;
  size_t need = layout(pl, (u32)tab.size(), nullptr, &b);
  s = ensure_ws(ctx, need);
  if (s != SKY_OK) return s;
  layout(pl, (u32)tab.size(), ctx->ws, &b);
  const u32 P = pl.P;
  const int D = pl.d;

  record(ctx, 0);
  const float* X = points;
  if (pl.x_on_host) {
    CK(cudaMemcpyAsync(b.X, points, n * d * sizeof(float), cudaMemcpyHostToDevice, st));
    X = b.X;
  }
  record(ctx, 1);
  CK(cudaMemsetAsync(b.words, 0, W_WORDS * sizeof(u32), st));
  CK(cudaMemsetAsync(b.stage_s, 0, n, st));
  u32* err = b.words + W_ERR;

  // ---- Partition(r, p): keys, sort, gather (Algorithm 2 first phase)
  PrepArgs pr{};
  pr.X = X;
  pr.n = n;
  pr.scheme = pl.scheme;
  pr.normalize = pl.normalize && (pl.scheme == SCHEME_GRID || pl.scheme == SCHEME_ANGULAR);
  pr.slice_dim = pl.slice_dim;
  pr.seed = pl.seed;
  for (int a = 0; a < 8; ++a) pr.slices[a] = pl.slices[a];
  pr.colmax = b.words + W_COLMAX;
  if (pl.scheme == SCHEME_ANGULAR) {
    CK(cudaMemcpyAsync(b.ang_table, tab.data(), tab.size() * sizeof(float), cudaMemcpyHostToDevice, st));
    for (int a = 0; a < 8; ++a) pr.ang_off[a] = ang_off[a];
  }
  pr.ang_table = b.ang_table;
  pr.keys = b.keys[0];
  pr.vals = b.vals[0];
  pr.err = err;
  if (pr.normalize) CK(launch_colmax(X, n, D, b.words + W_COLMAX, err, st));
  CK(launch_prep(pr, D, st));
  int sel = 0;
  if (pl.scheme == SCHEME_RANDOM || pl.scheme == SCHEME_SLICED) {
    CK(radix_sort(b.keys, b.vals, n, 0, 64, b.hist, b.scan_tmp, st, &sel));
    const u32* run_start = nullptr;
    if (pl.scheme == SCHEME_SLICED) {
      CK(launch_run_heads(b.keys[sel], n, b.head, st));
      CK(scan_u32(b.head, b.head, n, false, true, b.scan_tmp, st));
      run_start = b.head;
    }
    // rekey into the other buffer pair, then sort by (partition, score)
    CK(launch_rekey(X, n, D, b.vals[sel], run_start, P, b.keys[sel ^ 1], b.vals[sel ^ 1], st));
    u64* k2[2] = {b.keys[sel ^ 1], b.keys[sel]};
    u32* v2[2] = {b.vals[sel ^ 1], b.vals[sel]};
    int sel2 = 0;
    CK(radix_sort(k2, v2, n, 0, 32 + pl.pid_bits, b.hist, b.scan_tmp, st, &sel2));
    sel = sel2 == 0 ? (sel ^ 1) : sel;
  } else {
    int hi = (pl.scheme == SCHEME_NONE) ? 32 : 32 + pl.pid_bits;
    CK(radix_sort(b.keys, b.vals, n, 0, hi, b.hist, b.scan_tmp, st, &sel));
  }
  GatherArgs ga{};
  ga.X = X;
  ga.n = n;
  ga.keys = b.keys[sel];
  ga.vals = b.vals[sel];
  ga.P = P;
  ga.pts = b.pts;
  ga.hc = b.hc;
  ga.score = b.score;
  ga.orig = b.orig;
  ga.spid = b.spid;
  ga.alive = b.alive;
  ga.seg_off = b.seg_off;
  CK(launch_gather(ga, D, st));
  record(ctx, 2);

  // ---- Grid Filtering (3.2)
  const u8* dropped = nullptr;
  if (pl.scheme == SCHEME_GRID && pl.grid_filter) {
    GridDims gd;
    for (int a = 0; a < 8; ++a) gd.m[a] = pl.slices[a];
    CK(launch_grid_filter(b.seg_off, b.spid, n, D, gd, P, b.clos, b.dropped, b.alive, b.stage_s,
                          b.words + W_GRID_DROPPED, st));
    dropped = b.dropped;
  }
  // ---- Sorted representatives (4.1)
  if (pl.rep) {
    u32 nrep = P * pl.k;
    CK(launch_rep_select(b.seg_off, P, pl.k, dropped, b.pts, D, b.rep_pts, b.rep_alive, st));
    // R = Sky(reps): dominated representatives are discarded first
    CK(launch_relative(b.rep_pts, b.rep_alive, nrep, b.rep_pts, nrep, nullptr, D, st));
    CK(scan_u8(b.rep_alive, b.rep_excl, nrep, true, b.scan_tmp, st));
    CK(cudaMemcpyAsync(b.words + W_KEPT, b.scan_tmp + scan_total_index(nrep), sizeof(u32),
                       cudaMemcpyDeviceToDevice, st));
    CK(launch_compact_reps(b.rep_alive, b.rep_excl, nrep, D, b.rep_pts, b.kept_pts, st));
    CK(launch_relative(b.pts, b.alive, n, b.kept_pts, 0, b.words + W_KEPT, D, st));
    CK(launch_stamp_stage(b.alive, n, b.stage_s, ST_REP, st));
  }
  record(ctx, 3);

  // ---- ComputeLocalSet: u_i = Sky(r_i) for every partition
  SegArrays sa{b.pts, b.hc, b.score, b.alive, b.win, b.whc, b.dpos, b.dhc};
  CK(launch_build_segs(b.seg_off, P, dropped, sa, D, b.segs, st));
  CK(cudaMemsetAsync(b.tdoneA, 0, b.tcap * sizeof(u32), st));
  CK(cudaMemsetAsync(b.tdoneB, 0, b.tcap * sizeof(u32), st));
  EngineWork ew;
  ew.st = b.st;
  ew.done_round = b.done_round;
  ew.tdoneA = b.tdoneA;
  ew.tdoneB = b.tdoneB;
  ew.tcap = b.tcap;
  ew.ctl = b.ctl;
  const u32* maxround = b.ctl + engine_max_round_word();
  record(ctx, 8);
  if (pl.exec == SKY_EXEC_PERSISTENT) {
    CK(engine_run(b.segs, P, pl.cfg, ew, err, st));
    record(ctx, 9);
    CK(launch_fold_max(maxround, b.words + W_MAXROUND_LOCAL, st));
  } else {
    for (u32 q = 0; q < P; ++q) {
      CK(engine_run(b.segs + q, 1, pl.cfg, ew, err, st));
      CK(launch_fold_max(maxround, b.words + W_MAXROUND_LOCAL, st));
    }
    record(ctx, 9);
  }
  CK(launch_stamp_stage(b.alive, n, b.stage_s, ST_LOCAL, st));
  record(ctx, 4);

  // ---- final phase over u (sequential Sky(u), or NoSeq, Section 4.2)
  if (P > 1) {
    CK(scan_u8(b.alive, b.excl, n, true, b.scan_tmp, st));
    CK(cudaMemcpyAsync(b.words + W_NU, b.scan_tmp + scan_total_index(n), sizeof(u32), cudaMemcpyDeviceToDevice,
                       st));
    const bool seq = pl.merge == SKY_MERGE_SEQUENTIAL;
    CK(launch_compact_u(b.alive, b.excl, n, D, b.pts, b.hc, b.score, b.spid, b.upts, b.uhc, b.uscore, b.upos,
                        nullptr,
                        seq ? b.keys[0] : nullptr, seq ? b.vals[0] : nullptr, st));
    if (seq) {
      CK(cudaMemcpyAsync(ctx->pinned, b.words + W_NU, sizeof(u32), cudaMemcpyDeviceToHost, st));
      CK(cudaStreamSynchronize(st));
      const u64 nu = ctx->pinned[0];
      int msel = 0;
      CK(radix_sort(b.keys, b.vals, nu, 0, 32, b.hist, b.scan_tmp, st, &msel));
      CK(launch_gather_u(b.vals[msel], nu, D, b.upts, b.uhc, b.uscore, b.upos, b.mpts, b.mhc, b.mscore, b.mpos,
                         st));
      CK(cudaMemsetAsync(b.malive, 1, nu ? nu : 1, st));
      SegArrays ma{b.mpts, b.mhc, b.mscore, b.malive, b.win, b.whc, b.dpos, b.dhc};
      CK(launch_build_one_seg(ma, b.words + W_NU, D, b.segs, st));
      CK(cudaMemsetAsync(b.tdoneA, 0, b.tcap * sizeof(u32), st));
      CK(cudaMemsetAsync(b.tdoneB, 0, b.tcap * sizeof(u32), st));
      record(ctx, 10);
      CK(engine_run(b.segs, 1, pl.cfg, ew, err, st));
      record(ctx, 11);
      CK(launch_fold_max(maxround, b.words + W_MAXROUND_MERGE, st));
      CK(launch_scatter_alive(b.malive, b.mpos, nu, b.alive, b.stage_s, ST_MERGE, st));
    } else {
      CK(launch_useg(b.seg_off, P, b.excl, n, b.words + W_NU, b.useg, st));
      CK(cudaMemsetAsync(b.ualive, 1, n, st));
      NoSeqArgs na{};
      na.upts = reinterpret_cast<const float4*>(b.upts);
      na.uscore = b.uscore;
      na.useg = b.useg;
      na.ualive = b.ualive;
      na.P = P;
      na.scheme = pl.scheme;
      na.d = D;
      for (int a = 0; a < 8; ++a) na.gd.m[a] = pl.slices[a];
      na.dom_block = pl.cfg.dom_block;
      // keep the item count within 32 bits
      while (((n / 64 + P + 1) * (n / na.dom_block + 1)) >= (1ull << 31)) na.dom_block *= 2;
      record(ctx, 10);
      CK(launch_noseq(na, b.gcnt, b.gpre, b.scan_tmp, b.words + W_NU, b.ctl, st));
      record(ctx, 11);
      // u is a prefix of the sorted positions' survivors: upos maps back
      CK(cudaMemcpyAsync(ctx->pinned, b.words + W_NU, sizeof(u32), cudaMemcpyDeviceToHost, st));
      CK(cudaStreamSynchronize(st));
      const u64 nu = ctx->pinned[0];
      CK(launch_scatter_alive(b.ualive, b.upos, nu, b.alive, b.stage_s, ST_MERGE, st));
    }
  }
  record(ctx, 5);

  // ---- output: ascending indices of Sky(r)
  CK(launch_output(b.stage_s, b.orig, b.spid, n, b.mask, out_stage && is_device_ptr(out_stage) ? out_stage : nullptr,
                   out_pid && is_device_ptr(out_pid) ? out_pid : nullptr, st));
  CK(scan_u8(b.mask, b.excl, n, true, b.scan_tmp, st));
  CK(cudaMemcpyAsync(b.words + W_SKY, b.scan_tmp + scan_total_index(n), sizeof(u32), cudaMemcpyDeviceToDevice, st));
  const bool out_dev = is_device_ptr(out_idx);
  CK(launch_compact_idx(b.mask, b.excl, n, out_dev ? out_idx : b.out_dev, st));
  CK(launch_stage_hist(b.stage_s, n, b.words + W_HIST, st));
  record(ctx, 6);
  CK(cudaMemcpyAsync(ctx->pinned, b.words, W_WORDS * sizeof(u32), cudaMemcpyDeviceToHost, st));
  CK(cudaStreamSynchronize(st));
  u32 w[W_WORDS];
  memcpy(w, ctx->pinned, sizeof(w));
  if (w[W_ERR] & ERR_NAN) return fail(ctx, SKY_EINVAL, "input contains NaN");
  if (w[W_ERR] & ERR_TIMEOUT) return fail(ctx, SKY_ETIMEOUT, "a device-side wait timed out");
  if (w[W_ERR] & ERR_CAPACITY) return fail(ctx, SKY_ENOMEM, "device-side capacity exceeded");
  const u64 cnt = w[W_SKY];
  if (!out_dev && cnt) CK(cudaMemcpyAsync(out_idx, b.out_dev, cnt * sizeof(u32), cudaMemcpyDeviceToHost, st));
  // host-side diagnostics
  if (out_stage && !is_device_ptr(out_stage)) {
    CK(launch_output(b.stage_s, b.orig, b.spid, n, b.mask, reinterpret_cast<u8*>(b.keys[0]), b.vals[0], st));
    CK(cudaMemcpyAsync(out_stage, b.keys[0], n, cudaMemcpyDeviceToHost, st));
    if (out_pid && !is_device_ptr(out_pid)) CK(cudaMemcpyAsync(out_pid, b.vals[0], n * 4, cudaMemcpyDeviceToHost, st));
  } else if (out_pid && !is_device_ptr(out_pid)) {
    CK(launch_output(b.stage_s, b.orig, b.spid, n, b.mask, nullptr, b.vals[0], st));
    CK(cudaMemcpyAsync(out_pid, b.vals[0], n * 4, cudaMemcpyDeviceToHost, st));
  }
  record(ctx, 7);
  CK(cudaStreamSynchronize(st));
  *out_count = cnt;
  sky_stats& S = ctx->stats;
  S.rounds_local = w[W_MAXROUND_LOCAL];
  S.rounds_merge = w[W_MAXROUND_MERGE];
  S.reps_kept = pl.rep ? w[W_KEPT] : 0;
  S.grid_dropped = w[W_HIST + ST_GRID];
  S.rep_dropped = w[W_HIST + ST_REP];
  S.local_union = (u64)w[W_HIST + ST_MERGE] + w[W_HIST + ST_SKY];
  S.skyline = cnt;
  S.nonempty_partitions = 0;
  S.launches = launch_counter() - launches0;
  if (ctx->timing) {
    float ms = 0;
    cudaEventElapsedTime(&ms, ctx->ev[0], ctx->ev[7]);
    S.ms_total = ms;
    for (int i = 0; i < 6; ++i) {
      float t = 0;
      cudaEventElapsedTime(&t, ctx->ev[i + 1], ctx->ev[i + 2]);
      S.ms_phase[i] = t;
    }
    float tl = 0, tm = 0;
    cudaEventElapsedTime(&tl, ctx->ev[8], ctx->ev[9]);
    S.ms_dom_local = tl;
    if (P > 1) {
      cudaEventElapsedTime(&tm, ctx->ev[10], ctx->ev[11]);
      S.ms_dom_merge = tm;
    }
  }
  return SKY_OK;
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
  c->device = device;
  c->budget = mem_budget_bytes;
  if (cudaMallocHost(&c->pinned, PINNED_WORDS * sizeof(u32)) != cudaSuccess) {
    delete c;
    return SKY_ENOMEM;
  }
  for (int i = 0; i < 12; ++i) cudaEventCreate(&c->ev[i]);
  device_sm_count();
  memset(&c->stats, 0, sizeof(c->stats));
  *ctx = c;
  return SKY_OK;
}

sky_status sky_set_stream(sky_ctx* ctx, void* cuda_stream) {
  if (!ctx) return SKY_EINVAL;
  ctx->stream = reinterpret_cast<cudaStream_t>(cuda_stream);
  return SKY_OK;
}

sky_status sky_set_timing(sky_ctx* ctx, int on) {
  if (!ctx) return SKY_EINVAL;
  ctx->timing = on ? 1 : 0;
  return SKY_OK;
}

sky_status sky_skyline(sky_ctx* ctx, const float* points, uint64_t n, uint32_t d, const sky_params* params,
                       uint32_t* out_idx, uint64_t* out_count) {
  return run(ctx, points, n, d, params, out_idx, out_count, nullptr, nullptr);
}

sky_status sky_skyline_ex(sky_ctx* ctx, const float* points, uint64_t n, uint32_t d, const sky_params* params,
                          uint32_t* out_idx, uint64_t* out_count, uint32_t* out_pid, uint8_t* out_stage) {
  return run(ctx, points, n, d, params, out_idx, out_count, out_pid, out_stage);
}

sky_status sky_get_stats(sky_ctx* ctx, sky_stats* out) {
  if (!ctx || !out) return SKY_EINVAL;
  *out = ctx->stats;
  return SKY_OK;
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
  CK(cudaSetDevice(ctx->device));
  sky_status s = ensure_ws(ctx, 256);
  if (s != SKY_OK) return s;
  CK(probe_compare_rate(iterations, ctx->stream, compares_per_s, sm_count, reinterpret_cast<u32*>(ctx->ws)));
  return SKY_OK;
}

const char* sky_last_error(sky_ctx* ctx) { return ctx ? ctx->last_error.c_str() : "no context"; }

void sky_destroy(sky_ctx* ctx) {
  if (!ctx) return;
  cudaSetDevice(ctx->device);
  cudaStreamSynchronize(ctx->stream);
  if (ctx->ws) cudaFree(ctx->ws);
  if (ctx->pinned) cudaFreeHost(ctx->pinned);
  for (int i = 0; i < 12; ++i)
    if (ctx->ev[i]) cudaEventDestroy(ctx->ev[i]);
  delete ctx;
}

}  // extern "C"
