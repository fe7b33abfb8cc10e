// Host-side orchestration of Algorithm 2 (Section 3) with the optimisations
// of Sections 3.2 (Grid Filtering), 4.1 (Sorted representatives) and 4.2
// (NoSeq), over a batch of independent queries.  Every step runs in the
// kernels of sky_prep.cu, sky_prims.cu, sky_dom.cu and sky_engine.cu; the
// host sizes buffers, launches, and copies the results once at the end.
//
// Batching: the partitions of every query of a batch are segments of one
// persistent engine launch (the local phase), and the merge inputs of every
// query with a sequential final phase are segments of a second one, so the
// uneven work of many queries fills the GPU together.  There is no host
// round trip between the first launch and the final copy of the counts:
// sizes that are only known on the device (|u|) are read by the kernels.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <memory>
#include <nvtx3/nvToolsExt.h>
#include "sky_pipeline.cuh"

namespace sky {

namespace pipe {

// Bump allocator over one scratch block; sizes are rounded to 256 bytes.
struct Carve {
  char* base;
  size_t off;
  explicit Carve(char* b, size_t start = 0) : base(b), off(start) {}
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
  int images = SKY_IMAGES_VALUES;
  EngineCfg cfg{};
  int pid_bits = 0;
  bool x_on_host = false;
};

// Per-query device buffers.
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

// Engine state shared by the queries of a batch.
struct BatchBufs {
  SegDesc* segs;    // local-phase segments of every query
  SegDesc* msegs;   // merge segments (one per query with a sequential final phase)
  SegState* st;
  u32* tbase;
  u32* tdoneA;
  u32* tdoneB;
  u32* tstat;
  u64 tcap;
  void* tasks;
  u64 task_cap;
  u32* ctl;
};

// Local-phase launches with at most this many segments keep ordered dense
// lists by look-back (large chunks); launches with more have the last tile
// of each phase compact its chunk in order (many small chunks).
constexpr u32 ORDERED_MAX_SEGS = 8;

// word slots of Bufs::words
enum { W_ERR = 0, W_COLMAX = 1, W_GRID_DROPPED = 9, W_KEPT = 10, W_NU = 11, W_SKY = 12, W_MAXROUND_LOCAL = 13,
       W_MAXROUND_MERGE = 14, W_NONEMPTY = 15, W_HIST = 16, W_NOSEQ_CTR = 24,
       W_TESTS_LOCAL = 26, W_TESTS_MERGE = 28 /* u64 each: the engine's FP16 tests */, W_WORDS = 32 };

size_t layout(const Plan& pl, u32 ang_words, Carve& c, Bufs* b) {
  const size_t start = c.off;
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
  size_t scan_words = scan_tmp_words(std::max<u64>({n, (u64)P + 1, (u64)nrep}));
  b->scan_tmp = c.take<u32>(scan_words);
  b->hist = c.take<u32>(radix_work_words(n));
  b->win = c.take<float>(n * 4 * V);
  b->whc = c.take<uint4>(n + P + 2);  // pairs: every partition starts at an even entry
  b->dpos = c.take<u32>(n);
  b->dhc = c.take<uint4>(n + P + 2);
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
  return c.off - start;
}

void layout_batch(u64 total_pts, u32 total_segs, u32 nmerge, u32 chunk_min, Carve& c, BatchBufs* bb) {
  const u32 nseg = std::max(std::max(total_segs, nmerge), 1u);
  bb->segs = c.take<SegDesc>(std::max(total_segs, 1u));
  bb->msegs = c.take<SegDesc>(std::max(nmerge, 1u));
  bb->st = c.take<SegState>(nseg);
  bb->tbase = c.take<u32>(nseg);
  bb->tcap = engine_tile_capacity(std::max<u64>(total_pts, 1), nseg);
  bb->tdoneA = c.take<u32>(bb->tcap);
  bb->tdoneB = c.take<u32>(bb->tcap);
  bb->tstat = c.take<u32>(bb->tcap);
  bb->task_cap = engine_task_capacity(std::max<u64>(total_pts, 1), nseg, chunk_min);
  bb->tasks = c.take<char>(bb->task_cap * engine_task_bytes());
  bb->ctl = c.take<u32>(ENGINE_CTL_WORDS);
}

int bits_for(u64 v) {  // bits needed to represent values in [0, v)
  int b = 0;
  while (b < 64 && (1ull << b) < v) ++b;
  return b;
}

// Checks the arguments of one query and derives its plan; msg receives the
// reason of a failure.
sky_status validate(const float* points, u64 n, u32 d, const sky_params* pa, Plan* pl, std::string* msg) {
  auto bad = [&](const char* m) {
    *msg = m;
    return SKY_EINVAL;
  };
  if (d < 1 || d > 8) return bad("d must be in 1..8");
  if (n >= (1ull << 32) - 1) return bad("N must be below 2^32 - 1");
  if (n > 0 && !points) return bad("points is NULL");
  sky_params def;
  sky_params_init(&def);
  const sky_params& p = pa ? *pa : def;
  if (pa && pa->struct_size != sizeof(sky_params)) return bad("sky_params.struct_size mismatch");
  pl->n = n;
  pl->d = (int)d;
  pl->V = vec_of((int)d);
  pl->scheme = (int)p.scheme;
  pl->normalize = p.normalize ? 1 : 0;
  pl->seed = p.seed;
  pl->rep = (int)p.rep;
  if (p.rep != SKY_REP_NONE && p.rep != SKY_REP_SORTED && p.rep != SKY_REP_REGION) return bad("unknown rep mode");
  pl->k = p.reps_per_partition ? p.reps_per_partition : 1;
  if (p.merge != SKY_MERGE_SEQUENTIAL && p.merge != SKY_MERGE_NOSEQ) return bad("unknown merge");
  pl->merge = (int)p.merge;
  if (p.exec != SKY_EXEC_PERSISTENT && p.exec != SKY_EXEC_PLAIN) return bad("unknown exec");
  pl->exec = (int)p.exec;
  if (p.images != SKY_IMAGES_VALUES && p.images != SKY_IMAGES_RANKS) return bad("unknown images mode");
  pl->images = (int)p.images;
  u64 P = 1;
  switch (p.scheme) {
    case SKY_GRID:
      for (u32 a = 0; a < d; ++a) {
        if (p.slices[a] < 1) return bad("Grid slices must be >= 1");
        P *= p.slices[a];
        if (P > (1u << 20)) return bad("Grid cell count above 2^20");
        pl->slices[a] = p.slices[a];
      }
      pl->grid_filter = p.grid_filter != 0;
      break;
    case SKY_ANGULAR:
      for (u32 a = 0; a + 1 < d; ++a) {
        if (p.slices[a] < 1) return bad("Angular slices must be >= 1");
        P *= p.slices[a];
        if (P > (1u << 20)) return bad("Angular partition count above 2^20");
        pl->slices[a] = p.slices[a];
      }
      break;
    case SKY_RANDOM:
    case SKY_SLICED:
      P = p.num_partitions ? p.num_partitions : 1;
      if (P > (1u << 20)) return bad("partition count above 2^20");
      if (n > 0 && P > n) P = n;
      if (p.scheme == SKY_SLICED) {
        if (p.slice_dim >= d) return bad("slice_dim must be < d");
        pl->slice_dim = (int)p.slice_dim;
      }
      break;
    case SKY_NONE:
      P = 1;
      break;
    default:
      return bad("unknown partitioning scheme");
  }
  pl->P = (u32)P;
  if (pl->rep && (u64)pl->P * pl->k > (1u << 22)) return bad("too many representatives");
  if (pl->rep == SKY_REP_REGION && pl->k > 64) return bad("at most 64 Region representatives per partition");
  pl->pid_bits = bits_for(P);
  pl->cfg.chunk_min = p.chunk_min ? p.chunk_min : DEFAULT_CHUNK_MIN;
  pl->cfg.chunk_max = p.chunk_max ? p.chunk_max : DEFAULT_CHUNK_MAX;
  if (pl->cfg.chunk_max < pl->cfg.chunk_min) pl->cfg.chunk_max = pl->cfg.chunk_min;
  pl->cfg.alpha_x4 = p.chunk_alpha_x4 ? p.chunk_alpha_x4 : DEFAULT_ALPHA_X4;
  pl->cfg.dom_block = p.dom_block ? p.dom_block : DEFAULT_DOM_BLOCK;
  if (pl->cfg.dom_block % 32) return bad("dom_block must be a multiple of 32");
  if (pl->cfg.dom_block > engine_max_dom_block()) return bad("dom_block above the engine's maximum");
  if (pl->cfg.chunk_min > (1u << 24) || pl->cfg.chunk_max > (1u << 24)) return bad("chunk too large");
  if (!engine_shape_ok(p.engine_warps, p.engine_cands))
    return bad("engine_warps must be 0, 4 or 8 and engine_cands 0, 2 or 4");
  pl->cfg.warps = p.engine_warps ? p.engine_warps : DEFAULT_ENGINE_WARPS;
  pl->cfg.cands = p.engine_cands ? p.engine_cands : DEFAULT_ENGINE_CANDS;
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

// Everything the pipeline keeps about one query between its stages.
struct Work {
  Runner::Query* q;
  Plan pl;
  std::vector<float> tab;
  u32 ang_off[8] = {0};
  Bufs b;
  const float* X = nullptr;   // device copy of the input
  const u8* dropped = nullptr;
  u32 seg_base = 0;          // first local segment in the batch array
  int mseg = -1;             // merge segment, or -1
  bool out_dev = false;
  u32 words[W_WORDS] = {0};
  size_t tab_off = 0;        // angular table in the pinned staging (words)
  bool pid_dev = false;      // out_pid / out_stage are device memory
  bool stage_dev = false;
  int copy_ev = -1;          // event of the input's copy to the device (host input)
};

#define CK(expr)                                                                       \
  do {                                                                                 \
    cudaError_t e_ = (expr);                                                           \
    if (e_ != cudaSuccess) return fail(SKY_ECUDA, std::string(#expr) + ": " + cudaGetErrorString(e_)); \
  } while (0)

}  // namespace pipe

using namespace pipe;

// Everything one batch keeps between its stages (prepare, enqueue, finish).
struct BatchState {
  Runner::Query* queries = nullptr;
  u32 nq = 0;
  std::vector<Work> ws;
  BatchBufs bb{};
  bool empty = false;
  bool graph = false;         // captured into a CUDA graph: no host round trips
  Work* first_persistent = nullptr;
  u64 launches0 = 0;
  u64 kernels = 0;            // kernel launches the device work issues
};

sky_status validate_query(const float* points, u64 n, u32 d, const sky_params* params, std::string* msg) {
  Plan pl;
  return validate(points, n, d, params, &pl, msg);
}

int pointer_kind(const void* p) {
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return PTR_HOST;
  }
  if (a.type == cudaMemoryTypeManaged) return PTR_DEVICE;
  if (a.type != cudaMemoryTypeDevice) return PTR_HOST;
  int cur = -1;
  if (cudaGetDevice(&cur) != cudaSuccess) return PTR_OTHER_DEVICE;
  return a.device == cur ? PTR_DEVICE : PTR_OTHER_DEVICE;
}

bool is_device_ptr(const void* p) { return pointer_kind(p) == PTR_DEVICE; }

Runner::~Runner() {
  if (ws_ || pinned_ || ev_[0]) {
    cudaSetDevice(device);
    cudaStreamSynchronize(stream);
  }
  if (ws_) cudaFree(ws_);
  if (pinned_) cudaFreeHost(pinned_);
  for (auto& e : ev_)
    if (e) cudaEventDestroy(e);
  if (gate_ev_) cudaEventDestroy(gate_ev_);
  if (fork_ev_) cudaEventDestroy(fork_ev_);
  for (auto e : copy_ev_) cudaEventDestroy(e);
  for (int k = 0; k < NAUX; ++k) {
    if (aux_[k]) {
      cudaStreamSynchronize(aux_[k]);
      cudaStreamDestroy(aux_[k]);
    }
    if (join_ev_[k]) cudaEventDestroy(join_ev_[k]);
  }
}

sky_status Runner::init(int dev, size_t mem_budget) {
  device = dev;
  budget = mem_budget;
  if (cudaSetDevice(dev) != cudaSuccess) return SKY_ECUDA;
  for (auto& e : ev_)
    if (cudaEventCreate(&e) != cudaSuccess) return SKY_ECUDA;
  if (cudaEventCreateWithFlags(&gate_ev_, cudaEventDisableTiming) != cudaSuccess) return SKY_ECUDA;
  if (cudaEventCreateWithFlags(&fork_ev_, cudaEventDisableTiming) != cudaSuccess) return SKY_ECUDA;
  for (int k = 0; k < NAUX; ++k) {
    if (cudaStreamCreateWithFlags(&aux_[k], cudaStreamNonBlocking) != cudaSuccess) return SKY_ECUDA;
    if (cudaEventCreateWithFlags(&join_ev_[k], cudaEventDisableTiming) != cudaSuccess) return SKY_ECUDA;
  }
  return ensure_pinned(64);
}

void Runner::release() {
  if (ws_) {
    cudaSetDevice(device);
    cudaStreamSynchronize(stream);
    cudaFree(ws_);
  }
  ws_ = nullptr;
  ws_size_ = 0;
}

sky_status Runner::fail(sky_status s, const std::string& msg) {
  last_error = msg;
  return s;
}

sky_status Runner::ensure_ws(size_t bytes) {
  if (bytes <= ws_size_) return SKY_OK;
  if (budget && bytes > budget)
    return fail(SKY_ENOMEM, "scratch memory of " + std::to_string(bytes) + " bytes exceeds the budget");
  release();
  size_t grow = bytes + bytes / 8;
  if (budget && grow > budget) grow = bytes;
  cudaError_t e = cudaMalloc(&ws_, grow);
  if (e != cudaSuccess) {
    cudaGetLastError();
    ws_ = nullptr;
    return fail(SKY_ENOMEM, std::string("cudaMalloc: ") + cudaGetErrorString(e));
  }
  ws_size_ = grow;
  return SKY_OK;
}

sky_status Runner::ensure_pinned(size_t words) {
  if (words <= pinned_words_) return SKY_OK;
  if (pinned_) {
    cudaStreamSynchronize(stream);
    cudaFreeHost(pinned_);
    pinned_ = nullptr;
    pinned_words_ = 0;
  }
  if (cudaMallocHost(&pinned_, words * sizeof(u32)) != cudaSuccess) {
    cudaGetLastError();
    return fail(SKY_ENOMEM, "cudaMallocHost failed");
  }
  pinned_words_ = words;
  return SKY_OK;
}

size_t Runner::query_bytes(u64 n, u32 d, const sky_params* params) {
  Plan pl;
  std::string msg;
  if (validate(reinterpret_cast<const float*>(1), n, d, params, &pl, &msg) != SKY_OK) return 0;
  pl.x_on_host = true;
  std::vector<float> tab;
  u32 off[8];
  if (pl.scheme == SCHEME_ANGULAR) angular_table(pl, &tab, off);
  Bufs b;
  Carve c(nullptr);
  size_t q = layout(pl, (u32)std::max<size_t>(tab.size(), 1), c, &b);
  Carve c2(nullptr);
  BatchBufs bb;
  layout_batch(n, pl.P, 1, pl.cfg.chunk_min, c2, &bb);
  return q + c2.off;
}

sky_status Runner::run(Query* queries, u32 nq) {
  BatchState B;
  sky_status s = prepare(B, queries, nq, false);
  if (s == SKY_OK && !B.empty) s = enqueue(B);
  // the wait-test hooks apply to one call
  test_wait_ns = 0;
  test_withhold_task = 0;
  if (s != SKY_OK || B.empty) return s;
  return finish(B);
}

sky_status Runner::prepare(BatchState& B, Query* queries, u32 nq, bool graph) {
  B.queries = queries;
  B.nq = nq;
  B.graph = graph;
  B.launches0 = launch_counter();
  memset(&stats, 0, sizeof(stats));
  CK(cudaSetDevice(device));
  std::vector<Work>& ws = B.ws;
  ws.assign(nq, Work());
  // ---- validate and size
  u64 total_pts = 0;
  u32 total_segs = 0, nmerge = 0, min_chunk = 0xffffffffu;
  std::vector<size_t> offs(nq);
  size_t need = 0;
  for (u32 i = 0; i < nq; ++i) {
    Work& w = ws[i];
    Query& q = queries[i];
    w.q = &q;
    q.status = SKY_OK;
    memset(&q.stats, 0, sizeof(q.stats));
    std::string msg;
    sky_status s = validate(q.points, q.n, q.d, q.params, &w.pl, &msg);
    if (s == SKY_OK && !q.out_count) {
      s = SKY_EINVAL;
      msg = "out_count is NULL";
    }
    if (s == SKY_OK && q.n > 0 && !q.out_idx) {
      s = SKY_EINVAL;
      msg = "out_idx is NULL";
    }
    if (s != SKY_OK) {
      q.status = s;
      return fail(s, nq > 1 ? "query " + std::to_string(i) + ": " + msg : msg);
    }
    q.stats.n = q.n;
    q.stats.d = q.d;
    q.stats.partitions = w.pl.P;
    if (q.n == 0) continue;
    if (pointer_kind(q.points) == PTR_OTHER_DEVICE || pointer_kind(q.out_idx) == PTR_OTHER_DEVICE ||
        (q.out_pid && pointer_kind(q.out_pid) == PTR_OTHER_DEVICE) ||
        (q.out_stage && pointer_kind(q.out_stage) == PTR_OTHER_DEVICE)) {
      q.status = SKY_EINVAL;
      return fail(SKY_EINVAL, (nq > 1 ? "query " + std::to_string(i) + ": " : std::string()) +
                                  "a buffer is device memory of another GPU than the context's");
    }
    w.pl.x_on_host = !is_device_ptr(q.points);
    w.out_dev = is_device_ptr(q.out_idx);
    w.pid_dev = q.out_pid && is_device_ptr(q.out_pid);
    w.stage_dev = q.out_stage && is_device_ptr(q.out_stage);
    if (graph && (w.pl.x_on_host || !w.out_dev || (q.out_pid && !is_device_ptr(q.out_pid)) ||
                  (q.out_stage && !is_device_ptr(q.out_stage)))) {
      q.status = SKY_EINVAL;
      return fail(SKY_EINVAL, "a captured batch needs device inputs and outputs");
    }
    if (w.pl.scheme == SCHEME_ANGULAR) angular_table(w.pl, &w.tab, w.ang_off);
    Carve c(nullptr, need);
    offs[i] = need;
    need += layout(w.pl, (u32)std::max<size_t>(w.tab.size(), 1), c, &w.b);
    total_pts += q.n;
    total_segs += w.pl.P;
    min_chunk = std::min(min_chunk, w.pl.cfg.chunk_min);
    if (w.pl.P > 1 && w.pl.merge == SKY_MERGE_SEQUENTIAL) ++nmerge;
  }
  for (u32 i = 0; i < nq; ++i)
    if (queries[i].n == 0) *queries[i].out_count = 0;
  if (total_pts == 0) {
    B.empty = true;
    return SKY_OK;
  }
  BatchBufs& bb = B.bb;
  {
    Carve c(nullptr, need);
    layout_batch(total_pts, total_segs, nmerge, min_chunk, c, &bb);
    need = c.off;
  }
  sky_status s = ensure_ws(need);
  if (s != SKY_OK) return s;
  // pinned staging: the result words of every query, then the Angular
  // threshold tables (copied to the device from here)
  size_t pinned_words = (size_t)nq * W_WORDS;
  for (auto& w : ws) {
    w.tab_off = pinned_words;
    pinned_words += w.tab.size();
  }
  s = ensure_pinned(pinned_words);
  if (s != SKY_OK) return s;
  for (auto& w : ws)
    if (!w.tab.empty()) memcpy(pinned_ + w.tab_off, w.tab.data(), w.tab.size() * sizeof(float));
  {
    size_t batch_off = 0;
    for (u32 i = 0; i < nq; ++i) {
      Work& w = ws[i];
      if (w.q->n == 0) continue;
      Carve c(ws_, offs[i]);
      layout(w.pl, (u32)std::max<size_t>(w.tab.size(), 1), c, &w.b);
      batch_off = std::max(batch_off, c.off);
    }
    Carve c(ws_, batch_off);
    layout_batch(total_pts, total_segs, nmerge, min_chunk, c, &bb);
  }
  // Segment order: persistent queries first (one launch covers them), then
  // queries that ask for one launch per partition.
  {
    u32 sb = 0, mb = 0;
    for (int pass = 0; pass < 2; ++pass)
      for (auto& w : ws) {
        if (w.q->n == 0 || (w.pl.exec == SKY_EXEC_PLAIN) != (pass == 1)) continue;
        w.seg_base = sb;
        sb += w.pl.P;
        if (w.pl.P > 1 && w.pl.merge == SKY_MERGE_SEQUENTIAL) w.mseg = (int)mb++;
      }
  }

  return SKY_OK;
}

// Phase boundaries of a batch: CUDA events (when timing is on) and NVTX
// ranges on the host thread (one per phase, for a profiler's timeline; the
// calls do nothing unless a tool is attached).  Boundaries 1..6 open the
// phases below, 7 (in finish) closes the last; 0 and 8..11 are events only.
void Runner::record(int i, const BatchState& B) {
  if (timing && !B.graph) cudaEventRecord(ev_[i], stream);
  static const char* const kPhase[7] = {nullptr, "sky: partition", "sky: filters", "sky: local skylines",
                                        "sky: final phase", "sky: output", "sky: host copies"};
  if (B.graph || i < 1 || i > 7) return;
  if (i >= 2) nvtxRangePop();
  if (i <= 6) nvtxRangePushA(kPhase[i]);
}

sky_status Runner::enqueue(BatchState& B) {
  std::vector<Work>& ws = B.ws;
  BatchBufs& bb = B.bb;
  const u32 nq = B.nq;
  const cudaStream_t st = stream;
  const u64 k0 = launch_counter();
  // Per-query work runs on up to NAUX streams forked from `st` (the small
  // kernels of different queries overlap); the engine launches, which cover
  // every query, run on `st` between the joins.
  const bool multi = nq > 1;
  auto fork = [&]() -> cudaError_t {
    if (!multi) return cudaSuccess;
    cudaError_t r = cudaEventRecord(fork_ev_, st);
    for (int k = 0; k < NAUX && r == cudaSuccess; ++k) r = cudaStreamWaitEvent(aux_[k], fork_ev_, 0);
    return r;
  };
  auto join = [&]() -> cudaError_t {
    if (!multi) return cudaSuccess;
    cudaError_t r = cudaSuccess;
    for (int k = 0; k < NAUX && r == cudaSuccess; ++k) {
      r = cudaEventRecord(join_ev_[k], aux_[k]);
      if (r == cudaSuccess) r = cudaStreamWaitEvent(st, join_ev_[k], 0);
    }
    return r;
  };
  auto qstream = [&](const Work& w) -> cudaStream_t { return multi ? aux_[(&w - ws.data()) % NAUX] : stream; };
  record(0, B);
  record(1, B);

  // ---- Partition(r, p): keys, sort, gather (Algorithm 2 first phase)
  CK(fork());
  // Host inputs are copied to the device one after another on the main
  // stream, in query order, each at the whole copy bandwidth, and a query's
  // partitioning waits for its own copy only: later copies overlap earlier
  // queries' partitioning (copies issued on every query's stream at once
  // would share the bandwidth and all end together).
  {
    size_t k = 0;
    for (auto& w : ws) {
      if (w.q->n == 0 || !w.pl.x_on_host) continue;
      if (k == copy_ev_.size()) {
        cudaEvent_t e;
        CK(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
        copy_ev_.push_back(e);
      }
      CK(cudaMemcpyAsync(w.b.X, w.q->points, w.q->n * w.q->d * sizeof(float), cudaMemcpyHostToDevice, stream));
      CK(cudaEventRecord(copy_ev_[k], stream));
      w.copy_ev = (int)k++;
    }
  }
  for (auto& w : ws) {
    if (w.q->n == 0) continue;
    const cudaStream_t st = qstream(w);
    w.X = w.q->points;
    if (w.pl.x_on_host) {
      CK(cudaStreamWaitEvent(st, copy_ev_[w.copy_ev], 0));
      w.X = w.b.X;
    }
    const Plan& pl = w.pl;
    Bufs& b = w.b;
    const u64 n = pl.n;
    const int D = pl.d;
    u32* err = b.words + W_ERR;
    CK(cudaMemsetAsync(b.words, 0, W_WORDS * sizeof(u32), st));
    CK(cudaMemsetAsync(b.stage_s, 0, n, st));
    PrepArgs pr{};
    pr.X = w.X;
    pr.n = n;
    pr.scheme = pl.scheme;
    pr.normalize = pl.normalize && (pl.scheme == SCHEME_GRID || pl.scheme == SCHEME_ANGULAR);
    pr.slice_dim = pl.slice_dim;
    pr.seed = pl.seed;
    for (int a = 0; a < 8; ++a) pr.slices[a] = pl.slices[a];
    pr.colmax = b.words + W_COLMAX;
    if (pl.scheme == SCHEME_ANGULAR) {
      CK(cudaMemcpyAsync(b.ang_table, pinned_ + w.tab_off, w.tab.size() * sizeof(float), cudaMemcpyHostToDevice,
                         st));
      for (int a = 0; a < 8; ++a) pr.ang_off[a] = w.ang_off[a];
    }
    pr.ang_table = b.ang_table;
    pr.keys = b.keys[0];
    pr.vals = b.vals[0];
    pr.err = err;
    // column maxima: keys of normalised Grid / Angular, volumes of normalised
    // Region representatives
    if (pr.normalize || (pl.normalize && pl.rep == SKY_REP_REGION))
      CK(launch_colmax(w.X, n, D, b.words + W_COLMAX, err, st));
    // rank images (by original index) in the union's image buffer, which is
    // free until the local phase ends; the column ranks in the window's
    // point array (d x n words fit its 16 x vec_of(d) bytes per point), the
    // distinct counts in the merge's position array, both idle until the
    // local phase; keys, values, mask and head are rewritten by the prep and
    // the sorts below
    if (pl.images == SKY_IMAGES_RANKS) {
      RankScratch rs{{b.keys[0], b.keys[1]}, {b.vals[0], b.vals[1]}, b.hist, b.mask, b.head, b.scan_tmp,
                     reinterpret_cast<u32*>(b.win)};
      CK(launch_rank_space(w.X, n, (u32)D, rs, nullptr, nullptr, b.uhc, b.mpos, err, st));
    }
    CK(launch_prep(pr, D, st));
    int sel = 0;
    if (pl.scheme == SCHEME_RANDOM || pl.scheme == SCHEME_SLICED) {
      CK(radix_sort(b.keys, b.vals, n, 0, 64, b.hist, st, &sel, nullptr, err));
      const u32* run_start = nullptr;
      if (pl.scheme == SCHEME_SLICED) {
        CK(launch_run_heads(b.keys[sel], n, b.head, st));
        CK(scan_u32(b.head, b.head, n, false, true, b.scan_tmp, st));
        run_start = b.head;
      }
      // rekey into the other buffer pair, then sort by (partition, score)
      CK(launch_rekey(w.X, n, D, b.vals[sel], run_start, pl.P, b.keys[sel ^ 1], b.vals[sel ^ 1], st));
      u64* k2[2] = {b.keys[sel ^ 1], b.keys[sel]};
      u32* v2[2] = {b.vals[sel ^ 1], b.vals[sel]};
      int sel2 = 0;
      CK(radix_sort(k2, v2, n, 0, 32 + pl.pid_bits, b.hist, st, &sel2, nullptr, err));
      sel = sel2 == 0 ? (sel ^ 1) : sel;
    } else {
      int hi = (pl.scheme == SCHEME_NONE) ? 32 : 32 + pl.pid_bits;
      CK(radix_sort(b.keys, b.vals, n, 0, hi, b.hist, st, &sel, nullptr, err));
    }
    GatherArgs ga{};
    ga.X = w.X;
    ga.n = n;
    ga.keys = b.keys[sel];
    ga.vals = b.vals[sel];
    ga.P = pl.P;
    ga.pts = b.pts;
    ga.rcode = pl.images == SKY_IMAGES_RANKS ? b.uhc : nullptr;
    ga.hc = b.hc;
    ga.score = b.score;
    ga.orig = b.orig;
    ga.spid = b.spid;
    ga.alive = b.alive;
    ga.seg_off = b.seg_off;
    CK(launch_gather(ga, D, st));
  }
  CK(join());
  record(2, B);

  // ---- Grid Filtering (3.2), Sorted representatives (4.1), segments
  CK(fork());
  for (auto& w : ws) {
    if (w.q->n == 0) continue;
    const cudaStream_t st = qstream(w);
    const Plan& pl = w.pl;
    Bufs& b = w.b;
    const u64 n = pl.n;
    const int D = pl.d;
    const u32 P = pl.P;
    if (pl.scheme == SCHEME_GRID && pl.grid_filter) {
      GridDims gd;
      for (int a = 0; a < 8; ++a) gd.m[a] = pl.slices[a];
      CK(launch_grid_filter(b.seg_off, b.spid, n, D, gd, P, b.clos, b.dropped, b.alive, b.stage_s,
                            b.words + W_GRID_DROPPED, st));
      w.dropped = b.dropped;
    }
    if (pl.rep) {
      u32 nrep = P * pl.k;
      if (pl.rep == SKY_REP_REGION)
        CK(launch_rep_region(b.seg_off, P, pl.k, w.dropped, b.pts, b.orig, b.words + W_COLMAX, pl.normalize, D,
                             b.rep_pts, b.rep_alive, st));
      else
        CK(launch_rep_select(b.seg_off, P, pl.k, w.dropped, b.pts, D, b.rep_pts, b.rep_alive, st));
      // R = Sky(reps): dominated representatives are discarded first
      CK(launch_relative(b.rep_pts, b.rep_alive, nrep, b.rep_pts, nrep, nullptr, D, st));
      CK(scan_u8(b.rep_alive, b.rep_excl, nrep, true, b.scan_tmp, st));
      CK(cudaMemcpyAsync(b.words + W_KEPT, b.scan_tmp + scan_total_index(nrep), sizeof(u32),
                         cudaMemcpyDeviceToDevice, st));
      CK(launch_compact_reps(b.rep_alive, b.rep_excl, nrep, D, b.rep_pts, b.kept_pts, st));
      CK(launch_relative(b.pts, b.alive, n, b.kept_pts, 0, b.words + W_KEPT, D, st));
      CK(launch_stamp_stage(b.alive, n, b.stage_s, ST_REP, st));
    }
    SegArrays sa{b.pts, b.hc, b.score, b.alive, b.win, b.whc, b.dpos, b.dhc};
    CK(launch_build_segs(b.seg_off, P, w.dropped, sa, D, bb.segs + w.seg_base, b.words + W_NONEMPTY, st));
  }
  CK(join());
  record(3, B);

  // ---- ComputeLocalSet: u_i = Sky(r_i) for every partition of every query
  EngineWork ew;
  ew.st = bb.st;
  ew.tbase = bb.tbase;
  ew.tdoneA = bb.tdoneA;
  ew.tdoneB = bb.tdoneB;
  ew.tstat = bb.tstat;
  ew.tcap = bb.tcap;
  ew.tasks = bb.tasks;
  ew.task_cap = bb.task_cap;
  ew.ctl = bb.ctl;
  // the error word, round count and test counts of a launch go to one
  // query's words (err = words + W_ERR)
  auto engine = [&](const SegDesc* segs, u32 nseg, EngineCfg cfg, u32* err, u32* round_dst, u32 tests_word,
                    u32 ordered) -> cudaError_t {
    unsigned long long* tests_dst = reinterpret_cast<unsigned long long*>(err - W_ERR + tests_word);
    cfg.ordered = ordered;
    cfg.wait_ns = test_wait_ns;
    cfg.withhold_task = test_withhold_task;
    cudaError_t e = cudaMemsetAsync(bb.tdoneA, 0, bb.tcap * sizeof(u32), st);
    if (e == cudaSuccess) e = cudaMemsetAsync(bb.tdoneB, 0, bb.tcap * sizeof(u32), st);
    if (e != cudaSuccess) return e;
    if (gate) {
      std::lock_guard<std::mutex> g(gate->mu);
      if (gate->last) e = cudaStreamWaitEvent(st, gate->last, 0);
      if (e == cudaSuccess) e = engine_run(segs, nseg, cfg, ew, err, st);
      if (e == cudaSuccess) e = cudaEventRecord(gate_ev_, st);
      if (e == cudaSuccess) gate->last = gate_ev_;
    } else {
      e = engine_run(segs, nseg, cfg, ew, err, st);
    }
    if (e == cudaSuccess) e = launch_fold_engine(bb.ctl, round_dst, tests_dst, st);
    return e;
  };
  // the error word and round counter of a shared launch go to the first
  // query of the launch; the host folds them into every query of it
  Work*& first_persistent = B.first_persistent;
  first_persistent = nullptr;
  u32 persistent_segs = 0;
  for (auto& w : ws) {
    if (w.q->n == 0 || w.pl.exec == SKY_EXEC_PLAIN) continue;
    if (!first_persistent) first_persistent = &w;
    persistent_segs += w.pl.P;
  }
  record(8, B);
  if (first_persistent) {
    // the engine's chunk policy of a shared launch is the first query's
    // a local phase with few segments has large chunks, like the merge
    CK(engine(bb.segs, persistent_segs, first_persistent->pl.cfg, first_persistent->b.words + W_ERR,
              first_persistent->b.words + W_MAXROUND_LOCAL, W_TESTS_LOCAL,
              persistent_segs <= ORDERED_MAX_SEGS ? ORD_LOOKBACK : ORD_LAST));
  }
  for (auto& w : ws) {
    if (w.q->n == 0 || w.pl.exec != SKY_EXEC_PLAIN) continue;
    for (u32 p = 0; p < w.pl.P; ++p)
      CK(engine(bb.segs + w.seg_base + p, 1, w.pl.cfg, w.b.words + W_ERR, w.b.words + W_MAXROUND_LOCAL,
                W_TESTS_LOCAL, ORD_LOOKBACK));
  }
  record(9, B);
  CK(fork());
  for (auto& w : ws) {
    if (w.q->n == 0) continue;
    const cudaStream_t st = qstream(w);
    CK(launch_stamp_stage(w.b.alive, w.pl.n, w.b.stage_s, ST_LOCAL, st));
  }
  CK(join());
  record(4, B);

  // ---- final phase over u (sequential Sky(u), or NoSeq, Section 4.2)
  CK(fork());
  for (auto& w : ws) {
    if (w.q->n == 0 || w.pl.P <= 1) continue;
    const cudaStream_t st = qstream(w);
    const Plan& pl = w.pl;
    Bufs& b = w.b;
    const u64 n = pl.n;
    const int D = pl.d;
    const u32* nu_dev = b.words + W_NU;
    CK(scan_u8(b.alive, b.excl, n, true, b.scan_tmp, st));
    CK(cudaMemcpyAsync(b.words + W_NU, b.scan_tmp + scan_total_index(n), sizeof(u32), cudaMemcpyDeviceToDevice,
                       st));
    const bool seq = pl.merge == SKY_MERGE_SEQUENTIAL;
    CK(launch_compact_u(b.alive, b.excl, n, D, b.pts, b.hc, b.score, b.spid, b.upts, b.uhc, b.uscore, b.upos,
                        nullptr, seq ? b.keys[0] : nullptr, seq ? b.vals[0] : nullptr, st));
    if (seq) {
      // sort u by score; |u| is read on the device
      int msel = 0;
      CK(radix_sort(b.keys, b.vals, n, 0, 32, b.hist, st, &msel, nu_dev, b.words + W_ERR));
      CK(launch_gather_u(b.vals[msel], n, nu_dev, D, b.upts, b.uhc, b.uscore, b.upos, b.mpts, b.mhc, b.mscore,
                         b.mpos, st));
      CK(cudaMemsetAsync(b.malive, 1, n, st));
      SegArrays ma{b.mpts, b.mhc, b.mscore, b.malive, b.win, b.whc, b.dpos, b.dhc};
      CK(launch_build_one_seg(ma, nu_dev, D, bb.msegs + w.mseg, st));
    } else {
      CK(launch_useg(b.seg_off, pl.P, b.excl, n, nu_dev, b.useg, st));
      CK(cudaMemsetAsync(b.ualive, 1, n, st));
      NoSeqArgs na{};
      na.upts = reinterpret_cast<const float4*>(b.upts);
      na.uhc = b.uhc;
      na.uscore = b.uscore;
      na.useg = b.useg;
      na.ualive = b.ualive;
      na.P = pl.P;
      na.scheme = pl.scheme;
      na.d = D;
      for (int a = 0; a < 8; ++a) na.gd.m[a] = pl.slices[a];
      na.dom_block = pl.cfg.dom_block;
      // keep the item count within 32 bits
      while (((n / 64 + pl.P + 1) * (n / na.dom_block + 1)) >= (1ull << 31)) na.dom_block *= 2;
      CK(launch_noseq(na, b.gcnt, b.gpre, b.scan_tmp, nu_dev, b.words + W_NOSEQ_CTR, st));
      // u is a prefix of the sorted positions' survivors: upos maps back
      CK(launch_scatter_alive(b.ualive, b.upos, n, nu_dev, b.alive, b.stage_s, ST_MERGE, st));
    }
  }
  CK(join());
  record(10, B);
  {
    Work* first = nullptr;
    u32 cnt = 0;
    for (auto& w : ws)
      if (w.mseg >= 0 && w.pl.exec != SKY_EXEC_PLAIN) {
        if (!first) first = &w;
        ++cnt;
      }
    if (first)
      CK(engine(bb.msegs, cnt, first->pl.cfg, first->b.words + W_ERR, first->b.words + W_MAXROUND_MERGE,
                W_TESTS_MERGE, ORD_LOOKBACK));
    for (auto& w : ws)
      if (w.mseg >= 0 && w.pl.exec == SKY_EXEC_PLAIN)
        CK(engine(bb.msegs + w.mseg, 1, w.pl.cfg, w.b.words + W_ERR, w.b.words + W_MAXROUND_MERGE,
                  W_TESTS_MERGE, ORD_LOOKBACK));
  }
  record(11, B);
  CK(fork());
  for (auto& w : ws) {
    if (w.mseg < 0) continue;
    const cudaStream_t st = qstream(w);
    Bufs& b = w.b;
    CK(launch_scatter_alive(b.malive, b.mpos, w.pl.n, b.words + W_NU, b.alive, b.stage_s, ST_MERGE, st));
  }
  CK(join());
  record(5, B);

  // ---- output: ascending indices of Sky(r)
  CK(fork());
  for (u32 i = 0; i < nq; ++i) {
    Work& w = ws[i];
    if (w.q->n == 0) continue;
    const cudaStream_t st = qstream(w);
    Bufs& b = w.b;
    const u64 n = w.pl.n;
    u32* out_pid = w.q->out_pid;
    u8* out_stage = w.q->out_stage;
    CK(launch_output(b.stage_s, b.orig, b.spid, n, b.mask, w.stage_dev ? out_stage : nullptr,
                     w.pid_dev ? out_pid : nullptr, st));
    CK(scan_u8(b.mask, b.excl, n, true, b.scan_tmp, st));
    CK(cudaMemcpyAsync(b.words + W_SKY, b.scan_tmp + scan_total_index(n), sizeof(u32), cudaMemcpyDeviceToDevice,
                       st));
    CK(launch_compact_idx(b.mask, b.excl, n, w.out_dev ? w.q->out_idx : b.out_dev, st));
    CK(launch_stage_hist(b.stage_s, n, b.words + W_HIST, st));
  }
  CK(join());
  record(6, B);
  for (u32 i = 0; i < nq; ++i) {
    Work& w = ws[i];
    if (w.q->n == 0) continue;
    CK(cudaMemcpyAsync(pinned_ + (size_t)i * W_WORDS, w.b.words, W_WORDS * sizeof(u32), cudaMemcpyDeviceToHost,
                       st));
  }
  B.kernels = launch_counter() - k0;
  return SKY_OK;
}

sky_status Runner::finish(BatchState& B) {
  std::vector<Work>& ws = B.ws;
  const u32 nq = B.nq;
  Query* queries = B.queries;
  Work* first_persistent = B.first_persistent;
  const cudaStream_t st = stream;
  CK(cudaStreamSynchronize(st));
  // the error word and round counts of a shared engine launch were written
  // to its first query: every query of the launch shares them
  u32 shared_err = 0, shared_round_local = 0, shared_round_merge = 0;
  // dominance tests of the engine launches: every launch's went to one
  // query's words; a query of the shared launches reports theirs, a query
  // with launches of its own reports those, the batch reports all of them
  // k: 0 local, 1 merge
  u64 tests_all[2] = {0, 0}, tests_shared[2] = {0, 0};
  auto tests_of = [](const Work& w, int k) {
    u64 v;
    memcpy(&v, &w.words[k == 0 ? W_TESTS_LOCAL : W_TESTS_MERGE], sizeof(v));
    return v;
  };
  for (u32 i = 0; i < nq; ++i) {
    Work& w = ws[i];
    if (w.q->n == 0) continue;
    memcpy(w.words, pinned_ + (size_t)i * W_WORDS, sizeof(w.words));
    for (int k = 0; k < 2; ++k) {
      tests_all[k] += tests_of(w, k);
      if (w.pl.exec != SKY_EXEC_PLAIN) tests_shared[k] += tests_of(w, k);
    }
    if (&w == first_persistent) {
      shared_err = w.words[W_ERR] & (ERR_TIMEOUT | ERR_CAPACITY);
      shared_round_local = w.words[W_MAXROUND_LOCAL];
    }
    if (w.mseg >= 0 && w.pl.exec != SKY_EXEC_PLAIN) {
      shared_err |= w.words[W_ERR] & (ERR_TIMEOUT | ERR_CAPACITY);
      shared_round_merge = std::max(shared_round_merge, w.words[W_MAXROUND_MERGE]);
    }
  }
  sky_status first_bad = SKY_OK;
  std::string first_msg;
  for (u32 i = 0; i < nq; ++i) {
    Work& w = ws[i];
    Query& q = *w.q;
    if (q.n == 0) continue;
    u32 e = w.words[W_ERR];
    if (w.pl.exec != SKY_EXEC_PLAIN) e |= shared_err;
    sky_status qs = SKY_OK;
    std::string msg;
    if (e & ERR_NAN) {
      qs = SKY_EINVAL;
      msg = "input contains NaN";
    } else if (e & ERR_TIMEOUT) {
      qs = SKY_ETIMEOUT;
      msg = "a device-side wait timed out";
    } else if (e & ERR_CAPACITY) {
      qs = SKY_ENOMEM;
      msg = "device-side capacity exceeded";
    }
    q.status = qs;
    if (qs != SKY_OK) {
      if (first_bad == SKY_OK) {
        first_bad = qs;
        first_msg = nq > 1 ? "query " + std::to_string(i) + ": " + msg : msg;
      }
      continue;
    }
    const u64 cnt = w.words[W_SKY];
    Bufs& b = w.b;
    const u64 n = w.pl.n;
    if (!w.out_dev && cnt) CK(cudaMemcpyAsync(q.out_idx, b.out_dev, cnt * sizeof(u32), cudaMemcpyDeviceToHost, st));
    // host-side diagnostics
    if (q.out_stage && !w.stage_dev) {
      CK(launch_output(b.stage_s, b.orig, b.spid, n, b.mask, reinterpret_cast<u8*>(b.keys[0]), b.vals[0], st));
      CK(cudaMemcpyAsync(q.out_stage, b.keys[0], n, cudaMemcpyDeviceToHost, st));
      if (q.out_pid && !w.pid_dev) CK(cudaMemcpyAsync(q.out_pid, b.vals[0], n * 4, cudaMemcpyDeviceToHost, st));
    } else if (q.out_pid && !w.pid_dev) {
      CK(launch_output(b.stage_s, b.orig, b.spid, n, b.mask, nullptr, b.vals[0], st));
      CK(cudaMemcpyAsync(q.out_pid, b.vals[0], n * 4, cudaMemcpyDeviceToHost, st));
    }
    *q.out_count = cnt;
    sky_stats& S = q.stats;
    const bool shared = w.pl.exec != SKY_EXEC_PLAIN;
    S.rounds_local = shared ? shared_round_local : w.words[W_MAXROUND_LOCAL];
    S.rounds_merge = (shared && w.mseg >= 0) ? shared_round_merge : w.words[W_MAXROUND_MERGE];
    S.reps_kept = w.pl.rep ? w.words[W_KEPT] : 0;
    S.nonempty_partitions = w.words[W_NONEMPTY];
    S.grid_dropped = w.words[W_HIST + ST_GRID];
    S.rep_dropped = w.words[W_HIST + ST_REP];
    S.local_union = (u64)w.words[W_HIST + ST_MERGE] + w.words[W_HIST + ST_SKY];
    S.skyline = cnt;
    u64 t[2];
    for (int k = 0; k < 2; ++k) t[k] = shared ? tests_shared[k] : tests_of(w, k);
    S.tests_fp16 = t[0] + t[1];
    S.tests_fp16_local = t[0];
  }
  record(7, B);
  CK(cudaStreamSynchronize(st));
  // batch statistics: sums over the queries, maxima of the round counts
  for (u32 i = 0; i < nq; ++i) {
    const sky_stats& S = queries[i].stats;
    stats.n += S.n;
    stats.d = std::max(stats.d, S.d);
    stats.partitions += S.partitions;
    stats.nonempty_partitions += S.nonempty_partitions;
    stats.rounds_local = std::max(stats.rounds_local, S.rounds_local);
    stats.rounds_merge = std::max(stats.rounds_merge, S.rounds_merge);
    stats.reps_kept += S.reps_kept;
    stats.grid_dropped += S.grid_dropped;
    stats.rep_dropped += S.rep_dropped;
    stats.local_union += S.local_union;
    stats.skyline += S.skyline;
  }
  stats.tests_fp16 = tests_all[0] + tests_all[1];
  stats.tests_fp16_local = tests_all[0];
  stats.launches = B.graph ? B.kernels : launch_counter() - B.launches0;
  if (timing && !B.graph) {
    float ms = 0;
    cudaEventElapsedTime(&ms, ev_[0], ev_[7]);
    stats.ms_total = ms;
    for (int i = 0; i < 6; ++i) {
      float t = 0;
      cudaEventElapsedTime(&t, ev_[i + 1], ev_[i + 2]);
      stats.ms_phase[i] = t;
    }
    float tl = 0, tm = 0;
    cudaEventElapsedTime(&tl, ev_[8], ev_[9]);
    cudaEventElapsedTime(&tm, ev_[10], ev_[11]);
    stats.ms_dom_local = tl;
    stats.ms_dom_merge = tm;
  }
  if (first_bad != SKY_OK) return fail(first_bad, first_msg);
  return SKY_OK;
}

// ---------------------------------------------------------------- CUDA graphs

struct StreamHolder {
  cudaStream_t s = nullptr;
  ~StreamHolder() {
    if (s) cudaStreamDestroy(s);
  }
};

struct GraphRun {
  StreamHolder stream;  // destroyed after the Runner that uses it
  Runner R;
  BatchState B;
  std::vector<Runner::Query> qs;
  std::vector<u64> counts;
  cudaGraphExec_t exec = nullptr;
  cudaEvent_t dep = nullptr, e0 = nullptr, e1 = nullptr;
  ~GraphRun() {
    if (exec) cudaGraphExecDestroy(exec);
    for (cudaEvent_t e : {dep, e0, e1})
      if (e) cudaEventDestroy(e);
  }
};

sky_status graph_capture(int device, size_t budget, const Runner::Query* queries, u32 nq, GraphRun** out,
                         std::string* msg) {
  *out = nullptr;
  std::unique_ptr<GraphRun> g(new GraphRun());
  sky_status s = g->R.init(device, budget);
  if (s != SKY_OK) return s;
  if (cudaStreamCreateWithFlags(&g->stream.s, cudaStreamNonBlocking) != cudaSuccess) return SKY_ECUDA;
  g->R.stream = g->stream.s;
  for (cudaEvent_t* e : {&g->dep, &g->e0, &g->e1})
    if (cudaEventCreate(e) != cudaSuccess) return SKY_ECUDA;
  g->qs.assign(queries, queries + nq);
  g->counts.assign(nq, 0);
  for (u32 i = 0; i < nq; ++i) g->qs[i].out_count = &g->counts[i];
  s = g->R.prepare(g->B, g->qs.data(), nq, true);
  if (s != SKY_OK) {
    *msg = g->R.last_error;
    return s;
  }
  if (!g->B.empty) {
    if (cudaStreamBeginCapture(g->stream.s, cudaStreamCaptureModeThreadLocal) != cudaSuccess) return SKY_ECUDA;
    s = g->R.enqueue(g->B);
    cudaGraph_t graph = nullptr;
    cudaError_t e = cudaStreamEndCapture(g->stream.s, &graph);
    if (s != SKY_OK || e != cudaSuccess) {
      if (graph) cudaGraphDestroy(graph);
      cudaGetLastError();
      *msg = s != SKY_OK ? g->R.last_error : std::string("stream capture: ") + cudaGetErrorString(e);
      return s != SKY_OK ? s : SKY_ECUDA;
    }
    e = cudaGraphInstantiate(&g->exec, graph, 0);
    cudaGraphDestroy(graph);
    if (e != cudaSuccess) {
      cudaGetLastError();
      *msg = std::string("graph instantiation: ") + cudaGetErrorString(e);
      return SKY_ECUDA;
    }
  }
  *out = g.release();
  return SKY_OK;
}

sky_status graph_launch(GraphRun* g, cudaStream_t after, u64* counts, sky_status* statuses, double* ms,
                        sky_stats* stats, std::string* msg) {
  if (cudaSetDevice(g->R.device) != cudaSuccess) return SKY_ECUDA;
  sky_status s = SKY_OK;
  if (g->exec) {
    // the replay starts after the work already queued on the caller's stream
    if (cudaEventRecord(g->dep, after) != cudaSuccess || cudaStreamWaitEvent(g->stream.s, g->dep, 0) != cudaSuccess ||
        cudaEventRecord(g->e0, g->stream.s) != cudaSuccess || cudaGraphLaunch(g->exec, g->stream.s) != cudaSuccess ||
        cudaEventRecord(g->e1, g->stream.s) != cudaSuccess) {
      *msg = std::string("graph launch: ") + cudaGetErrorString(cudaGetLastError());
      return SKY_ECUDA;
    }
    s = g->R.finish(g->B);
    if (ms) {
      float t = 0;
      cudaEventElapsedTime(&t, g->e0, g->e1);
      *ms = t;
    }
    if (s != SKY_OK) *msg = g->R.last_error;
  } else if (ms) {
    *ms = 0;
  }
  for (size_t i = 0; i < g->qs.size(); ++i) {
    if (counts) counts[i] = g->counts[i];
    if (statuses) statuses[i] = g->qs[i].status;
  }
  if (stats) *stats = g->R.stats;
  return s;
}

void graph_destroy(GraphRun* g) {
  if (!g) return;
  cudaSetDevice(g->R.device);
  delete g;
}

}  // namespace sky
