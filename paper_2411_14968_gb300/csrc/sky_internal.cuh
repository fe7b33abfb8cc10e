// Internal declarations shared by the translation units of libskyline.
// Nothing here is part of the public C ABI (include/skyline.h).
#pragma once
#include <cstdint>
#include <cuda_runtime.h>
#include <type_traits>

namespace sky {

typedef uint32_t u32;
typedef uint64_t u64;
typedef uint8_t u8;

constexpr u32 FULL = 0xffffffffu;

// ---------------------------------------------------------------- numerics
// Monotone unsigned image of a non-NaN FP32 value (a < b <=> fkey(a) <
// fkey(b), given -0.0 was turned into +0.0).  Only sort keys use it;
// dominance always compares the FP32 values themselves.
__host__ __device__ inline u32 fkey(float x) {
#ifdef __CUDA_ARCH__
  u32 b = __float_as_uint(x);
#else
  u32 b;
  __builtin_memcpy(&b, &x, 4);
#endif
  return (b & 0x80000000u) ? ~b : (b | 0x80000000u);
}
__host__ __device__ inline float fkey_inv(u32 k) {
  u32 b = (k & 0x80000000u) ? (k & 0x7fffffffu) : ~k;
#ifdef __CUDA_ARCH__
  return __uint_as_float(b);
#else
  float x;
  __builtin_memcpy(&x, &b, 4);
  return x;
#endif
}

// Number of float4 per stored point: 1 for d <= 4, 2 for d <= 8.  Padding
// attributes are +0.0 in every point, so they never decide a dominance test.
__host__ __device__ constexpr int vec_of(int d) { return (d + 3) / 4; }

// Bits of the device error word.
enum : u32 {
  ERR_NAN = 1u,       // an input attribute is NaN
  ERR_TIMEOUT = 2u,   // a bounded wait gave up
  ERR_CAPACITY = 4u,  // a device-side capacity check failed
};

// Partition schemes (same numbering as the public enum).
enum : int { SCHEME_RANDOM = 0, SCHEME_GRID = 1, SCHEME_ANGULAR = 2, SCHEME_SLICED = 3, SCHEME_NONE = 4 };

// Stage codes written per point (same numbering as the public documentation).
enum : u8 { ST_SKY = 1, ST_GRID = 2, ST_REP = 3, ST_LOCAL = 4, ST_MERGE = 5 };

// Kernel launches issued by this library in the calling host thread (each
// launch site calls note_launch() right before its launch).
u64& launch_counter();
inline void note_launch() { ++launch_counter(); }

template <class F>
inline cudaError_t dispatch_d(int d, F&& f) {
  switch (d) {
    case 1: f(std::integral_constant<int, 1>()); break;
    case 2: f(std::integral_constant<int, 2>()); break;
    case 3: f(std::integral_constant<int, 3>()); break;
    case 4: f(std::integral_constant<int, 4>()); break;
    case 5: f(std::integral_constant<int, 5>()); break;
    case 6: f(std::integral_constant<int, 6>()); break;
    case 7: f(std::integral_constant<int, 7>()); break;
    case 8: f(std::integral_constant<int, 8>()); break;
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

// ---------------------------------------------------------------- primitives (sky_prims.cu)
// Device-wide scan of n values (u8 or u32 input) into u32 (add or max).
// tmp must hold scan_tmp_words(n) u32; tmp[scan_total_index(n)] receives the
// total.  In-place (in == out) is allowed for u32.
size_t scan_tmp_words(u64 n);
u64 scan_total_index(u64 n);
cudaError_t scan_u32(const u32* in, u32* out, u64 n, bool exclusive, bool use_max, u32* tmp,
                     cudaStream_t st);
cudaError_t scan_u8(const u8* in, u32* out, u64 n, bool exclusive, u32* tmp, cudaStream_t st);

// Stable LSD radix sort of (u64 key, u32 value) pairs on key bits [lo_bit,
// hi_bit) (at most 64 bits, n < 2^32).  Input in k[0], v[0]; *out_sel
// receives the index (0 or 1) of the buffer pair that holds the output.
// work: radix_work_words(n) u32 (zeroed by the sort itself).  With n_dev the
// element count is min(n, *n_dev), read on the device (n is the capacity the
// grids are sized for), so no host round trip is needed.  err (optional)
// receives ERR_TIMEOUT if a bounded look-back wait gave up.
size_t radix_work_words(u64 n);
cudaError_t radix_sort(u64* k[2], u32* v[2], u64 n, int lo_bit, int hi_bit, u32* work, cudaStream_t st,
                       int* out_sel, const u32* n_dev = nullptr, u32* err = nullptr);
// The same for 32-bit keys (hi_bit <= 32): 16 instead of 24 bytes moved per
// key and pass.
cudaError_t radix_sort(u32* k[2], u32* v[2], u64 n, int lo_bit, int hi_bit, u32* work, cudaStream_t st,
                       int* out_sel, const u32* n_dev = nullptr, u32* err = nullptr);

// ---------------------------------------------------------------- rank space (sky_rank.cu)
// Codes of the rank images: the finite non-negative FP16 bit patterns
// 0x0000..0x7BFF, in increasing order.
constexpr u32 RANK_CODES = 0x7C00;
// Order-preserving code of dense rank `rank` in a column of R distinct
// values: the rank itself when it fits, else rank scaled down (floor), which
// is non-decreasing in the rank and maps R - 1 to the largest code.
__host__ __device__ inline u32 rank_code(u32 rank, u32 R) {
  return R <= RANK_CODES ? rank : (u32)(((u64)rank * (RANK_CODES - 1)) / (R - 1));
}
struct RankScratch {
  u64* keys[2];   // n each (the sort uses them as 32-bit key arrays)
  u32* vals[2];   // n each
  u32* work;      // radix_work_words(n)
  u8* flag;       // n
  u32* incl;      // n
  u32* scan_tmp;  // scan_tmp_words(n)
  u32* cols;      // d x n: the ranks column by column
};
// Dense ranks of every column of X (N x d row-major, device) into s.cols and
// distinct[a] (device, d words), then row-major: ranks[i*d + a] (optional),
// codes[i*d + a] = rank_code(rank, distinct[a]) (optional), and the codes
// packed eight halves per point (optional).  NaN sets ERR_NAN in *err.
cudaError_t launch_rank_space(const float* X, u64 n, u32 d, const RankScratch& s, u32* ranks,
                              unsigned short* codes, uint4* packed, u32* distinct, u32* err, cudaStream_t st);

// ---------------------------------------------------------------- prep (sky_prep.cu)
struct PrepArgs {
  const float* X;        // row-major input, n x d
  u64 n;
  int scheme;
  int normalize;         // divide attributes by the column maximum for keys
  int slice_dim;
  u64 seed;
  u32 slices[8];
  const u32* colmax;     // fkey of the column maxima (normalize only)
  const float* ang_table;  // Angular thresholds tan^2(k pi / 2m), per angle
  u32 ang_off[8];
  u64* keys;             // out: first sort key
  u32* vals;             // out: point index
  u32* err;
};

struct GatherArgs {
  const float* X;
  u64 n;
  const u64* keys;       // sorted keys; partition id in bits 63..32
  const u32* vals;       // sorted point indices
  u32 P;                 // partitions
  float* pts;            // out: padded points in sorted order, vec_of(d) float4 each
  const uint4* rcode;    // rank images by original index (rank space), or NULL: FP16 round-down
  uint4* hc;             // out: images of the points (rcode's, else FP16 round-down)
  float* score;          // out: scores in sorted order
  u32* orig;             // out: original index of sorted position
  u32* spid;             // out: partition of sorted position
  u8* alive;             // out: 1
  u32* seg_off;          // out: P + 1 segment offsets
};

cudaError_t launch_colmax(const float* X, u64 n, int d, u32* colmax, u32* err, cudaStream_t st);
cudaError_t launch_prep(const PrepArgs& p, int d, cudaStream_t st);
cudaError_t launch_rekey(const float* X, u64 n, int d, const u32* sorted_idx, const u32* run_start,
                         u32 P, u64* keys, u32* vals, cudaStream_t st);
cudaError_t launch_run_heads(const u64* keys, u64 n, u32* head, cudaStream_t st);
cudaError_t launch_gather(const GatherArgs& g, int d, cudaStream_t st);

struct GridDims { u32 m[8]; };
cudaError_t launch_grid_filter(const u32* seg_off, const u32* spid, u64 n, int d, const GridDims& gd,
                               u32 P, u8* clos, u8* dropped, u8* alive, u8* stage_s, u32* counter,
                               cudaStream_t st);
// Sorted representatives (4.1): the first k points of every non-empty,
// non-dropped partition, packed; empty slots hold +inf points and
// rep_alive 0.
cudaError_t launch_rep_select(const u32* seg_off, u32 P, u32 k, const u8* dropped, const float* pts,
                              int d, float* rep_pts, u8* rep_alive, cudaStream_t st);
// Region representatives (Section 4.1): per segment the k points of largest
// dominance-region volume inside [0,1]^d (orig breaks ties); colmax (fkey
// column maxima) scales the attributes when normalize is set.
cudaError_t launch_rep_region(const u32* seg_off, u32 P, u32 k, const u8* dropped, const float* pts, const u32* orig,
                              const u32* colmax, int normalize, int d, float* rep_pts, u8* rep_alive, cudaStream_t st);

// Compaction of the points alive after the local phase into u (keeps the
// (partition, score, index) order).
cudaError_t launch_compact_u(const u8* alive, const u32* excl, u64 n, int d, const float* pts, const uint4* hc,
                             const float* score, const u32* spid, float* upts, uint4* uhc, float* uscore,
                             u32* upos, u32* upid, u64* ukey, u32* uval, cudaStream_t st);
// useg[s] = offset of u_s in u (P + 1 entries); total = device pointer to |u|.
cudaError_t launch_useg(const u32* seg_off, u32 P, const u32* excl, u64 n, const u32* total, u32* useg,
                        cudaStream_t st);
// u in score order: entry r of the merge array is u[order[r]], for r below
// n (capacity) and *n_dev (if given).
cudaError_t launch_gather_u(const u32* order, u64 n, const u32* n_dev, int d, const float* upts, const uint4* uhc,
                            const float* uscore, const u32* upos, float* mpts, uint4* mhc, float* mscore,
                            u32* mpos, cudaStream_t st);
// Points dead in a merge array (entries below n and *n_dev if given): their
// sorted-position flag is cleared and, if no stage was recorded yet, stage
// `code` is recorded.
cudaError_t launch_scatter_alive(const u8* malive, const u32* mpos, u64 n, const u32* n_dev, u8* alive,
                                 u8* stage_s, u8 code, cudaStream_t st);
// Points dead (alive == 0) with no stage recorded get `code`.
cudaError_t launch_stamp_stage(const u8* alive, u64 n, u8* stage_s, u8 code, cudaStream_t st);
// Output mask in input order; a point with no stage recorded is in the
// skyline (stage SKY).  Optional per-point diagnostics in input order.
cudaError_t launch_output(u8* stage_s, const u32* orig, const u32* spid, u64 n, u8* mask,
                          u8* stage_out, u32* pid_out, cudaStream_t st);
cudaError_t launch_compact_idx(const u8* mask, const u32* excl, u64 n, u32* out, cudaStream_t st);
cudaError_t launch_compact_reps(const u8* rep_alive, const u32* excl, u32 nrep, int d, const float* rep_pts,
                                float* kept_pts, cudaStream_t st);
cudaError_t launch_stage_hist(const u8* stage_s, u64 n, u32* hist6, cudaStream_t st);

// ---------------------------------------------------------------- dominance engine (sky_engine.cu)
// FP16 images of a point's attributes: __float2half_rd of each attribute
// clamped to [-65504, 65504], packed two per 32-bit word (attribute 2k in
// the low half), +0 padding.  Both maps are monotone, so w[a] > t[a]
// whenever code(w)[a] > code(t)[a]; images are finite and never -0 (the
// attributes' -0.0 is turned into +0.0 first).
//
// One segment (a partition, or the whole merge input) of the SFS engine.
// The points of a segment are sorted by score; win/whc and dpos/dhc have
// room for n entries each (whc and dhc for n + 1, rounded to whole pairs,
// starting at an even entry of their arrays).
struct SegDesc {
  const float4* pts;     // vec_of(d) float4 per point, sorted by score
  const uint4* hc;       // FP16 images of pts
  const float* score;
  u8* alive;
  float4* win;           // window: skyline points found so far (FP32)
  uint4* whc;            // window FP16 images, stored as pairs (32 bytes per two entries)
  u32* dpos;             // dense list of the round: segment-relative positions
  uint4* dhc;            // dense list FP16 images, stored as pairs
  u32 n;
  u32 d;                 // attributes (1..8)
};

// Round state of a segment (written by the CTA that starts the round).
struct SegState {
  u32 cur;      // first position of the current chunk
  u32 cend;     // end of the current chunk (never splits a run of equal scores)
  u32 wlen;     // window points visible to this round
  u32 wfill;    // window append cursor (atomic)
  u32 tiles;    // candidate tiles of the chunk (phase A)
  u32 dlen;     // dense-list length after phase A (atomic)
  u32 done_a;   // phase-A tiles finished (atomic)
  u32 done_b;   // phase-B tiles finished (atomic)
  u32 rounds;   // rounds completed
};

// Built-in defaults of the engine knobs (sky_params: 0 selects these).  A
// short first chunk builds a window quickly; later chunks are 8x the window.
constexpr u32 DEFAULT_CHUNK_MIN = 1024;
constexpr u32 DEFAULT_CHUNK_MAX = 262144;
constexpr u32 DEFAULT_ALPHA_X4 = 32;
constexpr u32 DEFAULT_DOM_BLOCK = 1024;
enum : u32 { ORD_NONE = 0, ORD_LOOKBACK = 1, ORD_LAST = 2 };
constexpr u32 ORD_LAST_MAX = 16384;

// Default launch shape of the engine: warps per CTA x candidates per lane.
constexpr u32 DEFAULT_ENGINE_WARPS = 4;
constexpr u32 DEFAULT_ENGINE_CANDS = 4;
// Smallest tile (candidates per work item) of any compiled shape: 4 warps x
// 32 lanes x 2 candidates.
constexpr u32 ENGINE_MIN_TILE = 256;

struct EngineCfg {
  u32 chunk_min, chunk_max, alpha_x4, dom_block;
  // launch shape: warps per CTA (4 or 8) and candidates per lane (2 or 4);
  // 0 selects the default
  u32 warps, cands;
  // How phase A builds a segment's dense list: ORD_NONE in arrival order
  // (phase B tests the whole dense square); ORD_LOOKBACK in position order,
  // each tile writing its survivors at the sum of its predecessors' counts
  // (decoupled look-back; phase B tests only the lower-score half of the
  // square; pays off for large chunks, the merge); ORD_LAST in position
  // order, written by the last tile of the phase over the whole chunk (the
  // half square without look-back waits; for many small chunks: a round
  // whose chunk is longer than ORD_LAST_MAX points uses ORD_NONE instead,
  // since one CTA compacts the chunk)
  u32 ordered;
  // Test hooks, zero unless set through sky_diag_engine_wait_test: the bound
  // of every device-side wait without progress (0 = the built-in 4 s), and
  // the 1-based index of a task of the launch that is reserved but never
  // published (0 = none), which makes the waits for it run out.
  u64 wait_ns;
  u32 withhold_task;
};

struct EngineWork {
  SegState* st;       // nseg
  u32* tbase;         // nseg
  u32* tdoneA;        // engine_tile_capacity(...) counters, zero before the first launch
  u32* tdoneB;        // same
  u32* tstat;         // same count of tile status words
  u64 tcap;
  void* tasks;        // engine_task_capacity(...) x engine_task_bytes() bytes
  u64 task_cap;
  u32* ctl;           // ENGINE_CTL_WORDS control words
};
constexpr int ENGINE_CTL_WORDS = 16;
u64 engine_tile_capacity(u64 total_points, u32 nseg);
// Tasks (phases of segments) one launch can publish at most.
u64 engine_task_capacity(u64 total_points, u32 nseg, u32 chunk_min);
size_t engine_task_bytes();
// Control word that receives the largest round count of a launch.
u32 engine_max_round_word();
u32 engine_tests_word();  // the u64 control word counting the launch's FP16 dominance tests
// Largest dominator block (points) the engine stages in shared memory.
u32 engine_max_dom_block();

// Local skylines of segs[0..nseg) in one persistent launch (grid = the
// co-resident capacity) driven by a device-side work queue.  Kills dominated
// points (alive = 0) and leaves each segment's skyline in its window.
cudaError_t engine_run(const SegDesc* segs_dev, u32 nseg, const EngineCfg& cfg, const EngineWork& w, u32* err,
                       cudaStream_t st);
// Whether (warps, cands) names a compiled launch shape (0 = default).
bool engine_shape_ok(u32 warps, u32 cands);
// engine_run for one compiled shape (sky_engine_w<W>r<R>.cu).
template <int W, int RR>
cudaError_t engine_run_variant(const SegDesc* segs_dev, u32 nseg, const EngineCfg& cfg, const EngineWork& w,
                               u32* err, cudaStream_t st);

// Segment descriptors (sky_dom.cu).
struct SegArrays {
  const float* pts;
  const uint4* hc;
  const float* score;
  u8* alive;
  float* win;
  uint4* whc;
  u32* dpos;
  uint4* dhc;
};
// nonempty (may be NULL): incremented once per partition that holds a point
// (before Grid Filtering).
cudaError_t launch_build_segs(const u32* seg_off, u32 P, const u8* dropped, const SegArrays& a, int d,
                              SegDesc* segs, u32* nonempty, cudaStream_t st);
cudaError_t launch_build_one_seg(const SegArrays& a, const u32* n_dev, int d, SegDesc* seg, cudaStream_t st);
// After an engine launch (whose control words are ctl): the launch's round
// count into *round_dst (maximum) and its test count into *tests_dst (sum).
cudaError_t launch_fold_engine(const u32* ctl, u32* round_dst, unsigned long long* tests_dst, cudaStream_t st);

// Relative skyline (Section 4.2 definition): kill every alive candidate of
// cand[0..nc) dominated by one of dom[0..nd) (nd = *nd_dev if given, else
// nd_host).
cudaError_t launch_relative(const float* cand, u8* alive, u64 nc, const float* dom, u32 nd_host,
                            const u32* nd_dev, int d, cudaStream_t st);

// NoSeq final phase: u sorted by (partition, score) with offsets useg[P+1];
// t in u_i is killed iff some s in pd_i dominates it.
struct NoSeqArgs {
  const float4* upts;
  const uint4* uhc;  // FP16 round-down images of u (packed, two per word)
  const float* uscore;
  const u32* useg;   // P + 1
  u8* ualive;
  u32 P;
  int scheme;
  int d;
  GridDims gd;       // Grid: slices per attribute
  u32 dom_block;
};
// counter: one device word, the kernel's work counter (zeroed here).
cudaError_t launch_noseq(const NoSeqArgs& a, u32* gcnt, u32* gpre, u32* scan_tmp, const u32* nu_dev, u32* counter,
                         cudaStream_t st);

int device_sm_count();

// Compare-throughput probe (sky_probe.cu).
cudaError_t probe_compare_rate(u32 iters, cudaStream_t st, double* per_s, u32* sms_out, u32* sink);
cudaError_t probe_reject_rate(u32 iters, cudaStream_t st, double* per_s, u32* sms_out, u32* sink);

}  // namespace sky
