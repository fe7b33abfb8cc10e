// Local-skyline engine: Algorithm 1 (SFS) run on every partition of
// Algorithm 2 at once, in one persistent cooperative launch.
//
// Exactness rests on one fact: t is outside Sky(r) iff some point of r
// dominates t, whether or not that point is in the skyline itself (a minimal
// dominator exists because dominance is a strict partial order on a finite
// set, and it lies in the skyline).  So a candidate may be tested against any
// superset of its skyline dominators and the result is still exact.  Score
// order (f = attribute sum, monotone) bounds where those dominators are:
// s < t implies f(s) <= f(t).
//
// SFS in rounds.  The points of a segment are sorted by f.  A round takes the
// next chunk of the segment (cut only between different scores), so every
// point of the window -- the skyline points of the earlier chunks -- has a
// strictly lower score than every chunk point, and every skyline dominator of
// a chunk point is either in the window or in the chunk itself.  A round has
// two phases separated by a grid barrier:
//   A. every chunk point is tested against the first window block (the
//      strongest, lowest-score skyline points); the survivors of each tile of
//      the chunk are compacted into the segment's dense list;
//   B. every dense-list point is tested against the rest of the window and
//      against the whole dense list (a chunk dominator killed in phase A was
//      itself dominated by a window point that also dominates the candidate,
//      so the dense list holds every chunk dominator that matters); the
//      survivors are appended to the window.
// The last tile of a segment plans the segment's next round.
//
// Dominance test.  Every point carries, next to its FP32 attributes, their
// round-down FP16 images packed two per 32-bit word.  Round-down is monotone,
// so if any FP16 image of w exceeds t's, then w exceeds t in that attribute
// and cannot dominate t: the FP16 test rejects exactly, two attributes per
// half2 compare, and only pairs it passes are tested in FP32 (Def. 1).
//
// Work items are (tile of 8 warps x 32 lanes x R candidates, dominator block
// of DB points), numbered block-major so that the strongest window points run
// first.  A CTA stages the block's FP16 images in shared memory with one
// cp.async.bulk copy completing on an mbarrier; each warp scans it with
// broadcast shared loads and leaves the item when a ballot shows all its
// candidates dead.  Every wait (mbarrier, grid barrier) is bounded by
// %globaltimer and reports ERR_TIMEOUT instead of hanging.
#include <algorithm>
#include <cuda_fp16.h>
#include "sky_internal.cuh"

namespace sky {

namespace {

constexpr int WARPS = 8;
constexpr int THREADS = WARPS * 32;
constexpr int R = 4;                    // candidates per lane
constexpr int GS = 32 * R;              // candidates per warp
constexpr int TILE = WARPS * GS;        // candidates per tile (CTA item)
constexpr u32 DBMAX = 2048;             // dominator block capacity (points)
constexpr u32 A_BLOCKS = 1;             // window blocks of phase A
constexpr u32 MAX_SEG = 4096;           // segments per launch (shared-memory prefix)
constexpr u64 WAIT_NS = 4000000000ull;  // bound of every wait

enum { C_A0 = 0, C_A1 = 1, C_B0 = 2, C_B1 = 3, C_BAR_COUNT = 4, C_BAR_GEN = 5, C_ABORT = 6, C_MAXROUND = 7,
       C_PROGRESS = 8 };

__device__ __forceinline__ u64 globaltimer() {
  u64 t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}
__device__ __forceinline__ u32 ld_cg_u32(const u32* p) { return __ldcg(p); }
__device__ __forceinline__ u32 ld_vol_u32(const u32* p) { return *(const volatile u32*)p; }
__device__ __forceinline__ u8 ld_cg_u8(const u8* p) { return (u8)__ldcg(reinterpret_cast<const unsigned char*>(p)); }
__device__ __forceinline__ u32 smem_addr(const void* p) { return (u32)__cvta_generic_to_shared(p); }

// ------------------------------------------------------------ mbarrier + bulk copy

__device__ __forceinline__ void mbar_init(u64* bar) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_addr(bar)) : "memory");
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
__device__ __forceinline__ void mbar_expect_tx(u64* bar, u32 bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)), "r"(bytes)
               : "memory");
}
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, u32 bytes, u64* bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
          smem_addr(dst)),
      "l"(src), "r"(bytes), "r"(smem_addr(bar))
      : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(u64* bar, u32 parity) {
  u32 ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(smem_addr(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}
// Bounded wait for phase `parity` of the barrier.  On timeout the error and
// abort words are set and false is returned.
__device__ bool mbar_wait(u64* bar, u32 parity, u32* err, u32* ctl) {
  if (mbar_try_wait(bar, parity)) return true;
  u64 t0 = globaltimer();
  while (!mbar_try_wait(bar, parity)) {
    if (globaltimer() - t0 > WAIT_NS) {
      atomicOr(err, ERR_TIMEOUT);
      atomicExch(ctl + C_ABORT, 1u);
      return false;
    }
  }
  return true;
}
// Generic-proxy writes of global memory made visible to later bulk copies.
__device__ __forceinline__ void fence_proxy_async() { asm volatile("fence.proxy.async.global;" ::: "memory"); }

// Grid-wide barrier of the cooperative launch.  The wait is bounded by
// progress, not by its length: a CTA gives up (ERR_TIMEOUT, abort) only
// after WAIT_NS in which no work item anywhere completed, so a long round
// of a large input is not mistaken for a hang.
__device__ bool grid_barrier(u32* ctl, u32* err) {
  __shared__ int s_ok;
  __syncthreads();
  if (threadIdx.x == 0) {
    u32 gen = ld_vol_u32(ctl + C_BAR_GEN);
    __threadfence();
    fence_proxy_async();
    u32 arrived = atomicAdd(ctl + C_BAR_COUNT, 1u);
    bool ok = true;
    if (arrived == gridDim.x - 1) {
      atomicExch(ctl + C_BAR_COUNT, 0u);
      __threadfence();
      atomicAdd(ctl + C_BAR_GEN, 1u);
    } else {
      u64 t0 = globaltimer();
      u32 seen = ld_vol_u32(ctl + C_PROGRESS);
      while (ld_vol_u32(ctl + C_BAR_GEN) == gen) {
        if (ld_vol_u32(ctl + C_ABORT)) { ok = false; break; }
        const u32 now = ld_vol_u32(ctl + C_PROGRESS);
        if (now != seen) {
          seen = now;
          t0 = globaltimer();
        }
        if (globaltimer() - t0 > WAIT_NS) {
          atomicOr(err, ERR_TIMEOUT);
          atomicExch(ctl + C_ABORT, 1u);
          ok = false;
          break;
        }
        __nanosleep(64);
      }
    }
    __threadfence();
    s_ok = ok && !ld_vol_u32(ctl + C_ABORT);
  }
  __syncthreads();
  return s_ok;
}

// ------------------------------------------------------------ dominance test

template <int D>
struct HW {
  static constexpr int value = (D + 1) / 2;  // half2 words that hold D attributes
};

__device__ __forceinline__ bool hle2(u32 a, u32 b) {
  return __hble2(*reinterpret_cast<const __half2*>(&a), *reinterpret_cast<const __half2*>(&b));
}

// All FP16 images of w <= those of t (necessary for w to dominate t).
template <int D>
__device__ __forceinline__ bool codes_le(const uint4& w, const uint4& t) {
  bool le = hle2(w.x, t.x);
  if (HW<D>::value > 1) le &= hle2(w.y, t.y);
  if (HW<D>::value > 2) le &= hle2(w.z, t.z);
  if (HW<D>::value > 3) le &= hle2(w.w, t.w);
  return le;
}

// Def. 1 on the FP32 attributes.
template <int D>
__device__ __forceinline__ bool dominates_fp32(const float4* w, const float4* t) {
  float4 a = w[0], b = t[0];
  float wa[8] = {a.x, a.y, a.z, a.w, 0, 0, 0, 0};
  float ta[8] = {b.x, b.y, b.z, b.w, 0, 0, 0, 0};
  if (D > 4) {
    float4 c = w[1], e = t[1];
    wa[4] = c.x; wa[5] = c.y; wa[6] = c.z; wa[7] = c.w;
    ta[4] = e.x; ta[5] = e.y; ta[6] = e.z; ta[7] = e.w;
  }
  bool le = true, ne = false;
#pragma unroll
  for (int k = 0; k < D; ++k) {
    le &= wa[k] <= ta[k];
    ne |= wa[k] != ta[k];
  }
  return le && ne;
}

constexpr u32 NEG_INF2 = 0xFC00FC00u;  // (-inf, -inf)
constexpr u32 POS_INF2 = 0x7C007C00u;  // (+inf, +inf)

// The candidates of one lane.
struct Cands {
  uint4 c[R];    // FP16 images (-inf when dead)
  u32 pos[R];    // segment-relative position
  bool alive[R];
  bool was[R];
};

// Where the FP32 attributes of dominator j of a staged block live: win[base
// + j] (window) or pts[map[base + j]] (dense list).
struct DomSrc {
  const float4* fp32;
  const u32* map;
  u32 base;
};

template <int D>
__device__ __forceinline__ const float4* dom_fp32(const DomSrc& s, u32 j) {
  constexpr int V = vec_of(D);
  u32 idx = s.base + j;
  if (s.map) idx = __ldcg(s.map + idx);
  return s.fp32 + (u64)idx * V;
}

// Scans the staged block sb[0..cnt) for the warp's candidates.
template <int D>
__device__ __forceinline__ void scan_smem(const uint4* sb, u32 cnt, const DomSrc& src, const float4* pts,
                                          Cands& c) {
  constexpr int V = vec_of(D);
  constexpr int U = 4;
  for (u32 j = 0; j < cnt; j += U) {
    uint4 w[U];
#pragma unroll
    for (int u = 0; u < U; ++u) w[u] = (j + u < cnt) ? sb[j + u] : make_uint4(POS_INF2, POS_INF2, POS_INF2, POS_INF2);
    bool hit = false;
#pragma unroll
    for (int u = 0; u < U; ++u)
#pragma unroll
      for (int r = 0; r < R; ++r) hit |= codes_le<D>(w[u], c.c[r]);
    if (hit) {
#pragma unroll
      for (int u = 0; u < U; ++u)
#pragma unroll
        for (int r = 0; r < R; ++r) {
          if (c.alive[r] && j + u < cnt && codes_le<D>(w[u], c.c[r])) {
            // for window dominators the FP32 copy may have been written in
            // an earlier round by another SM: read it through L2
            const float4* wp = dom_fp32<D>(src, j + u);
            float4 wv[2], tv[2];
            wv[0] = __ldcg(wp);
            tv[0] = __ldg(pts + (u64)c.pos[r] * V);
            if (V > 1) {
              wv[1] = __ldcg(wp + 1);
              tv[1] = __ldg(pts + (u64)c.pos[r] * V + 1);
            }
            if (dominates_fp32<D>(wv, tv)) {
              c.alive[r] = false;
              c.c[r] = make_uint4(NEG_INF2, NEG_INF2, NEG_INF2, NEG_INF2);
            }
          }
        }
    }
    if ((j & 31) == 28) {
      bool any = false;
#pragma unroll
      for (int r = 0; r < R; ++r) any |= c.alive[r];
      if (!__any_sync(FULL, any)) break;
    }
  }
}

__device__ __forceinline__ bool any_alive(const Cands& c) {
  bool a = false;
#pragma unroll
  for (int r = 0; r < R; ++r) a |= c.alive[r];
  return a;
}

__device__ __forceinline__ u32 ceil_div(u32 a, u32 b) { return (a + b - 1) / b; }

// ------------------------------------------------------------ rounds

struct Params {
  const SegDesc* segs;
  u32 nseg;
  EngineCfg cfg;
  SegState* st;        // 2 * nseg
  u32* done_round;     // nseg
  u32* tdoneA;         // per tile of phase A (capacity tcap)
  u32* tdoneB;         // per tile of phase B (capacity tcap)
  u64 tcap;
  u32* ctl;
  u32* err;
};

__device__ __forceinline__ u32 upper_bound_score(const float* __restrict__ score, u32 from, u32 n, float v) {
  u32 lo = from, hi = n;
  while (lo < hi) {
    u32 mid = lo + ((hi - lo) >> 1);
    if (__ldg(score + mid) <= v) lo = mid + 1;
    else hi = mid;
  }
  return lo;
}

// Next chunk of a segment: nominal length from the window size, extended to
// the end of a run of equal scores.
__device__ void plan_round(const SegDesc& sd, const EngineCfg& cfg, SegState& s) {
  s.dlen = 0;
  s.done_a = 0;
  s.done_b = 0;
  if (s.cur >= sd.n) {
    s.cend = sd.n;
    s.tiles = 0;
    return;
  }
  u64 k = ((u64)s.wlen * cfg.alpha_x4) / 4;
  k = k < cfg.chunk_min ? cfg.chunk_min : k;
  k = k > cfg.chunk_max ? cfg.chunk_max : k;
  u64 e = (u64)s.cur + k;
  if (e >= sd.n) s.cend = sd.n;
  else s.cend = upper_bound_score(sd.score, (u32)e, sd.n, __ldg(sd.score + e - 1));
  s.tiles = ceil_div(s.cend - s.cur, TILE);
}

__device__ __forceinline__ u32 items_a(const SegState& s, u32 DB) {
  u32 wb = ceil_div(s.wlen, DB);
  return s.tiles * max(1u, min(wb, A_BLOCKS));
}
__device__ __forceinline__ u32 dtiles_of(const SegState& s) { return ceil_div(s.dlen, TILE); }
__device__ __forceinline__ u32 items_b(const SegState& s, u32 DB) {
  u32 wb = ceil_div(s.wlen, DB);
  u32 wbB = wb > A_BLOCKS ? wb - A_BLOCKS : 0;
  return dtiles_of(s) * (wbB + ceil_div(s.dlen, DB));
}

// One work item as the producer thread planned it.
struct Meta {
  u32 item;    // item index of the phase (>= total: no item)
  u32 s;       // segment
  u32 tile;    // candidate tile (phase A) or dense-list tile (phase B)
  u32 tgid;    // global tile id (completion counters)
  u32 cnt;     // dominators staged in the item's buffer
  u32 base;    // index of the first staged dominator in its source
  u32 dense;   // 1: the dominators are dense-list points (FP32 via dpos)
  u32 copied;  // 1: a bulk copy into the item's buffer was issued
};

struct Shared {
  Meta meta[2];
  u64 bar[2];
  u32 bar_phase[2];
  u32 flag;
  u32 warp_tot[WARPS];
  u32 carry;
};

// Exclusive prefix over segments of the item count (phase 0: A, 1: B) and
// of the tile count, into out_items / out_tiles [nseg + 1].
__device__ void prefix_segments(const Params& P, const SegState* cur, u32 round, int phase, u32* out_items,
                                u32* out_tiles, Shared& S) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const u32 DB = P.cfg.dom_block;
  for (int pass = 0; pass < 2; ++pass) {
    u32* out = pass == 0 ? out_items : out_tiles;
    if (threadIdx.x == 0) S.carry = 0;
    __syncthreads();
    for (u32 base = 0; base < P.nseg; base += THREADS) {
      u32 i = base + threadIdx.x;
      u32 v = 0;
      if (i < P.nseg && ld_cg_u32(P.done_round + i) > round) {
        SegState s;
        s.wlen = ld_cg_u32(&cur[i].wlen);
        s.tiles = ld_cg_u32(&cur[i].tiles);
        s.dlen = ld_cg_u32(&cur[i].dlen);
        if (phase == 0) v = pass == 0 ? items_a(s, DB) : s.tiles;
        else v = pass == 0 ? items_b(s, DB) : dtiles_of(s);
      }
      u32 x = v;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        u32 y = __shfl_up_sync(FULL, x, o);
        if (lane >= o) x += y;
      }
      if (lane == 31) S.warp_tot[warp] = x;
      __syncthreads();
      u32 pre = S.carry;
      for (int w2 = 0; w2 < warp; ++w2) pre += S.warp_tot[w2];
      if (i < P.nseg) out[i] = pre + x - v;
      __syncthreads();
      if (threadIdx.x == THREADS - 1) S.carry = pre + x;
      __syncthreads();
    }
    if (threadIdx.x == 0) out[P.nseg] = S.carry;
    __syncthreads();
  }
}

__device__ __forceinline__ u32 find_segment(const u32* pre, u32 nseg, u32 it) {
  u32 lo = 0, hi = nseg;
  while (hi - lo > 1) {
    u32 mid = (lo + hi) >> 1;
    if (pre[mid] <= it) lo = mid;
    else hi = mid;
  }
  return lo;
}

// Producer (thread 0 only): takes the next item of the phase and starts the
// bulk copy of its dominator block's FP16 images into buffer `slot`.  The
// buffer is free: every warp has passed the end of the item that used it.
__device__ void produce(const Params& P, int phase, const SegState* cur, const u32* s_items, const u32* s_tiles,
                        u32 total, u32* counter, uint4* buf, int slot, Shared& S) {
  Meta m;
  m.item = atomicAdd(counter, 1u);
  m.copied = 0;
  m.cnt = 0;
  if (m.item < total) {
    const u32 DB = P.cfg.dom_block;
    m.s = find_segment(s_items, P.nseg, m.item);
    const u32 l = m.item - s_items[m.s];
    const u32 tiles_s = s_tiles[m.s + 1] - s_tiles[m.s];
    m.tile = l % tiles_s;  // block-major numbering: item l = block * tiles + tile
    const u32 b = l / tiles_s;
    m.tgid = s_tiles[m.s] + m.tile;
    const u32 wlen = ld_cg_u32(&cur[m.s].wlen);
    const uint4* codes;
    if (phase == 0) {
      m.cnt = min(wlen, DB);
      m.base = 0;
      m.dense = 0;
      codes = P.segs[m.s].whc;
    } else {
      const u32 dlen = ld_cg_u32(&cur[m.s].dlen);
      const u32 wb = ceil_div(wlen, DB);
      const u32 wbB = wb > A_BLOCKS ? wb - A_BLOCKS : 0;
      if (b < wbB) {
        m.base = (A_BLOCKS + b) * DB;
        m.cnt = min(DB, wlen - m.base);
        m.dense = 0;
        codes = P.segs[m.s].whc + m.base;
      } else {
        m.base = (b - wbB) * DB;
        m.cnt = min(DB, dlen - m.base);
        m.dense = 1;
        codes = P.segs[m.s].dhc + m.base;
      }
    }
    if (m.cnt) {
      fence_proxy_async();
      mbar_expect_tx(&S.bar[slot], m.cnt * 16u);
      bulk_g2s(buf, codes, m.cnt * 16u, &S.bar[slot]);
      m.copied = 1;
    }
  }
  S.meta[slot] = m;
}

template <int D>
__device__ void load_cand(const SegDesc& sd, u32 pos, bool valid, Cands& c, int r) {
  bool ok = valid && ld_cg_u8(sd.alive + pos);
  c.alive[r] = ok;
  c.was[r] = ok;
  c.pos[r] = pos;
  c.c[r] = ok ? __ldg(sd.hc + pos) : make_uint4(NEG_INF2, NEG_INF2, NEG_INF2, NEG_INF2);
}

// Phase A item: tile `tile` of the chunk against window block 0.
template <int D>
__device__ void item_a(const Params& P, const SegDesc& sd, SegState* cur, SegState* nxt, const Meta& mt,
                       const uint4* staged, u32 round, Shared& S) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const u32 DB = P.cfg.dom_block;
  const u32 s = mt.s, tgid = mt.tgid;
  SegState cs;
  cs.cur = ld_cg_u32(&cur[s].cur);
  cs.cend = ld_cg_u32(&cur[s].cend);
  cs.wlen = ld_cg_u32(&cur[s].wlen);
  cs.tiles = ld_cg_u32(&cur[s].tiles);
  const u32 cnt = mt.cnt;
  const u32 per_tile = max(1u, min(ceil_div(cs.wlen, DB), A_BLOCKS));
  const u32 gbase = cs.cur + mt.tile * TILE + warp * GS;

  if (cnt) {
    Cands c;
#pragma unroll
    for (int r = 0; r < R; ++r) {
      u32 pos = gbase + r * 32 + lane;
      load_cand<D>(sd, pos, pos < cs.cend, c, r);
    }
    if (__any_sync(FULL, any_alive(c))) {
      DomSrc src{sd.win, nullptr, 0};
      scan_smem<D>(staged, cnt, src, sd.pts, c);
#pragma unroll
      for (int r = 0; r < R; ++r)
        if (c.was[r] && !c.alive[r]) sd.alive[c.pos[r]] = 0;
    }
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    __threadfence();
    u32 old = atomicAdd(P.tdoneA + tgid, 1u);
    S.flag = (old == per_tile - 1);
    if (S.flag) P.tdoneA[tgid] = 0;
  }
  __syncthreads();
  if (!S.flag) return;
  __threadfence();
  // the tile's flags are final for phase A: compact its survivors
#pragma unroll
  for (int r = 0; r < R; ++r) {
    u32 pos = gbase + r * 32 + lane;
    bool a = pos < cs.cend && ld_cg_u8(sd.alive + pos);
    u32 m = __ballot_sync(FULL, a);
    u32 base = 0;
    if (lane == 0 && m) base = atomicAdd(&cur[s].dlen, (u32)__popc(m));
    base = __shfl_sync(FULL, base, 0);
    if (a) {
      u32 slot = base + __popc(m & ((1u << lane) - 1u));
      sd.dpos[slot] = pos;
      sd.dhc[slot] = __ldg(sd.hc + pos);
    }
  }
  __threadfence();
  fence_proxy_async();
  __syncthreads();
  if (threadIdx.x == 0) {
    u32 old = atomicAdd(&cur[s].done_a, 1u);
    if (old == cs.tiles - 1) {
      __threadfence();
      u32 dl = atomicAdd(&cur[s].dlen, 0u);
      if (dl == 0) {
        // nothing survived phase A: the next round starts now
        SegState nx;
        nx.cur = cs.cend;
        nx.wlen = ld_cg_u32(&cur[s].wlen);
        nx.wfill = nx.wlen;
        nx.rounds = ld_cg_u32(&cur[s].rounds) + 1;
        plan_round(sd, P.cfg, nx);
        nxt[s] = nx;
        if (nx.tiles == 0) P.done_round[s] = round + 1;
        atomicMax(P.ctl + C_MAXROUND, nx.rounds);
      }
    }
  }
}

// Phase B item: dense tile `dt` against window block A_BLOCKS + b, or dense
// block b - (window blocks of phase B).
template <int D>
__device__ void item_b(const Params& P, const SegDesc& sd, SegState* cur, SegState* nxt, const Meta& mt,
                       const uint4* staged, u32 round, Shared& S) {
  constexpr int V = vec_of(D);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const u32 DB = P.cfg.dom_block;
  const u32 s = mt.s, tgid = mt.tgid;
  SegState cs;
  cs.cur = ld_cg_u32(&cur[s].cur);
  cs.cend = ld_cg_u32(&cur[s].cend);
  cs.wlen = ld_cg_u32(&cur[s].wlen);
  cs.dlen = ld_cg_u32(&cur[s].dlen);
  cs.rounds = ld_cg_u32(&cur[s].rounds);
  const u32 wb = ceil_div(cs.wlen, DB);
  const u32 wbB = wb > A_BLOCKS ? wb - A_BLOCKS : 0;
  const u32 dtiles = ceil_div(cs.dlen, TILE);
  const u32 per_tile = wbB + ceil_div(cs.dlen, DB);
  const u32 dbase = mt.tile * TILE + warp * GS;
  const u32 cnt = mt.cnt;
  const DomSrc src = mt.dense ? DomSrc{sd.pts, sd.dpos, mt.base} : DomSrc{sd.win, nullptr, mt.base};
  Cands c;
#pragma unroll
  for (int r = 0; r < R; ++r) {
    u32 e = dbase + r * 32 + lane;
    bool valid = e < cs.dlen;
    u32 pos = valid ? __ldcg(sd.dpos + e) : 0;
    load_cand<D>(sd, pos, valid, c, r);
  }
  if (__any_sync(FULL, any_alive(c))) {
    scan_smem<D>(staged, cnt, src, sd.pts, c);
#pragma unroll
    for (int r = 0; r < R; ++r)
      if (c.was[r] && !c.alive[r]) sd.alive[c.pos[r]] = 0;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    __threadfence();
    u32 old = atomicAdd(P.tdoneB + tgid, 1u);
    S.flag = (old == per_tile - 1);
    if (S.flag) P.tdoneB[tgid] = 0;
  }
  __syncthreads();
  if (!S.flag) return;
  __threadfence();
  // the dense tile's flags are final: append its survivors to the window
#pragma unroll
  for (int r = 0; r < R; ++r) {
    u32 e = dbase + r * 32 + lane;
    u32 pos = e < cs.dlen ? __ldcg(sd.dpos + e) : 0;
    bool a = e < cs.dlen && ld_cg_u8(sd.alive + pos);
    u32 m = __ballot_sync(FULL, a);
    u32 base = 0;
    if (lane == 0 && m) base = atomicAdd(&cur[s].wfill, (u32)__popc(m));
    base = __shfl_sync(FULL, base, 0);
    if (a) {
      u32 slot = base + __popc(m & ((1u << lane) - 1u));
      const float4* src4 = sd.pts + (u64)pos * V;
      float4* dst4 = sd.win + (u64)slot * V;
#pragma unroll
      for (int v = 0; v < V; ++v) dst4[v] = __ldg(src4 + v);
      sd.whc[slot] = __ldg(sd.hc + pos);
    }
  }
  __threadfence();
  fence_proxy_async();
  __syncthreads();
  if (threadIdx.x == 0) {
    u32 old = atomicAdd(&cur[s].done_b, 1u);
    if (old == dtiles - 1) {
      __threadfence();
      SegState nx;
      nx.cur = cs.cend;
      nx.wlen = atomicAdd(&cur[s].wfill, 0u);
      nx.wfill = nx.wlen;
      nx.rounds = cs.rounds + 1;
      plan_round(sd, P.cfg, nx);
      nxt[s] = nx;
      if (nx.tiles == 0) P.done_round[s] = round + 1;
      atomicMax(P.ctl + C_MAXROUND, nx.rounds);
    }
  }
}

template <int D>
__device__ void run_item(int phase, const Params& P, const SegDesc& sd, SegState* cur, SegState* nxt, const Meta& m,
                         const uint4* staged, u32 round, Shared& S) {
  if (phase == 0) item_a<D>(P, sd, cur, nxt, m, staged, round, S);
  else item_b<D>(P, sd, cur, nxt, m, staged, round, S);
}

__global__ void __launch_bounds__(THREADS) k_engine(Params P) {
  extern __shared__ __align__(128) unsigned char dyn[];
  __shared__ Shared S;
  const u32 DB = P.cfg.dom_block;
  uint4* const buf0 = reinterpret_cast<uint4*>(dyn);  // two buffers of DB FP16 images
  u32* s_items = reinterpret_cast<u32*>(dyn + 2 * (size_t)DB * 16);  // nseg + 1
  u32* s_tiles = s_items + (P.nseg + 1);                             // nseg + 1
  const u32 nseg = P.nseg;

  if (threadIdx.x == 0) {
    mbar_init(&S.bar[0]);
    mbar_init(&S.bar[1]);
    S.bar_phase[0] = S.bar_phase[1] = 0;
    for (u32 s = blockIdx.x; s < nseg; s += gridDim.x) {
      SegState z;
      z.cur = 0;
      z.wlen = 0;
      z.wfill = 0;
      z.rounds = 0;
      plan_round(P.segs[s], P.cfg, z);
      P.st[s] = z;
      P.st[nseg + s] = z;
      P.done_round[s] = z.tiles ? 0xffffffffu : 0u;
    }
  }
  if (!grid_barrier(P.ctl, P.err)) return;

  for (u32 round = 0;; ++round) {
    SegState* cur = P.st + (round & 1) * nseg;
    SegState* nxt = P.st + ((round + 1) & 1) * nseg;
    for (int phase = 0; phase < 2; ++phase) {
      prefix_segments(P, cur, round, phase, s_items, s_tiles, S);
      const u32 total = s_items[nseg];
      if (phase == 0 && total == 0) return;  // every segment is done
      if (s_tiles[nseg] > P.tcap) {
        if (threadIdx.x == 0) {
          atomicOr(P.err, ERR_CAPACITY);
          atomicExch(P.ctl + C_ABORT, 1u);
        }
        return;
      }
      // the counter of the next phase is idle now: clear it
      if (blockIdx.x == 0 && threadIdx.x == 0) {
        if (phase == 0) P.ctl[C_B0 + (round & 1)] = 0;
        else P.ctl[C_A0 + ((round + 1) & 1)] = 0;
      }
      u32* counter = P.ctl + (phase == 0 ? C_A0 : C_B0) + (round & 1);
      // software pipeline: while the CTA scans item k from one buffer,
      // thread 0 has already taken item k + 1 and its bulk copy is filling
      // the other buffer
      if (threadIdx.x == 0) produce(P, phase, cur, s_items, s_tiles, total, counter, buf0, 0, S);
      __syncthreads();
      bool aborted = false;
      for (u32 k = 0;; ++k) {
        const int slot = k & 1;
        const Meta m = S.meta[slot];
        if (m.item >= total) break;
        if (m.copied && !mbar_wait(&S.bar[slot], S.bar_phase[slot], P.err, P.ctl)) {
          aborted = true;
          break;
        }
        __syncthreads();
        if (threadIdx.x == 0) {
          if (m.copied) S.bar_phase[slot] ^= 1u;
          produce(P, phase, cur, s_items, s_tiles, total, counter, buf0 + (size_t)(slot ^ 1) * DB, slot ^ 1, S);
        }
        const SegDesc sd = P.segs[m.s];
        const uint4* staged = buf0 + (size_t)slot * DB;
        switch (sd.d) {
          case 1: run_item<1>(phase, P, sd, cur, nxt, m, staged, round, S); break;
          case 2: run_item<2>(phase, P, sd, cur, nxt, m, staged, round, S); break;
          case 3: run_item<3>(phase, P, sd, cur, nxt, m, staged, round, S); break;
          case 4: run_item<4>(phase, P, sd, cur, nxt, m, staged, round, S); break;
          case 5: run_item<5>(phase, P, sd, cur, nxt, m, staged, round, S); break;
          case 6: run_item<6>(phase, P, sd, cur, nxt, m, staged, round, S); break;
          case 7: run_item<7>(phase, P, sd, cur, nxt, m, staged, round, S); break;
          default: run_item<8>(phase, P, sd, cur, nxt, m, staged, round, S); break;
        }
        if (threadIdx.x == 0) atomicAdd(P.ctl + C_PROGRESS, 1u);
        __syncthreads();
        if (ld_vol_u32(P.ctl + C_ABORT)) {
          aborted = true;
          // the copy of the prefetched item may still be in flight
          const Meta mn = S.meta[slot ^ 1];
          if (mn.item < total && mn.copied) mbar_wait(&S.bar[slot ^ 1], S.bar_phase[slot ^ 1], P.err, P.ctl);
          break;
        }
      }
      if (aborted) return;
      if (!grid_barrier(P.ctl, P.err)) return;
    }
  }
}

int g_sms = 0;

}  // namespace

u64 engine_tile_capacity(u64 total_points, u32 nseg) { return total_points / TILE + nseg + 1; }

cudaError_t engine_run(const SegDesc* segs_dev, u32 nseg, const EngineCfg& cfg, const EngineWork& w, u32* err,
                       cudaStream_t st) {
  if (nseg == 0) return cudaSuccess;
  if (nseg > MAX_SEG) {
    for (u32 s0 = 0; s0 < nseg; s0 += MAX_SEG) {
      cudaError_t e = engine_run(segs_dev + s0, std::min(MAX_SEG, nseg - s0), cfg, w, err, st);
      if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
  }
  if (cfg.dom_block == 0 || cfg.dom_block > DBMAX) return cudaErrorInvalidValue;
  Params P;
  P.segs = segs_dev;
  P.nseg = nseg;
  P.cfg = cfg;
  P.st = w.st;
  P.done_round = w.done_round;
  P.tdoneA = w.tdoneA;
  P.tdoneB = w.tdoneB;
  P.tcap = w.tcap;
  P.ctl = w.ctl;
  P.err = err;
  size_t smem = 2 * (size_t)cfg.dom_block * sizeof(uint4) + 2 * (size_t)(nseg + 1) * sizeof(u32);
  cudaError_t e = cudaFuncSetAttribute(k_engine, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  int per_sm = 0;
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_engine, THREADS, smem);
  if (e != cudaSuccess) return e;
  if (per_sm <= 0) return cudaErrorInvalidConfiguration;
  if (!g_sms) g_sms = device_sm_count();
  unsigned grid = (unsigned)(g_sms * per_sm);
  e = cudaMemsetAsync(w.ctl, 0, ENGINE_CTL_WORDS * sizeof(u32), st);
  if (e != cudaSuccess) return e;
  cudaLaunchConfig_t lc = {};
  lc.gridDim = dim3(grid);
  lc.blockDim = dim3(THREADS);
  lc.dynamicSmemBytes = smem;
  lc.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeCooperative;
  attr[0].val.cooperative = 1;
  lc.attrs = attr;
  lc.numAttrs = 1;
  note_launch();
  return cudaLaunchKernelEx(&lc, k_engine, P);
}

u32 engine_max_round_word() { return C_MAXROUND; }
u32 engine_max_dom_block() { return DBMAX; }

}  // namespace sky
