// Dominance kernels: the local-skyline engine (Algorithm 1, SFS, run on every
// partition of Algorithm 2 at once), the representative filter (Section 4.1)
// and the NoSeq final phase (Section 4.2).
//
// Exactness rests on one fact: t is outside Sky(r) iff some point of r
// dominates t, whether or not that point is itself in the skyline (a minimal
// dominator exists because dominance is a strict partial order on a finite
// set, and it is in the skyline).  So a candidate may be tested against any
// superset of its skyline dominators -- dead points included -- and the
// result is still exact.  Score order (f = attribute sum, monotone) bounds
// where the dominators can be: s < t implies f(s) <= f(t).
//
// SFS in rounds.  The points of a segment are sorted by f.  A round takes
// the next chunk of the segment (cut only between different scores) and
// tests every chunk point against (a) the window -- the skyline points of
// all earlier chunks, whose scores are strictly lower -- and (b) the chunk
// points with score <= its own.  A minimal dominator of a chunk point is in
// one of those two sets, so the chunk's survivors are exactly its skyline
// points, and they are appended to the window.
//
// Work decomposition.  A group is 32 * R consecutive chunk points held in
// the registers of one warp (R per lane).  A work item is (group, dominator
// block of DB points); items are numbered dominator-block-major so that
// early blocks (strongest window points) run first and later items find
// their candidates already dead.  Each item's warp scans its block with
// uniform loads, tests all R x 32 candidates per dominator with FP32
// compares, and exits as soon as a warp ballot shows every candidate dead.
// The last item to finish a group appends the group's survivors to the
// window; the last group of a segment sets up the segment's next round.
#include <algorithm>
#include <cstdio>
#include "sky_internal.cuh"

namespace sky {

namespace {

constexpr int WARPS = 8;
constexpr int THREADS = WARPS * 32;
constexpr int R = 2;             // candidates per lane
constexpr int GS = 32 * R;       // candidates per group
constexpr int IB = 4;            // items taken per atomic fetch
constexpr u32 MAX_SEG = 8192;    // segments per engine launch
constexpr u64 BARRIER_TIMEOUT_NS = 4000000000ull;

// control words
enum { C_ITEMS0 = 0, C_ITEMS1 = 1, C_BAR_COUNT = 2, C_BAR_GEN = 3, C_ABORT = 4, C_MAXROUND = 5,
       C_NOSEQ_ITEMS = 6, C_REL_ITEMS = 7 };

__device__ __forceinline__ u64 globaltimer() {
  u64 t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

__device__ __forceinline__ u32 ld_cg_u32(const u32* p) { return __ldcg(p); }
__device__ __forceinline__ u32 ld_vol_u32(const u32* p) { return *(const volatile u32*)p; }
__device__ __forceinline__ u8 ld_cg_u8(const u8* p) {
  return (u8)__ldcg(reinterpret_cast<const unsigned char*>(p));
}

// Grid-wide barrier of a cooperative launch (all blocks co-resident).  The
// wait is bounded: after BARRIER_TIMEOUT_NS it sets ERR_TIMEOUT and the abort
// word, and every block leaves the kernel at its next check.
__device__ bool grid_barrier(u32* ctl, u32* err) {
  __shared__ int s_ok;
  __syncthreads();
  if (threadIdx.x == 0) {
    u32 gen = ld_vol_u32(ctl + C_BAR_GEN);
    __threadfence();
    u32 arrived = atomicAdd(ctl + C_BAR_COUNT, 1u);
    bool ok = true;
    if (arrived == gridDim.x - 1) {
      atomicExch(ctl + C_BAR_COUNT, 0u);
      __threadfence();
      atomicAdd(ctl + C_BAR_GEN, 1u);
    } else {
      u64 t0 = globaltimer();
      while (ld_vol_u32(ctl + C_BAR_GEN) == gen) {
        if (ld_vol_u32(ctl + C_ABORT)) { ok = false; break; }
        if (globaltimer() - t0 > BARRIER_TIMEOUT_NS) {
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

// ------------------------------------------------------------ dominance scan

// Candidates of one lane: R points of D attributes.  A dead candidate's
// coordinates are set to -inf so that no dominator passes its "all <=" test.
template <int D>
struct Cand {
  float t[R][D];
  bool alive[R];
};

template <int D>
__device__ __forceinline__ void load_point(const float4* __restrict__ p, bool cg, float (&w)[8]) {
  float4 a = cg ? __ldcg(p) : __ldg(p);
  w[0] = a.x; w[1] = a.y; w[2] = a.z; w[3] = a.w;
  if (D > 4) {
    float4 b = cg ? __ldcg(p + 1) : __ldg(p + 1);
    w[4] = b.x; w[5] = b.y; w[6] = b.z; w[7] = b.w;
  } else {
    w[4] = w[5] = w[6] = w[7] = 0.0f;
  }
}

template <int D>
__device__ __forceinline__ bool all_le(const float (&w)[8], const float (&t)[D]) {
  bool le = true;
#pragma unroll
  for (int a = 0; a < D; ++a) le &= (w[a] <= t[a]);
  return le;
}

template <int D>
__device__ __forceinline__ bool any_ne(const float (&w)[8], const float (&t)[D]) {
  bool ne = false;
#pragma unroll
  for (int a = 0; a < D; ++a) ne |= (w[a] != t[a]);
  return ne;
}

// Tests the warp's candidates against dominators dom[0..cnt) (vec float4
// per point).  Returns when every candidate of the warp is dead or the block
// is exhausted.
template <int D>
__device__ __forceinline__ void scan_block(const float4* __restrict__ dom, u32 cnt, bool cg, Cand<D>& c) {
  constexpr int V = vec_of(D);
  constexpr int U = D <= 4 ? 8 : 4;
  for (u32 j = 0; j < cnt; j += U) {
    float w[U][8];
#pragma unroll
    for (int u = 0; u < U; ++u) {
      if (j + u < cnt) {
        load_point<D>(dom + (u64)(j + u) * V, cg, w[u]);
      } else {
#pragma unroll
        for (int a = 0; a < 8; ++a) w[u][a] = INFINITY;
      }
    }
    bool hit = false;
#pragma unroll
    for (int u = 0; u < U; ++u)
#pragma unroll
      for (int r = 0; r < R; ++r) hit |= all_le<D>(w[u], c.t[r]);
    if (hit) {
#pragma unroll
      for (int u = 0; u < U; ++u)
#pragma unroll
        for (int r = 0; r < R; ++r)
          if (c.alive[r] && j + u < cnt && all_le<D>(w[u], c.t[r]) && any_ne<D>(w[u], c.t[r])) {
            c.alive[r] = false;
#pragma unroll
            for (int a = 0; a < D; ++a) c.t[r][a] = -INFINITY;
          }
    }
    if ((j & (8 * U - 1)) == 8 * U - U) {
      bool any = false;
#pragma unroll
      for (int r = 0; r < R; ++r) any |= c.alive[r];
      if (!__any_sync(FULL, any)) break;
    }
  }
}

// Loads the group's candidates at positions base + r * 32 + lane < end.
template <int D>
__device__ __forceinline__ void load_cands(const float4* __restrict__ pts, const u8* alive, u32 base,
                                           u32 end, int lane, Cand<D>& c, bool (&was)[R]) {
  constexpr int V = vec_of(D);
#pragma unroll
  for (int r = 0; r < R; ++r) {
    u32 pos = base + r * 32 + lane;
    bool ok = pos < end && ld_cg_u8(alive + pos);
    c.alive[r] = ok;
    was[r] = ok;
    float w[8];
    if (ok) {
      load_point<D>(pts + (u64)pos * V, false, w);
#pragma unroll
      for (int a = 0; a < D; ++a) c.t[r][a] = w[a];
    } else {
#pragma unroll
      for (int a = 0; a < D; ++a) c.t[r][a] = -INFINITY;
    }
  }
}

template <int D>
__device__ __forceinline__ void store_kills(u8* alive, u32 base, int lane, const Cand<D>& c,
                                            const bool (&was)[R]) {
#pragma unroll
  for (int r = 0; r < R; ++r)
    if (was[r] && !c.alive[r]) alive[base + r * 32 + lane] = 0;
}

// First position >= from in [from, n) whose score exceeds v (scores sorted).
__device__ __forceinline__ u32 upper_bound_score(const float* __restrict__ score, u32 from, u32 n, float v) {
  u32 lo = from, hi = n;
  while (lo < hi) {
    u32 mid = lo + ((hi - lo) >> 1);
    if (__ldg(score + mid) <= v) lo = mid + 1;
    else hi = mid;
  }
  return lo;
}

// End of the chunk that starts at `start` with nominal length k: extended so
// that a run of equal scores is never split.
__device__ __forceinline__ u32 chunk_end(const SegDesc& sd, u32 start, u32 k) {
  u64 e = (u64)start + k;
  if (e >= sd.n) return sd.n;
  return upper_bound_score(sd.score, (u32)e, sd.n, __ldg(sd.score + e - 1));
}

__device__ __forceinline__ u32 ceil_div(u32 a, u32 b) { return (a + b - 1) / b; }

__device__ __forceinline__ void plan_round(const SegDesc& sd, const EngineCfg& cfg, SegState& s) {
  if (s.cur >= sd.n) {
    s.cend = sd.n;
    s.groups = 0;
    s.items = 0;
    return;
  }
  u64 k = ((u64)s.wlen * cfg.alpha_x4) / 4;
  k = k < cfg.chunk_min ? cfg.chunk_min : k;
  k = k > cfg.chunk_max ? cfg.chunk_max : k;
  s.cend = chunk_end(sd, s.cur, (u32)k);
  u32 len = s.cend - s.cur;
  s.groups = ceil_div(len, GS);
  s.items = s.groups * (ceil_div(s.wlen, cfg.dom_block) + ceil_div(len, cfg.dom_block));
}

// Block-wide exclusive scan of vals (n entries) into out[0..n]; out[n] = total.
__device__ void block_scan_to_smem(const SegState* st, const u32* done_round, u32 round, u32 n, bool groups,
                                   u32* out) {
  __shared__ u32 warp_tot[WARPS];
  __shared__ u32 carry;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  if (threadIdx.x == 0) carry = 0;
  __syncthreads();
  for (u32 base = 0; base < n; base += THREADS) {
    u32 i = base + threadIdx.x;
    u32 v = 0;
    // a segment that finished in an earlier round contributes nothing; one
    // that finishes during this round keeps its count until the round ends
    if (i < n && ld_cg_u32(done_round + i) > round)
      v = groups ? ld_cg_u32(&st[i].groups) : ld_cg_u32(&st[i].items);
    u32 x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      u32 y = __shfl_up_sync(FULL, x, o);
      if (lane >= o) x += y;
    }
    if (lane == 31) warp_tot[warp] = x;
    __syncthreads();
    u32 pre = carry;
    for (int w2 = 0; w2 < warp; ++w2) pre += warp_tot[w2];
    if (i < n) out[i] = pre + x - v;
    __syncthreads();
    if (threadIdx.x == THREADS - 1) carry = pre + x;
    __syncthreads();
  }
  if (threadIdx.x == 0) out[n] = carry;
  __syncthreads();
}

// ------------------------------------------------------------ engine

struct EngineParams {
  const SegDesc* segs;
  u32 nseg;
  EngineCfg cfg;
  SegState* st;       // 2 * nseg, alternating by round parity
  u32* done_round;    // nseg: first round in which the segment has no work
  u32* gdone;
  u64 gcap;
  u32* ctl;
  u32* err;
};

// One work item of the engine for segment sd: group g against dominator
// block b of this round.
template <int D>
__device__ void engine_item(const EngineParams& P, const SegDesc& sd, u32 s, const SegState& S, u32 b,
                            u32 g, u32 gid, SegState* cur, SegState* nxt, u32 round, int lane) {
  constexpr int V = vec_of(D);
  const u32 DB = P.cfg.dom_block;
  const u32 wblocks = ceil_div(S.wlen, DB);
  const u32 len = S.cend - S.cur;
  const u32 cblocks = ceil_div(len, DB);
  const u32 base = S.cur + g * GS;
  const u32 gend = min(base + GS, S.cend);

  Cand<D> c;
  bool was[R];
  load_cands<D>(sd.pts, sd.alive, base, gend, lane, c, was);
  bool any = false;
#pragma unroll
  for (int r = 0; r < R; ++r) any |= c.alive[r];
  if (__any_sync(FULL, any)) {
    if (b < wblocks) {
      u32 lo = b * DB;
      u32 cnt = min(DB, S.wlen - lo);
      scan_block<D>(sd.win + (u64)lo * V, cnt, true, c);
    } else {
      u32 lo = S.cur + (b - wblocks) * DB;
      // chunk dominators with score <= the group's largest score
      u32 hi = upper_bound_score(sd.score, gend - 1, S.cend, __ldg(sd.score + gend - 1));
      hi = min(hi, lo + DB);
      if (lo < hi) scan_block<D>(sd.pts + (u64)lo * V, hi - lo, false, c);
    }
    store_kills<D>(sd.alive, base, lane, c, was);
  }

  // completion of the group
  __syncwarp();
  u32 last = 0;
  if (lane == 0) {
    __threadfence();
    u32 old = atomicAdd(P.gdone + gid, 1u);
    last = (old == wblocks + cblocks - 1);
    if (last) P.gdone[gid] = 0;
  }
  last = __shfl_sync(FULL, last, 0);
  if (!last) return;
  __threadfence();
  // every item of the group is done: the flags are final
  bool surv[R];
  u32 cnt = 0;
#pragma unroll
  for (int r = 0; r < R; ++r) {
    u32 pos = base + r * 32 + lane;
    surv[r] = pos < gend && ld_cg_u8(sd.alive + pos);
    cnt += __popc(__ballot_sync(FULL, surv[r]));
  }
  u32 wbase = 0;
  if (lane == 0 && cnt) wbase = atomicAdd(&cur[s].wfill, cnt);
  wbase = __shfl_sync(FULL, wbase, 0);
  u32 off = 0;
#pragma unroll
  for (int r = 0; r < R; ++r) {
    u32 m = __ballot_sync(FULL, surv[r]);
    if (surv[r]) {
      u32 slot = wbase + off + __popc(m & ((1u << lane) - 1u));
      u32 pos = base + r * 32 + lane;
      const float4* src = sd.pts + (u64)pos * V;
      float4* dst = sd.win + (u64)slot * V;
#pragma unroll
      for (int v = 0; v < V; ++v) dst[v] = __ldg(src + v);
      if (sd.wpos) sd.wpos[slot] = pos;
    }
    off += __popc(m);
  }
  __threadfence();
  if (lane == 0) {
    u32 old = atomicAdd(&cur[s].done_groups, 1u);
    if (old == S.groups - 1) {
      // last group of the segment: plan the next round
      __threadfence();
      SegState nx;
      nx.cur = S.cend;
      nx.wlen = atomicAdd(&cur[s].wfill, 0u);
      nx.wfill = nx.wlen;
      nx.done_groups = 0;
      nx.rounds = S.rounds + 1;
      plan_round(sd, P.cfg, nx);
      nxt[s] = nx;
      if (nx.items == 0) P.done_round[s] = round + 1;
      atomicMax(P.ctl + C_MAXROUND, nx.rounds);
    }
  }
}

__global__ void __launch_bounds__(THREADS) k_engine(EngineParams P) {
  extern __shared__ u32 sh[];
  u32* s_items = sh;                  // nseg + 1
  u32* s_groups = sh + (P.nseg + 1);  // nseg + 1
  const int lane = threadIdx.x & 31;
  const u32 nseg = P.nseg;

  // round 0 plans
  if (threadIdx.x == 0) {
    for (u32 s = blockIdx.x; s < nseg; s += gridDim.x) {
      SegState z;
      z.cur = 0; z.wlen = 0; z.wfill = 0; z.done_groups = 0; z.rounds = 0;
      plan_round(P.segs[s], P.cfg, z);
      P.st[s] = z;
      SegState y = z;
      y.items = 0;
      y.groups = 0;
      P.st[nseg + s] = y;
      P.done_round[s] = z.items ? 0xffffffffu : 0u;
    }
  }
  if (!grid_barrier(P.ctl, P.err)) return;

  for (u32 round = 0;; ++round) {
    SegState* cur = P.st + (round & 1) * nseg;
    SegState* nxt = P.st + ((round + 1) & 1) * nseg;
    block_scan_to_smem(cur, P.done_round, round, nseg, false, s_items);
    block_scan_to_smem(cur, P.done_round, round, nseg, true, s_groups);
    const u32 total = s_items[nseg];
    if (total == 0) break;
    if (s_groups[nseg] > P.gcap) {
      if (threadIdx.x == 0) {
        atomicOr(P.err, ERR_CAPACITY);
        atomicExch(P.ctl + C_ABORT, 1u);
      }
      return;
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) P.ctl[(round + 1) & 1] = 0;
    u32* counter = P.ctl + (round & 1);
    for (;;) {
      u32 first = 0;
      if (lane == 0) first = atomicAdd(counter, (u32)IB);
      first = __shfl_sync(FULL, first, 0);
      if (first >= total) break;
      u32 lim = min(first + IB, total);
      for (u32 it = first; it < lim; ++it) {
        // segment of item `it`: last s with s_items[s] <= it
        u32 lo = 0, hi = nseg;
        while (hi - lo > 1) {
          u32 mid = (lo + hi) >> 1;
          if (s_items[mid] <= it) lo = mid;
          else hi = mid;
        }
        const u32 s = lo;
        const SegDesc sd = P.segs[s];
        SegState S;
        S.cur = ld_cg_u32(&cur[s].cur);
        S.cend = ld_cg_u32(&cur[s].cend);
        S.wlen = ld_cg_u32(&cur[s].wlen);
        S.groups = ld_cg_u32(&cur[s].groups);
        S.rounds = ld_cg_u32(&cur[s].rounds);
        u32 l = it - s_items[s];
        u32 b = l / S.groups, g = l % S.groups;
        u32 gid = s_groups[s] + g;
        switch (sd.d) {
          case 1: engine_item<1>(P, sd, s, S, b, g, gid, cur, nxt, round, lane); break;
          case 2: engine_item<2>(P, sd, s, S, b, g, gid, cur, nxt, round, lane); break;
          case 3: engine_item<3>(P, sd, s, S, b, g, gid, cur, nxt, round, lane); break;
          case 4: engine_item<4>(P, sd, s, S, b, g, gid, cur, nxt, round, lane); break;
          case 5: engine_item<5>(P, sd, s, S, b, g, gid, cur, nxt, round, lane); break;
          case 6: engine_item<6>(P, sd, s, S, b, g, gid, cur, nxt, round, lane); break;
          case 7: engine_item<7>(P, sd, s, S, b, g, gid, cur, nxt, round, lane); break;
          default: engine_item<8>(P, sd, s, S, b, g, gid, cur, nxt, round, lane); break;
        }
      }
    }
    if (!grid_barrier(P.ctl, P.err)) return;
  }
}

// ------------------------------------------------------------ relative skyline

// Kill every alive candidate dominated by one of dom[0..*nd) (the kept
// representatives).  One warp per group of GS candidates.
template <int D>
__global__ void __launch_bounds__(THREADS) k_relative(const float4* __restrict__ cand, u8* alive, u64 nc,
                                                      const float4* __restrict__ dom, u32 nd_host,
                                                      const u32* nd_dev) {
  const int lane = threadIdx.x & 31;
  const u64 group = (u64)blockIdx.x * WARPS + (threadIdx.x >> 5);
  const u64 base64 = group * GS;
  if (base64 >= nc) return;
  const u32 base = (u32)base64;
  const u32 end = (u32)(nc < base64 + GS ? nc : base64 + GS);
  Cand<D> c;
  bool was[R];
  load_cands<D>(cand, alive, base, end, lane, c, was);
  bool any = false;
#pragma unroll
  for (int r = 0; r < R; ++r) any |= c.alive[r];
  if (!__any_sync(FULL, any)) return;
  scan_block<D>(dom, nd_dev ? *nd_dev : nd_host, false, c);
  store_kills<D>(alive, base, lane, c, was);
}

// ------------------------------------------------------------ NoSeq

// pd_i membership (Section 4.2): Sliced j < i; Grid cell j componentwise <=
// cell i (weak grid dominance, j != i); Random / Angular / none: j != i.
__device__ __forceinline__ bool in_pd(const NoSeqArgs& a, u32 i, u32 j) {
  if (i == j) return false;
  if (a.scheme == SCHEME_SLICED) return j < i;
  if (a.scheme == SCHEME_GRID) {
    u32 ci = i, cj = j;
    for (int k = 0; k < a.d; ++k) {
      u32 m = a.gd.m[k];
      if (cj % m > ci % m) return false;
      ci /= m;
      cj /= m;
    }
    return true;
  }
  return true;
}

// Items: (group of u_i, dominator block of u).  gpre[P + 1]: prefix of the
// group counts per partition (computed on the device).
template <int D>
__global__ void __launch_bounds__(THREADS) k_noseq(NoSeqArgs a, const u32* __restrict__ gpre, const u32* nu_dev,
                                                   u32* ctl) {
  constexpr int V = vec_of(D);
  const int lane = threadIdx.x & 31;
  const u32 nu = *nu_dev;
  const u32 ngroups = gpre[a.P];
  const u32 DB = a.dom_block;
  const u32 nblocks = (nu + DB - 1) / DB;
  const u64 total = (u64)ngroups * nblocks;
  for (;;) {
    u32 first = 0;
    if (lane == 0) first = atomicAdd(ctl + C_NOSEQ_ITEMS, (u32)IB);
    first = __shfl_sync(FULL, first, 0);
    if (first >= total) break;
    u64 lim = (u64)first + IB < total ? (u64)first + IB : total;
    for (u64 it = first; it < lim; ++it) {
      u32 b = (u32)(it / ngroups), G = (u32)(it % ngroups);
      // partition i of global group G
      u32 lo = 0, hi = a.P;
      while (hi - lo > 1) {
        u32 mid = (lo + hi) >> 1;
        if (__ldg(gpre + mid) <= G) lo = mid;
        else hi = mid;
      }
      const u32 i = lo;
      const u32 ibeg = __ldg(a.useg + i), iend = __ldg(a.useg + i + 1);
      const u32 base = ibeg + (G - __ldg(gpre + i)) * GS;
      const u32 gend = min(base + GS, iend);
      const float fmax = __ldg(a.uscore + gend - 1);
      // dominator block [blo, bhi) of u; visit the partitions it overlaps
      const u32 blo = b * DB, bhi = min(blo + DB, nu);
      Cand<D> c;
      bool was[R];
      bool loaded = false;
      u32 pos = blo;
      while (pos < bhi) {
        // partition j holding u position pos
        u32 l2 = 0, h2 = a.P;
        while (h2 - l2 > 1) {
          u32 mid = (l2 + h2) >> 1;
          if (__ldg(a.useg + mid) <= pos) l2 = mid;
          else h2 = mid;
        }
        const u32 j = l2;
        const u32 jend = min(__ldg(a.useg + j + 1), bhi);
        if (in_pd(a, i, j)) {
          // u_j is sorted by score: only points with score <= fmax can dominate
          u32 cut = jend;
          {
            u32 lo3 = pos, hi3 = jend;
            while (lo3 < hi3) {
              u32 mid = lo3 + ((hi3 - lo3) >> 1);
              if (__ldg(a.uscore + mid) <= fmax) lo3 = mid + 1;
              else hi3 = mid;
            }
            cut = lo3;
          }
          if (cut > pos) {
            if (!loaded) {
              load_cands<D>(a.upts, a.ualive, base, gend, lane, c, was);
              loaded = true;
            }
            bool any = false;
#pragma unroll
            for (int r = 0; r < R; ++r) any |= c.alive[r];
            if (!__any_sync(FULL, any)) break;
            scan_block<D>(a.upts + (u64)pos * V, cut - pos, false, c);
          }
        }
        pos = jend;
      }
      if (loaded) store_kills<D>(a.ualive, base, lane, c, was);
    }
  }
}

__global__ void k_noseq_groups(const u32* __restrict__ useg, u32 P, u32* __restrict__ cnt) {
  u64 i = (u64)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < P) cnt[i] = (useg[i + 1] - useg[i] + GS - 1) / GS;
}

// Segment descriptors of the local phase from the partition offsets;
// partitions removed by Grid Filtering get no work.
__global__ void k_build_segs(const u32* __restrict__ seg_off, u32 P, const u8* __restrict__ dropped,
                             const float4* pts, const float* score, u8* alive, float4* win, u32* wpos,
                             int d, SegDesc* segs) {
  u64 s = (u64)blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= P) return;
  const int V = vec_of(d);
  u32 o = seg_off[s];
  SegDesc sd;
  sd.pts = pts + (u64)o * V;
  sd.score = score + o;
  sd.alive = alive + o;
  sd.win = win + (u64)o * V;
  sd.wpos = wpos ? wpos + o : nullptr;
  sd.n = (dropped && dropped[s]) ? 0u : seg_off[s + 1] - o;
  sd.d = (u32)d;
  segs[s] = sd;
}

__global__ void k_build_one_seg(const float4* pts, const float* score, u8* alive, float4* win,
                                const u32* n_dev, int d, SegDesc* seg) {
  SegDesc sd;
  sd.pts = pts;
  sd.score = score;
  sd.alive = alive;
  sd.win = win;
  sd.wpos = nullptr;
  sd.n = *n_dev;
  sd.d = (u32)d;
  *seg = sd;
}

__global__ void k_fold_max(const u32* src, u32* dst) { atomicMax(dst, *src); }

int g_sm_count = 0;

}  // namespace

cudaError_t launch_build_segs(const u32* seg_off, u32 P, const u8* dropped, const float* pts, const float* score,
                              u8* alive, float* win, u32* wpos, int d, SegDesc* segs, cudaStream_t st) {
  if (P == 0) return cudaSuccess;
  note_launch();
  k_build_segs<<<(P + 255) / 256, 256, 0, st>>>(seg_off, P, dropped, reinterpret_cast<const float4*>(pts), score,
                                                alive, reinterpret_cast<float4*>(win), wpos, d, segs);
  return cudaGetLastError();
}

cudaError_t launch_build_one_seg(const float* pts, const float* score, u8* alive, float* win, const u32* n_dev,
                                 int d, SegDesc* seg, cudaStream_t st) {
  note_launch();
  k_build_one_seg<<<1, 1, 0, st>>>(reinterpret_cast<const float4*>(pts), score, alive,
                                   reinterpret_cast<float4*>(win), n_dev, d, seg);
  return cudaGetLastError();
}

cudaError_t launch_fold_max(const u32* ctl, u32* dst, cudaStream_t st) {
  note_launch();
  k_fold_max<<<1, 1, 0, st>>>(ctl + C_MAXROUND, dst);
  return cudaGetLastError();
}

int device_sm_count() {
  int dev = 0;
  cudaGetDevice(&dev);
  int n = 0;
  cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
  g_sm_count = n;
  return n;
}

u64 engine_group_capacity(u64 total_points, u32 nseg) { return total_points / GS + nseg + 1; }

cudaError_t engine_run(const SegDesc* segs_dev, u32 nseg, u32 max_vec, const EngineCfg& cfg,
                       const EngineWork& w, u32* err, cudaStream_t st) {
  (void)max_vec;
  if (nseg == 0) return cudaSuccess;
  if (nseg > MAX_SEG) {
    // more segments than one launch's shared-memory prefix holds: batches
    for (u32 s0 = 0; s0 < nseg; s0 += MAX_SEG) {
      cudaError_t e = engine_run(segs_dev + s0, std::min(MAX_SEG, nseg - s0), max_vec, cfg, w, err, st);
      if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
  }
  EngineParams P;
  P.segs = segs_dev;
  P.nseg = nseg;
  P.cfg = cfg;
  P.st = w.st;
  P.done_round = w.done_round;
  P.gdone = w.gdone;
  P.gcap = w.gcap;
  P.ctl = w.ctl;
  P.err = err;
  size_t smem = 2 * (size_t)(nseg + 1) * sizeof(u32);
  cudaError_t e = cudaFuncSetAttribute(k_engine, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  int per_sm = 0;
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_engine, THREADS, smem);
  if (e != cudaSuccess) return e;
  if (per_sm <= 0) return cudaErrorInvalidConfiguration;
  int sms = g_sm_count ? g_sm_count : device_sm_count();
  unsigned grid = (unsigned)(sms * per_sm);
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

cudaError_t launch_relative(const float* cand, u8* alive, u64 nc, const float* dom, u32 nd_host,
                            const u32* nd_dev, int d, cudaStream_t st) {
  if (nc == 0) return cudaSuccess;
  u64 groups = (nc + GS - 1) / GS;
  unsigned grid = (unsigned)((groups + WARPS - 1) / WARPS);
  return dispatch_d(d, [&](auto D) {
    note_launch();
    k_relative<decltype(D)::value><<<grid, THREADS, 0, st>>>(reinterpret_cast<const float4*>(cand), alive, nc,
                                                             reinterpret_cast<const float4*>(dom), nd_host, nd_dev);
  });
}

cudaError_t launch_noseq(const NoSeqArgs& a, u32* gcnt, u32* gpre, u32* scan_tmp, const u32* nu_dev, u32* ctl,
                         cudaStream_t st) {
  if (a.P == 0) return cudaSuccess;
  note_launch();
  k_noseq_groups<<<(a.P + 255) / 256, 256, 0, st>>>(a.useg, a.P, gcnt);
  cudaError_t e = scan_u32(gcnt, gpre, a.P, true, false, scan_tmp, st);
  if (e != cudaSuccess) return e;
  // gpre[P] = total groups
  e = cudaMemcpyAsync(gpre + a.P, scan_tmp + scan_total_index(a.P), sizeof(u32), cudaMemcpyDeviceToDevice, st);
  if (e != cudaSuccess) return e;
  e = cudaMemsetAsync(ctl + C_NOSEQ_ITEMS, 0, sizeof(u32), st);
  if (e != cudaSuccess) return e;
  int sms = g_sm_count ? g_sm_count : device_sm_count();
  return dispatch_d(a.d, [&](auto D) {
    int per_sm = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_noseq<decltype(D)::value>, THREADS, 0);
    if (per_sm <= 0) per_sm = 1;
    note_launch();
    k_noseq<decltype(D)::value><<<(unsigned)(sms * per_sm), THREADS, 0, st>>>(a, gpre, nu_dev, ctl);
  });
}

}  // namespace sky
