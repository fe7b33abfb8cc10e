// Local-skyline engine: Algorithm 1 (SFS) run on every partition of
// Algorithm 2 -- of every query of a batch -- at once, in one persistent
// launch driven by a device-side work queue.
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
// two phases:
//   A. every chunk point is tested against the first window block (the
//      strongest, lowest-score skyline points); the survivors of each tile of
//      the chunk are compacted into the segment's dense list;
//   B. every dense-list point is tested against the rest of the window and
//      against the dense-list points of lower or equal score (a chunk
//      dominator killed in phase A was itself dominated by a window point
//      that also dominates the candidate, so the dense list holds every chunk
//      dominator that matters); the survivors are appended to the window.
// When the dense list is kept in position (= score) order, phase B tests a
// dense tile only against the dense entries up to its end (extended over a
// run of equal scores), half of the square.  The merge (and a local phase
// of few segments) keeps the order by decoupled look-back: each tile writes
// its survivors at the sum of its predecessors' counts.  The look-back makes
// a tile wait for the scans of the tiles before it, which pays off for large
// chunks but blocks CTAs when many small segments interleave, so a local
// phase of many segments keeps the order differently: its phase-A tiles
// only count, and the phase's last tile compacts the whole chunk in order.
// One CTA does that pass, so a round whose chunk is long falls back to
// arrival order and tests the whole dense square.
//
// Work queue.  Segments advance through their rounds independently; there
// is no grid-wide barrier.  A phase of a segment is a task of items (tile of
// WARPS warps x 32 lanes x R candidates, dominator block of DB points, numbered
// block-major so the strongest window points run first).  Publishing a task
// reserves a contiguous range of tickets with one 64-bit atomic (task index
// and ticket range together, so both orders agree) and then marks the task
// valid.  A CTA claims tickets one at a time and finds the task of its
// ticket by a galloping search from the task of its previous ticket.  The
// CTA that completes the last tile of a phase publishes the segment's next
// phase (or its next round's phase A, or finishes the segment); when the
// last segment finishes, the CTAs still waiting for tickets leave.
// Segments of different sizes and queries of a batch thus overlap freely,
// and a segment's long phase never holds up the others.
//
// Dominance test.  Every point carries, next to its FP32 attributes, their
// 16-bit images packed two per 32-bit word: the round-down FP16 values, or
// the rank codes of sky_rank.cu (finite non-negative FP16 bit patterns).
// Both are non-decreasing in the value, so if any image of w exceeds t's,
// then w exceeds t in that attribute and cannot dominate t: the FP16 test
// (the signs of f16x2 differences; a
// candidate's images are duplicated per word and staged dominators come in
// pairs, so one subtraction tests one attribute of two pairs) rejects
// exactly, and only pairs it passes are tested in FP32 (Def. 1).  A warp
// compacts its live candidates into fewer slots per lane as they die, so
// dead lanes stop costing tests.
//
// Pipeline.  The first warp to finish its part of the current item claims
// the next item (while the other warps still scan) and starts the bulk copy
// (cp.async.bulk, completing on an mbarrier) of the next item's dominator
// block into the second of two shared-memory buffers; each warp scans the
// staged block with broadcast
// shared loads and leaves the item when a ballot shows all its candidates
// dead.  Every wait (mbarrier, waiting for a ticket's task) is bounded: it
// gives up with ERR_TIMEOUT when no item anywhere has completed for WAIT_NS
// (a launch may set a shorter limit: EngineCfg::wait_ns).
//
// This file is the engine's implementation for one launch shape: it is
// included by one translation unit per shape (sky_engine_w<W>r<R>.cu), which
// defines SKY_ENGINE_WARPS (warps per CTA) and SKY_ENGINE_R (candidates per
// lane) first; sky_engine.cu dispatches a launch to the shape its EngineCfg
// asks for.
#include <algorithm>
#include "sky_internal.cuh"

#if !defined(SKY_ENGINE_WARPS) || !defined(SKY_ENGINE_R)
#error "define SKY_ENGINE_WARPS and SKY_ENGINE_R before including sky_engine_impl.cuh"
#endif

namespace sky {

namespace {

// Warps per CTA and candidates per lane of this launch shape.  The default
// (4 warps, 4 candidates) runs four 128-thread CTAs per SM: an item ends when
// its slowest warp has scanned its candidates, and four CTAs of four warps
// per SM lose less to that wait than two CTAs of eight (measured 484 vs 462
// M points/s on the benchmark's batch with the default knobs).  Two
// candidates per lane halve the tile, for segments too small to fill the
// GPU with 512-candidate tiles.  The autotuner picks among the shapes.
constexpr int WARPS = SKY_ENGINE_WARPS;
constexpr int THREADS = WARPS * 32;
constexpr int R = SKY_ENGINE_R;         // candidates per lane
static_assert((WARPS == 4 || WARPS == 8) && (R == 2 || R == 4), "compiled engine shapes");
static_assert(WARPS * 32 * R >= ENGINE_MIN_TILE, "tile capacity is sized for the smallest tile");
constexpr int GS = 32 * R;              // candidates per warp
constexpr int TILE = WARPS * GS;        // candidates per tile (CTA item)
constexpr u32 DBMAX = 2048;             // dominator block capacity (points)
// Window blocks of phase A.  Must stay 1 while merges use the ordered
// compaction: a tile's look-back runs in the item that completes the tile,
// and only with one phase-A item per tile is that item's ticket above every
// item of the tiles before it, so the CTAs it waits for never wait for it.
constexpr u32 A_BLOCKS = 1;
constexpr u64 WAIT_NS = 4000000000ull;  // default bound of every wait (without progress)

// Control words of a launch (zeroed by the host before it).  The queue word
// is 64-bit: (tasks published << 32) | tickets reserved.
enum { C_TICKET = 0, C_QUEUE = 2, C_LIVE = 4, C_FINISHED = 5, C_ABORT = 6, C_MAXROUND = 7, C_PROGRESS = 8,
       C_TESTS = 10 /* u64: the launch's FP16 tests */ };

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
__device__ bool mbar_wait(u64* bar, u32 parity, u64 limit_ns, u32* err, u32* ctl) {
  if (mbar_try_wait(bar, parity)) return true;
  u64 t0 = globaltimer();
  while (!mbar_try_wait(bar, parity)) {
    if (globaltimer() - t0 > limit_ns) {
      atomicOr(err, ERR_TIMEOUT);
      atomicExch(ctl + C_ABORT, 1u);
      return false;
    }
  }
  return true;
}
// Generic-proxy writes of global memory made visible to later bulk copies.
__device__ __forceinline__ void fence_proxy_async() { asm volatile("fence.proxy.async.global;" ::: "memory"); }
// A thread's generic-proxy reads of a staging buffer ordered before the
// async-proxy writes of a later bulk copy into the same buffer (issued by
// one thread after a CTA barrier that every reader has passed).
__device__ __forceinline__ void fence_proxy_async_smem() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}


// ------------------------------------------------------------ dominance test

template <int D>
struct HW {
  static constexpr int value = (D + 1) / 2;  // half2 words that hold D attributes
};

// Sign bits of t - w per FP16 half, ORed over the image words: bit 15 / 31
// is clear iff every attribute of the low / high halves has w <= t.  The
// subtraction's sign is exact: t - w rounds to a value of the sign of the
// exact difference (a nonzero difference of two FP16 numbers is at least
// the smallest subnormal, so it never rounds to zero), t - t is +0, the
// images are finite and never -0, and overflow keeps the sign; a dead
// candidate (-inf) or a padding dominator (+inf) gives -inf.
__device__ __forceinline__ u32 hsub2_bits(u32 t, u32 w) {
  u32 r;
  asm("sub.rn.f16x2 %0, %1, %2;" : "=r"(r) : "r"(t), "r"(w));
  return r;
}
// A candidate's images are kept duplicated, word k = (image k, image k); a
// staged dominator pair is kept as word k = (image k of the first, image k
// of the second).  One f16x2 subtraction per attribute then tests the
// candidate against both dominators: bit 15 / 31 of the OR over the
// attributes is clear iff every attribute of the first / second dominator
// is <= the candidate's (the FP16 part of Def. 1's first condition).
template <int D>
__device__ __forceinline__ u32 pair_fail(const u32 (&t)[D], const u32 (&w)[D]) {
  u32 x = hsub2_bits(t[0], w[0]);
#pragma unroll
  for (int k = 1; k < D; ++k) x |= hsub2_bits(t[k], w[k]);
  return x;
}

// Packed images (two attributes per word, attribute 2i in the low half) to
// duplicated words and back.
template <int D>
__device__ __forceinline__ void unpack_dup(const uint4& p, u32 (&t)[D]) {
  const u32 w[4] = {p.x, p.y, p.z, p.w};
#pragma unroll
  for (int k = 0; k < D; ++k) t[k] = __byte_perm(w[k / 2], 0u, (k & 1) ? 0x3232u : 0x1010u);
}
template <int D>
__device__ __forceinline__ uint4 pack_dup(const u32 (&t)[D]) {
  u32 w[4];
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const u32 lo = 2 * i < D ? t[2 * i] : 0u, hi = 2 * i + 1 < D ? t[2 * i + 1] : 0u;
    w[i] = __byte_perm(lo, hi, 0x5410u);
  }
  return make_uint4(w[0], w[1], w[2], w[3]);
}

// Window and dense-list images are stored as pairs: entries 2i and 2i+1
// share 32 bytes (two uint4), word k = (image k of entry 2i, image k of
// entry 2i+1), so a bulk copy of a block lands in shared memory as the
// dominator pairs the scan tests.  Writes entry j's D images (two-byte
// stores into its half of the pair's words).
template <int D>
__device__ __forceinline__ void put_pair_entry(uint4* arr, u32 j, const uint4& packed) {
  unsigned short* h = reinterpret_cast<unsigned short*>(arr) + (size_t)(j >> 1) * 16 + (j & 1);
  const u32 w[4] = {packed.x, packed.y, packed.z, packed.w};
#pragma unroll
  for (int k = 0; k < D; ++k) h[2 * k] = (unsigned short)((k & 1) ? (w[k / 2] >> 16) : (w[k / 2] & 0xffffu));
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

// Staging buffer entries beyond dom_block: a scan step may read past a
// block's last entry up to the next multiple of 8 (blocks hold at most
// dom_block entries, a multiple of 32).
constexpr u32 STAGE_PAD = 4;
constexpr u32 NEG_INF2 = 0xFC00FC00u;  // (-inf, -inf)

// The candidates of one lane: RR slots (R when an item starts; fewer once
// the warp's live candidates have been compacted).
template <int D, int RR>
struct CandsT {
  u32 t[RR][D];   // duplicated FP16 images (-inf when dead)
  u32 pos[RR];    // segment-relative position
  bool alive[RR];
  bool was[RR];
};

template <int D>
__device__ __forceinline__ void set_dead(u32 (&t)[D]) {
#pragma unroll
  for (int k = 0; k < D; ++k) t[k] = NEG_INF2;
}

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

template <int D, int RR>
__device__ __forceinline__ u32 alive_count(const CandsT<D, RR>& c) {
  u32 n = 0;
#pragma unroll
  for (int r = 0; r < RR; ++r) n += __popc(__ballot_sync(FULL, c.alive[r]));
  return n;
}

// Records the warp's kills (candidates alive at load, dead now).
template <int D, int RR>
__device__ __forceinline__ void write_kills(const CandsT<D, RR>& c, u8* alive) {
#pragma unroll
  for (int r = 0; r < RR; ++r)
    if (c.was[r] && !c.alive[r]) alive[c.pos[r]] = 0;
}

// Moves the warp's live candidates (at most 32 x RB of them) into RB slots
// per lane, in slot-major order, through the warp's shared scratch; kills
// are recorded first.
template <int D, int RA, int RB>
__device__ __forceinline__ void compact(const CandsT<D, RA>& a, CandsT<D, RB>& b, uint4* sc, u32* sp, u8* alive) {
  const int lane = threadIdx.x & 31;
  const u32 lt = (1u << lane) - 1u;
  write_kills(a, alive);
  u32 k0 = 0;
#pragma unroll
  for (int r = 0; r < RA; ++r) {
    const u32 m = __ballot_sync(FULL, a.alive[r]);
    if (a.alive[r]) {
      const u32 k = k0 + __popc(m & lt);
      sc[k] = pack_dup<D>(a.t[r]);
      sp[k] = a.pos[r];
    }
    k0 += __popc(m);
  }
  __syncwarp();
#pragma unroll
  for (int r = 0; r < RB; ++r) {
    const u32 k = r * 32 + lane;
    const bool v = k < k0;
    b.alive[r] = v;
    b.was[r] = v;
    if (v) {
      unpack_dup<D>(sc[k], b.t[r]);
    } else {
      set_dead<D>(b.t[r]);
    }
    b.pos[r] = v ? sp[k] : 0u;
  }
  __syncwarp();
}

// Dominance tests of a CTA (shared memory), added to the launch's total
// when the CTA leaves: candidate slots x dominators the FP16 test covered
// (dead slots included).  Counted per scan call, outside the scan loop.
struct EngineCounts {
  unsigned long long n16;
};

__device__ __forceinline__ void count_fp16(EngineCounts* k, u32 j0, u32 j1, u32 cnt, u32 slots) {
  const u32 e = j1 < cnt ? j1 : cnt;
  if ((threadIdx.x & 31) == 0 && e > j0) atomicAdd(&k->n16, (unsigned long long)(e - j0) * 32ull * slots);
}

// Scans the staged block sb[j..cnt) (dominator pairs, see put_pair_entry) for
// the warp's candidates, RR slots per lane.  Every 32 dominators the warp
// counts its live candidates; it stops early when none is left or when they
// fit in half the slots (the caller compacts them and goes on with fewer
// slots, so dead lanes stop costing compares).  Returns the position
// reached; *n_alive = live candidates.
template <int D, int RR>
__device__ __forceinline__ u32 scan_steps(const uint4* sb, u32 j, u32 cnt, const DomSrc& src, const float4* pts,
                                          CandsT<D, RR>& c, u32* n_alive) {
  constexpr int V = vec_of(D);
  // dominator pairs per step: more with fewer candidate slots (the step's
  // fixed cost is spread over more tests); the kernel needs 120 registers,
  // within the budget of four 128-thread CTAs per SM
  constexpr int UP = 2 * (RR == 1 ? 2 : 1);
  // the last step may read pairs past the block's end (whatever the
  // buffer held): the FP32 path checks the bound, so a spurious pass there
  // costs time only
  while (j < cnt) {
    u32 w[UP][D];
#pragma unroll
    for (int q = 0; q < UP; ++q) {
      const uint4 a = sb[j + 2 * q];
      w[q][0] = a.x;
      if (D > 1) w[q][1 < D ? 1 : 0] = a.y;
      if (D > 2) w[q][2 < D ? 2 : 0] = a.z;
      if (D > 3) w[q][3 < D ? 3 : 0] = a.w;
      if (D > 4) {
        const uint4 b = sb[j + 2 * q + 1];
        w[q][4 < D ? 4 : 0] = b.x;
        if (D > 5) w[q][5 < D ? 5 : 0] = b.y;
        if (D > 6) w[q][6 < D ? 6 : 0] = b.z;
        if (D > 7) w[q][7 < D ? 7 : 0] = b.w;
      }
    }
    // fast rejection: acc keeps bits 15 and 31 set while every candidate
    // fails against both dominators of every pair of the step, and clears
    // one for every (candidate, dominator) that the exact FP16 test passes
    u32 acc = 0xffffffffu;
#pragma unroll
    for (int q = 0; q < UP; ++q)
#pragma unroll
      for (int r = 0; r < RR; ++r) acc &= pair_fail<D>(c.t[r], w[q]);
    if ((acc & 0x80008000u) != 0x80008000u) {
#pragma unroll
      for (int q = 0; q < UP; ++q)
#pragma unroll
        for (int r = 0; r < RR; ++r) {
          const u32 x = pair_fail<D>(c.t[r], w[q]);
#pragma unroll
          for (int h = 0; h < 2; ++h) {
            const u32 jd = j + 2 * q + h;
            if (c.alive[r] && !((x >> (15 + 16 * h)) & 1u) && jd < cnt) {
              // for window dominators the FP32 copy may have been written
              // in an earlier round by another SM: read it through L2
              const float4* wp = dom_fp32<D>(src, jd);
              float4 wv[2], tv[2];
              wv[0] = __ldcg(wp);
              tv[0] = __ldg(pts + (u64)c.pos[r] * V);
              if (V > 1) {
                wv[1] = __ldcg(wp + 1);
                tv[1] = __ldg(pts + (u64)c.pos[r] * V + 1);
              }
              if (dominates_fp32<D>(wv, tv)) {
                c.alive[r] = false;
                set_dead<D>(c.t[r]);
              }
            }
          }
        }
    }
    j += 2 * UP;
    if ((j & 31) == 0) {
      const u32 n = alive_count(c);
      if (n == 0 || (RR > 1 && n <= 32u * (RR / 2))) {
        *n_alive = n;
        return j;
      }
    }
  }
  *n_alive = alive_count(c);
  return j;
}

// Scans the staged block sb[0..cnt) for the warp's candidates and records
// their kills in `alive`.  Starts with R slots per lane and compacts the
// live candidates into 2, then 1, slot as they die; sc/sp are the warp's
// shared scratch (GS entries).
template <int D>
__device__ __forceinline__ void scan_smem(const uint4* sb, u32 cnt, const DomSrc& src, const float4* pts,
                                          CandsT<D, R>& c,
                                          uint4* sc, u32* sp, u8* alive, EngineCounts* k) {
  u32 n = alive_count(c);
  u32 j = 0;
  if constexpr (R == 2) {
    // 2 slots per lane, then 1
    if (n > 32) {
      j = scan_steps<D, 2>(sb, 0, cnt, src, pts, c, &n);
      count_fp16(k, 0, j, cnt, 2);
      if (j >= cnt || n == 0) {
        write_kills(c, alive);
        return;
      }
    }
    CandsT<D, 1> c1;
    compact(c, c1, sc, sp, alive);
    if (n == 0) return;
    count_fp16(k, j, scan_steps<D, 1>(sb, j, cnt, src, pts, c1, &n), cnt, 1);
    write_kills(c1, alive);
  } else {
    // 4 slots per lane, then 2, then 1
    if (n > 64) {
      j = scan_steps<D, 4>(sb, 0, cnt, src, pts, c, &n);
      count_fp16(k, 0, j, cnt, 4);
      if (j >= cnt || n == 0) {
        write_kills(c, alive);
        return;
      }
    }
    CandsT<D, 1> c1;
    if (n > 32) {
      CandsT<D, 2> c2;
      compact(c, c2, sc, sp, alive);
      const u32 j2 = scan_steps<D, 2>(sb, j, cnt, src, pts, c2, &n);
      count_fp16(k, j, j2, cnt, 2);
      j = j2;
      if (j >= cnt || n == 0) {
        write_kills(c2, alive);
        return;
      }
      compact(c2, c1, sc, sp, alive);
    } else {
      compact(c, c1, sc, sp, alive);
      if (n == 0) return;
    }
    count_fp16(k, j, scan_steps<D, 1>(sb, j, cnt, src, pts, c1, &n), cnt, 1);
    write_kills(c1, alive);
  }
}

template <int D>
__device__ __forceinline__ bool any_alive(const CandsT<D, R>& c) {
  bool a = false;
#pragma unroll
  for (int r = 0; r < R; ++r) a |= c.alive[r];
  return a;
}

__device__ __forceinline__ u32 ceil_div(u32 a, u32 b) { return (a + b - 1) / b; }

// ------------------------------------------------------------ work queue

struct Task {
  u64 tv;       // (first ticket << 32) | 1, written last (release); 0 until published
  u32 s;        // segment
  u32 phase;    // 0: A, 1: B
  u32 tiles;    // candidate tiles of the phase
  u32 items;    // work items (tiles x dominator blocks)
  u32 pad[2];
};

__device__ __forceinline__ u64 ld_acquire_u64(const u64* p) {
  u64 v;
  asm volatile("ld.acquire.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ void st_release_u64(u64* p, u64 v) {
  asm volatile("st.release.gpu.global.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}

struct Params {
  const SegDesc* segs;
  u32 nseg;
  EngineCfg cfg;
  SegState* st;    // nseg
  u32* tbase;      // nseg: first completion counter of each segment
  u32* tdoneA;     // completion counters of phase-A tiles (capacity tcap)
  u32* tdoneB;     // completion counters of phase-B tiles (capacity tcap)
  u32* tstat;      // phase-A tile status for the ordered compaction (capacity tcap)
  u64 tcap;
  Task* tasks;     // task_cap entries, valid flags zero before the launch
  u32 task_cap;
  u32* ctl;
  u32* err;
  u64 wait_ns;     // bound of every wait without progress
};

__device__ __forceinline__ void abort_launch(const Params& P, u32 code) {
  atomicOr(P.err, code);
  atomicExch(P.ctl + C_ABORT, 1u);
}

__device__ __forceinline__ u32 upper_bound_score(const float* __restrict__ score, u32 from, u32 n, float v) {
  u32 lo = from, hi = n;
  while (lo < hi) {
    u32 mid = lo + ((hi - lo) >> 1);
    if (__ldg(score + mid) <= v) lo = mid + 1;
    else hi = mid;
  }
  return lo;
}

// Next chunk of a segment: nominal length alpha/4 x the window size, and at
// least an eighth of the points already processed (so a segment whose window
// stays small still needs only logarithmically many rounds), clamped, then
// extended to the end of a run of equal scores.
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
  if (k < s.cur / 8) k = s.cur / 8;
  k = k < cfg.chunk_min ? cfg.chunk_min : k;
  k = k > cfg.chunk_max ? cfg.chunk_max : k;
  u64 e = (u64)s.cur + k;
  if (e >= sd.n) s.cend = sd.n;
  else s.cend = upper_bound_score(sd.score, (u32)e, sd.n, __ldg(sd.score + e - 1));
  s.tiles = ceil_div(s.cend - s.cur, TILE);
}

// How the round whose chunk is [cur, cend) builds its dense list: the
// launch's mode, except that ORD_LAST falls back to arrival order for a
// chunk longer than ORD_LAST_MAX (one CTA would compact it alone).
__device__ __forceinline__ u32 round_ord(const EngineCfg& cfg, u32 cur, u32 cend) {
  return cfg.ordered == ORD_LAST && cend - cur > ORD_LAST_MAX ? ORD_NONE : cfg.ordered;
}

// Publishes a task (one thread).  The 64-bit atomic reserves the task index
// and its ticket range together.
__device__ void publish(const Params& P, u32 s, u32 phase, u32 tiles, u32 items) {
  unsigned long long* q = reinterpret_cast<unsigned long long*>(P.ctl + C_QUEUE);
  const u64 old = atomicAdd(q, (1ull << 32) | (u64)items);
  const u32 idx = (u32)(old >> 32), t0 = (u32)old;
  if (idx >= P.task_cap || (u64)t0 + items >= 0xffff0000ull) {
    abort_launch(P, ERR_CAPACITY);
    return;
  }
  // test hook (EngineCfg::withhold_task): the task keeps its tickets but is
  // never marked published, so the CTAs that draw them wait until the
  // bounded wait gives up
  if (P.cfg.withhold_task && idx + 1 == P.cfg.withhold_task) return;
  Task* t = P.tasks + idx;
  t->s = s;
  t->phase = phase;
  t->tiles = tiles;
  t->items = items;
  __threadfence();
  st_release_u64(&t->tv, ((u64)t0 << 32) | 1ull);
}

__device__ void finish_segment(const Params& P) {
  __threadfence();
  if (atomicSub(P.ctl + C_LIVE, 1u) == 1u) {
    __threadfence();
    atomicExch(P.ctl + C_FINISHED, 1u);
  }
}

// Plans segment s's next round from nx (cur, wlen, rounds set) and publishes
// its phase A, or finishes the segment.
__device__ void start_round(const Params& P, const SegDesc& sd, u32 s, SegState nx) {
  nx.wfill = nx.wlen;
  plan_round(sd, P.cfg, nx);
  P.st[s] = nx;
  atomicMax(P.ctl + C_MAXROUND, nx.rounds);
  if (nx.tiles == 0) {
    finish_segment(P);
    return;
  }
  __threadfence();
  const u32 per_tile = max(1u, min(ceil_div(nx.wlen, P.cfg.dom_block), A_BLOCKS));
  publish(P, s, 0, nx.tiles, nx.tiles * per_tile);
}

// Finds the task of ticket t: 1 found (*idx), 0 not known yet (retry), -1
// no more work.  `cursor` is the task of the CTA's previous ticket, a lower
// bound because a CTA's tickets increase.  The task is the last one whose
// first ticket is <= t: the search gallops forward from the cursor (the
// CTA's next task is usually near its last one), then bisects; each probe is
// one acquire load of a task's (first ticket, published) word.
__device__ int find_task(const Params& P, u32 t, u32* cursor, u32* idx_out) {
  const volatile unsigned long long* q = reinterpret_cast<const volatile unsigned long long*>(P.ctl + C_QUEUE);
  u64 qv = *q;
  if (t >= (u32)qv) {
    if (!ld_vol_u32(P.ctl + C_FINISHED)) return 0;
    __threadfence();
    qv = *q;  // nothing is published once every segment has finished
    if (t >= (u32)qv) return -1;
  }
  u32 lo = *cursor, hi = (u32)(qv >> 32);
  if (hi > P.task_cap) hi = P.task_cap;
  for (u32 step = 1; lo + step < hi; step <<= 1) {
    const u64 w = ld_acquire_u64(&P.tasks[lo + step].tv);
    if (!(w & 1ull)) return 0;  // reserved, not yet published
    if ((u32)(w >> 32) > t) {
      hi = lo + step;
      break;
    }
    lo += step;
  }
  while (hi - lo > 1) {
    const u32 mid = lo + ((hi - lo) >> 1);
    const u64 w = ld_acquire_u64(&P.tasks[mid].tv);
    if (!(w & 1ull)) return 0;
    if ((u32)(w >> 32) <= t) lo = mid;
    else hi = mid;
  }
  // orders the reads of the task's fields after its publication
  if (!(ld_acquire_u64(&P.tasks[lo].tv) & 1ull)) return 0;
  *cursor = lo;
  *idx_out = lo;
  return 1;
}

// ------------------------------------------------------------ items

// One work item as the producer thread planned it.
enum : u32 { M_EMPTY = 0, M_PENDING = 1, M_READY = 2, M_DONE = 3 };
struct Meta {
  u32 state;
  u32 ticket;
  u32 s;       // segment
  u32 phase;
  u32 tile;    // candidate tile (phase A) or dense-list tile (phase B)
  u32 tgid;    // completion counter of the tile
  u32 cnt;     // dominators staged in the item's buffer
  u32 base;    // index of the first staged dominator in its source
  u32 dense;   // 1: the dominators are dense-list points (FP32 via dpos)
  u32 copied;  // 1: a bulk copy into the item's buffer was issued
  u32 counted; // 1: the producer counted the item towards its tile (empty item completing the tile)
  u32 parity;  // phase parity of the buffer's barrier that the copy completes
};

struct Shared {
  uint4 scode[WARPS][GS];  // per-warp compaction scratch of the scan
  u32 spos[WARPS][GS];
  Meta meta[2];
  u64 bar[2];
  u32 cursor;
  u32 flag;
  u32 wtot[WARPS];
  u32 tile_base;
  u32 pclaim;   // warps past their scan of the current item (the first one produces)
  int pslot;    // buffer slot of the next item
  uint4* pbuf;  // and its buffer
  u32 abort_seen;  // the launch's abort flag was seen set
  u32 pcopies[2];  // bulk copies issued into each buffer (by its producers, one at a time)
  EngineCounts counts;
};

// Tile status words of the ordered compaction (decoupled look-back): the
// tile's survivor count, or the inclusive prefix of survivor counts up to
// and including the tile.
constexpr u32 TS_AGG = 1u << 30, TS_INC = 2u << 30, TS_VAL = TS_AGG - 1;

// Empty items (dense blocks past a tile's triangular bound) the producer may
// retire in one call before it hands the CTA a ticket still pending.
constexpr int SKIP_MAX = 32;

// Producer (one thread at a time: thread 0 while the CTA waits for work, else
// lane 0 of the warp that finished the current item first; never blocks):
// claims a ticket for buffer `slot` if it has none, and once the ticket's
// task is known plans the item and starts the bulk copy of its dominator
// block's FP16 images.  The buffer is free: every warp has finished the item
// that used it.  A phase-B item whose
// dense block lies past its tile's triangular bound tests nothing: the
// producer counts it towards its tile's completion itself and claims the
// next ticket, unless the item is the one that completes the tile (then the
// CTA runs it, already counted, to append the tile's survivors).
__device__ void produce(const Params& P, Shared& S, int slot, uint4* buf) {
  Meta& m = S.meta[slot];
  for (int skips = 0;; ++skips) {
  if (m.state == M_EMPTY) {
    m.ticket = atomicAdd(P.ctl + C_TICKET, 1u);
    m.state = M_PENDING;
  }
  if (m.state != M_PENDING || skips == SKIP_MAX) return;
  u32 idx = 0;
  const int f = find_task(P, m.ticket, &S.cursor, &idx);
  if (f < 0) {
    m.state = M_DONE;
    return;
  }
  if (f == 0) return;
  m.counted = 0;
  const Task* tk = P.tasks + idx;
  const u32 DB = P.cfg.dom_block;
  m.s = __ldcg(&tk->s);
  m.phase = __ldcg(&tk->phase);
  const u32 tiles = __ldcg(&tk->tiles);
  const u32 l = m.ticket - (u32)(__ldcg(reinterpret_cast<const unsigned long long*>(&tk->tv)) >> 32);
  m.tile = l % tiles;  // block-major: item l = block * tiles + tile
  const u32 b = l / tiles;
  m.tgid = __ldcg(P.tbase + m.s) + m.tile;
  const u32 wlen = ld_cg_u32(&P.st[m.s].wlen);
  const SegDesc* sd = P.segs + m.s;
  const uint4* codes;
  if (m.phase == 0) {
    m.cnt = min(wlen, DB);
    m.base = 0;
    m.dense = 0;
    codes = sd->whc;
  } else {
    const u32 dlen = ld_cg_u32(&P.st[m.s].dlen);
    const u32 wb = ceil_div(wlen, DB);
    const u32 wbB = wb > A_BLOCKS ? wb - A_BLOCKS : 0;
    if (b < wbB) {
      m.base = (A_BLOCKS + b) * DB;
      m.cnt = min(DB, wlen - m.base);
      m.dense = 0;
      codes = sd->whc + m.base;
    } else {
      // the dense list is in position (= score) order: a candidate of dense
      // tile t can only be dominated by dense entries up to the end of the
      // tile, extended over a run of scores equal to its last one (the end
      // the last phase-A tile wrote into the tile's status word)
      const u32 ord = round_ord(P.cfg, ld_cg_u32(&P.st[m.s].cur), ld_cg_u32(&P.st[m.s].cend));
      const u32 e = ord != ORD_NONE ? ld_cg_u32(P.tstat + m.tgid) : dlen;
      m.base = (b - wbB) * DB;
      m.cnt = m.base < e ? min(DB, e - m.base) : 0;
      m.dense = 1;
      codes = sd->dhc + m.base;
      const u32 per_tile = wbB + ceil_div(dlen, DB);
      if (m.cnt == 0 && per_tile > 1) {
        // nothing to test (no kills to publish, so no fence before the count)
        const u32 old = atomicAdd(P.tdoneB + m.tgid, 1u);
        if (old != per_tile - 1) {
          m.state = M_EMPTY;
          continue;
        }
        P.tdoneB[m.tgid] = 0;
        m.counted = 1;
      }
    }
  }
  m.copied = 0;
  if (m.cnt) {
    // whole pairs: m.base is even, the block is m.cnt entries rounded up
    const u32 bytes = ((m.cnt + 1) & ~1u) * 16u;
    m.parity = S.pcopies[slot] & 1u;
    ++S.pcopies[slot];
    fence_proxy_async();
    mbar_expect_tx(&S.bar[slot], bytes);
    bulk_g2s(buf, codes, bytes, &S.bar[slot]);
    m.copied = 1;
  }
  m.state = M_READY;
  return;
  }
}

// The first warp to finish its scan of the current item plans the next one
// (produce), so the producer's memory round trips delay no warp that still
// has candidates to test.
__device__ __forceinline__ void produce_next(const Params& P, Shared& S) {
  if ((threadIdx.x & 31) == 0 && atomicAdd(&S.pclaim, 1u) == 0) {
    produce(P, S, S.pslot, S.pbuf);
    // the abort flag for the check after the item, read off its critical path
    if (ld_vol_u32(P.ctl + C_ABORT)) S.abort_seen = 1;
  }
  __syncwarp();
}

template <int D>
__device__ void load_cand(const SegDesc& sd, u32 pos, bool valid, CandsT<D, R>& c, int r) {
  // the images are loaded beside the flag, not after it (one round trip)
  const uint4 h = valid ? __ldg(sd.hc + pos) : make_uint4(0u, 0u, 0u, 0u);
  bool ok = valid && ld_cg_u8(sd.alive + pos);
  c.alive[r] = ok;
  c.was[r] = ok;
  c.pos[r] = pos;
  if (ok) {
    unpack_dup<D>(h, c.t[r]);
  } else {
    set_dead<D>(c.t[r]);
  }
}

// After the last tile of a phase A (one thread): publish phase B over the
// dense list of dl points, or the next round if nothing survived.
__device__ void after_phase_a(const Params& P, const SegDesc& sd, u32 s, const SegState& cs, u32 dl) {
  if (dl == 0) {
    SegState nx;
    nx.cur = cs.cend;
    nx.wlen = cs.wlen;
    nx.rounds = cs.rounds + 1;
    start_round(P, sd, s, nx);
  } else {
    const u32 DB = P.cfg.dom_block;
    const u32 wb = ceil_div(cs.wlen, DB);
    const u32 wbB = wb > A_BLOCKS ? wb - A_BLOCKS : 0;
    const u32 dtiles = ceil_div(dl, TILE);
    publish(P, s, 1, dtiles, dtiles * (wbB + ceil_div(dl, DB)));
  }
}

// The survivors of the chunk [cur, cend) of a segment, compacted by the whole
// CTA into the dense list in position order (ORD_LAST, by the phase's last
// tile once every tile's flags are final); sets the list's length and
// returns it.  Thread t takes PER consecutive positions of each step, so a
// block-wide exclusive scan of the threads' counts gives every survivor its
// slot.
template <int D>
__device__ u32 compact_chunk(const SegDesc& sd, SegState* st, u32 cur, u32 cend, Shared& S) {
  constexpr u32 PER = 8;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  u32 base = 0;
  for (u32 p0 = cur; p0 < cend; p0 += THREADS * PER) {
    const u32 q0 = p0 + threadIdx.x * PER;
    u32 fl = 0;
#pragma unroll
    for (u32 i = 0; i < PER; ++i)
      if (q0 + i < cend && ld_cg_u8(sd.alive + q0 + i)) fl |= 1u << i;
    const u32 c = __popc(fl);
    u32 x = c;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const u32 y = __shfl_up_sync(FULL, x, o);
      if (lane >= o) x += y;
    }
    if (lane == 31) S.wtot[warp] = x;
    __syncthreads();
    u32 off = base + x - c;
    u32 tot = 0;
#pragma unroll
    for (int w = 0; w < WARPS; ++w) {
      const u32 v = S.wtot[w];
      if (w < warp) off += v;
      tot += v;
    }
    while (fl) {
      const u32 i = __ffs(fl) - 1;
      fl &= fl - 1;
      const u32 pos = q0 + i;
      sd.dpos[off] = pos;
      put_pair_entry<D>(sd.dhc, off, __ldg(sd.hc + pos));
      ++off;
    }
    base += tot;
    __syncthreads();  // S.wtot is rewritten by the next step
  }
  if (threadIdx.x == 0) st->dlen = base;
  __threadfence();
  fence_proxy_async();
  __syncthreads();
  return base;
}

// Phase A item: tile `tile` of the chunk against window block 0.
template <int D>
__device__ void item_a(const Params& P, const SegDesc& sd, const Meta& mt, const uint4* staged, Shared& S) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const u32 DB = P.cfg.dom_block;
  const u32 s = mt.s;
  SegState* st = P.st + s;
  SegState cs;
  cs.cur = ld_cg_u32(&st->cur);
  cs.cend = ld_cg_u32(&st->cend);
  const u32 cnt = mt.cnt;
  const u32 gbase = cs.cur + mt.tile * TILE + warp * GS;

  if (cnt) {
    CandsT<D, R> c;
#pragma unroll
    for (int r = 0; r < R; ++r) {
      u32 pos = gbase + r * 32 + lane;
      load_cand<D>(sd, pos, pos < cs.cend, c, r);
    }
    if (__any_sync(FULL, any_alive(c))) {
      DomSrc src{sd.win, nullptr, 0};
      scan_smem<D>(staged, cnt, src, sd.pts, c, S.scode[warp], S.spos[warp], sd.alive, &S.counts);
    }
  }
  // the staged buffer is refilled by a bulk copy once every warp is past
  // the barrier below
  fence_proxy_async_smem();
  produce_next(P, S);
  // the round state the completion needs (read after the scan: fewer
  // registers live across it)
  cs.wlen = ld_cg_u32(&st->wlen);
  cs.tiles = ld_cg_u32(&st->tiles);
  cs.rounds = ld_cg_u32(&st->rounds);
  const u32 ord = round_ord(P.cfg, cs.cur, cs.cend);
  const u32 per_tile = max(1u, min(ceil_div(cs.wlen, DB), A_BLOCKS));
  __syncthreads();
  // with one item per tile (always so while A_BLOCKS is 1) the item
  // completes its tile and needs no completion counter
  if (per_tile > 1) {
    if (threadIdx.x == 0) {
      __threadfence();
      u32 old = atomicAdd(P.tdoneA + mt.tgid, 1u);
      S.flag = (old == per_tile - 1);
      if (S.flag) P.tdoneA[mt.tgid] = 0;
    }
    __syncthreads();
    if (!S.flag) return;
  }
  __threadfence();
  // The tile's flags are final for phase A: compact its survivors into the
  // dense list in position order.  The tile's offset is the sum of its
  // predecessors' survivor counts, found by decoupled look-back over the
  // status words of the earlier tiles (all of which hold smaller tickets, so
  // every one of them is being or has been processed).
  if (ord == ORD_NONE) {
    // unordered compaction: the warp's slots from one atomic
    bool a[R];
    u32 m[R];
    u32 tot = 0;
#pragma unroll
    for (int r = 0; r < R; ++r) {
      const u32 pos = gbase + r * 32 + lane;
      a[r] = pos < cs.cend && ld_cg_u8(sd.alive + pos);
      m[r] = __ballot_sync(FULL, a[r]);
      tot += __popc(m[r]);
    }
    u32 base = 0;
    if (lane == 0 && tot) base = atomicAdd(&st->dlen, tot);
    base = __shfl_sync(FULL, base, 0);
#pragma unroll
    for (int r = 0; r < R; ++r) {
      if (a[r]) {
        const u32 pos = gbase + r * 32 + lane;
        const u32 slot = base + __popc(m[r] & ((1u << lane) - 1u));
        sd.dpos[slot] = pos;
        put_pair_entry<D>(sd.dhc, slot, __ldg(sd.hc + pos));
      }
      base += __popc(m[r]);
    }
  } else if (ord == ORD_LOOKBACK) {
  bool a[R];
  u32 bal[R];
  u32 wcount = 0;
#pragma unroll
  for (int r = 0; r < R; ++r) {
    u32 pos = gbase + r * 32 + lane;
    a[r] = pos < cs.cend && ld_cg_u8(sd.alive + pos);
    bal[r] = __ballot_sync(FULL, a[r]);
    wcount += __popc(bal[r]);
  }
  if (lane == 0) S.wtot[warp] = wcount;
  __syncthreads();
  if (threadIdx.x == 0) {
    u32 cnt_t = 0;
    for (int w = 0; w < WARPS; ++w) cnt_t += S.wtot[w];
    u32* stat = P.tstat + __ldcg(P.tbase + s);
    u32 excl = 0;
    if (mt.tile == 0) {
      atomicExch(stat, TS_INC | cnt_t);
    } else {
      atomicExch(stat + mt.tile, TS_AGG | cnt_t);
      u64 t0 = 0;
      u32 seen = 0;
      for (int j = (int)mt.tile - 1; j >= 0;) {
        const u32 v = ld_vol_u32(stat + j);
        if (v & TS_INC) {
          excl += v & TS_VAL;
          break;
        }
        if (v & TS_AGG) {
          excl += v & TS_VAL;
          --j;
          continue;
        }
        // the predecessor has not counted its survivors yet: bounded wait
        const u32 now = ld_vol_u32(P.ctl + C_PROGRESS);
        if (t0 == 0 || now != seen) {
          seen = now;
          t0 = globaltimer();
        } else if (globaltimer() - t0 > P.wait_ns || ld_vol_u32(P.ctl + C_ABORT)) {
          abort_launch(P, ERR_TIMEOUT);
          break;
        }
      }
      atomicExch(stat + mt.tile, TS_INC | (excl + cnt_t));
    }
    S.tile_base = excl;
  }
  __syncthreads();
  {
    u32 off = S.tile_base;
    for (int w = 0; w < warp; ++w) off += S.wtot[w];
    const u32 lt = (1u << lane) - 1u;
#pragma unroll
    for (int r = 0; r < R; ++r) {
      if (a[r]) {
        const u32 slot = off + __popc(bal[r] & lt);
        const u32 pos = gbase + r * 32 + lane;
        sd.dpos[slot] = pos;
        put_pair_entry<D>(sd.dhc, slot, __ldg(sd.hc + pos));
      }
      off += __popc(bal[r]);
    }
    if (lane == 0 && wcount) atomicAdd(&st->dlen, wcount);
  }
  }
  __threadfence();
  fence_proxy_async();
  __syncthreads();
  if (ord == ORD_NONE) {
    // one thread counts the tile and, for the phase's last tile, publishes
    // phase B: the other threads have nothing left to do in this item
    if (threadIdx.x == 0) {
      const u32 old = atomicAdd(&st->done_a, 1u);
      if (old == cs.tiles - 1) {
        __threadfence();
        after_phase_a(P, sd, s, cs, atomicAdd(&st->dlen, 0u));
      }
    }
    return;
  }
  if (threadIdx.x == 0) {
    const u32 old = atomicAdd(&st->done_a, 1u);
    S.flag = old == cs.tiles - 1;
    if (S.flag) {
      __threadfence();
      S.tile_base = atomicAdd(&st->dlen, 0u);
    }
  }
  __syncthreads();
  if (!S.flag) return;
  // ORD_LAST: every tile's flags are final; the last one compacts the chunk
  const u32 dl = ord == ORD_LAST ? compact_chunk<D>(sd, st, cs.cur, cs.cend, S) : S.tile_base;
  {
    // last tile of phase A: every tile has finished its look-back, so its
    // status word is free.  It now holds the dense tile's end for phase B:
    // the tile's last position, or the whole list when a run of equal
    // scores straddles it (zero past the dense tiles, for the next round)
    u32* stat = P.tstat + __ldcg(P.tbase + s);
    for (u32 j = threadIdx.x; j < cs.tiles; j += THREADS) {
      const u32 tend = min(dl, (j + 1) * TILE);
      u32 e = j * TILE < dl ? tend : 0u;
      if (e && tend < dl) {
        const float last = __ldg(sd.score + __ldcg(sd.dpos + tend - 1));
        const float next = __ldg(sd.score + __ldcg(sd.dpos + tend));
        if (next == last) e = dl;
      }
      stat[j] = e;
    }
    __threadfence();
    __syncthreads();
  }
  if (threadIdx.x == 0) after_phase_a(P, sd, s, cs, dl);
}

// Phase B item: dense tile against window block A_BLOCKS + b, or dense block
// b - (window blocks of phase B).
template <int D>
__device__ void item_b(const Params& P, const SegDesc& sd, const Meta& mt, const uint4* staged, Shared& S) {
  constexpr int V = vec_of(D);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const u32 DB = P.cfg.dom_block;
  const u32 s = mt.s;
  SegState* st = P.st + s;
  SegState cs;
  cs.dlen = ld_cg_u32(&st->dlen);
  const u32 dbase = mt.tile * TILE + warp * GS;
  const u32 cnt = mt.cnt;
  const DomSrc src = mt.dense ? DomSrc{sd.pts, sd.dpos, mt.base} : DomSrc{sd.win, nullptr, mt.base};
  if (cnt) {  // an item past the triangular bound has nothing to test
    CandsT<D, R> c;
#pragma unroll
    for (int r = 0; r < R; ++r) {
      u32 e = dbase + r * 32 + lane;
      bool valid = e < cs.dlen;
      u32 pos = valid ? __ldcg(sd.dpos + e) : 0;
      load_cand<D>(sd, pos, valid, c, r);
    }
    if (__any_sync(FULL, any_alive(c))) {
      scan_smem<D>(staged, cnt, src, sd.pts, c, S.scode[warp], S.spos[warp], sd.alive, &S.counts);
    }
  }
  fence_proxy_async_smem();  // as in item_a
  produce_next(P, S);
  // the round state the completion needs (read after the scan, as in item_a)
  cs.cur = ld_cg_u32(&st->cur);
  cs.cend = ld_cg_u32(&st->cend);
  cs.wlen = ld_cg_u32(&st->wlen);
  cs.rounds = ld_cg_u32(&st->rounds);
  const u32 ord = round_ord(P.cfg, cs.cur, cs.cend);
  const u32 wb = ceil_div(cs.wlen, DB);
  const u32 wbB = wb > A_BLOCKS ? wb - A_BLOCKS : 0;
  const u32 dtiles = ceil_div(cs.dlen, TILE);
  const u32 per_tile = wbB + ceil_div(cs.dlen, DB);
  __syncthreads();
  if (per_tile > 1) {
    if (threadIdx.x == 0) {
      if (mt.counted) {
        S.flag = 1;
      } else {
        __threadfence();
        u32 old = atomicAdd(P.tdoneB + mt.tgid, 1u);
        S.flag = (old == per_tile - 1);
        if (S.flag) P.tdoneB[mt.tgid] = 0;
      }
    }
    __syncthreads();
    if (!S.flag) return;
  }
  __threadfence();
  // the dense tile's flags are final: append its survivors to the window
  // (the warp's slots from one atomic; the window's order does not matter)
  u32 wpos[R], wm[R];
  bool wa[R];
  u32 tot = 0;
#pragma unroll
  for (int r = 0; r < R; ++r) {
    const u32 e = dbase + r * 32 + lane;
    wpos[r] = e < cs.dlen ? __ldcg(sd.dpos + e) : 0;
  }
#pragma unroll
  for (int r = 0; r < R; ++r) {
    const u32 e = dbase + r * 32 + lane;
    wa[r] = e < cs.dlen && ld_cg_u8(sd.alive + wpos[r]);
    wm[r] = __ballot_sync(FULL, wa[r]);
    tot += __popc(wm[r]);
  }
  u32 base = 0;
  if (lane == 0 && tot) base = atomicAdd(&st->wfill, tot);
  base = __shfl_sync(FULL, base, 0);
#pragma unroll
  for (int r = 0; r < R; ++r) {
    const u32 pos = wpos[r];
    const bool a = wa[r];
    const u32 m = wm[r];
    const u32 slot = base + __popc(m & ((1u << lane) - 1u));
    base += __popc(m);
    if (a) {
      const float4* src4 = sd.pts + (u64)pos * V;
      float4* dst4 = sd.win + (u64)slot * V;
#pragma unroll
      for (int v = 0; v < V; ++v) dst4[v] = __ldg(src4 + v);
      put_pair_entry<D>(sd.whc, slot, __ldg(sd.hc + pos));
    }
  }
  __threadfence();
  fence_proxy_async();
  __syncthreads();
  if (threadIdx.x == 0) {
    u32 old = atomicAdd(&st->done_b, 1u);
    if (old == dtiles - 1) {
      // last dense tile: clear the tile ends for the next round's phase A,
      // then the next round
      if (ord != ORD_NONE) {
        u32* stat = P.tstat + __ldcg(P.tbase + s);
        for (u32 j = 0; j < dtiles; ++j) stat[j] = 0;
      }
      __threadfence();
      SegState nx;
      nx.cur = cs.cend;
      nx.wlen = atomicAdd(&st->wfill, 0u);
      nx.rounds = cs.rounds + 1;
      start_round(P, sd, s, nx);
    }
  }
}

template <int D>
__device__ void run_item(const Params& P, const SegDesc& sd, const Meta& m, const uint4* staged, Shared& S) {
  if (m.phase == 0) item_a<D>(P, sd, m, staged, S);
  else item_b<D>(P, sd, m, staged, S);
}

// Prologue of CTA 0: completion-counter bases of the segments, then round 0
// of every segment (published or finished at once).
__device__ bool prologue(const Params& P) {
  __shared__ u32 s_carry;
  __shared__ u32 s_warp[WARPS];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  if (threadIdx.x == 0) s_carry = 0;
  __syncthreads();
  for (u32 base = 0; base < P.nseg; base += THREADS) {
    const u32 i = base + threadIdx.x;
    // a phase of segment i has at most ceil(n / TILE) tiles
    const u32 v = i < P.nseg ? ceil_div(P.segs[i].n, TILE) + 1 : 0;
    u32 x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      u32 y = __shfl_up_sync(FULL, x, o);
      if (lane >= o) x += y;
    }
    if (lane == 31) s_warp[warp] = x;
    __syncthreads();
    u32 pre = s_carry;
    for (int w2 = 0; w2 < warp; ++w2) pre += s_warp[w2];
    if (i < P.nseg) P.tbase[i] = pre + x - v;
    __syncthreads();
    if (threadIdx.x == THREADS - 1) s_carry = pre + x;
    __syncthreads();
  }
  if (s_carry > P.tcap) {
    if (threadIdx.x == 0) abort_launch(P, ERR_CAPACITY);
    return false;
  }
  if (threadIdx.x == 0) {
    P.ctl[C_LIVE] = P.nseg;
    if (P.nseg == 0) P.ctl[C_FINISHED] = 1;
  }
  __threadfence();
  __syncthreads();
  for (u32 i = threadIdx.x; i < P.nseg; i += THREADS) {
    SegState z;
    z.cur = 0;
    z.wlen = 0;
    z.rounds = 0;
    start_round(P, P.segs[i], i, z);
  }
  return true;
}

// 16 warps per SM in every shape: up to 128 registers a thread, no spills
__global__ void __launch_bounds__(THREADS, 16 / WARPS) k_engine(Params P) {
  extern __shared__ __align__(128) unsigned char dyn[];
  __shared__ Shared S;
  const u32 DB = P.cfg.dom_block;
  uint4* const buf0 = reinterpret_cast<uint4*>(dyn);  // two buffers of DB (+ padding) FP16 images
  const u32 BUFN = DB + STAGE_PAD;

  if (threadIdx.x == 0) {
    mbar_init(&S.bar[0]);
    mbar_init(&S.bar[1]);
    S.cursor = 0;
    S.meta[0].state = M_EMPTY;
    S.meta[1].state = M_EMPTY;
    S.abort_seen = 0;
    S.counts.n16 = 0;
    S.pcopies[0] = S.pcopies[1] = 0;
  }
  __syncthreads();
  if (blockIdx.x == 0 && !prologue(P)) return;

  if (threadIdx.x == 0) produce(P, S, 0, buf0);
  for (u32 k = 0;; ++k) {
    const int slot = k & 1;
    uint4* const cur_buf = buf0 + (size_t)slot * BUFN;
    // wait until the slot's ticket has a task (or there is no more work)
    if (threadIdx.x == 0) {
      // every warp is past the previous item's last CTA barrier, so every
      // thread has copied that item's plan and left its producer call: its
      // buffer slot is free for the next plan
      if (k > 0) S.meta[slot ^ 1].state = M_EMPTY;
      S.pclaim = 0;
      S.pslot = slot ^ 1;
      S.pbuf = buf0 + (size_t)(slot ^ 1) * BUFN;
      u64 t0 = 0;
      u32 seen = 0;
      while (S.meta[slot].state == M_PENDING) {
        produce(P, S, slot, cur_buf);
        if (S.meta[slot].state != M_PENDING) break;
        if (ld_vol_u32(P.ctl + C_ABORT)) {
          S.meta[slot].state = M_DONE;
          break;
        }
        const u32 now = ld_vol_u32(P.ctl + C_PROGRESS);
        if (t0 == 0 || now != seen) {
          seen = now;
          t0 = globaltimer();
        } else if (globaltimer() - t0 > P.wait_ns) {
          abort_launch(P, ERR_TIMEOUT);
          S.meta[slot].state = M_DONE;
          break;
        }
        __nanosleep(128);
      }
    }
    __syncthreads();
    const Meta m = S.meta[slot];
    if (m.state != M_READY) break;
    if (m.copied) {
      if (!mbar_wait(&S.bar[slot], m.parity, P.wait_ns, P.err, P.ctl)) break;
    }
    const SegDesc sd = P.segs[m.s];
    switch (sd.d) {
      case 1: run_item<1>(P, sd, m, cur_buf, S); break;
      case 2: run_item<2>(P, sd, m, cur_buf, S); break;
      case 3: run_item<3>(P, sd, m, cur_buf, S); break;
      case 4: run_item<4>(P, sd, m, cur_buf, S); break;
      case 5: run_item<5>(P, sd, m, cur_buf, S); break;
      case 6: run_item<6>(P, sd, m, cur_buf, S); break;
      case 7: run_item<7>(P, sd, m, cur_buf, S); break;
      default: run_item<8>(P, sd, m, cur_buf, S); break;
    }
    if (threadIdx.x == 0) atomicAdd(P.ctl + C_PROGRESS, 1u);
    // No CTA barrier here: past the item's last barrier the threads read
    // only abort_seen (set before it, in produce_next) and, on an abort, the
    // prefetched plan; thread 0 rewrites neither before the next item's
    // first barrier.  An abort raised while this item ran is seen after the
    // next one.
    if (S.abort_seen) {
      // the copy of the prefetched item may still be in flight
      const Meta mn = S.meta[slot ^ 1];
      if (mn.state == M_READY && mn.copied) mbar_wait(&S.bar[slot ^ 1], mn.parity, P.wait_ns, P.err, P.ctl);
      break;
    }
  }
  // the CTA's test counts into the launch's (every warp is past its last
  // scan when the loop ends normally; after an abort the counts are partial)
  if (threadIdx.x == 0) {
    unsigned long long* tot = reinterpret_cast<unsigned long long*>(P.ctl + C_TESTS);
    const unsigned long long a = atomicExch(&S.counts.n16, 0ull);
    if (a) atomicAdd(tot, a);
  }
}


int g_sms = 0;

}  // namespace

template <>
cudaError_t engine_run_variant<WARPS, R>(const SegDesc* segs_dev, u32 nseg, const EngineCfg& cfg,
                                         const EngineWork& w, u32* err, cudaStream_t st) {
  if (nseg == 0) return cudaSuccess;
  if (cfg.dom_block == 0 || cfg.dom_block > DBMAX) return cudaErrorInvalidValue;
  if (w.task_cap > 0xffffffffull) return cudaErrorInvalidValue;
  Params P;
  P.segs = segs_dev;
  P.nseg = nseg;
  P.cfg = cfg;
  P.st = w.st;
  P.tbase = w.tbase;
  P.tdoneA = w.tdoneA;
  P.tdoneB = w.tdoneB;
  P.tstat = w.tstat;
  P.tcap = w.tcap;
  P.tasks = reinterpret_cast<Task*>(w.tasks);
  P.task_cap = (u32)w.task_cap;
  P.ctl = w.ctl;
  P.err = err;
  P.wait_ns = cfg.wait_ns ? cfg.wait_ns : WAIT_NS;
  size_t smem = 2 * ((size_t)cfg.dom_block + STAGE_PAD) * sizeof(uint4);
  cudaError_t e = cudaFuncSetAttribute(k_engine, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  int per_sm = 0;
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_engine, THREADS, smem);
  if (e != cudaSuccess) return e;
  if (per_sm <= 0) return cudaErrorInvalidConfiguration;
  if (!g_sms) g_sms = device_sm_count();
  unsigned grid = (unsigned)(g_sms * per_sm);
  // a small launch (few tiles in any phase) gets fewer CTAs: any grid size
  // is correct (no CTA waits for one that is not resident), and the CTAs
  // that would find no work still cost their scheduling and exit
  const u64 want = 4 * w.tcap > 16 ? 4 * w.tcap : 16;
  if (want < grid) grid = (unsigned)want;
  e = cudaMemsetAsync(w.ctl, 0, ENGINE_CTL_WORDS * sizeof(u32), st);
  if (e == cudaSuccess) e = cudaMemsetAsync(w.tasks, 0, w.task_cap * sizeof(Task), st);
  if (e == cudaSuccess) e = cudaMemsetAsync(w.tstat, 0, w.tcap * sizeof(u32), st);
  if (e != cudaSuccess) return e;
  // One CTA per resident slot.  No CTA ever waits for one that is not
  // resident: a CTA waits only for work published by CTAs that hold
  // earlier tickets (or, in the ordered compaction, for earlier tiles), and
  // a CTA takes a ticket only once it runs, so the launch needs no
  // co-residency guarantee (and can be captured into a CUDA graph).
  note_launch();
  k_engine<<<grid, THREADS, smem, st>>>(P);
  return cudaGetLastError();
}

#if SKY_ENGINE_WARPS == 4 && SKY_ENGINE_R == 4
// Facts of the engine that every shape shares.
u32 engine_max_round_word() { return C_MAXROUND; }
u32 engine_tests_word() { return C_TESTS; }
u32 engine_max_dom_block() { return DBMAX; }
size_t engine_task_bytes() { return sizeof(Task); }
#endif

}  // namespace sky
