// Dominance kernels outside the local-skyline engine: the representative
// filter (Section 4.1, a relative skyline: kill candidates dominated by a
// point of a second set) and the NoSeq final phase (Section 4.2, Prop. 2),
// plus the segment descriptors the engine (sky_engine.cu) runs on.
//
// Both kernels are exact for the same reason as the engine: t is outside
// Sky(r) iff some point of r dominates t, so testing a candidate against any
// set of real input points never kills a skyline point.  A group is 32 * R
// candidates in the registers of one warp (R per lane); the warp leaves as
// soon as a ballot shows every candidate dead.  The representative filter
// scans its few dominators with uniform loads and FP32 compares (Def. 1);
// NoSeq stages blocks of u in shared memory and rejects pairs on their FP16
// images first.
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

__device__ __forceinline__ u8 ld_cg_u8(const u8* p) {
  return (u8)__ldcg(reinterpret_cast<const unsigned char*>(p));
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

// NoSeq's dominance test runs on the FP16 round-down images of u, as the
// local-skyline engine's does.  Round-down is monotone, so an image of s
// above t's means s is above t in that attribute and cannot dominate t; the
// sign of an f16x2 difference t - s is the sign of the exact difference of
// the images (a nonzero difference of two FP16 numbers never rounds to zero,
// the images are finite), so the FP16 test only rejects pairs that fail
// Def. 1, and every pair it passes is decided in FP32.  A candidate holds
// its images duplicated per word, word k = (image k, image k); dominators
// are staged as pairs, word k = (image k of the first, image k of the
// second), so one subtraction per attribute tests two dominators.
// NoSeq candidates per lane: 4 above d = 4, where skylines are large and a
// group's candidates mostly survive (more candidates share each staged
// dominator); 2 up to d = 4, where most of u dies within a few dominators
// and smaller groups leave earlier.
__host__ __device__ constexpr int ns_r(int d) { return d <= 4 ? 2 : 4; }
constexpr u32 INF2 = 0x7C007C00u;    // (+inf, +inf): a padding dominator fails every test
constexpr u32 NEG_INF2 = 0xFC00FC00u;  // (-inf, -inf): a dead candidate passes no test

__device__ __forceinline__ u32 hsub2_bits(u32 t, u32 w) {
  u32 r;
  asm("sub.rn.f16x2 %0, %1, %2;" : "=r"(r) : "r"(t), "r"(w));
  return r;
}
// Bit 15 / 31 clear iff every attribute of the first / second dominator of
// the pair is <= the candidate's (in FP16 images).
template <int D>
__device__ __forceinline__ u32 pair_fail(const u32 (&t)[D], const u32 (&w)[D]) {
  u32 x = hsub2_bits(t[0], w[0]);
#pragma unroll
  for (int k = 1; k < D; ++k) x |= hsub2_bits(t[k], w[k]);
  return x;
}

// A lane's NoSeq candidates in NR slots: ns_r(D) when a group is loaded,
// fewer once its live candidates have been compacted.
template <int D, int NR>
struct NCand {
  u32 t[NR][D];   // duplicated FP16 images (-inf when dead)
  u32 pos[NR];    // position in u
  bool alive[NR];
  bool was[NR];
};

template <int D, int NR>
__device__ __forceinline__ u32 ns_live(const NCand<D, NR>& c) {
  u32 n = 0;
#pragma unroll
  for (int r = 0; r < NR; ++r) n += __popc(__ballot_sync(FULL, c.alive[r]));
  return n;
}

// Loads the group's candidates at u positions base + r * 32 + lane < end.
template <int D, int NR>
__device__ __forceinline__ void ns_load(const NoSeqArgs& a, u32 base, u32 end, int lane, NCand<D, NR>& c) {
#pragma unroll
  for (int r = 0; r < NR; ++r) {
    const u32 pos = base + r * 32 + lane;
    const bool ok = pos < end && ld_cg_u8(a.ualive + pos);
    const uint4 h = ok ? __ldg(a.uhc + pos) : make_uint4(0u, 0u, 0u, 0u);
    const u32 w[4] = {h.x, h.y, h.z, h.w};
    c.alive[r] = ok;
    c.was[r] = ok;
    c.pos[r] = pos;
#pragma unroll
    for (int k = 0; k < D; ++k) c.t[r][k] = ok ? __byte_perm(w[k / 2], 0u, (k & 1) ? 0x3232u : 0x1010u) : NEG_INF2;
  }
}

// Records the kills of the lane's slots (alive when loaded, dead now).
template <int D, int NR>
__device__ __forceinline__ void ns_write_kills(const NoSeqArgs& a, const NCand<D, NR>& c) {
#pragma unroll
  for (int r = 0; r < NR; ++r)
    if (c.was[r] && !c.alive[r]) a.ualive[c.pos[r]] = 0;
}

// Moves the warp's live candidates of a (at most 32 x NB of them) into NB
// slots per lane, slot-major, through the warp's shared scratch (sc: images,
// one uint4 per candidate, sp: positions); a's kills are recorded first.
template <int D, int NA, int NB>
__device__ __forceinline__ void ns_compact(const NoSeqArgs& a, const NCand<D, NA>& ca, NCand<D, NB>& cb, uint4* sc,
                                           u32* sp) {
  const int lane = threadIdx.x & 31;
  const u32 lt = (1u << lane) - 1u;
  ns_write_kills(a, ca);
  u32 k0 = 0;
#pragma unroll
  for (int r = 0; r < NA; ++r) {
    const u32 m = __ballot_sync(FULL, ca.alive[r]);
    if (ca.alive[r]) {
      const u32 k = k0 + __popc(m & lt);
      u32 w[4];
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const u32 lo = 2 * q < D ? ca.t[r][2 * q < D ? 2 * q : 0] : 0u;
        const u32 hi = 2 * q + 1 < D ? ca.t[r][2 * q + 1 < D ? 2 * q + 1 : 0] : 0u;
        w[q] = __byte_perm(lo, hi, 0x5410u);
      }
      sc[k] = make_uint4(w[0], w[1], w[2], w[3]);
      sp[k] = ca.pos[r];
    }
    k0 += __popc(m);
  }
  __syncwarp();
#pragma unroll
  for (int r = 0; r < NB; ++r) {
    const u32 k = r * 32 + lane;
    const bool v = k < k0;
    cb.alive[r] = v;
    cb.was[r] = v;
    cb.pos[r] = v ? sp[k] : 0u;
    const uint4 h = v ? sc[k] : make_uint4(0u, 0u, 0u, 0u);
    const u32 w[4] = {h.x, h.y, h.z, h.w};
#pragma unroll
    for (int q = 0; q < D; ++q) cb.t[r][q] = v ? __byte_perm(w[q / 2], 0u, (q & 1) ? 0x3232u : 0x1010u) : NEG_INF2;
  }
  __syncwarp();
}

// Def. 1 on the FP32 attributes: does u[j] dominate u[i]?
template <int D>
__device__ __forceinline__ bool dominates_u(const float4* __restrict__ upts, u32 j, u32 i) {
  constexpr int V = vec_of(D);
  float w[8], t[8];
  load_point<D>(upts + (u64)j * V, false, w);
  load_point<D>(upts + (u64)i * V, false, t);
  bool le = true, ne = false;
#pragma unroll
  for (int k = 0; k < D; ++k) {
    le &= w[k] <= t[k];
    ne |= w[k] != t[k];
  }
  return le && ne;
}

// Tests the warp's candidates against u[lo..hi): 64 entries at a time are
// staged as 32 dominator pairs in the warp's shared buffer sp (64 uint4; a
// tail is padded with +inf images), then scanned with broadcast shared
// loads, two pairs per step; the next 64 entries are loaded from global
// memory while the current ones are scanned.  Every 16 entries the warp
// counts its live candidates and stops when none is left or when they fit
// in half the slots (the caller compacts them and goes on with fewer).
// Returns the position reached (every entry before it has been tested);
// *n_live = live candidates.
template <int D, int NR>
__device__ u32 ns_scan_range(const NoSeqArgs& a, u32 lo, u32 hi, uint4* sp, NCand<D, NR>& c, u32* n_live) {
  const int lane = threadIdx.x & 31;
  const uint4 z = make_uint4(INF2, INF2, INF2, INF2);
  uint4 p0, p1;  // this lane's two entries of the next stage
  {
    const u32 e0 = lo + 2 * lane;
    p0 = e0 < hi ? __ldg(a.uhc + e0) : z;
    p1 = e0 + 1 < hi ? __ldg(a.uhc + e0 + 1) : z;
  }
  for (u32 j0 = lo; j0 < hi; j0 += 64) {
    {
      const u32 x0[4] = {p0.x, p0.y, p0.z, p0.w}, x1[4] = {p1.x, p1.y, p1.z, p1.w};
      u32 w[8];
#pragma unroll
      for (int k = 0; k < 8; ++k) w[k] = __byte_perm(x0[k / 2], x1[k / 2], (k & 1) ? 0x7632u : 0x5410u);
      sp[2 * lane] = make_uint4(w[0], w[1], w[2], w[3]);
      sp[2 * lane + 1] = make_uint4(w[4], w[5], w[6], w[7]);
    }
    __syncwarp();
    if (j0 + 64 < hi) {
      const u32 e0 = j0 + 64 + 2 * lane;
      p0 = e0 < hi ? __ldg(a.uhc + e0) : z;
      p1 = e0 + 1 < hi ? __ldg(a.uhc + e0 + 1) : z;
    }
    const u32 npairs = min(32u, (hi - j0 + 1) / 2);
    for (u32 q = 0; q < npairs; q += 2) {
      // pairs q and q + 1 (q + 1 <= 31; past the range it holds +inf images)
      u32 w[2][D];
#pragma unroll
      for (int g = 0; g < 2; ++g) {
        const uint4 a0 = sp[2 * (q + g)];
        w[g][0] = a0.x;
        if (D > 1) w[g][1 < D ? 1 : 0] = a0.y;
        if (D > 2) w[g][2 < D ? 2 : 0] = a0.z;
        if (D > 3) w[g][3 < D ? 3 : 0] = a0.w;
        if (D > 4) {
          const uint4 a1 = sp[2 * (q + g) + 1];
          w[g][4 < D ? 4 : 0] = a1.x;
          if (D > 5) w[g][5 < D ? 5 : 0] = a1.y;
          if (D > 6) w[g][6 < D ? 6 : 0] = a1.z;
          if (D > 7) w[g][7 < D ? 7 : 0] = a1.w;
        }
      }
      u32 acc = 0xffffffffu;
#pragma unroll
      for (int g = 0; g < 2; ++g)
#pragma unroll
        for (int r = 0; r < NR; ++r) acc &= pair_fail<D>(c.t[r], w[g]);
      if ((acc & 0x80008000u) != 0x80008000u) {
#pragma unroll
        for (int g = 0; g < 2; ++g)
#pragma unroll
          for (int r = 0; r < NR; ++r) {
            const u32 x = pair_fail<D>(c.t[r], w[g]);
#pragma unroll
            for (int h = 0; h < 2; ++h) {
              const u32 jd = j0 + 2 * (q + g) + h;
              if (c.alive[r] && !((x >> (15 + 16 * h)) & 1u) && jd < hi && dominates_u<D>(a.upts, jd, c.pos[r])) {
                c.alive[r] = false;
#pragma unroll
                for (int k = 0; k < D; ++k) c.t[r][k] = NEG_INF2;
              }
            }
          }
      }
      if ((q & 6) == 6) {
        const u32 n = ns_live(c);
        if (n == 0 || (NR > 1 && n <= 32u * (NR / 2))) {
          __syncwarp();
          *n_live = n;
          return min(j0 + 2 * (q + 2), hi);
        }
      }
    }
    __syncwarp();  // the buffer is restaged only after every lane's reads
  }
  *n_live = ns_live(c);
  return hi;
}

// The rest of one item from u position pos: every partition j of u[pos,
// bhi) that is a potential dominator of partition i, cut at the group's
// largest score fmax (u_j is sorted by score, so later points cannot
// dominate), scanned with the NR-slot candidates; when they fit in fewer
// slots they are compacted and the item goes on with those.  Records the
// kills.
template <int D, int NR>
__device__ void ns_rest(const NoSeqArgs& a, u32 i, float fmax, u32 pos, u32 bhi, NCand<D, NR>& c, u32 n,
                        uint4* sp, uint4* sc, u32* spos) {
  while (pos < bhi && n > 0) {
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
      u32 lo3 = pos, hi3 = jend;
      while (lo3 < hi3) {
        u32 mid = lo3 + ((hi3 - lo3) >> 1);
        if (__ldg(a.uscore + mid) <= fmax) lo3 = mid + 1;
        else hi3 = mid;
      }
      const u32 cut = lo3;
      if (cut > pos) {
        const u32 reached = ns_scan_range<D, NR>(a, pos, cut, sp, c, &n);
        if (reached < cut) {
          if (n == 0) break;
          if constexpr (NR > 1) {
            NCand<D, NR / 2> c2;
            ns_compact<D, NR, NR / 2>(a, c, c2, sc, spos);
            ns_rest<D, NR / 2>(a, i, fmax, reached, bhi, c2, n, sp, sc, spos);
            return;
          }
        }
      }
    }
    pos = jend;
  }
  ns_write_kills(a, c);
}

// Items: (group of u_i, dominator block of u).  gpre[P + 1]: prefix of the
// group counts per partition (computed on the device).
template <int D>
__global__ void __launch_bounds__(THREADS) k_noseq(NoSeqArgs a, const u32* __restrict__ gpre, const u32* nu_dev,
                                                   u32* counter) {
  constexpr int NR0 = ns_r(D);
  __shared__ uint4 s_pairs[WARPS][64];
  __shared__ uint4 s_cimg[WARPS][32 * NR0];  // compaction scratch: images
  __shared__ u32 s_cpos[WARPS][32 * NR0];    // and positions
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const u32 nu = *nu_dev;
  const u32 ngroups = gpre[a.P];
  const u32 DB = a.dom_block;
  const u32 nblocks = (nu + DB - 1) / DB;
  const u64 total = (u64)ngroups * nblocks;
  for (;;) {
    u32 first = 0;
    if (lane == 0) first = atomicAdd(counter, (u32)IB);
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
      constexpr u32 NGS = 32 * NR0;  // candidates per group
      const u32 base = ibeg + (G - __ldg(gpre + i)) * NGS;
      const u32 gend = min(base + NGS, iend);
      const float fmax = __ldg(a.uscore + gend - 1);
      // dominator block [blo, bhi) of u: its first partition that holds
      // potential dominators (the candidates are loaded only if there is one)
      const u32 blo = b * DB, bhi = min(blo + DB, nu);
      u32 pos = blo;
      while (pos < bhi) {
        u32 l2 = 0, h2 = a.P;
        while (h2 - l2 > 1) {
          u32 mid = (l2 + h2) >> 1;
          if (__ldg(a.useg + mid) <= pos) l2 = mid;
          else h2 = mid;
        }
        if (in_pd(a, i, l2) && __ldg(a.uscore + pos) <= fmax) break;
        pos = min(__ldg(a.useg + l2 + 1), bhi);
      }
      if (pos >= bhi) continue;
      NCand<D, NR0> c;
      ns_load<D, NR0>(a, base, gend, lane, c);
      const u32 n = ns_live(c);
      if (n == 0) continue;
      ns_rest<D, NR0>(a, i, fmax, pos, bhi, c, n, s_pairs[warp], s_cimg[warp], s_cpos[warp]);
    }
  }
}

__global__ void k_noseq_groups(const u32* __restrict__ useg, u32 P, u32 ngs, u32* __restrict__ cnt) {
  u64 i = (u64)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < P) cnt[i] = (useg[i + 1] - useg[i] + ngs - 1) / ngs;
}

// Segment descriptors of the local phase from the partition offsets;
// partitions removed by Grid Filtering get no work.  Every per-point array
// of a segment is the slice [seg_off[s], seg_off[s + 1]) of the whole array.
__global__ void k_build_segs(const u32* __restrict__ seg_off, u32 P, const u8* __restrict__ dropped, SegArrays a,
                             int d, SegDesc* segs, u32* nonempty) {
  u64 s = (u64)blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= P) return;
  if (nonempty && seg_off[s + 1] > seg_off[s]) atomicAdd(nonempty, 1u);
  const int V = vec_of(d);
  u32 o = seg_off[s];
  SegDesc sd;
  sd.pts = reinterpret_cast<const float4*>(a.pts) + (u64)o * V;
  sd.hc = a.hc + o;
  sd.score = a.score + o;
  sd.alive = a.alive + o;
  sd.win = reinterpret_cast<float4*>(a.win) + (u64)o * V;
  // image arrays of pairs: each segment starts at an even entry, with one
  // entry of slack per segment (the arrays hold n + P + 2 entries)
  const u64 q = ((u64)o + s + 1) & ~1ull;
  sd.whc = a.whc + q;
  sd.dpos = a.dpos + o;
  sd.dhc = a.dhc + q;
  sd.n = (dropped && dropped[s]) ? 0u : seg_off[s + 1] - o;
  sd.d = (u32)d;
  segs[s] = sd;
}

__global__ void k_build_one_seg(SegArrays a, const u32* n_dev, int d, SegDesc* seg) {
  SegDesc sd;
  sd.pts = reinterpret_cast<const float4*>(a.pts);
  sd.hc = a.hc;
  sd.score = a.score;
  sd.alive = a.alive;
  sd.win = reinterpret_cast<float4*>(a.win);
  sd.whc = a.whc;
  sd.dpos = a.dpos;
  sd.dhc = a.dhc;
  sd.n = *n_dev;
  sd.d = (u32)d;
  *seg = sd;
}

// After an engine launch: its round count into the query's maximum, its
// test count into the query's sum.
__global__ void k_fold_engine(const u32* ctl, u32 round_word, u32 tests_word, u32* round_dst,
                              unsigned long long* tests_dst) {
  atomicMax(round_dst, ctl[round_word]);
  atomicAdd(tests_dst, *reinterpret_cast<const unsigned long long*>(ctl + tests_word));
}

int g_sm_count = 0;

}  // namespace

cudaError_t launch_build_segs(const u32* seg_off, u32 P, const u8* dropped, const SegArrays& a, int d,
                              SegDesc* segs, u32* nonempty, cudaStream_t st) {
  if (P == 0) return cudaSuccess;
  note_launch();
  k_build_segs<<<(P + 255) / 256, 256, 0, st>>>(seg_off, P, dropped, a, d, segs, nonempty);
  return cudaGetLastError();
}

cudaError_t launch_build_one_seg(const SegArrays& a, const u32* n_dev, int d, SegDesc* seg, cudaStream_t st) {
  note_launch();
  k_build_one_seg<<<1, 1, 0, st>>>(a, n_dev, d, seg);
  return cudaGetLastError();
}

cudaError_t launch_fold_engine(const u32* ctl, u32* round_dst, unsigned long long* tests_dst, cudaStream_t st) {
  note_launch();
  k_fold_engine<<<1, 1, 0, st>>>(ctl, engine_max_round_word(), engine_tests_word(), round_dst, tests_dst);
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

cudaError_t launch_noseq(const NoSeqArgs& a, u32* gcnt, u32* gpre, u32* scan_tmp, const u32* nu_dev, u32* counter,
                         cudaStream_t st) {
  if (a.P == 0) return cudaSuccess;
  note_launch();
  k_noseq_groups<<<(a.P + 255) / 256, 256, 0, st>>>(a.useg, a.P, 32u * ns_r(a.d), gcnt);
  cudaError_t e = scan_u32(gcnt, gpre, a.P, true, false, scan_tmp, st);
  if (e != cudaSuccess) return e;
  // gpre[P] = total groups
  e = cudaMemcpyAsync(gpre + a.P, scan_tmp + scan_total_index(a.P), sizeof(u32), cudaMemcpyDeviceToDevice, st);
  if (e != cudaSuccess) return e;
  e = cudaMemsetAsync(counter, 0, sizeof(u32), st);
  if (e != cudaSuccess) return e;
  int sms = g_sm_count ? g_sm_count : device_sm_count();
  return dispatch_d(a.d, [&](auto D) {
    int per_sm = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_noseq<decltype(D)::value>, THREADS, 0);
    if (per_sm <= 0) per_sm = 1;
    note_launch();
    k_noseq<decltype(D)::value><<<(unsigned)(sms * per_sm), THREADS, 0, st>>>(a, gpre, nu_dev, counter);
  });
}

}  // namespace sky
