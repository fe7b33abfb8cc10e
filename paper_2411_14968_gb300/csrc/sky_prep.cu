// HBM-bound passes of the pipeline: validation and scores, partition
// assignment (Sections 3.1-3.4), gather into the sorted padded layout, Grid
// Filtering (Section 3.2), Sorted representatives (Section 4.1), compaction
// of the local skylines and the final compaction into ascending indices.
#include <algorithm>
#include <cuda_fp16.h>
#include "sky_internal.cuh"

namespace sky {

namespace {

constexpr int PT = 256;

inline unsigned grid_for(u64 n) { return (unsigned)((n + PT - 1) / PT); }

// Score f(t) of Section 2: FP32 sum of the d attributes added left to right,
// round-to-nearest, no contraction.
template <int D>
__device__ __forceinline__ float score_of(const float (&x)[8]) {
  float f = x[0];
#pragma unroll
  for (int a = 1; a < D; ++a) f = __fadd_rn(f, x[a]);
  // a point holding both +inf and -inf has no sum (inf - inf): it scores
  // +inf, which keeps the score monotone under dominance (such a point
  // dominates only points holding +inf in the same attribute)
  return f != f ? __int_as_float(0x7f800000) : f;
}

// FP16 round-down images of the 8 (padded) attributes, two per word,
// clamped to the finite FP16 range (clamping is monotone too, and keeps the
// images finite, so differences of two images never produce NaN).
__device__ __forceinline__ u32 pack_rd(float lo, float hi) {
  constexpr float HMAX = 65504.0f;
  __half a = __float2half_rd(fminf(fmaxf(lo, -HMAX), HMAX)), b = __float2half_rd(fminf(fmaxf(hi, -HMAX), HMAX));
  return (u32)__half_as_ushort(a) | ((u32)__half_as_ushort(b) << 16);
}
__device__ __forceinline__ uint4 fp16_codes(const float (&x)[8]) {
  return make_uint4(pack_rd(x[0], x[1]), pack_rd(x[2], x[3]), pack_rd(x[4], x[5]), pack_rd(x[6], x[7]));
}

// Reads point i of the row-major input with -0.0 turned into +0.0 (x + 0.0
// is +0.0 for both zeros under round-to-nearest); flags NaN.
template <int D>
__device__ __forceinline__ void load_row(const float* __restrict__ X, u64 i, float (&x)[8],
                                         u32* err) {
  const float* r = X + i * D;
  bool nan = false;
#pragma unroll
  for (int a = 0; a < 8; ++a) {
    float v = a < D ? r[a] : 0.0f;
    nan |= (v != v);
    x[a] = __fadd_rn(v, 0.0f);
  }
  if (nan && err) atomicOr(err, ERR_NAN);
}

// SplitMix64 (Steele, Lea & Flood, OOPSLA 2014): output number i (from 0) of
// the generator whose state starts at `seed`.
__device__ __forceinline__ u64 splitmix64(u64 seed, u64 i) {
  u64 z = seed + (i + 1) * 0x9E3779B97F4A7C15ull;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

// Coordinate used by the Grid / Angular keys: the attribute itself, or the
// attribute divided by its column maximum when normalising (keys only).
__device__ __forceinline__ float key_coord(const float (&x)[8], int a, const float (&sc)[8],
                                           int normalize) {
  return normalize ? __fdiv_rn(x[a], sc[a]) : x[a];
}

// Section 3.2: cell = sum_i clamp(floor(x_i * m_i), 0, m_i - 1) * prod_{j<i} m_j.
template <int D>
__device__ __forceinline__ u32 grid_cell(const float (&x)[8], const float (&sc)[8], const PrepArgs& p) {
  u64 id = 0, w = 1;
#pragma unroll
  for (int a = 0; a < D; ++a) {
    u32 m = p.slices[a];
    float v = __fmul_rn(key_coord(x, a, sc, p.normalize), (float)m);
    float fl = floorf(v);
    u32 c;
    if (!(fl > 0.0f)) c = 0;
    else if (fl >= (float)(m - 1)) c = m - 1;
    else c = (u32)fl;
    id += (u64)c * w;
    w *= m;
  }
  return (u32)id;
}

// Section 3.3, Eq. (index-angular), without transcendentals: the digit of
// angle i counts the thresholds k pi / (2 m_i) that phi_i reaches, i.e.
// #{k in 1..m_i-1 : S_i >= x_i^2 tan^2(k pi / (2 m_i))}, S_i the suffix sum of
// squares accumulated from the last attribute.  The thresholds increase with
// k, so the count is found by bisection.
template <int D>
__device__ __forceinline__ u32 angular_cell(const float (&x)[8], const float (&sc)[8], const PrepArgs& p) {
  float k[8], S[8];
#pragma unroll
  for (int a = 0; a < 8; ++a) { k[a] = 0.0f; S[a] = 0.0f; }
#pragma unroll
  for (int a = 0; a < D; ++a) k[a] = key_coord(x, a, sc, p.normalize);
  float acc = 0.0f;
#pragma unroll
  for (int a = D - 1; a >= 1; --a) {
    float sq = __fmul_rn(k[a], k[a]);
    acc = (a == D - 1) ? sq : __fadd_rn(sq, acc);
    S[a - 1] = acc;
  }
  u64 id = 0, w = 1;
#pragma unroll
  for (int a = 0; a + 1 < D; ++a) {
    u32 m = p.slices[a];
    float xx = __fmul_rn(k[a], k[a]);
    const float* T = p.ang_table + p.ang_off[a];
    u32 lo = 0, hi = m - 1;
    while (lo < hi) {
      u32 mid = (lo + hi + 1) >> 1;
      if (S[a] >= __fmul_rn(xx, T[mid - 1])) lo = mid;
      else hi = mid - 1;
    }
    id += (u64)lo * w;
    w *= m;
  }
  return (u32)id;
}

__global__ void k_colmax_init(u32* colmax) {
  if (threadIdx.x < 8) colmax[threadIdx.x] = 0;
}

// Column maxima (as fkey) for the normalised keys.
template <int D>
__global__ void k_colmax(const float* __restrict__ X, u64 n, u32* colmax, u32* err) {
  __shared__ u32 sm[8];
  if (threadIdx.x < 8) sm[threadIdx.x] = 0;
  __syncthreads();
  u32 loc[8];
#pragma unroll
  for (int a = 0; a < 8; ++a) loc[a] = 0;
  for (u64 i = (u64)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (u64)gridDim.x * blockDim.x) {
    float x[8];
    load_row<D>(X, i, x, err);
#pragma unroll
    for (int a = 0; a < D; ++a) loc[a] = max(loc[a], fkey(x[a]));
  }
#pragma unroll
  for (int a = 0; a < D; ++a) atomicMax(&sm[a], loc[a]);
  __syncthreads();
  if (threadIdx.x < D) atomicMax(&colmax[threadIdx.x], sm[threadIdx.x]);
}

// First pass: validation, scores and the first sort key of every scheme.
template <int D>
__global__ void k_prep(PrepArgs p) {
  u64 i = (u64)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= p.n) return;
  float x[8];
  load_row<D>(p.X, i, x, p.err);
  float sc[8];
#pragma unroll
  for (int a = 0; a < 8; ++a) sc[a] = 1.0f;
  if (p.normalize) {
    // the column maximum when positive and finite, else 1
#pragma unroll
    for (int a = 0; a < D; ++a) {
      float mx = fkey_inv(p.colmax[a]);
      sc[a] = (mx > 0.0f && mx <= 3.402823466e38f) ? mx : 1.0f;
    }
  }
  float f = score_of<D>(x);
  u64 key;
  switch (p.scheme) {
    case SCHEME_GRID: key = ((u64)grid_cell<D>(x, sc, p) << 32) | fkey(f); break;
    case SCHEME_ANGULAR: key = ((u64)angular_cell<D>(x, sc, p) << 32) | fkey(f); break;
    case SCHEME_RANDOM: key = splitmix64(p.seed, i); break;
    case SCHEME_SLICED: {
      float xs = 0.0f;
#pragma unroll
      for (int a = 0; a < D; ++a)
        if (a == p.slice_dim) xs = x[a];
      key = ((u64)fkey(xs) << 32) | fkey(f);
      break;
    }
    default: key = fkey(f); break;
  }
  p.keys[i] = key;
  p.vals[i] = (u32)i;
}

// Random (3.1) and Sliced (3.4): the point at sorted rank r goes to partition
// floor(start * p / N), start = r (Random) or the first rank of its run of
// equal (x_dim, f) keys (Sliced).  Writes the (partition, score) key back at
// the point's own index so that a second stable sort groups the partitions.
template <int D>
__global__ void k_rekey_rank(const float* __restrict__ X, u64 n, const u32* __restrict__ sorted_idx,
                             const u32* __restrict__ run_start, u32 P, u64* __restrict__ keys,
                             u32* __restrict__ vals) {
  u64 r = (u64)blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= n) return;
  u32 i = sorted_idx[r];
  u64 start = run_start ? run_start[r] : r;
  u32 pid = (u32)((start * (u64)P) / n);
  float x[8];
  load_row<D>(X, i, x, nullptr);
  keys[i] = ((u64)pid << 32) | fkey(score_of<D>(x));
  vals[i] = i;
}

// Sliced: head[r] = r at the first element of a run of equal keys, else 0;
// a max-scan of head gives the run start of every rank.
__global__ void k_run_heads(const u64* __restrict__ keys, u64 n, u32* __restrict__ head) {
  u64 r = (u64)blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= n) return;
  head[r] = (r == 0 || keys[r] != keys[r - 1]) ? (u32)r : 0u;
}

// Gather into the sorted padded layout; segment offsets per partition.
template <int D>
__global__ void k_gather(GatherArgs g) {
  u64 r = (u64)blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= g.n) return;
  u32 i = g.vals[r];
  float x[8];
  load_row<D>(g.X, i, x, nullptr);
  constexpr int V = vec_of(D);
  float4* dst = reinterpret_cast<float4*>(g.pts) + r * V;
  dst[0] = make_float4(x[0], x[1], x[2], x[3]);
  if (V > 1) dst[1] = make_float4(x[4], x[5], x[6], x[7]);
  g.hc[r] = g.rcode ? g.rcode[i] : fp16_codes(x);
  g.score[r] = score_of<D>(x);
  g.orig[r] = i;
  g.alive[r] = 1;
  u32 pid = (u32)(g.keys[r] >> 32);
  g.spid[r] = pid;
  long long prev = r == 0 ? -1 : (long long)(u32)(g.keys[r - 1] >> 32);
  for (long long q = prev + 1; q <= (long long)pid; ++q) g.seg_off[q] = (u32)r;
  if (r == g.n - 1)
    for (u64 q = (u64)pid + 1; q <= g.P; ++q) g.seg_off[q] = (u32)g.n;
}

// ------------------------------------------------------------ Grid Filtering

__global__ void k_occupied(const u32* __restrict__ seg_off, u32 P, u8* __restrict__ clos) {
  u64 c = (u64)blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= P) return;
  clos[c] = seg_off[c + 1] > seg_off[c] ? 1 : 0;
}

// One pass of the componentwise-<= closure of occupancy: prefix OR along
// axis k (cell stride `stride`, m cells along the axis).
__global__ void k_closure_axis(u8* __restrict__ clos, u32 P, u32 m, u32 stride) {
  u64 line = (u64)blockIdx.x * blockDim.x + threadIdx.x;
  u64 nlines = P / m;
  if (line >= nlines) return;
  u64 lo = line % stride, hi = line / stride;
  u64 base = hi * stride * m + lo;
  u8 acc = 0;
  for (u32 j = 0; j < m; ++j) {
    u64 c = base + (u64)j * stride;
    acc |= clos[c];
    clos[c] = acc;
  }
}

// Cell h is dropped iff some non-empty cell is strictly smaller in every
// coordinate (grid dominance), i.e. the closure at h - (1, ..., 1) is set.
__global__ void k_grid_dropped(const u8* __restrict__ clos, u32 P, int d, GridDims gd,
                               u8* __restrict__ dropped) {
  u64 h = (u64)blockIdx.x * blockDim.x + threadIdx.x;
  if (h >= P) return;
  u64 rest = h, below = 0, w = 1;
  bool ok = true;
  for (int a = 0; a < d; ++a) {
    u32 c = (u32)(rest % gd.m[a]);
    rest /= gd.m[a];
    if (c == 0) ok = false;
    else below += (u64)(c - 1) * w;
    w *= gd.m[a];
  }
  dropped[h] = ok ? clos[below] : 0;
}

__global__ void k_apply_dropped(const u32* __restrict__ spid, u64 n, const u8* __restrict__ dropped,
                                u8* __restrict__ alive, u8* __restrict__ stage_s, u32* counter) {
  u64 r = (u64)blockIdx.x * blockDim.x + threadIdx.x;
  bool dr = false;
  if (r < n && dropped[spid[r]]) {
    alive[r] = 0;
    stage_s[r] = ST_GRID;
    dr = true;
  }
  u32 b = __ballot_sync(FULL, dr);
  if ((threadIdx.x & 31) == 0 && b) atomicAdd(counter, __popc(b));
}

// ------------------------------------------- Sorted representatives (4.1)

// The first k points of every non-dropped, non-empty partition (the sort put
// them in (f, index) order), packed; empty slots hold +inf points, which
// dominate nothing.
template <int D>
__global__ void k_rep_select(const u32* __restrict__ seg_off, u32 P, u32 k,
                             const u8* __restrict__ dropped, const float* __restrict__ pts,
                             float* __restrict__ rep_pts, u8* __restrict__ rep_alive) {
  u64 t = (u64)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= (u64)P * k) return;
  u32 s = (u32)(t / k), j = (u32)(t % k);
  u32 len = seg_off[s + 1] - seg_off[s];
  bool ok = j < len && !(dropped && dropped[s]);
  rep_alive[t] = ok ? 1 : 0;
  constexpr int V = vec_of(D);
  const float4* src = reinterpret_cast<const float4*>(pts);
  float4* dst = reinterpret_cast<float4*>(rep_pts) + t * V;
  float4 inf = make_float4(INFINITY, INFINITY, INFINITY, INFINITY);
#pragma unroll
  for (int v = 0; v < V; ++v) dst[v] = ok ? src[(u64)(seg_off[s] + j) * V + v] : inf;
}

// Region representatives (Section 4.1): the k points of each segment with
// the largest volume of the dominance region inside the unit cube, V(t) =
// prod (1 - c_a) in double, factors left to right, c_a the attribute (over
// the column scale when normalising) clamped to [0, 1]; ties by original
// index.  One block per segment; pass r finds the best point after the
// winner of pass r - 1 in the order (V descending, index ascending).
__device__ __forceinline__ bool region_better(double v, u32 id, double bv, u32 bid) {
  return v > bv || (v == bv && id < bid);
}

template <int D>
__global__ void __launch_bounds__(256) k_rep_region(const u32* __restrict__ seg_off, u32 P, u32 k,
                                                    const u8* __restrict__ dropped, const float* __restrict__ pts,
                                                    const u32* __restrict__ orig, const u32* __restrict__ colmax,
                                                    int normalize, float* __restrict__ rep_pts,
                                                    u8* __restrict__ rep_alive) {
  __shared__ double s_v[8];
  __shared__ u32 s_id[8], s_pos[8];
  __shared__ double s_limv;
  __shared__ u32 s_limid;
  constexpr int V = vec_of(D);
  const u32 s = blockIdx.x;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const u32 o = seg_off[s];
  const u32 len = (dropped && dropped[s]) ? 0u : seg_off[s + 1] - o;
  float sc[8];
#pragma unroll
  for (int a = 0; a < 8; ++a) sc[a] = 1.0f;
  if (normalize) {
#pragma unroll
    for (int a = 0; a < D; ++a) {
      float mx = fkey_inv(colmax[a]);
      sc[a] = (mx > 0.0f && mx <= 3.402823466e38f) ? mx : 1.0f;
    }
  }
  const float4* src = reinterpret_cast<const float4*>(pts);
  bool have_lim = false;
  double limv = 0.0;
  u32 limid = 0;
  for (u32 r = 0; r < k; ++r) {
    double bv = -1.0;
    u32 bid = 0xffffffffu, bpos = 0xffffffffu;
    for (u32 j = threadIdx.x; j < len; j += blockDim.x) {
      float x[8];
      float4 q0 = src[(u64)(o + j) * V];
      x[0] = q0.x; x[1] = q0.y; x[2] = q0.z; x[3] = q0.w;
      if (V > 1) {
        float4 q1 = src[(u64)(o + j) * V + 1];
        x[4] = q1.x; x[5] = q1.y; x[6] = q1.z; x[7] = q1.w;
      }
      double v = 1.0;
#pragma unroll
      for (int a = 0; a < D; ++a) {
        double c = normalize ? (double)__fdiv_rn(x[a], sc[a]) : (double)x[a];
        c = c < 0.0 ? 0.0 : (c > 1.0 ? 1.0 : c);
        v = __dmul_rn(v, 1.0 - c);
      }
      const u32 id = orig[o + j];
      const bool after = !have_lim || v < limv || (v == limv && id > limid);
      if (after && region_better(v, id, bv, bid)) {
        bv = v;
        bid = id;
        bpos = o + j;
      }
    }
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
      double ov = __shfl_down_sync(FULL, bv, off);
      u32 oid = __shfl_down_sync(FULL, bid, off);
      u32 opos = __shfl_down_sync(FULL, bpos, off);
      if (region_better(ov, oid, bv, bid)) {
        bv = ov;
        bid = oid;
        bpos = opos;
      }
    }
    if (lane == 0) {
      s_v[warp] = bv;
      s_id[warp] = bid;
      s_pos[warp] = bpos;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      for (int w = 1; w < (int)(blockDim.x >> 5); ++w)
        if (region_better(s_v[w], s_id[w], bv, bid)) {
          bv = s_v[w];
          bid = s_id[w];
          bpos = s_pos[w];
        }
      const u64 t = (u64)s * k + r;
      const bool ok = bpos != 0xffffffffu;
      rep_alive[t] = ok ? 1 : 0;
      float4* dst = reinterpret_cast<float4*>(rep_pts) + t * V;
      const float4 inf = make_float4(INFINITY, INFINITY, INFINITY, INFINITY);
#pragma unroll
      for (int v = 0; v < V; ++v) dst[v] = ok ? src[(u64)bpos * V + v] : inf;
      s_limv = bv;
      s_limid = bid;
    }
    __syncthreads();
    have_lim = true;
    limv = s_limv;
    limid = s_limid;
    __syncthreads();
  }
}

// Kept representatives packed after R = Sky(reps) was computed in place.
template <int D>
__global__ void k_compact_reps(const u8* __restrict__ rep_alive, const u32* __restrict__ excl, u32 nrep,
                               const float* __restrict__ rep_pts, float* __restrict__ kept_pts) {
  u32 t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= nrep || !rep_alive[t]) return;
  constexpr int V = vec_of(D);
  const float4* src = reinterpret_cast<const float4*>(rep_pts) + (u64)t * V;
  float4* dst = reinterpret_cast<float4*>(kept_pts) + (u64)excl[t] * V;
#pragma unroll
  for (int v = 0; v < V; ++v) dst[v] = src[v];
}

// Histogram of the stage codes 0..5.
__global__ void k_stage_hist(const u8* __restrict__ stage_s, u64 n, u32* hist6) {
  __shared__ u32 h[6];
  if (threadIdx.x < 6) h[threadIdx.x] = 0;
  __syncthreads();
  for (u64 r = (u64)blockIdx.x * blockDim.x + threadIdx.x; r < n; r += (u64)gridDim.x * blockDim.x) {
    u8 s = stage_s[r];
    if (s < 6) atomicAdd(&h[s], 1u);
  }
  __syncthreads();
  if (threadIdx.x < 6) atomicAdd(&hist6[threadIdx.x], h[threadIdx.x]);
}

// ------------------------------------------------------------------ u and output

// Points alive after the local phase, compacted into u in (partition, f,
// index) order.
template <int D>
__global__ void k_compact_u(const u8* __restrict__ alive, const u32* __restrict__ excl, u64 n,
                            const float* __restrict__ pts, const uint4* __restrict__ hc,
                            const float* __restrict__ score, const u32* __restrict__ spid,
                            float* __restrict__ upts, uint4* __restrict__ uhc, float* __restrict__ uscore,
                            u32* __restrict__ upos, u32* __restrict__ upid,
                            u64* __restrict__ ukey, u32* __restrict__ uval) {
  u64 r = (u64)blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= n || !alive[r]) return;
  u32 j = excl[r];
  constexpr int V = vec_of(D);
  const float4* src = reinterpret_cast<const float4*>(pts) + r * V;
  float4* dst = reinterpret_cast<float4*>(upts) + (u64)j * V;
#pragma unroll
  for (int v = 0; v < V; ++v) dst[v] = src[v];
  uhc[j] = hc[r];
  float f = score[r];
  uscore[j] = f;
  upos[j] = (u32)r;
  if (upid) upid[j] = spid[r];
  if (ukey) {
    ukey[j] = fkey(f);
    uval[j] = j;
  }
}

__global__ void k_useg(const u32* __restrict__ seg_off, u32 P, const u32* __restrict__ excl, u64 n,
                       const u32* __restrict__ total, u32* __restrict__ useg) {
  u64 s = (u64)blockIdx.x * blockDim.x + threadIdx.x;
  if (s > P) return;
  u32 o = seg_off[s];
  useg[s] = o < n ? excl[o] : *total;
}

// u in score order for the sequential final phase.
template <int D>
__global__ void k_gather_u(const u32* __restrict__ order, u64 n, const u32* __restrict__ n_dev,
                           const float* __restrict__ upts,
                           const uint4* __restrict__ uhc, const float* __restrict__ uscore,
                           const u32* __restrict__ upos, float* __restrict__ mpts, uint4* __restrict__ mhc,
                           float* __restrict__ mscore, u32* __restrict__ mpos) {
  u64 r = (u64)blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= n || (n_dev && r >= *n_dev)) return;
  u32 j = order[r];
  constexpr int V = vec_of(D);
  const float4* src = reinterpret_cast<const float4*>(upts) + (u64)j * V;
  float4* dst = reinterpret_cast<float4*>(mpts) + r * V;
#pragma unroll
  for (int v = 0; v < V; ++v) dst[v] = src[v];
  mhc[r] = uhc[j];
  mscore[r] = uscore[j];
  mpos[r] = upos[j];
}

__global__ void k_scatter_alive(const u8* __restrict__ malive, const u32* __restrict__ mpos, u64 n,
                                const u32* __restrict__ n_dev, u8* __restrict__ alive, u8* __restrict__ stage_s,
                                u8 code) {
  u64 r = (u64)blockIdx.x * blockDim.x + threadIdx.x;
  if (n_dev && r >= *n_dev) return;
  if (r >= n || malive[r]) return;
  u32 p = mpos[r];
  alive[p] = 0;
  if (stage_s[p] == 0) stage_s[p] = code;
}

__global__ void k_stamp_stage(const u8* __restrict__ alive, u64 n, u8* __restrict__ stage_s, u8 code) {
  u64 r = (u64)blockIdx.x * blockDim.x + threadIdx.x;
  if (r < n && !alive[r] && stage_s[r] == 0) stage_s[r] = code;
}

// Final stage per sorted position: alive points are the skyline.  Writes the
// output mask (input order) and the optional per-point diagnostics.
__global__ void k_output(u8* __restrict__ stage_s, const u32* __restrict__ orig,
                         const u32* __restrict__ spid, u64 n, u8* __restrict__ mask,
                         u8* __restrict__ stage_out, u32* __restrict__ pid_out) {
  u64 r = (u64)blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= n) return;
  u32 i = orig[r];
  u8 s = stage_s[r];
  if (s == 0) {
    s = ST_SKY;
    stage_s[r] = s;
  }
  mask[i] = (s == ST_SKY);
  if (stage_out) stage_out[i] = s;
  if (pid_out) pid_out[i] = spid[r];
}

__global__ void k_compact_idx(const u8* __restrict__ mask, const u32* __restrict__ excl, u64 n,
                              u32* __restrict__ out) {
  u64 i = (u64)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n && mask[i]) out[excl[i]] = (u32)i;
}

}  // namespace

cudaError_t launch_colmax(const float* X, u64 n, int d, u32* colmax, u32* err, cudaStream_t st) {
  note_launch();
  k_colmax_init<<<1, 32, 0, st>>>(colmax);
  unsigned g = (unsigned)std::min<u64>((n + PT - 1) / PT, 4096);
  if (g == 0) return cudaGetLastError();
  note_launch();
  return dispatch_d(d, [&](auto D) { k_colmax<decltype(D)::value><<<g, PT, 0, st>>>(X, n, colmax, err); });
}

cudaError_t launch_prep(const PrepArgs& p, int d, cudaStream_t st) {
  if (p.n == 0) return cudaSuccess;
  note_launch();
  return dispatch_d(d, [&](auto D) { k_prep<decltype(D)::value><<<grid_for(p.n), PT, 0, st>>>(p); });
}

cudaError_t launch_rekey(const float* X, u64 n, int d, const u32* sorted_idx, const u32* run_start,
                         u32 P, u64* keys, u32* vals, cudaStream_t st) {
  if (n == 0) return cudaSuccess;
  return dispatch_d(d, [&](auto D) {
    note_launch();
    k_rekey_rank<decltype(D)::value><<<grid_for(n), PT, 0, st>>>(X, n, sorted_idx, run_start, P, keys, vals);
  });
}

cudaError_t launch_run_heads(const u64* keys, u64 n, u32* head, cudaStream_t st) {
  if (n == 0) return cudaSuccess;
  note_launch();
  k_run_heads<<<grid_for(n), PT, 0, st>>>(keys, n, head);
  return cudaGetLastError();
}

cudaError_t launch_gather(const GatherArgs& g, int d, cudaStream_t st) {
  if (g.n == 0) return cudaSuccess;
  note_launch();
  return dispatch_d(d, [&](auto D) { k_gather<decltype(D)::value><<<grid_for(g.n), PT, 0, st>>>(g); });
}

cudaError_t launch_grid_filter(const u32* seg_off, const u32* spid, u64 n, int d, const GridDims& gd,
                               u32 P, u8* clos, u8* dropped, u8* alive, u8* stage_s, u32* counter,
                               cudaStream_t st) {
  note_launch();
  k_occupied<<<grid_for(P), PT, 0, st>>>(seg_off, P, clos);
  u32 stride = 1;
  for (int a = 0; a < d; ++a) {
    u64 nlines = P / gd.m[a];
    if (nlines) {
      note_launch();
      k_closure_axis<<<grid_for(nlines), PT, 0, st>>>(clos, P, gd.m[a], stride);
    }
    stride *= gd.m[a];
  }
  note_launch();
  k_grid_dropped<<<grid_for(P), PT, 0, st>>>(clos, P, d, gd, dropped);
  if (n) {
    note_launch();
    k_apply_dropped<<<grid_for(n), PT, 0, st>>>(spid, n, dropped, alive, stage_s, counter);
  }
  return cudaGetLastError();
}

cudaError_t launch_rep_select(const u32* seg_off, u32 P, u32 k, const u8* dropped, const float* pts,
                              int d, float* rep_pts, u8* rep_alive, cudaStream_t st) {
  u64 cnt = (u64)P * k;
  if (cnt == 0) return cudaSuccess;
  return dispatch_d(d, [&](auto D) {
    note_launch();
    k_rep_select<decltype(D)::value><<<grid_for(cnt), PT, 0, st>>>(seg_off, P, k, dropped, pts, rep_pts, rep_alive);
  });
}

cudaError_t launch_rep_region(const u32* seg_off, u32 P, u32 k, const u8* dropped, const float* pts, const u32* orig,
                              const u32* colmax, int normalize, int d, float* rep_pts, u8* rep_alive, cudaStream_t st) {
  if (P == 0 || k == 0) return cudaSuccess;
  return dispatch_d(d, [&](auto D) {
    note_launch();
    k_rep_region<decltype(D)::value><<<P, 256, 0, st>>>(seg_off, P, k, dropped, pts, orig, colmax, normalize, rep_pts,
                                                         rep_alive);
  });
}

cudaError_t launch_compact_reps(const u8* rep_alive, const u32* excl, u32 nrep, int d, const float* rep_pts,
                                float* kept_pts, cudaStream_t st) {
  if (nrep == 0) return cudaSuccess;
  return dispatch_d(d, [&](auto D) {
    note_launch();
    k_compact_reps<decltype(D)::value><<<grid_for(nrep), PT, 0, st>>>(rep_alive, excl, nrep, rep_pts, kept_pts);
  });
}

cudaError_t launch_stage_hist(const u8* stage_s, u64 n, u32* hist6, cudaStream_t st) {
  cudaError_t e = cudaMemsetAsync(hist6, 0, 6 * sizeof(u32), st);
  if (e != cudaSuccess || n == 0) return e;
  unsigned g = (unsigned)std::min<u64>(grid_for(n), 1024);
  note_launch();
  k_stage_hist<<<g, PT, 0, st>>>(stage_s, n, hist6);
  return cudaGetLastError();
}

cudaError_t launch_compact_u(const u8* alive, const u32* excl, u64 n, int d, const float* pts, const uint4* hc,
                             const float* score, const u32* spid, float* upts, uint4* uhc, float* uscore,
                             u32* upos, u32* upid, u64* ukey, u32* uval, cudaStream_t st) {
  if (n == 0) return cudaSuccess;
  return dispatch_d(d, [&](auto D) {
    note_launch();
    k_compact_u<decltype(D)::value><<<grid_for(n), PT, 0, st>>>(alive, excl, n, pts, hc, score, spid, upts,
                                                               uhc, uscore, upos, upid, ukey, uval);
  });
}

cudaError_t launch_useg(const u32* seg_off, u32 P, const u32* excl, u64 n, const u32* total, u32* useg,
                        cudaStream_t st) {
  note_launch();
  k_useg<<<grid_for((u64)P + 1), PT, 0, st>>>(seg_off, P, excl, n, total, useg);
  return cudaGetLastError();
}

cudaError_t launch_gather_u(const u32* order, u64 n, const u32* n_dev, int d, const float* upts, const uint4* uhc,
                            const float* uscore, const u32* upos, float* mpts, uint4* mhc, float* mscore,
                            u32* mpos, cudaStream_t st) {
  if (n == 0) return cudaSuccess;
  return dispatch_d(d, [&](auto D) {
    note_launch();
    k_gather_u<decltype(D)::value><<<grid_for(n), PT, 0, st>>>(order, n, n_dev, upts, uhc, uscore, upos, mpts, mhc,
                                                              mscore, mpos);
  });
}

cudaError_t launch_scatter_alive(const u8* malive, const u32* mpos, u64 n, const u32* n_dev, u8* alive,
                                 u8* stage_s, u8 code, cudaStream_t st) {
  if (n == 0) return cudaSuccess;
  note_launch();
  k_scatter_alive<<<grid_for(n), PT, 0, st>>>(malive, mpos, n, n_dev, alive, stage_s, code);
  return cudaGetLastError();
}

cudaError_t launch_stamp_stage(const u8* alive, u64 n, u8* stage_s, u8 code, cudaStream_t st) {
  if (n == 0) return cudaSuccess;
  note_launch();
  k_stamp_stage<<<grid_for(n), PT, 0, st>>>(alive, n, stage_s, code);
  return cudaGetLastError();
}

cudaError_t launch_output(u8* stage_s, const u32* orig, const u32* spid, u64 n, u8* mask,
                          u8* stage_out, u32* pid_out, cudaStream_t st) {
  if (n == 0) return cudaSuccess;
  note_launch();
  k_output<<<grid_for(n), PT, 0, st>>>(stage_s, orig, spid, n, mask, stage_out, pid_out);
  return cudaGetLastError();
}

cudaError_t launch_compact_idx(const u8* mask, const u32* excl, u64 n, u32* out, cudaStream_t st) {
  if (n == 0) return cudaSuccess;
  note_launch();
  k_compact_idx<<<grid_for(n), PT, 0, st>>>(mask, excl, n, out);
  return cudaGetLastError();
}

}  // namespace sky
