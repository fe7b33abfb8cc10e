// Device-wide scan and stable LSD radix sort used by the skyline pipeline
// (the monotone-score sort of Algorithm 1's presorting step and the
// partition-keyed segmented sort of Algorithm 2's Partition phase).
#include "sky_internal.cuh"

namespace sky {

namespace {

constexpr int SCAN_T = 256;
constexpr int SCAN_IPT = 8;
constexpr u64 SCAN_TILE = SCAN_T * SCAN_IPT;

struct OpAdd {
  __device__ u32 operator()(u32 a, u32 b) const { return a + b; }
  static constexpr u32 identity = 0;
};
struct OpMax {
  __device__ u32 operator()(u32 a, u32 b) const { return a > b ? a : b; }
  static constexpr u32 identity = 0;
};

// Inclusive scan across the block of one value per thread; returns the
// inclusive prefix and writes the block aggregate to *agg.
template <class Op>
__device__ u32 block_scan_incl(u32 v, u32* sh, u32* agg, Op op) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int nw = blockDim.x >> 5;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    u32 y = __shfl_up_sync(FULL, v, o);
    if (lane >= o) v = op(v, y);
  }
  if (lane == 31) sh[warp] = v;
  __syncthreads();
  if (warp == 0) {
    u32 w = lane < nw ? sh[lane] : Op::identity;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      u32 y = __shfl_up_sync(FULL, w, o);
      if (lane >= o) w = op(w, y);
    }
    sh[lane] = w;
  }
  __syncthreads();
  u32 pre = warp > 0 ? sh[warp - 1] : Op::identity;
  u32 res = op(pre, v);
  *agg = sh[nw - 1];
  __syncthreads();
  return res;
}

template <class In, class Op>
__global__ void k_scan_reduce(const In* __restrict__ in, u64 n, u32* __restrict__ part) {
  __shared__ u32 sh[32];
  Op op;
  u64 base = (u64)blockIdx.x * SCAN_TILE;
  u32 acc = Op::identity;
#pragma unroll
  for (int i = 0; i < SCAN_IPT; ++i) {
    u64 e = base + (u64)i * SCAN_T + threadIdx.x;
    if (e < n) acc = op(acc, (u32)in[e]);
  }
  u32 agg;
  block_scan_incl(acc, sh, &agg, op);
  if (threadIdx.x == 0) part[blockIdx.x] = agg;
}

// One block: exclusive scan of the nb partials in place; part[nb] = total.
template <class Op>
__global__ void k_scan_partials(u32* part, u64 nb) {
  __shared__ u32 sh[32];
  __shared__ u32 buf[1024];
  Op op;
  u32 carry = Op::identity;
  for (u64 c = 0; c < nb; c += blockDim.x) {
    u64 e = c + threadIdx.x;
    u32 v = e < nb ? part[e] : Op::identity;
    u32 agg;
    u32 inc = block_scan_incl(v, sh, &agg, op);
    buf[threadIdx.x] = inc;
    __syncthreads();
    u32 ex = threadIdx.x > 0 ? buf[threadIdx.x - 1] : Op::identity;
    if (e < nb) part[e] = op(carry, ex);
    carry = op(carry, agg);
    __syncthreads();
  }
  if (threadIdx.x == 0) part[nb] = carry;
}

template <class In, class Op>
__global__ void k_scan_down(const In* __restrict__ in, u32* __restrict__ out, u64 n,
                            const u32* __restrict__ part, bool exclusive) {
  __shared__ u32 sh[32];
  Op op;
  u64 base = (u64)blockIdx.x * SCAN_TILE + (u64)threadIdx.x * SCAN_IPT;
  u32 v[SCAN_IPT];
  u32 acc = Op::identity;
#pragma unroll
  for (int i = 0; i < SCAN_IPT; ++i) {
    u64 e = base + i;
    v[i] = e < n ? (u32)in[e] : Op::identity;
    acc = op(acc, v[i]);
  }
  u32 agg;
  u32 inc = block_scan_incl(acc, sh, &agg, op);
  // exclusive prefix of this thread's run within the block
  __shared__ u32 buf[SCAN_T];
  buf[threadIdx.x] = inc;
  __syncthreads();
  u32 run_excl = threadIdx.x > 0 ? buf[threadIdx.x - 1] : Op::identity;
  u32 run = op(part[blockIdx.x], run_excl);
#pragma unroll
  for (int i = 0; i < SCAN_IPT; ++i) {
    u64 e = base + i;
    u32 nxt = op(run, v[i]);
    if (e < n) out[e] = exclusive ? run : nxt;
    run = nxt;
  }
}

// Scans of at most SCAN_SMALL_MAX elements (latency-bound): one block walks
// the tiles in order with a running carry, in one launch instead of three;
// the total goes to the same word as in the three-kernel scan.  In-place
// use is safe: a thread reads its elements before the block writes any.
constexpr u64 SCAN_SMALL_MAX = 8 * SCAN_TILE;

template <class In, class Op>
__global__ void k_scan_small(const In* in, u32* out, u64 n, u32* total, bool exclusive) {
  __shared__ u32 sh[32];
  __shared__ u32 buf[SCAN_T];
  Op op;
  u32 carry = Op::identity;
  for (u64 b0 = 0; b0 < n; b0 += SCAN_TILE) {
    const u64 base = b0 + (u64)threadIdx.x * SCAN_IPT;
    u32 v[SCAN_IPT];
    u32 acc = Op::identity;
#pragma unroll
    for (int i = 0; i < SCAN_IPT; ++i) {
      const u64 e = base + i;
      v[i] = e < n ? (u32)in[e] : Op::identity;
      acc = op(acc, v[i]);
    }
    u32 agg;
    const u32 inc = block_scan_incl(acc, sh, &agg, op);
    buf[threadIdx.x] = inc;
    __syncthreads();
    u32 run = op(carry, threadIdx.x > 0 ? buf[threadIdx.x - 1] : Op::identity);
#pragma unroll
    for (int i = 0; i < SCAN_IPT; ++i) {
      const u64 e = base + i;
      const u32 nxt = op(run, v[i]);
      if (e < n) out[e] = exclusive ? run : nxt;
      run = nxt;
    }
    carry = op(carry, agg);
    __syncthreads();  // buf is rewritten by the next tile
  }
  if (threadIdx.x == 0) *total = carry;
}

template <class In, class Op>
cudaError_t scan_impl(const In* in, u32* out, u64 n, bool exclusive, u32* tmp, cudaStream_t st) {
  u64 nb = (n + SCAN_TILE - 1) / SCAN_TILE;
  if (nb == 0) {
    return cudaMemsetAsync(tmp, 0, sizeof(u32), st);
  }
  if (n <= SCAN_SMALL_MAX) {
    note_launch();
    k_scan_small<In, Op><<<1, SCAN_T, 0, st>>>(in, out, n, tmp + nb, exclusive);
    return cudaGetLastError();
  }
  note_launch();
  k_scan_reduce<In, Op><<<(unsigned)nb, SCAN_T, 0, st>>>(in, n, tmp);
  note_launch();
  k_scan_partials<Op><<<1, 1024, 0, st>>>(tmp, nb);
  note_launch();
  k_scan_down<In, Op><<<(unsigned)nb, SCAN_T, 0, st>>>(in, out, n, tmp, exclusive);
  return cudaGetLastError();
}

// ---------------------------------------------------------------- radix sort
//
// Stable LSD radix sort with 8-bit digits, one kernel per digit (the
// single-pass scheme with decoupled look-back of Adinets & Merrill,
// "Onesweep", 2022): one kernel counts every digit of every pass up front,
// one block scans those counts into global digit offsets, and each pass's
// kernel then claims tiles in order, counts its tile's digits, publishes
// them and looks back over the earlier tiles' published counts for its
// offsets, and scatters its keys stably.

constexpr int RT = 256;       // threads per block == radix buckets
constexpr int RIPT = 16;      // keys per thread
constexpr u64 RTILE = (u64)RT * RIPT;
constexpr int MAX_PASS = 8;   // 64-bit keys
constexpr u64 WAIT_NS_SORT = 2000000000ull;  // bound of a look-back wait without progress

// Tile status word: bits 62..63 flag (1 = this tile's count, 2 = inclusive
// count of tiles 0..this), bits 32..39 the pass (1-based, so a word from an
// earlier pass of the same sort is not taken for this one), bits 0..31 the
// count.  The status array is zeroed at the start of every sort.
constexpr u64 ST_AGG = 1ull << 62, ST_INC = 2ull << 62;

// Layout of the work buffer (u32 words): ghist[MAX_PASS][RT], tile counters
// [MAX_PASS] (+ padding to 8 bytes), then the tile status words (u64).
constexpr size_t W_GHIST = 0;
constexpr size_t W_CTR = (size_t)MAX_PASS * RT;
constexpr size_t W_STATUS = W_CTR + MAX_PASS + 8;  // even, so the u64 array is aligned

// n_dev (optional): the element count lives in device memory and may be
// below the capacity n the grid was sized for; blocks past it do nothing.
__device__ __forceinline__ u64 radix_count(u64 n, const u32* n_dev) {
  if (!n_dev) return n;
  u64 m = *n_dev;
  return m < n ? m : n;
}

// The lanes of the warp holding the same digit as this lane (8-bit digits;
// invalid lanes, dg = ~0, are nobody's peers): one ballot per digit bit,
// so the cost does not depend on how many distinct digits the warp holds.
__device__ __forceinline__ u32 digit_peers(u32 dg, bool valid) {
  u32 peers = __ballot_sync(FULL, valid);
#pragma unroll
  for (int b = 0; b < 8; ++b) {
    const bool bit = (dg >> b) & 1u;
    const u32 bal = __ballot_sync(FULL, bit);
    peers &= bit ? bal : ~bal;
  }
  return peers;
}

__device__ __forceinline__ u64 sort_timer() {
  u64 t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// Counts the digits of every pass over one tile per block.  K is the key
// type (u64, or u32 for keys of at most 32 bits: a third less traffic per
// pass).
template <class K>
__global__ void k_sort_hist(const K* __restrict__ k, u64 n, const u32* __restrict__ n_dev, int lo_bit,
                            int npass, int last_bits, u32* __restrict__ ghist) {
  __shared__ u32 h[MAX_PASS][RT];
  const int tid = threadIdx.x;
  for (int p = 0; p < npass; ++p) h[p][tid] = 0;
  __syncthreads();
  n = radix_count(n, n_dev);
  const u64 base = (u64)blockIdx.x * RTILE;
  // the tile's keys are loaded together (one memory latency), then counted
  K kr[RIPT];
#pragma unroll
  for (int r = 0; r < RIPT; ++r) {
    const u64 e = base + (u64)r * RT + tid;
    kr[r] = e < n ? k[e] : (K)0;
  }
#pragma unroll
  for (int r = 0; r < RIPT; ++r) {
    if (base + (u64)r * RT + tid >= n) break;
    for (int p = 0; p < npass; ++p) {
      const u32 mask = p == npass - 1 ? (1u << last_bits) - 1u : 0xffu;
      atomicAdd(&h[p][(u32)(kr[r] >> (lo_bit + 8 * p)) & mask], 1u);
    }
  }
  __syncthreads();
  for (int p = 0; p < npass; ++p)
    if (h[p][tid]) atomicAdd(&ghist[(size_t)p * RT + tid], h[p][tid]);
}

// One block: exclusive scan of each pass's RT digit counts, in place.
__global__ void k_sort_scan(u32* ghist, int npass) {
  __shared__ u32 sh[32];
  for (int p = 0; p < npass; ++p) {
    u32* g = ghist + (size_t)p * RT;
    const u32 v = g[threadIdx.x];
    u32 agg;
    const u32 inc = block_scan_incl(v, sh, &agg, OpAdd());
    g[threadIdx.x] = inc - v;
  }
}

// One digit pass.  Blocks claim tiles in order, so the tiles a block looks
// back over are held by blocks that are running; a wait for one of them is
// bounded anyway (error word, then the block carries on with what it saw).
// Warp w of a block owns the tile's keys [w * KPW, (w + 1) * KPW), lane-
// strided, so the order (warp, iteration, lane) is the keys' input order:
// each warp counts its digits in a private row, one scan across the rows
// gives every warp its start per digit, and the warp then scatters its keys
// in the same order, keeping them stable inside each digit.
constexpr int KPW = RIPT * 32;  // keys per warp of a tile
constexpr int LBW = 8;          // predecessor status words read per look-back step

// (Two blocks per SM, as the kernel ran before the ballots: unbounded, the
// unrolled ballots of the 16 keys per thread take 254 registers.)
template <class K>
__global__ void __launch_bounds__(RT, 2) k_sort_pass(const K* __restrict__ kin, const u32* __restrict__ vin, K* __restrict__ kout,
                            u32* __restrict__ vout, u64 n, const u32* __restrict__ n_dev, int shift, u32 mask,
                            const u32* __restrict__ gofs, u64* status, u32* tile_ctr, u32 pass_tag, u32* err) {
  __shared__ u32 s_tile;
  __shared__ u32 s_base[RT];
  __shared__ u32 s_w[RT / 32][RT];  // per-warp digit counts, then per-warp digit starts
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const u32 lt = (1u << lane) - 1u;
  n = radix_count(n, n_dev);
  if (tid == 0) s_tile = atomicAdd(tile_ctr, 1u);
#pragma unroll
  for (int w = 0; w < RT / 32; ++w) s_w[w][tid] = 0;
  __syncthreads();
  const u64 t = s_tile;
  const u64 base = t * RTILE;
  if (base >= n) return;
  const u64 wbase = base + (u64)warp * KPW;
  // the warp's keys and values are loaded together up front (one memory
  // latency for the tile instead of one per iteration of the passes below)
  K kr[RIPT];
  u32 vr[RIPT];
#pragma unroll
  for (int r = 0; r < RIPT; ++r) {
    const u64 e = wbase + (u64)r * 32 + lane;
    kr[r] = e < n ? kin[e] : (K)0;
  }
#pragma unroll
  for (int r = 0; r < RIPT; ++r) {
    const u64 e = wbase + (u64)r * 32 + lane;
    vr[r] = e < n ? vin[e] : 0u;
  }
  // this warp's digit counts (a digit's leader lane adds its peers; leaders
  // of one iteration hold distinct digits, so no atomics are needed), and
  // each key's rank among the warp's keys of its digit (two 16-bit ranks
  // per word), which the scatter below reuses
  u32 wr[RIPT / 2];
#pragma unroll
  for (int r = 0; r < RIPT; ++r) {
    const u64 e = wbase + (u64)r * 32 + lane;
    const bool valid = e < n;
    const u32 dg = valid ? (u32)(kr[r] >> shift) & mask : 0xffffffffu;
    const u32 peers = digit_peers(dg, valid);
    const u32 rk = (valid ? s_w[warp][dg] : 0u) + __popc(peers & lt);
    if (r & 1) wr[r / 2] |= rk << 16;
    else wr[r / 2] = rk;
    __syncwarp();
    if (valid && lane == __ffs(peers) - 1) s_w[warp][dg] += __popc(peers);
    __syncwarp();
  }
  __syncthreads();
  // per digit (one per thread): the tile's count, and each warp's start
  // within the tile
  u32 c = 0;
#pragma unroll
  for (int w = 0; w < RT / 32; ++w) {
    const u32 cw = s_w[w][tid];
    s_w[w][tid] = c;
    c += cw;
  }
  // decoupled look-back, one digit per thread
  {
    volatile u64* st = status + t * RT + tid;
    const u64 tag = (u64)pass_tag << 32;
    u32 excl = 0;
    if (t == 0) {
      *st = ST_INC | tag | c;
    } else {
      *st = ST_AGG | tag | c;
      // walk back over the predecessors LBW at a time (their status words
      // are loaded together, so a walk over k tiles costs k / LBW round
      // trips), summing aggregates up to the first inclusive prefix
      u64 i = t;  // tiles below i are still to be read, from i - 1 down
      u64 t0 = 0;
      bool fin = false;
      while (!fin) {
        u64 v[LBW];
#pragma unroll
        for (int w = 0; w < LBW; ++w)
          v[w] = i > (u64)w ? *(volatile const u64*)(status + (i - 1 - w) * RT + tid) : 0ull;
        // take the ready words in order, stopping at the first one not ready
        int adv = 0;
#pragma unroll
        for (int w = 0; w < LBW; ++w) {
          if (fin || adv != w || i <= (u64)w) continue;
          const bool ready = ((v[w] >> 32) & 0xffu) == pass_tag && (v[w] >> 62) != 0;
          if (!ready) continue;
          excl += (u32)v[w];
          if ((v[w] & ST_INC) || i - 1 - (u64)w == 0) fin = true;
          adv = w + 1;
        }
        if (fin) break;
        if (adv == 0) {
          // the nearest predecessor has not counted yet: bounded wait
          if (t0 == 0) {
            t0 = sort_timer();
          } else if (sort_timer() - t0 > WAIT_NS_SORT) {
            if (err) atomicOr(err, ERR_TIMEOUT);
            break;
          }
          continue;
        }
        t0 = 0;
        i -= (u64)adv;
      }
      *st = ST_INC | tag | (excl + c);
    }
    s_base[tid] = gofs[tid] + excl;
  }
  __syncthreads();
  // stable scatter: a key goes to its digit's start in the output, plus its
  // warp's start within the tile's keys of that digit, plus its rank within
  // the warp's keys of that digit (from the count pass)
#pragma unroll
  for (int r = 0; r < RIPT; ++r) {
    const u64 e = wbase + (u64)r * 32 + lane;
    if (e >= n) continue;
    const K key = kr[r];
    const u32 dg = (u32)(key >> shift) & mask;
    const u32 pos = s_base[dg] + s_w[warp][dg] + ((wr[r / 2] >> (16 * (r & 1))) & 0xffffu);
    if (pos < n) {  // always, unless a look-back wait gave up (then err is set)
      kout[pos] = key;
      vout[pos] = vr[r];
    }
  }
}

// Inputs of at most SMALL_SORT_MAX keys are latency-bound: one block sorts
// them with the same stable LSD passes in one launch instead of two plus one
// per pass.  The keys and values of a pass are read from shared memory; the
// pass scatters them into the other global buffer of the pair (L2-resident
// at this size) and the next pass loads them back.  Warp w owns the
// elements [w * per, (w + 1) * per) in lane-strided order, so (warp,
// iteration, lane) is the input order, as in k_sort_pass, and the
// permutation is the same.
constexpr u32 SMALL_SORT_MAX = 4096;
constexpr size_t SMALL_DSMEM = (size_t)SMALL_SORT_MAX * (sizeof(u64) + sizeof(u32));

template <class K>
__global__ void __launch_bounds__(RT) k_sort_small(K* k0, K* k1, u32* v0, u32* v1, u64 n,
                                                   const u32* __restrict__ n_dev, int lo_bit, int npass,
                                                   int last_bits) {
  extern __shared__ __align__(16) unsigned char s_dyn[];
  __shared__ u32 s_w[RT / 32][RT];  // per-warp digit counts, then per-warp digit starts
  __shared__ u32 s_start[RT];       // start of each digit in the output
  __shared__ u32 s_sc[32];
  K* ks = reinterpret_cast<K*>(s_dyn);
  u32* vs = reinterpret_cast<u32*>(ks + SMALL_SORT_MAX);
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const u32 lt = (1u << lane) - 1u;
  const u32 m = (u32)radix_count(n, n_dev);
  // elements per warp, a multiple of 32 so every lane runs the same loop
  const u32 per = (m + RT - 1) / RT * 32;
  const u32 wb = warp * per;
  for (int p = 0; p < npass; ++p) {
    // pass p reads buffer p % 2 and writes buffer (p + 1) % 2
    const K* kin = (p & 1) ? k1 : k0;
    const u32* vin = (p & 1) ? v1 : v0;
    K* kout = (p & 1) ? k0 : k1;
    u32* vout = (p & 1) ? v0 : v1;
    for (u32 i = tid; i < m; i += RT) {
      ks[i] = kin[i];
      vs[i] = vin[i];
    }
    const int shift = lo_bit + 8 * p;
    const u32 mask = p == npass - 1 ? (1u << last_bits) - 1u : 0xffu;
#pragma unroll
    for (int w = 0; w < RT / 32; ++w) s_w[w][tid] = 0;
    __syncthreads();
    for (u32 it = 0; it < per; it += 32) {
      const u32 e = wb + it + lane;
      const bool valid = e < m;
      const u32 dg = valid ? (u32)(ks[e] >> shift) & mask : 0xffffffffu;
      const u32 peers = digit_peers(dg, valid);
      if (valid && lane == __ffs(peers) - 1) s_w[warp][dg] += __popc(peers);
      __syncwarp();
    }
    __syncthreads();
    u32 c = 0;
#pragma unroll
    for (int w = 0; w < RT / 32; ++w) {
      const u32 cw = s_w[w][tid];
      s_w[w][tid] = c;
      c += cw;
    }
    u32 agg;
    s_start[tid] = block_scan_incl(c, s_sc, &agg, OpAdd()) - c;
    __syncthreads();
    for (u32 it = 0; it < per; it += 32) {
      const u32 e = wb + it + lane;
      const bool valid = e < m;
      const K key = valid ? ks[e] : (K)0;
      const u32 dg = valid ? (u32)(key >> shift) & mask : 0xffffffffu;
      const u32 peers = digit_peers(dg, valid);
      if (valid) {
        const u32 pos = s_start[dg] + s_w[warp][dg] + __popc(peers & lt);
        kout[pos] = key;
        vout[pos] = vs[e];
      }
      __syncwarp();
      if (valid && lane == __ffs(peers) - 1) s_w[warp][dg] += __popc(peers);
      __syncwarp();
    }
    // the next pass reloads the buffer the block has just written
    __syncthreads();
  }
}

}  // namespace

size_t scan_tmp_words(u64 n) { return (size_t)((n + SCAN_TILE - 1) / SCAN_TILE) + 2; }
u64 scan_total_index(u64 n) { return (n + SCAN_TILE - 1) / SCAN_TILE; }

cudaError_t scan_u32(const u32* in, u32* out, u64 n, bool exclusive, bool use_max, u32* tmp,
                     cudaStream_t st) {
  return use_max ? scan_impl<u32, OpMax>(in, out, n, exclusive, tmp, st)
                 : scan_impl<u32, OpAdd>(in, out, n, exclusive, tmp, st);
}

cudaError_t scan_u8(const u8* in, u32* out, u64 n, bool exclusive, u32* tmp, cudaStream_t st) {
  return scan_impl<u8, OpAdd>(in, out, n, exclusive, tmp, st);
}

size_t radix_work_words(u64 n) {
  const u64 nb = (n + RTILE - 1) / RTILE;
  return W_STATUS + 2 * (size_t)RT * (size_t)(nb ? nb : 1);
}

namespace {

template <class K>
cudaError_t radix_sort_impl(K* k[2], u32* v[2], u64 n, int lo_bit, int hi_bit, u32* work, cudaStream_t st,
                            int* out_sel, const u32* n_dev, u32* err) {
  *out_sel = 0;
  if (n <= 1 || hi_bit <= lo_bit) return cudaSuccess;
  const int bits = hi_bit - lo_bit;
  const int npass = (bits + 7) / 8;
  if (npass > MAX_PASS || n >= (1ull << 32) || hi_bit > (int)(8 * sizeof(K))) return cudaErrorInvalidValue;
  const int last_bits = bits - 8 * (npass - 1);
  if (n <= SMALL_SORT_MAX) {
    cudaError_t e = cudaFuncSetAttribute(k_sort_small<K>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)SMALL_DSMEM);
    if (e != cudaSuccess) return e;
    note_launch();
    k_sort_small<K><<<1, RT, SMALL_DSMEM, st>>>(k[0], k[1], v[0], v[1], n, n_dev, lo_bit, npass, last_bits);
    *out_sel = npass & 1;  // the last pass wrote buffer npass % 2
    return cudaGetLastError();
  }
  const u64 nb = (n + RTILE - 1) / RTILE;
  u32* ghist = work + W_GHIST;
  u32* ctr = work + W_CTR;
  u64* status = reinterpret_cast<u64*>(work + W_STATUS);
  cudaError_t e = cudaMemsetAsync(work, 0, radix_work_words(n) * sizeof(u32), st);
  if (e != cudaSuccess) return e;
  note_launch();
  k_sort_hist<K><<<(unsigned)nb, RT, 0, st>>>(k[0], n, n_dev, lo_bit, npass, last_bits, ghist);
  note_launch();
  k_sort_scan<<<1, RT, 0, st>>>(ghist, npass);
  int sel = 0;
  for (int p = 0; p < npass; ++p) {
    const int shift = lo_bit + 8 * p;
    const u32 mask = p == npass - 1 ? (1u << last_bits) - 1u : 0xffu;
    note_launch();
    k_sort_pass<K><<<(unsigned)nb, RT, 0, st>>>(k[sel], v[sel], k[sel ^ 1], v[sel ^ 1], n, n_dev, shift, mask,
                                                ghist + (size_t)p * RT, status, ctr + p, (u32)(p + 1), err);
    sel ^= 1;
  }
  *out_sel = sel;
  return cudaGetLastError();
}

}  // namespace

cudaError_t radix_sort(u64* k[2], u32* v[2], u64 n, int lo_bit, int hi_bit, u32* work, cudaStream_t st,
                       int* out_sel, const u32* n_dev, u32* err) {
  return radix_sort_impl<u64>(k, v, n, lo_bit, hi_bit, work, st, out_sel, n_dev, err);
}

cudaError_t radix_sort(u32* k[2], u32* v[2], u64 n, int lo_bit, int hi_bit, u32* work, cudaStream_t st,
                       int* out_sel, const u32* n_dev, u32* err) {
  return radix_sort_impl<u32>(k, v, n, lo_bit, hi_bit, work, st, out_sel, n_dev, err);
}

}  // namespace sky
