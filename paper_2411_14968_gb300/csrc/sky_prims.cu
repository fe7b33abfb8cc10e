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

template <class In, class Op>
cudaError_t scan_impl(const In* in, u32* out, u64 n, bool exclusive, u32* tmp, cudaStream_t st) {
  u64 nb = (n + SCAN_TILE - 1) / SCAN_TILE;
  if (nb == 0) {
    return cudaMemsetAsync(tmp, 0, sizeof(u32), st);
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

constexpr int RT = 256;       // threads per block == radix buckets
constexpr int RIPT = 16;      // keys per thread
constexpr u64 RTILE = (u64)RT * RIPT;

// n_dev (optional): the element count lives in device memory and may be
// below the capacity n the grid was sized for; blocks past it count nothing.
__device__ __forceinline__ u64 radix_count(u64 n, const u32* n_dev) {
  if (!n_dev) return n;
  u64 m = *n_dev;
  return m < n ? m : n;
}

__global__ void k_radix_hist(const u64* __restrict__ k, u64 n, const u32* __restrict__ n_dev, int shift, u32 mask,
                             u32* __restrict__ hist, u32 nb) {
  __shared__ u32 h[RT];
  const int tid = threadIdx.x, lane = tid & 31;
  n = radix_count(n, n_dev);
  h[tid] = 0;
  __syncthreads();
  u64 base = (u64)blockIdx.x * RTILE;
  for (int r = 0; r < RIPT; ++r) {
    u64 e = base + (u64)r * RT + tid;
    bool valid = e < n;
    u32 dg = valid ? (u32)(k[e] >> shift) & mask : 0xffffffffu;
    u32 peers = __match_any_sync(FULL, dg);
    if (valid && lane == __ffs(peers) - 1) atomicAdd(&h[dg], __popc(peers));
  }
  __syncthreads();
  hist[(u64)tid * nb + blockIdx.x] = h[tid];
}

// Stable scatter: elements keep their input order inside each digit.
__global__ void k_radix_scatter(const u64* __restrict__ kin, const u32* __restrict__ vin,
                                u64* __restrict__ kout, u32* __restrict__ vout, u64 n,
                                const u32* __restrict__ n_dev, int shift, u32 mask,
                                const u32* __restrict__ offs, u32 nb) {
  __shared__ u32 s_base[RT];
  __shared__ u32 s_w[RT / 32][RT];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  n = radix_count(n, n_dev);
  if ((u64)blockIdx.x * RTILE >= n) return;
  s_base[tid] = offs[(u64)tid * nb + blockIdx.x];
#pragma unroll
  for (int w = 0; w < RT / 32; ++w) s_w[w][tid] = 0;
  __syncthreads();
  u64 base = (u64)blockIdx.x * RTILE;
  for (int r = 0; r < RIPT; ++r) {
    u64 e = base + (u64)r * RT + tid;
    bool valid = e < n;
    u64 key = valid ? kin[e] : 0;
    u32 val = valid ? vin[e] : 0;
    u32 dg = valid ? (u32)(key >> shift) & mask : 0xffffffffu;
    u32 peers = __match_any_sync(FULL, dg);
    u32 rank = __popc(peers & ((1u << lane) - 1u));
    if (valid && lane == __ffs(peers) - 1) s_w[warp][dg] = __popc(peers);
    __syncthreads();
    {
      u32 run = s_base[tid];
#pragma unroll
      for (int w = 0; w < RT / 32; ++w) {
        u32 c = s_w[w][tid];
        s_w[w][tid] = run;
        run += c;
      }
      s_base[tid] = run;
    }
    __syncthreads();
    if (valid) {
      u32 pos = s_w[warp][dg] + rank;
      kout[pos] = key;
      vout[pos] = val;
    }
    __syncthreads();
#pragma unroll
    for (int w = 0; w < RT / 32; ++w) s_w[w][tid] = 0;
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

size_t radix_hist_words(u64 n) { return (size_t)RT * (size_t)((n + RTILE - 1) / RTILE) + 1; }

cudaError_t radix_sort(u64* k[2], u32* v[2], u64 n, int lo_bit, int hi_bit, u32* hist, u32* tmp,
                       cudaStream_t st, int* out_sel, const u32* n_dev) {
  int sel = 0;
  u64 nb = (n + RTILE - 1) / RTILE;
  if (n <= 1 || hi_bit <= lo_bit) {
    *out_sel = 0;
    return cudaSuccess;
  }
  for (int shift = lo_bit; shift < hi_bit; shift += 8) {
    int bits = hi_bit - shift < 8 ? hi_bit - shift : 8;
    u32 mask = (1u << bits) - 1u;
    note_launch();
    k_radix_hist<<<(unsigned)nb, RT, 0, st>>>(k[sel], n, n_dev, shift, mask, hist, (u32)nb);
    cudaError_t e = scan_u32(hist, hist, (u64)RT * nb, true, false, tmp, st);
    if (e != cudaSuccess) return e;
    note_launch();
    k_radix_scatter<<<(unsigned)nb, RT, 0, st>>>(k[sel], v[sel], k[sel ^ 1], v[sel ^ 1], n, n_dev, shift,
                                                  mask, hist, (u32)nb);
    sel ^= 1;
  }
  *out_sel = sel;
  return cudaGetLastError();
}

}  // namespace sky
