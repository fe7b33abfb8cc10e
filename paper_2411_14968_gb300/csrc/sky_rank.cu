// Rank space of a point set: every attribute replaced by its dense rank in
// its column.  Def. 1 compares each attribute of two points only by order,
// so a strictly increasing map of each column (the dense rank is one) keeps
// every dominance relation, and with it every skyline.
//
// The engine uses the ranks as the 16-bit images of its first test (the
// FP16 sign test of sky_engine_impl.cuh, which needs images that are
// non-decreasing in the value and finite): code = rank while the column has
// at most RANK_CODES distinct values -- the bit patterns 0x0000..0x7BFF are
// the finite non-negative FP16 numbers in increasing order, so distinct
// values keep distinct codes -- else rank scaled down to RANK_CODES levels.
// Unlike the FP16 rounding of the values themselves, these images separate
// the values of a column however they are spread (a common offset, very
// large or very small magnitudes).
//
// One column at a time: sort (value key, index) pairs by the value's
// monotone unsigned image (the radix sort of sky_prims.cu, on 32-bit keys),
// flag the sorted positions whose value differs from the previous one, an
// inclusive scan of the flags gives rank + 1 (and, as its total, the number
// of distinct values), and a scatter writes the rank at the point's own
// index of the column's rank array.  One last kernel then writes ranks and
// codes row-major from the column arrays.
#include <cstring>
#include <string>
#include "sky_pipeline.cuh"

namespace sky {

namespace {

constexpr int RT = 256;
inline unsigned rgrid(u64 n) { return (unsigned)((n + RT - 1) / RT); }

// Sort keys of attribute a: fkey of the value (-0.0 read as +0.0), with the
// point's index as the sort's value.  A NaN is flagged (and sorted as 0).
__global__ void k_rank_keys(const float* __restrict__ X, u64 n, u32 d, u32 a, u32* __restrict__ keys,
                            u32* __restrict__ vals, u32* err) {
  const u64 i = (u64)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  float v = X[i * d + a];
  if (v != v) {
    atomicOr(err, ERR_NAN);
    v = 0.0f;
  }
  keys[i] = fkey(__fadd_rn(v, 0.0f));
  vals[i] = (u32)i;
}

// flag[r] = 1 where sorted position r starts a run of equal values.
__global__ void k_rank_heads(const u32* __restrict__ keys, u64 n, u8* __restrict__ flag) {
  const u64 r = (u64)blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= n) return;
  flag[r] = (r == 0 || keys[r] != keys[r - 1]) ? 1 : 0;
}

// incl[r] - 1 is the dense rank of the value at sorted position r; it goes
// to the point's own index in the column's rank array (random 4-byte writes
// into one n-word array, which stays in L2 for the columns of up to tens of
// millions of points), and *total (the scan's total, the column's number of
// distinct values) to distinct[a].
__global__ void k_rank_scatter(const u32* __restrict__ sorted_idx, const u32* __restrict__ incl, u64 n,
                               const u32* __restrict__ total, u32* __restrict__ col, u32* __restrict__ distinct,
                               u32 a) {
  const u64 r = (u64)blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= n) return;
  col[sorted_idx[r]] = incl[r] - 1;
  if (r == 0) distinct[a] = *total;
}

// Row-major outputs from the column rank arrays (cols[a * n + i]), one
// point per thread, coalesced on both sides: ranks[i*d + a] (optional), the
// codes of the rank images -- codes[i*d + a] (optional), or packed as one
// uint4 of eight halves per point with the halves past d zero (optional).
__global__ void k_rank_pack(const u32* __restrict__ cols, u64 n, u32 d, const u32* __restrict__ distinct,
                            u32* __restrict__ ranks, unsigned short* __restrict__ codes,
                            uint4* __restrict__ packed) {
  const u64 i = (u64)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  u32 c[8];
#pragma unroll
  for (int a = 0; a < 8; ++a) {
    c[a] = 0;
    if ((u32)a < d) {
      const u32 rank = cols[(u64)a * n + i];
      if (ranks) ranks[i * d + a] = rank;
      c[a] = rank_code(rank, distinct[a]);
      if (codes) codes[i * d + a] = (unsigned short)c[a];
    }
  }
  if (packed) packed[i] = make_uint4(c[0] | c[1] << 16, c[2] | c[3] << 16, c[4] | c[5] << 16, c[6] | c[7] << 16);
}

// Bump allocator over the Runner's workspace (sizes rounded to 256 bytes).
struct Bump {
  char* base;
  size_t off = 0;
  template <class T>
  T* take(size_t count) {
    const size_t bytes = (count * sizeof(T) + 255) & ~(size_t)255;
    T* p = base ? reinterpret_cast<T*>(base + off) : nullptr;
    off += bytes ? bytes : 256;
    return p;
  }
};

}  // namespace

cudaError_t launch_rank_space(const float* X, u64 n, u32 d, const RankScratch& s, u32* ranks,
                              unsigned short* codes, uint4* packed, u32* distinct, u32* err, cudaStream_t st) {
  if (n == 0) return cudaSuccess;
  const u32* total = s.scan_tmp + scan_total_index(n);
  // 32-bit sort keys in the key buffers
  u32* k2[2] = {reinterpret_cast<u32*>(s.keys[0]), reinterpret_cast<u32*>(s.keys[1])};
  for (u32 a = 0; a < d; ++a) {
    note_launch();
    k_rank_keys<<<rgrid(n), RT, 0, st>>>(X, n, d, a, k2[0], s.vals[0], err);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    u32* v2[2] = {s.vals[0], s.vals[1]};
    int sel = 0;
    e = radix_sort(k2, v2, n, 0, 32, s.work, st, &sel, nullptr, err);
    if (e != cudaSuccess) return e;
    note_launch();
    k_rank_heads<<<rgrid(n), RT, 0, st>>>(k2[sel], n, s.flag);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    e = scan_u8(s.flag, s.incl, n, false, s.scan_tmp, st);
    if (e != cudaSuccess) return e;
    note_launch();
    k_rank_scatter<<<rgrid(n), RT, 0, st>>>(s.vals[sel], s.incl, n, total, s.cols + (u64)a * n, distinct, a);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  }
  note_launch();
  k_rank_pack<<<rgrid(n), RT, 0, st>>>(s.cols, n, d, distinct, ranks, codes, packed);
  return cudaGetLastError();
}

#define RCK(expr)                                                                              \
  do {                                                                                         \
    cudaError_t e_ = (expr);                                                                   \
    if (e_ != cudaSuccess) return fail(SKY_ECUDA, std::string(#expr) + ": " + cudaGetErrorString(e_)); \
  } while (0)

sky_status Runner::rank_space(const float* points, u64 n, u32 d, u32* out_ranks, u32* out_distinct,
                              unsigned short* out_codes) {
  memset(&stats, 0, sizeof(stats));
  RCK(cudaSetDevice(device));
  if (d < 1 || d > 8) return fail(SKY_EINVAL, "d must be in 1..8");
  if (n >= (1ull << 32) - 1) return fail(SKY_EINVAL, "N must be below 2^32 - 1");
  if (n > 0 && !points) return fail(SKY_EINVAL, "points is NULL");
  for (const void* p : {(const void*)points, (const void*)out_ranks, (const void*)out_distinct,
                        (const void*)out_codes})
    if (p && pointer_kind(p) == PTR_OTHER_DEVICE)
      return fail(SKY_EINVAL, "a buffer is device memory of another GPU than the context's");
  const bool distinct_dev = out_distinct && is_device_ptr(out_distinct);
  if (n == 0) {
    if (out_distinct) {
      if (distinct_dev) {
        RCK(cudaMemsetAsync(out_distinct, 0, d * sizeof(u32), stream));
        RCK(cudaStreamSynchronize(stream));
      } else {
        memset(out_distinct, 0, d * sizeof(u32));
      }
    }
    return SKY_OK;
  }
  const bool x_host = !is_device_ptr(points);
  const bool ranks_host = out_ranks && !is_device_ptr(out_ranks);
  const bool codes_host = out_codes && !is_device_ptr(out_codes);
  const u64 L = n * d;
  auto lay = [&](Bump& c, RankScratch* s, const float** X, u32** rk, unsigned short** cd, u32** dist, u32** err) {
    *X = x_host ? c.take<float>(L) : points;
    s->keys[0] = c.take<u64>(n);
    s->keys[1] = c.take<u64>(n);
    s->vals[0] = c.take<u32>(n);
    s->vals[1] = c.take<u32>(n);
    s->work = c.take<u32>(radix_work_words(n));
    s->flag = c.take<u8>(n);
    s->incl = c.take<u32>(n);
    s->scan_tmp = c.take<u32>(scan_tmp_words(n));
    s->cols = c.take<u32>(L);
    *rk = ranks_host ? c.take<u32>(L) : out_ranks;
    *cd = codes_host ? c.take<unsigned short>(L) : out_codes;
    *dist = c.take<u32>(8);
    *err = c.take<u32>(1);
  };
  RankScratch s{};
  const float* X = nullptr;
  u32 *rk = nullptr, *dist = nullptr, *err = nullptr;
  unsigned short* cd = nullptr;
  Bump sizing{nullptr};
  lay(sizing, &s, &X, &rk, &cd, &dist, &err);
  sky_status ss = ensure_ws(sizing.off);
  if (ss != SKY_OK) return ss;
  ss = ensure_pinned(9);
  if (ss != SKY_OK) return ss;
  Bump c{ws_};
  lay(c, &s, &X, &rk, &cd, &dist, &err);
  const u64 l0 = launch_counter();
  if (x_host) RCK(cudaMemcpyAsync(const_cast<float*>(X), points, L * sizeof(float), cudaMemcpyHostToDevice, stream));
  RCK(cudaMemsetAsync(err, 0, sizeof(u32), stream));
  if (timing) RCK(cudaEventRecord(ev_[0], stream));
  RCK(launch_rank_space(X, n, d, s, rk, cd, nullptr, dist, err, stream));
  if (timing) RCK(cudaEventRecord(ev_[1], stream));
  if (ranks_host) RCK(cudaMemcpyAsync(out_ranks, rk, L * sizeof(u32), cudaMemcpyDeviceToHost, stream));
  if (codes_host) RCK(cudaMemcpyAsync(out_codes, cd, L * sizeof(unsigned short), cudaMemcpyDeviceToHost, stream));
  if (out_distinct)
    RCK(cudaMemcpyAsync(out_distinct, dist, d * sizeof(u32),
                        distinct_dev ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, stream));
  RCK(cudaMemcpyAsync(pinned_, err, sizeof(u32), cudaMemcpyDeviceToHost, stream));
  RCK(cudaStreamSynchronize(stream));
  stats.n = n;
  stats.d = d;
  stats.launches = launch_counter() - l0;
  if (timing) {
    float ms = 0;
    RCK(cudaEventElapsedTime(&ms, ev_[0], ev_[1]));
    stats.ms_total = ms;  // the kernels only (no host copies)
  }
  const u32 e = pinned_[0];
  if (e & ERR_NAN) return fail(SKY_EINVAL, "input contains NaN");
  if (e & ERR_TIMEOUT) return fail(SKY_ETIMEOUT, "a device-side wait timed out");
  return SKY_OK;
}

}  // namespace sky
