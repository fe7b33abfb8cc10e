// sky_skyline_static: the skyline of a small device-resident point set
// computed without allocating any memory.
//
// Some callers cannot call cudaMalloc at the moment they need a skyline: a
// host thread that runs under an allocator which forbids new device
// allocations (a framework that owns every byte of the GPU through its own
// pool), a latency-critical loop in which an allocation (and the device-wide
// synchronisation cudaFree may cause) is not acceptable, or code that must
// keep a fixed, known memory footprint.  For them this entry point runs the
// dominance kernel of the representative filter (every candidate tested
// against every point, Def. 1) with all of its scratch -- the padded points,
// the alive flags, the scan of the compaction and the error word -- in one
// file-scope device array whose size is fixed when the library is built.
// Every GPU that loads the library holds that array until the process exits.
//
// In host code the array's name only stands in for it: its device address
// is taken with cudaGetSymbolAddress once per device, on the first call made
// with that device current, and cached.  That first call should therefore
// come before any stream capture.  Inputs and outputs must be device memory
// of the current device (or managed memory); memory of another GPU is
// refused, since the kernels would read or write it through the peer path.
// Every call shares the array and finds the previous call's contents in it,
// so the call clears what must start at zero itself; calls whose work
// overlaps on the GPU (several host threads, or several streams) race on
// the array and must not be made.
#include <cstring>
#include <mutex>
#include "../../include/skyline.h"
#include "sky_internal.cuh"

namespace sky {
namespace {

constexpr size_t align256(size_t b) { return (b + 255) & ~(size_t)255; }

// Layout of the array (byte offsets).  The scan partials need
// scan_tmp_words(n) words, checked against the reserved room on every call.
constexpr u64 MAXN = SKY_STATIC_MAX_POINTS;
constexpr size_t OFF_PTS = 0;                                      // 2 float4 per point
constexpr size_t OFF_ALIVE = OFF_PTS + align256(MAXN * 32);        // u8 per point
constexpr size_t OFF_EXCL = OFF_ALIVE + align256(MAXN);            // u32 per point
constexpr size_t OFF_TMP = OFF_EXCL + align256(MAXN * 4);          // scan partials
constexpr size_t TMP_WORDS = 4096;
constexpr size_t OFF_ERR = OFF_TMP + align256(TMP_WORDS * 4);      // error word
constexpr size_t STATIC_BYTES = OFF_ERR + 256;

static __device__ __align__(256) unsigned char g_static_scratch[STATIC_BYTES];

constexpr int MAX_DEVICES = 64;
std::mutex g_mu;
unsigned char* g_addr[MAX_DEVICES] = {};

// Row-major input to padded points (+0.0 padding, -0.0 read as +0.0),
// every alive flag set, NaN flagged.
template <int D>
__global__ void k_static_pack(const float* __restrict__ X, u32 n, float4* __restrict__ pts, u8* __restrict__ alive,
                              u32* __restrict__ err) {
  u32 i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  float x[8] = {0, 0, 0, 0, 0, 0, 0, 0};
  bool nan = false;
#pragma unroll
  for (int a = 0; a < D; ++a) {
    float v = X[(u64)i * D + a];
    nan |= v != v;
    x[a] = v + 0.0f;
  }
  if (nan) atomicOr(err, ERR_NAN);
  constexpr int V = vec_of(D);
  pts[(u64)i * V] = make_float4(x[0], x[1], x[2], x[3]);
  if (V > 1) pts[(u64)i * V + 1] = make_float4(x[4], x[5], x[6], x[7]);
  alive[i] = 1;
}

// Device address of the array on the current device.  Set-up, on the first
// call with a device current: cudaGetSymbolAddress, cached per device.  A
// cached address is used only while the runtime still reports it as device
// memory of the current device; after a cudaDeviceReset the module (and the
// array) is loaded again, the old address is no longer valid, and the set-up
// runs again.
bool is_current_device_mem(const void* p) {
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  if (a.type == cudaMemoryTypeManaged) return true;
  int cur = -1;
  if (a.type != cudaMemoryTypeDevice || cudaGetDevice(&cur) != cudaSuccess) return false;
  return a.device == cur;
}

cudaError_t scratch_address(unsigned char** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= MAX_DEVICES) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> g(g_mu);
  if (!g_addr[dev] || !is_current_device_mem(g_addr[dev])) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_static_scratch);
    if (e != cudaSuccess) return e;
    g_addr[dev] = static_cast<unsigned char*>(p);
  }
  *out = g_addr[dev];
  return cudaSuccess;
}

}  // namespace
}  // namespace sky

using namespace sky;

extern "C" sky_status sky_skyline_static(const float* points, uint64_t n, uint32_t d, uint32_t* out_idx,
                                         uint64_t* out_count, void* cuda_stream) {
  if (!out_count) return SKY_EINVAL;
  *out_count = 0;
  if (d < 1 || d > 8) return SKY_EINVAL;
  if (n > SKY_STATIC_MAX_POINTS) return SKY_EINVAL;
  if (n == 0) return SKY_OK;
  if (!points || !out_idx || !is_current_device_mem(points) || !is_current_device_mem(out_idx)) return SKY_EINVAL;
  if (scan_tmp_words(n) > TMP_WORDS) return SKY_EINVAL;
  cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
  unsigned char* base = nullptr;
  if (scratch_address(&base) != cudaSuccess) return SKY_ECUDA;
  float* pts = reinterpret_cast<float*>(base + OFF_PTS);
  u8* alive = base + OFF_ALIVE;
  u32* excl = reinterpret_cast<u32*>(base + OFF_EXCL);
  u32* tmp = reinterpret_cast<u32*>(base + OFF_TMP);
  u32* err = reinterpret_cast<u32*>(base + OFF_ERR);
  const u32 nn = (u32)n;
  // the error word keeps the previous call's value: clear it
  if (cudaMemsetAsync(err, 0, sizeof(u32), st) != cudaSuccess) return SKY_ECUDA;
  cudaError_t e = dispatch_d((int)d, [&](auto D) {
    note_launch();
    k_static_pack<decltype(D)::value>
        <<<(nn + 255) / 256, 256, 0, st>>>(points, nn, reinterpret_cast<float4*>(pts), alive, err);
  });
  if (e != cudaSuccess) return SKY_ECUDA;
  // Def. 1 against every point: a point never dominates itself or a copy
  // of itself, so the survivors are exactly Sky(points)
  if (launch_relative(pts, alive, n, pts, nn, nullptr, (int)d, st) != cudaSuccess) return SKY_ECUDA;
  if (scan_u8(alive, excl, n, true, tmp, st) != cudaSuccess) return SKY_ECUDA;
  if (launch_compact_idx(alive, excl, n, out_idx, st) != cudaSuccess) return SKY_ECUDA;
  u32 words[2] = {0, 0};
  if (cudaMemcpyAsync(&words[0], tmp + scan_total_index(n), sizeof(u32), cudaMemcpyDeviceToHost, st) != cudaSuccess)
    return SKY_ECUDA;
  if (cudaMemcpyAsync(&words[1], err, sizeof(u32), cudaMemcpyDeviceToHost, st) != cudaSuccess) return SKY_ECUDA;
  if (cudaStreamSynchronize(st) != cudaSuccess) return SKY_ECUDA;
  if (words[1] & ERR_NAN) return SKY_EINVAL;
  *out_count = words[0];
  return SKY_OK;
}
