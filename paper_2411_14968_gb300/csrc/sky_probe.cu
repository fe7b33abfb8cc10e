// Compare-throughput probe (include/skyline_diag.h): the roofline
// denominator of the dominance kernels.  Each thread runs 8 independent
// predicate chains of FP32 "<=" compares (setp.le.and.f32, the form a
// dominance test's "all attributes <=" takes) over 64 distinct register
// operand pairs that change every iteration (8 FP32 adds per 64 compares),
// so the loop is compare-issue bound.
#include <cstdint>
#include "sky_internal.cuh"

namespace sky {
namespace {

__global__ void __launch_bounds__(256) k_probe_cmp(u32 iters, float seed, u32* sink) {
  float t0 = seed + threadIdx.x * 1e-7f, t1 = t0 + 0.5f, t2 = t0 + 0.25f, t3 = t0 + 0.125f;
  float t4 = t0 + 0.0625f, t5 = t0 + 0.375f, t6 = t0 + 0.625f, t7 = t0 + 0.75f;
  float w0 = 0.0f, w1 = 0.1f, w2 = 0.2f, w3 = 0.3f, w4 = 0.4f, w5 = 0.6f, w6 = 0.7f, w7 = 0.8f;
  u32 acc = 0;
  for (u32 i = 0; i < iters; ++i) {
    u32 r;
    // 64 distinct compares t_i <= w_j in 8 predicate chains (one per t_i)
    asm volatile(
        "{\n\t"
        ".reg .pred p0, p1, p2, p3, p4, p5, p6, p7;\n\t"
        "setp.le.f32 p0, %1, %9;\n\t"
        "setp.le.f32 p1, %2, %9;\n\t"
        "setp.le.f32 p2, %3, %9;\n\t"
        "setp.le.f32 p3, %4, %9;\n\t"
        "setp.le.f32 p4, %5, %9;\n\t"
        "setp.le.f32 p5, %6, %9;\n\t"
        "setp.le.f32 p6, %7, %9;\n\t"
        "setp.le.f32 p7, %8, %9;\n\t"
        "setp.le.and.f32 p0, %1, %10, p0;\n\t"
        "setp.le.and.f32 p1, %2, %10, p1;\n\t"
        "setp.le.and.f32 p2, %3, %10, p2;\n\t"
        "setp.le.and.f32 p3, %4, %10, p3;\n\t"
        "setp.le.and.f32 p4, %5, %10, p4;\n\t"
        "setp.le.and.f32 p5, %6, %10, p5;\n\t"
        "setp.le.and.f32 p6, %7, %10, p6;\n\t"
        "setp.le.and.f32 p7, %8, %10, p7;\n\t"
        "setp.le.and.f32 p0, %1, %11, p0;\n\t"
        "setp.le.and.f32 p1, %2, %11, p1;\n\t"
        "setp.le.and.f32 p2, %3, %11, p2;\n\t"
        "setp.le.and.f32 p3, %4, %11, p3;\n\t"
        "setp.le.and.f32 p4, %5, %11, p4;\n\t"
        "setp.le.and.f32 p5, %6, %11, p5;\n\t"
        "setp.le.and.f32 p6, %7, %11, p6;\n\t"
        "setp.le.and.f32 p7, %8, %11, p7;\n\t"
        "setp.le.and.f32 p0, %1, %12, p0;\n\t"
        "setp.le.and.f32 p1, %2, %12, p1;\n\t"
        "setp.le.and.f32 p2, %3, %12, p2;\n\t"
        "setp.le.and.f32 p3, %4, %12, p3;\n\t"
        "setp.le.and.f32 p4, %5, %12, p4;\n\t"
        "setp.le.and.f32 p5, %6, %12, p5;\n\t"
        "setp.le.and.f32 p6, %7, %12, p6;\n\t"
        "setp.le.and.f32 p7, %8, %12, p7;\n\t"
        "setp.le.and.f32 p0, %1, %13, p0;\n\t"
        "setp.le.and.f32 p1, %2, %13, p1;\n\t"
        "setp.le.and.f32 p2, %3, %13, p2;\n\t"
        "setp.le.and.f32 p3, %4, %13, p3;\n\t"
        "setp.le.and.f32 p4, %5, %13, p4;\n\t"
        "setp.le.and.f32 p5, %6, %13, p5;\n\t"
        "setp.le.and.f32 p6, %7, %13, p6;\n\t"
        "setp.le.and.f32 p7, %8, %13, p7;\n\t"
        "setp.le.and.f32 p0, %1, %14, p0;\n\t"
        "setp.le.and.f32 p1, %2, %14, p1;\n\t"
        "setp.le.and.f32 p2, %3, %14, p2;\n\t"
        "setp.le.and.f32 p3, %4, %14, p3;\n\t"
        "setp.le.and.f32 p4, %5, %14, p4;\n\t"
        "setp.le.and.f32 p5, %6, %14, p5;\n\t"
        "setp.le.and.f32 p6, %7, %14, p6;\n\t"
        "setp.le.and.f32 p7, %8, %14, p7;\n\t"
        "setp.le.and.f32 p0, %1, %15, p0;\n\t"
        "setp.le.and.f32 p1, %2, %15, p1;\n\t"
        "setp.le.and.f32 p2, %3, %15, p2;\n\t"
        "setp.le.and.f32 p3, %4, %15, p3;\n\t"
        "setp.le.and.f32 p4, %5, %15, p4;\n\t"
        "setp.le.and.f32 p5, %6, %15, p5;\n\t"
        "setp.le.and.f32 p6, %7, %15, p6;\n\t"
        "setp.le.and.f32 p7, %8, %15, p7;\n\t"
        "setp.le.and.f32 p0, %1, %16, p0;\n\t"
        "setp.le.and.f32 p1, %2, %16, p1;\n\t"
        "setp.le.and.f32 p2, %3, %16, p2;\n\t"
        "setp.le.and.f32 p3, %4, %16, p3;\n\t"
        "setp.le.and.f32 p4, %5, %16, p4;\n\t"
        "setp.le.and.f32 p5, %6, %16, p5;\n\t"
        "setp.le.and.f32 p6, %7, %16, p6;\n\t"
        "setp.le.and.f32 p7, %8, %16, p7;\n\t"
        "and.pred p0, p0, p1;\n\t and.pred p2, p2, p3;\n\t and.pred p4, p4, p5;\n\t"
        "and.pred p6, p6, p7;\n\t or.pred p0, p0, p2;\n\t or.pred p4, p4, p6;\n\t"
        "or.pred p0, p0, p4;\n\t"
        "selp.u32 %0, 1, 0, p0;\n\t"
        "}\n"
        : "=r"(r)
        : "f"(t0), "f"(t1), "f"(t2), "f"(t3), "f"(t4), "f"(t5), "f"(t6), "f"(t7),
          "f"(w0), "f"(w1), "f"(w2), "f"(w3), "f"(w4), "f"(w5), "f"(w6), "f"(w7));
    acc += r;
    w0 += 1e-6f;
    w1 += 1e-6f;
    w2 += 1e-6f;
    w3 += 1e-6f;
    w4 += 1e-6f;
    w5 += 1e-6f;
    w6 += 1e-6f;
    w7 += 1e-6f;
  }
  if (acc == 0xffffffffu) sink[0] = acc;  // keeps the loop live
}

}  // namespace

cudaError_t probe_compare_rate(u32 iters, cudaStream_t st, double* per_s, u32* sms_out, u32* sink) {
  int sms = device_sm_count();
  int per_sm = 0;
  cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_probe_cmp, 256, 0);
  if (e != cudaSuccess) return e;
  unsigned grid = (unsigned)(sms * (per_sm > 0 ? per_sm : 1));
  cudaEvent_t a, b;
  cudaEventCreate(&a);
  cudaEventCreate(&b);
  note_launch();
  k_probe_cmp<<<grid, 256, 0, st>>>(iters / 8 + 1, 0.5f, sink);  // warm-up
  cudaEventRecord(a, st);
  note_launch();
  k_probe_cmp<<<grid, 256, 0, st>>>(iters, 0.5f, sink);
  cudaEventRecord(b, st);
  e = cudaEventSynchronize(b);
  float ms = 0;
  cudaEventElapsedTime(&ms, a, b);
  cudaEventDestroy(a);
  cudaEventDestroy(b);
  if (e != cudaSuccess) return e;
  double compares = 64.0 * (double)iters * (double)grid * 256.0;
  *per_s = compares / (ms * 1e-3);
  *sms_out = (u32)sms;
  return cudaGetLastError();
}

}  // namespace sky
