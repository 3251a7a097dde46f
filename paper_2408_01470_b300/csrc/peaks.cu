// Throughput probes of the SM pipes the hot path is bound by (the denominators of its roofline):
// FP32 FMA (scalar and the packed .f32x2 form), FP64 FMA and the MUFU ex2 approximation.
//
// Each thread runs 8 independent dependency chains of one operation for `iters` rounds, so the
// pipe, not the latency of one chain, limits the rate; the grid is a whole number of CTAs per SM.
// The kernels time themselves with CUDA events on the caller's stream after one warm-up launch
// (no clock or power setting is touched).  Built as its own library (libsabr_peaks.so): it is
// measurement infrastructure, not part of the calibration's C-ABI.
#include <cuda_runtime.h>
#include <cstdint>

namespace {

template <int KIND>
__global__ void __launch_bounds__(256) peak_kernel(int iters, float a, float b, double ad, double bd, float* sink,
                                                   double* sinkd) {
  if constexpr (KIND == 0) {   // FP32 FMA, scalar
    float x[8];
#pragma unroll
    for (int j = 0; j < 8; ++j) x[j] = (float)(threadIdx.x + j) * 1e-3f;
    for (int i = 0; i < iters; ++i)
#pragma unroll
      for (int j = 0; j < 8; ++j) x[j] = fmaf(x[j], a, b);
    float s = 0.f;
#pragma unroll
    for (int j = 0; j < 8; ++j) s += x[j];
    if (s == 1234.5f) sink[threadIdx.x] = s;
  } else if constexpr (KIND == 1) {   // FP32 FMA on register pairs (.f32x2): 2 FMAs per instruction
    float2 x[8];
#pragma unroll
    for (int j = 0; j < 8; ++j) x[j] = make_float2((float)(threadIdx.x + j) * 1e-3f, (float)j * 1e-3f);
    const float2 a2 = make_float2(a, a), b2 = make_float2(b, b);
    for (int i = 0; i < iters; ++i)
#pragma unroll
      for (int j = 0; j < 8; ++j) x[j] = __ffma2_rn(x[j], a2, b2);
    float s = 0.f;
#pragma unroll
    for (int j = 0; j < 8; ++j) s += x[j].x + x[j].y;
    if (s == 1234.5f) sink[threadIdx.x] = s;
  } else if constexpr (KIND == 2) {   // FP64 FMA
    double x[8];
#pragma unroll
    for (int j = 0; j < 8; ++j) x[j] = (double)(threadIdx.x + j) * 1e-3;
    for (int i = 0; i < iters; ++i)
#pragma unroll
      for (int j = 0; j < 8; ++j) x[j] = fma(x[j], ad, bd);
    double s = 0.0;
#pragma unroll
    for (int j = 0; j < 8; ++j) s += x[j];
    if (s == 1234.5) sinkd[threadIdx.x] = s;
  } else {   // MUFU: x <- 2^(-x), a contraction onto a fixed point in (0, 1) (no subnormals)
    float x[8];
#pragma unroll
    for (int j = 0; j < 8; ++j) x[j] = 0.5f + (float)j * 1e-2f;
    for (int i = 0; i < iters; ++i)
#pragma unroll
      for (int j = 0; j < 8; ++j) {
        float r;
        asm volatile("ex2.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(-x[j]));
        x[j] = r;
      }
    float s = 0.f;
#pragma unroll
    for (int j = 0; j < 8; ++j) s += x[j];
    if (s == 1234.5f) sink[threadIdx.x] = s;
  }
}

template <int KIND>
cudaError_t run(int blocks, int threads, int iters, cudaStream_t s, float* sink, double* sinkd) {
  peak_kernel<KIND><<<blocks, threads, 0, s>>>(iters, 0.999f, 1e-4f, 0.999, 1e-4, sink, sinkd);
  return cudaGetLastError();
}

}  // namespace

// kind: 0 FP32 FMA, 1 FP32 FMA on pairs, 2 FP64 FMA, 3 MUFU ex2.  Runs `blocks` CTAs of `threads`
// threads (<= 256), `iters` rounds of 8 operations per thread (x2 for kind 1), once untimed and
// once timed with events on `stream`.  Outputs: *seconds (device time of the timed launch) and
// *ops (operations of the timed launch: FMAs for kinds 0-2, ex2 evaluations for kind 3).  Returns
// 0, or the CUDA error code.
extern "C" int sabr_peak_probe(int kind, int blocks, int threads, int iters, void* stream, double* seconds,
                               double* ops) {
  if (kind < 0 || kind > 3 || blocks < 1 || threads < 32 || threads > 256 || iters < 1 || !seconds || !ops)
    return (int)cudaErrorInvalidValue;
  cudaStream_t s = (cudaStream_t)stream;
  float* sink = nullptr;
  double* sinkd = nullptr;
  cudaError_t e = cudaMalloc(&sink, 256 * sizeof(float));
  if (e == cudaSuccess) e = cudaMalloc(&sinkd, 256 * sizeof(double));
  cudaEvent_t a = nullptr, b = nullptr;
  if (e == cudaSuccess) e = cudaEventCreate(&a);
  if (e == cudaSuccess) e = cudaEventCreate(&b);
  auto launch = [&]() {
    switch (kind) {
      case 0: return run<0>(blocks, threads, iters, s, sink, sinkd);
      case 1: return run<1>(blocks, threads, iters, s, sink, sinkd);
      case 2: return run<2>(blocks, threads, iters, s, sink, sinkd);
      default: return run<3>(blocks, threads, iters, s, sink, sinkd);
    }
  };
  if (e == cudaSuccess) e = launch();
  if (e == cudaSuccess) e = cudaEventRecord(a, s);
  if (e == cudaSuccess) e = launch();
  if (e == cudaSuccess) e = cudaEventRecord(b, s);
  if (e == cudaSuccess) e = cudaEventSynchronize(b);
  float ms = 0.f;
  if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, a, b);
  if (a) cudaEventDestroy(a);
  if (b) cudaEventDestroy(b);
  if (sink) cudaFree(sink);
  if (sinkd) cudaFree(sinkd);
  if (e != cudaSuccess) return (int)e;
  *seconds = ms * 1e-3;
  *ops = (double)blocks * threads * (double)iters * 8.0 * (kind == 1 ? 2.0 : 1.0);
  return 0;
}
