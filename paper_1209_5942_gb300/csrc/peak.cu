// peak.cu -- measured arithmetic peaks of the GPU the context runs on, the
// denominators of the roofline fractions of ALU-bound kernels: the IEEE-FP64
// hop is bound by the FP64 pipe and the float-float hop by the FP32 pipe,
// while the copy-bandwidth figure only bounds the memory-bound ones.
//
// Each thread runs 8 independent fused multiply-add chains x <- x * a + b
// (so the pipe, not the FMA latency, is the limit) over a grid of 8 blocks
// of 256 threads per SM; the FP32 form uses the packed two-lane FFMA2 of
// sm_100+ (two FMAs per instruction), which is how the float-float kernels
// issue most of their arithmetic.  The timed launch follows one warm-up
// launch; 2 flops per FMA.
#include <cuda_runtime.h>

#include "internal.h"

namespace lqcd {

__global__ void __launch_bounds__(256) fma_f64_kernel(double *out, int iters, double a, double b) {
  double x[8];
#pragma unroll
  for (int k = 0; k < 8; k++) x[k] = 1e-3 * (threadIdx.x + k);
#pragma unroll 2
  for (int i = 0; i < iters; i++) {
#pragma unroll
    for (int k = 0; k < 8; k++) x[k] = __fma_rn(x[k], a, b);
  }
  double s = 0.0;
#pragma unroll
  for (int k = 0; k < 8; k++) s += x[k];
  if (s == 12345.678) out[blockIdx.x] = s;  // never true: keeps the chains alive
}

__global__ void __launch_bounds__(256) fma_f32x2_kernel(float *out, int iters, float a, float b) {
  float2 x[8];
#pragma unroll
  for (int k = 0; k < 8; k++) x[k] = make_float2(1e-3f * (threadIdx.x + k), 2e-3f * (threadIdx.x + k));
  const float2 a2 = make_float2(a, a), b2 = make_float2(b, b);
#pragma unroll 2
  for (int i = 0; i < iters; i++) {
#pragma unroll
    for (int k = 0; k < 8; k++) x[k] = __ffma2_rn(x[k], a2, b2);
  }
  float s = 0.0f;
#pragma unroll
  for (int k = 0; k < 8; k++) s += x[k].x + x[k].y;
  if (s == 12345.678f) out[blockIdx.x] = s;
}

}  // namespace lqcd

using namespace lqcd;

extern "C" int lqcd_measure_peaks(lqcd_ctx *ctx, double *fp64_tflops, double *fp32_tflops) {
  if (!ctx || !fp64_tflops || !fp32_tflops) return LQCD_ERR_INVALID;
  LQCD_TRY(ensure_partials(ctx, 8 * (size_t)ctx->num_sms));
  const unsigned grid = 8u * (unsigned)ctx->num_sms;
  const unsigned block = 256;
  const int it64 = 1 << 12, it32 = 1 << 16;
  cudaEvent_t e0, e1;
  LQCD_CUDA(ctx, cudaEventCreate(&e0));
  if (cudaEventCreate(&e1) != cudaSuccess) {
    cudaEventDestroy(e0);
    return fail(ctx, LQCD_ERR_CUDA, "cudaEventCreate failed");
  }
  float ms64 = 0.0f, ms32 = 0.0f;
  cudaStream_t st = ctx->stream;
  fma_f64_kernel<<<grid, block, 0, st>>>(ctx->partials, it64, 0.999999, 1e-7);
  cudaEventRecord(e0, st);
  fma_f64_kernel<<<grid, block, 0, st>>>(ctx->partials, it64, 0.999999, 1e-7);
  cudaEventRecord(e1, st);
  cudaError_t e = cudaEventSynchronize(e1);
  if (e == cudaSuccess) e = cudaEventElapsedTime(&ms64, e0, e1);
  if (e == cudaSuccess) {
    fma_f32x2_kernel<<<grid, block, 0, st>>>((float *)ctx->partials, it32, 0.9999f, 1e-5f);
    cudaEventRecord(e0, st);
    fma_f32x2_kernel<<<grid, block, 0, st>>>((float *)ctx->partials, it32, 0.9999f, 1e-5f);
    cudaEventRecord(e1, st);
    e = cudaEventSynchronize(e1);
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms32, e0, e1);
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (e != cudaSuccess) return cuda_check(ctx, e, "peak microbenchmark");
  LQCD_CUDA(ctx, cudaGetLastError());
  const double threads = (double)grid * block;
  *fp64_tflops = threads * it64 * 8 * 2.0 / (ms64 * 1e-3) / 1e12;
  *fp32_tflops = threads * it32 * 8 * 2 * 2.0 / (ms32 * 1e-3) / 1e12;
  return LQCD_OK;
}
