// lsas_peak.cu -- FP32 FMA-pipe throughput microbenchmark.
//
// The fused receiver's FFT runs on the CUDA cores' FP32 pipe; its ALU
// roofline needs that pipe's peak as measured on this GPU, not a nominal
// lanes x clock figure.  fma_peak_kernel keeps NACC independent packed
// (f32x2) FMA chains per thread, so every warp always has an instruction
// ready and the pipe, not dependencies, sets the pace.
#include <cuda_runtime.h>

#include "lsas.h"

namespace {

constexpr int kNacc = 8;

__global__ void __launch_bounds__(512) fma_peak_kernel(int iters, float2 a, float2 b, float* out) {
  float2 acc[kNacc];
#pragma unroll
  for (int i = 0; i < kNacc; ++i)
    acc[i] = make_float2(static_cast<float>(threadIdx.x + i), static_cast<float>(blockIdx.x - i));
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int i = 0; i < kNacc; ++i) acc[i] = __ffma2_rn(acc[i], a, b);
  }
  float s = 0.f;
#pragma unroll
  for (int i = 0; i < kNacc; ++i) s += acc[i].x + acc[i].y;
  out[static_cast<size_t>(blockIdx.x) * blockDim.x + threadIdx.x] = s;
}

}  // namespace

extern "C" lsas_status lsas_fma_peak_run(int blocks, int threads, int iters, float* d_out,
                                         double* flops, void* stream) {
  if (blocks < 1 || threads < 32 || threads > 512 || threads % 32 != 0 || iters < 1 || !d_out)
    return LSAS_ERR_INVALID_ARG;
  // a and b keep every chain finite: acc -> 0.5 acc + 0.25 converges to 0.5
  fma_peak_kernel<<<blocks, threads, 0, static_cast<cudaStream_t>(stream)>>>(
      iters, make_float2(0.5f, 0.5f), make_float2(0.25f, 0.25f), d_out);
  if (cudaGetLastError() != cudaSuccess) return LSAS_ERR_CUDA;
  if (flops)
    *flops = static_cast<double>(blocks) * threads * static_cast<double>(iters) * kNacc * 2.0 * 2.0;
  return LSAS_OK;
}
