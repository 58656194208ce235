// lsas_inst.cuh -- launch wrapper of one FFT length; each lsas_inst_n*.cu
// includes it once so that the six lengths compile in parallel.
#pragma once
#include "lsas_kernels.cuh"
#include "lsas_warp.cuh"
#include "lsas_hyb.cuh"
#include "lsas_pair.cuh"
#include "lsas_twin.cuh"
#include "lsas_twinpair.cuh"

namespace lsas {

template <int LOG2N, bool FC32>
static cudaError_t launch_t(int kind, const KParams& p, int grid, int smem, cudaStream_t st) {
  void (*fn)(const KParams) = nullptr;
  int threads = Geo<LOG2N>::TW;
  int slot = kind;   // entry of the shared-memory attribute cache below
  if (kind == kKindFrame) {
    // fused receiver: from aligned sc16 rows, two symbols per step for
    // N = 1024 (and N = 256, 512 with enough antennas; per-warp pipelines)
    // and N = 2048 (pipelines of warp pairs), or, opt-in at N = 1024, the
    // second FFT pass on the tensor cores; otherwise one symbol per step: per-warp pipelines up to
    // N = 1024, pipelines of warp pairs for N = 2048 from sc16 rows and the
    // warp-specialised producer/consumer kernel for N = 2048 from fc32 rows
    if constexpr (LOG2N == 10 && !FC32) {
      if (p.hybrid && p.use_tma) {
        fn = hyb_kernel<false>;
        threads = kHyThreads;
        smem = kHySmem;
        slot = 3;
      } else if (p.twin && p.use_tma && (p.mode == kModeRun || p.mode == kModePartial)) {
        fn = twin_kernel<LOG2N>;
        slot = 4;
        threads = kTwThreads;
        smem = make_twlayout().total;
      } else {
        fn = warp_kernel<LOG2N, FC32>;
        threads = 32 * wgeo_warps(4);
      }
    } else if constexpr ((LOG2N == 8 || LOG2N == 9) && !FC32) {
      // p.twin is set by the plan only with enough antennas at these sizes
      if (p.twin && p.use_tma && (p.mode == kModeRun || p.mode == kModePartial)) {
        fn = twin_kernel<LOG2N>;
        slot = 4;
        threads = kTwThreads;
        smem = make_twlayout().total;
      } else {
        fn = warp_kernel<LOG2N, FC32>;
        threads = 32 * wgeo_warps(4);
      }
    } else if constexpr (LOG2N <= 10) {
      fn = warp_kernel<LOG2N, FC32>;
      threads = 32 * wgeo_warps(FC32 ? 8 : 4);
    } else if constexpr (!FC32) {
      if (p.twin && p.use_tma && (p.mode == kModeRun || p.mode == kModePartial)) {
        fn = twinpair_kernel<LOG2N>;
        threads = kTpThreads;
        smem = make_tplayout().total;
        slot = 4;
      } else {
        fn = pair_kernel<LOG2N>;
        threads = kPThreads;
      }
    } else {
      fn = frame_kernel<LOG2N, FC32>;
      threads = Geo<LOG2N>::T;
    }
  } else if (kind == kKindEstimate) {
    fn = estimate_kernel<LOG2N, FC32>;
  } else {
    fn = fft_kernel<LOG2N, FC32>;
  }
  // raise the kernel's dynamic shared memory limit once per device
  static int limit[5][64] = {};
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= 64 || smem > limit[slot][dev]) {
    e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e != cudaSuccess) return e;
    if (dev >= 0 && dev < 64) limit[slot][dev] = smem;
  }
  // group layers (partial mode, small batches): the two-symbol kernel groups
  // the data symbols its own way
  const int gz = !p.group_z ? 1 : (slot == 4 ? twin_groups(p.D) : p.groups);
  fn<<<dim3(grid, p.grid_y > 1 ? p.grid_y : 1, gz), threads, smem, st>>>(p);
  return cudaGetLastError();
}

template <int LOG2N>
cudaError_t launch_n(int kind, bool fc32, const KParams& p, int grid, int smem,
                     cudaStream_t st) {
  return fc32 ? launch_t<LOG2N, true>(kind, p, grid, smem, st)
              : launch_t<LOG2N, false>(kind, p, grid, smem, st);
}

}  // namespace lsas
