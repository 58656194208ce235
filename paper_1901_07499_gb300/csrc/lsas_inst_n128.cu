// Kernels for N = 128 subcarriers.
#include "lsas_inst.cuh"

namespace lsas {
cudaError_t launch_n128(int kind, bool fc32, const KParams& p, int grid, int smem,
                      cudaStream_t st) {
  return launch_n<7>(kind, fc32, p, grid, smem, st);
}
}  // namespace lsas
