// Kernels for N = 2048 subcarriers.
#include "lsas_inst.cuh"

namespace lsas {
cudaError_t launch_n2048(int kind, bool fc32, const KParams& p, int grid, int smem,
                      cudaStream_t st) {
  return launch_n<11>(kind, fc32, p, grid, smem, st);
}
}  // namespace lsas
