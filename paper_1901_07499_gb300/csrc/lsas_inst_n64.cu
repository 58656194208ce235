// Kernels for N = 64 subcarriers.
#include "lsas_inst.cuh"

namespace lsas {
cudaError_t launch_n64(int kind, bool fc32, const KParams& p, int grid, int smem,
                      cudaStream_t st) {
  return launch_n<6>(kind, fc32, p, grid, smem, st);
}
}  // namespace lsas
