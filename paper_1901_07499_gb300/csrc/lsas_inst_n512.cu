// Kernels for N = 512 subcarriers.
#include "lsas_inst.cuh"

namespace lsas {
cudaError_t launch_n512(int kind, bool fc32, const KParams& p, int grid, int smem,
                      cudaStream_t st) {
  return launch_n<9>(kind, fc32, p, grid, smem, st);
}
}  // namespace lsas
