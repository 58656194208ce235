// Kernels for N = 1024 subcarriers.
#include "lsas_inst.cuh"

namespace lsas {
cudaError_t launch_n1024(int kind, bool fc32, const KParams& p, int grid, int smem,
                      cudaStream_t st) {
  return launch_n<10>(kind, fc32, p, grid, smem, st);
}
}  // namespace lsas
