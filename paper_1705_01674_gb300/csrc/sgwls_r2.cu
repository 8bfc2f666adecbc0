// Kernels of one SG-WLS pass instantiated for neighbourhood radius r = 2.
#include "sgwls_launch.cuh"

namespace sgwls {
cudaError_t launch_pass_r2(const PassArgs& a, const Plan& pl, int CC, cudaStream_t st) {
  return launch_pass_r<2>(a, pl, CC, st);
}
}  // namespace sgwls
