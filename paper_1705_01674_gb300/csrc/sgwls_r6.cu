// Kernels of one SG-WLS pass instantiated for neighbourhood radius r = 6.
#include "sgwls_launch.cuh"

namespace sgwls {
cudaError_t launch_pass_r6(const PassArgs& a, const Plan& pl, int CC, cudaStream_t st) {
#ifdef SGWLS_STUB_RADIUS
  (void)a, (void)pl, (void)CC, (void)st;
  return cudaErrorNotSupported;
#else
  return launch_pass_r<6>(a, pl, CC, st);
#endif
}

cudaError_t launch_batch_r6(const BatchArgs& ba, const BatchLaunch& bl, int CC, cudaStream_t st) {
#ifdef SGWLS_STUB_RADIUS
  (void)ba, (void)bl, (void)CC, (void)st;
  return cudaErrorNotSupported;
#else
  return launch_batch_r<6>(ba, bl, CC, st);
#endif
}
}  // namespace sgwls
