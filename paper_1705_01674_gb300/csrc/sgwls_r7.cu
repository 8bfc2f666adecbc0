// Kernels of one SG-WLS pass instantiated for neighbourhood radius r = 7.
#include "sgwls_launch.cuh"

namespace sgwls {
cudaError_t launch_pass_r7(const PassArgs& a, const Plan& pl, int CC, cudaStream_t st) {
#ifdef SGWLS_STUB_RADIUS
  (void)a, (void)pl, (void)CC, (void)st;
  return cudaErrorNotSupported;
#else
  return launch_pass_r<7>(a, pl, CC, st);
#endif
}

cudaError_t launch_batch_r7(const BatchArgs& ba, const BatchLaunch& bl, int CC, cudaStream_t st) {
#ifdef SGWLS_STUB_RADIUS
  (void)ba, (void)bl, (void)CC, (void)st;
  return cudaErrorNotSupported;
#else
  return launch_batch_r<7>(ba, bl, CC, st);
#endif
}
}  // namespace sgwls
