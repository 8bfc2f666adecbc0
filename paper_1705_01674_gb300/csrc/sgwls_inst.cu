// One (radius, channel group) of the SG-WLS pass kernels.  build.py compiles
// this file once per pair with SGWLS_R (1..8) and SGWLS_CC (1..4) defined;
// with SGWLS_STUB_RADIUS the launchers only report "not supported" (the
// development shortcut that builds a subset of the radii).
#include "sgwls_launch.cuh"

#if !defined(SGWLS_R) || !defined(SGWLS_CC)
#error "compile with -DSGWLS_R=<radius> -DSGWLS_CC=<channels>"
#endif

namespace sgwls {

template <int R, int CC>
cudaError_t launch_pass_inst(const PassArgs& a, const Plan& pl, bool bwd, cudaStream_t st) {
#ifdef SGWLS_STUB_RADIUS
  (void)a, (void)pl, (void)bwd, (void)st;
  return cudaErrorNotSupported;
#else
  if (bwd) {
    // the backward solves u and v together: an even number of right-hand sides
    if constexpr (CC == 2 || CC == 4) return launch_pass_rc<R, CC, true>(a, pl, st);
    return cudaErrorInvalidValue;
  }
  return launch_pass_rc<R, CC, false>(a, pl, st);
#endif
}

template <int R, int CC>
cudaError_t launch_batch_inst(const BatchArgs& ba, const BatchLaunch& bl, cudaStream_t st) {
#ifdef SGWLS_STUB_RADIUS
  (void)ba, (void)bl, (void)st;
  return cudaErrorNotSupported;
#else
  return launch_batch_rc<R, CC>(ba, bl, st);
#endif
}

template cudaError_t launch_pass_inst<SGWLS_R, SGWLS_CC>(const PassArgs&, const Plan&, bool, cudaStream_t);
template cudaError_t launch_batch_inst<SGWLS_R, SGWLS_CC>(const BatchArgs&, const BatchLaunch&, cudaStream_t);

}  // namespace sgwls
