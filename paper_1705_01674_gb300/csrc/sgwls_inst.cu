// One (radius, channel group) of the SG-WLS pass kernels.  build.py compiles
// this file once per pair with SGWLS_R (1..8) and SGWLS_CC (1..4) defined,
// and once with SGWLS_R = 1, SGWLS_CC = 6 (the backward's u and v of three
// channels, backward kernels only);
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
    if constexpr (CC % 2 == 0) return launch_pass_rc<R, CC, true>(a, pl, st);
    return cudaErrorInvalidValue;
  }
  // more than kGroupMax right-hand sides: the backward's wide group only
  if constexpr (CC <= kGroupMax) return launch_pass_rc<R, CC, false>(a, pl, st);
  return cudaErrorInvalidValue;
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
#if SGWLS_CC <= 4
template cudaError_t launch_batch_inst<SGWLS_R, SGWLS_CC>(const BatchArgs&, const BatchLaunch&, cudaStream_t);
#endif

}  // namespace sgwls
