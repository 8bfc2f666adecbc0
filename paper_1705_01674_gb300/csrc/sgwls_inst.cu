// One (radius, channel group) of the SG-WLS pass kernels.  build.py compiles
// this file once per pair with SGWLS_R (1..8) and SGWLS_CC (1..4) defined,
// and once with SGWLS_R = 1, SGWLS_CC = 6 (the backward's u and v of three
// channels, backward kernels only); even CC also carry the batched
// backward's kernels (u and v of CC / 2 channels);
// with SGWLS_STUB_RADIUS the launchers only report "not supported" (the
// development shortcut that builds a subset of the radii).
#include "sgwls_launch.cuh"
#include "sgwls_line.cuh"

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

template <int R, int CC>
cudaError_t launch_batch_bwd_inst(const BatchArgs& ba, const BatchLaunch& bl, cudaStream_t st) {
#ifdef SGWLS_STUB_RADIUS
  (void)ba, (void)bl, (void)st;
  return cudaErrorNotSupported;
#else
  return launch_batch_bwd_rc<R, CC>(ba, bl, st);
#endif
}

template <int R, int CC>
cudaError_t launch_line_inst(const LineArgs& a, cudaStream_t st) {
#ifdef SGWLS_STUB_RADIUS
  (void)a, (void)st;
  return cudaErrorNotSupported;
#else
  const int nlines = a.dir == 1 ? a.H : a.W;
  cudaError_t e = launch_pdl(k_line_pass<R, CC>, dim3((nlines + 127) / 128), dim3(128), 0, st, a);
  return e != cudaSuccess ? e : cudaGetLastError();
#endif
}

template cudaError_t launch_pass_inst<SGWLS_R, SGWLS_CC>(const PassArgs&, const Plan&, bool, cudaStream_t);
#if SGWLS_R <= 4 && SGWLS_CC <= 4
template cudaError_t launch_line_inst<SGWLS_R, SGWLS_CC>(const LineArgs&, cudaStream_t);
#endif
#if SGWLS_CC % 2 == 0
template cudaError_t launch_batch_bwd_inst<SGWLS_R, SGWLS_CC>(const BatchArgs&, const BatchLaunch&, cudaStream_t);
#endif
#if SGWLS_CC <= 4
template cudaError_t launch_batch_inst<SGWLS_R, SGWLS_CC>(const BatchArgs&, const BatchLaunch&, cudaStream_t);
#endif

}  // namespace sgwls
