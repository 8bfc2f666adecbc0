// sgwls_launch.cuh -- launch plan of one pass and the per-radius launchers.
#pragma once

#include "sgwls_pass.cuh"

namespace sgwls {

struct Plan {
  int h;          // lines per chunk
  int P;          // chunks per subsystem
  int warps_rec;  // warps (chunks) per k_recover block
  size_t smem_rec;
};

// Launches the kernels of one pass for a group of CC <= 4 channels.
using PassLauncher = cudaError_t (*)(const PassArgs&, const Plan&, int CC, cudaStream_t);

template <int R, int CC>
cudaError_t launch_pass_rc(const PassArgs& a, const Plan& pl, cudaStream_t st) {
  static_assert(R >= 1 && R <= kRMax, "radius");
  constexpr int OB = 32 - 2 * R;
  if (pl.smem_rec > 48 * 1024) {
    cudaError_t e = cudaFuncSetAttribute(k_recover<R, CC>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)pl.smem_rec);
    if (e != cudaSuccess) return e;
  }
  if (a.P > 1) {
    dim3 bs(32, 4), gs((a.nsys + 31) / 32, (a.P + 3) / 4);
    k_summary<R, CC><<<gs, bs, 0, st>>>(a);
    k_reduced<R, CC><<<(a.nsys + 127) / 128, 128, 0, st>>>(a);
  }
  dim3 br(32, pl.warps_rec), gr((a.D + OB - 1) / OB, (a.P + pl.warps_rec - 1) / pl.warps_rec);
  k_recover<R, CC><<<gr, br, pl.smem_rec, st>>>(a);
  return cudaGetLastError();
}

template <int R>
cudaError_t launch_pass_r(const PassArgs& a, const Plan& pl, int CC, cudaStream_t st) {
  switch (CC) {
    case 1: return launch_pass_rc<R, 1>(a, pl, st);
    case 2: return launch_pass_rc<R, 2>(a, pl, st);
    case 3: return launch_pass_rc<R, 3>(a, pl, st);
    case 4: return launch_pass_rc<R, 4>(a, pl, st);
    default: return cudaErrorInvalidValue;
  }
}

cudaError_t launch_pass_r1(const PassArgs&, const Plan&, int, cudaStream_t);
cudaError_t launch_pass_r2(const PassArgs&, const Plan&, int, cudaStream_t);
cudaError_t launch_pass_r3(const PassArgs&, const Plan&, int, cudaStream_t);
cudaError_t launch_pass_r4(const PassArgs&, const Plan&, int, cudaStream_t);
cudaError_t launch_pass_r5(const PassArgs&, const Plan&, int, cudaStream_t);
cudaError_t launch_pass_r6(const PassArgs&, const Plan&, int, cudaStream_t);
cudaError_t launch_pass_r7(const PassArgs&, const Plan&, int, cudaStream_t);
cudaError_t launch_pass_r8(const PassArgs&, const Plan&, int, cudaStream_t);

}  // namespace sgwls
