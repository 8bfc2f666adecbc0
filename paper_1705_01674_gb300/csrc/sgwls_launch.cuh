// sgwls_launch.cuh -- launch plan of one pass and the per-radius launchers.
#pragma once

#include <algorithm>

#include "sgwls_batch.cuh"

namespace sgwls {

struct Plan {
  int h;          // lines per chunk
  int P;          // chunks per subsystem
  int G;          // chunks (warps) per block
  int NG;         // chunk groups = ceil(P / G)
  size_t smem_sum, smem_rec;
  int queue = 0;  // the pass runs as the queue-scheduled k_pass_q
  int nslot = 0;  // its factor-store ring slots (0: one per band)
};

// Least number of bands between a band's summary items and the
// back-substitution items of the queue-scheduled pass; a ring needs at least
// look-ahead + 2 slots.
constexpr int kLookahead = 2;

// Shared memory of the two tiled kernels for a plan (bytes); gc guidance
// planes.
inline size_t tile_floats(int r, int CC, int h, int G, int step = 1, int gc = 1) {
  const int ncol = tile_ncol(r, step);
  return (size_t)(CC + gc) * tile_pstride(G * h + 2, std::max(tile_pitch_n(ncol, 0), tile_pitch_n(ncol, 1)));
}
// k_summary: the strip tile and the chunk 2-ports (in the same memory for
// radius <= 3, see tile_over_2ports).
inline size_t smem_summary(int r, int CC, int h, int G, int step = 1, int gc = 1) {
  const size_t tile = tile_floats(r, CC, h, G, step, gc), ports = (size_t)G * (3 * r * r + 2 * r * CC) * 32;
  return 4 * (tile_over_2ports(r) ? std::max(tile, ports) : tile + ports);
}
inline size_t smem_recover(int r, int CC, int h, int G, bool bwd = false) {
  const int n = 2 * r + 1;
  const size_t merge = (size_t)(G - 1) * (3 * r * r + r * CC) * 32 + 2 * (size_t)r * CC * 32;
  const int nout = bwd ? CC / 2 : CC;
  const size_t otile = (size_t)nout * (32 - 2 * r) * ((G * h) | 1);
  const size_t gacc = bwd ? (size_t)(G * h + 2) * (32 + 2 * r) : 0;
  return 4 * (tile_floats(r, CC, h, G) + (size_t)G * 2 * r * CC * 32 + merge + (size_t)G * h * n * (r + CC) * 32 +
              otile + gacc);
}

// k_backsub: group ports and merge factors, plus the row-direction output
// staging; with a sliding step > 1 also each warp's accumulation rows; the
// adjoint (bwd, CC = u and v planes) writes CC / 2 planes and adds the
// guidance tile and its dLoss/dG accumulators.
// dir < 0: the larger of the two directions; the column direction's
// forward pass at step 1 writes its output lines directly (no output tile).
inline size_t smem_backsub(int r, int CC, int h, int G, int step = 1, bool bwd = false, int dir = -1) {
  const size_t merge = (size_t)(G - 1) * (3 * r * r + r * CC) * 32 + 2 * (size_t)r * CC * 32;
  const bool no_otile = dir == 0 && step == 1 && !bwd;
  const size_t otile = no_otile ? 0 : (size_t)(bwd ? CC / 2 : CC) * step_own_max(r, step) * ((G * h) | 1);
  const size_t accum = step > 1 ? (size_t)G * (CC + 1) * step_acc_width(r, step) : 0;
  const size_t gtile = bwd ? 2 * (size_t)(G * h + 2) * (32 + 2 * r) : 0;
  return 4 * ((size_t)G * 2 * r * CC * 32 + merge + otile + accum + gtile);
}

constexpr size_t kReducedSmemMax = 96 * 1024;


// Launch with programmatic stream serialization (the kernels synchronise
// with griddep_wait before they consume the previous kernel's output).
template <typename... KArgs, typename... Args>
cudaError_t launch_pdl(void (*kernel)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t st,
                       Args&&... args) {
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, kernel, std::forward<Args>(args)...);
}

// Raises a kernel's dynamic shared-memory limit once per (kernel, device):
// later launches (for example inside a CUDA-graph capture) make no call.
cudaError_t set_smem_raw(const void* kernel, size_t bytes);

// Blocks of `kernel` (32 x G threads, `smem` dynamic bytes) resident on the
// whole current device, cached per (kernel, G, smem, device).
cudaError_t resident_blocks(const void* kernel, int G, size_t smem, int* out);

// (The default limit of 48 KB covers static and dynamic shared memory
// together: the batched kernels hold their argument block in static shared
// memory, so the attribute is raised from 32 KB of dynamic memory on.)
template <typename K>
cudaError_t set_smem(K kernel, size_t bytes) {
  if (bytes <= 32 * 1024) return cudaSuccess;
  return set_smem_raw(reinterpret_cast<const void*>(kernel), bytes);
}

template <int R, int CC, bool BWD = false>
cudaError_t launch_pass_rc(const PassArgs& a, const Plan& pl, cudaStream_t st);

// Refined pass (refine = 1): first solve keeping every entry's solution,
// the FP32 residual, the solve of the residual (same factors recomputed
// from the same tile) adding the first solution, then the averaging.
template <int R, int CC>
cudaError_t launch_refined_pass(const PassArgs& a, const Plan& pl, cudaStream_t st) {
  cudaError_t e;
  PassArgs b = a;
  b.refine = 0;
  b.xmode = 1;
  b.rhs = nullptr;
  if ((e = launch_pass_rc<R, CC>(b, pl, st)) != cudaSuccess) return e;
  b.rhs = a.rhs;
  const int gy = pl.G;
  e = launch_pdl(k_resid<R, CC>, dim3((a.nsys + 31) / 32, (a.L + 4 * gy - 1) / (4 * gy)), dim3(32, gy), 0, st, b);
  if (e != cudaSuccess) return e;
  b.xmode = 2;
  return launch_pass_rc<R, CC>(b, pl, st);
}

template <int R, int CC, bool BWD>
cudaError_t launch_pass_rc(const PassArgs& a, const Plan& pl, cudaStream_t st) {
  static_assert(R >= 1 && R <= kRMax, "radius");
  if constexpr (!BWD) {
    if (a.refine) return launch_refined_pass<R, CC>(a, pl, st);
  }
  constexpr int OB = 32 - 2 * R;
  cudaError_t e;
  PassArgs b = a;
  b.early_stage = a.P > 1 ? 1 : 0;   // k_recover follows k_summary
  // factors are kept by k_summary for k_backsub (one chunk: k_recover alone);
  // the adjoint keeps them for k_backsub's adjoint mode at step 1 only
  if (a.P < 2 || (BWD && a.step != 1)) b.fac = b.psi = nullptr;
  // a vector guidance is read by the keeping k_summary<..., 3> alone
  if (a.gc > 1 && (!b.fac || b.rhs)) return cudaErrorInvalidValue;
  if (a.P > 1) {
    const size_t chain = (size_t)pl.NG * (3 * R * R + 2 * R * CC) * 32 * sizeof(float);
    b.chain_smem = (pl.NG > 1 && chain <= kReducedSmemMax) ? 1 : 0;
    const size_t smem = b.chain_smem ? std::max(pl.smem_sum, chain) : pl.smem_sum;
    if constexpr (!BWD) {
      if (pl.queue) {
        // one persistent kernel: summary and back-substitution items
        if (!b.fac || a.step != 1 || a.gc > 1 || b.rhs || b.xmode != 0 || !b.qctl) return cudaErrorInvalidValue;
        b.tma = 0;   // its blocks stage many tiles; the tensor-copy path is single-use
        const size_t qsmem = std::max(smem, smem_backsub(R, CC, a.h, pl.G, 1));
        if ((e = set_smem(k_pass_q<R, CC>, qsmem)) != cudaSuccess) return e;
        int res = 0;
        if ((e = resident_blocks(reinterpret_cast<const void*>(k_pass_q<R, CC>), pl.G, qsmem, &res)) != cudaSuccess)
          return e;
        if (res < 1) return cudaErrorInvalidConfiguration;
        // look-ahead: by default about one generation of resident blocks
        // (a band's summary items finish before the items that need it are
        // taken); a ring of S slots allows at most S - 2
        int la = a.lookahead > 0 ? a.lookahead : std::max(kLookahead, res / (2 * pl.NG) + 2);
        if (pl.nslot > 0) la = std::min(la, pl.nslot - 2);
        b.lookahead = la;
        const long long items = (long long)pl.NG * (((a.nsys + 31) >> 5) + (a.D + OB - 1) / OB);
        const int grid = (int)std::min<long long>(items, res);
        e = launch_pdl(k_pass_q<R, CC>, dim3(grid), dim3(32, pl.G), qsmem, st, b);
        if (e != cudaSuccess) return e;
        return cudaGetLastError();
      }
    }
    void (*ks)(PassArgs) = k_summary<R, CC, 0>;
    if constexpr (!BWD) {
      if (b.rhs)
        ks = k_summary<R, CC, 2>;
      else if (b.fac)
        ks = a.gc > 1 ? k_summary<R, CC, 3> : k_summary<R, CC, 1>;
    } else {
      if (b.fac) ks = k_summary<R, CC, 1>;
    }
    if ((e = set_smem(ks, smem)) != cudaSuccess) return e;
    e = launch_pdl(ks, dim3((a.nsys + 31) / 32, pl.NG), dim3(32, pl.G), smem, st, b);
    if (e != cudaSuccess) return e;
  }
  if constexpr (BWD) {
    if (b.fac) {   // adjoint back-substitution from the kept factors
      const size_t smem = smem_backsub(R, CC, a.h, pl.G, 1, true);
      if ((e = set_smem(k_backsub<R, CC, 3>, smem)) != cudaSuccess) return e;
      e = launch_pdl(k_backsub<R, CC, 3>, dim3((a.D + OB - 1) / OB, pl.NG), dim3(32, pl.G), smem, st, b);
      if (e != cudaSuccess) return e;
      return cudaGetLastError();
    }
  } else {
    if (b.fac) {   // the factors were kept by k_summary
      const size_t smem = smem_backsub(R, CC, a.h, pl.G, a.step, false, b.xmode != 0 ? -1 : a.dir);
      const int nbx = a.step == 1 ? (a.D + OB - 1) / OB : (a.nsys + step_owned_lanes(R, a.step) - 1) /
                                                              step_owned_lanes(R, a.step);
      auto kern = a.step != 1 ? k_backsub<R, CC, 1> : (b.xmode != 0 ? k_backsub<R, CC, 2> : k_backsub<R, CC, 0>);
      if ((e = set_smem(kern, smem)) != cudaSuccess) return e;
      e = launch_pdl(kern, dim3(nbx, pl.NG), dim3(32, pl.G), smem, st, b);
      if (e != cudaSuccess) return e;
      return cudaGetLastError();
    }
  }
  if ((e = set_smem(k_recover<R, CC, BWD>, pl.smem_rec)) != cudaSuccess) return e;
  e = launch_pdl(k_recover<R, CC, BWD>, dim3((a.D + OB - 1) / OB, pl.NG), dim3(32, pl.G), pl.smem_rec, st, b);
  if (e != cudaSuccess) return e;
  return cudaGetLastError();
}

// Batched pass: one launch per kernel over all images of `ba`.
struct BatchLaunch {
  int nblk[3];       // blocks of the summary / reduced / recover launches
  int G;             // chunks (warps) per block, common to all images
  size_t smem[3];
  bool red_smem;     // reduced chain in shared memory
  bool any_multi;    // some image has more than one chunk
  bool any_red;      // some image has more than one chunk group
  bool keep;         // k_summary keeps the chunk factors, k_backsub follows
};

template <int R, int CC>
cudaError_t launch_batch_rc(const BatchArgs& ba, const BatchLaunch& bl, cudaStream_t st) {
  cudaError_t e;
  BatchArgs b = ba;
  b.base.early_stage = bl.any_multi ? 1 : 0;   // k_recover follows k_summary
  b.base.chain_smem = bl.red_smem ? 1 : 0;
  if (bl.any_multi) {
    const size_t smem = bl.red_smem ? std::max(bl.smem[0], bl.smem[1]) : bl.smem[0];
    auto ks = bl.keep ? k_summary_b<R, CC, 1> : k_summary_b<R, CC, 0>;
    if ((e = set_smem(ks, smem)) != cudaSuccess) return e;
    if ((e = launch_pdl(ks, dim3(bl.nblk[0]), dim3(32, bl.G), smem, st, b)) != cudaSuccess) return e;
  }
  if (bl.keep && bl.any_multi) {
    if ((e = set_smem(k_backsub_b<R, CC>, bl.smem[2])) != cudaSuccess) return e;
    if ((e = launch_pdl(k_backsub_b<R, CC>, dim3(bl.nblk[2]), dim3(32, bl.G), bl.smem[2], st, b)) != cudaSuccess)
      return e;
    return cudaGetLastError();
  }
  if ((e = set_smem(k_recover_b<R, CC>, bl.smem[2])) != cudaSuccess) return e;
  if ((e = launch_pdl(k_recover_b<R, CC>, dim3(bl.nblk[2]), dim3(32, bl.G), bl.smem[2], st, b)) != cudaSuccess)
    return e;
  return cudaGetLastError();
}

// Batched adjoint pass: one launch per kernel over all images of `ba` (CC =
// u and v planes of CC / 2 channels).  The summaries keep their factors for
// the adjoint back-substitution (bl.keep), or k_recover recomputes them.
template <int R, int CC>
cudaError_t launch_batch_bwd_rc(const BatchArgs& ba, const BatchLaunch& bl, cudaStream_t st) {
  cudaError_t e;
  BatchArgs b = ba;
  b.base.early_stage = bl.any_multi ? 1 : 0;
  b.base.chain_smem = bl.red_smem ? 1 : 0;
  if (bl.any_multi) {
    const size_t smem = bl.red_smem ? std::max(bl.smem[0], bl.smem[1]) : bl.smem[0];
    auto ks = bl.keep ? k_summary_b<R, CC, 1> : k_summary_b<R, CC, 0>;
    if ((e = set_smem(ks, smem)) != cudaSuccess) return e;
    if ((e = launch_pdl(ks, dim3(bl.nblk[0]), dim3(32, bl.G), smem, st, b)) != cudaSuccess) return e;
  }
  if (bl.keep && bl.any_multi) {
    if ((e = set_smem(k_backsub_b<R, CC, 3>, bl.smem[2])) != cudaSuccess) return e;
    if ((e = launch_pdl(k_backsub_b<R, CC, 3>, dim3(bl.nblk[2]), dim3(32, bl.G), bl.smem[2], st, b)) != cudaSuccess)
      return e;
    return cudaGetLastError();
  }
  if ((e = set_smem(k_recover_b<R, CC, true>, bl.smem[2])) != cudaSuccess) return e;
  if ((e = launch_pdl(k_recover_b<R, CC, true>, dim3(bl.nblk[2]), dim3(32, bl.G), bl.smem[2], st, b)) != cudaSuccess)
    return e;
  return cudaGetLastError();
}

// The launchers are instantiated one (radius, channel group) per object
// file (sgwls_inst.cu, compiled once per pair by build.py, so the builds of
// the kernels run in parallel); the dispatchers switch on the runtime r and
// group size.  CC < 0 in launch_pass_any: the backward pass over -CC
// right-hand sides (u and v planes of -CC/2 channels).
template <int R, int CC>
cudaError_t launch_pass_inst(const PassArgs& a, const Plan& pl, bool bwd, cudaStream_t st);
template <int R, int CC>
cudaError_t launch_batch_inst(const BatchArgs& ba, const BatchLaunch& bl, cudaStream_t st);
template <int R, int CC>
cudaError_t launch_batch_bwd_inst(const BatchArgs& ba, const BatchLaunch& bl, cudaStream_t st);
cudaError_t launch_batch_bwd_any(int r, int CC, const BatchArgs& ba, const BatchLaunch& bl, cudaStream_t st);
struct LineArgs;
template <int R, int CC>
cudaError_t launch_line_inst(const LineArgs& a, cudaStream_t st);
cudaError_t launch_pass_any(int r, int CC, const PassArgs& a, const Plan& pl, cudaStream_t st);
cudaError_t launch_batch_any(int r, int CC, const BatchArgs& ba, const BatchLaunch& bl, cudaStream_t st);

}  // namespace sgwls
