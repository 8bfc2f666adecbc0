// sgwls_api.cu -- the C ABI declared in include/sgwls.h: argument checks,
// workspace layout, the sequence of passes (Sec. 2.3) and kernel dispatch.
#include <math.h>
#include <stdint.h>
#include <string.h>

#include <algorithm>
#include <cstdio>
#include <map>
#include <mutex>
#include <tuple>
#include <vector>

#include "../../include/sgwls.h"
#include "sgwls_launch.cuh"
#include "sgwls_line.cuh"

namespace sgwls {

cudaError_t set_smem_raw(const void* kernel, size_t bytes) {
  static std::mutex mu;
  static std::map<std::pair<const void*, int>, size_t> done;
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  std::lock_guard<std::mutex> lock(mu);
  size_t& cur = done[{kernel, dev}];
  if (cur >= bytes) return cudaSuccess;
  e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
  if (e == cudaSuccess) cur = bytes;
  return e;
}

cudaError_t resident_blocks(const void* kernel, int G, size_t smem, int* out) {
  static std::mutex mu;
  static std::map<std::tuple<const void*, int, size_t, int>, int> done;
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  std::lock_guard<std::mutex> lock(mu);
  const auto key = std::make_tuple(kernel, G, smem, dev);
  auto it = done.find(key);
  if (it != done.end()) {
    *out = it->second;
    return cudaSuccess;
  }
  int per_sm = 0, nsm = 0;
  if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, 32 * G, smem)) != cudaSuccess) return e;
  if ((e = cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return e;
  *out = done[key] = per_sm * nsm;
  return cudaSuccess;
}

namespace {

thread_local char g_cuda_err[256] = "";

// Device word that a kernel sets when one of its bounded waits gave up
// (the queue-scheduled pass); read and cleared by sgwls_device_flag.  The
// name is a host-side stand-in: its device address is looked up once per
// device, with that device current.
__device__ unsigned g_device_flag;
constexpr int kMaxDevices = 64;
std::mutex g_flag_mu;
unsigned* g_flag_ptr[kMaxDevices] = {};

cudaError_t device_flag_ptr(unsigned** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lock(g_flag_mu);
  if (!g_flag_ptr[dev]) {
    void* p = nullptr;
    if ((e = cudaGetSymbolAddress(&p, g_device_flag)) != cudaSuccess) return e;
    g_flag_ptr[dev] = static_cast<unsigned*>(p);
  }
  *out = g_flag_ptr[dev];
  return cudaSuccess;
}

// Launch counter: every kernel the library launches adds one.
unsigned long long g_launches = 0;

sgwls_status cuda_fail(cudaError_t e) {
  snprintf(g_cuda_err, sizeof(g_cuda_err), "%s: %s", cudaGetErrorName(e), cudaGetErrorString(e));
  return SGWLS_E_CUDA;
}

size_t dt_size(int dt) { return dt == DT_F32 ? 4 : 2; }
size_t align256(size_t x) { return (x + 255) & ~size_t(255); }

// Resident-warp target used to size the chunking: 152 SMs x 16 warps.
constexpr int kTargetWarps = 152 * 16;
constexpr size_t kSmemBlockTarget = 110 * 1024;   // two blocks per SM
constexpr size_t kSmemBlockMax = 200 * 1024;
constexpr int kGMax = 8;

// Chunk length of a pass that keeps its chunk factors, by radius (measured
// on GB300 over 1024x768 RGB r = 1 and 1920x1080 RGB r = 2, 3, 5: long
// enough that a thread's sweep outweighs the per-chunk staging and merge
// work, short enough for many warps per SM); shorter when that would leave
// fewer than kTargetWarps chunk-warps.
inline int keep_lines(int r) { return r == 1 ? 6 : r == 2 ? 12 : r == 3 ? 8 : 16; }

// Chunk length of a sliding-step (tau > 1) pass, by radius and step: the
// fastest of 3..12 lines on GB300 for a 1-megapixel RGB image, T = 3, with
// tensor-copy staging (8 lines where the sweep found no better length, and
// beyond r = 5 or tau = 5).
inline int step_lines(int r, int step) {
  if (r == 2 && step == 2) return 6;
  if (r == 3) return step == 2 ? 6 : step == 3 ? 12 : 8;
  if (r == 4) return step == 2 ? 6 : 8;
  if (r == 5) return (step == 3 || step == 4) ? 6 : step == 5 ? 12 : 8;
  return 8;
}

// Subsystems of a pass across D offsets with sliding step `step`: the
// regular centres r, r + step, ... <= D-1-r, and the last centre D-1-r
// appended when the stride misses it (every line stays covered).  *nreg:
// regular ones.
int n_centres(int D, int r, int step, int* nreg) {
  const int nr = (D - 1 - 2 * r) / step + 1;
  if (nreg) *nreg = nr;
  return nr + (((nr - 1) * step != D - 1 - 2 * r) ? 1 : 0);
}

// keep: the pass keeps its chunk factors (k_backsub follows k_summary; no
// k_recover tile), so only the summary's tile and 2-ports bound the block.
Plan make_plan(int L, int D, int r, int CC, int chunk_lines, bool bwd = false, bool keep = false, int step = 1,
               int gc = 1, int gmax = kGMax) {
  const int bands = step == 1 ? (D + (32 - 2 * r) - 1) / (32 - 2 * r) : (n_centres(D, r, step, nullptr) + 31) / 32;
  auto second = [&](int hh, int G) {
    return keep ? smem_backsub(r, CC, hh, G, step, bwd) : smem_recover(r, CC, hh, G, bwd);
  };
  // k_summary's tile and chunk 2-ports counted side by side (they share
  // memory in the kernel): the chunk-warp counts below were tuned on GB300
  // with this measure, which also keeps the large radii (255 registers a
  // thread) at four chunk-warps a block
  auto block = [&](int hh, int G) {
    return std::max(second(hh, G),
                    4 * (tile_floats(r, CC, hh, G, step, gc) + (size_t)G * (3 * r * r + 2 * r * CC) * 32));
  };
  int h;
  if (keep && step > 1) {
    // sliding step: fewer subsystems, so fewer warps (see step_lines)
    h = step_lines(r, step);
  } else if (keep) {
    h = keep_lines(r);
    while (h > 1 && (long long)L * bands / h < kTargetWarps) --h;
  } else {
    // enough chunks for ~kTargetWarps warps in flight: h <= L * bands / target
    h = std::max(1, (int)(((long long)L * bands) / kTargetWarps));
    // blocks of G = 8 chunk-warps, two blocks per SM: shrink h to fit
    while (h > 1 && block(h, gmax) > kSmemBlockTarget) --h;
  }
  if (chunk_lines > 0) h = std::min(chunk_lines, L);
  while (h > 1 && block(h, 1) > kSmemBlockMax) --h;
  h = std::min(h, L);
  Plan pl;
  pl.h = h;
  pl.P = (L + h - 1) / h;
  // keep: as many chunk-warps per block as fit two blocks per SM
  const size_t gcap = keep ? kSmemBlockTarget : kSmemBlockMax;
  int G = 1;
  while (G < gmax && G < pl.P && block(h, 2 * G) <= gcap) G *= 2;
  pl.G = G;
  pl.NG = (pl.P + G - 1) / G;
  pl.smem_sum = smem_summary(r, CC, h, G, step, gc);
  pl.smem_rec = smem_recover(r, CC, h, G, bwd);
  return pl;
}

int n_fields(int r, int CC) { return 3 * r * r + 2 * r * CC; }
int n_mfields(int r, int CC) { return 3 * r * r + r * CC; }

struct Layout {
  size_t img_off, img_bytes;
  size_t summ_off, summ_bytes;
  size_t xsep_off, xsep_bytes;
  size_t mdata_off, mdata_bytes;
  size_t cnt_off, cnt_bytes;   // per-band block counters of k_summary
  size_t fac_off, fac_bytes;   // chunk factors kept between the kernels of a pass
  size_t psi_off, psi_bytes;
  size_t rhs_off, xent_off, ent_bytes;   // refinement: residual and first-solve entries
  size_t total;
};

// Chunk factors of one pass over CC channels: (2r + CC) values per vector
// entry (L * (2r+1) entries per subsystem), r * r per chunk for psi.
constexpr size_t kFactorCacheBytes = size_t(4) << 30;
size_t fac_bytes(int L, int r, int CC, int sstride) {
  return (size_t)L * (2 * r + 1) * (2 * r + CC) * sstride * sizeof(float);
}
size_t psi_bytes(int P, int r, int sstride) { return (size_t)P * r * r * sstride * sizeof(float); }
// Factor-store ring of the queue-scheduled pass: as many band slots as fit
// this budget (well inside GB300's 126 MB L2, next to the pass's images).
constexpr size_t kRingBytes = size_t(64) << 20;
// Guidance planes of a call (guide_channels 0 and 1: one plane).
int guide_planes(const sgwls_params* p) { return p->guide_channels > 1 ? p->guide_channels : 1; }
// Plan of one forward pass; *keep: its chunk factors are kept between the
// two kernels (needs at least two chunks).
Plan fwd_plan(const sgwls_params* p, int L, int D, int CC, int sstride, bool* keep) {
  // the sliding step, the refinement and a vector guidance run on kept
  // factors only
  const int gc = guide_planes(p);
  const bool need = p->step > 1 || p->refine || gc > 1;
  bool k = need || p->factor_cache == 1 ||
           (p->factor_cache == 0 && fac_bytes(L, p->r, CC, sstride) <= kFactorCacheBytes);
  const int gmax = p->group_warps > 0 ? p->group_warps : kGMax;
  Plan pl = make_plan(L, D, p->r, CC, p->chunk_lines, false, k, p->step, k ? gc : 1, gmax);
  // keeping factors needs at least two chunks
  if (k && need && pl.P < 2 && L >= 2)
    pl = make_plan(L, D, p->r, CC, (L + 1) / 2, false, true, p->step, gc, gmax);
  if (k && pl.P < 2) {
    k = false;
    pl = make_plan(L, D, p->r, CC, p->chunk_lines, false, false, 1, 1, gmax);
  }
  *keep = k;
  // on request (schedule = 2) a plain forward pass with kept factors runs as
  // one queue-scheduled kernel whose factor store is a ring of band slots
  // (measured on GB300 at 1920 x 1080 RGB, r = 1..5: at best 3 % faster than
  // the two kernels, mostly slower, so not the default)
  if (k && p->step == 1 && !p->refine && gc == 1 && p->schedule == 2) {
    pl.queue = 1;
    const int nb = sstride / 32;
    const size_t band = fac_bytes(L, p->r, CC, 32) + psi_bytes(pl.P, p->r, 32);
    const int slots = p->ring_slots > 0
                          ? p->ring_slots
                          : (int)std::max<size_t>(kRingBytes / band, (size_t)kLookahead + 2);
    pl.nslot = slots >= nb ? 0 : slots;
  }
  return pl;
}

// Control words of a pass, per band of 32 subsystems of the longer
// direction: k_summary's block tickets, then (queue-scheduled pass) the
// done flags and reader counts, then the queue and exit counters.
int counter_bands(int H, int W, int r) { return (std::max(H, W) - 2 * r + 31) / 32; }
size_t counter_bytes(int H, int W, int r) {
  return align256(((size_t)3 * counter_bands(H, W, r) + 2) * sizeof(int));
}

// Largest per-pass scratch over both directions and all channel groups.
Layout make_layout(int H, int W, int C, const sgwls_params* p) {
  Layout lo;
  const int r = p->r;
  size_t summ = 0, xsep = 0, mdata = 0, fac = 0, psi = 0, ent = 0;
  for (int dir = 0; dir < 2; ++dir) {
    const int L = dir == 0 ? H : W;
    const int D = dir == 0 ? W : H;
    const int nsys = (n_centres(D, r, p->step, nullptr) + 31) / 32 * 32;   // padded subsystem stride
    for (int c0 = 0; c0 < C; c0 += kGroupMax) {
      const int CC = std::min(kGroupMax, C - c0);
      bool keep = false;
      const Plan pl = fwd_plan(p, L, D, CC, nsys, &keep);
      summ = std::max(summ, (size_t)pl.NG * n_fields(r, CC) * nsys * sizeof(float));
      xsep = std::max(xsep, (size_t)std::max(pl.NG - 1, 1) * r * CC * nsys * sizeof(float));
      mdata = std::max(mdata, (size_t)pl.NG * std::max(pl.G - 1, 1) * n_mfields(r, CC) * nsys * sizeof(float));
      if (keep) {
        fac = std::max(fac, pl.nslot ? fac_bytes(L, r, CC, 32 * pl.nslot) : fac_bytes(L, r, CC, nsys));
        psi = std::max(psi, pl.nslot ? psi_bytes(pl.P, r, 32 * pl.nslot) : psi_bytes(pl.P, r, nsys));
        if (p->refine) {
          ent = std::max(ent, (size_t)L * (2 * r + 1) * CC * nsys * sizeof(float));
        }
      }
    }
  }
  // Intermediate estimates ping-pong between u and one workspace image when
  // both have the same storage type; otherwise between two workspace images
  // (u is then written by the last pass only).
  const int n_img = (p->iters > 0) ? (p->inter_storage == p->storage ? 1 : 2) : 0;
  const size_t img = (size_t)n_img * C * H * W * dt_size(p->inter_storage);
  lo.img_off = 0;
  lo.img_bytes = align256(img);
  lo.summ_off = lo.img_off + lo.img_bytes;
  lo.summ_bytes = align256(summ);
  lo.xsep_off = lo.summ_off + lo.summ_bytes;
  lo.xsep_bytes = align256(xsep);
  lo.mdata_off = lo.xsep_off + lo.xsep_bytes;
  lo.mdata_bytes = align256(mdata);
  lo.cnt_off = lo.mdata_off + lo.mdata_bytes;
  lo.cnt_bytes = counter_bytes(H, W, r);
  lo.fac_off = lo.cnt_off + lo.cnt_bytes;
  lo.fac_bytes = align256(fac);
  lo.psi_off = lo.fac_off + lo.fac_bytes;
  lo.psi_bytes = align256(psi);
  lo.ent_bytes = align256(ent);
  lo.rhs_off = lo.psi_off + lo.psi_bytes;
  lo.xent_off = lo.rhs_off + lo.ent_bytes;
  lo.total = lo.xent_off + lo.ent_bytes;
  return lo;
}

sgwls_status check_params(int H, int W, int C, const sgwls_params* p) {
  if (!p) return SGWLS_E_INVALID;
  if (p->r < 1 || p->r > SGWLS_R_MAX) return SGWLS_E_INVALID;
  if (p->iters < 0 || p->step < 1 || p->step > 2 * p->r + 1) return SGWLS_E_INVALID;
  if (p->axis_order != 0 && p->axis_order != 1) return SGWLS_E_INVALID;
  if (p->weight != SGWLS_W_EXP && p->weight != SGWLS_W_FRAC) return SGWLS_E_INVALID;
  if (p->weight == SGWLS_W_EXP && !(p->sigma_s > 0.f && p->sigma_r > 0.f)) return SGWLS_E_INVALID;
  if (p->weight == SGWLS_W_FRAC && !(p->eps > 0.f && p->alpha_s >= 0.f && p->alpha_r >= 0.f)) return SGWLS_E_INVALID;
  if (!isfinite(p->sigma_s) || !isfinite(p->sigma_r) || !isfinite(p->alpha_s) || !isfinite(p->alpha_r) ||
      !isfinite(p->eps))
    return SGWLS_E_INVALID;
  if (p->refine < 0 || p->refine > 1) return SGWLS_E_INVALID;
  if (p->chunk_lines < 0) return SGWLS_E_INVALID;
  if (p->factor_cache < 0 || p->factor_cache > 2) return SGWLS_E_INVALID;
  if (p->guide_channels < 0 || p->guide_channels > SGWLS_GUIDE_MAX) return SGWLS_E_INVALID;
  if (p->schedule < 0 || p->schedule > 2) return SGWLS_E_INVALID;
  if (p->group_warps != 0 && p->group_warps != 1 && p->group_warps != 2 && p->group_warps != 4 &&
      p->group_warps != 8)
    return SGWLS_E_INVALID;
  if (p->ring_slots < 0 || (p->ring_slots > 0 && p->ring_slots < kLookahead + 2)) return SGWLS_E_INVALID;
  if (p->lookahead < 0 || p->lookahead > 4096) return SGWLS_E_INVALID;
  if ((p->storage != SGWLS_F32 && p->storage != SGWLS_BF16) ||
      (p->inter_storage != SGWLS_F32 && p->inter_storage != SGWLS_BF16))
    return SGWLS_E_DTYPE;
  if (C < 1 || C > SGWLS_C_MAX) return SGWLS_E_SHAPE;
  if (H < 2 * p->r + 1 || W < 2 * p->r + 1) return SGWLS_E_SHAPE;
  if (H > 65536 || W > 65536 || (long long)H * W > (1LL << 31) / 4) return SGWLS_E_SHAPE;
  return SGWLS_OK;
}

// The sliding step tau > 1, the refinement and a vector guidance run on the
// kernels that keep chunk factors: they need them kept in every pass (not
// factor_cache = 2, not beyond the factor-store budget, at least two lines
// per subsystem).
sgwls_status check_step(int H, int W, int C, const sgwls_params* p) {
  // refinement (refine = 1) reuses the keep path at step 1; its FP64
  // residual reads a single guidance plane
  if (p->refine && (p->step != 1 || guide_planes(p) > 1)) return SGWLS_E_UNSUPPORTED;
  if (p->step == 1 && !p->refine && guide_planes(p) == 1) return SGWLS_OK;
  for (int dir = 0; dir < 2; ++dir) {
    const int L = dir == 0 ? H : W;
    const int D = dir == 0 ? W : H;
    const int nsys = (n_centres(D, p->r, p->step, nullptr) + 31) / 32 * 32;
    for (int c0 = 0; c0 < C; c0 += kGroupMax) {
      bool keep = false;
      fwd_plan(p, L, D, std::min(kGroupMax, C - c0), nsys, &keep);
      if (!keep || p->factor_cache == 2) return SGWLS_E_UNSUPPORTED;
      if (fac_bytes(L, p->r, std::min(kGroupMax, C - c0), nsys) > kFactorCacheBytes && p->factor_cache != 1)
        return SGWLS_E_UNSUPPORTED;
    }
  }
  return SGWLS_OK;
}

// Fills the parts of the argument block that depend only on the parameters.
void fill_weights(PassArgs& a, const sgwls_params* p, float lambda) {
  const int r = p->r;
  const int n = 2 * r + 1;
  a.lam = lambda;
  a.weight = p->weight;
  if (p->weight == SGWLS_W_EXP) {
    a.range_k = (float)(-1.4426950408889634 / (2.0 * (double)p->sigma_r * (double)p->sigma_r));
  } else {
    a.range_k = p->alpha_r;
  }
  a.eps = p->eps;
  a.dgk = (float)(1.0 / ((double)p->sigma_r * (double)p->sigma_r));
  // Spatial factor of the pair (p, p+t) with j = p % n: same line -> distance
  // t; next line -> one line over and |4r + 1 - 2j - t| across (the snake
  // turns), for both directions.
  for (int j = 0; j < n; ++j) {
    for (int t = 1; t <= r; ++t) {
      double d2;
      if (j + t < n) {
        d2 = (double)t * t;
      } else {
        const double dx = (double)(4 * r + 1 - 2 * j - t);
        d2 = 1.0 + dx * dx;
      }
      double sp;
      if (p->weight == SGWLS_W_EXP) {
        sp = exp(-d2 / (2.0 * (double)p->sigma_s * (double)p->sigma_s));
      } else {
        sp = 1.0 / (pow(sqrt(d2), (double)p->alpha_s) + (double)p->eps);
      }
      a.sp[j * r + t - 1] = (float)(lambda * sp);
      a.sp0[j * r + t - 1] = (float)sp;
    }
  }
}

__global__ void k_convert(const void* src, int sdt, void* dst, int ddt, long long count) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < count) st_px(dst, i, ddt, ld_px(src, i, sdt));
}

sgwls_status copy_image(const void* src, int sdt, void* dst, int ddt, long long count, cudaStream_t st) {
  if (sdt == ddt) {
    cudaError_t e = cudaMemcpyAsync(dst, src, (size_t)count * dt_size(sdt), cudaMemcpyDeviceToDevice, st);
    return e == cudaSuccess ? SGWLS_OK : cuda_fail(e);
  }
  k_convert<<<(unsigned)((count + 255) / 256), 256, 0, st>>>(src, sdt, dst, ddt, count);
  __atomic_add_fetch(&g_launches, 1ull, __ATOMIC_RELAXED);
  cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? SGWLS_OK : cuda_fail(e);
}

}  // namespace

// Argument checks of a single pass, in the order sgwls_filter_pass applies
// them (shared with the no-allocation pass so both return the same codes).
sgwls_status check_pass_params(int H, int W, int C, const sgwls_params* p) {
  sgwls_status s = check_params(H, W, C, p);
  if (s == SGWLS_OK) s = check_step(H, W, C, p);
  return s;
}

// Dispatch to the (radius, channel group) instantiations.
#define SGWLS_CASE_CC(R)                                                         \
  case R:                                                                        \
    switch (CC < 0 ? -CC : CC) {                                                 \
      case 1: return launch_pass_inst<R, 1>(a, pl, CC < 0, st);                 \
      case 2: return launch_pass_inst<R, 2>(a, pl, CC < 0, st);                 \
      case 3: return launch_pass_inst<R, 3>(a, pl, CC < 0, st);                 \
      case 4: return launch_pass_inst<R, 4>(a, pl, CC < 0, st);                 \
      default: return cudaErrorInvalidValue;                                     \
    }
cudaError_t launch_pass_any(int r, int CC, const PassArgs& a, const Plan& pl, cudaStream_t st) {
  // the backward's six right-hand sides (u and v of three channels): r = 1
  if (CC == -kBwdWideRhs) return r == 1 ? launch_pass_inst<1, kBwdWideRhs>(a, pl, true, st) : cudaErrorInvalidValue;
  switch (r) {
    SGWLS_CASE_CC(1) SGWLS_CASE_CC(2) SGWLS_CASE_CC(3) SGWLS_CASE_CC(4)
    SGWLS_CASE_CC(5) SGWLS_CASE_CC(6) SGWLS_CASE_CC(7) SGWLS_CASE_CC(8)
    default: return cudaErrorInvalidValue;
  }
}
#undef SGWLS_CASE_CC
#define SGWLS_CASE_CC(R)                                                         \
  case R:                                                                        \
    switch (CC) {                                                                \
      case 1: return launch_batch_inst<R, 1>(ba, bl, st);                        \
      case 2: return launch_batch_inst<R, 2>(ba, bl, st);                        \
      case 3: return launch_batch_inst<R, 3>(ba, bl, st);                        \
      case 4: return launch_batch_inst<R, 4>(ba, bl, st);                        \
      default: return cudaErrorInvalidValue;                                     \
    }
cudaError_t launch_batch_any(int r, int CC, const BatchArgs& ba, const BatchLaunch& bl, cudaStream_t st) {
  switch (r) {
    SGWLS_CASE_CC(1) SGWLS_CASE_CC(2) SGWLS_CASE_CC(3) SGWLS_CASE_CC(4)
    SGWLS_CASE_CC(5) SGWLS_CASE_CC(6) SGWLS_CASE_CC(7) SGWLS_CASE_CC(8)
    default: return cudaErrorInvalidValue;
  }
}
#undef SGWLS_CASE_CC
#define SGWLS_CASE_CC(R)                                                         \
  case R:                                                                        \
    switch (CC) {                                                                \
      case 2: return launch_batch_bwd_inst<R, 2>(ba, bl, st);                    \
      case 4: return launch_batch_bwd_inst<R, 4>(ba, bl, st);                    \
      default: return cudaErrorInvalidValue;                                     \
    }
// CC: u and v planes of CC / 2 channels (6 at r = 1 only)
cudaError_t launch_batch_bwd_any(int r, int CC, const BatchArgs& ba, const BatchLaunch& bl, cudaStream_t st) {
  if (CC == kBwdWideRhs) return r == 1 ? launch_batch_bwd_inst<1, kBwdWideRhs>(ba, bl, st) : cudaErrorInvalidValue;
  switch (r) {
    SGWLS_CASE_CC(1) SGWLS_CASE_CC(2) SGWLS_CASE_CC(3) SGWLS_CASE_CC(4)
    SGWLS_CASE_CC(5) SGWLS_CASE_CC(6) SGWLS_CASE_CC(7) SGWLS_CASE_CC(8)
    default: return cudaErrorInvalidValue;
  }
}
#undef SGWLS_CASE_CC


// Tensor-copy (TMA) descriptors of the column direction's tile staging.
// The driver's encoder is looked up once through the runtime (no link
// against the driver library).
using TmaEncodeFn = CUresult (*)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                 const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                 CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);
TmaEncodeFn tma_encoder() {
  static std::once_flag once;
  static TmaEncodeFn fn = nullptr;
  std::call_once(once, [] {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
            cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<TmaEncodeFn>(p);
  });
  return fn;
}

// Fills a.tm_in / a.tm_g for a column-direction pass and returns true when
// the tensor-copy staging applies: FP32 estimate and guidance, one guidance
// plane, one input source, rows and plane bases 16-byte aligned (W a
// multiple of 4), the box (tile pitch x G h + 2 lines) at most 256 per
// dimension.  Every box then starts on a 16-byte boundary (x = 32 band step,
// or the back-substitution block's first column rounded down to 4).
bool setup_tma(PassArgs& a, const Plan& pl, int r, int CC) {
  if (a.dir != 0 || a.gc != 1 || a.in_dt != DT_F32 || a.g_dt != DT_F32 || a.in2 != a.in) return false;
  if ((a.W & 3) || (reinterpret_cast<uintptr_t>(a.in) & 15) || (reinterpret_cast<uintptr_t>(a.g) & 15)) return false;
  // the tile of a band: 32 + 2r columns at step 1, 31 step + 2r + 1 beyond
  const int pitch = tile_pitch_n(tile_ncol(r, a.step), 0);
  const int ntl = pl.G * pl.h + 2;
  if (ntl > 256 || pitch > 256) return false;
  TmaEncodeFn enc = tma_encoder();
  if (!enc) return false;
  const cuuint64_t W = (cuuint64_t)a.W, H = (cuuint64_t)a.H;
  const cuuint64_t dims3[3] = {W, H, (cuuint64_t)CC};
  const cuuint64_t str3[2] = {W * 4, W * H * 4};
  const cuuint32_t box3[3] = {(cuuint32_t)pitch, (cuuint32_t)ntl, 1};
  const cuuint32_t es[3] = {1, 1, 1};
  if (enc(&a.tm_in, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, const_cast<void*>(a.in), dims3, str3, box3, es,
          CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
          CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
    return false;
  const cuuint64_t dims2[2] = {W, H};
  const cuuint64_t str2[1] = {W * 4};
  const cuuint32_t box2[2] = {(cuuint32_t)pitch, (cuuint32_t)ntl};
  if (enc(&a.tm_g, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, const_cast<void*>(a.g), dims2, str2, box2, es,
          CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
          CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
    return false;
  return true;
}

// One pass along `dir` (Sec. 2.3, the four steps): out = pass(in).
sgwls_status run_pass(const void* in, int in_dt, void* out, int out_dt, const void* g, int H, int W, int C,
                      float lambda, const sgwls_params* p, int dir, void* ws, cudaStream_t st, bool zero_counters) {
  const Layout lo = make_layout(H, W, C, p);
  char* wsb = static_cast<char*>(ws);
  if (zero_counters) {
    cudaError_t e = cudaMemsetAsync(wsb + lo.cnt_off, 0, lo.cnt_bytes, st);
    if (e != cudaSuccess) return cuda_fail(e);
  }
  const long long plane = (long long)H * W;
  PassArgs a;
  memset(&a, 0, sizeof(a));
  a.g = g;
  a.plane = plane;
  a.H = H;
  a.W = W;
  a.g_dt = p->storage;
  a.in_dt = in_dt;
  a.out_dt = out_dt;
  a.dir = dir;
  a.L = dir == 0 ? H : W;
  a.D = dir == 0 ? W : H;
  a.step = p->step;
  a.gc = guide_planes(p);
  a.nsys = n_centres(a.D, p->r, p->step, &a.nreg);
  a.sstride = (a.nsys + 31) / 32 * 32;
  a.summ = reinterpret_cast<float*>(wsb + lo.summ_off);
  a.xsep = reinterpret_cast<float*>(wsb + lo.xsep_off);
  a.mdata = reinterpret_cast<float*>(wsb + lo.mdata_off);
  a.band_cnt = reinterpret_cast<int*>(wsb + lo.cnt_off);
  {
    const int nbc = counter_bands(H, W, p->r);
    a.done = a.band_cnt + nbc;
    a.rdcnt = a.done + nbc;
    a.qctl = a.rdcnt + nbc;
    a.lookahead = p->lookahead;   // 0: chosen at launch
    cudaError_t e = device_flag_ptr(&a.err);
    if (e != cudaSuccess) return cuda_fail(e);
  }
  fill_weights(a, p, lambda);
  for (int c0 = 0; c0 < C; c0 += kGroupMax) {
    const int CC = std::min(kGroupMax, C - c0);
    bool keep = false;
    const Plan pl = fwd_plan(p, a.L, a.D, CC, a.sstride, &keep);
    a.h = pl.h;
    a.P = pl.P;
    a.ngroups = pl.NG;
    a.in = static_cast<const char*>(in) + (size_t)c0 * plane * dt_size(in_dt);
    a.in2 = a.in;
    a.n_in1 = CC;
    a.out = static_cast<char*>(out) + (size_t)c0 * plane * dt_size(out_dt);
    a.fac = keep ? reinterpret_cast<float*>(wsb + lo.fac_off) : nullptr;
    a.psi = keep ? reinterpret_cast<float*>(wsb + lo.psi_off) : nullptr;
    a.refine = (keep && p->refine) ? 1 : 0;
    a.rhs = a.refine ? reinterpret_cast<float*>(wsb + lo.rhs_off) : nullptr;
    a.xent = a.refine ? reinterpret_cast<float*>(wsb + lo.xent_off) : nullptr;
    a.xmode = 0;
    a.nslot = pl.nslot;
    a.tma = (!pl.queue && setup_tma(a, pl, p->r, CC)) ? 1 : 0;
    cudaError_t e = launch_pass_any(p->r, CC, a, pl, st);
    if (e != cudaSuccess) return cuda_fail(e);
    __atomic_add_fetch(&g_launches, (unsigned long long)(a.refine ? 5 : (pl.queue || pl.P < 2) ? 1 : 2),
                       __ATOMIC_RELAXED);
  }
  return SGWLS_OK;
}

// Runs all passes of one image.  Shared by the public entry points.
sgwls_status run_filter(const void* f, const void* g, void* u, int H, int W, int C, float lambda,
                        const sgwls_params* p, void* ws, void* saved, cudaStream_t st) {
  const Layout lo = make_layout(H, W, C, p);
  const long long count = (long long)H * W * C;
  const int sdt = p->storage, idt = p->inter_storage;
  if (p->iters == 0) return copy_image(f, sdt, u, sdt, count, st);

  char* wsb = static_cast<char*>(ws);
  void* img = wsb + lo.img_off;
  const int npass = 2 * p->iters;
  const size_t inter_bytes = (size_t)count * dt_size(idt);
  if (saved) {
    sgwls_status s = copy_image(f, sdt, saved, idt, count, st);
    if (s != SGWLS_OK) return s;
  }
  const void* cur = f;
  int cur_dt = sdt;
  for (int t = 0; t < npass; ++t) {
    const int dir = ((t & 1) == 0) ? p->axis_order : 1 - p->axis_order;
    void* dst;
    int dst_dt;
    if (t == npass - 1) {
      dst = u;
      dst_dt = sdt;
    } else if (saved) {
      dst = static_cast<char*>(saved) + (size_t)(t + 1) * inter_bytes;
      dst_dt = idt;
    } else if (idt == sdt) {
      dst = ((npass - 1 - t) & 1) ? img : u;
      dst_dt = sdt;
    } else {
      dst = static_cast<char*>(img) + (size_t)(t & 1) * inter_bytes;
      dst_dt = idt;
    }
    sgwls_status s = run_pass(cur, cur_dt, dst, dst_dt, g, H, W, C, lambda, p, dir, ws, st, t == 0);
    if (s != SGWLS_OK) return s;
    cur = dst;
    cur_dt = dst_dt;
  }
  return SGWLS_OK;
}

// ---------------------------------------------------------------------------
// Guided sparse interpolation (Eq. 21): filter [F, Hm] as C + 1 channels of
// one image (one factorisation per subsystem for up to four channels), then
// divide.  Workspace: the stacked input, the filtered stack, the filter's own
// workspace.

namespace {

struct InterpLayout {
  size_t stack_in, stack_out, filt, total;
};

InterpLayout make_interp_layout(int H, int W, int C, const sgwls_params* p) {
  InterpLayout lo;
  const size_t plane = (size_t)H * W * sizeof(float);
  lo.stack_in = 0;
  lo.stack_out = align256((size_t)(C + 1) * plane);
  lo.filt = lo.stack_out + align256((size_t)(C + 1) * plane);
  lo.total = lo.filt + make_layout(H, W, C + 1, p).total;
  return lo;
}

// u[c] = x[c] / x[C] where the filtered index map x[C] is positive, else 0.
__global__ void k_ratio(const float* __restrict__ x, float* __restrict__ u, long long plane, int C) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= plane) return;
  const float d = x[(long long)C * plane + i];
  const float inv = d > 0.f ? 1.0f / d : 0.f;
  for (int c = 0; c < C; ++c) u[(long long)c * plane + i] = x[(long long)c * plane + i] * inv;
}

}  // namespace

sgwls_status run_interpolate(const float* f, const float* hmap, const float* g, float* u, int H, int W, int C,
                             float lambda, const sgwls_params* p, void* ws, cudaStream_t st) {
  const InterpLayout lo = make_interp_layout(H, W, C, p);
  char* wsb = static_cast<char*>(ws);
  float* xin = reinterpret_cast<float*>(wsb + lo.stack_in);
  float* xout = reinterpret_cast<float*>(wsb + lo.stack_out);
  const size_t plane = (size_t)H * W;
  cudaError_t e = cudaMemcpyAsync(xin, f, (size_t)C * plane * sizeof(float), cudaMemcpyDeviceToDevice, st);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(xin + (size_t)C * plane, hmap, plane * sizeof(float), cudaMemcpyDeviceToDevice, st);
  if (e != cudaSuccess) return cuda_fail(e);
  sgwls_status s = run_filter(xin, g, xout, H, W, C + 1, lambda, p, wsb + lo.filt, nullptr, st);
  if (s != SGWLS_OK) return s;
  k_ratio<<<(unsigned)((plane + 255) / 256), 256, 0, st>>>(xout, u, (long long)plane, C);
  __atomic_add_fetch(&g_launches, 1ull, __ATOMIC_RELAXED);
  e = cudaGetLastError();
  return e == cudaSuccess ? SGWLS_OK : cuda_fail(e);
}

// ---------------------------------------------------------------------------
// Batched filter: many images of uneven sizes, one launch per kernel per pass.

namespace {

// Whether the passes of a batched call keep their chunk factors: every
// image's factors within the single-image budget (or factor_cache = 1).
bool batch_keep(int B, const sgwls_image* imgs, const sgwls_params* p) {
  if (p->factor_cache == 2) return false;
  if (p->factor_cache == 1) return true;
  for (int i = 0; i < B; ++i) {
    for (int dir = 0; dir < 2; ++dir) {
      const int L = dir == 0 ? imgs[i].H : imgs[i].W;
      const int D = dir == 0 ? imgs[i].W : imgs[i].H;
      const int nsys = ((D - 2 * p->r) + 31) / 32 * 32;
      if (fac_bytes(L, p->r, imgs[i].C, nsys) > kFactorCacheBytes) return false;
    }
  }
  return true;
}

// Lines per chunk shared by every image of a batch (blocks of kGMax chunks,
// two blocks per SM).
int batch_h(int r, int CC, bool keep, int chunk_lines) {
  int h = chunk_lines > 0 ? chunk_lines : keep ? keep_lines(r) : 64;
  auto block = [&](int hh) {
    return keep ? std::max(smem_summary(r, CC, hh, kGMax), smem_backsub(r, CC, hh, kGMax))
                : smem_recover(r, CC, hh, kGMax);
  };
  while (h > 1 && block(h) > kSmemBlockTarget) --h;
  return h;
}

Plan batch_plan(int L, int r, int CC, int h0) {
  Plan pl;
  pl.h = std::min(h0, L);
  pl.P = (L + pl.h - 1) / pl.h;
  pl.G = kGMax;
  pl.NG = (pl.P + kGMax - 1) / kGMax;
  pl.smem_sum = smem_summary(r, CC, h0, kGMax);
  pl.smem_rec = smem_recover(r, CC, h0, kGMax);
  return pl;
}

struct BatchImgLayout {
  size_t img, summ, xsep, mdata, cnt, fac, psi, end;
};

// Workspace of image i starts at `base`; returns its layout.
BatchImgLayout batch_img_layout(size_t base, int H, int W, int C, const sgwls_params* p, bool keep) {
  const int r = p->r;
  const int h0 = batch_h(r, C, keep, p->chunk_lines);
  size_t summ = 0, xsep = 0, mdata = 0, fac = 0, psi = 0;
  for (int dir = 0; dir < 2; ++dir) {
    const int L = dir == 0 ? H : W;
    const int D = dir == 0 ? W : H;
    const int nsys = ((D - 2 * r) + 31) / 32 * 32;   // padded subsystem stride
    const Plan pl = batch_plan(L, r, C, h0);
    summ = std::max(summ, (size_t)pl.NG * n_fields(r, C) * nsys * sizeof(float));
    xsep = std::max(xsep, (size_t)std::max(pl.NG - 1, 1) * r * C * nsys * sizeof(float));
    mdata = std::max(mdata, (size_t)pl.NG * (kGMax - 1) * n_mfields(r, C) * nsys * sizeof(float));
    if (keep) {
      fac = std::max(fac, fac_bytes(L, r, C, nsys));
      psi = std::max(psi, psi_bytes(pl.P, r, nsys));
    }
  }
  const int n_img = (p->iters > 0) ? (p->inter_storage == p->storage ? 1 : 2) : 0;
  BatchImgLayout lo;
  lo.img = base;
  lo.summ = lo.img + align256((size_t)n_img * C * H * W * dt_size(p->inter_storage));
  lo.xsep = lo.summ + align256(summ);
  lo.mdata = lo.xsep + align256(xsep);
  lo.cnt = 0;   // (counters live in the batch's shared counter region)
  lo.fac = lo.mdata + align256(mdata);
  lo.psi = lo.fac + align256(fac);
  lo.end = lo.psi + align256(psi);
  return lo;
}

sgwls_status check_batch(int B, const sgwls_image* imgs, const sgwls_params* p) {
  if (B < 1 || !imgs || !p) return SGWLS_E_INVALID;
  sgwls_status s0 = check_params(imgs[0].H, imgs[0].W, imgs[0].C, p);   // out-of-range values first
  if (s0 != SGWLS_OK) return s0;
  // sliding step, refinement, vector guidance: single images
  if (p->step != 1 || p->refine || p->guide_channels > 1) return SGWLS_E_UNSUPPORTED;
  for (int i = 0; i < B; ++i) {
    const sgwls_image& im = imgs[i];
    sgwls_status s = check_params(im.H, im.W, im.C, p);
    if (s != SGWLS_OK) return s;
    if (!im.f || !im.g || !im.u || im.f == im.u || im.g == im.u) return SGWLS_E_INVALID;
    if (!(im.lambda >= 0.f) || !isfinite(im.lambda)) return SGWLS_E_INVALID;
  }
  return SGWLS_OK;
}

// Batched workspace: the band counters of all images first (one region,
// cleared once per call), then every image's layout.
size_t batch_counters(int B, const sgwls_image* imgs, const sgwls_params* p) {
  size_t c = 0;
  for (int i = 0; i < B; ++i) c += counter_bytes(imgs[i].H, imgs[i].W, p->r);
  return c;
}

size_t batch_workspace(int B, const sgwls_image* imgs, const sgwls_params* p) {
  const bool keep = batch_keep(B, imgs, p);
  size_t off = batch_counters(B, imgs, p);
  for (int i = 0; i < B; ++i) off = batch_img_layout(off, imgs[i].H, imgs[i].W, imgs[i].C, p, keep).end;
  return off;
}

// Images of any channel count: every image is split into channel groups of
// at most kGroupMax channels (views of its input and output at a channel
// offset; same guidance and lambda), and the groups are gathered by size
// into uniform batches, sets[CC - 1] holding the groups of CC channels.
// strides[CC - 1][k]: elements between the per-pass checkpoints of group k
// (its image's C H W: a group's checkpoint of pass t is its channels of the
// image's checkpoint t).
void channel_group_sets(int B, const sgwls_image* imgs, const sgwls_params* p,
                        std::vector<sgwls_image> (&sets)[kGroupMax], std::vector<long long> (&strides)[kGroupMax]) {
  const size_t el = dt_size(p->storage), eli = dt_size(p->inter_storage);
  for (int i = 0; i < B; ++i) {
    const sgwls_image& im = imgs[i];
    const size_t plane = (size_t)im.H * im.W;
    for (int c0 = 0; c0 < im.C; c0 += kGroupMax) {
      sgwls_image v = im;
      v.C = std::min(kGroupMax, im.C - c0);
      v.f = static_cast<const char*>(im.f) + (size_t)c0 * plane * el;
      v.u = static_cast<char*>(im.u) + (size_t)c0 * plane * el;
      v.saved = im.saved ? static_cast<char*>(im.saved) + (size_t)c0 * plane * eli : nullptr;
      sets[v.C - 1].push_back(v);
      strides[v.C - 1].push_back((long long)im.C * (long long)plane);
    }
  }
}

// Workspace of a batch of any channel counts: the uniform batches one after
// another, each 256-byte aligned.
size_t batch_workspace_any(int B, const sgwls_image* imgs, const sgwls_params* p) {
  std::vector<sgwls_image> sets[kGroupMax];
  std::vector<long long> strides[kGroupMax];
  channel_group_sets(B, imgs, p, sets, strides);
  size_t off = 0;
  for (auto& v : sets)
    if (!v.empty()) off = align256(off + batch_workspace((int)v.size(), v.data(), p));
  return off;
}

}  // namespace

sgwls_status run_batched(int B, const sgwls_image* imgs, const sgwls_params* p, void* ws, cudaStream_t st,
                         const long long* saved_stride);

// Batched filter of images of any channel counts: one uniform batch per
// channel-group size present (see channel_group_sets).
sgwls_status run_batched_any(int B, const sgwls_image* imgs, const sgwls_params* p, void* ws, cudaStream_t st) {
  std::vector<sgwls_image> sets[kGroupMax];
  std::vector<long long> strides[kGroupMax];
  channel_group_sets(B, imgs, p, sets, strides);
  size_t off = 0;
  for (int k = 0; k < kGroupMax; ++k) {
    std::vector<sgwls_image>& v = sets[k];
    if (v.empty()) continue;
    const sgwls_status s =
        run_batched((int)v.size(), v.data(), p, static_cast<char*>(ws) + off, st, strides[k].data());
    if (s != SGWLS_OK) return s;
    off = align256(off + batch_workspace((int)v.size(), v.data(), p));
  }
  return SGWLS_OK;
}

// A uniform batch: every image has the same channel count C <= kGroupMax.
// saved_stride[i] (null: C H W): elements between image i's checkpoints.
sgwls_status run_batched(int B, const sgwls_image* imgs, const sgwls_params* p, void* ws, cudaStream_t st,
                         const long long* saved_stride) {
  const int C = imgs[0].C;
  const int r = p->r;
  const int sdt = p->storage, idt = p->inter_storage;
  char* wsb = static_cast<char*>(ws);
  if (p->iters == 0) {
    for (int i = 0; i < B; ++i) {
      sgwls_status s = copy_image(imgs[i].f, sdt, imgs[i].u, sdt, (long long)imgs[i].H * imgs[i].W * C, st);
      if (s != SGWLS_OK) return s;
    }
    return SGWLS_OK;
  }
  const bool keep = batch_keep(B, imgs, p);
  const int h0 = batch_h(r, C, keep, p->chunk_lines);
  const int OB = 32 - 2 * r;
  const int npass = 2 * p->iters;
  std::vector<BatchImgLayout> lay(B);
  std::vector<size_t> cnt_off(B);
  {
    const size_t ncnt = batch_counters(B, imgs, p);
    size_t off = ncnt, coff = 0;
    for (int i = 0; i < B; ++i) {
      lay[i] = batch_img_layout(off, imgs[i].H, imgs[i].W, C, p, keep);
      off = lay[i].end;
      cnt_off[i] = coff;
      coff += counter_bytes(imgs[i].H, imgs[i].W, r);
    }
    // the band counters of all images, cleared once (each pass leaves them at 0)
    cudaError_t e = cudaMemsetAsync(wsb, 0, ncnt, st);
    if (e != cudaSuccess) return cuda_fail(e);
  }
  // checkpoints: pass 0's input is a copy of f
  for (int i = 0; i < B; ++i) {
    if (!imgs[i].saved) continue;
    const sgwls_status s = copy_image(imgs[i].f, sdt, imgs[i].saved, idt, (long long)imgs[i].H * imgs[i].W * C, st);
    if (s != SGWLS_OK) return s;
  }
  static thread_local BatchArgs batch_args;   // host-side argument block (the kernels get a copy)
  BatchArgs* ba = &batch_args;
  for (int t = 0; t < npass; ++t) {
    const int dir = ((t & 1) == 0) ? p->axis_order : 1 - p->axis_order;
    for (int i0 = 0; i0 < B; i0 += kBatchMax) {
      const int nb = std::min(kBatchMax, B - i0);
      memset(ba, 0, sizeof(BatchArgs));
      PassArgs& a = ba->base;
      a.dir = dir;
      a.in_dt = t == 0 ? sdt : idt;
      a.g_dt = sdt;
      a.n_in1 = C;
      a.step = 1;
      fill_weights(a, p, 1.0f);   // sp0 (lambda applied per image)
      ba->nimg = nb;
      BatchLaunch bl = {};
      bl.G = kGMax;
      bl.keep = keep;
      size_t red_max = 0;
      int b[3] = {0, 0, 0};
      for (int k = 0; k < nb; ++k) {
        const sgwls_image& im = imgs[i0 + k];
        const BatchImgLayout& lo = lay[i0 + k];
        ImgDesc& d = ba->img[k];
        const size_t count = (size_t)im.H * im.W * C;
        const size_t ib = count * dt_size(idt);
        void* img = wsb + lo.img;
        // with checkpoints, pass t reads checkpoint t and writes checkpoint t + 1
        char* const sv = static_cast<char*>(im.saved);
        const size_t sb = (size_t)(saved_stride ? saved_stride[i0 + k] : (long long)count) * dt_size(idt);
        const void* src;
        void* dst;
        if (t == 0) {
          src = im.f;
        } else if (sv) {
          src = sv + (size_t)t * sb;
        } else if (idt == sdt) {
          src = ((npass - t) & 1) ? img : im.u;
        } else {
          src = static_cast<char*>(img) + (size_t)((t - 1) & 1) * ib;
        }
        if (t == npass - 1) {
          dst = im.u;
        } else if (sv) {
          dst = sv + (size_t)(t + 1) * sb;
        } else if (idt == sdt) {
          dst = ((npass - 1 - t) & 1) ? img : im.u;
        } else {
          dst = static_cast<char*>(img) + (size_t)(t & 1) * ib;
        }
        d.in = src;
        d.g = im.g;
        d.out = dst;
        d.summ = reinterpret_cast<float*>(wsb + lo.summ);
        d.xsep = reinterpret_cast<float*>(wsb + lo.xsep);
        d.mdata = reinterpret_cast<float*>(wsb + lo.mdata);
        d.band_cnt = reinterpret_cast<int*>(wsb + cnt_off[i0 + k]);
        d.fac = keep ? reinterpret_cast<float*>(wsb + lo.fac) : nullptr;
        d.psi = keep ? reinterpret_cast<float*>(wsb + lo.psi) : nullptr;
        d.plane = (long long)im.H * im.W;
        d.H = im.H;
        d.W = im.W;
        d.L = dir == 0 ? im.H : im.W;
        d.D = dir == 0 ? im.W : im.H;
        d.nsys = d.D - 2 * r;
        d.sstride = (d.nsys + 31) / 32 * 32;
        const Plan pl = batch_plan(d.L, r, C, h0);
        d.h = pl.h;
        d.P = pl.P;
        d.ngroups = pl.NG;
        d.lam = im.lambda;
        d.nbx[0] = (d.nsys + 31) / 32;
        d.nbx[1] = (d.nsys + 31) / 32;
        d.nbx[2] = (d.D + OB - 1) / OB;
        d.b0[0] = b[0];
        d.b0[1] = b[1];
        d.b0[2] = b[2];
        b[0] += d.nbx[0] * pl.NG;
        b[1] += d.nbx[1];
        b[2] += d.nbx[2] * pl.NG;
        bl.any_multi |= pl.P > 1;
        bl.any_red |= pl.NG > 1;
        red_max = std::max(red_max, (size_t)pl.NG * n_fields(r, C) * 32 * sizeof(float));
        bl.smem[0] = pl.smem_sum;
        bl.smem[2] = keep ? smem_backsub(r, C, h0, kGMax) : pl.smem_rec;
      }
      // the output type of intermediate passes is the intermediate type
      a.out_dt = (t == npass - 1) ? sdt : (idt == sdt ? sdt : idt);
      bl.nblk[0] = b[0];
      bl.nblk[1] = b[1];
      bl.nblk[2] = b[2];
      bl.red_smem = red_max <= kReducedSmemMax;
      bl.smem[1] = bl.red_smem ? red_max : 0;
      cudaError_t e = launch_batch_any(r, C, *ba, bl, st);
      if (e != cudaSuccess) return cuda_fail(e);
      __atomic_add_fetch(&g_launches, (unsigned long long)(1 + (bl.any_multi ? 1 : 0)), __ATOMIC_RELAXED);
    }
  }
  return SGWLS_OK;
}

// ---------------------------------------------------------------------------
// Backward (adjoint) of the filter.

namespace {

struct BwdLayout {
  size_t img0, img1, gbuf, summ, xsep, mdata, fac, psi, cnt, total;
  bool keep;   // the adjoint passes keep their chunk factors
};

// Channels per backward group (u and v of each solved against one factor):
// three at r = 1 (six right-hand sides), two otherwise.
int bwd_group(int r) { return r == 1 ? kBwdWideRhs / 2 : 2; }

// Whether the adjoint passes of an H x W x C image keep their chunk factors
// (k_summary then k_backsub's adjoint mode) instead of recomputing them in
// k_recover: as in the forward, unless factor_cache = 2 or the factors of
// a pass exceed the factor budget (factor_cache = 1: always).
bool bwd_keep(int H, int W, int C, const sgwls_params* p) {
  if (p->factor_cache == 2) return false;
  if (p->factor_cache == 1) return true;
  const int CC = 2 * std::min(bwd_group(p->r), C);
  for (int dir = 0; dir < 2; ++dir) {
    const int L = dir == 0 ? H : W;
    const int D = dir == 0 ? W : H;
    const int nsys = ((D - 2 * p->r) + 31) / 32 * 32;
    if (fac_bytes(L, p->r, CC, nsys) > kFactorCacheBytes) return false;
  }
  return true;
}

// Plan of one adjoint pass over CC right-hand sides.
Plan bwd_plan(int L, int D, int CC, const sgwls_params* p, bool keep) {
  return make_plan(L, D, p->r, CC, p->chunk_lines, true, keep, 1, 1, p->group_warps > 0 ? p->group_warps : kGMax);
}

BwdLayout make_bwd_layout(int H, int W, int C, const sgwls_params* p) {
  const int r = p->r;
  const int gch = bwd_group(r);
  const bool keep = bwd_keep(H, W, C, p);
  size_t summ = 0, xsep = 0, mdata = 0, fac = 0, psi = 0;
  for (int dir = 0; dir < 2; ++dir) {
    const int L = dir == 0 ? H : W;
    const int D = dir == 0 ? W : H;
    const int nsys = ((D - 2 * r) + 31) / 32 * 32;   // padded subsystem stride
    for (int c0 = 0; c0 < C; c0 += gch) {
      const int CC = 2 * std::min(gch, C - c0);
      const Plan pl = bwd_plan(L, D, CC, p, keep);
      summ = std::max(summ, (size_t)pl.NG * n_fields(r, CC) * nsys * sizeof(float));
      xsep = std::max(xsep, (size_t)std::max(pl.NG - 1, 1) * r * CC * nsys * sizeof(float));
      mdata = std::max(mdata, (size_t)pl.NG * std::max(pl.G - 1, 1) * n_mfields(r, CC) * nsys * sizeof(float));
      if (keep && pl.P > 1) {
        fac = std::max(fac, fac_bytes(L, r, CC, nsys));
        psi = std::max(psi, psi_bytes(pl.P, r, nsys));
      }
    }
  }
  const size_t img = align256((size_t)C * H * W * sizeof(float));
  BwdLayout lo;
  lo.keep = keep;
  lo.img0 = 0;
  lo.img1 = img;
  lo.gbuf = 2 * img;
  lo.summ = lo.gbuf + align256(((size_t)H * W + 64) * sizeof(float));
  lo.xsep = lo.summ + align256(summ);
  lo.mdata = lo.xsep + align256(xsep);
  lo.fac = lo.mdata + align256(mdata);
  lo.psi = lo.fac + align256(fac);
  lo.cnt = lo.psi + align256(psi);
  lo.total = lo.cnt + counter_bytes(H, W, r);
  return lo;
}

// vbar' = vbar / (number of subsystems containing the pixel), for the pass
// direction `dir` (the transpose of step 4 of Sec. 2.3).
__global__ void k_bwd_scale(const float* __restrict__ vin, float* __restrict__ vout, int H, int W, int C, int r,
                            int dir) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  const long long plane = (long long)H * W;
  if (i >= plane * C) return;
  const long long pix = i % plane;
  const int y = (int)(pix / W), x = (int)(pix - (long long)y * W);
  const int o = dir == 0 ? x : y;
  const int D = dir == 0 ? W : H;
  const int lo = max(r, o - r), hi = min(D - 1 - r, o + r);
  vout[i] = vin[i] / (float)(hi - lo + 1);
}

}  // namespace

sgwls_status run_backward(const float* grad_u, const float* g, const float* saved, int H, int W, int C,
                          float lambda, const sgwls_params* p, float* grad_f, float* grad_g, float* grad_lam,
                          void* ws, cudaStream_t st) {
  const BwdLayout lo = make_bwd_layout(H, W, C, p);
  char* wsb = static_cast<char*>(ws);
  float* w0 = reinterpret_cast<float*>(wsb + lo.img0);   // vbar / count
  float* w1 = reinterpret_cast<float*>(wsb + lo.img1);   // vbar of the next pass down
  float* gb = reinterpret_cast<float*>(wsb + lo.gbuf);
  if (!grad_g) grad_g = gb;
  if (!grad_lam) grad_lam = gb + (size_t)H * W;
  const long long plane = (long long)H * W;
  const long long count = plane * C;
  cudaError_t e;
  if ((e = cudaMemsetAsync(grad_g, 0, (size_t)plane * sizeof(float), st)) != cudaSuccess) return cuda_fail(e);
  if ((e = cudaMemsetAsync(grad_lam, 0, sizeof(float), st)) != cudaSuccess) return cuda_fail(e);
  if ((e = cudaMemsetAsync(wsb + lo.cnt, 0, lo.total - lo.cnt, st)) != cudaSuccess) return cuda_fail(e);
  const int npass = 2 * p->iters;
  if (npass == 0) {
    e = cudaMemcpyAsync(grad_f, grad_u, (size_t)count * sizeof(float), cudaMemcpyDeviceToDevice, st);
    return e == cudaSuccess ? SGWLS_OK : cuda_fail(e);
  }
  const float* vbar = grad_u;
  for (int t = npass - 1; t >= 0; --t) {
    const int dir = ((t & 1) == 0) ? p->axis_order : 1 - p->axis_order;
    k_bwd_scale<<<(unsigned)((count + 255) / 256), 256, 0, st>>>(vbar, w0, H, W, C, p->r, dir);
    __atomic_add_fetch(&g_launches, 1ull, __ATOMIC_RELAXED);
    if ((e = cudaGetLastError()) != cudaSuccess) return cuda_fail(e);
    float* dst = t == 0 ? grad_f : w1;
    const float* uin = saved + (size_t)t * count;
    PassArgs a;
    memset(&a, 0, sizeof(a));
    a.g = g;
    a.plane = plane;
    a.H = H;
    a.W = W;
    a.g_dt = DT_F32;
    a.in_dt = DT_F32;
    a.out_dt = DT_F32;
    a.dir = dir;
    a.L = dir == 0 ? H : W;
    a.D = dir == 0 ? W : H;
    a.nsys = a.D - 2 * p->r;
    a.step = 1;
    a.nreg = a.nsys;
    a.sstride = (a.nsys + 31) / 32 * 32;
    a.summ = reinterpret_cast<float*>(wsb + lo.summ);
    a.xsep = reinterpret_cast<float*>(wsb + lo.xsep);
    a.mdata = reinterpret_cast<float*>(wsb + lo.mdata);
    a.band_cnt = reinterpret_cast<int*>(wsb + lo.cnt);
    a.grad_g = grad_g;
    a.grad_lam = grad_lam;
    fill_weights(a, p, lambda);
    const int gch = bwd_group(p->r);
    for (int c0 = 0; c0 < C; c0 += gch) {
      const int nch = std::min(gch, C - c0);
      const Plan pl = bwd_plan(a.L, a.D, 2 * nch, p, lo.keep);
      a.h = pl.h;
      a.P = pl.P;
      a.ngroups = pl.NG;
      a.fac = lo.keep && pl.P > 1 ? reinterpret_cast<float*>(wsb + lo.fac) : nullptr;
      a.psi = lo.keep && pl.P > 1 ? reinterpret_cast<float*>(wsb + lo.psi) : nullptr;
      a.in = uin + (size_t)c0 * plane;
      a.in2 = w0 + (size_t)c0 * plane;
      a.n_in1 = nch;
      a.out = dst + (size_t)c0 * plane;
      e = launch_pass_any(p->r, -2 * nch, a, pl, st);
      if (e != cudaSuccess) return cuda_fail(e);
      __atomic_add_fetch(&g_launches, (unsigned long long)(a.refine ? 5 : (pl.P > 1 ? 2 : 1)), __ATOMIC_RELAXED);
    }
    vbar = dst;
  }
  return SGWLS_OK;
}

// ---------------------------------------------------------------------------
// Batched backward: the adjoint of a batched forward, every pass one launch
// per kernel over all images (grouped by channel-group size).

namespace {

constexpr int kScaleMax = 64;   // images per batched scale launch

// Every image's vbar / count of one pass direction (k_bwd_scale over a batch:
// a flat index over all images' elements, the image by binary search).
struct ScaleTab {
  int n, r, dir;
  const float* vin[kScaleMax];
  float* vout[kScaleMax];
  int H[kScaleMax], W[kScaleMax];
  long long start[kScaleMax + 1];   // first element of each image
};

__global__ void k_bwd_scale_b(const __grid_constant__ ScaleTab t) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= t.start[t.n]) return;
  int lo = 0, hi = t.n - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (t.start[mid] <= i) lo = mid; else hi = mid - 1;
  }
  const long long k = i - t.start[lo];
  const int H = t.H[lo], W = t.W[lo];
  const long long pix = k % ((long long)H * W);
  const int y = (int)(pix / W), x = (int)(pix - (long long)y * W);
  const int o = t.dir == 0 ? x : y;
  const int D = t.dir == 0 ? W : H;
  const int lo_c = max(t.r, o - t.r), hi_c = min(D - 1 - t.r, o + t.r);
  t.vout[lo][k] = t.vin[lo][k] / (float)(hi_c - lo_c + 1);
}

// Lines per chunk of a batched adjoint pass (blocks of kGMax chunks).
int batch_h_bwd(int r, int CC, int chunk_lines, bool keep) {
  int h = chunk_lines > 0 ? chunk_lines : keep ? keep_lines(r) : 64;
  auto block = [&](int hh) {
    return keep ? std::max(smem_summary(r, CC, hh, kGMax), smem_backsub(r, CC, hh, kGMax, 1, true))
                : smem_recover(r, CC, hh, kGMax, true);
  };
  while (h > 1 && block(h) > kSmemBlockTarget) --h;
  return h;
}

// One channel group of one image of a batched backward.
struct BwdJob {
  int img, c0, nch;
};

struct BwdBatchLayout {
  std::vector<size_t> w0, w1, gbuf;                 // per image
  std::vector<size_t> summ, xsep, mdata, cnt;       // per job
  std::vector<size_t> fac, psi;                     // per job (keep)
  std::vector<BwdJob> jobs[kGroupMax];              // by nch - 1 (nch <= 3)
  std::vector<size_t> jobpos[kGroupMax];            // index into summ / xsep / ...
  size_t ncnt = 0, total = 0;
  bool keep = false;   // the adjoint passes keep their chunk factors
};

// Keep the adjoint's chunk factors for every image of a batched backward,
// or for none (each job has its own factor store).
bool bwd_batch_keep(int B, const sgwls_grad_image* imgs, const sgwls_params* p) {
  for (int i = 0; i < B; ++i)
    if (!bwd_keep(imgs[i].H, imgs[i].W, imgs[i].C, p)) return false;
  return true;
}

BwdBatchLayout bwd_batch_layout(int B, const sgwls_grad_image* imgs, const sgwls_params* p) {
  BwdBatchLayout lo;
  const int r = p->r;
  const int gch = bwd_group(r);
  lo.keep = bwd_batch_keep(B, imgs, p);
  std::vector<BwdJob> all;
  for (int i = 0; i < B; ++i)
    for (int c0 = 0; c0 < imgs[i].C; c0 += gch) all.push_back({i, c0, std::min(gch, imgs[i].C - c0)});
  // counters of every job first (one region, cleared once per call)
  size_t off = 0;
  for (const BwdJob& j : all) {
    lo.cnt.push_back(off);
    off += counter_bytes(imgs[j.img].H, imgs[j.img].W, r);
  }
  lo.ncnt = off;
  off = align256(off);
  for (int i = 0; i < B; ++i) {
    const size_t img = align256((size_t)imgs[i].C * imgs[i].H * imgs[i].W * sizeof(float));
    lo.w0.push_back(off);
    lo.w1.push_back(off + img);
    lo.gbuf.push_back(off + 2 * img);
    off += 2 * img + align256(((size_t)imgs[i].H * imgs[i].W + 64) * sizeof(float));
  }
  for (size_t k = 0; k < all.size(); ++k) {
    const BwdJob& j = all[k];
    const int CC = 2 * j.nch;
    const int h0 = batch_h_bwd(r, CC, p->chunk_lines, lo.keep);
    size_t summ = 0, xsep = 0, mdata = 0, fac = 0, psi = 0;
    for (int dir = 0; dir < 2; ++dir) {
      const int L = dir == 0 ? imgs[j.img].H : imgs[j.img].W;
      const int D = dir == 0 ? imgs[j.img].W : imgs[j.img].H;
      const int nsys = ((D - 2 * r) + 31) / 32 * 32;
      const Plan pl = batch_plan(L, r, CC, h0);
      summ = std::max(summ, (size_t)pl.NG * n_fields(r, CC) * nsys * sizeof(float));
      xsep = std::max(xsep, (size_t)std::max(pl.NG - 1, 1) * r * CC * nsys * sizeof(float));
      mdata = std::max(mdata, (size_t)pl.NG * (kGMax - 1) * n_mfields(r, CC) * nsys * sizeof(float));
      if (lo.keep) {
        fac = std::max(fac, fac_bytes(L, r, CC, nsys));
        psi = std::max(psi, psi_bytes(pl.P, r, nsys));
      }
    }
    lo.summ.push_back(off);
    lo.xsep.push_back(off + align256(summ));
    lo.mdata.push_back(off + align256(summ) + align256(xsep));
    off += align256(summ) + align256(xsep) + align256(mdata);
    lo.fac.push_back(off);
    lo.psi.push_back(off + align256(fac));
    off += align256(fac) + align256(psi);
    lo.jobs[j.nch - 1].push_back(j);
    lo.jobpos[j.nch - 1].push_back(k);
  }
  lo.total = off;
  return lo;
}

sgwls_status check_batch_bwd(int B, const sgwls_grad_image* imgs, const sgwls_params* p) {
  if (B < 1 || !imgs || !p) return SGWLS_E_INVALID;
  sgwls_status s0 = check_params(imgs[0].H, imgs[0].W, imgs[0].C, p);
  if (s0 != SGWLS_OK) return s0;
  if (p->storage != SGWLS_F32 || p->inter_storage != SGWLS_F32) return SGWLS_E_UNSUPPORTED;
  if (p->weight == SGWLS_W_FRAC && p->alpha_r < 1.f) return SGWLS_E_UNSUPPORTED;
  if (p->step != 1 || p->refine || p->guide_channels > 1) return SGWLS_E_UNSUPPORTED;
  for (int i = 0; i < B; ++i) {
    const sgwls_grad_image& im = imgs[i];
    sgwls_status s = check_params(im.H, im.W, im.C, p);
    if (s != SGWLS_OK) return s;
    if (!im.grad_u || !im.g || !im.grad_f || (p->iters > 0 && !im.saved)) return SGWLS_E_INVALID;
    if (im.grad_f == im.grad_u) return SGWLS_E_INVALID;
    if (!(im.lambda >= 0.f) || !isfinite(im.lambda)) return SGWLS_E_INVALID;
  }
  return SGWLS_OK;
}

}  // namespace

sgwls_status run_backward_batched(int B, const sgwls_grad_image* imgs, const sgwls_params* p, void* ws,
                                  cudaStream_t st) {
  const BwdBatchLayout lo = bwd_batch_layout(B, imgs, p);
  char* wsb = static_cast<char*>(ws);
  const int r = p->r;
  const int npass = 2 * p->iters;
  cudaError_t e;
  std::vector<float*> gg(B), gl(B);
  std::vector<const float*> vbar(B);
  for (int i = 0; i < B; ++i) {
    const size_t plane = (size_t)imgs[i].H * imgs[i].W;
    float* gb = reinterpret_cast<float*>(wsb + lo.gbuf[i]);
    gg[i] = imgs[i].grad_g ? imgs[i].grad_g : gb;
    gl[i] = imgs[i].grad_lambda ? imgs[i].grad_lambda : gb + plane;
    if ((e = cudaMemsetAsync(gg[i], 0, plane * sizeof(float), st)) != cudaSuccess) return cuda_fail(e);
    if ((e = cudaMemsetAsync(gl[i], 0, sizeof(float), st)) != cudaSuccess) return cuda_fail(e);
    vbar[i] = imgs[i].grad_u;
    if (npass == 0) {
      e = cudaMemcpyAsync(imgs[i].grad_f, imgs[i].grad_u, plane * imgs[i].C * sizeof(float),
                          cudaMemcpyDeviceToDevice, st);
      if (e != cudaSuccess) return cuda_fail(e);
    }
  }
  if (npass == 0) return SGWLS_OK;
  if ((e = cudaMemsetAsync(wsb, 0, lo.ncnt, st)) != cudaSuccess) return cuda_fail(e);
  static thread_local ScaleTab scale_tab;
  static thread_local BatchArgs batch_args;
  const int OB = 32 - 2 * r;
  for (int t = npass - 1; t >= 0; --t) {
    const int dir = ((t & 1) == 0) ? p->axis_order : 1 - p->axis_order;
    // vbar / count of every image, one launch per 64 images
    for (int i0 = 0; i0 < B; i0 += kScaleMax) {
      ScaleTab& tb = scale_tab;
      memset(&tb, 0, sizeof(tb));
      tb.n = std::min(kScaleMax, B - i0);
      tb.r = r;
      tb.dir = dir;
      tb.start[0] = 0;
      for (int k = 0; k < tb.n; ++k) {
        const sgwls_grad_image& im = imgs[i0 + k];
        tb.vin[k] = vbar[i0 + k];
        tb.vout[k] = reinterpret_cast<float*>(wsb + lo.w0[i0 + k]);
        tb.H[k] = im.H;
        tb.W[k] = im.W;
        tb.start[k + 1] = tb.start[k] + (long long)im.C * im.H * im.W;
      }
      k_bwd_scale_b<<<(unsigned)((tb.start[tb.n] + 255) / 256), 256, 0, st>>>(tb);
      __atomic_add_fetch(&g_launches, 1ull, __ATOMIC_RELAXED);
      if ((e = cudaGetLastError()) != cudaSuccess) return cuda_fail(e);
    }
    // the adjoint pass of every channel group, one uniform batch per group size
    for (int gsz = 1; gsz <= kGroupMax; ++gsz) {
      const std::vector<BwdJob>& jobs = lo.jobs[gsz - 1];
      const std::vector<size_t>& pos = lo.jobpos[gsz - 1];
      const int CC = 2 * gsz;
      const int h0 = batch_h_bwd(r, CC, p->chunk_lines, lo.keep);
      for (size_t j0 = 0; j0 < jobs.size(); j0 += kBatchMax) {
        const int nb = (int)std::min<size_t>(kBatchMax, jobs.size() - j0);
        BatchArgs* ba = &batch_args;
        memset(ba, 0, sizeof(BatchArgs));
        PassArgs& a = ba->base;
        a.dir = dir;
        a.in_dt = a.out_dt = a.g_dt = DT_F32;
        a.n_in1 = gsz;
        a.step = 1;
        fill_weights(a, p, 1.0f);   // sp0 (lambda applied per image)
        ba->nimg = nb;
        BatchLaunch bl = {};
        bl.G = kGMax;
        bl.keep = lo.keep;
        size_t red_max = 0;
        int b[3] = {0, 0, 0};
        for (int k = 0; k < nb; ++k) {
          const BwdJob& jb = jobs[j0 + k];
          const size_t q = pos[j0 + k];
          const sgwls_grad_image& im = imgs[jb.img];
          const size_t plane = (size_t)im.H * im.W;
          const size_t count = plane * im.C;
          ImgDesc& d = ba->img[k];
          d.in = im.saved + (size_t)t * count + (size_t)jb.c0 * plane;
          d.in2 = reinterpret_cast<const float*>(wsb + lo.w0[jb.img]) + (size_t)jb.c0 * plane;
          d.out = (t == 0 ? im.grad_f : reinterpret_cast<float*>(wsb + lo.w1[jb.img])) + (size_t)jb.c0 * plane;
          d.g = im.g;
          d.grad_g = gg[jb.img];
          d.grad_lam = gl[jb.img];
          d.summ = reinterpret_cast<float*>(wsb + lo.summ[q]);
          d.xsep = reinterpret_cast<float*>(wsb + lo.xsep[q]);
          d.mdata = reinterpret_cast<float*>(wsb + lo.mdata[q]);
          d.band_cnt = reinterpret_cast<int*>(wsb + lo.cnt[q]);
          d.fac = lo.keep ? reinterpret_cast<float*>(wsb + lo.fac[q]) : nullptr;
          d.psi = lo.keep ? reinterpret_cast<float*>(wsb + lo.psi[q]) : nullptr;
          d.plane = (long long)plane;
          d.H = im.H;
          d.W = im.W;
          d.L = dir == 0 ? im.H : im.W;
          d.D = dir == 0 ? im.W : im.H;
          d.nsys = d.D - 2 * r;
          d.sstride = (d.nsys + 31) / 32 * 32;
          const Plan pl = batch_plan(d.L, r, CC, h0);
          d.h = pl.h;
          d.P = pl.P;
          d.ngroups = pl.NG;
          d.lam = im.lambda;
          d.nbx[0] = (d.nsys + 31) / 32;
          d.nbx[1] = (d.nsys + 31) / 32;
          d.nbx[2] = (d.D + OB - 1) / OB;
          d.b0[0] = b[0];
          d.b0[1] = b[1];
          d.b0[2] = b[2];
          b[0] += d.nbx[0] * pl.NG;
          b[1] += d.nbx[1];
          b[2] += d.nbx[2] * pl.NG;
          bl.any_multi |= pl.P > 1;
          bl.any_red |= pl.NG > 1;
          red_max = std::max(red_max, (size_t)pl.NG * n_fields(r, CC) * 32 * sizeof(float));
          bl.smem[0] = smem_summary(r, CC, h0, kGMax);
          bl.smem[2] = lo.keep ? smem_backsub(r, CC, h0, kGMax, 1, true) : smem_recover(r, CC, h0, kGMax, true);
        }
        bl.nblk[0] = b[0];
        bl.nblk[1] = b[1];
        bl.nblk[2] = b[2];
        bl.red_smem = red_max <= kReducedSmemMax;
        bl.smem[1] = bl.red_smem ? red_max : 0;
        if ((e = launch_batch_bwd_any(r, CC, *ba, bl, st)) != cudaSuccess) return cuda_fail(e);
        __atomic_add_fetch(&g_launches, (unsigned long long)(1 + (bl.any_multi ? 1 : 0)), __ATOMIC_RELAXED);
      }
    }
    for (int i = 0; i < B; ++i) vbar[i] = t == 0 ? imgs[i].grad_f : reinterpret_cast<float*>(wsb + lo.w1[i]);
  }
  return SGWLS_OK;
}

// ---------------------------------------------------------------------------
// Line relaxation (opt-in variant): T x (first direction, second direction)
// block-Jacobi passes of the dense 2D WLS system, one banded solve per line.

#define SGWLS_LINE_CC(R)                                                         \
  case R:                                                                        \
    switch (CC) {                                                                \
      case 1: return launch_line_inst<R, 1>(a, st);                              \
      case 2: return launch_line_inst<R, 2>(a, st);                              \
      case 3: return launch_line_inst<R, 3>(a, st);                              \
      case 4: return launch_line_inst<R, 4>(a, st);                              \
      default: return cudaErrorInvalidValue;                                     \
    }
cudaError_t launch_line_any(int r, int CC, const LineArgs& a, cudaStream_t st) {
  switch (r) {
    SGWLS_LINE_CC(1) SGWLS_LINE_CC(2) SGWLS_LINE_CC(3) SGWLS_LINE_CC(4)
    default: return cudaErrorInvalidValue;
  }
}
#undef SGWLS_LINE_CC

namespace {

struct LineLayout {
  size_t img, scratch, total;
};

LineLayout line_layout(int H, int W, int C, const sgwls_params* p) {
  LineLayout lo;
  lo.img = 0;
  const size_t img = p->iters > 0 ? align256((size_t)C * H * W * sizeof(float)) : 0;
  lo.scratch = img;
  const int CCmax = std::min(kGroupMax, C);
  lo.total = img + align256((size_t)H * W * (p->r + CCmax) * sizeof(float));
  return lo;
}

sgwls_status check_line(int H, int W, int C, const sgwls_params* p) {
  sgwls_status s = check_params(H, W, C, p);
  if (s != SGWLS_OK) return s;
  if (p->storage != SGWLS_F32 || p->inter_storage != SGWLS_F32) return SGWLS_E_UNSUPPORTED;
  if (p->r > kLineRMax || p->step != 1 || p->refine || p->guide_channels > 1) return SGWLS_E_UNSUPPORTED;
  return SGWLS_OK;
}

}  // namespace

sgwls_status run_line_relax(const float* f, const float* g, float* u, int H, int W, int C, float lambda,
                            const sgwls_params* p, void* ws, cudaStream_t st) {
  const LineLayout lo = line_layout(H, W, C, p);
  char* wsb = static_cast<char*>(ws);
  const long long plane = (long long)H * W;
  cudaError_t e;
  const int npass = 2 * p->iters;
  if (npass == 0) {
    e = cudaMemcpyAsync(u, f, (size_t)plane * C * sizeof(float), cudaMemcpyDeviceToDevice, st);
    return e == cudaSuccess ? SGWLS_OK : cuda_fail(e);
  }
  LineArgs a;
  memset(&a, 0, sizeof(a));
  a.g = g;
  a.plane = plane;
  a.H = H;
  a.W = W;
  a.weight = p->weight;
  a.range_k = p->weight == SGWLS_W_EXP ? (float)(-1.4426950408889634 / (2.0 * (double)p->sigma_r * p->sigma_r))
                                       : p->alpha_r;
  a.eps = p->eps;
  const int r = p->r, S = 2 * r + 1;
  for (int dy = -r; dy <= r; ++dy)
    for (int dx = -r; dx <= r; ++dx) {
      const double d2 = (double)dx * dx + (double)dy * dy;
      const double sp = p->weight == SGWLS_W_EXP ? exp(-d2 / (2.0 * (double)p->sigma_s * p->sigma_s))
                                                 : 1.0 / (pow(sqrt(d2), (double)p->alpha_s) + (double)p->eps);
      a.wsp[(dy + r) * S + dx + r] = (float)(lambda * sp);
    }
  a.scratch = reinterpret_cast<float*>(wsb + lo.scratch);
  float* img = reinterpret_cast<float*>(wsb + lo.img);
  const float* cur = f;
  for (int t = 0; t < npass; ++t) {
    a.dir = ((t & 1) == 0) ? p->axis_order : 1 - p->axis_order;
    float* dst = (t == npass - 1) ? u : (((npass - 1 - t) & 1) ? img : u);
    for (int c0 = 0; c0 < C; c0 += kGroupMax) {
      const int CC = std::min(kGroupMax, C - c0);
      a.f = f + (size_t)c0 * plane;
      a.uin = cur + (size_t)c0 * plane;
      a.uout = dst + (size_t)c0 * plane;
      if ((e = launch_line_any(r, CC, a, st)) != cudaSuccess) return cuda_fail(e);
      __atomic_add_fetch(&g_launches, 1ull, __ATOMIC_RELAXED);
    }
    cur = dst;
  }
  return SGWLS_OK;
}

}  // namespace sgwls

using namespace sgwls;

extern "C" {

void sgwls_params_default(sgwls_params* p) {
  if (!p) return;
  p->weight = SGWLS_W_EXP;
  p->sigma_s = 1.0f;
  p->sigma_r = 0.1f;
  p->alpha_s = 1.2f;
  p->alpha_r = 1.2f;
  p->eps = 1e-4f;
  p->r = 1;
  p->iters = 1;
  p->step = 1;
  p->axis_order = 0;
  p->refine = 0;
  p->storage = SGWLS_F32;
  p->inter_storage = SGWLS_F32;
  p->chunk_lines = 0;
  p->factor_cache = 0;
  p->guide_channels = 1;
  p->schedule = 0;
  p->ring_slots = 0;
  p->group_warps = 0;
  p->lookahead = 0;
}

const char* sgwls_status_string(sgwls_status s) {
  switch (s) {
    case SGWLS_OK: return "SGWLS_OK";
    case SGWLS_E_INVALID: return "SGWLS_E_INVALID: invalid argument";
    case SGWLS_E_SHAPE: return "SGWLS_E_SHAPE: invalid image shape";
    case SGWLS_E_DTYPE: return "SGWLS_E_DTYPE: unknown storage type";
    case SGWLS_E_WORKSPACE: return "SGWLS_E_WORKSPACE: workspace missing or too small";
    case SGWLS_E_CUDA: return "SGWLS_E_CUDA: CUDA error";
    case SGWLS_E_DEVICE_FLAG: return "SGWLS_E_DEVICE_FLAG: kernel reported an error";
    case SGWLS_E_UNSUPPORTED: return "SGWLS_E_UNSUPPORTED: not implemented in this build";
  }
  return "SGWLS_E_?: unknown status";
}

const char* sgwls_last_cuda_error(void) { return g_cuda_err; }

size_t sgwls_workspace_bytes(int H, int W, int C, const sgwls_params* p) {
  if (check_params(H, W, C, p) != SGWLS_OK || check_step(H, W, C, p) != SGWLS_OK) return 0;
  return make_layout(H, W, C, p).total;
}

sgwls_status sgwls_filter(const void* f, const void* g, void* u, int H, int W, int C, float lambda,
                          const sgwls_params* p, void* ws, size_t ws_bytes, void* saved, void* stream) {
  const sgwls_status s = check_pass_params(H, W, C, p);
  if (s != SGWLS_OK) return s;
  if (!f || !g || !u || f == u || g == u) return SGWLS_E_INVALID;
  if (!(lambda >= 0.f) || !isfinite(lambda)) return SGWLS_E_INVALID;
  const size_t need = make_layout(H, W, C, p).total;
  if (need > 0 && (!ws || ws_bytes < need || (reinterpret_cast<uintptr_t>(ws) & 255))) return SGWLS_E_WORKSPACE;
  return run_filter(f, g, u, H, W, C, lambda, p, ws, saved, static_cast<cudaStream_t>(stream));
}

sgwls_status sgwls_filter_pass(const void* f, const void* g, void* u, int H, int W, int C, float lambda,
                               const sgwls_params* p, int direction, void* ws, size_t ws_bytes, void* stream) {
  const sgwls_status s = check_pass_params(H, W, C, p);
  if (s != SGWLS_OK) return s;
  if (!f || !g || !u || f == u || g == u) return SGWLS_E_INVALID;
  if (direction != 0 && direction != 1) return SGWLS_E_INVALID;
  if (!(lambda >= 0.f) || !isfinite(lambda)) return SGWLS_E_INVALID;
  const Layout lo = make_layout(H, W, C, p);
  if (!ws || ws_bytes < lo.total || (reinterpret_cast<uintptr_t>(ws) & 255)) return SGWLS_E_WORKSPACE;
  return run_pass(f, p->storage, u, p->storage, g, H, W, C, lambda, p, direction, ws,
                  static_cast<cudaStream_t>(stream), true);
}

size_t sgwls_interpolate_workspace_bytes(int H, int W, int C, const sgwls_params* p) {
  if (C < 1 || C + 1 > SGWLS_C_MAX || check_params(H, W, C + 1, p) != SGWLS_OK) return 0;
  if (check_step(H, W, C + 1, p) != SGWLS_OK) return 0;
  return make_interp_layout(H, W, C, p).total;
}

sgwls_status sgwls_interpolate(const void* f, const void* hmap, const void* g, void* u, int H, int W, int C,
                               float lambda, const sgwls_params* p, void* ws, size_t ws_bytes, void* stream) {
  if (C < 1 || C + 1 > SGWLS_C_MAX) return SGWLS_E_SHAPE;
  sgwls_status s = check_params(H, W, C + 1, p);
  if (s == SGWLS_OK) s = check_step(H, W, C + 1, p);
  if (s != SGWLS_OK) return s;
  if (p->storage != SGWLS_F32 || p->inter_storage != SGWLS_F32) return SGWLS_E_UNSUPPORTED;
  if (!f || !hmap || !g || !u || u == f || u == hmap) return SGWLS_E_INVALID;
  if (!(lambda >= 0.f) || !isfinite(lambda)) return SGWLS_E_INVALID;
  const size_t need = make_interp_layout(H, W, C, p).total;
  if (!ws || ws_bytes < need || (reinterpret_cast<uintptr_t>(ws) & 255)) return SGWLS_E_WORKSPACE;
  return run_interpolate(static_cast<const float*>(f), static_cast<const float*>(hmap), static_cast<const float*>(g),
                         static_cast<float*>(u), H, W, C, lambda, p, ws, static_cast<cudaStream_t>(stream));
}

unsigned long long sgwls_launch_count(void) { return __atomic_load_n(&g_launches, __ATOMIC_RELAXED); }

sgwls_status sgwls_device_flag(int clear) {
  unsigned* ptr = nullptr;
  cudaError_t e = device_flag_ptr(&ptr);
  if (e != cudaSuccess) return cuda_fail(e);
  unsigned v = 0;
  if ((e = cudaMemcpy(&v, ptr, sizeof(v), cudaMemcpyDeviceToHost)) != cudaSuccess) return cuda_fail(e);
  if (clear && v != 0u && (e = cudaMemset(ptr, 0, sizeof(unsigned))) != cudaSuccess) return cuda_fail(e);
  return v ? SGWLS_E_DEVICE_FLAG : SGWLS_OK;
}

}  // extern "C"

extern "C" {

size_t sgwls_backward_workspace_bytes(int H, int W, int C, const sgwls_params* p) {
  if (check_params(H, W, C, p) != SGWLS_OK || p->step != 1) return 0;
  return make_bwd_layout(H, W, C, p).total;
}

sgwls_status sgwls_filter_backward(const void* grad_u, const void* g, const void* saved, int H, int W, int C,
                                   float lambda, const sgwls_params* p, void* grad_f, void* grad_g,
                                   float* grad_lambda, void* ws, size_t ws_bytes, void* stream) {
  sgwls_status s = check_params(H, W, C, p);
  if (s != SGWLS_OK) return s;
  if (!grad_u || !g || !grad_f || (p->iters > 0 && !saved)) return SGWLS_E_INVALID;
  if (grad_f == grad_u) return SGWLS_E_INVALID;
  if (!(lambda >= 0.f) || !isfinite(lambda)) return SGWLS_E_INVALID;
  if (p->storage != SGWLS_F32 || p->inter_storage != SGWLS_F32) return SGWLS_E_UNSUPPORTED;
  if (p->weight == SGWLS_W_FRAC && p->alpha_r < 1.f) return SGWLS_E_UNSUPPORTED;
  if (p->step != 1 || p->refine || p->guide_channels > 1) return SGWLS_E_UNSUPPORTED;
  const size_t need = make_bwd_layout(H, W, C, p).total;
  if (!ws || ws_bytes < need || (reinterpret_cast<uintptr_t>(ws) & 255)) return SGWLS_E_WORKSPACE;
  return run_backward(static_cast<const float*>(grad_u), static_cast<const float*>(g),
                      static_cast<const float*>(saved), H, W, C, lambda, p, static_cast<float*>(grad_f),
                      static_cast<float*>(grad_g), grad_lambda, ws, static_cast<cudaStream_t>(stream));
}

}  // extern "C"

extern "C" {

size_t sgwls_batched_workspace_bytes(int B, const sgwls_image* imgs, const sgwls_params* p) {
  if (check_batch(B, imgs, p) != SGWLS_OK) return 0;
  return batch_workspace_any(B, imgs, p);
}

size_t sgwls_line_relax_workspace_bytes(int H, int W, int C, const sgwls_params* p) {
  if (check_line(H, W, C, p) != SGWLS_OK) return 0;
  return line_layout(H, W, C, p).total;
}

sgwls_status sgwls_line_relax(const void* f, const void* g, void* u, int H, int W, int C, float lambda,
                              const sgwls_params* p, void* ws, size_t ws_bytes, void* stream) {
  sgwls_status s = check_line(H, W, C, p);
  if (s != SGWLS_OK) return s;
  if (!f || !g || !u || f == u || g == u) return SGWLS_E_INVALID;
  if (!(lambda >= 0.f) || !isfinite(lambda)) return SGWLS_E_INVALID;
  const size_t need = line_layout(H, W, C, p).total;
  if (!ws || ws_bytes < need || (reinterpret_cast<uintptr_t>(ws) & 255)) return SGWLS_E_WORKSPACE;
  return run_line_relax(static_cast<const float*>(f), static_cast<const float*>(g), static_cast<float*>(u), H, W,
                        C, lambda, p, ws, static_cast<cudaStream_t>(stream));
}

size_t sgwls_backward_batched_workspace_bytes(int B, const sgwls_grad_image* imgs, const sgwls_params* p) {
  if (check_batch_bwd(B, imgs, p) != SGWLS_OK) return 0;
  return bwd_batch_layout(B, imgs, p).total;
}

sgwls_status sgwls_filter_backward_batched(int B, const sgwls_grad_image* imgs, const sgwls_params* p, void* ws,
                                           size_t ws_bytes, void* stream) {
  sgwls_status s = check_batch_bwd(B, imgs, p);
  if (s != SGWLS_OK) return s;
  const size_t need = bwd_batch_layout(B, imgs, p).total;
  if (!ws || ws_bytes < need || (reinterpret_cast<uintptr_t>(ws) & 255)) return SGWLS_E_WORKSPACE;
  return run_backward_batched(B, imgs, p, ws, static_cast<cudaStream_t>(stream));
}

sgwls_status sgwls_filter_batched(int B, const sgwls_image* imgs, const sgwls_params* p, void* ws, size_t ws_bytes,
                                  void* stream) {
  sgwls_status s = check_batch(B, imgs, p);
  if (s != SGWLS_OK) return s;
  const size_t need = batch_workspace_any(B, imgs, p);
  if (need > 0 && (!ws || ws_bytes < need || (reinterpret_cast<uintptr_t>(ws) & 255))) return SGWLS_E_WORKSPACE;
  return run_batched_any(B, imgs, p, ws, static_cast<cudaStream_t>(stream));
}

}  // extern "C"
