// sgwls_common.cuh -- argument block and small device helpers shared by the
// SG-WLS pass kernels.
//
// Geometry of one pass (Sec. 2.1).  A pass runs along one direction:
//   dir 0 ("column direction"): centres are columns k, the formed vector runs
//        down the image rows; lines = rows (L = H), across = columns (D = W).
//   dir 1 ("row direction"): centres are rows k, the vector runs along the
//        columns; lines = columns (L = W), across = rows (D = H).
// Entry p of the vector of centre k sits on line p / n at across-offset
//   k - r + j   (line even, 0-based; the paper's odd 1-based rows), or
//   k + r - j   (line odd: reversed), with j = p % n and n = 2r + 1.
#pragma once

#include <cuda.h>   // CUtensorMap (the tensor-copy descriptors of the tile staging)
#include <cuda_runtime.h>
#include <cuda_bf16.h>
#include <stdint.h>

#include <type_traits>
#include <utility>

namespace sgwls {

constexpr int kRMax = 8;
constexpr int kGroupMax = 4;   // channels solved together against one factor
constexpr int kBwdWideRhs = 6; // right-hand sides of the backward's widest group (r = 1)

enum : int { DT_F32 = 0, DT_BF16 = 1 };

struct PassArgs {
  const void* in;      // C planes, dtype in_dt
  const void* g;       // guidance planes (gc of them, planar), dtype g_dt
  int gc;              // guidance channels: 1, or 2..4 (vector guidance, |G_i - G_j| the Euclidean norm)
  void* out;           // C planes, dtype out_dt
  long long plane;     // H * W (elements per plane)
  int H, W;
  int in_dt, g_dt, out_dt;
  int dir;             // 0 column direction, 1 row direction
  int D;               // extent across the lines (number of columns for dir 0)
  int L;               // number of lines (rows for dir 0)
  int nsys;            // number of centres (subsystems): D - 2r for step 1
  int step;            // sliding step tau between centres (Sec. 2.3)
  int nreg;            // regular centres r + s step, s < nreg; centre nsys-1 = D-1-r when nsys > nreg
  int sstride;         // subsystem stride of the scratch arrays: nsys rounded up to 32
  int h;               // lines per chunk
  int P;               // chunks per subsystem
  int ngroups;         // chunk groups (one block of G chunks each)
  float lam;           // lambda
  int weight;          // 0 exp, 1 frac
  float range_k;       // exp: -log2(e) / (2 sigma_r^2);  frac: alpha_r
  float eps;           // frac epsilon
  // lambda * spatial factor of the pair (p, p+t) for j = p % n, t = 1..r:
  // sp[j * r + t - 1]
  float sp[(2 * kRMax + 1) * kRMax];
  float* summ;         // group 2-ports     [NG][Fields::N][nsys]
  float* xsep;         // group separators  [NG-1][r*CC][nsys]
  float* mdata;        // merge factors     [NG][G-1][MFields::N][nsys]
  int early_stage;     // k_recover may stage its tile before griddep_wait
  int* band_cnt;       // per band of 32 subsystems: k_summary blocks finished (0 between passes)
  int chain_smem;      // the reduced chain of a band fits in k_summary's shared memory
  // Chunk factors kept between the two kernels of a pass (null: k_recover
  // recomputes them), per band of 32 subsystems (sys = 32 band + lane):
  // fac[band][e][f][lane] for vector entry e of an interior: f < r:
  // L[e, e-1..e-r]; then z0 = D^-1 L^-1 f (CC values); then Phi =
  // -D^-1 L^-1 A(I, S_top) (r values, chunks with a top separator).
  // psi[band][c][k][i][lane]: the bottom-separator column i of
  // -D^-1 L^-1 A(I, S_bot) at chunk c's k-th of its last r interior entries
  // (the only rows where it is not zero).
  float* fac;
  float* psi;
  // Queue-scheduled pass (k_pass_q): the factor store is a ring of nslot
  // band slots (0: one slot per band, the two-kernel pass); per band
  // `done` (its summary items and reduced system finished) and `rdcnt`
  // (back-substitution items that finished reading it); qctl[0] the work
  // queue, qctl[1] the count of blocks that left; `lookahead` bands between
  // a band's summary items and the back-substitution items that need it.
  // `err` (device word, shared by all calls) is set when a wait gives up.
  int nslot;
  int lookahead;
  int* done;
  int* rdcnt;
  int* qctl;
  unsigned* err;
  // Tensor-copy (TMA) staging of the column direction's tiles (FP32, step
  // 1, one guidance plane, 16-byte-aligned rows): tm_in maps the CC
  // estimate planes as a 3D tensor (W, H, CC), tm_g the guidance as 2D
  // (W, H); both boxes are pitch x (G h + 2) floats.  0: the other staging.
  int tma;
  CUtensorMap tm_in;
  CUtensorMap tm_g;
  // Refinement of each subsystem solve (refine = 1): first solve with
  // xmode 1 (every entry's solution to xent, no averaging); k_resid forms
  // rho = f - A u in FP32 (A's identity kept apart) into rhs; second solve with rhs as the
  // right-hand side and xmode 2 (xent added before the averaging).  Both
  // buffers are [band][e][CC][32] (e = vector entry, 32 subsystems a band).
  float* rhs;
  float* xent;
  int xmode;
  int refine;          // host: this pass runs the two solves and the residual
  // Planes 0 .. n_in1-1 come from `in`, planes n_in1 .. CC-1 from `in2`
  // (the backward solves u = A^-1 f and v = A^-1 ubar together).
  const void* in2;
  int n_in1;
  // backward only: accumulated d loss / d guidance (FP32, the pass's pixel
  // grid) and d loss / d lambda (one float); the spatial factor without
  // lambda, sp0[j * r + t - 1]; dgk = 1 / sigma_r^2 (exp weights)
  float* grad_g;
  float* grad_lam;
  float sp0[(2 * kRMax + 1) * kRMax];
  float dgk;
};

// Across-offset of the centre of subsystem s: r + s step for the regular
// centres; the last centre D-1-r is appended when the stride misses it
// (Sec. 2.3 sliding construction; every line stays covered).
__device__ __forceinline__ int centre_of(const PassArgs& a, int s, int r) {
  return s < a.nreg ? r + s * a.step : a.D - 1 - r;
}

__device__ __forceinline__ float ld_px(const void* base, long long idx, int dt) {
  if (dt == DT_F32) return __ldg(reinterpret_cast<const float*>(base) + idx);
  const unsigned short raw = __ldg(reinterpret_cast<const unsigned short*>(base) + idx);
  return __uint_as_float(static_cast<unsigned>(raw) << 16);
}

__device__ __forceinline__ void st_px(void* base, long long idx, int dt, float v) {
  if (dt == DT_F32) {
    reinterpret_cast<float*>(base)[idx] = v;
  } else {
    reinterpret_cast<__nv_bfloat16*>(base)[idx] = __float2bfloat16_rn(v);
  }
}

// Pixel index of (line, across-offset) for the pass direction.
__device__ __forceinline__ long long pix_index(const PassArgs& a, int line, int off) {
  return a.dir == 0 ? (long long)line * a.W + off : (long long)off * a.W + line;
}

__device__ __forceinline__ float fast_ex2(float x) {
  float y;
  asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}

// Range factor of Eq. 2 for the guidance difference dg: exp weights use the
// hardware base-2 exponential on dg^2 * (-log2(e) / (2 sigma_r^2)).
__device__ __forceinline__ float range_factor(const PassArgs& a, float dg) {
  if (a.weight == 0) return fast_ex2(dg * dg * a.range_k);
  return 1.0f / (powf(fabsf(dg), a.range_k) + a.eps);
}

// The same for a vector guidance, from the squared norm d2 of the
// difference: exp(-d2 / (2 sigma_r^2)), or 1 / (d2^(alpha_r / 2) + eps).
__device__ __forceinline__ float range_factor_sq(const PassArgs& a, float d2) {
  if (a.weight == 0) return fast_ex2(d2 * a.range_k);
  return 1.0f / (powf(d2, 0.5f * a.range_k) + a.eps);
}

// Programmatic dependent launch: wait for the preceding kernel of the stream
// to complete (its memory is then visible), and allow the next kernel to be
// scheduled.  Every kernel here calls launch_dependents only after its own
// wait, so a kernel that runs code before its wait may read anything written
// two or more kernels earlier.
__device__ __forceinline__ void griddep_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void griddep_launch() { asm volatile("griddepcontrol.launch_dependents;" :::); }

// Nanoseconds of the global timer (for the time limit of a wait).
__device__ __forceinline__ unsigned long long global_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

__device__ __forceinline__ int ld_acquire(const int* p) {
  int v;
  asm volatile("ld.acquire.gpu.global.b32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

// Waits (one thread) until *p >= v.  Gives up, sets bit `code` of *err and
// returns false after at least 2^20 polls and 2 s of global time (both, so
// that time the context spends switched out does not count alone), or as
// soon as another block has set *err; the caller then skips its work and the
// host reads the flag (sgwls_device_flag).  Every wait of this library is
// on work that an earlier-scheduled, already running block holds, so the
// limit is not reached in a correct run.
__device__ __forceinline__ bool wait_geq(const int* p, int v, unsigned* err, unsigned code) {
  if (ld_acquire(p) >= v) return true;
  const unsigned long long t0 = global_ns();
  for (unsigned it = 1;; ++it) {
    __nanosleep(it < 16 ? 32 : 256);
    if (ld_acquire(p) >= v) return true;
    if ((it & 63) == 0) {
      if (*reinterpret_cast<const volatile unsigned*>(err) != 0u) return false;
      if (it >= (1u << 20) && global_ns() - t0 > 2000000000ull) {
        atomicOr(err, code);
        return false;
      }
    }
  }
}

// ---- tensor copies (TMA) completed on a shared-memory mbarrier
__device__ __forceinline__ unsigned smem_u32(const void* p) {
  return static_cast<unsigned>(__cvta_generic_to_shared(p));
}
__device__ __forceinline__ void mbar_init(unsigned long long* bar, unsigned count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
  // make the initialised barrier visible to the tensor-copy (async) proxy
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}
__device__ __forceinline__ void mbar_expect_tx(unsigned long long* bar, unsigned bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes) : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(unsigned long long* bar, unsigned parity) {
  unsigned ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}
// 2D / 3D box of a tensor map into shared memory (coordinates in elements,
// innermost first), completing `bar` with the box's bytes.
__device__ __forceinline__ void tma_load_2d(float* dst, const CUtensorMap* map, int x, int y,
                                            unsigned long long* bar) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];"
      ::"r"(smem_u32(dst)), "l"(reinterpret_cast<unsigned long long>(map)), "r"(x), "r"(y), "r"(smem_u32(bar))
      : "memory");
}
__device__ __forceinline__ void tma_load_3d(float* dst, const CUtensorMap* map, int x, int y, int z,
                                            unsigned long long* bar) {
  asm volatile(
      "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], "
      "[%5];"
      ::"r"(smem_u32(dst)), "l"(reinterpret_cast<unsigned long long>(map)), "r"(x), "r"(y), "r"(z),
        "r"(smem_u32(bar))
      : "memory");
}
// Waits (every thread) for phase `parity` of `bar`: at least 2^20 polls and
// 2 s, then the error flag is set and the wait continues for as long again
// (the copies in flight target this block's shared memory) before it gives
// up; returns false if it timed out.
__device__ __forceinline__ bool mbar_wait_bounded(unsigned long long* bar, unsigned parity, unsigned* err) {
  if (mbar_try_wait(bar, parity)) return true;
  unsigned long long t0 = global_ns();
  bool flagged = false;
  for (unsigned it = 1;; ++it) {
    if (mbar_try_wait(bar, parity)) return !flagged;
    if ((it & 63) == 0 && it >= (1u << 20) && global_ns() - t0 > 2000000000ull) {
      if (flagged) return false;
      if (err) atomicOr(err, 4u);
      flagged = true;
      it = 0;
      t0 = global_ns();
    }
  }
}

__device__ __forceinline__ float fast_rcp(float x) {
  float y;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}

}  // namespace sgwls
