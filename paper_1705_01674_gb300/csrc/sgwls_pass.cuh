// sgwls_pass.cuh -- one SG-WLS pass (Sec. 2.3) as two kernels.
//
// Every subsystem A_s u = f (Eq. 5) of a pass is a symmetric positive
// definite banded matrix of half-bandwidth r and length s = (2r+1) * lines.
// A_s is strictly diagonally dominant (diagonal minus the off-diagonal sum is
// 1, from the Eq. 4 form), so an FP32 LDL^T without pivoting is stable.  The
// paper factors each subsystem serially (its r-band LU, Eqs. 9-20); a GPU
// needs far more parallelism than one thread per subsystem, so each
// subsystem is split along its lines into P chunks and solved exactly by
// Schur-complement (nested dissection) reduction:
//
//   chunk c covers lines [c h, min((c+1) h, L)), vector entries [b, end);
//   its last r entries S_c (c < P-1) are the separator shared with chunk
//   c+1; the rest is the interior I_c = [b, e).  Interiors couple only to
//   the separators on both sides (bandwidth r < 2r+1 = entries per line).
//
// Eliminating a chunk's interior leaves a "2-port" on (S_{c-1}, S_c): the
// Schur complement's couplings among the separator entries, the margins
// (row sums) it passes on to them, and the reduced right-hand sides, with
// A(I,I) = L D L^T, Y_T = L^-1 A(I,S_{c-1}), Y_B = L^-1 A(I,S_c) and
// y = L^-1 f(I).  Every pivot is formed as a margin plus coupling
// magnitudes, a sum of non-negative terms (see gth_row), in the sweeps and
// in the merges, so FP32 keeps the identity of A_s even where lambda w is
// ~1e7.  Consecutive 2-ports merge by eliminating their shared separator
// (an associative operation), so the reduction is hierarchical:
//
//   k_summary   block = 32 neighbouring subsystems (lanes) x G chunks (warps).
//               The block stages its strip tile (estimate planes and guidance)
//               in shared memory, every thread eliminates its chunk's
//               interior (forward sweep) and, when the pass keeps its factors,
//               stores each entry's LDL^T row, z0 = D^-1 L^-1 f and top-port
//               column; the warps then merge the block's G chunk 2-ports into
//               one group 2-port as a binary tree, keeping the merge factors
//               for the back-fill.  The last block of each band to finish
//               solves the band's reduced system: the chain of the group
//               2-ports, eliminated separator by separator in margin form
//               (r x r blocks), split into segments that the warps fold in
//               parallel.
//   k_backsub   block = 32 neighbouring centres x G chunks.  The warps
//               back-fill the separators inside the group down the merge
//               tree; every thread back-substitutes its interior from the kept
//               factors, writes the solution back into the strip and averages
//               each pixel's 2r+1 values across the neighbouring centres'
//               lanes with warp shuffles (steps 3-4 of Sec. 2.3), one output
//               line at a time.
//   k_recover   the same without kept factors: it re-stages the tile and
//               repeats the forward sweep into shared memory before the
//               backward sweep (also the adjoint pass of the backward).
//   k_resid     the refinement's residual f - A u for every vector entry,
//               in FP32 with A's identity kept apart from its Laplacian.
//   k_pass_q    a forward pass with kept factors at step 1 as ONE
//               persistent kernel: its blocks take k_summary and k_backsub
//               work items from a queue, band by band, so a band's factors
//               (a ring of band slots) are read back while still in L2.
//
// Compile-time modes: k_summary keeps its factors or not, takes its
// right-hand sides from the tile or from the refinement's residual, and
// reads one guidance plane or several (the norm of the guidance
// difference); k_backsub runs step 1, a sliding step > 1 (a lane per
// centre, averaging through shared memory) or the refinement's two solves.
//
// The sweeps run one line of the vector at a time with the line's parity
// (snake direction) and its first/last role fixed at compile time, so every
// index inside a line is static.
#pragma once

#include "sgwls_common.cuh"
#include "sgwls_sched.h"

namespace sgwls {

// 2-port fields (chunk 2-port, and group 2-port in the same format), all
// in margin form: KTT off the diagonal the magnitude of the T_i - T_m
// coupling Y_T' D^-1 Y_T induces, on it the margin the eliminated entries
// pass to T_i; KTB the magnitude of the T_i - B_m coupling (Y_T' D^-1 Y_B);
// DS off the diagonal the magnitude of the B_i - B_m coupling (A's own plus
// Y_B' D^-1 Y_B), on it B_i's margin (its own 1 plus what it received); HT
// the right-hand side the eliminated entries add to T_i (-Y_T' D^-1 y); GS
// B_i's reduced right-hand side (f(S_c) - Y_B' D^-1 y).
template <int R, int CC>
struct Fields {
  static constexpr int KTT = 0;
  static constexpr int KTB = R * R;
  static constexpr int DS = 2 * R * R;
  static constexpr int HT = 3 * R * R;
  static constexpr int GS = 3 * R * R + R * CC;
  static constexpr int N = 3 * R * R + 2 * R * CC;
};

// Merge factors kept for the back-fill (see fold_2ports): LM the eliminated
// separator's L^T multipliers below the diagonal and reciprocal pivots on
// it, U and V its couplings to the outer ports and W its right-hand side,
// each divided by its entry's pivot.
template <int R, int CC>
struct MFields {
  static constexpr int LM = 0;
  static constexpr int U = R * R;
  static constexpr int V = 2 * R * R;
  static constexpr int W = 3 * R * R;
  static constexpr int N = 3 * R * R + R * CC;
};

// ---------------------------------------------------------------------------
// Shared-memory strip tile: planes 0..CC-1 = estimate channels, then the
// guidance plane(s); tile[plane * pstride + tl * pitch + col] holds (line
// tl0 + tl, across-offset off0 + col), zero outside the image.  pitch is odd
// so the transposed staging of the row direction is free of bank conflicts;
// pstride (>= ntl * pitch) is a multiple of 32 floats, so every plane starts
// on a 128-byte boundary (the destination alignment of a tensor copy).
struct Tile {
  float* p;
  int tl0, ntl, off0, pitch;
  int pstride;   // floats between planes
  int cs;        // physical column of across-offset off0 (vector-aligned staging)
  int ncol;      // staged columns (runtime-width staging of the sliding-step path)
  __device__ __forceinline__ const float* row(int plane, int line) const {
    return p + plane * pstride + (line - tl0) * pitch + cs;
  }
};

// k_summary writes its chunk 2-ports over the strip tile (radius <= 3).
__host__ __device__ constexpr bool tile_over_2ports(int r) { return r <= 3; }

// Floats between tile planes for ntl lines of `pitch` floats.
__host__ __device__ constexpr int tile_pstride(int ntl, int pitch) { return (ntl * pitch + 31) / 32 * 32; }

// Tile columns of a band of 32 subsystems: their strips of 2r+1 offsets,
// centres step apart (the appended last centre lies inside that span).
__host__ __device__ constexpr int tile_ncol(int r, int step) { return 31 * step + 2 * r + 1; }
// Row pitch of the tile in floats: column direction, rows of whole 16-byte
// quads starting at the 16-byte boundary at or before off0; row direction,
// an odd pitch (transposed staging without bank conflicts).
__host__ __device__ constexpr int tile_pitch_n(int ncol, int dir) {
  return dir == 0 ? 4 * ((ncol + 3 + 3) / 4) : (ncol | 1);
}
__host__ __device__ constexpr int tile_pitch(int r, int dir) { return tile_pitch_n(32 + 2 * r, dir); }
__host__ __device__ constexpr int tile_pitch_max(int r) {
  return tile_pitch(r, 0) > tile_pitch(r, 1) ? tile_pitch(r, 0) : tile_pitch(r, 1);
}

// Sliding step > 1 (k_backsub): each warp's lanes are 32 consecutive
// subsystems, ceil(r / step) + 1 of them on each side halo lanes whose
// values reach the owned columns (the + 1: the appended last centre lies
// less than step beyond the last regular one, so it reaches one subsystem
// further back); a warp owns the columns from its first owned centre to the
// next warp's (at most step per owned lane, plus the border columns before
// the first centre and after the last).
__host__ __device__ constexpr int step_halo(int r, int step) { return step == 1 ? r : (r + step - 1) / step + 1; }
__host__ __device__ constexpr int step_owned_lanes(int r, int step) { return 32 - 2 * step_halo(r, step); }
__host__ __device__ constexpr int step_own_max(int r, int step) {
  return step == 1 ? 32 - 2 * r : step_owned_lanes(r, step) * step + 2 * r + 1;
}
__host__ __device__ constexpr int step_acc_width(int r, int step) { return 32 * step + 2 * r + 2; }

// Base of tile plane pl: estimate planes from `in` (then `in2`), the
// guidance planes last.  `elem` is the element size of plane pl's type.
template <int CC>
__device__ __forceinline__ const char* plane_base(const PassArgs& a, int pl, int elem) {
  if (pl < a.n_in1) return static_cast<const char*>(a.in) + (size_t)pl * a.plane * elem;
  if (pl < CC) return static_cast<const char*>(a.in2) + (size_t)(pl - a.n_in1) * a.plane * elem;
  return static_cast<const char*>(a.g) + (size_t)(pl - CC) * a.plane * elem;
}

// Mixed storage types (BF16 guidance with FP32 estimates): plain loop.
template <int CC>
__device__ __noinline__ void stage_tile_mixed(const PassArgs& a, const Tile& t, int ncol, int p0, int p1) {
  const int nthreads = blockDim.x * blockDim.y;
  const int tid = threadIdx.y * blockDim.x + threadIdx.x;
  const int per_plane = t.ntl * ncol;
  for (int idx = tid; idx < (p1 - p0) * per_plane; idx += nthreads) {
    const int pl = p0 + idx / per_plane;
    const int rest = idx - (pl - p0) * per_plane;
    const int tl = rest / ncol, col = rest - tl * ncol;
    const int line = t.tl0 + tl, off = t.off0 + col;
    float v = 0.f;
    if (line >= 0 && line < a.L && off >= 0 && off < a.D) {
      const long long pix = pix_index(a, line, off);
      v = pl < CC ? ld_px(plane_base<CC>(a, pl, a.in_dt == DT_F32 ? 4 : 2), pix, a.in_dt)
                  : ld_px(plane_base<CC>(a, pl, a.g_dt == DT_F32 ? 4 : 2), pix, a.g_dt);
    }
    t.p[pl * t.pstride + tl * t.pitch + col] = v;
  }
}

// Loads one value of plane `pl` (a.in channels, then the guidance).
template <bool F32>
__device__ __forceinline__ float ld_plane(const void* base, long long idx) {
  if (F32) return __ldg(reinterpret_cast<const float*>(base) + idx);
  const unsigned short raw = __ldg(reinterpret_cast<const unsigned short*>(base) + idx);
  return __uint_as_float(static_cast<unsigned>(raw) << 16);
}

// Stages planes x lines x ncol values, zero outside the image.  Column
// direction: lanes along the offsets (contiguous in memory), warps over the
// lines.  Row direction: lanes along the lines (contiguous in memory), warps
// over the offsets.  Each thread issues U loads before its stores.
template <int CC, bool F32>
__device__ __noinline__ void stage_tile_t(const PassArgs& a, const Tile& t, int ncol, int p0, int p1) {
  const int lane = threadIdx.x, warp = threadIdx.y, nw = blockDim.y;
  constexpr int U = 4;
#pragma unroll 1
  for (int pl = p0; pl < p1; ++pl) {
    const char* base = plane_base<CC>(a, pl, F32 ? 4 : 2);
    float* dplane = t.p + pl * t.pstride;
    if (a.dir == 0) {
      // rows = lines; 2 columns per lane cover ncol <= 64
      for (int tl0 = warp; tl0 < t.ntl; tl0 += U * nw) {
        float v[U][2];
#pragma unroll
        for (int u = 0; u < U; ++u) {
          const int tl = tl0 + u * nw;
          const int line = t.tl0 + tl;
          const bool lok = tl < t.ntl && line >= 0 && line < a.L;
          const char* rowp = base + (size_t)(lok ? line : 0) * a.W * (F32 ? 4 : 2);
#pragma unroll
          for (int k = 0; k < 2; ++k) {
            const int off = t.off0 + lane + 32 * k;
            const bool ok = lok && lane + 32 * k < ncol && off >= 0 && off < a.D;
            v[u][k] = ok ? ld_plane<F32>(rowp, off) : 0.f;
          }
        }
#pragma unroll
        for (int u = 0; u < U; ++u) {
          const int tl = tl0 + u * nw;
          if (tl < t.ntl) {
#pragma unroll
            for (int k = 0; k < 2; ++k)
              if (lane + 32 * k < ncol) dplane[tl * t.pitch + lane + 32 * k] = v[u][k];
          }
        }
      }
    } else {
      // rows of the image = offsets; lanes along the lines
      for (int c0 = warp; c0 < ncol; c0 += U * nw) {
        for (int tb = 0; tb < t.ntl; tb += 32) {
          const int tl = tb + lane;
          const int line = t.tl0 + tl;
          const bool lok = tl < t.ntl && line >= 0 && line < a.L;
          float v[U];
#pragma unroll
          for (int u = 0; u < U; ++u) {
            const int col = c0 + u * nw;
            const int off = t.off0 + col;
            const bool ok = lok && col < ncol && off >= 0 && off < a.D;
            const char* rowp = base + (size_t)(ok ? off : 0) * a.W * (F32 ? 4 : 2);
            v[u] = ok ? ld_plane<F32>(rowp, line) : 0.f;
          }
#pragma unroll
          for (int u = 0; u < U; ++u) {
            const int col = c0 + u * nw;
            if (col < ncol && tl < t.ntl) dplane[tl * t.pitch + col] = v[u];
          }
        }
      }
    }
  }
}

// FP32 tiles: every element is an asynchronous 4-byte global->shared copy
// (cp.async; zero-filled outside the image), all of a thread's copies in
// flight at once.  The caller waits with cp_async_wait_all + __syncthreads.
__device__ __forceinline__ void cp_async4(float* dst, const float* src, bool ok) {
  const unsigned d = static_cast<unsigned>(__cvta_generic_to_shared(dst));
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;" ::"r"(d), "l"(src), "r"(ok ? 4 : 0) : "memory");
}
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;" ::: "memory"); }

template <int CC, int NCOL>
__device__ __noinline__ void stage_tile_async(const PassArgs& a, const Tile& t, int p0, int p1) {
  const int tid = threadIdx.y * blockDim.x + threadIdx.x;
  const int nthreads = blockDim.x * blockDim.y;
  const long long W = a.W;
#pragma unroll 1
  for (int pl = p0; pl < p1; ++pl) {
    const float* base = reinterpret_cast<const float*>(plane_base<CC>(a, pl, 4));
    float* dplane = t.p + pl * t.pstride;
    if (a.dir == 0) {
      // flat over (line, offset); NCOL is a compile-time constant
      const int nel = t.ntl * NCOL;
      for (int idx = tid; idx < nel; idx += nthreads) {
        const int tl = idx / NCOL;
        const int col = idx - tl * NCOL;
        const int line = t.tl0 + tl, off = t.off0 + col;
        const bool ok = line >= 0 && line < a.L && off >= 0 && off < a.D;
        const float* src = ok ? base + (line * W + off) : base;
        cp_async4(dplane + tl * t.pitch + col, src, ok);
      }
    } else {
      // 8 lines x 4 offsets per warp instruction: lanes along the lines are
      // contiguous in memory (one 32-byte sector per offset)
      constexpr int NCB = (NCOL + 3) / 4;
      const int nlb = (t.ntl + 7) / 8;
      const int ls = threadIdx.x & 7, cs = threadIdx.x >> 3;
      for (int tile = threadIdx.y; tile < nlb * NCB; tile += blockDim.y) {
        const int lb = tile / NCB;
        const int cb = tile - lb * NCB;
        const int tl = lb * 8 + ls, col = cb * 4 + cs;
        const int line = t.tl0 + tl, off = t.off0 + col;
        const bool in_tile = tl < t.ntl && col < NCOL;
        const bool ok = in_tile && line >= 0 && line < a.L && off >= 0 && off < a.D;
        const float* src = ok ? base + (off * W + line) : base;
        if (in_tile) cp_async4(dplane + tl * t.pitch + col, src, ok);
      }
    }
  }
}

// 16-byte asynchronous global->shared copy; bytes past src_bytes are zero.
__device__ __forceinline__ void cp_async16(float* dst, const float* src, int src_bytes) {
  const unsigned d = static_cast<unsigned>(__cvta_generic_to_shared(dst));
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(d), "l"(src), "r"(src_bytes) : "memory");
}

// Four consecutive BF16 values (8-byte aligned) widened to FP32.
__device__ __forceinline__ float4 ld_bf16x4(const unsigned short* p) {
  const uint2 raw = __ldg(reinterpret_cast<const uint2*>(p));
  return make_float4(__uint_as_float(raw.x << 16), __uint_as_float(raw.x & 0xffff0000u),
                     __uint_as_float(raw.y << 16), __uint_as_float(raw.y & 0xffff0000u));
}
__device__ __forceinline__ float ld_bf16(const unsigned short* p) {
  return __uint_as_float(static_cast<unsigned>(__ldg(p)) << 16);
}

// One tile plane with 4-element transfers (image rows 16-byte aligned for
// FP32, 8-byte aligned for BF16).  Column direction: quads along the
// offsets into quads of the tile (its column origin is the quad boundary,
// cs = off0 mod 4): FP32 as asynchronous 16-byte copies, BF16 as 8-byte
// loads widened in registers (U in flight per thread); only quads that
// start left of the image use scalar loads.  Row direction: each warp
// instruction loads 8 quads (32 consecutive lines) of 4 image rows, U loads
// in flight per thread, scattered into the transposed tile.
template <bool F32, int NCOL>
__device__ __forceinline__ void stage_plane_vec(const PassArgs& a, const Tile& t, const void* vbase, float* dplane) {
  const int tid = threadIdx.y * blockDim.x + threadIdx.x;
  const int nthreads = blockDim.x * blockDim.y;
  const long long W = a.W;
  const float* fb = reinterpret_cast<const float*>(vbase);
  const unsigned short* hb = reinterpret_cast<const unsigned short*>(vbase);
  constexpr int U = 4;
  if (a.dir == 0) {
    constexpr int PQ = (NCOL + 3 + 3) / 4;
    const int x0 = t.off0 - t.cs;
    const int nq = t.ntl * PQ;
    if constexpr (F32) {
      for (int idx = tid; idx < nq; idx += nthreads) {
        const int tl = idx / PQ;
        const int q = idx - tl * PQ;
        const int line = t.tl0 + tl;
        const int x = x0 + 4 * q;
        float* dst = dplane + tl * t.pitch + 4 * q;
        const bool lok = line >= 0 && line < a.L;
        if (x >= 0) {
          const int valid = lok ? max(0, min(4, a.D - x)) : 0;
          cp_async16(dst, valid > 0 ? fb + (line * W + x) : fb, 4 * valid);
        } else {
          const float* rp = fb + (lok ? line : 0) * W;
#pragma unroll
          for (int i = 0; i < 4; ++i) dst[i] = (lok && x + i >= 0 && x + i < a.D) ? __ldg(rp + x + i) : 0.f;
        }
      }
    } else {
      for (int i0 = tid; i0 < nq; i0 += U * nthreads) {
        float4 v[U];
#pragma unroll
        for (int u = 0; u < U; ++u) {
          const int idx = i0 + u * nthreads;
          const int tl = idx / PQ;
          const int q = idx - tl * PQ;
          const int line = t.tl0 + tl;
          const int x = x0 + 4 * q;
          v[u] = make_float4(0.f, 0.f, 0.f, 0.f);
          if (idx < nq && line >= 0 && line < a.L) {
            const unsigned short* rp = hb + line * W;
            if (x >= 0 && x + 3 < a.D) {
              v[u] = ld_bf16x4(rp + x);
            } else {
              if (x >= 0 && x < a.D) v[u].x = ld_bf16(rp + x);
              if (x + 1 >= 0 && x + 1 < a.D) v[u].y = ld_bf16(rp + x + 1);
              if (x + 2 >= 0 && x + 2 < a.D) v[u].z = ld_bf16(rp + x + 2);
              if (x + 3 >= 0 && x + 3 < a.D) v[u].w = ld_bf16(rp + x + 3);
            }
          }
        }
#pragma unroll
        for (int u = 0; u < U; ++u) {
          const int idx = i0 + u * nthreads;
          if (idx >= nq) continue;
          const int tl = idx / PQ;
          const int q = idx - tl * PQ;
          *reinterpret_cast<float4*>(dplane + tl * t.pitch + 4 * q) = v[u];
        }
      }
    }
  } else {
    constexpr int NCB = (NCOL + 3) / 4;
    const int x0 = t.tl0 & ~3;                 // first quad's line
    const int nql = (t.tl0 + t.ntl - x0 + 3) / 4;
    const int nqb = (nql + 7) / 8;
    const int qs = threadIdx.x & 7, csub = threadIdx.x >> 3;
    const int ntile = nqb * NCB;
    for (int tb = threadIdx.y; tb < ntile; tb += U * blockDim.y) {
      float4 v[U];
#pragma unroll
      for (int u = 0; u < U; ++u) {
        const int tile = tb + u * blockDim.y;
        const int qb = tile / NCB;
        const int cb = tile - qb * NCB;
        const int q = qb * 8 + qs, col = cb * 4 + csub;
        const int off = t.off0 + col;
        const int x = x0 + 4 * q;
        v[u] = make_float4(0.f, 0.f, 0.f, 0.f);
        if (tile < ntile && q < nql && col < NCOL && off >= 0 && off < a.D) {
          if constexpr (F32) {
            const float* rp = fb + off * W;
            if (x >= 0 && x + 3 < a.L) {
              v[u] = __ldg(reinterpret_cast<const float4*>(rp + x));
            } else {
              if (x >= 0 && x < a.L) v[u].x = __ldg(rp + x);
              if (x + 1 >= 0 && x + 1 < a.L) v[u].y = __ldg(rp + x + 1);
              if (x + 2 >= 0 && x + 2 < a.L) v[u].z = __ldg(rp + x + 2);
              if (x + 3 >= 0 && x + 3 < a.L) v[u].w = __ldg(rp + x + 3);
            }
          } else {
            const unsigned short* rp = hb + off * W;
            if (x >= 0 && x + 3 < a.L) {
              v[u] = ld_bf16x4(rp + x);
            } else {
              if (x >= 0 && x < a.L) v[u].x = ld_bf16(rp + x);
              if (x + 1 >= 0 && x + 1 < a.L) v[u].y = ld_bf16(rp + x + 1);
              if (x + 2 >= 0 && x + 2 < a.L) v[u].z = ld_bf16(rp + x + 2);
              if (x + 3 >= 0 && x + 3 < a.L) v[u].w = ld_bf16(rp + x + 3);
            }
          }
        }
      }
#pragma unroll
      for (int u = 0; u < U; ++u) {
        const int tile = tb + u * blockDim.y;
        const int qb = tile / NCB;
        const int cb = tile - qb * NCB;
        const int q = qb * 8 + qs, col = cb * 4 + csub;
        if (tile >= ntile || q >= nql || col >= NCOL) continue;
        const int tlq = x0 + 4 * q - t.tl0;   // tile line of v.x
        const float e[4] = {v[u].x, v[u].y, v[u].z, v[u].w};
#pragma unroll
        for (int i = 0; i < 4; ++i)
          if (tlq + i >= 0 && tlq + i < t.ntl) dplane[(tlq + i) * t.pitch + col] = e[i];
      }
    }
  }
}

// Every plane with 4-element transfers, each in its own storage type.
template <int CC, int NCOL>
__device__ __forceinline__ void stage_tile_vec(const PassArgs& a, const Tile& t, int p0, int p1) {
#pragma unroll 1
  for (int pl = p0; pl < p1; ++pl) {
    const int dt = pl < CC ? a.in_dt : a.g_dt;
    const void* base = plane_base<CC>(a, pl, dt == DT_F32 ? 4 : 2);
    float* dplane = t.p + pl * t.pstride;
    if (dt == DT_F32)
      stage_plane_vec<true, NCOL>(a, t, base, dplane);
    else
      stage_plane_vec<false, NCOL>(a, t, base, dplane);
  }
}

// The 4-element staging applies when every plane's rows start on a 4-element
// boundary of its type (16 bytes for FP32, 8 for BF16).
__device__ __forceinline__ bool vec_staging(const PassArgs& a) {
  if (a.W & 3) return false;
  const uintptr_t m_in = a.in_dt == DT_F32 ? 15 : 7;
  const uintptr_t m_g = a.g_dt == DT_F32 ? 15 : 7;
  return ((reinterpret_cast<uintptr_t>(a.in) | reinterpret_cast<uintptr_t>(a.in2)) & m_in) == 0 &&
         (reinterpret_cast<uintptr_t>(a.g) & m_g) == 0;
}

// Dispatch: 4-element transfers when aligned; otherwise per-element copies
// (asynchronous for FP32, plain loads for BF16 or mixed types).  Planes
// [p0, p1): the estimate planes are 0 .. CC-1, the guidance plane CC.
template <int CC, int NCOL>
__device__ __forceinline__ void stage_tile(const PassArgs& a, const Tile& t, int p0 = 0, int p1 = CC + 1) {
  const int ncol = NCOL;
  if (vec_staging(a))
    stage_tile_vec<CC, NCOL>(a, t, p0, p1);
  else if (a.in_dt == DT_F32 && a.g_dt == DT_F32)
    stage_tile_async<CC, NCOL>(a, t, p0, p1);
  else if (a.in_dt == DT_BF16 && a.g_dt == DT_BF16)
    stage_tile_t<CC, false>(a, t, ncol, p0, p1);
  else
    stage_tile_mixed<CC>(a, t, ncol, p0, p1);
}

// Tiles of a runtime width (sliding step > 1): one warp per tile row (a
// line for the column direction, an across-offset for the row direction),
// lanes along the image's contiguous axis; plain loads, zero outside the
// image.  Planes [p0, p1).
template <int CC>
__device__ __noinline__ void stage_tile_rt(const PassArgs& a, const Tile& t, int p0, int p1) {
#pragma unroll 1
  for (int pl = p0; pl < p1; ++pl) {
    const int dt = pl < CC ? a.in_dt : a.g_dt;
    const void* base = plane_base<CC>(a, pl, dt == DT_F32 ? 4 : 2);
    float* dplane = t.p + pl * t.pstride;
    if (a.dir == 0) {
      for (int tl = threadIdx.y; tl < t.ntl; tl += blockDim.y) {
        const int line = t.tl0 + tl;
        const bool lok = line >= 0 && line < a.L;
        for (int col = threadIdx.x; col < t.ncol; col += 32) {
          const int off = t.off0 + col;
          dplane[tl * t.pitch + col] =
              (lok && off >= 0 && off < a.D) ? ld_px(base, (long long)line * a.W + off, dt) : 0.f;
        }
      }
    } else {
      for (int col = threadIdx.y; col < t.ncol; col += blockDim.y) {
        const int off = t.off0 + col;
        const bool ook = off >= 0 && off < a.D;
        for (int tl = threadIdx.x; tl < t.ntl; tl += 32) {
          const int line = t.tl0 + tl;
          dplane[tl * t.pitch + col] =
              (ook && line >= 0 && line < a.L) ? ld_px(base, (long long)off * a.W + line, dt) : 0.f;
        }
      }
    }
  }
}

// Column (relative to the lane's strip start) of entry j of a line.
template <int R, bool ODD>
__device__ __forceinline__ constexpr int ecol(int j) { return ODD ? 2 * R - j : j; }

// Entries of a line handled per loop trip: all of them (static indices) for
// r <= 3, one (a rolled loop, smaller code) for larger r.
template <int R>
struct LineUnroll {
  static constexpr int value = R <= 3 ? 2 * R + 1 : 1;
};

// lambda * w(p, p+t), t = 1..R, for entry j of a line (Eq. 2).  gr / gnr:
// guidance rows of this line and the next (lane-relative); `end_ok`: the next
// line exists (pairs that cross into it are inside the vector).  GCM: a.gc
// guidance planes gs floats apart (the norm of the difference vector).
template <int R, bool ODD, bool GCM = false>
__device__ __forceinline__ void forward_weights(const PassArgs& a, const float* gr, const float* gnr, int j,
                                                bool end_ok, float (&wf)[R], int gs = 0) {
  constexpr int n = 2 * R + 1;
  const float g0 = gr[ecol<R, ODD>(j)];
#pragma unroll
  for (int t = 1; t <= R; ++t) {
    const int jt = j + t;
    float w;
    if constexpr (GCM) {
      const float* gp = gr + ecol<R, ODD>(j);
      const float* gq = jt < n ? gr + ecol<R, ODD>(jt) : gnr + ecol<R, !ODD>(jt - n);
      float d2 = 0.f;
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        if (k < a.gc) {
          const float d = gp[k * gs] - gq[k * gs];
          d2 += d * d;
        }
      }
      w = a.sp[j * R + t - 1] * range_factor_sq(a, d2);
    } else {
      const float gq = jt < n ? gr[ecol<R, ODD>(jt)] : gnr[ecol<R, !ODD>(jt - n)];
      w = a.sp[j * R + t - 1] * range_factor(a, g0 - gq);
    }
    wf[t - 1] = (jt < n || end_ok) ? w : 0.f;
  }
}

// lambda * w(p, p+t) of the entries j = J0 .. J1-1 of a line (t = 1..r), one
// branch on the weight form per call instead of one per pair.
template <int R, bool ODD, bool GCM = false, int J0 = 0, int J1 = 2 * R + 1>
__device__ __forceinline__ void line_weights(const PassArgs& a, const float* gr, const float* gnr, bool end_ok,
                                             float (&wl)[2 * R + 1][R], int gs = 0) {
  constexpr int n = 2 * R + 1;
  constexpr int GE = J1 + R;   // guidance values g[J0 .. GE-1] are read
  float g[n + R];   // guidance of the line's entries, then of the next line's first r
  if constexpr (GCM) {
    // squared norms of the guidance differences, plane by plane
    float d2[n][R];
#pragma unroll
    for (int j = J0; j < J1; ++j)
#pragma unroll
      for (int t = 0; t < R; ++t) d2[j][t] = 0.f;
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      if (k < a.gc) {
#pragma unroll
        for (int j = J0; j < n && j < GE; ++j) g[j] = gr[k * gs + ecol<R, ODD>(j)];
#pragma unroll
        for (int m = 0; m < R && n + m < GE; ++m) g[n + m] = gnr[k * gs + ecol<R, !ODD>(m)];
#pragma unroll
        for (int j = J0; j < J1; ++j)
#pragma unroll
          for (int t = 1; t <= R; ++t) {
            const float d = g[j] - g[j + t];
            d2[j][t - 1] += d * d;
          }
      }
    }
#pragma unroll
    for (int j = J0; j < J1; ++j)
#pragma unroll
      for (int t = 1; t <= R; ++t) wl[j][t - 1] = a.sp[j * R + t - 1] * range_factor_sq(a, d2[j][t - 1]);
  } else {
#pragma unroll
    for (int j = J0; j < n && j < GE; ++j) g[j] = gr[ecol<R, ODD>(j)];
#pragma unroll
    for (int k = 0; k < R && n + k < GE; ++k) g[n + k] = gnr[ecol<R, !ODD>(k)];
    if (a.weight == 0) {
#pragma unroll
      for (int j = J0; j < J1; ++j)
#pragma unroll
        for (int t = 1; t <= R; ++t) {
          const float d = g[j] - g[j + t];
          wl[j][t - 1] = a.sp[j * R + t - 1] * fast_ex2(d * d * a.range_k);
        }
    } else {
#pragma unroll
      for (int j = J0; j < J1; ++j)
#pragma unroll
        for (int t = 1; t <= R; ++t)
          wl[j][t - 1] = a.sp[j * R + t - 1] / (powf(fabsf(g[j] - g[j + t]), a.range_k) + a.eps);
    }
  }
  if (!end_ok) {
#pragma unroll
    for (int j = J0; j < J1; ++j)
#pragma unroll
      for (int t = 1; t <= R; ++t)
        if (j + t >= n) wl[j][t - 1] = 0.f;
  }
}

template <int R>
__device__ __forceinline__ void push_weights(float (&wh)[R][R], const float (&wf)[R]) {
#pragma unroll
  for (int u = R - 1; u > 0; --u)
#pragma unroll
    for (int t = 0; t < R; ++t) wh[u][t] = wh[u - 1][t];
#pragma unroll
  for (int t = 0; t < R; ++t) wh[0][t] = wf[t];
}

// One LDL^T row for entry p, with a subtraction-free pivot.
//
// A_s = I + lambda L has unit row sums (Eq. 4), so row p of every Schur
// complement on the way has a non-negative "margin" (its row sum: 1 plus
// what the eliminated entries passed on) and non-positive off-diagonals;
// its diagonal is the margin plus the magnitudes of the off-diagonals.
// Forming the pivot that way, as a sum of non-negative terms, instead of as
// 1 + lambda sum w - sum (fill), keeps the identity's 1 when lambda w is
// ~1e7 (the frac weights' settings of Sec. 3), where the subtraction loses
// it to FP32 rounding.  This is Grassmann, Taksar and Heyman's elimination
// for M-matrices applied to the band.
//
// In:  wh[u-1][t-1] = lambda w(p-u, p-u+t); Lw[u-1][v-1] = L[p-u, p-u-v];
//      Dw[u-1] = 1/D[p-u]; mw[u-1] = margin of p-u; Uw[u-1][t-1] =
//      |S[p-u, p-u+t]| (the couplings of p-u to later entries when it was
//      pivoted; read for t < r); wf[t-1] = lambda w(p, p+t); mbase = 1 plus
//      the couplings of p to entries outside the factored matrix that are
//      counted as margin; bit t-1 of `keep` clear: entry p+t lies outside
//      the factored matrix (its coupling is part of mbase instead).
//      Entries p-t with t > lim are outside the interior.
// Out: Lrow[t-1] = L[p, p-t], m = margin of p, Up[t-1] = |S[p, p+t]|;
//      returns m + sum_t Up[t-1] (the pivot less any couplings the caller
//      tracks separately).
template <int R>
__device__ __forceinline__ float gth_row(float mbase, const float (&wf)[R], const float (&wh)[R][R],
                                         const float (&Lw)[R][R], const float (&Dw)[R], const float (&mw)[R],
                                         const float (&Uw)[R][R], int lim, unsigned keep, float (&Lrow)[R],
                                         float& m, float (&Up)[R]) {
  float Wt[R];
#pragma unroll
  for (int t = R; t >= 1; --t) {
    float acc = -wh[t - 1][t - 1];
#pragma unroll
    for (int v = t + 1; v <= R; ++v) acc -= Wt[v - 1] * Lw[t - 1][v - t - 1];
    const bool in = t <= lim;
    Wt[t - 1] = in ? acc : 0.f;
    Lrow[t - 1] = in ? acc * Dw[t - 1] : 0.f;
  }
  m = mbase;
#pragma unroll
  for (int t = 0; t < R; ++t) m -= Lrow[t] * mw[t];
  float D = m;
#pragma unroll
  for (int t = 1; t <= R; ++t) {
    float u = wf[t - 1];
    // at distance r no earlier entry couples to both: the coupling is still
    // A's own, lambda w(p-v, p+t) (wh), so Uw is read for shorter ones only
#pragma unroll
    for (int v = 1; v <= R - t; ++v) u -= Lrow[v - 1] * (t + v == R ? wh[v - 1][R - 1] : Uw[v - 1][t + v - 1]);
    Up[t - 1] = ((keep >> (t - 1)) & 1u) ? u : 0.f;
    D += Up[t - 1];
  }
  return D;
}

// Shifts the margin and upper-coupling windows by one entry.
template <int R>
__device__ __forceinline__ void push_gth(float (&mw)[R], float (&Uw)[R][R], float mp, const float (&Up)[R]) {
#pragma unroll
  for (int u = R - 1; u > 0; --u) {
    mw[u] = mw[u - 1];
#pragma unroll
    for (int t = 0; t < R; ++t) Uw[u][t] = Uw[u - 1][t];
  }
  mw[0] = mp;
#pragma unroll
  for (int t = 0; t < R; ++t) Uw[0][t] = Up[t];
}

template <int R>
__device__ __forceinline__ void push_factor(float (&Lw)[R][R], float (&Dw)[R], const float (&Lrow)[R], float dinv) {
#pragma unroll
  for (int u = R - 1; u > 0; --u) {
#pragma unroll
    for (int v = 0; v < R; ++v) Lw[u][v] = Lw[u - 1][v];
    Dw[u] = Dw[u - 1];
  }
#pragma unroll
  for (int v = 0; v < R; ++v) Lw[0][v] = Lrow[v];
  Dw[0] = dinv;
}

template <int R, int K>
__device__ __forceinline__ void push_vec(float (&w)[R][K], const float (&x)[K]) {
#pragma unroll
  for (int u = R - 1; u > 0; --u)
#pragma unroll
    for (int i = 0; i < K; ++i) w[u][i] = w[u - 1][i];
#pragma unroll
  for (int i = 0; i < K; ++i) w[0][i] = x[i];
}

// y -= sum_t L[p, p-t] win[t-1]  (forward substitution, K columns)
template <int R, int K>
__device__ __forceinline__ void fwd_subst(const float (&Lrow)[R], const float (&win)[R][K], float (&y)[K]) {
#pragma unroll
  for (int t = 0; t < R; ++t)
#pragma unroll
    for (int i = 0; i < K; ++i) y[i] -= Lrow[t] * win[t][i];
}

// Runs body(odd, first, last, line) over the lines [line0, line1): the
// parity and the last-line role are compile-time constants, the first-line
// role a runtime flag (keeps the kernels' code small).
template <typename Body>
__device__ __forceinline__ void for_lines(int line0, int line1, Body&& body) {
  auto dispatch = [&](bool first, auto last, int line) {
    if (line & 1)
      body(std::true_type{}, first, last, line);
    else
      body(std::false_type{}, first, last, line);
  };
  for (int line = line0; line < line1 - 1; ++line) dispatch(line == line0, std::false_type{}, line);
  dispatch(line1 - 1 == line0, std::true_type{}, line1 - 1);
}

// Backward order: body(odd, last, line) over lines line1-1 down to line0.
template <typename Body>
__device__ __forceinline__ void for_lines_rev(int line0, int line1, Body&& body) {
  auto dispatch = [&](auto last, int line) {
    if (line & 1)
      body(std::true_type{}, last, line);
    else
      body(std::false_type{}, last, line);
  };
  dispatch(std::true_type{}, line1 - 1);
  for (int line = line1 - 2; line >= line0; --line) dispatch(std::false_type{}, line);
}

// ---------------------------------------------------------------------------
struct Chunk {
  int line0, line1;     // lines [line0, line1)
  int b, e, end;        // interior [b, e), chunk entries [b, end)
  bool top, bot;        // has a separator above / below
};

template <int R>
__device__ __forceinline__ Chunk make_chunk(const PassArgs& a, int c) {
  constexpr int n = 2 * R + 1;
  Chunk ch;
  ch.line0 = c * a.h;
  ch.line1 = min(ch.line0 + a.h, a.L);
  ch.b = ch.line0 * n;
  ch.end = ch.line1 * n;
  ch.top = c > 0;
  ch.bot = c < a.P - 1;
  ch.e = ch.bot ? ch.end - R : ch.end;
  return ch;
}

// Weights of the line above a chunk (its top separator's line) into wh.
template <int R, int CC, bool GCM = false>
__device__ __forceinline__ void prologue_weights(const PassArgs& a, const Tile& t, int lane, int line,
                                                 float (&wh)[R][R]) {
  constexpr int n = 2 * R + 1;
  auto pro = [&](auto odd) {
    constexpr bool ODD = decltype(odd)::value;
    const float* gr = t.row(CC, line) + lane;
    const float* gnr = t.row(CC, line + 1) + lane;
    float wf[R];
#pragma unroll LineUnroll<R>::value
    for (int j = 0; j < n; ++j) {
      forward_weights<R, ODD, GCM>(a, gr, gnr, j, true, wf, t.pstride);
      push_weights<R>(wh, wf);
    }
  };
  if (line & 1) pro(std::true_type{}); else pro(std::false_type{});
}

// Strided access to the field block of one lane: base[field * stride].
struct Strided {
  float* base;
  int stride;
  __device__ __forceinline__ float& operator[](int field) const { return base[field * stride]; }
};
struct StridedG {
  float* base;
  long long stride;
  __device__ __forceinline__ float& operator[](int field) const { return base[field * stride]; }
};

// ---------------------------------------------------------------------------
// Forward sweep of one chunk for the summary: eliminates the interior and
// writes its 2-port to `out`.
// Factor store of one subsystem (band of 32 subsystems, lane in the band):
// fac[band][e][2r + CC fields x 32 lanes, grouped as in st_fields] with
// e = line * (2r+1) + j over the L lines; psi[band][c][k][i][32].  Inside a
// band every offset is a compile-time multiple of 32 floats from the line's
// base.
// With a.nslot > 0 the store is a ring of a.nslot band slots (the
// queue-scheduled pass reuses a slot once every reader of its band is done).
__device__ __forceinline__ size_t fac_slot(const PassArgs& a, int sys) {
  const int band = sys >> 5;
  return (size_t)(a.nslot > 0 ? band % a.nslot : band);
}
template <int R, int CC>
__device__ __forceinline__ float* fac_lane(const PassArgs& a, int sys) {
  const size_t band = (size_t)a.L * (2 * R + 1) * (2 * R + CC) * 32;
  return a.fac + fac_slot(a, sys) * band + (sys & 31);
}
// Factor-store entry of a band: NF fields x 32 lanes, the fields in groups
// of four, then a pair, then a single one (NF = 4k + 2a + b); in the block
// of group [f, f + w) lane l's w fields are one w x 4-byte word at
// entry + f * 32 + w * l.  So a lane stores and loads an entry with a few
// wide accesses, and a warp's lanes of one band touch contiguous memory.
template <int NF>
__device__ __forceinline__ void st_fields(float* eb, int l, const float (&v)[NF]) {
  int f = 0;
#pragma unroll
  for (; f + 4 <= NF; f += 4)
    *reinterpret_cast<float4*>(eb + f * 32 + 4 * l) = make_float4(v[f], v[f + 1], v[f + 2], v[f + 3]);
  if constexpr (NF % 4 >= 2) {
    *reinterpret_cast<float2*>(eb + (NF / 4 * 4) * 32 + 2 * l) = make_float2(v[NF / 4 * 4], v[NF / 4 * 4 + 1]);
  }
  if constexpr (NF % 2 == 1) eb[(NF - 1) * 32 + l] = v[NF - 1];
}
template <int NF>
__device__ __forceinline__ void ld_fields(const float* eb, int l, float (&v)[NF]) {
#pragma unroll
  for (int f = 0; f + 4 <= NF; f += 4) {
    const float4 q = __ldcg(reinterpret_cast<const float4*>(eb + f * 32 + 4 * l));
    v[f] = q.x;
    v[f + 1] = q.y;
    v[f + 2] = q.z;
    v[f + 3] = q.w;
  }
  if constexpr (NF % 4 >= 2) {
    const float2 q = __ldcg(reinterpret_cast<const float2*>(eb + (NF / 4 * 4) * 32 + 2 * l));
    v[NF / 4 * 4] = q.x;
    v[NF / 4 * 4 + 1] = q.y;
  }
  if constexpr (NF % 2 == 1) v[NF - 1] = __ldcg(eb + (NF - 1) * 32 + l);
}

// Per-entry buffers of the refinement (rhs, xent): [band][e][CC][32].
template <int R, int CC>
__device__ __forceinline__ float* ent_lane(const PassArgs& a, float* buf, int sys) {
  const size_t band = (size_t)a.L * (2 * R + 1) * CC * 32;
  return buf + (size_t)(sys >> 5) * band + (sys & 31);
}
template <int R>
__device__ __forceinline__ float* psi_lane(const PassArgs& a, int sys) {
  const size_t band = (size_t)a.P * R * R * 32;
  return a.psi + fac_slot(a, sys) * band + (sys & 31);
}
// With a.fac set it also keeps, per interior entry, the factor row, z0 and
// Phi for k_backsub, and psi for the last r interior entries.
template <int R, int CC, bool KEEP, bool RHSB = false, bool GCM = false, typename Out>
__device__ __forceinline__ void chunk_summary(const PassArgs& a, const Tile& t, int col, int sys, int c,
                                              Out&& out) {
  const int lane = col;   // tile column of the lane's strip
  constexpr int n = 2 * R + 1;
  constexpr int NFAC = 2 * R + CC;
  constexpr bool LW = LineUnroll<R>::value > 1;   // a line's weights computed together
  using F = Fields<R, CC>;
  const Chunk q = make_chunk<R>(a, c);
  const int pstride = t.pstride;
  // the band's factor store and the lane in it (st_fields layout)
  float* const fac = KEEP ? fac_lane<R, CC>(a, sys) - (sys & 31) : nullptr;
  // RHSB: the right-hand side of every entry comes from a.rhs (the
  // refinement's residual) instead of the estimate planes of the tile
  const float* const rhs = RHSB ? ent_lane<R, CC>(a, a.rhs, sys) : nullptr;

  float wh[R][R] = {};
  float Lw[R][R] = {};
  float Dw[R] = {};
  float yw[R][CC] = {};
  float YTw[R][R] = {};
  float YBw[R][R] = {};
  float KTT[R][R] = {}, KTB[R][R] = {}, KBB[R][R] = {};
  float HT[R][CC] = {}, HB[R][CC] = {};
  float DS[R][R] = {};
  float FS[R][CC] = {};
  float mw[R] = {};        // margins of the last R interior entries
  float Uw[R][R] = {};     // their couplings to later entries
  float tauT[R] = {}, tauB[R] = {};   // margin passed to the separators

  if (q.top) prologue_weights<R, CC, GCM>(a, t, lane, q.line0 - 1, wh);

  for_lines(q.line0, q.line1, [&](auto odd, const bool FIRST, auto last, int line) {
    constexpr bool ODD = decltype(odd)::value;
    constexpr bool LAST = decltype(last)::value;
    const float* gr = t.row(CC, line) + lane;
    const float* gnr = t.row(CC, line + 1) + lane;
    const float* fr = t.row(0, line) + lane;
    const bool end_ok = line + 1 < a.L;
    // a line's weights: all at once for r <= 2; for r = 3 in two halves
    // (fewer registers live)
    constexpr int JH = R == 3 ? R + 1 : n;
    float wl[LW ? n : 1][R];
    if constexpr (LW) line_weights<R, ODD, GCM, 0, JH>(a, gr, gnr, end_ok, wl, pstride);
    (void)wl;
#pragma unroll LineUnroll<R>::value
    for (int j = 0; j < n; ++j) {
      if constexpr (LW && JH < n) {
        if (j == JH) line_weights<R, ODD, GCM, JH, n>(a, gr, gnr, end_ok, wl, pstride);
      }
      float wf[R];
      if constexpr (LW) {
#pragma unroll
        for (int tt = 0; tt < R; ++tt) wf[tt] = wl[LW ? j : 0][tt];
      } else {
        forward_weights<R, ODD, GCM>(a, gr, gnr, j, end_ok, wf, pstride);
      }
      float fj[CC];
#pragma unroll
      for (int ch = 0; ch < CC; ++ch) {
        if constexpr (RHSB)
          fj[ch] = __ldcg(rhs + ((line * n + j) * CC + ch) * 32);
        else
          fj[ch] = fr[ch * pstride + ecol<R, ODD>(j)];
      }
      const bool sep = LAST && q.bot && j >= n - R;
      if (!sep) {
        const int lim = FIRST ? min(j, R) : R;
        float Lrow[R], mp, Up[R];
        // the couplings to the bottom separator count among the later
        // entries', those to the top separator are -YT (added below)
        float piv = gth_row<R>(1.f, wf, wh, Lw, Dw, mw, Uw, lim, ~0u, Lrow, mp, Up);
        float y[CC];
#pragma unroll
        for (int ch = 0; ch < CC; ++ch) y[ch] = fj[ch];
        fwd_subst<R, CC>(Lrow, yw, y);
        float YT[R];
#pragma unroll
        for (int i = 0; i < R; ++i) YT[i] = 0.f;
        // Top-separator terms, tracked in every chunk: without a separator
        // above (chunk 0) the prologue weights wh are zero, so YT, KTT and
        // HT stay zero and no branch is needed.
        // E_T[p][i] = A[p, b-R+i] = -lambda w(p-tt, p), tt = j + R - i
#pragma unroll
        for (int i = 0; i < R; ++i)
#pragma unroll
          for (int tt = 1; tt <= R; ++tt)
            if (tt == j + R - i) YT[i] = FIRST ? -wh[tt - 1][tt - 1] : 0.f;
        fwd_subst<R, R>(Lrow, YTw, YT);
#pragma unroll
        for (int i = 0; i < R; ++i) piv -= YT[i];
        const float dinv = fast_rcp(piv);
#pragma unroll
        for (int i = 0; i < R; ++i) {
          const float yd = YT[i] * dinv;
#pragma unroll
          for (int m = 0; m < R; ++m)
            if (m > i) KTT[i][m] += yd * YT[m];   // symmetric: the upper part
          tauT[i] -= yd * mp;
#pragma unroll
          for (int ch = 0; ch < CC; ++ch) HT[i][ch] += yd * y[ch];
        }
        if constexpr (KEEP) {
          float fv[NFAC];
#pragma unroll
          for (int tt = 0; tt < R; ++tt) fv[tt] = Lrow[tt];
#pragma unroll
          for (int ch = 0; ch < CC; ++ch) fv[R + ch] = y[ch] * dinv;
#pragma unroll
          for (int i = 0; i < R; ++i) fv[R + CC + i] = -YT[i] * dinv;
          st_fields<NFAC>(fac + ((line * n + j) * NFAC) * 32, sys & 31, fv);
        }
        float YB[R];
#pragma unroll
        for (int i = 0; i < R; ++i) YB[i] = 0.f;
        if (LAST) {
          if (q.bot && j >= n - 2 * R) {
            // E_B[p][i] = A[p, e+i] = -lambda w(p, p+tt), tt = (n - R - j) + i
#pragma unroll
            for (int i = 0; i < R; ++i)
#pragma unroll
              for (int tt = 1; tt <= R; ++tt)
                if (tt == n - R - j + i) YB[i] = -wf[tt - 1];
            fwd_subst<R, R>(Lrow, YBw, YB);
#pragma unroll
            for (int i = 0; i < R; ++i) {
              const float yd = YB[i] * dinv;
#pragma unroll
              for (int m = 0; m < R; ++m) {
                if (m > i) KBB[i][m] += yd * YB[m];
                KTB[m][i] += yd * YT[m];
              }
              tauB[i] -= yd * mp;
#pragma unroll
              for (int ch = 0; ch < CC; ++ch) HB[i][ch] += yd * y[ch];
            }
            if constexpr (KEEP) {
              float* pe = psi_lane<R>(a, sys) + ((c * R + (j - (n - 2 * R))) * R) * 32;
#pragma unroll
              for (int i = 0; i < R; ++i) pe[i * 32] = -YB[i] * dinv;
            }
          }
          push_vec<R, R>(YBw, YB);
        }
        push_factor<R>(Lw, Dw, Lrow, dinv);
        push_gth<R>(mw, Uw, mp, Up);
        push_vec<R, CC>(yw, y);
        push_vec<R, R>(YTw, YT);
      } else {
        // separator entry e + i: its own margin 1, the magnitudes of its
        // couplings inside S_c, f(S_c)
        const int isep = j - (n - R);
#pragma unroll
        for (int i = 0; i < R; ++i) {
          if (i == isep) {
            DS[i][i] = 1.f;
#pragma unroll
            for (int m = 0; m < i; ++m) {  // |A[e+i, e+m]| = lambda w(e+m, e+i)
              DS[i][m] = wh[i - m - 1][i - m - 1];
              DS[m][i] = DS[i][m];
            }
#pragma unroll
            for (int ch = 0; ch < CC; ++ch) FS[i][ch] = fj[ch];
          }
        }
      }
      push_weights<R>(wh, wf);
    }
  });

  // the 2-port in margin form (see Fields)
#pragma unroll
  for (int i = 0; i < R; ++i) {
#pragma unroll
    for (int m = 0; m < R; ++m) {
      out[F::KTT + i * R + m] = m == i ? tauT[i] : KTT[min(i, m)][max(i, m)];
      out[F::KTB + i * R + m] = KTB[i][m];
      out[F::DS + i * R + m] = m == i ? DS[i][i] + tauB[i] : DS[i][m] + KBB[min(i, m)][max(i, m)];
    }
#pragma unroll
    for (int ch = 0; ch < CC; ++ch) {
      out[F::HT + i * CC + ch] = -HT[i][ch];
      out[F::GS + i * CC + ch] = FS[i][ch] - HB[i][ch];
    }
  }
}

// Tensor-copy staging of a fixed-width column-direction tile (a.tma): thread
// (0, 0) issues one box per plane [p0, p1) into the tile -- the estimate
// planes through the 3D map tm_in, the guidance through tm_g -- starting at
// the 16-byte boundary x = off0 - cs and line tl0 (negative or past the image:
// zeros).  The boxes complete `bar`, whose expected bytes the caller set.
template <int CC>
__device__ __forceinline__ void tma_stage(const PassArgs& a, const Tile& t, int p0, int p1, unsigned long long* bar) {
  if (threadIdx.x != 0 || threadIdx.y != 0) return;
  const int x = t.off0 - t.cs, y = t.tl0;
  for (int pl = p0; pl < p1; ++pl) {
    float* dst = t.p + pl * t.pstride;
    if (pl < CC)
      tma_load_3d(dst, &a.tm_in, x, y, pl, bar);
    else
      tma_load_2d(dst, &a.tm_g, x, y, bar);
  }
}

// Bytes of the CC + 1 boxes of a tensor-copy tile.
__device__ __forceinline__ unsigned tma_tile_bytes(const Tile& t, int planes) {
  return (unsigned)(planes * t.ntl * t.pitch * sizeof(float));
}

// Tile geometry of a block of G chunks starting at chunk c0.
// ncol columns from off0; fixed: the 32 + 2r columns of step 1 (staged with
// 4-element transfers when aligned), otherwise the runtime-width staging.
__device__ __forceinline__ void group_tile(const PassArgs& a, int c0, int G, int off0, int ncol, bool fixed, float* p,
                                           Tile& t) {
  t.tl0 = c0 * a.h - 1;
  // with tensor-copy staging every block's tile has the box's G h + 2 lines
  // (lines past the image are filled with zeros by the copy)
  const bool tma = a.tma && a.dir == 0;
  t.ntl = tma ? G * a.h + 2 : min((c0 + G) * a.h, a.L) + 1 - t.tl0;
  t.off0 = off0;
  t.cs = (a.dir == 0 && (tma || (fixed && vec_staging(a)))) ? (off0 & 3) : 0;
  t.pitch = tile_pitch_n(ncol, a.dir);
  t.pstride = tile_pstride(t.ntl, t.pitch);
  t.ncol = ncol;
  t.p = p;
}

// Folds n consecutive 2-ports (Fields format; in(i) addresses element i's
// fields) into one by eliminating the n-1 separators between them, left to
// right.  Element 0 has a top port iff acc_top; element i has a bottom port
// iff has_bot(i).  Merge i (1 <= i < n) eliminates separator Y (element
// i-1's bottom = element i's top) from the rows of Y, X (the fold's top) and
// Z (element i's bottom) of the reduced system, entry by entry and without
// subtraction: Y's rows have margin DS_{i-1} + KTT_i on the diagonal slots,
// couplings |Y_a - Y_b| = the two off-diagonal parts summed, |Y - X| =
// KTB_{i-1}^T, |Y - Z| = KTB_i and right-hand side GS_{i-1} + HT_i; the
// pivot of Y_a is its margin plus its remaining couplings, and eliminating
// it passes c = coupling / pivot times its margin, couplings and right-hand
// side on to every row it couples to.  Merge i keeps, through mf(i), what
// the back-fill needs: LM (below the diagonal c of the later Y entries,
// on it 1 / pivot), U = |Y - X| / pivot, V = |Y - Z| / pivot and
// W = rhs_Y / pivot, each taken when its entry was pivoted.  out receives
// the folded 2-port.  Lane = subsystem.
template <int R, int CC, typename In, typename HasBot, typename Mf, typename Out>
__device__ __forceinline__ void fold_2ports(int n, bool acc_top, In&& in, HasBot&& has_bot, Mf&& mf, Out&& out) {
  using F = Fields<R, CC>;
  using MF = MFields<R, CC>;
  auto cs = in(0);
  // the fold so far: X (its top), B (its bottom, the next Y)
  float XX[R][R], XB[R][R], BB[R][R], bX[R][CC], bB[R][CC];
#pragma unroll
  for (int i = 0; i < R; ++i) {
#pragma unroll
    for (int m = 0; m < R; ++m) {
      XX[i][m] = cs[F::KTT + i * R + m];
      XB[i][m] = cs[F::KTB + i * R + m];
      BB[i][m] = cs[F::DS + i * R + m];
    }
#pragma unroll
    for (int ch = 0; ch < CC; ++ch) {
      bX[i][ch] = cs[F::HT + i * CC + ch];
      bB[i][ch] = cs[F::GS + i * CC + ch];
    }
  }
  // Element i's KTT, KTB and HT (the fields its merge needs first) are read
  // one merge ahead, its DS and GS (needed after the separator's pivots) at
  // the start of its merge; both before merge i writes its factors, which
  // may overwrite element i in place.  The loads leave the serial path.
  float pT[R][R], pK[R][R], pH[R][CC];
  auto load_early = [&](int i) {
    auto src = in(i);
#pragma unroll
    for (int y = 0; y < R; ++y) {
#pragma unroll
      for (int m = 0; m < R; ++m) {
        pT[y][m] = src[F::KTT + y * R + m];
        pK[y][m] = src[F::KTB + y * R + m];
      }
#pragma unroll
      for (int ch = 0; ch < CC; ++ch) pH[y][ch] = src[F::HT + y * CC + ch];
    }
  };
  if (n > 1) load_early(1);
  for (int i = 1; i < n; ++i) {
    const bool zb = has_bot(i);
    auto direct = in(i);
    float YY[R][R], YX[R][R], YZ[R][R], bY[R][CC], ZZ[R][R], bZ[R][CC], XZ[R][R];
#pragma unroll
    for (int y = 0; y < R; ++y) {
#pragma unroll
      for (int m = 0; m < R; ++m) {
        YY[y][m] = BB[y][m] + pT[y][m];
        YX[y][m] = acc_top ? XB[m][y] : 0.f;
        YZ[y][m] = zb ? pK[y][m] : 0.f;
        ZZ[y][m] = zb ? direct[F::DS + y * R + m] : 0.f;
        XZ[y][m] = 0.f;
      }
#pragma unroll
      for (int ch = 0; ch < CC; ++ch) {
        bY[y][ch] = bB[y][ch] + pH[y][ch];
        bZ[y][ch] = zb ? direct[F::GS + y * CC + ch] : 0.f;
      }
    }
    if (i + 1 < n) load_early(i + 1);
    auto md = mf(i);
#pragma unroll
    for (int y = 0; y < R; ++y) {
      float d = YY[y][y];
#pragma unroll
      for (int m = 0; m < R; ++m) {
        if (m > y) d += YY[y][m];
        d += YX[y][m] + YZ[y][m];
      }
      const float dinv = fast_rcp(d);
#pragma unroll
      for (int m = 0; m < R; ++m) {
        md[MF::LM + m * R + y] = m == y ? dinv : (m > y ? YY[y][m] * dinv : 0.f);
        md[MF::U + y * R + m] = YX[y][m] * dinv;
        md[MF::V + y * R + m] = YZ[y][m] * dinv;
      }
#pragma unroll
      for (int ch = 0; ch < CC; ++ch) md[MF::W + y * CC + ch] = bY[y][ch] * dinv;
      // pass Y_y's margin, couplings and right-hand side on
#pragma unroll
      for (int y2 = y + 1; y2 < R; ++y2) {
        const float c = YY[y][y2] * dinv;
        YY[y2][y2] += c * YY[y][y];
#pragma unroll
        for (int y3 = y + 1; y3 < R; ++y3)
          if (y3 != y2) YY[y2][y3] += c * YY[y][y3];
#pragma unroll
        for (int m = 0; m < R; ++m) {
          YX[y2][m] += c * YX[y][m];
          YZ[y2][m] += c * YZ[y][m];
        }
#pragma unroll
        for (int ch = 0; ch < CC; ++ch) bY[y2][ch] += c * bY[y][ch];
      }
      if (acc_top) {
#pragma unroll
        for (int x = 0; x < R; ++x) {
          const float c = YX[y][x] * dinv;
          XX[x][x] += c * YY[y][y];
#pragma unroll
          for (int x2 = 0; x2 < R; ++x2)
            if (x2 != x) XX[x][x2] += c * YX[y][x2];
#pragma unroll
          for (int z = 0; z < R; ++z) XZ[x][z] += c * YZ[y][z];
#pragma unroll
          for (int ch = 0; ch < CC; ++ch) bX[x][ch] += c * bY[y][ch];
        }
      }
      if (zb) {
#pragma unroll
        for (int z = 0; z < R; ++z) {
          const float c = YZ[y][z] * dinv;
          ZZ[z][z] += c * YY[y][y];
#pragma unroll
          for (int z2 = 0; z2 < R; ++z2)
            if (z2 != z) ZZ[z][z2] += c * YZ[y][z2];
#pragma unroll
          for (int ch = 0; ch < CC; ++ch) bZ[z][ch] += c * bY[y][ch];
        }
      }
    }
#pragma unroll
    for (int y = 0; y < R; ++y) {
#pragma unroll
      for (int m = 0; m < R; ++m) {
        XB[y][m] = XZ[y][m];
        BB[y][m] = ZZ[y][m];
      }
#pragma unroll
      for (int ch = 0; ch < CC; ++ch) bB[y][ch] = bZ[y][ch];
    }
  }
#pragma unroll
  for (int i = 0; i < R; ++i) {
#pragma unroll
    for (int m = 0; m < R; ++m) {
      out[F::KTT + i * R + m] = XX[i][m];
      out[F::KTB + i * R + m] = XB[i][m];
      out[F::DS + i * R + m] = BB[i][m];
    }
#pragma unroll
    for (int ch = 0; ch < CC; ++ch) {
      out[F::HT + i * CC + ch] = bX[i][ch];
      out[F::GS + i * CC + ch] = bB[i][ch];
    }
  }
}

// Back-fill of a fold: given the outer separators xX (above element 0, used
// iff acc_top) and xZ (below element n-1, used iff has_bot(n-1)), recovers
// the separators between the elements, bottom to top: put(i, x) receives the
// separator between elements i-1 and i,
//   x_Y[y] = W[y] + U[y] xX + V[y] xZ + sum_{m > y} LM[m][y] x_Y[m].
template <int R, int CC, typename HasBot, typename Mf, typename Put>
__device__ __forceinline__ void backfill_2ports(int n, bool acc_top, const float (&xX)[R][CC], float (&xZ)[R][CC],
                                                HasBot&& has_bot, Mf&& mf, Put&& put) {
  using MF = MFields<R, CC>;
  // small factor sets: merge i-1's are read while merge i is solved (put
  // may write memory the factors live in as far as the compiler knows)
  constexpr bool PREF = MF::N <= 40;
  constexpr int NB = PREF ? MF::N : 1;
  float nb[NB], cb[NB];
  auto load = [&](int i) {
    auto src = mf(i);
#pragma unroll
    for (int f = 0; f < NB; ++f) nb[f] = src[f];
  };
  if (PREF && n > 1) load(n - 1);
  for (int i = n - 1; i >= 1; --i) {
    const bool b_bot = has_bot(i);
    auto direct = mf(i);
    if constexpr (PREF) {
#pragma unroll
      for (int f = 0; f < NB; ++f) cb[f] = nb[f];
      if (i > 1) load(i - 1);
    }
    auto md = [&](int f) -> float { if constexpr (PREF) return cb[f < NB ? f : 0]; else return direct[f]; };
    float v[R][CC];
#pragma unroll
    for (int y = R - 1; y >= 0; --y) {
#pragma unroll
      for (int ch = 0; ch < CC; ++ch) {
        float acc = md(MF::W + y * CC + ch);
#pragma unroll
        for (int m = 0; m < R; ++m) {
          if (acc_top) acc += md(MF::U + y * R + m) * xX[m][ch];
          if (b_bot) acc += md(MF::V + y * R + m) * xZ[m][ch];
          if (m > y) acc += md(MF::LM + m * R + y) * v[m][ch];
        }
        v[y][ch] = acc;
      }
    }
    put(i, v);
#pragma unroll
    for (int y = 0; y < R; ++y)
#pragma unroll
      for (int ch = 0; ch < CC; ++ch) xZ[y][ch] = v[y][ch];
  }
}

// Merges the block's chunk 2-ports into the group 2-port as a binary tree:
// at level l warp w merges the node of chunks [2w 2^l, (2w+1) 2^l) with its
// right neighbour (in place, slot of the left node), so the serial depth is
// log2(G) merges instead of G-1.  Merge (l, w) keeps its factors in mdata
// slot G - (G >> l) + w of the group (lane = subsystem).  The group 2-port
// goes to summ.  Every thread of the block calls this (barriers).
template <int R, int CC>
__device__ __forceinline__ void merge_tree(const PassArgs& a, float* csum, int lane, int sys, int grp, int c0,
                                           int nch, int G, bool active) {
  using F = Fields<R, CC>;
  using MF = MFields<R, CC>;
  const long long ns = a.sstride;
  auto slot = [&](int i) { return Strided{csum + i * F::N * 32 + lane, 32}; };
  for (int span = 1; span < nch; span *= 2) {
    const int left = threadIdx.y * 2 * span;
    if (active && left + span < nch) {
      const int id = G - G / span + threadIdx.y;   // G - (G >> l) + w
      const int last = min(left + 2 * span, nch) - 1;
      fold_2ports<R, CC>(
          2, c0 + left > 0, [&](int i) { return slot(left + i * span); },
          [&](int) { return c0 + last < a.P - 1; },
          [&](int) { return StridedG{a.mdata + ((long long)(grp * (G - 1) + id) * MF::N) * ns + sys, ns}; },
          slot(left));
    }
    __syncthreads();
  }
  if (threadIdx.y == 0 && active) {
    const Strided g0 = slot(0);
    StridedG gs{a.summ + (long long)grp * F::N * ns + sys, ns};
#pragma unroll
    for (int f = 0; f < F::N; ++f) gs[f] = g0[f];
  }
}

// The separator system of NG consecutive 2-ports of one subsystem (the
// serial chain): fold_2ports over all of them (the first has no top port,
// the last no bottom port), merge g's factors written over 2-port g in
// place, then the back-fill.  `fld(g, field)` addresses the 2-ports; the
// value of the separator between 2-ports g and g+1 goes to xsep as group
// separator xidx(g) (skipped when !store).
template <int R, int CC, typename Fld, typename Xidx>
__device__ __forceinline__ void reduced_chain(const PassArgs& a, int sys, int NG, bool store, Fld&& fld,
                                              Xidx&& xidx) {
  using F = Fields<R, CC>;
  const long long ns = a.sstride;
  struct Slot {
    Fld* f;
    int g;
    __device__ __forceinline__ float& operator[](int field) const { return (*f)(g, field); }
  };
  auto slot = [&](int g) { return Slot{&fld, g}; };
  auto has_bot = [&](int g) { return g < NG - 1; };
  float sink[F::N];   // the folded 2-port of the whole subsystem has no ports
  fold_2ports<R, CC>(NG, false, slot, has_bot, slot, sink);
  float xX[R][CC] = {}, xZ[R][CC] = {};
  backfill_2ports<R, CC>(NG, false, xX, xZ, has_bot, slot, [&](int i, const float (&v)[R][CC]) {
    if (!store) return;
    const long long xb = (long long)xidx(i - 1) * R * CC;
#pragma unroll
    for (int y = 0; y < R; ++y)
#pragma unroll
      for (int ch = 0; ch < CC; ++ch) a.xsep[(xb + y * CC + ch) * ns + sys] = v[y][ch];
  });
}

// Segment length of the reduced chain of NG group 2-ports run by nw warps:
// about sqrt(NG) segments of m 2-ports (a fold step costs about 1.5 chain
// steps), at most nw of them; the last segment may be shorter.
__host__ __device__ inline int chain_segment_len(int NG, int nw) {
  int S = 1;
  while ((S + 1) * (S + 1) <= (NG * 6) / 5) ++S;
  int m = (NG + S - 1) / S;
  while ((NG + m - 1) / m > nw) ++m;
  return m;
}

// Reduced system of one band (32 subsystems).  When the band's group
// 2-ports fit in shared memory (copied there through L2: other blocks wrote
// them) the chain is split into S segments: warp s folds segment s's 2-ports
// into one (in place: the merge factors of its i-th merge overwrite 2-port
// i, the folded 2-port its first), warp 0 solves the chain of the S segment
// 2-ports, then warp s back-fills the separators inside segment s.  Serial
// depth about 2 sqrt(NG) instead of 2 NG.  Otherwise warp 0 runs the whole
// chain from global memory.  Lane = subsystem.
template <int R, int CC>
__device__ __forceinline__ void band_chain(const PassArgs& a, int bx, float* smem) {
  using F = Fields<R, CC>;
  const int lane = threadIdx.x;
  const int sys = bx * 32 + lane;
  const int NG = a.ngroups;
  const long long ns = a.sstride;
  const bool ok = sys < a.nsys;
  if (!a.chain_smem) {
    if (threadIdx.y != 0) return;
    float* const S = a.summ;
    reduced_chain<R, CC>(
        a, sys, NG, ok, [&](int g, int field) -> float& { return S[((long long)g * F::N + field) * ns + sys]; },
        [](int g) { return g; });
    return;
  }
  // rows of 32 subsystems are 128-byte lines (the stride is a multiple of
  // 32): 16-byte asynchronous copies, all in flight at once (through L2)
  const int nq = NG * F::N * 8;
  const int tid = threadIdx.y * 32 + lane;
  for (int q = tid; q < nq; q += 32 * blockDim.y) {
    const int row = q >> 3, qq = q & 7;
    cp_async16(smem + row * 32 + qq * 4, a.summ + (long long)row * ns + bx * 32 + qq * 4, 16);
  }
  cp_async_wait_all();
  __syncthreads();
  auto slot = [&](int g) { return Strided{smem + g * F::N * 32 + lane, 32}; };
  const int m = chain_segment_len(NG, blockDim.y);
  const int S = (NG + m - 1) / m;
  if (S < 2) {
    if (threadIdx.y != 0) return;
    reduced_chain<R, CC>(
        a, sys, NG, ok, [&](int g, int field) -> float& { return smem[(g * F::N + field) * 32 + lane]; },
        [](int g) { return g; });
    return;
  }
  const int w = threadIdx.y;
  auto seg0 = [&](int sg) { return min(sg * m, NG); };   // first group of segment sg
  const int g0 = seg0(w), g1 = seg0(w + 1);
  auto has_bot = [&](int i) { return g0 + i < NG - 1; };
  auto mf = [&](int i) { return slot(g0 + i); };
  if (w < S) fold_2ports<R, CC>(g1 - g0, g0 > 0, [&](int i) { return slot(g0 + i); }, has_bot, mf, slot(g0));
  __syncthreads();
  if (w == 0)
    reduced_chain<R, CC>(
        a, sys, S, ok, [&](int sg, int field) -> float& { return smem[(seg0(sg) * F::N + field) * 32 + lane]; },
        [&](int sg) { return seg0(sg + 1) - 1; });
  __syncthreads();   // the segment separators (global, this block's writes) are visible
  if (w >= S || !ok) return;
  constexpr int XS = R * CC;
  float xX[R][CC], xZ[R][CC];
#pragma unroll
  for (int i = 0; i < R; ++i)
#pragma unroll
    for (int ch = 0; ch < CC; ++ch) {
      xX[i][ch] = g0 > 0 ? a.xsep[((long long)(g0 - 1) * XS + i * CC + ch) * ns + sys] : 0.f;
      xZ[i][ch] = g1 < NG ? a.xsep[((long long)(g1 - 1) * XS + i * CC + ch) * ns + sys] : 0.f;
    }
  backfill_2ports<R, CC>(g1 - g0, g0 > 0, xX, xZ, has_bot, mf, [&](int i, const float (&v)[R][CC]) {
    const long long xb = (long long)(g0 + i - 1) * XS;
#pragma unroll
    for (int y = 0; y < R; ++y)
#pragma unroll
      for (int ch = 0; ch < CC; ++ch) a.xsep[(xb + y * CC + ch) * ns + sys] = v[y][ch];
  });
}

// SM 0: the factors are not kept (k_recover follows); 1: kept (a.fac,
// k_backsub follows); 2: kept, right-hand sides from a.rhs (the
// refinement's second solve); 3: kept, a vector guidance of a.gc planes.
// One instantiation per mode keeps the unused sweeps out of each kernel's
// code.
// Returns true (in every thread) when this block completed its band: it
// solved the band's reduced system, or the band has a single chunk group.
template <int R, int CC, int SM>
__device__ __forceinline__ bool body_summary(const PassArgs& a, int bx, int by, float* smem) {
  using F = Fields<R, CC>;
  using MF = MFields<R, CC>;
  const int lane = threadIdx.x;
  const int G = blockDim.y;
  const int sys = bx * 32 + lane;
  const int grp = by;
  const int c0 = grp * G;
  const int nch = min(G, a.P - c0);
  const int c = c0 + threadIdx.y;

  // the band's strips start at its first subsystem's: offset 32 bx for step
  // 1, that centre minus r in general
  const bool unit = a.step == 1;
  const int off0 = unit ? bx * 32 : centre_of(a, bx * 32, R) - R;
  Tile t;
  group_tile(a, c0, G, off0, unit ? 32 + 2 * R : tile_ncol(R, a.step), unit, smem, t);
  // SM 3: a guidance of a.gc planes (tile planes CC .. CC + gc - 1)
  const int np = CC + (SM == 3 ? a.gc : 1);
  // [G][F::N][32]: the chunk 2-ports.  Radius <= 3: written over the tile
  // once every warp finished its sweep (a block holds the tile or the
  // 2-ports, not both); larger radii (2-ports of 60+ values, too many to
  // hold across the barrier) after the tile.
  constexpr bool OVER = tile_over_2ports(R);
  float* csum = OVER ? smem : smem + np * t.pstride;
  // The guidance is an input of the whole filter (no kernel of the filter
  // writes it): its planes are staged before the wait, overlapping the
  // preceding kernel's tail; the estimate planes after it.
  if (a.tma) {   // (a sliding step's wider tile too: its box starts at 32 bx step, 16-byte aligned)
    __shared__ unsigned long long s_bar;
    if (threadIdx.x == 0 && threadIdx.y == 0) mbar_init(&s_bar, 1);
    __syncthreads();
    if (threadIdx.x == 0 && threadIdx.y == 0) mbar_expect_tx(&s_bar, tma_tile_bytes(t, np));
    tma_stage<CC>(a, t, CC, np, &s_bar);
    griddep_wait();
    griddep_launch();
    tma_stage<CC>(a, t, 0, CC, &s_bar);
    mbar_wait_bounded(&s_bar, 0, a.err);
  } else {
    if (unit) stage_tile<CC, 32 + 2 * R>(a, t, CC, np); else stage_tile_rt<CC>(a, t, CC, np);
    griddep_wait();
    griddep_launch();
    if (unit) stage_tile<CC, 32 + 2 * R>(a, t, 0, CC); else stage_tile_rt<CC>(a, t, 0, CC);
    cp_async_wait_all();
  }
  __syncthreads();

  const bool active = sys < a.nsys;
  const bool mine = active && threadIdx.y < nch;
  const int col = unit ? lane : centre_of(a, sys, R) - R - off0;   // the lane's strip in the tile
  if constexpr (OVER) {
    float outv[F::N];
    if (mine) chunk_summary<R, CC, SM != 0, SM == 2, SM == 3>(a, t, col, sys, c, outv);
    __syncthreads();   // the tile is read no more
    if (mine) {
#pragma unroll
      for (int f = 0; f < F::N; ++f) csum[(threadIdx.y * F::N + f) * 32 + lane] = outv[f];
    }
  } else {
    if (mine)
      chunk_summary<R, CC, SM != 0, SM == 2, SM == 3>(a, t, col, sys, c, Strided{csum + threadIdx.y * F::N * 32 + lane, 32});
  }
  __syncthreads();
  merge_tree<R, CC>(a, csum, lane, sys, grp, c0, nch, G, active);
  if (a.ngroups < 2) return true;   // one group: no reduced system
  // The last block of this band of 32 subsystems to finish (an atomic ticket
  // taken after a memory fence; nothing waits) solves the band's reduced
  // system on the group separators, overlapping the other bands' work.
  __shared__ int s_last;
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0 && threadIdx.y == 0) s_last = atomicAdd(&a.band_cnt[bx], 1) == a.ngroups - 1;
  __syncthreads();
  if (!s_last) return false;
  __threadfence();
  band_chain<R, CC>(a, bx, smem);
  if (threadIdx.x == 0 && threadIdx.y == 0) a.band_cnt[bx] = 0;   // ready for the next pass
  return true;
}

// Blocks of 256 threads per SM that the registers must allow (the block's
// shared memory allows them): four at radius 1, three at radius 2, two at
// radius 3; larger radii keep their r x r windows in up to 255 registers.
template <int R, int CC, int SM>
__global__ void __launch_bounds__(256, R == 1 ? 4 : R == 2 ? 3 : R == 3 ? 2 : 1)
    k_summary(const __grid_constant__ PassArgs a) {
  extern __shared__ __align__(128) float smem[];
  body_summary<R, CC, SM>(a, blockIdx.x, blockIdx.y, smem);
}

// Separator values of every chunk of a group (one block): loads the group's
// merge factors (asynchronous copies) and its two outer separators, then
// back-fills the separators between its chunks down the merge tree of
// merge_tree, one warp per merge of a level (lane = subsystem).
// ports[(i * 2 + side) * r*CC * 32 + lane] receives the top (side 0) and
// bottom (side 1) separator of chunk c0 + i; mbuf holds the merge factors.
// Waits for all of the block's asynchronous copies.
template <int R, int CC>
__device__ __forceinline__ void group_ports(const PassArgs& a, int grp, int c0, int nch, int sys, int lane,
                                            float* ports, float* mbuf) {
  using MF = MFields<R, CC>;
  constexpr int XS = R * CC;
  const int G = blockDim.y;
  const long long ns = a.sstride;
  // (the tree's merge slots are not contiguous when nch < G: copy all G-1)
  for (int i = threadIdx.y; i < (nch > 1 ? G - 1 : 0); i += G) {
    const float* src = a.mdata + ((long long)(grp * (G - 1) + i) * MF::N) * ns + sys;
    float* dst = mbuf + i * MF::N * 32 + lane;
#pragma unroll
    for (int f = 0; f < MF::N; ++f) cp_async4(dst + f * 32, src + f * ns, true);
  }
  if (threadIdx.y == G - 1) {
    float* dst = mbuf + (G - 1) * MF::N * 32 + lane;
#pragma unroll
    for (int i = 0; i < XS; ++i) {
      dst[i * 32] = c0 > 0 ? a.xsep[((long long)(grp - 1) * XS + i) * ns + sys] : 0.f;
      dst[(XS + i) * 32] = grp < a.ngroups - 1 ? a.xsep[((long long)grp * XS + i) * ns + sys] : 0.f;
    }
  }
  cp_async_wait_all();
  __syncthreads();
  // the group's outer separators: top of its first chunk, bottom of its last
  if (threadIdx.y == 0) {
    const float* xo = mbuf + (G - 1) * MF::N * 32 + lane;
    float* pp = ports + lane;
    float* pl = ports + ((nch - 1) * 2 + 1) * XS * 32 + lane;
#pragma unroll
    for (int i = 0; i < XS; ++i) {
      pp[i * 32] = xo[i * 32];
      pl[i * 32] = xo[(XS + i) * 32];
    }
  }
  __syncthreads();
  // back-fill down the merge tree (the merges of merge_tree in reverse): the
  // separator of merge (l, w) lies between chunks left+span-1 and left+span
  int top = 1;
  while (top < nch) top *= 2;
  for (int span = top / 2; span >= 1; span /= 2) {
    const int left = threadIdx.y * 2 * span;
    if (left + span < nch) {
      const int id = G - G / span + threadIdx.y;
      const int last = min(left + 2 * span, nch) - 1;
      float xX[R][CC], xZ[R][CC];
      const float* pt = ports + (left * 2) * XS * 32 + lane;        // top of chunk left
      const float* pb = ports + (last * 2 + 1) * XS * 32 + lane;    // bottom of chunk last
#pragma unroll
      for (int i = 0; i < R; ++i)
#pragma unroll
        for (int ch = 0; ch < CC; ++ch) {
          xX[i][ch] = pt[(i * CC + ch) * 32];
          xZ[i][ch] = pb[(i * CC + ch) * 32];
        }
      backfill_2ports<R, CC>(
          2, c0 + left > 0, xX, xZ, [&](int) { return c0 + last < a.P - 1; },
          [&](int) { return Strided{mbuf + id * MF::N * 32 + lane, 32}; },
          [&](int, const float (&v)[R][CC]) {
            float* p0 = ports + ((left + span - 1) * 2 + 1) * XS * 32 + lane;   // bottom of chunk left+span-1
            float* p1 = ports + ((left + span) * 2) * XS * 32 + lane;           // top of chunk left+span
#pragma unroll
            for (int y = 0; y < R; ++y)
#pragma unroll
              for (int ch = 0; ch < CC; ++ch) {
                p0[(y * CC + ch) * 32] = v[y][ch];
                p1[(y * CC + ch) * 32] = v[y][ch];
              }
          });
    }
    __syncthreads();
  }
}

// Row direction: writes the block's staged output lines ([NOUT][OB][lines],
// pitch opitch; across-offsets o0 .. o0 + nown - 1, OB rows per channel)
// along the image rows.
template <int NOUT, int OB>
__device__ __forceinline__ void flush_otile(const PassArgs& a, int bx, int c0, const float* otile, int opitch,
                                            int o0 = -1, int nown = OB) {
  const int G = blockDim.y;
  const int oline0 = c0 * a.h;
  const int nl = min((c0 + G) * a.h, a.L) - oline0;
  if (o0 < 0) o0 = bx * OB;
  for (int row = threadIdx.y; row < NOUT * OB; row += G) {
    const int ch = row / OB;
    const int o = row - ch * OB;
    const int oabs = o0 + o;
    if (o >= nown || oabs >= a.D) continue;
    const float* src = otile + row * opitch;
    const long long gbase = ch * a.plane + (long long)oabs * a.W + oline0;
    float* const outw = reinterpret_cast<float*>(a.out);
    for (int l = threadIdx.x; l < nl; l += 32) {
      if (a.out_dt == DT_F32)
        outw[gbase + l] = src[l];
      else
        st_px(a.out, gbase + l, a.out_dt, src[l]);
    }
  }
}

// flush_otile with a runtime number of rows per channel (own), writing
// across-offsets o0 .. o0 + nown - 1.
template <int NOUT>
__device__ __forceinline__ void flush_otile_n(const PassArgs& a, int c0, const float* otile, int opitch, int own,
                                              int o0, int nown) {
  const int G = blockDim.y;
  const int oline0 = c0 * a.h;
  const int nl = min((c0 + G) * a.h, a.L) - oline0;
  for (int row = threadIdx.y; row < NOUT * nown; row += G) {
    const int ch = row / nown;
    const int o = row - ch * nown;
    const float* src = otile + (ch * own + o) * opitch;
    const long long gbase = ch * a.plane + (long long)(o0 + o) * a.W + oline0;
    for (int l = threadIdx.x; l < nl; l += 32) {
      if (a.out_dt == DT_F32)
        reinterpret_cast<float*>(a.out)[gbase + l] = src[l];
      else
        st_px(a.out, gbase + l, a.out_dt, src[l]);
    }
  }
}

// ---------------------------------------------------------------------------
// k_recover: back-fill of the group's separators, exact interior solves with
// known separators, write-back and averaging.  Grid (ceil(D / OB), NG),
// block (32, G); lane = centre, warp = chunk.
//
// BWD: the adjoint of the pass.  The CC right-hand sides are u-planes (the
// pass input, NOUT = CC/2 channels) and v-planes (dLoss/d(pass output) /
// count); the kernel writes dLoss/d(pass input) = sum over subsystems of v,
// and accumulates dLoss/dG and dLoss/dlambda from every pair of entries.
template <int R, int CC, bool BWD = false>
__device__ __forceinline__ void body_recover(const PassArgs& a, int bx, int by, float* smem) {
  constexpr int n = 2 * R + 1;
  constexpr int NF = R + CC;       // stored per entry: L[p, p-1..p-R], z
  constexpr int OB = 32 - 2 * R;   // outputs per warp
  constexpr int XS = R * CC;       // values per separator
  constexpr int NOUT = BWD ? CC / 2 : CC;   // output channels
  constexpr int NCOL = 32 + 2 * R;
  using MF = MFields<R, CC>;
  const int lane = threadIdx.x;
  const int G = blockDim.y;
  const int grp = by;
  const int c0 = grp * G;
  const int nch = min(G, a.P - c0);
  const int c = c0 + threadIdx.y;
  const int kc = bx * OB - R + lane;  // this lane's centre
  const int sys_raw = kc - R;
  const bool valid = sys_raw >= 0 && sys_raw < a.nsys;
  const int sys = min(max(sys_raw, 0), a.nsys - 1);
  const int mcap = a.h * n;

  Tile t;
  group_tile(a, c0, G, bx * OB - 2 * R, 32 + 2 * R, true, smem, t);
  float* ports = smem + (CC + 1) * t.pstride;   // [G][2][XS][32]
  float* mbuf = ports + G * 2 * XS * 32;               // [G-1][MF::N][32] merge factors + [2][XS][32]
  float* store = mbuf + (G - 1) * MF::N * 32 + 2 * XS * 32;   // [G][mcap][NF][32]
  // The input tile comes from the pass before the preceding k_summary, which
  // completed before that k_summary passed its own wait; with a single chunk
  // (no k_summary) the preceding kernel produced the input, so wait first.
  if (!BWD && a.tma) {
    __shared__ unsigned long long s_bar;
    if (threadIdx.x == 0 && threadIdx.y == 0) mbar_init(&s_bar, 1);
    __syncthreads();
    if (!a.early_stage) griddep_wait();
    if (threadIdx.x == 0 && threadIdx.y == 0) mbar_expect_tx(&s_bar, tma_tile_bytes(t, CC + 1));
    tma_stage<CC>(a, t, 0, CC + 1, &s_bar);
    if (a.early_stage) griddep_wait();
    griddep_launch();
    mbar_wait_bounded(&s_bar, 0, a.err);
  } else {
    if (!a.early_stage) griddep_wait();
    stage_tile<CC, 32 + 2 * R>(a, t);
    if (a.early_stage) griddep_wait();
    griddep_launch();
  }
  group_ports<R, CC>(a, grp, c0, nch, sys, lane, ports, mbuf);
  // Row direction: the block's output lines are staged as [CC][OB][lines]
  // (odd pitch) and written out along the lines at the end.
  const int oline0 = c0 * a.h;
  const int opitch = (G * a.h) | 1;
  float* const otile = store + G * mcap * NF * 32;
  float* const gacc = otile + NOUT * OB * opitch;   // BWD: [ntl][NCOL] dLoss/dG
  float lam_acc = 0.f;
  const bool owner = valid && lane >= R && lane < 32 - R;
  if constexpr (BWD) {
    for (int i = threadIdx.y * 32 + lane; i < t.ntl * NCOL; i += G * 32) gacc[i] = 0.f;
    __syncthreads();
  }

  if (threadIdx.y < nch) {  // warp-uniform
  const Chunk q = make_chunk<R>(a, c);
  float xT[R][CC], xB[R][CC];
  {
    const float* pp = ports + (threadIdx.y * 2) * XS * 32 + lane;
#pragma unroll
    for (int i = 0; i < R; ++i)
#pragma unroll
      for (int ch = 0; ch < CC; ++ch) {
        xT[i][ch] = pp[(i * CC + ch) * 32];
        xB[i][ch] = pp[(XS + i * CC + ch) * 32];
      }
  }
  float* const st = store + threadIdx.y * mcap * NF * 32 + lane;

  // ---- forward sweep over the interior: L row and z = y / D per entry
  const int pstride = t.pstride;
  {
    float wh[R][R] = {};
    float Lw[R][R] = {};
    float Dw[R] = {};
    float mw[R] = {};
    float Uw[R][R] = {};
    float yw[R][CC] = {};
    if (q.top) prologue_weights<R, CC>(a, t, lane, q.line0 - 1, wh);
    for_lines(q.line0, q.line1, [&](auto odd, const bool FIRST, auto last, int line) {
      constexpr bool ODD = decltype(odd)::value;
      constexpr bool LAST = decltype(last)::value;
      const float* gr = t.row(CC, line) + lane;
      const float* gnr = t.row(CC, line + 1) + lane;
      const float* fr = t.row(0, line) + lane;
      const bool end_ok = line + 1 < a.L;
      float* lslot = st + (line - q.line0) * n * NF * 32;
#pragma unroll LineUnroll<R>::value
      for (int j = 0; j < n; ++j) {
        float wf[R];
        forward_weights<R, ODD>(a, gr, gnr, j, end_ok, wf);
        const bool sep = LAST && q.bot && j >= n - R;
        if (!sep) {
          // the factored matrix is the interior alone: the couplings to the
          // separators (known values, moved to the right-hand side below)
          // count as margin
          float mbase = 1.f;
          unsigned keep = ~0u;
          if (FIRST && q.top) {
#pragma unroll
            for (int i = 0; i < R; ++i)
#pragma unroll
              for (int tt = 1; tt <= R; ++tt)
                if (tt == j + R - i) mbase += wh[tt - 1][tt - 1];
          }
          if (LAST && q.bot) {
#pragma unroll
            for (int tt = 1; tt <= R; ++tt)
              if (j + tt >= n - R) {
                mbase += wf[tt - 1];
                keep &= ~(1u << (tt - 1));
              }
          }
          float Lrow[R], mp, Up[R];
          const float dinv =
              fast_rcp(gth_row<R>(mbase, wf, wh, Lw, Dw, mw, Uw, FIRST ? min(j, R) : R, keep, Lrow, mp, Up));
          float y[CC];
#pragma unroll
          for (int ch = 0; ch < CC; ++ch) y[ch] = fr[ch * pstride + ecol<R, ODD>(j)];
          if (FIRST) {
            if (q.top) {
              // + lambda w(p-tt, p) x(b-R+i) for separator entries above, tt = j + R - i
#pragma unroll
              for (int i = 0; i < R; ++i)
#pragma unroll
                for (int tt = 1; tt <= R; ++tt)
                  if (tt == j + R - i)
#pragma unroll
                    for (int ch = 0; ch < CC; ++ch) y[ch] += wh[tt - 1][tt - 1] * xT[i][ch];
            }
          }
          if (LAST) {
            if (q.bot) {
              // + lambda w(p, p+tt) x(e+i) for separator entries below, i = j + tt - (n - R)
#pragma unroll
              for (int i = 0; i < R; ++i)
#pragma unroll
                for (int tt = 1; tt <= R; ++tt)
                  if (i == j + tt - (n - R))
#pragma unroll
                    for (int ch = 0; ch < CC; ++ch) y[ch] += wf[tt - 1] * xB[i][ch];
            }
          }
          fwd_subst<R, CC>(Lrow, yw, y);
          float* slot = lslot + j * NF * 32;
#pragma unroll
          for (int tt = 0; tt < R; ++tt) slot[tt * 32] = Lrow[tt];
#pragma unroll
          for (int ch = 0; ch < CC; ++ch) slot[(R + ch) * 32] = y[ch] * dinv;
          push_factor<R>(Lw, Dw, Lrow, dinv);
          push_gth<R>(mw, Uw, mp, Up);
          push_vec<R, CC>(yw, y);
        }
        push_weights<R>(wh, wf);
      }
    });
  }

  // ---- backward sweep, write-back and averaging per line
  const int o = kc;  // output across-offset of this lane
  const bool writer = lane >= R && lane < 32 - R && o >= 0 && o < a.D;
  float inv_cnt = 0.f;
  if (writer) {
    const int lo = max(R, o - R), hi = min(a.D - 1 - R, o + R);
    inv_cnt = 1.0f / (float)(hi - lo + 1);
  }
  float Lb[R][R] = {};   // Lb[u-1][t-1] = L[p+u, p+u-t]
  float xw[R][CC] = {};  // x of entries p+1 .. p+R (interior only)
  float xpw[R][CC] = {}; // BWD: x of entries p+1 .. p+R of the chunk (with its separator)
  // BWD pair term of entries p (line lp, entry jp) and q = p + tq, owned by
  // this chunk: dLoss/dG and dLoss/dlambda contributions.
  auto pair_terms = [&](auto oddp, int lp, int jp, const float (&xp)[CC], int tq, const float (&xq)[CC]) {
    constexpr bool ODDP = decltype(oddp)::value;
    const int jq = jp + tq;
    const int lq = jq < n ? lp : lp + 1;
    const int colp = lane + ecol<R, ODDP>(jp);
    const int colq = lane + (jq < n ? ecol<R, ODDP>(jq) : ecol<R, !ODDP>(jq - n));
    const float gp = t.row(CC, lp)[colp];
    const float gq = t.row(CC, lq)[colq];
    float sdot = 0.f;
#pragma unroll
    for (int ch = 0; ch < NOUT; ++ch) sdot += (xp[NOUT + ch] - xq[NOUT + ch]) * (xp[ch] - xq[ch]);
    const float dg = gp - gq;
    const float sp = a.sp0[jp * R + tq - 1];
    float w, dw;
    if (a.weight == 0) {
      w = sp * fast_ex2(dg * dg * a.range_k);
      dw = -w * dg * a.dgk;
    } else {
      const float ad = fabsf(dg);
      const float hh = 1.0f / (powf(ad, a.range_k) + a.eps);
      w = sp * hh;
      dw = ad > 0.f ? -sp * hh * hh * a.range_k * powf(ad, a.range_k - 1.0f) * (dg > 0.f ? 1.f : -1.f) : 0.f;
    }
    lam_acc -= w * sdot;
    const float gb = -a.lam * sdot * dw;
    atomicAdd_block(&gacc[(lp - t.tl0) * NCOL + colp], gb);
    atomicAdd_block(&gacc[(lq - t.tl0) * NCOL + colq], -gb);
  };
  const long long ostride = a.dir == 0 ? 1 : a.W;
  const long long lstride = a.dir == 0 ? a.W : 1;
  float* const outp = reinterpret_cast<float*>(a.out);
  constexpr bool XREG = LineUnroll<R>::value > 1;   // line values in registers
  for_lines_rev(q.line0, q.line1, [&](auto odd, auto last, int line) {
    constexpr bool ODD = decltype(odd)::value;
    constexpr bool LAST = decltype(last)::value;
    float xl[XREG ? n : 1][CC];
    (void)xl;
    float* lslot = st + (line - q.line0) * n * NF * 32;
#pragma unroll LineUnroll<R>::value
    for (int j = n - 1; j >= 0; --j) {
      float x[CC];
      float* slot = lslot + j * NF * 32;
      if (LAST && q.bot && j >= n - R) {
#pragma unroll
        for (int i = 0; i < R; ++i)
          if (i == j - (n - R))
#pragma unroll
            for (int ch = 0; ch < CC; ++ch) x[ch] = xB[i][ch];
      } else {
        float Lrow[R];
#pragma unroll
        for (int tt = 0; tt < R; ++tt) Lrow[tt] = slot[tt * 32];
#pragma unroll
        for (int ch = 0; ch < CC; ++ch) x[ch] = slot[(R + ch) * 32];
#pragma unroll
        for (int tt = 1; tt <= R; ++tt)
#pragma unroll
          for (int ch = 0; ch < CC; ++ch) x[ch] -= Lb[tt - 1][tt - 1] * xw[tt - 1][ch];
#pragma unroll
        for (int u = R - 1; u > 0; --u)
#pragma unroll
          for (int tt = 0; tt < R; ++tt) Lb[u][tt] = Lb[u - 1][tt];
#pragma unroll
        for (int tt = 0; tt < R; ++tt) Lb[0][tt] = Lrow[tt];
        push_vec<R, CC>(xw, x);
      }
      if constexpr (BWD) {
        if (owner) {
#pragma unroll
          for (int tq = 1; tq <= R; ++tq)
            if (!LAST || j + tq < n) pair_terms(odd, line, j, x, tq, xpw[tq - 1]);
        }
        push_vec<R, CC>(xpw, x);
      }
      if constexpr (XREG) {
#pragma unroll
        for (int ch = 0; ch < CC; ++ch) xl[j][ch] = x[ch];
      } else {
#pragma unroll
        for (int ch = 0; ch < CC; ++ch) slot[(R + ch) * 32] = x[ch];
      }
    }
    // inverse construction + averaging: value at across-offset kc - R + e
    const long long pix = (long long)line * lstride + (long long)o * ostride;
    constexpr int CH0 = BWD ? NOUT : 0;   // BWD: the v-planes
    const float scale = BWD ? 1.f : inv_cnt;
#pragma unroll
    for (int ch = 0; ch < NOUT; ++ch) {
      float voff[n];
#pragma unroll
      for (int e2 = 0; e2 < n; ++e2) {
        float v;
        if constexpr (XREG) v = xl[ecol<R, ODD>(e2)][CH0 + ch];
        else v = lslot[ecol<R, ODD>(e2) * NF * 32 + (R + CH0 + ch) * 32];
        voff[e2] = valid ? v : 0.f;
      }
      float sum = voff[R];
#pragma unroll
      for (int d = 1; d <= R; ++d) {
        sum += __shfl_down_sync(0xffffffffu, voff[R - d], d);  // from centre kc + d
        sum += __shfl_up_sync(0xffffffffu, voff[R + d], d);    // from centre kc - d
      }
      if (writer) {
        if (a.dir != 0)
          otile[(ch * OB + (lane - R)) * opitch + (line - oline0)] = sum * scale;
        else if (a.out_dt == DT_F32)
          outp[pix + ch * a.plane] = sum * scale;
        else
          st_px(a.out, pix + ch * a.plane, a.out_dt, sum * scale);
      }
    }
  });
  if constexpr (BWD) {
    // pairs from the separator above into this chunk's first entries
    if (q.top && owner) {
      const int lp = q.line0 - 1;
      auto virt = [&](auto oddp) {
#pragma unroll
        for (int d = 1; d <= R; ++d) {
          float xv[CC];
#pragma unroll
          for (int ch = 0; ch < CC; ++ch) xv[ch] = xT[R - d][ch];
#pragma unroll
          for (int tq = 1; tq <= R; ++tq)
            if (tq >= d) pair_terms(oddp, lp, n - d, xv, tq, xpw[tq - 1]);
          push_vec<R, CC>(xpw, xv);
        }
      };
      if (lp & 1) virt(std::true_type{}); else virt(std::false_type{});
    }
  }
  }  // this warp's chunk

  if (a.dir != 0 || BWD) __syncthreads();
  if (a.dir != 0) flush_otile<NOUT, OB>(a, bx, c0, otile, opitch);
  if constexpr (BWD) {
    // dLoss/dlambda: warp sum, one atomic per warp
#pragma unroll
    for (int d = 16; d >= 1; d >>= 1) lam_acc += __shfl_down_sync(0xffffffffu, lam_acc, d);
    if (lane == 0 && lam_acc != 0.f) atomicAdd(a.grad_lam, lam_acc);
    // dLoss/dG of this block's pairs
    for (int i = threadIdx.y * 32 + lane; i < t.ntl * NCOL; i += G * 32) {
      const float v = gacc[i];
      if (v == 0.f) continue;
      const int tl = i / NCOL;
      const int col = i - tl * NCOL;
      const int line = t.tl0 + tl, off = t.off0 + col;
      if (line >= 0 && line < a.L && off >= 0 && off < a.D) atomicAdd(a.grad_g + pix_index(a, line, off), v);
    }
  }
}

template <int R, int CC, bool BWD>
__global__ void __launch_bounds__(256) k_recover(const __grid_constant__ PassArgs a) {
  extern __shared__ __align__(128) float smem[];
  body_recover<R, CC, BWD>(a, blockIdx.x, blockIdx.y, smem);
}

// ---------------------------------------------------------------------------
// k_backsub: the second kernel of a pass when k_summary kept the chunk
// factors (a.fac).  Back-fills the group's separators, then every thread
// runs the backward substitution of its chunk from the kept rows,
//   x_e = z0_e + Phi_e xT + Psi_e xB - sum_t L[e+t, e] x_{e+t},
// and averages each pixel's 2r+1 values across the neighbouring centres'
// lanes.  No tile, no weights: the factors come from L2.  Grid (ceil(D / OB),
// NG), block (32, G); lane = centre, warp = chunk.
// MODE 0: step 1; 1: step > 1; 2: step 1 with the refinement's entry
// buffers (xmode).
template <int R, int CC, int MODE>
__device__ __forceinline__ void body_backsub(const PassArgs& a, int bx, int by, float* smem) {
  constexpr int n = 2 * R + 1;
  constexpr int NFAC = 2 * R + CC;
  constexpr int OB = 32 - 2 * R;
  constexpr int XS = R * CC;
  using MF = MFields<R, CC>;
  const int lane = threadIdx.x;
  const int G = blockDim.y;
  const int grp = by;
  const int c0 = grp * G;
  const int nch = min(G, a.P - c0);
  const int c = c0 + threadIdx.y;
  // step 1: lane = across-offset kc (the centre of subsystem kc - r when
  // that exists), 2r halo lanes; step > 1: lane = subsystem, HL halo lanes
  constexpr bool unit = MODE != 1;   // MODE 1: the launch's step is > 1
  const int HL = step_halo(R, a.step);
  const int SB = 32 - 2 * HL;
  const int kc = bx * OB - R + lane;
  const int sys_raw = unit ? kc - R : bx * SB - HL + lane;
  const bool valid = sys_raw >= 0 && sys_raw < a.nsys;
  const int sys = min(max(sys_raw, 0), a.nsys - 1);
  const int OWN = unit ? OB : step_own_max(R, a.step);   // otile rows per channel
  // MODE 3: the adjoint pass from kept factors (planes 0 .. CC/2-1 hold u,
  // CC/2 .. CC-1 v): its output is the sum of the v values a pixel
  // received, plus the pair terms of dLoss/dG and dLoss/dlambda
  constexpr bool BWD = MODE == 3;
  constexpr int NOUT = BWD ? CC / 2 : CC;   // output planes
  constexpr int NCOL = 32 + 2 * R;           // BWD: columns of the guidance tile

  float* ports = smem;                                  // [G][2][XS][32]
  float* mbuf = ports + G * 2 * XS * 32;                // [G-1][MF::N][32] + [2][XS][32]
  float* otile = mbuf + (G - 1) * MF::N * 32 + 2 * XS * 32;   // [NOUT][OWN][opitch]
  const int opitch = (G * a.h) | 1;
  // BWD: the guidance tile of the group's lines (one line of halo above)
  // and the block's dLoss/dG accumulators, both [ntl][NCOL], columns from
  // the first lane's strip (across-offset bx OB - 2r)
  const int gtl0 = c0 * a.h - 1;
  const int gntl = min((c0 + G) * a.h, a.L) + 1 - gtl0;
  float* const gtile = otile + NOUT * OWN * opitch;
  float* const gacc = gtile + gntl * NCOL;
  float lam_acc = 0.f;
  if constexpr (BWD) {
    // the guidance is an input of the whole filter: staged before the wait
    const int off0 = bx * OB - 2 * R;
    for (int i = threadIdx.y * 32 + lane; i < gntl * NCOL; i += G * 32) {
      const int tl = i / NCOL, col = i - tl * NCOL;
      const int line = gtl0 + tl, off = off0 + col;
      gtile[i] = (line >= 0 && line < a.L && off >= 0 && off < a.D) ? ld_px(a.g, pix_index(a, line, off), a.g_dt) : 0.f;
      gacc[i] = 0.f;
    }
  }
  // step > 1: per warp, CC accumulation rows and one of reciprocal counts
  const int AW = step_acc_width(R, a.step);
  float* const accw = otile + CC * OWN * opitch + threadIdx.y * (CC + 1) * AW;
  float* const invw = accw + CC * AW;
  // columns owned by this lane (step > 1): from its centre to the next
  // (from 0 for the first subsystem, to D for the last)
  const bool owner = !unit && valid && lane >= HL && lane < 32 - HL;
  const int own_lo = (sys == 0) ? 0 : centre_of(a, sys, R);
  const int own_hi = (sys == a.nsys - 1) ? a.D : centre_of(a, sys + 1, R);
  const int wsys0 = bx * SB;   // first owned subsystem of the block
  const int wlo = wsys0 == 0 ? 0 : centre_of(a, min(wsys0, a.nsys - 1), R);
  const int whi = min(wsys0 + SB, a.nsys) == a.nsys ? a.D : centre_of(a, wsys0 + SB, R);
  const int abase = centre_of(a, max(wsys0 - HL, 0), R) - R;   // offset of accw[0]
  const int lcol = centre_of(a, sys, R) - R - abase;           // the lane's strip in accw
  griddep_wait();
  griddep_launch();
  group_ports<R, CC>(a, grp, c0, nch, sys, lane, ports, mbuf);
  const int oline0 = c0 * a.h;
  if (!unit && threadIdx.y < nch) {  // (compile-time false for step 1)
    // coverage counts of the warp's columns (every column has a centre
    // within r), then their reciprocals in the owned columns
    for (int i = lane; i < (CC + 1) * AW; i += 32) accw[i] = 0.f;
    __syncwarp();
    if (valid)
      for (int e2 = 0; e2 < n; ++e2) atomicAdd(&invw[lcol + e2], 1.0f);
    __syncwarp();
    if (owner)
      for (int o = own_lo; o < own_hi; ++o) invw[o - abase] = 1.0f / invw[o - abase];
    __syncwarp();
  }

  if (threadIdx.y < nch) {  // warp-uniform
    const Chunk q = make_chunk<R>(a, c);
    float xT[R][CC], xB[R][CC];
    {
      const float* pp = ports + (threadIdx.y * 2) * XS * 32 + lane;
#pragma unroll
      for (int i = 0; i < R; ++i)
#pragma unroll
        for (int ch = 0; ch < CC; ++ch) {
          xT[i][ch] = pp[(i * CC + ch) * 32];
          xB[i][ch] = pp[(XS + i * CC + ch) * 32];
        }
    }
    const int o = kc;
    const bool writer = lane >= R && lane < 32 - R && o >= 0 && o < a.D;
    float inv_cnt = 0.f;
    if (writer) {
      const int lo = max(R, o - R), hi = min(a.D - 1 - R, o + R);
      inv_cnt = 1.0f / (float)(hi - lo + 1);
    }
    // the band's factor store and the lane in it (st_fields layout)
    const float* const fac = fac_lane<R, CC>(a, sys) - (sys & 31);
    const int flane = sys & 31;
    const float* const psi = psi_lane<R>(a, sys);
    float Lb[R][R] = {};   // Lb[u-1][t-1] = L[p+u, p+u-t]
    float xw[R][CC] = {};  // x of entries p+1 .. p+R (interior only)
    // BWD: x of entries p+1 .. p+R of the chunk (its bottom separator too);
    // a subsystem's pair terms are added by the one block that owns it
    float xpw[R][CC] = {};
    (void)xpw;
    const bool bowner = BWD && valid && lane >= R && lane < 32 - R;
    // BWD pair term of entries p (line lp, entry jp) and q = p + tq (the
    // derivative of Eq. 2's weight through Eq. 4): dLoss/dlambda and
    // dLoss/dG contributions, from the u and v values of both entries
    auto pair_terms = [&](auto oddp, int lp, int jp, const float (&xp)[CC], int tq, const float (&xq)[CC]) {
      constexpr bool ODDP = decltype(oddp)::value;
      const int jq = jp + tq;
      const int lq = jq < n ? lp : lp + 1;
      const int colp = lane + ecol<R, ODDP>(jp);
      const int colq = lane + (jq < n ? ecol<R, ODDP>(jq) : ecol<R, !ODDP>(jq - n));
      const float gp = gtile[(lp - gtl0) * NCOL + colp];
      const float gq = gtile[(lq - gtl0) * NCOL + colq];
      float sdot = 0.f;
#pragma unroll
      for (int ch = 0; ch < NOUT; ++ch) sdot += (xp[NOUT + ch] - xq[NOUT + ch]) * (xp[ch] - xq[ch]);
      const float dg = gp - gq;
      const float sp = a.sp0[jp * R + tq - 1];
      float w, dw;
      if (a.weight == 0) {
        w = sp * fast_ex2(dg * dg * a.range_k);
        dw = -w * dg * a.dgk;
      } else {
        const float ad = fabsf(dg);
        const float hh = 1.0f / (powf(ad, a.range_k) + a.eps);
        w = sp * hh;
        dw = ad > 0.f ? -sp * hh * hh * a.range_k * powf(ad, a.range_k - 1.0f) * (dg > 0.f ? 1.f : -1.f) : 0.f;
      }
      lam_acc -= w * sdot;
      const float gb = -a.lam * sdot * dw;
      atomicAdd_block(&gacc[(lp - gtl0) * NCOL + colp], gb);
      atomicAdd_block(&gacc[(lq - gtl0) * NCOL + colq], -gb);
    };
    (void)pair_terms;
    const long long ostride = a.dir == 0 ? 1 : a.W;
    const long long lstride = a.dir == 0 ? a.W : 1;
    float* const outp = reinterpret_cast<float*>(a.out);
    // r = 1 (few factor values a line): the next line's factor rows are
    // loaded into registers while the current line is solved, so the loads
    // of two lines are in flight at once
    constexpr bool PIPE = R == 1 && !BWD;
    float fnext[PIPE ? n : 1][PIPE ? NFAC : 1];
    auto load_line = [&](int l) {
      if constexpr (PIPE) {
        const float* f0 = fac + l * n * NFAC * 32;
#pragma unroll
        for (int j = 0; j < n; ++j) ld_fields<NFAC>(f0 + j * NFAC * 32, flane, fnext[j]);
      }
    };
    if constexpr (PIPE) load_line(q.line1 - 1);
    for_lines_rev(q.line0, q.line1, [&](auto odd, auto last, int line) {
      constexpr bool ODD = decltype(odd)::value;
      constexpr bool LAST = decltype(last)::value;
      float fcur[PIPE ? n : 1][PIPE ? NFAC : 1];
      if constexpr (PIPE) {
#pragma unroll
        for (int j = 0; j < n; ++j)
#pragma unroll
          for (int f = 0; f < NFAC; ++f) fcur[j][f] = fnext[j][f];
        if (line > q.line0) load_line(line - 1);
      }
      (void)fcur;
      float xl[n][CC];
      const float* fl = fac + line * n * NFAC * 32;
#pragma unroll LineUnroll<R>::value
      for (int j = n - 1; j >= 0; --j) {
        float x[CC];
        if (LAST && q.bot && j >= n - R) {
#pragma unroll
          for (int i = 0; i < R; ++i)
            if (i == j - (n - R))
#pragma unroll
              for (int ch = 0; ch < CC; ++ch) x[ch] = xB[i][ch];
        } else {
          float fe[PIPE ? 1 : NFAC];
          if constexpr (!PIPE) ld_fields<NFAC>(fl + j * NFAC * 32, flane, fe);
          auto fv = [&](int f) -> float {
            if constexpr (PIPE) return fcur[j][f]; else return fe[f];
          };
          float Lrow[R];
#pragma unroll
          for (int tt = 0; tt < R; ++tt) Lrow[tt] = fv(tt);
#pragma unroll
          for (int ch = 0; ch < CC; ++ch) x[ch] = fv(R + ch);
          if (q.top) {
#pragma unroll
            for (int i = 0; i < R; ++i) {
              const float ph = fv(R + CC + i);
#pragma unroll
              for (int ch = 0; ch < CC; ++ch) x[ch] += ph * xT[i][ch];
            }
          }
          if (LAST && q.bot && j >= n - 2 * R) {
            const float* pe = psi + ((c * R + (j - (n - 2 * R))) * R) * 32;
#pragma unroll
            for (int i = 0; i < R; ++i) {
              const float ps = __ldcg(pe + i * 32);
#pragma unroll
              for (int ch = 0; ch < CC; ++ch) x[ch] += ps * xB[i][ch];
            }
          }
#pragma unroll
          for (int tt = 1; tt <= R; ++tt)
#pragma unroll
            for (int ch = 0; ch < CC; ++ch) x[ch] -= Lb[tt - 1][tt - 1] * xw[tt - 1][ch];
#pragma unroll
          for (int u = R - 1; u > 0; --u)
#pragma unroll
            for (int tt = 0; tt < R; ++tt) Lb[u][tt] = Lb[u - 1][tt];
#pragma unroll
          for (int tt = 0; tt < R; ++tt) Lb[0][tt] = Lrow[tt];
          push_vec<R, CC>(xw, x);
        }
        if constexpr (BWD) {
          if (bowner) {
#pragma unroll
            for (int tq = 1; tq <= R; ++tq)
              if (!LAST || j + tq < n) pair_terms(odd, line, j, x, tq, xpw[tq - 1]);
          }
          push_vec<R, CC>(xpw, x);
        }
        // (registers for r <= 3; the rolled loop of larger r indexes xl
        // dynamically, which places it in local memory)
#pragma unroll
        for (int ch = 0; ch < CC; ++ch) xl[j][ch] = x[ch];
      }

      // refinement: xmode 1 keeps every entry's solution (no averaging),
      // xmode 2 adds the kept first solution to this correction
      if (MODE == 2 && a.xmode != 0) {
        float* const xe = ent_lane<R, CC>(a, a.xent, sys) + line * n * CC * 32;
        if (a.xmode == 1) {
          if (valid) {
#pragma unroll LineUnroll<R>::value
            for (int j = 0; j < n; ++j)
#pragma unroll
              for (int ch = 0; ch < CC; ++ch) xe[(j * CC + ch) * 32] = xl[j][ch];
          }
          return;
        }
#pragma unroll LineUnroll<R>::value
        for (int j = 0; j < n; ++j)
#pragma unroll
          for (int ch = 0; ch < CC; ++ch) xl[j][ch] += __ldcg(xe + (j * CC + ch) * 32);
      }
      // inverse construction + averaging: value at across-offset kc - R + e
      if constexpr (!unit) {
        // step > 1: the strips of neighbouring lanes overlap irregularly;
        // every valid lane adds its 2r+1 values into the warp's rows, the
        // owners read their columns and scale by 1 / count
        if (valid) {
#pragma unroll
          for (int ch = 0; ch < CC; ++ch)
#pragma unroll
            for (int e2 = 0; e2 < n; ++e2) atomicAdd(&accw[ch * AW + lcol + e2], xl[ecol<R, ODD>(e2)][ch]);
        }
        __syncwarp();
        if (owner) {
          for (int oo = own_lo; oo < own_hi; ++oo) {
            const float ic = invw[oo - abase];
#pragma unroll
            for (int ch = 0; ch < CC; ++ch) {
              const float v = accw[ch * AW + oo - abase] * ic;
              if (a.dir != 0)
                otile[(ch * OWN + (oo - wlo)) * opitch + (line - oline0)] = v;
              else if (a.out_dt == DT_F32)
                outp[(long long)line * lstride + oo + ch * a.plane] = v;
              else
                st_px(a.out, (long long)line * lstride + oo + ch * a.plane, a.out_dt, v);
            }
          }
        }
        __syncwarp();
        if (valid) {
#pragma unroll
          for (int ch = 0; ch < CC; ++ch)
#pragma unroll
            for (int e2 = 0; e2 < n; ++e2) accw[ch * AW + lcol + e2] = 0.f;
        }
        __syncwarp();
        return;
      }
      const long long pix = (long long)line * lstride + (long long)o * ostride;
      // (BWD: the sum of the v planes, no division: the caller divided
      // dLoss/d(pass output) by the counts before the pass)
      constexpr int CH0 = BWD ? NOUT : 0;
      const float scale = BWD ? 1.f : inv_cnt;
#pragma unroll
      for (int ch = 0; ch < NOUT; ++ch) {
        float voff[n];
#pragma unroll
        for (int e2 = 0; e2 < n; ++e2) voff[e2] = valid ? xl[ecol<R, ODD>(e2)][CH0 + ch] : 0.f;
        float sum = voff[R];
#pragma unroll
        for (int d = 1; d <= R; ++d) {
          sum += __shfl_down_sync(0xffffffffu, voff[R - d], d);  // from centre kc + d
          sum += __shfl_up_sync(0xffffffffu, voff[R + d], d);    // from centre kc - d
        }
        if (writer) {
          if (a.dir != 0)
            otile[(ch * OB + (lane - R)) * opitch + (line - oline0)] = sum * scale;
          else if (a.out_dt == DT_F32)
            outp[pix + ch * a.plane] = sum * scale;
          else
            st_px(a.out, pix + ch * a.plane, a.out_dt, sum * scale);
        }
      }
    });
    if constexpr (BWD) {
      // pairs from the separator above into this chunk's first entries
      if (q.top && bowner) {
        const int lp = q.line0 - 1;
        auto virt = [&](auto oddp) {
#pragma unroll
          for (int d = 1; d <= R; ++d) {
            float xv[CC];
#pragma unroll
            for (int ch = 0; ch < CC; ++ch) xv[ch] = xT[R - d][ch];
#pragma unroll
            for (int tq = 1; tq <= R; ++tq)
              if (tq >= d) pair_terms(oddp, lp, n - d, xv, tq, xpw[tq - 1]);
            push_vec<R, CC>(xpw, xv);
          }
        };
        if (lp & 1) virt(std::true_type{}); else virt(std::false_type{});
      }
    }
  }
  if (a.dir != 0 && !(MODE == 2 && a.xmode == 1)) {
    __syncthreads();
    if constexpr (unit)
      flush_otile<NOUT, OB>(a, bx, c0, otile, opitch);
    else
      flush_otile_n<CC>(a, c0, otile, opitch, OWN, wlo, whi - wlo);
  }
  if constexpr (BWD) {
    // dLoss/dlambda: warp sum, one atomic per warp; dLoss/dG of the block
    __syncthreads();
#pragma unroll
    for (int d = 16; d >= 1; d >>= 1) lam_acc += __shfl_down_sync(0xffffffffu, lam_acc, d);
    if (lane == 0 && lam_acc != 0.f) atomicAdd(a.grad_lam, lam_acc);
    const int off0 = bx * OB - 2 * R;
    for (int i = threadIdx.y * 32 + lane; i < gntl * NCOL; i += G * 32) {
      const float v = gacc[i];
      if (v == 0.f) continue;
      const int tl = i / NCOL, col = i - tl * NCOL;
      const int line = gtl0 + tl, off = off0 + col;
      if (line >= 0 && line < a.L && off >= 0 && off < a.D) atomicAdd(a.grad_g + pix_index(a, line, off), v);
    }
  }
}

template <int R, int CC, int MODE>
__global__ void __launch_bounds__(256) k_backsub(const __grid_constant__ PassArgs a) {
  extern __shared__ __align__(128) float smem[];
  body_backsub<R, CC, MODE>(a, blockIdx.x, blockIdx.y, smem);
}

// ---------------------------------------------------------------------------
// k_pass_q: one forward pass (sliding step 1, kept chunk factors) as a
// single persistent kernel.  Its blocks take work items from an atomic
// queue in the order of QueueSched (sgwls_sched.h): summary items (the body
// of k_summary for one chunk group of one band, the band's last one solving
// its reduced system) and back-substitution items (the body of k_backsub)
// a few bands behind them.  Compared with the two-kernel pass the factors of
// a band are read back soon after they are written, so with the factor
// store a ring of a.nslot band slots they stay in L2 instead of streaming
// through HBM, and the summary and back-substitution work of different
// bands share the SMs (no wave tail between two grids).  A back-substitution
// item waits for its bands' done flags; a summary item whose ring slot still
// holds an older band waits until that band's readers finished.  Both waits
// are bounded (wait_geq); a block whose wait gives up skips its item.
// Grid: at most the resident blocks; block (32, G).
__device__ __forceinline__ void st_release(int* p, int v) {
  asm volatile("st.release.gpu.global.b32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}
__device__ __forceinline__ bool flag_set(const unsigned* err) {
  return *reinterpret_cast<const volatile unsigned*>(err) != 0u;
}

template <int R, int CC>
__global__ void __launch_bounds__(256) k_pass_q(const __grid_constant__ PassArgs a) {
  extern __shared__ __align__(128) float smem[];
  __shared__ int s_item, s_ok;
  QueueSched q;
  q.nb = (a.nsys + 31) >> 5;
  q.OB = 32 - 2 * R;
  q.nbx = (a.D + q.OB - 1) / q.OB;
  q.NG = a.ngroups;
  q.LA = a.lookahead;
  q.r = R;
  const int total = q.total();
  const bool lead = threadIdx.x == 0 && threadIdx.y == 0;
  griddep_wait();     // the queue words were reset by the previous pass's last block
  griddep_launch();
  for (;;) {
    if (lead) s_item = atomicAdd(&a.qctl[0], 1);
    __syncthreads();
    const int item = s_item;
    if (item >= total) break;   // uniform
    int band, bx, grp;
    if (q.decode(item, &band, &bx, &grp)) {
      if (lead) {
        bool ok = !flag_set(a.err);
        if (ok && a.nslot > 0 && band >= a.nslot) {
          const int old = band - a.nslot;   // the band whose factors occupy this slot
          ok = wait_geq(&a.rdcnt[old], q.NG * q.readers(old), a.err, 1u);
        }
        s_ok = ok;
      }
      __syncthreads();
      if (s_ok) {
        const bool done = body_summary<R, CC, 1>(a, band, grp, smem);
        __threadfence();
        __syncthreads();
        if (done && lead) st_release(&a.done[band], 1);
      }
    } else {
      const int blo = q.band_lo(bx), bhi = q.band_hi(bx);
      if (lead)
        s_ok = !flag_set(a.err) && wait_geq(&a.done[blo], 1, a.err, 2u) && wait_geq(&a.done[bhi], 1, a.err, 2u);
      __syncthreads();
      if (s_ok) body_backsub<R, CC, 0>(a, bx, grp, smem);
      __syncthreads();   // every thread's factor loads have returned
      if (lead) {
        __threadfence();
        atomicAdd(&a.rdcnt[blo], 1);
        if (bhi != blo) atomicAdd(&a.rdcnt[bhi], 1);
      }
    }
    __syncthreads();
  }
  // The last block to leave resets the control words for the next pass
  // (which reads them only after its griddep_wait).
  __syncthreads();
  if (lead) {
    __threadfence();
    s_item = atomicAdd(&a.qctl[1], 1) == (int)(gridDim.x - 1);
  }
  __syncthreads();
  if (s_item) {
    const int nt = blockDim.x * blockDim.y;
    for (int b = threadIdx.y * 32 + threadIdx.x; b < q.nb; b += nt) {
      a.done[b] = 0;
      a.rdcnt[b] = 0;
    }
    if (lead) {
      a.qctl[0] = 0;
      a.qctl[1] = 0;
    }
  }
}

// ---------------------------------------------------------------------------
// k_resid: the refinement's residual rho = f - A u for every entry of every
// subsystem, in FP32, with u the first solve's entries (xent).  A = I +
// lambda L (Eq. 4, Eq. 5) is never formed: row e of A u is
//   u_e + sum_q lambda w(e, q) (u_e - u_q)
// over the entries q within r of e along the vector, so the identity's
// contribution is not rounded away next to lambda w ~ 1e7 (frac weights on
// flat guidance), which is what makes the FP32 diagonal 1 + lambda sum w
// inaccurate.  The pair weights are Eq. 2 in FP32 from the guidance, the
// same expression the forward sweep uses.  Grid (ceil(nsys / 32), ceil(L /
// (4 lines x blockDim.y))), block (32, G); lane = subsystem, each warp 4
// lines.
template <int R, int CC>
__global__ void __launch_bounds__(256) k_resid(const __grid_constant__ PassArgs a) {
  constexpr int n = 2 * R + 1;
  constexpr int LPW = 4;   // lines per warp
  const int lane = threadIdx.x;
  const int sys = blockIdx.x * 32 + lane;
  const int l0 = (blockIdx.y * blockDim.y + threadIdx.y) * LPW;
  griddep_wait();
  griddep_launch();
  if (sys >= a.nsys || l0 >= a.L) return;
  const int kc = centre_of(a, sys, R);
  const int s_len = a.L * n;
  const float* const xe = ent_lane<R, CC>(a, a.xent, sys);
  float* const re = ent_lane<R, CC>(a, a.rhs, sys);
  // pixel of entry e (line e / n, snake order within the line)
  auto pix = [&](int e) {
    const int line = e / n, j = e - line * n;
    const int off = kc - R + ((line & 1) ? 2 * R - j : j);
    return pix_index(a, line, off);
  };
  const int l1 = min(l0 + LPW, a.L);
  for (int e = l0 * n; e < l1 * n; ++e) {
    const long long pe = pix(e);
    const float ge = ld_px(a.g, pe, a.g_dt);
    float xv[CC], acc[CC];
#pragma unroll
    for (int ch = 0; ch < CC; ++ch) {
      xv[ch] = __ldcg(xe + (e * CC + ch) * 32);
      acc[ch] = ld_px(plane_base<CC>(a, ch, a.in_dt == DT_F32 ? 4 : 2), pe, a.in_dt) - xv[ch];
    }
#pragma unroll
    for (int t = 1; t <= R; ++t) {
#pragma unroll
      for (int side = 0; side < 2; ++side) {   // pairs (e, e + t) and (e - t, e)
        const int q = side == 0 ? e + t : e - t;
        if (q < 0 || q >= s_len) continue;
        const int p0 = side == 0 ? e : q;   // first entry of the pair: its position in the line picks sp
        const float w = a.sp[(p0 % n) * R + t - 1] * range_factor(a, ge - ld_px(a.g, pix(q), a.g_dt));
#pragma unroll
        for (int ch = 0; ch < CC; ++ch) acc[ch] -= w * (xv[ch] - __ldcg(xe + (q * CC + ch) * 32));
      }
    }
#pragma unroll
    for (int ch = 0; ch < CC; ++ch) re[(e * CC + ch) * 32] = acc[ch];
  }
}

}  // namespace sgwls
