// sgwls_pass.cuh -- one SG-WLS pass (Sec. 2.3) as three kernels.
//
// Every subsystem A_s u = f (Eq. 5) of a pass is a symmetric positive
// definite banded matrix of half-bandwidth r and length s = (2r+1) * lines.
// A_s is strictly diagonally dominant (diagonal minus the off-diagonal sum is
// 1, from the Eq. 4 form), so an FP32 LDL^T without pivoting is stable.  The
// paper factors each subsystem serially (its r-band LU, Eqs. 9-20); a GPU
// needs more parallelism than one thread per subsystem, so each subsystem is
// split along its lines into P chunks and solved exactly by one level of
// Schur-complement (nested dissection) reduction:
//
//   chunk c covers lines [c h, min((c+1) h, L)), vector entries [b, end);
//   its last r entries S_c (c < P-1) are the separator shared with chunk
//   c+1; the rest is the interior I_c = [b, e).  Interiors couple only to
//   the separators on both sides (bandwidth r < 2r+1 = entries per line).
//
//   k_summary   one thread per (subsystem, chunk): factors A(I_c) = L D L^T,
//               forms Y_T = L^{-1} A(I_c, S_{c-1}), Y_B = L^{-1} A(I_c, S_c),
//               y = L^{-1} f(I_c) and writes the chunk's Schur contributions
//                 KTT = Y_T' D^-1 Y_T, KTB = Y_T' D^-1 Y_B,
//                 DS  = A(S_c, S_c) - Y_B' D^-1 Y_B,
//                 HT  = Y_T' D^-1 y,   G = f(S_c) - Y_B' D^-1 y.
//   k_reduced   one thread per subsystem: block Cholesky of the reduced block
//               tridiagonal system on the separators (r x r blocks)
//                 diag_c = DS_c - KTT_{c+1},  off_{c,c+1} = -KTB_{c+1},
//                 rhs_c  = G_c - HT_{c+1},
//               and back substitution -> separator values x(S_c).
//   k_recover   one warp per (32 neighbouring centres, chunk): refactors the
//               interior, solves A(I_c) x = f - A(I,S) x(S) (forward sweep
//               into shared memory, backward sweep), writes the solution back
//               into the strip and averages each pixel's 2r+1 values across
//               the neighbouring centres' lanes with warp shuffles (steps 3-4
//               of Sec. 2.3), then stores the output line by line.
#pragma once

#include "sgwls_common.cuh"

namespace sgwls {

template <int R, int CC>
struct Fields {
  static constexpr int KTT = 0;
  static constexpr int KTB = R * R;
  static constexpr int DS = 2 * R * R;
  static constexpr int HT = 3 * R * R;
  static constexpr int GS = 3 * R * R + R * CC;
  static constexpr int N = 3 * R * R + 2 * R * CC;
};

// Loads the guidance values of one line in vector order (entry j of the line).
template <int R>
__device__ __forceinline__ void load_g_line(const PassArgs& a, int k, int line, float (&gl)[2 * R + 1]) {
  constexpr int n = 2 * R + 1;
  if (line < 0 || line >= a.L) {
#pragma unroll
    for (int j = 0; j < n; ++j) gl[j] = 0.f;
    return;
  }
  const bool rev = line & 1;
#pragma unroll
  for (int j = 0; j < n; ++j) {
    const int off = rev ? (k + R - j) : (k - R + j);
    gl[j] = ld_px(a.g, pix_index(a, line, off), a.g_dt);
  }
}

template <int R, int CC>
__device__ __forceinline__ void load_f_line(const PassArgs& a, int k, int line, float (&fl)[2 * R + 1][CC]) {
  constexpr int n = 2 * R + 1;
  const bool rev = line & 1;
#pragma unroll
  for (int j = 0; j < n; ++j) {
    const int off = rev ? (k + R - j) : (k - R + j);
    const long long idx = pix_index(a, line, off);
#pragma unroll
    for (int ch = 0; ch < CC; ++ch) fl[j][ch] = ld_px(a.in, idx + ch * a.plane, a.in_dt);
  }
}

// lambda * w(p, p+t), t = 1..R, for entry j of the current line (Eq. 2).
template <int R>
__device__ __forceinline__ void forward_weights(const PassArgs& a, int j, int p, int s,
                                                const float (&gc)[2 * R + 1], const float (&gn)[2 * R + 1],
                                                float (&wf)[R]) {
  constexpr int n = 2 * R + 1;
#pragma unroll
  for (int t = 1; t <= R; ++t) {
    const float gq = (j + t < n) ? gc[(j + t) % n] : gn[(j + t) % n];
    const float w = a.sp[j * R + t - 1] * range_factor(a, gc[j] - gq);
    wf[t - 1] = (p + t < s) ? w : 0.f;
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

// One LDL^T row for entry p.  wh[u-1][t-1] = lambda w(p-u, p-u+t); Lw[u-1][v-1]
// = L[p-u, p-u-v]; Dw[u-1] = 1/D[p-u].  `lim` = number of previous entries
// that belong to the factored interior (entries p-t with t > lim are outside).
// Returns Lrow[t-1] = L[p, p-t] and 1/D[p].
template <int R>
__device__ __forceinline__ float ldl_row(float diag, const float (&wh)[R][R], const float (&Lw)[R][R],
                                         const float (&Dw)[R], int lim, float (&Lrow)[R]) {
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
  float D = diag;
#pragma unroll
  for (int t = 0; t < R; ++t) D -= Wt[t] * Lrow[t];
  return fast_rcp(D);
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

// y = rhs - sum_t L[p, p-t] win[t-1]  (forward substitution, K columns)
template <int R, int K>
__device__ __forceinline__ void fwd_subst(const float (&Lrow)[R], const float (&win)[R][K], float (&y)[K]) {
#pragma unroll
  for (int t = 0; t < R; ++t)
#pragma unroll
    for (int i = 0; i < K; ++i) y[i] -= Lrow[t] * win[t][i];
}

// ---------------------------------------------------------------------------
// Chunk geometry shared by the kernels.
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

// ---------------------------------------------------------------------------
// k_summary: forward sweep of one chunk and its Schur contributions.
template <int R, int CC>
__global__ void __launch_bounds__(128) k_summary(const PassArgs a) {
  constexpr int n = 2 * R + 1;
  using F = Fields<R, CC>;
  const int sys = blockIdx.x * 32 + threadIdx.x;
  const int c = blockIdx.y * blockDim.y + threadIdx.y;
  if (sys >= a.nsys || c >= a.P) return;
  const int k = sys + R;
  const int s = a.L * n;
  const Chunk q = make_chunk<R>(a, c);

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
  float gc[n], gn[n];
  float wf[R];

  if (q.top) {  // weights of the line above the chunk (the top separator's line)
    load_g_line<R>(a, k, q.line0 - 1, gc);
    load_g_line<R>(a, k, q.line0, gn);
#pragma unroll
    for (int j = 0; j < n; ++j) {
      forward_weights<R>(a, j, (q.line0 - 1) * n + j, s, gc, gn, wf);
      push_weights<R>(wh, wf);
    }
  }
  load_g_line<R>(a, k, q.line0, gc);
  for (int line = q.line0; line < q.line1; ++line) {
    load_g_line<R>(a, k, line + 1, gn);
    float fl[n][CC];
    load_f_line<R, CC>(a, k, line, fl);
    const bool first = line == q.line0;
    const bool last = line == q.line1 - 1;
#pragma unroll
    for (int j = 0; j < n; ++j) {
      const int p = line * n + j;
      forward_weights<R>(a, j, p, s, gc, gn, wf);
      float diag = 1.f;
#pragma unroll
      for (int t = 0; t < R; ++t) diag += wf[t] + wh[t][t];
      const bool sep = last && q.bot && (j >= n - R);
      if (!sep) {
        const int lim = first ? j : R;
        float Lrow[R];
        const float dinv = ldl_row<R>(diag, wh, Lw, Dw, lim, Lrow);
        float y[CC];
#pragma unroll
        for (int ch = 0; ch < CC; ++ch) y[ch] = fl[j][ch];
        fwd_subst<R, CC>(Lrow, yw, y);
        float z[CC];
#pragma unroll
        for (int ch = 0; ch < CC; ++ch) z[ch] = y[ch] * dinv;
        float YT[R];
        if (q.top) {
          // E_T[p][i] = A[p, b-R+i] = -lambda w(p-t, p), t = j + R - i (first line)
#pragma unroll
          for (int i = 0; i < R; ++i) {
            const int t = j + R - i;
            YT[i] = (first && t >= 1 && t <= R) ? -wh[(t - 1) % R][(t - 1) % R] : 0.f;
          }
          fwd_subst<R, R>(Lrow, YTw, YT);
#pragma unroll
          for (int i = 0; i < R; ++i) {
            const float yd = YT[i] * dinv;
#pragma unroll
            for (int m = 0; m < R; ++m) KTT[i][m] += yd * YT[m];
#pragma unroll
            for (int ch = 0; ch < CC; ++ch) HT[i][ch] += YT[i] * z[ch];
          }
        } else {
#pragma unroll
          for (int i = 0; i < R; ++i) YT[i] = 0.f;
        }
        float YB[R];
#pragma unroll
        for (int i = 0; i < R; ++i) YB[i] = 0.f;
        if (q.bot && last && j >= n - 2 * R) {
          // E_B[p][i] = A[p, e+i] = -lambda w(p, p+t), t = (n - R - j) + i
#pragma unroll
          for (int i = 0; i < R; ++i) {
            const int t = (n - R - j) + i;
            YB[i] = (t >= 1 && t <= R) ? -wf[(t - 1) % R] : 0.f;
          }
          fwd_subst<R, R>(Lrow, YBw, YB);
#pragma unroll
          for (int i = 0; i < R; ++i) {
            const float yd = YB[i] * dinv;
#pragma unroll
            for (int m = 0; m < R; ++m) {
              KBB[i][m] += yd * YB[m];
              KTB[m][i] += yd * YT[m];
            }
#pragma unroll
            for (int ch = 0; ch < CC; ++ch) HB[i][ch] += YB[i] * z[ch];
          }
        }
        push_factor<R>(Lw, Dw, Lrow, dinv);
        push_vec<R, CC>(yw, y);
        push_vec<R, R>(YTw, YT);
        push_vec<R, R>(YBw, YB);
      } else {
        const int i = j - (n - R);
#pragma unroll
        for (int m = 0; m < R; ++m) {
          if (m == i) DS[i][i] = diag;
          // A[e+i, e+i-t] = -lambda w(e+i-t, e+i), t = i - m
          if (m < i) {
            const int t = i - m;
            DS[i][m] = -wh[(t - 1) % R][(t - 1) % R];
            DS[m][i] = DS[i][m];
          }
        }
#pragma unroll
        for (int ch = 0; ch < CC; ++ch) FS[i][ch] = fl[j][ch];
      }
      push_weights<R>(wh, wf);
    }
#pragma unroll
    for (int j = 0; j < n; ++j) gc[j] = gn[j];
  }

  float* base = a.summ + (long long)c * F::N * a.nsys + sys;
  auto put = [&](int field, float v) { base[(long long)field * a.nsys] = v; };
  if (q.top) {
#pragma unroll
    for (int i = 0; i < R; ++i) {
#pragma unroll
      for (int m = 0; m < R; ++m) {
        put(F::KTT + i * R + m, KTT[i][m]);
        put(F::KTB + i * R + m, KTB[i][m]);
      }
#pragma unroll
      for (int ch = 0; ch < CC; ++ch) put(F::HT + i * CC + ch, HT[i][ch]);
    }
  }
  if (q.bot) {
#pragma unroll
    for (int i = 0; i < R; ++i) {
#pragma unroll
      for (int m = 0; m < R; ++m) put(F::DS + i * R + m, DS[i][m] - KBB[i][m]);
#pragma unroll
      for (int ch = 0; ch < CC; ++ch) put(F::GS + i * CC + ch, FS[i][ch] - HB[i][ch]);
    }
  }
}

// ---------------------------------------------------------------------------
// Small dense helpers for the reduced solve (R x R blocks, registers).

// In-place Cholesky M = L L^T (lower triangle of M overwritten by L; the
// diagonal holds 1/L_ii for cheap solves).
template <int R>
__device__ __forceinline__ void chol_inplace(float (&M)[R][R]) {
#pragma unroll
  for (int j = 0; j < R; ++j) {
    float d = M[j][j];
#pragma unroll
    for (int m = 0; m < j; ++m) d -= M[j][m] * M[j][m];
    const float inv = rsqrtf(d);
    M[j][j] = inv;
#pragma unroll
    for (int i = j + 1; i < R; ++i) {
      float v = M[i][j];
#pragma unroll
      for (int m = 0; m < j; ++m) v -= M[i][m] * M[j][m];
      M[i][j] = v * inv;
    }
  }
}

// X <- L^{-1} X for the Cholesky factor stored by chol_inplace.
template <int R, int K>
__device__ __forceinline__ void lsolve(const float (&Lm)[R][R], float (&X)[R][K]) {
#pragma unroll
  for (int i = 0; i < R; ++i) {
#pragma unroll
    for (int col = 0; col < K; ++col) {
      float v = X[i][col];
#pragma unroll
      for (int m = 0; m < i; ++m) v -= Lm[i][m] * X[m][col];
      X[i][col] = v * Lm[i][i];
    }
  }
}

// X <- L^{-T} X
template <int R, int K>
__device__ __forceinline__ void ltsolve(const float (&Lm)[R][R], float (&X)[R][K]) {
#pragma unroll
  for (int i = R - 1; i >= 0; --i) {
#pragma unroll
    for (int col = 0; col < K; ++col) {
      float v = X[i][col];
#pragma unroll
      for (int m = i + 1; m < R; ++m) v -= Lm[m][i] * X[m][col];
      X[i][col] = v * Lm[i][i];
    }
  }
}

// k_reduced: block Cholesky of the separator system, one thread per subsystem.
// Overwrites DS_c with the factor L_c, GS_c with w_c = L_c^{-1}(...), KTB_c with
// Z_c = L_{c-1}^{-1} (-KTB_c), and writes the separator values to xsep.
template <int R, int CC>
__global__ void __launch_bounds__(128) k_reduced(const PassArgs a) {
  using F = Fields<R, CC>;
  const int sys = blockIdx.x * blockDim.x + threadIdx.x;
  if (sys >= a.nsys || a.P < 2) return;
  const long long ns = a.nsys;
  auto fld = [&](int c, int field) -> float* { return a.summ + ((long long)c * F::N + field) * ns + sys; };

  float Lp[R][R];    // L_{c-1}
  float wp[R][CC];   // w_{c-1}
  for (int c = 0; c <= a.P - 2; ++c) {
    float M[R][R];
    float rhs[R][CC];
#pragma unroll
    for (int i = 0; i < R; ++i) {
#pragma unroll
      for (int m = 0; m < R; ++m) M[i][m] = *fld(c, F::DS + i * R + m) - *fld(c + 1, F::KTT + i * R + m);
#pragma unroll
      for (int ch = 0; ch < CC; ++ch) rhs[i][ch] = *fld(c, F::GS + i * CC + ch) - *fld(c + 1, F::HT + i * CC + ch);
    }
    if (c >= 1) {
      float Z[R][R];
#pragma unroll
      for (int i = 0; i < R; ++i)
#pragma unroll
        for (int m = 0; m < R; ++m) Z[i][m] = -*fld(c, F::KTB + i * R + m);
      lsolve<R, R>(Lp, Z);
#pragma unroll
      for (int i = 0; i < R; ++i) {
#pragma unroll
        for (int m = 0; m < R; ++m) {
          float v = 0.f;
#pragma unroll
          for (int l = 0; l < R; ++l) v += Z[l][i] * Z[l][m];
          M[i][m] -= v;
          *fld(c, F::KTB + i * R + m) = Z[i][m];
        }
#pragma unroll
        for (int ch = 0; ch < CC; ++ch) {
          float v = 0.f;
#pragma unroll
          for (int l = 0; l < R; ++l) v += Z[l][i] * wp[l][ch];
          rhs[i][ch] -= v;
        }
      }
    }
    chol_inplace<R>(M);
    lsolve<R, CC>(M, rhs);
#pragma unroll
    for (int i = 0; i < R; ++i) {
#pragma unroll
      for (int m = 0; m < R; ++m) {
        *fld(c, F::DS + i * R + m) = M[i][m];
        Lp[i][m] = M[i][m];
      }
#pragma unroll
      for (int ch = 0; ch < CC; ++ch) {
        *fld(c, F::GS + i * CC + ch) = rhs[i][ch];
        wp[i][ch] = rhs[i][ch];
      }
    }
  }
  // back substitution
  float x[R][CC];
  for (int c = a.P - 2; c >= 0; --c) {
    float Lc[R][R];
    float v[R][CC];
#pragma unroll
    for (int i = 0; i < R; ++i) {
#pragma unroll
      for (int m = 0; m < R; ++m) Lc[i][m] = *fld(c, F::DS + i * R + m);
#pragma unroll
      for (int ch = 0; ch < CC; ++ch) v[i][ch] = *fld(c, F::GS + i * CC + ch);
    }
    if (c < a.P - 2) {
#pragma unroll
      for (int i = 0; i < R; ++i)
#pragma unroll
        for (int m = 0; m < R; ++m) {
          const float zz = *fld(c + 1, F::KTB + i * R + m);
#pragma unroll
          for (int ch = 0; ch < CC; ++ch) v[i][ch] -= zz * x[m][ch];
        }
    }
    ltsolve<R, CC>(Lc, v);
#pragma unroll
    for (int i = 0; i < R; ++i)
#pragma unroll
      for (int ch = 0; ch < CC; ++ch) {
        x[i][ch] = v[i][ch];
        a.xsep[((long long)c * R * CC + i * CC + ch) * ns + sys] = v[i][ch];
      }
  }
}

// ---------------------------------------------------------------------------
// k_recover: exact interior solve with known separators, write-back and
// averaging.  Block = (32, warps); lane = centre, warp = chunk.
template <int R, int CC>
__global__ void __launch_bounds__(128) k_recover(const PassArgs a) {
  constexpr int n = 2 * R + 1;
  constexpr int NF = R + 1 + CC;   // stored per entry: L[p, p-1..p-R], 1/D, z
  constexpr int OB = 32 - 2 * R;   // outputs per warp
  extern __shared__ float smem[];
  const int lane = threadIdx.x;
  const int c = blockIdx.y * blockDim.y + threadIdx.y;
  if (c >= a.P) return;  // warp-uniform
  const int kc = blockIdx.x * OB - R + lane;  // this lane's centre
  const int sys_raw = kc - R;
  const bool valid = sys_raw >= 0 && sys_raw < a.nsys;
  const int sys = min(max(sys_raw, 0), a.nsys - 1);
  const int k = sys + R;
  const int s = a.L * n;
  const Chunk q = make_chunk<R>(a, c);
  const int mcap = a.h * n;
  float* st = smem + (size_t)threadIdx.y * mcap * NF * 32 + lane;

  // separator values from the reduced solve
  float xT[R][CC], xB[R][CC];
  const long long ns = a.nsys;
#pragma unroll
  for (int i = 0; i < R; ++i)
#pragma unroll
    for (int ch = 0; ch < CC; ++ch) {
      xT[i][ch] = q.top ? a.xsep[((long long)(c - 1) * R * CC + i * CC + ch) * ns + sys] : 0.f;
      xB[i][ch] = q.bot ? a.xsep[((long long)c * R * CC + i * CC + ch) * ns + sys] : 0.f;
    }

  // ---- forward sweep over the interior, storing L row, 1/D and z per entry
  {
    float wh[R][R] = {};
    float Lw[R][R] = {};
    float Dw[R] = {};
    float yw[R][CC] = {};
    float gc[n], gn[n];
    float wf[R];
    if (q.top) {
      load_g_line<R>(a, k, q.line0 - 1, gc);
      load_g_line<R>(a, k, q.line0, gn);
#pragma unroll
      for (int j = 0; j < n; ++j) {
        forward_weights<R>(a, j, (q.line0 - 1) * n + j, s, gc, gn, wf);
        push_weights<R>(wh, wf);
      }
    }
    load_g_line<R>(a, k, q.line0, gc);
    for (int line = q.line0; line < q.line1; ++line) {
      load_g_line<R>(a, k, line + 1, gn);
      float fl[n][CC];
      load_f_line<R, CC>(a, k, line, fl);
      const bool first = line == q.line0;
      const bool last = line == q.line1 - 1;
#pragma unroll
      for (int j = 0; j < n; ++j) {
        const int p = line * n + j;
        forward_weights<R>(a, j, p, s, gc, gn, wf);
        const bool sep = last && q.bot && (j >= n - R);
        if (!sep) {
          float diag = 1.f;
#pragma unroll
          for (int t = 0; t < R; ++t) diag += wf[t] + wh[t][t];
          float Lrow[R];
          const float dinv = ldl_row<R>(diag, wh, Lw, Dw, first ? j : R, Lrow);
          float y[CC];
#pragma unroll
          for (int ch = 0; ch < CC; ++ch) y[ch] = fl[j][ch];
          if (first && q.top) {
            // + lambda w(p-t, p) x(b-R+i) for separator entries above, i = j + R - t
#pragma unroll
            for (int t = j + 1; t <= R; ++t)
#pragma unroll
              for (int ch = 0; ch < CC; ++ch) y[ch] += wh[t - 1][t - 1] * xT[j + R - t][ch];
          }
          if (last && q.bot) {
            // + lambda w(p, p+t) x(e+i) for separator entries below, i = j + t - (n - R)
#pragma unroll
            for (int t = 1; t <= R; ++t) {
              const int i = j + t - (n - R);
              if (i >= 0 && i < R) {
#pragma unroll
                for (int ch = 0; ch < CC; ++ch) y[ch] += wf[t - 1] * xB[i][ch];
              }
            }
          }
          fwd_subst<R, CC>(Lrow, yw, y);
          float* slot = st + (size_t)(p - q.b) * NF * 32;
#pragma unroll
          for (int t = 0; t < R; ++t) slot[t * 32] = Lrow[t];
          slot[R * 32] = dinv;
#pragma unroll
          for (int ch = 0; ch < CC; ++ch) slot[(R + 1 + ch) * 32] = y[ch] * dinv;
          push_factor<R>(Lw, Dw, Lrow, dinv);
          push_vec<R, CC>(yw, y);
        }
        push_weights<R>(wh, wf);
      }
#pragma unroll
      for (int j = 0; j < n; ++j) gc[j] = gn[j];
    }
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
  for (int line = q.line1 - 1; line >= q.line0; --line) {
    const bool last = line == q.line1 - 1;
    float xl[n][CC];
#pragma unroll
    for (int jj = n - 1; jj >= 0; --jj) {
      const int p = line * n + jj;
      if (last && q.bot && jj >= n - R) {
#pragma unroll
        for (int ch = 0; ch < CC; ++ch) xl[jj][ch] = xB[jj - (n - R)][ch];
        continue;
      }
      const float* slot = st + (size_t)(p - q.b) * NF * 32;
      float Lrow[R];
#pragma unroll
      for (int t = 0; t < R; ++t) Lrow[t] = slot[t * 32];
      float x[CC];
#pragma unroll
      for (int ch = 0; ch < CC; ++ch) x[ch] = slot[(R + 1 + ch) * 32];
#pragma unroll
      for (int t = 1; t <= R; ++t)
#pragma unroll
        for (int ch = 0; ch < CC; ++ch) x[ch] -= Lb[t - 1][t - 1] * xw[t - 1][ch];
#pragma unroll
      for (int u = R - 1; u > 0; --u)
#pragma unroll
        for (int t = 0; t < R; ++t) Lb[u][t] = Lb[u - 1][t];
#pragma unroll
      for (int t = 0; t < R; ++t) Lb[0][t] = Lrow[t];
      push_vec<R, CC>(xw, x);
#pragma unroll
      for (int ch = 0; ch < CC; ++ch) xl[jj][ch] = x[ch];
    }
    // inverse construction + averaging: value at across-offset kc - R + e
    const bool rev = line & 1;
#pragma unroll
    for (int ch = 0; ch < CC; ++ch) {
      float voff[n];
#pragma unroll
      for (int e2 = 0; e2 < n; ++e2) voff[e2] = valid ? (rev ? xl[n - 1 - e2][ch] : xl[e2][ch]) : 0.f;
      float sum = voff[R];
#pragma unroll
      for (int d = 1; d <= R; ++d) {
        sum += __shfl_down_sync(0xffffffffu, voff[R - d], d);  // from centre kc + d
        sum += __shfl_up_sync(0xffffffffu, voff[R + d], d);    // from centre kc - d
      }
      if (writer) st_px(a.out, pix_index(a, line, o) + ch * a.plane, a.out_dt, sum * inv_cnt);
    }
  }
}

}  // namespace sgwls
