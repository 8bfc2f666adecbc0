// sgwls_line.cuh -- line relaxation of the 2D WLS model (an opt-in variant,
// not the paper's SG-WLS subsystem).
//
// Each pass solves one banded system per image line (rows for the row
// direction, columns for the column direction): for pixel p of the line,
//   (1 + lambda sum_{q in N(p)} w_pq) u_p - lambda sum_{q in N(p) on the line} w_pq u_q
//       = F_p + lambda sum_{q in N(p) off the line} w_pq U_q,
// N(p) the (2r+1) x (2r+1) square neighbourhood (Eq. 4's convention), w the
// Eq. 2 weight, F the filter's input, U the estimate the pass starts from: a
// block-Jacobi step on the dense 2D WLS system of Eqs. 1-4.  The line
// matrix is symmetric, banded (half-bandwidth r) and strictly diagonally
// dominant, so an FP32 LDL^T without pivoting is stable.
//
// k_line_pass: one thread per line.  The forward sweep forms every entry's
// weights from the guidance, its right-hand side (F plus the off-line
// neighbours' estimates) and its LDL^T row, and keeps L[e, e-1..e-r] and
// z = D^-1 L^-1 b in a scratch array laid out [entry][field][line] (lines
// fastest: coalesced across the threads of a warp); the backward sweep
// reads them back in reverse order and writes the solution.
#pragma once

#include "sgwls_common.cuh"

namespace sgwls {

constexpr int kLineRMax = 4;   // radii of the line-relaxation kernels

struct LineArgs {
  const float* f;      // F: CC planes (the data term)
  const float* uin;    // U: CC planes (the estimate the pass starts from)
  const float* g;      // guidance plane
  float* uout;         // CC output planes
  float* scratch;      // [n][R + CC][nlines]
  long long plane;     // H * W
  int H, W;
  int dir;             // 0: lines are columns (column direction); 1: lines are rows
  int weight;          // 0 exp, 1 frac
  float range_k;       // exp: -log2(e) / (2 sigma_r^2); frac: alpha_r
  float eps;
  // lambda * spatial factor of the neighbour (dy, dx):
  // wsp[(dy + r) * (2r + 1) + dx + r]
  float wsp[(2 * kLineRMax + 1) * (2 * kLineRMax + 1)];
};

template <int R, int CC>
__global__ void __launch_bounds__(128) k_line_pass(const __grid_constant__ LineArgs a) {
  constexpr int NF = R + CC;
  constexpr int S = 2 * R + 1;
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  const int nlines = a.dir == 1 ? a.H : a.W;
  const int n = a.dir == 1 ? a.W : a.H;
  griddep_wait();
  griddep_launch();
  if (k >= nlines) return;
  const long long W = a.W;
  float* const sc = a.scratch + k;
  const size_t fstride = (size_t)nlines;   // between fields of an entry
  auto at = [&](int e, int f) -> float* { return sc + ((size_t)e * NF + f) * fstride; };

  float wa[R][R] = {};    // wa[u-1][t-1] = lambda w(e-u, e-u+t): in-line weights ahead of entry e-u
  float Lw[R][R] = {};    // Lw[u-1][v-1] = L[e-u, e-u-v]
  float Di[R] = {};       // Di[u-1] = 1 / D[e-u]
  float yw[R][CC] = {};   // yw[u-1][c] = y[e-u] (forward-substituted right-hand side)
  for (int e = 0; e < n; ++e) {
    const int y = a.dir == 1 ? k : e, x = a.dir == 1 ? e : k;
    const long long pp = (long long)y * W + x;
    const float gp = __ldg(a.g + pp);
    float diag = 1.f;
    float b[CC];
#pragma unroll
    for (int c = 0; c < CC; ++c) b[c] = __ldg(a.f + c * a.plane + pp);
    float ahead[R];
#pragma unroll
    for (int t = 0; t < R; ++t) ahead[t] = 0.f;
#pragma unroll
    for (int dy = -R; dy <= R; ++dy) {
#pragma unroll
      for (int dx = -R; dx <= R; ++dx) {
        if (dy == 0 && dx == 0) continue;
        const int qy = y + dy, qx = x + dx;
        if (qy < 0 || qy >= a.H || qx < 0 || qx >= a.W) continue;
        const long long qq = (long long)qy * W + qx;
        const float dg = gp - __ldg(a.g + qq);
        const float rf = a.weight == 0 ? fast_ex2(dg * dg * a.range_k)
                                       : 1.0f / (powf(fabsf(dg), a.range_k) + a.eps);
        const float w = a.wsp[(dy + R) * S + dx + R] * rf;
        diag += w;
        const int along = a.dir == 1 ? dx : dy, across = a.dir == 1 ? dy : dx;
        if (across != 0) {
#pragma unroll
          for (int c = 0; c < CC; ++c) b[c] += w * __ldg(a.uin + c * a.plane + qq);
        } else if (along > 0) {
#pragma unroll
          for (int t = 1; t <= R; ++t)
            if (t == along) ahead[t - 1] = w;
        }
      }
    }
    // LDL^T row of entry e: A[e, e-t] = -lambda w(e-t, e) = -wa[t-1][t-1]
    float Wt[R], Lrow[R];
#pragma unroll
    for (int t = R; t >= 1; --t) {
      float acc = -wa[t - 1][t - 1];
#pragma unroll
      for (int v = t + 1; v <= R; ++v) acc -= Wt[v - 1] * Lw[t - 1][v - t - 1];
      Wt[t - 1] = acc;
      Lrow[t - 1] = acc * Di[t - 1];   // 0 before the line's start (Di = 0 there)
    }
    float D = diag;
#pragma unroll
    for (int t = 0; t < R; ++t) D -= Wt[t] * Lrow[t];
    const float dinv = 1.0f / D;
    float yv[CC];
#pragma unroll
    for (int c = 0; c < CC; ++c) {
      float v = b[c];
#pragma unroll
      for (int t = 0; t < R; ++t) v -= Lrow[t] * yw[t][c];
      yv[c] = v;
    }
#pragma unroll
    for (int t = 0; t < R; ++t) *at(e, t) = Lrow[t];
#pragma unroll
    for (int c = 0; c < CC; ++c) *at(e, R + c) = yv[c] * dinv;
    // shift the windows by one entry
#pragma unroll
    for (int u = R - 1; u > 0; --u) {
#pragma unroll
      for (int v = 0; v < R; ++v) {
        wa[u][v] = wa[u - 1][v];
        Lw[u][v] = Lw[u - 1][v];
      }
      Di[u] = Di[u - 1];
#pragma unroll
      for (int c = 0; c < CC; ++c) yw[u][c] = yw[u - 1][c];
    }
#pragma unroll
    for (int v = 0; v < R; ++v) {
      wa[0][v] = ahead[v];
      Lw[0][v] = Lrow[v];
    }
    Di[0] = dinv;
#pragma unroll
    for (int c = 0; c < CC; ++c) yw[0][c] = yv[c];
  }
  // back substitution: x[e] = z[e] - sum_t L[e+t, e] x[e+t]
  float Lb[R][R] = {};    // Lb[u-1][t-1] = L[e+u, e+u-t]
  float xw[R][CC] = {};   // x[e+u]
  for (int e = n - 1; e >= 0; --e) {
    float Lrow[R], xv[CC];
#pragma unroll
    for (int t = 0; t < R; ++t) Lrow[t] = *at(e, t);
#pragma unroll
    for (int c = 0; c < CC; ++c) {
      float v = *at(e, R + c);
#pragma unroll
      for (int t = 1; t <= R; ++t) v -= Lb[t - 1][t - 1] * xw[t - 1][c];
      xv[c] = v;
    }
    const int y = a.dir == 1 ? k : e, x = a.dir == 1 ? e : k;
    const long long pp = (long long)y * W + x;
#pragma unroll
    for (int c = 0; c < CC; ++c) a.uout[c * a.plane + pp] = xv[c];
#pragma unroll
    for (int u = R - 1; u > 0; --u) {
#pragma unroll
      for (int t = 0; t < R; ++t) Lb[u][t] = Lb[u - 1][t];
#pragma unroll
      for (int c = 0; c < CC; ++c) xw[u][c] = xw[u - 1][c];
    }
#pragma unroll
    for (int t = 0; t < R; ++t) Lb[0][t] = Lrow[t];
#pragma unroll
    for (int c = 0; c < CC; ++c) xw[0][c] = xv[c];
  }
}

}  // namespace sgwls
