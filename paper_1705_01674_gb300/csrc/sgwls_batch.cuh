// sgwls_batch.cuh -- one launch per kernel per pass for many images of
// uneven sizes (a flat queue of blocks over all images).
//
// The per-image descriptors travel in the kernel parameters (no upload, so
// a batched call can be captured in a CUDA graph).  Each block finds its
// image by binary search over the per-image block prefixes, assembles that
// image's argument block in shared memory and runs the same kernel body as
// the single-image launch.
#pragma once

#include "sgwls_pass.cuh"

namespace sgwls {

constexpr int kBatchMax = 64;   // images per batched launch

struct ImgDesc {
  const void* in;
  const void* in2;   // backward: the v-bar planes (null: in)
  const void* g;
  void* out;
  float* grad_g;     // backward: this image's dLoss/dG and dLoss/dlambda
  float* grad_lam;
  float* summ;
  float* xsep;
  float* mdata;
  int* band_cnt;
  float* fac;   // kept chunk factors (batches whose passes keep them)
  float* psi;
  long long plane;
  int H, W, L, D, nsys, sstride, h, P, ngroups;
  float lam;
  int b0[3];    // first block of this image in the summary / (unused) / recover or backsub launch
  int nbx[3];   // blocks along the across direction in each launch
};

struct BatchArgs {
  PassArgs base;   // fields shared by all images (direction, types, weight constants)
  int nimg;
  ImgDesc img[kBatchMax];
};

__device__ __forceinline__ int find_image(const BatchArgs& ba, int kind, int block) {
  int lo = 0, hi = ba.nimg - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (ba.img[mid].b0[kind] <= block) lo = mid; else hi = mid - 1;
  }
  return lo;
}

// Copies the shared argument block into shared memory and applies image i's
// fields (lambda scales the spatial table).
__device__ __forceinline__ void build_args(const BatchArgs& ba, int i, PassArgs& sa) {
  const int tid = threadIdx.y * blockDim.x + threadIdx.x;
  const int nthreads = blockDim.x * blockDim.y;
  const unsigned* src = reinterpret_cast<const unsigned*>(&ba.base);
  unsigned* dst = reinterpret_cast<unsigned*>(&sa);
  constexpr int nw = sizeof(PassArgs) / sizeof(unsigned);
  for (int w = tid; w < nw; w += nthreads) dst[w] = src[w];
  __syncthreads();
  const ImgDesc& d = ba.img[i];
  constexpr int nsp = (2 * kRMax + 1) * kRMax;
  for (int k = tid; k < nsp; k += nthreads) sa.sp[k] = d.lam * ba.base.sp0[k];
  if (tid == 0) {
    sa.in = d.in;
    sa.in2 = d.in2 ? d.in2 : d.in;
    sa.g = d.g;
    sa.grad_g = d.grad_g;
    sa.grad_lam = d.grad_lam;
    sa.out = d.out;
    sa.summ = d.summ;
    sa.xsep = d.xsep;
    sa.mdata = d.mdata;
    sa.band_cnt = d.band_cnt;
    sa.fac = d.fac;
    sa.psi = d.psi;
    sa.plane = d.plane;
    sa.H = d.H;
    sa.W = d.W;
    sa.L = d.L;
    sa.D = d.D;
    sa.nsys = d.nsys;
    sa.nreg = d.nsys;
    sa.sstride = d.sstride;
    sa.h = d.h;
    sa.P = d.P;
    sa.ngroups = d.ngroups;
    sa.lam = d.lam;
  }
  __syncthreads();
}

template <int R, int CC, int SM>
__global__ void __launch_bounds__(256) k_summary_b(const __grid_constant__ BatchArgs ba) {
  extern __shared__ __align__(128) float smem[];
  __shared__ PassArgs sa;
  const int i = find_image(ba, 0, blockIdx.x);
  const int local = blockIdx.x - ba.img[i].b0[0];
  const int by = local / ba.img[i].nbx[0];
  build_args(ba, i, sa);
  body_summary<R, CC, SM>(sa, local - by * ba.img[i].nbx[0], by, smem);
}

// BWD: the adjoint pass of every image (u from the checkpoint planes `in`,
// v from the v-bar planes `in2`, gradients to the image's own buffers).
template <int R, int CC, bool BWD = false>
__global__ void __launch_bounds__(256) k_recover_b(const __grid_constant__ BatchArgs ba) {
  extern __shared__ __align__(128) float smem[];
  __shared__ PassArgs sa;
  const int i = find_image(ba, 2, blockIdx.x);
  const int local = blockIdx.x - ba.img[i].b0[2];
  const int by = local / ba.img[i].nbx[2];
  build_args(ba, i, sa);
  body_recover<R, CC, BWD>(sa, local - by * ba.img[i].nbx[2], by, smem);
}

// MODE 0: forward back-substitution; 3: the adjoint's (CC = u and v planes)
template <int R, int CC, int MODE = 0>
__global__ void __launch_bounds__(256) k_backsub_b(const __grid_constant__ BatchArgs ba) {
  extern __shared__ __align__(128) float smem[];
  __shared__ PassArgs sa;
  const int i = find_image(ba, 2, blockIdx.x);
  const int local = blockIdx.x - ba.img[i].b0[2];
  const int by = local / ba.img[i].nbx[2];
  build_args(ba, i, sa);
  body_backsub<R, CC, MODE>(sa, local - by * ba.img[i].nbx[2], by, smem);
}

}  // namespace sgwls
