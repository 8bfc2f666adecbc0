// sgwls_sched.h -- work-queue order of the queue-scheduled pass (k_pass_q).
//
// One forward pass (sliding step 1, kept chunk factors) has two kinds of
// work item, each one block of G chunk-warps:
//   summary item  (band b, group g): the forward sweeps of chunk group g of
//                 the 32 subsystems of band b (centres 32 b .. 32 b + 31);
//                 the band's last summary item also solves its reduced
//                 system, after which the band is "done";
//   back-substitution item (block x, group g): the back substitution and
//                 averaging of output columns x OB .. x OB + OB - 1
//                 (OB = 32 - 2r), which reads the factors of subsystems
//                 x OB - 2r .. x OB - 2r + 31: bands lo(x) and hi(x)
//                 (at most two; both must be done first).
// Items are taken from an atomic counter in "rounds": round k holds the
// summary items of band k (k < nb) followed by the back-substitution items
// of the blocks whose last band is k - LA (all remaining blocks in the last
// round).  A back-substitution item therefore comes after every summary
// item it needs, with LA bands of slack.  When the factor store is a ring
// of S band slots, the summary items of band b reuse the slot of band b - S
// only after all readers of band b - S finished; those readers sit in
// rounds <= b - S + 1 + LA < b for S >= LA + 2.  Every wait is thus on an
// item taken earlier by a block that is already running, and blocks take a
// new item only after finishing the last one: no wait can be circular.
#pragma once

#ifdef __CUDACC__
#define SGWLS_HD __host__ __device__ __forceinline__
#else
#define SGWLS_HD inline
#endif

namespace sgwls {

struct QueueSched {
  int nb;    // bands of 32 subsystems (summary bands)
  int nbx;   // back-substitution blocks (output columns / OB)
  int NG;    // chunk groups per subsystem
  int LA;    // rounds between a band's summary items and the blocks needing it
  int r;     // radius
  int OB;    // output columns per back-substitution block: 32 - 2r

  SGWLS_HD static int imin(int a, int b) { return a < b ? a : b; }
  SGWLS_HD static int imax(int a, int b) { return a > b ? a : b; }

  // bands read by back-substitution block x
  SGWLS_HD int band_lo(int x) const { return imax(x * OB - 2 * r, 0) >> 5; }
  SGWLS_HD int band_hi(int x) const { return imin(nb - 1, (x * OB - 2 * r + 31) >> 5); }
  // number of blocks x whose last band is below k
  SGWLS_HD int blocks_below(int k) const {
    if (k <= 0) return 0;
    if (k >= nb) return nbx;
    return imin(nbx, (32 * k - 31 + 2 * r + OB - 1) / OB);
  }
  // number of blocks that read band b
  SGWLS_HD int readers(int b) const {
    return imin(nbx, (32 * b + 31 + 2 * r) / OB + 1) - blocks_below(b);
  }
  SGWLS_HD int rounds() const { return nb + LA; }
  SGWLS_HD int total() const { return NG * (nb + nbx); }
  // items before round k
  SGWLS_HD int before(int k) const { return NG * (imin(k, nb) + blocks_below(imin(imax(k - LA, 0), nb))); }

  // Decodes item i (0 <= i < total()): summary items give *band, back-
  // substitution items *bx; *grp is the chunk group.  Returns true for a
  // summary item.
  SGWLS_HD bool decode(int i, int* band, int* bx, int* grp) const {
    int lo = 0, hi = rounds() - 1;
    while (lo < hi) {
      const int mid = (lo + hi + 1) >> 1;
      if (before(mid) <= i) lo = mid; else hi = mid - 1;
    }
    int j = i - before(lo);
    if (lo < nb) {
      if (j < NG) {
        *band = lo;
        *bx = -1;
        *grp = j;
        return true;
      }
      j -= NG;
    }
    *band = -1;
    *bx = blocks_below(imin(imax(lo - LA, 0), nb)) + j / NG;
    *grp = j % NG;
    return false;
  }
};

}  // namespace sgwls
