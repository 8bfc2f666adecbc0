// Host check of the work-queue order of the queue-scheduled pass
// (paper_1705_01674_gb300/csrc/sgwls_sched.h), built and run by
// tests/test_sched_host.py.  For every shape: every item is decoded exactly
// once; every back-substitution item comes after every summary item of the
// bands its subsystems lie in; with a ring of S band slots every summary
// item comes after every reader of the band whose slot it reuses; the
// reader counts match the items that read each band.
#include <cstdio>
#include <vector>

#include "../paper_1705_01674_gb300/csrc/sgwls_sched.h"

static int fail(const char* what, int D, int r, int NG, int LA, int S, int i) {
  std::printf("FAIL %s D=%d r=%d NG=%d LA=%d S=%d item=%d\n", what, D, r, NG, LA, S, i);
  return 1;
}

static int check(int D, int r, int NG, int LA, int S) {
  const int nsys = D - 2 * r;
  sgwls::QueueSched q;
  q.nb = (nsys + 31) / 32;
  q.OB = 32 - 2 * r;
  q.nbx = (D + q.OB - 1) / q.OB;
  q.NG = NG;
  q.LA = LA;
  q.r = r;
  const int n = q.total();
  std::vector<int> pos_s(q.nb * NG, -1), pos_b(q.nbx * NG, -1);
  for (int i = 0; i < n; ++i) {
    int band, bx, grp;
    if (q.decode(i, &band, &bx, &grp)) {
      if (band < 0 || band >= q.nb || grp < 0 || grp >= NG || pos_s[band * NG + grp] >= 0)
        return fail("summary decode", D, r, NG, LA, S, i);
      pos_s[band * NG + grp] = i;
    } else {
      if (bx < 0 || bx >= q.nbx || grp < 0 || grp >= NG || pos_b[bx * NG + grp] >= 0)
        return fail("backsub decode", D, r, NG, LA, S, i);
      pos_b[bx * NG + grp] = i;
    }
  }
  std::vector<int> rd(q.nb, 0);
  for (int x = 0; x < q.nbx; ++x) {
    // bands of the subsystems the block reads (clamped to the valid ones)
    int lo = 1 << 30, hi = -1;
    for (int lane = 0; lane < 32; ++lane) {
      int s = x * q.OB - 2 * r + lane;
      s = s < 0 ? 0 : (s >= nsys ? nsys - 1 : s);
      lo = lo < s / 32 ? lo : s / 32;
      hi = hi > s / 32 ? hi : s / 32;
    }
    if (q.band_lo(x) != lo || q.band_hi(x) != hi) return fail("band range", D, r, NG, LA, S, x);
    for (int g = 0; g < NG; ++g) {
      const int pb = pos_b[x * NG + g];
      for (int b = lo; b <= hi; ++b)
        for (int g2 = 0; g2 < NG; ++g2)
          if (pos_s[b * NG + g2] >= pb) return fail("backsub before its summary", D, r, NG, LA, S, pb);
    }
    for (int b = lo; b <= hi; ++b) rd[b] += NG;
  }
  for (int b = 0; b < q.nb; ++b)
    if (rd[b] != NG * q.readers(b)) return fail("reader count", D, r, NG, LA, S, b);
  if (S > 0) {
    for (int b = S; b < q.nb; ++b)
      for (int g = 0; g < NG; ++g) {
        const int ps = pos_s[b * NG + g];
        for (int x = 0; x < q.nbx; ++x)
          if (q.band_lo(x) <= b - S && b - S <= q.band_hi(x))
            for (int g2 = 0; g2 < NG; ++g2)
              if (pos_b[x * NG + g2] >= ps) return fail("slot reused before its readers", D, r, NG, LA, S, ps);
      }
  }
  return 0;
}

int main() {
  int bad = 0, n = 0;
  const int Ds[] = {3, 5, 17, 31, 32, 33, 37, 63, 64, 65, 100, 127, 128, 129, 200, 511, 768, 1024, 1080, 1920, 4099};
  for (int D : Ds)
    for (int r = 1; r <= 8; ++r) {
      if (D < 2 * r + 1) continue;
      for (int NG : {1, 2, 3, 12})
        for (int LA : {0, 1, 2, 3})
          for (int S : {0, LA + 2, LA + 3, 7, 11}) {
            bad += check(D, r, NG, LA, S);
            ++n;
          }
    }
  std::printf("%s %d shapes\n", bad ? "FAILED" : "ok", n);
  return bad ? 1 : 0;
}
