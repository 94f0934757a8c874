// raylut.cpp — ray-mask lookup tables (Sec. 3.1.1).
//
// Definition (sweep test): in cell units, cell v is in the mask of
// (beg = b, end = e) iff the box [b, b+1]^3 moved by t*(e - b), t in [0,1],
// meets the interior of [v, v+1]^3, i.e. some t in [0,1] has
// |b_k + t (e_k - b_k) - v_k| < 1 on all three axes.
//
// Construction here: each axis condition holds on an interval of t, and by
// Helly's theorem on the line three intervals share a point iff every pair
// does.  So the 3-D mask is the AND of three 2-D "pair" tables (x,y), (y,z),
// (x,z), all one table P(b_a, b_b, e_a, e_b) of R^2 bits.  P is filled by an
// exact scan t = k/M with M = 2(R-1)^2 + 1 in integers: a non-empty feasible
// set of t contains 0 or 1, or an open interval between fractions with
// denominators <= R-1, which is longer than 1/M, so the scan finds it.
#include <cstdlib>
#include <cstring>
#include <mutex>

#include "internal.h"

namespace sc {

void raylut_pair2d(int R, std::vector<uint64_t>& out) {
  const int R2 = R * R;
  out.assign((size_t)R2 * R2, 0ULL);
  const long M = 2L * (R - 1) * (R - 1) + 1;
  for (int ba = 0; ba < R; ++ba)
    for (int bb = 0; bb < R; ++bb)
      for (int ea = 0; ea < R; ++ea)
        for (int eb = 0; eb < R; ++eb) {
          uint64_t m = 0;
          for (int va = 0; va < R; ++va)
            for (int vb = 0; vb < R; ++vb) {
              for (long k = 0; k <= M; ++k) {
                long qa = M * (ba - va) + k * (ea - ba);
                long qb = M * (bb - vb) + k * (eb - bb);
                if (std::labs(qa) < M && std::labs(qb) < M) {
                  m |= 1ULL << (va + R * vb);
                  break;
                }
              }
            }
          out[(((size_t)ba * R + bb) * R + ea) * R + eb] = m;
        }
}

void raylut_full(int R, uint32_t* out) {
  std::vector<uint64_t> P;
  raylut_pair2d(R, P);
  const int R3 = R * R * R, W = mask_words(R);
  auto pidx = [R](int ba, int bb, int ea, int eb) {
    return (((size_t)ba * R + bb) * R + ea) * R + eb;
  };
  std::memset(out, 0, sizeof(uint32_t) * (size_t)R3 * R3 * W);
  for (int beg = 0; beg < R3; ++beg) {
    const int bx = beg % R, by = (beg / R) % R, bz = beg / (R * R);
    for (int end = 0; end < R3; ++end) {
      const int ex = end % R, ey = (end / R) % R, ez = end / (R * R);
      const uint64_t pxy = P[pidx(bx, by, ex, ey)];
      const uint64_t pyz = P[pidx(by, bz, ey, ez)];
      const uint64_t pxz = P[pidx(bx, bz, ex, ez)];
      uint32_t* m = out + ((size_t)beg * R3 + end) * W;
      for (int z = 0; z < R; ++z)
        for (int y = 0; y < R; ++y)
          for (int x = 0; x < R; ++x)
            if (((pxy >> (x + R * y)) & 1) && ((pyz >> (y + R * z)) & 1) &&
                ((pxz >> (x + R * z)) & 1)) {
              int bit = x + R * y + R * R * z;
              m[bit >> 5] |= 1u << (bit & 31);
            }
    }
  }
}

}  // namespace sc
