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

// The table at R_ray = 2R (Sec. 4.2): begin and end cells on the 2R grid
// (x + 2R y + 4R^2 z), one R^3-bit row per pair, a mask cell set iff the
// sweep on the 2R grid sets one of its eight sub-cells.  Same construction as
// raylut_full one level finer: per axis pair a 2-D table of 2R rows of 2R
// bits (exact scan of t), the Helly product row by row, and each 2R row
// folded to R bits (bit i kept iff sub-bit 2i or 2i+1 is set).
void raylut2r_full(int R, uint32_t* out) {
  const int R2 = 2 * R, W = mask_words(R);
  if (R2 > 16) fail(SC_ERR_UNSUPPORTED, "R_ray = 2R table for R = %d", R);
  const int64_t R23 = (int64_t)R2 * R2 * R2;
  const long M = 2L * (R2 - 1) * (R2 - 1) + 1;
  // Q[((ba*R2 + bb)*R2 + ea)*R2 + eb][vb]: bits va
  std::vector<uint16_t> Q((size_t)R2 * R2 * R2 * R2 * R2, 0);
  parallel_for((int64_t)R2 * R2, resolve_threads(0), 1, [&](int64_t ab) {
    const int ba = (int)(ab / R2), bb = (int)(ab % R2);
    for (int ea = 0; ea < R2; ++ea)
      for (int eb = 0; eb < R2; ++eb) {
        uint16_t* q = &Q[((((size_t)ba * R2 + bb) * R2 + ea) * R2 + eb) * R2];
        for (int vb = 0; vb < R2; ++vb)
          for (int va = 0; va < R2; ++va)
            for (long k = 0; k <= M; ++k) {
              const long qa = M * (ba - va) + k * (ea - ba);
              const long qb = M * (bb - vb) + k * (eb - bb);
              if (std::labs(qa) < M && std::labs(qb) < M) {
                q[vb] |= (uint16_t)(1u << va);
                break;
              }
            }
      }
  });
  auto rows = [&](int ba, int bb, int ea, int eb) {
    return &Q[((((size_t)ba * R2 + bb) * R2 + ea) * R2 + eb) * R2];
  };
  auto fold = [R](uint32_t x) {
    uint32_t f = 0;
    for (int i = 0; i < R; ++i)
      if ((x >> (2 * i)) & 3u) f |= 1u << i;
    return f;
  };
  parallel_for(R23 * R23, resolve_threads(0), 4096, [&](int64_t row) {
    const int beg = (int)(row / R23), end = (int)(row % R23);
    const int bx = beg % R2, by = (beg / R2) % R2, bz = beg / (R2 * R2);
    const int ex = end % R2, ey = (end / R2) % R2, ez = end / (R2 * R2);
    const uint16_t* xy = rows(bx, by, ex, ey);  // [y] -> x bits
    const uint16_t* yz = rows(by, bz, ey, ez);  // [z] -> y bits
    const uint16_t* xz = rows(bx, bz, ex, ez);  // [z] -> x bits
    uint32_t* m = out + (size_t)row * W;
    std::memset(m, 0, sizeof(uint32_t) * W);
    for (int z = 0; z < R2; ++z)
      for (int y = 0; y < R2; ++y) {
        if (!((yz[z] >> y) & 1u)) continue;
        const uint32_t xs = fold((uint32_t)(xy[y] & xz[z]));
        for (int x = 0; x < R; ++x)
          if ((xs >> x) & 1u) {
            const int bit = x + R * (y / 2) + R * R * (z / 2);
            m[bit >> 5] |= 1u << (bit & 31);
          }
      }
  });
}

}  // namespace sc
