// Checks the FP32 filter of the SAT triangle/box test (mask_math.h) against
// the FP64 test: wherever the filter decides, it must give the FP64 answer.
// Cases: random triangles and boxes at several scales and offsets, and
// adversarial ones whose triangle planes, edges or vertices lie on, or a
// few ulps off, the box faces.  Prints the number of cases, the number the
// filter left undecided, the number of disagreements, and the cases and
// undecided ones among the random (non-adversarial) pairs.
#include <cstdint>
#include <cstdio>
#include <cmath>

#include "host/mask_math.h"

namespace {
uint64_t state = 0x9E3779B97F4A7C15ull;
uint64_t next_u64() {  // splitmix64
  uint64_t z = (state += 0x9E3779B97F4A7C15ull);
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}
double uni() { return (double)(next_u64() >> 11) * (1.0 / 9007199254740992.0); }
}  // namespace

int main() {
  long cases = 0, open = 0, wrong = 0, rnd = 0, rnd_open = 0;
  const double scales[4] = {1e-4, 1e-2, 1.0, 30.0};
  for (int rep = 0; rep < 400000; ++rep) {
    const double s = scales[rep % 4];
    const double off = (rep % 3) * 1.7;
    double bmin[3], bmax[3];
    for (int k = 0; k < 3; ++k) {
      bmin[k] = off + s * uni();
      bmax[k] = bmin[k] + s * (0.05 + uni());
    }
    float t9[9];
    const int kind = (int)(next_u64() % 4);
    for (int i = 0; i < 3; ++i)
      for (int k = 0; k < 3; ++k) {
        double x = bmin[k] + (bmax[k] - bmin[k]) * (2.0 * uni() - 0.5);
        if (kind == 1 && k == (rep % 3)) x = (i == 0 || uni() < 0.5) ? bmin[k] : bmax[k];
        t9[3 * i + k] = (float)x;
      }
    if (kind == 2) {  // a vertex on a box corner, nudged by a few ulps
      for (int k = 0; k < 3; ++k) {
        float f = (float)((next_u64() & 1) ? bmin[k] : bmax[k]);
        const int n = (int)(next_u64() % 5) - 2;
        for (int j = 0; j < (n < 0 ? -n : n); ++j) f = nextafterf(f, n < 0 ? -INFINITY : INFINITY);
        t9[k] = f;
      }
    }
    if (kind == 3) {  // a triangle in the plane of a face
      const int k = rep % 3;
      const float f = (float)((next_u64() & 1) ? bmin[k] : bmax[k]);
      for (int i = 0; i < 3; ++i) t9[3 * i + k] = f;
    }
    double v[9];
    for (int i = 0; i < 9; ++i) v[i] = (double)t9[i];
    const int f = sc::mm::tri_box_overlap_f32(v, bmin, bmax);
    const int d = sc::mm::tri_box_overlap(v, bmin, bmax) ? 1 : 0;
    ++cases;
    if (kind == 0) ++rnd;
    if (f < 0) {
      ++open;
      if (kind == 0) ++rnd_open;
    } else if (f != d) {
      ++wrong;
    }
  }
  printf("%ld %ld %ld %ld %ld\n", cases, open, wrong, rnd, rnd_open);
  return wrong != 0;
}
