// Checks the FP32 filter of the SAT triangle/box test (mask_math.h) against
// the FP64 test: wherever the filter decides, it must give the FP64 answer.
// Cases: random triangles and boxes at several scales and offsets, and
// adversarial ones whose triangle planes, edges or vertices lie on, or a
// few ulps off, the box faces.  Prints the number of cases, the number the
// filter left undecided, the number of disagreements, and the cases and
// undecided ones among the random (non-adversarial) pairs.  Given a file of
// triangles, checks the pairs a mask build of that scene meets instead.
#include <cstdint>
#include <cstdio>
#include <cstdlib>
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

// Realistic pairs: triangles (float32[n][9], binary, from argv[1]) grouped
// four at a time into a slot whose box is their bounding box, as a leaf of
// the builder; each triangle against every candidate voxel of that slot's
// R = 6 grid (the builder's own Grid) dilated by 2^-16 of the scene's
// largest extent.  Prints pairs, undecided and disagreements.
static int check_file(const char* path) {
  FILE* f = fopen(path, "rb");
  if (!f) return 2;
  fseek(f, 0, SEEK_END);
  const long bytes = ftell(f);
  fseek(f, 0, SEEK_SET);
  const long n = bytes / 36;
  float* t = (float*)malloc((size_t)bytes);
  if (!t || fread(t, 36, (size_t)n, f) != (size_t)n) return 3;
  fclose(f);
  float slo[3] = {INFINITY, INFINITY, INFINITY}, shi[3] = {-INFINITY, -INFINITY, -INFINITY};
  for (long i = 0; i < n * 3; ++i)
    for (int k = 0; k < 3; ++k) {
      slo[k] = fminf(slo[k], t[3 * i + k]);
      shi[k] = fmaxf(shi[k], t[3 * i + k]);
    }
  double diag = 0.0;
  for (int k = 0; k < 3; ++k) diag = fmax(diag, (double)shi[k] - (double)slo[k]);
  const double eps = diag * (1.0 / 65536.0);
  long pairs = 0, open = 0, wrong = 0;
  for (long g0 = 0; g0 + 4 <= n; g0 += 4) {
    float box[6] = {INFINITY, INFINITY, INFINITY, -INFINITY, -INFINITY, -INFINITY};
    for (long i = g0; i < g0 + 4; ++i)
      for (int v = 0; v < 3; ++v)
        for (int k = 0; k < 3; ++k) {
          box[k] = fminf(box[k], t[9 * i + 3 * v + k]);
          box[3 + k] = fmaxf(box[3 + k], t[9 * i + 3 * v + k]);
        }
    sc::mm::Grid g;
    g.init(box, 6, eps);
    for (long i = g0; i < g0 + 4; ++i) {
      double v[9];
      for (int j = 0; j < 9; ++j) v[j] = (double)t[9 * i + j];
      int r0[3], r1[3];
      for (int k = 0; k < 3; ++k) {
        const double lo = fmin(fmin(v[k], v[3 + k]), v[6 + k]);
        const double hi = fmax(fmax(v[k], v[3 + k]), v[6 + k]);
        g.candidates(k, lo, hi, r0[k], r1[k]);
      }
      for (int z = r0[2]; z <= r1[2]; ++z)
        for (int y = r0[1]; y <= r1[1]; ++y)
          for (int x = r0[0]; x <= r1[0]; ++x) {
            const double bmin[3] = {g.b0[0][x], g.b0[1][y], g.b0[2][z]};
            const double bmax[3] = {g.b1[0][x], g.b1[1][y], g.b1[2][z]};
            const int fr = sc::mm::tri_box_overlap_f32(v, bmin, bmax);
            const int d = sc::mm::tri_box_overlap(v, bmin, bmax) ? 1 : 0;
            ++pairs;
            if (fr < 0) ++open;
            else if (fr != d) ++wrong;
          }
    }
  }
  free(t);
  printf("%ld %ld %ld\n", pairs, open, wrong);
  return wrong != 0;
}

int main(int argc, char** argv) {
  if (argc > 1) return check_file(argv[1]);
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
