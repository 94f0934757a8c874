/*
 * scenegen.c — seeded synthetic scenes and rays (inputs only; see scenegen.h).
 *
 * The scenes stand in for the paper's hair assets (Curly Hair, 12.1M thin
 * tilted triangles, Sec. 4 / Fig. 7), which are not available: the hair
 * generator makes thin, diagonal ribbons, the geometry for which the paper
 * reports its largest culling gains (Sec. 4.1, Table 1).
 */
#include "scenegen.h"

#include <math.h>
#include <string.h>

/* ---------------------------------------------------------------- RNG --- */

static uint64_t splitmix64(uint64_t x) {
  uint64_t z = x + 0x9E3779B97F4A7C15ULL;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
  return z ^ (z >> 31);
}

typedef struct {
  uint64_t state;
  uint64_t inc;
} sg_pcg32;

static uint32_t pcg_next(sg_pcg32* g) {
  uint64_t old = g->state;
  g->state = old * 6364136223846793005ULL + g->inc;
  uint32_t xs = (uint32_t)(((old >> 18) ^ old) >> 27);
  uint32_t rot = (uint32_t)(old >> 59);
  return (xs >> rot) | (xs << ((32u - rot) & 31u));
}

static void pcg_seed(sg_pcg32* g, uint64_t seed, uint64_t stream) {
  uint64_t initstate = splitmix64(seed);
  uint64_t initseq = splitmix64(seed + 1ULL) ^ stream;
  g->state = 0;
  g->inc = (initseq << 1) | 1ULL;
  (void)pcg_next(g);
  g->state += initstate;
  (void)pcg_next(g);
}

static double pcg_uniform(sg_pcg32* g) {
  return (double)(pcg_next(g) >> 8) * (1.0 / 16777216.0);
}

double sg_uniform(uint64_t seed, uint64_t stream, int k) {
  sg_pcg32 g;
  pcg_seed(&g, seed, stream);
  double u = 0.0;
  for (int i = 0; i <= k; ++i) u = pcg_uniform(&g);
  return u;
}

/* ------------------------------------------------- elementary functions --- */

static const double SG_PI = 3.14159265358979311600;
static const double SG_TWO_PI = 6.28318530717958623200;

/* sin and cos by argument reduction to [-pi, pi] and Taylor series in
   nested (Horner) form; only + - * / are used, so the result is the same on
   every IEEE host. */
void sg_sincos(double x, double* s, double* c) {
  double k = floor(x / SG_TWO_PI + 0.5);
  double r = x - k * SG_TWO_PI;
  double r2 = r * r;
  double ps = 1.0, pc = 1.0;
  for (int n = 28; n >= 2; n -= 2) {
    ps = 1.0 - ps * r2 / ((double)n * (double)(n + 1));
    pc = 1.0 - pc * r2 / ((double)(n - 1) * (double)n);
  }
  *s = r * ps;
  *c = pc;
}

double sg_exp(double x) {
  static const double LN2 = 0.69314718055994528623;
  double k = floor(x / LN2 + 0.5);
  double r = x - k * LN2;
  double p = 1.0;
  for (int n = 20; n >= 1; --n) p = 1.0 + p * r / (double)n;
  return ldexp(p, (int)k);
}

/* -------------------------------------------------------- 3-vectors --- */

typedef struct {
  double x, y, z;
} v3;

static v3 v3_make(double x, double y, double z) {
  v3 r = {x, y, z};
  return r;
}
static v3 v3_add(v3 a, v3 b) { return v3_make(a.x + b.x, a.y + b.y, a.z + b.z); }
static v3 v3_sub(v3 a, v3 b) { return v3_make(a.x - b.x, a.y - b.y, a.z - b.z); }
static v3 v3_scale(v3 a, double s) { return v3_make(a.x * s, a.y * s, a.z * s); }
static double v3_dot(v3 a, v3 b) { return (a.x * b.x + a.y * b.y) + a.z * b.z; }
static v3 v3_cross(v3 a, v3 b) {
  return v3_make(a.y * b.z - a.z * b.y, a.z * b.x - a.x * b.z,
                 a.x * b.y - a.y * b.x);
}
static double v3_len(v3 a) { return sqrt(v3_dot(a, a)); }
static v3 v3_div(v3 a, double s) { return v3_make(a.x / s, a.y / s, a.z / s); }

static void put_tri(float* t, v3 a, v3 b, v3 c) {
  t[0] = (float)a.x; t[1] = (float)a.y; t[2] = (float)a.z;
  t[3] = (float)b.x; t[4] = (float)b.y; t[5] = (float)b.z;
  t[6] = (float)c.x; t[7] = (float)c.y; t[8] = (float)c.z;
}

/* Uniform direction by rejection from the cube [-1,1]^3 (no trigonometry). */
static v3 rand_dir(sg_pcg32* g) {
  for (;;) {
    double x = 2.0 * pcg_uniform(g) - 1.0;
    double y = 2.0 * pcg_uniform(g) - 1.0;
    double z = 2.0 * pcg_uniform(g) - 1.0;
    double r2 = (x * x + y * y) + z * z;
    if (r2 > 1e-8 && r2 <= 1.0) {
      double l = sqrt(r2);
      return v3_make(x / l, y / l, z / l);
    }
  }
}

/* --------------------------------------------------------------- hair --- */

int64_t sg_hair_count(int64_t strands, int segs, int ground) {
  return strands * (int64_t)segs * 2 + (ground ? 2 : 0);
}

void sg_hair(uint64_t seed, int64_t strands, int segs, int ground,
             int64_t s_begin, int64_t s_end, float* tris) {
  const double radius = 0.02, pitch = 0.05, length = 0.5, half_w = 5e-4;
  if (s_begin < 0) s_begin = 0;
  if (s_end > strands) s_end = strands;
  for (int64_t s = s_begin; s < s_end; ++s) {
    sg_pcg32 g;
    pcg_seed(&g, seed, (uint64_t)s);
    double z = 2.0 * pcg_uniform(&g) - 1.0;
    double phi = SG_TWO_PI * pcg_uniform(&g);
    double phi0 = SG_TWO_PI * pcg_uniform(&g);
    double rr = 1.0 - z * z;
    rr = rr > 0.0 ? sqrt(rr) : 0.0;
    double sp, cp;
    sg_sincos(phi, &sp, &cp);
    v3 n = v3_make(rr * cp, rr * sp, z);
    v3 a = fabs(n.y) > 0.9 ? v3_cross(n, v3_make(1, 0, 0))
                           : v3_cross(n, v3_make(0, 1, 0));
    a = v3_div(a, v3_len(a));
    v3 b = v3_cross(n, a);
    v3 prev = n;
    for (int k = 0; k <= segs; ++k) {
      double sk = (double)k / (double)segs;
      double axial = length * sk;
      double theta = phi0 + SG_TWO_PI * axial / pitch;
      double st, ct;
      sg_sincos(theta, &st, &ct);
      v3 p = v3_add(v3_add(n, v3_scale(n, axial)),
                    v3_scale(v3_add(v3_scale(a, ct), v3_scale(b, st)), radius));
      if (k > 0) {
        v3 seg = v3_sub(p, prev);
        v3 side = v3_cross(seg, n);
        double ls = v3_len(side);
        side = ls > 1e-12 ? v3_div(side, ls) : a;
        v3 off = v3_scale(side, half_w);
        v3 am = v3_sub(prev, off), ap = v3_add(prev, off);
        v3 bm = v3_sub(p, off), bp = v3_add(p, off);
        int64_t t = 2 * (s * (int64_t)segs + (k - 1));
        put_tri(tris + 9 * t, am, ap, bp);
        put_tri(tris + 9 * (t + 1), am, bp, bm);
      }
      prev = p;
    }
  }
  if (ground && s_end == strands) {
    int64_t t = strands * (int64_t)segs * 2;
    v3 c0 = v3_make(-4, -1.2, -4), c1 = v3_make(4, -1.2, -4);
    v3 c2 = v3_make(4, -1.2, 4), c3 = v3_make(-4, -1.2, 4);
    put_tri(tris + 9 * t, c0, c1, c2);
    put_tri(tris + 9 * (t + 1), c0, c2, c3);
  }
}

/* --------------------------------------------------------------- soup --- */

void sg_soup(uint64_t seed, int64_t i_begin, int64_t i_end, float* tris) {
  static const double LN10 = 2.30258509299404590109;
  for (int64_t i = i_begin; i < i_end; ++i) {
    sg_pcg32 g;
    pcg_seed(&g, seed, (uint64_t)i);
    v3 c = v3_make(pcg_uniform(&g), pcg_uniform(&g), pcg_uniform(&g));
    double ell = sg_exp((-4.0 + 3.0 * pcg_uniform(&g)) * LN10);
    if ((i & 1) == 0) {
      v3 ax = rand_dir(&g);
      v3 w;
      for (;;) {
        v3 r = rand_dir(&g);
        w = v3_sub(r, v3_scale(ax, v3_dot(r, ax)));
        double lw = v3_len(w);
        if (lw > 1e-3) {
          w = v3_div(w, lw);
          break;
        }
      }
      v3 v0 = v3_sub(c, v3_scale(ax, 0.5 * ell));
      v3 v1 = v3_add(c, v3_scale(ax, 0.5 * ell));
      v3 v2 = v3_add(c, v3_scale(w, ell / 1000.0));
      put_tri(tris + 9 * i, v0, v1, v2);
    } else {
      int k = (int)(pcg_uniform(&g) * 3.0);
      if (k > 2) k = 2;
      double leg1 = ell * (pcg_uniform(&g) < 0.5 ? -1.0 : 1.0);
      double leg2 = ell * (0.1 + 0.9 * pcg_uniform(&g)) *
                    (pcg_uniform(&g) < 0.5 ? -1.0 : 1.0);
      double p1[3] = {c.x, c.y, c.z}, p2[3] = {c.x, c.y, c.z};
      p1[(k + 1) % 3] += leg1;
      p2[(k + 2) % 3] += leg2;
      put_tri(tris + 9 * i, c, v3_make(p1[0], p1[1], p1[2]),
              v3_make(p2[0], p2[1], p2[2]));
    }
  }
}

/* --------------------------------------------------------------- rays --- */

static void put_ray(float* r, v3 o, v3 d) {
  r[0] = (float)o.x; r[1] = (float)o.y; r[2] = (float)o.z; r[3] = 0.0f;
  r[4] = (float)d.x; r[5] = (float)d.y; r[6] = (float)d.z; r[7] = INFINITY;
}

void sg_rays_pinhole(int W, int H, uint64_t jitter_seed, float* rays,
                     int32_t* pix) {
  const double tan_half = 0.36397023426620236; /* tan(20 degrees) */
  const double aspect = (double)W / (double)H;
  const int TW = 8, TH = 4;
  int ntx = (W + TW - 1) / TW, nty = (H + TH - 1) / TH;
  int64_t r = 0;
  v3 eye = v3_make(0, 0, 3);
  for (int ty = 0; ty < nty; ++ty)
    for (int tx = 0; tx < ntx; ++tx)
      for (int yy = 0; yy < TH; ++yy)
        for (int xx = 0; xx < TW; ++xx) {
          int i = tx * TW + xx, j = ty * TH + yy;
          if (i >= W || j >= H) continue;
          double fx = 0.5, fy = 0.5;
          if (jitter_seed) {
            sg_pcg32 g;
            pcg_seed(&g, jitter_seed, (uint64_t)j * (uint64_t)W + (uint64_t)i);
            fx = pcg_uniform(&g);
            fy = pcg_uniform(&g);
          }
          double px = ((double)i + fx) / (double)W;
          double py = ((double)j + fy) / (double)H;
          v3 d = v3_make((2.0 * px - 1.0) * aspect * tan_half,
                         (1.0 - 2.0 * py) * tan_half, -1.0);
          d = v3_div(d, v3_len(d));
          put_ray(rays + 8 * r, eye, d);
          if (pix) pix[r] = j * W + i;
          ++r;
        }
}

void sg_rays_random(uint64_t seed, int64_t r_begin, int64_t r_end,
                    float* rays) {
  for (int64_t r = r_begin; r < r_end; ++r) {
    sg_pcg32 g;
    pcg_seed(&g, seed, (uint64_t)r);
    v3 o = v3_make(pcg_uniform(&g), pcg_uniform(&g), pcg_uniform(&g));
    v3 d = rand_dir(&g);
    put_ray(rays + 8 * r, o, d);
  }
}
