/*
 * oracle.c — plain CPU oracle for BVH traversal with subspace culling.
 *
 * TEST INFRASTRUCTURE ONLY: used by tests/, by __graft_entry__.smoke() and by
 * bench.py's CPU baseline; never by the product path.  Every function below
 * is a direct, slow restatement of a definition or algorithm of the paper
 * (Yoshimura & Harada, "Subspace Culling for Ray-Box Intersection", 2023),
 * cited at the function.  Where the paper is silent the reading taken is
 * stated at the function.  Built with -ffp-contract=off -fno-fast-math so
 * that every float operation is one correctly rounded IEEE operation.
 */
#include "oracle.h"

#include <math.h>
#include <pthread.h>
#include <stdatomic.h>
#include <stdlib.h>
#include <string.h>
#include <unistd.h>

/* ------------------------------------------------------------ helpers --- */

int or_mask_words(int R) { return (R * R * R + 31) / 32; }

static void bit_set(uint32_t* m, int bit) { m[bit >> 5] |= 1u << (bit & 31); }
static int bit_get(const uint32_t* m, int bit) {
  return (int)((m[bit >> 5] >> (bit & 31)) & 1u);
}
static int popcount_mask(const uint32_t* m, int W) {
  int c = 0;
  for (int w = 0; w < W; ++w)
    for (int i = 0; i < 32; ++i) c += (int)((m[w] >> i) & 1u);
  return c;
}
static int cell_bit(int R, int x, int y, int z) { return x + R * y + R * R * z; }
static double dmin(double a, double b) { return a < b ? a : b; }
static double dmax(double a, double b) { return a > b ? a : b; }

/* ------------------------------------------------------------ threads --- */
/* The build's independent pieces (subtrees of the BVH, the slots of one
   depth level of the masks, the slots' LUT encodings) may run on several
   threads.  Each piece is computed by the same code whatever the thread, so
   the results do not depend on the thread count. */
static int g_threads = 0; /* 0: every online core */
static int64_t g_task_tris = 0; /* 0: automatic subtree task size */

void or_set_threads(int threads, int64_t task_tris) {
  g_threads = threads < 0 ? 0 : threads;
  g_task_tris = task_tris < 0 ? 0 : task_tris;
}

static int num_threads(void) {
  if (g_threads > 0) return g_threads;
  long n = sysconf(_SC_NPROCESSORS_ONLN);
  return n > 0 ? (int)(n > 256 ? 256 : n) : 1;
}

typedef struct {
  void (*fn)(void* ctx, int64_t i);
  void* ctx;
  int64_t n, grain;
  atomic_llong next;
} Jobs;

static void* jobs_worker(void* arg) {
  Jobs* j = (Jobs*)arg;
  for (;;) {
    int64_t i0 = atomic_fetch_add(&j->next, j->grain);
    if (i0 >= j->n) break;
    int64_t i1 = i0 + j->grain < j->n ? i0 + j->grain : j->n;
    for (int64_t i = i0; i < i1; ++i) j->fn(j->ctx, i);
  }
  return NULL;
}

/* fn(ctx, i) for every i in [0, n), on up to num_threads() threads. */
static void run_jobs(void (*fn)(void*, int64_t), void* ctx, int64_t n, int64_t grain) {
  Jobs j;
  j.fn = fn;
  j.ctx = ctx;
  j.n = n;
  j.grain = grain > 0 ? grain : 1;
  atomic_init(&j.next, 0);
  int t = num_threads();
  if ((int64_t)t > (n + j.grain - 1) / j.grain) t = (int)((n + j.grain - 1) / j.grain);
  if (t <= 1) {
    jobs_worker(&j);
    return;
  }
  pthread_t* th = (pthread_t*)malloc(sizeof(pthread_t) * (size_t)t);
  int started = 0;
  for (int k = 0; k < t - 1; ++k)
    if (pthread_create(&th[k], NULL, jobs_worker, &j) == 0) ++started;
    else break;
  jobs_worker(&j);
  for (int k = 0; k < started; ++k) pthread_join(th[k], NULL);
  free(th);
}

/* ------------------------------------------- ray-mask LUT (Sec. 3.1.1) --- */
/*
 * The ray-mask table is keyed by the discretised begin and end positions of
 * the ray inside the box (a six-dimensional key) and is built with an
 * AABB-AABB sweep test, because the sweep of the begin cell towards the end
 * cell contains every ray segment between the two cells (Sec. 3.1.1).
 *
 * Reading (the paper does not say whether touching counts): in cell units,
 * cell c is [c, c+1]^3; the sweep is the box [b, b+1]^3 translated by
 * t*(e-b), t in [0,1]; cell v is set iff the *interiors* of the moving box
 * and of cell v meet for some t, i.e. there is t in [0,1] with
 * |b_k + t*(e_k - b_k) - v_k| < 1 on every axis k.  Each axis gives an open
 * interval of t; the cell is set iff max(lower bounds, 0) < min(upper
 * bounds, 1).  All bounds are fractions with integer numerator and
 * denominator, compared exactly by cross-multiplication.
 */
int or_raylut_cell(int R, const int* b, const int* e, const int* v) {
  (void)R;
  /* lower bound lo_n/lo_d (starts at 0/1), upper bound hi_n/hi_d (1/1) */
  long lo_n = 0, lo_d = 1, hi_n = 1, hi_d = 1;
  for (int k = 0; k < 3; ++k) {
    long a = (long)b[k] - (long)v[k];
    long dl = (long)e[k] - (long)b[k];
    long ln, hn, den;
    if (dl == 0) {
      if (a != 0) return 0; /* |a| < 1 with integer a means a == 0 */
      continue;
    } else if (dl > 0) {
      ln = -1 - a; hn = 1 - a; den = dl;
    } else {
      ln = a - 1; hn = a + 1; den = -dl;
    }
    if (ln * lo_d > lo_n * den) { lo_n = ln; lo_d = den; }
    if (hn * hi_d < hi_n * den) { hi_n = hn; hi_d = den; }
  }
  return lo_n * hi_d < hi_n * lo_d;
}

void or_raylut(int R, uint32_t* lut) {
  int R3 = R * R * R, W = or_mask_words(R);
  memset(lut, 0, sizeof(uint32_t) * (size_t)R3 * (size_t)R3 * (size_t)W);
  for (int beg = 0; beg < R3; ++beg)
    for (int end = 0; end < R3; ++end) {
      int b[3] = {beg % R, (beg / R) % R, beg / (R * R)};
      int e[3] = {end % R, (end / R) % R, end / (R * R)};
      uint32_t* m = lut + ((size_t)beg * R3 + end) * W;
      for (int z = 0; z < R; ++z)
        for (int y = 0; y < R; ++y)
          for (int x = 0; x < R; ++x) {
            int v[3] = {x, y, z};
            if (or_raylut_cell(R, b, e, v)) bit_set(m, cell_bit(R, x, y, z));
          }
    }
}

/*
 * Ray-mask table at the finer resolution R_ray = 2R (Sec. 4.2).  The begin
 * and end positions are discretised on the 2R grid; each 2R cell lies in
 * exactly one mask cell (the one holding its 2x2x2 block), so the row of
 * (beg, end) sets mask cell v iff the sweep test above, run on the 2R grid,
 * sets one of v's eight sub-cells.  Rows are indexed beg * (2R)^3 + end with
 * beg = x + 2R y + 4R^2 z; each row is an R^3-bit mask of W words.  Only
 * sub-cells within one of the segment's bounding box on every axis can pass
 * (|b_k + t (e_k - b_k) - v_k| < 1 keeps v_k strictly between min - 1 and
 * max + 1), so the scan stops there.  Rows [row_begin, row_end) are filled,
 * so that callers can split the table across threads.
 */
void or_raylut2r_rows(int R, int64_t row_begin, int64_t row_end, uint32_t* lut) {
  const int R2 = 2 * R, R23 = R2 * R2 * R2, W = or_mask_words(R);
  for (int64_t row = row_begin; row < row_end; ++row) {
    const int beg = (int)(row / R23), end = (int)(row % R23);
    const int b[3] = {beg % R2, (beg / R2) % R2, beg / (R2 * R2)};
    const int e[3] = {end % R2, (end / R2) % R2, end / (R2 * R2)};
    int lo[3], hi[3];
    for (int k = 0; k < 3; ++k) {
      lo[k] = (b[k] < e[k] ? b[k] : e[k]);
      hi[k] = (b[k] > e[k] ? b[k] : e[k]);
    }
    uint32_t* m = lut + (size_t)row * W;
    memset(m, 0, sizeof(uint32_t) * (size_t)W);
    for (int z = lo[2]; z <= hi[2]; ++z)
      for (int y = lo[1]; y <= hi[1]; ++y)
        for (int x = lo[0]; x <= hi[0]; ++x) {
          const int v[3] = {x, y, z};
          if (or_raylut_cell(R2, b, e, v)) bit_set(m, cell_bit(R, x / 2, y / 2, z / 2));
        }
  }
}

/* ----------------------------- conservative voxelization (Sec. 3.1.1) --- */
/*
 * Triangle-box overlap by the separating axis theorem (Akenine-Moeller,
 * "Fast 3D Triangle-Box Overlap Testing", 2001): the triangle and the box are
 * disjoint iff they are separated along one of 13 axes (3 box normals, the
 * triangle normal, 9 edge x box-axis cross products).  Touching counts as
 * overlap.  Double precision throughout.
 */
int or_tri_box(const double* tri9, const double* bmin, const double* bmax) {
  double c[3], h[3], a[3][3], e[3][3];
  for (int k = 0; k < 3; ++k) {
    c[k] = 0.5 * (bmin[k] + bmax[k]);
    h[k] = 0.5 * (bmax[k] - bmin[k]);
  }
  for (int i = 0; i < 3; ++i)
    for (int k = 0; k < 3; ++k) a[i][k] = tri9[3 * i + k] - c[k];
  /* box normals */
  for (int k = 0; k < 3; ++k) {
    double mn = dmin(dmin(a[0][k], a[1][k]), a[2][k]);
    double mx = dmax(dmax(a[0][k], a[1][k]), a[2][k]);
    if (mn > h[k] || mx < -h[k]) return 0;
  }
  /* edges */
  for (int k = 0; k < 3; ++k) {
    e[0][k] = a[1][k] - a[0][k];
    e[1][k] = a[2][k] - a[1][k];
    e[2][k] = a[0][k] - a[2][k];
  }
  /* triangle normal: plane n.x = n.a0 against the box's projection radius */
  {
    double n[3] = {e[0][1] * e[1][2] - e[0][2] * e[1][1],
                   e[0][2] * e[1][0] - e[0][0] * e[1][2],
                   e[0][0] * e[1][1] - e[0][1] * e[1][0]};
    double d = (n[0] * a[0][0] + n[1] * a[0][1]) + n[2] * a[0][2];
    double r = (h[0] * fabs(n[0]) + h[1] * fabs(n[1])) + h[2] * fabs(n[2]);
    if (fabs(d) > r) return 0;
  }
  /* nine edge x axis cross products */
  for (int i = 0; i < 3; ++i) {
    for (int k = 0; k < 3; ++k) {
      double ax[3];
      if (k == 0) { ax[0] = 0.0; ax[1] = e[i][2]; ax[2] = -e[i][1]; }
      else if (k == 1) { ax[0] = -e[i][2]; ax[1] = 0.0; ax[2] = e[i][0]; }
      else { ax[0] = e[i][1]; ax[1] = -e[i][0]; ax[2] = 0.0; }
      double p0 = (ax[0] * a[0][0] + ax[1] * a[0][1]) + ax[2] * a[0][2];
      double p1 = (ax[0] * a[1][0] + ax[1] * a[1][1]) + ax[2] * a[1][2];
      double p2 = (ax[0] * a[2][0] + ax[1] * a[2][1]) + ax[2] * a[2][2];
      double mn = dmin(dmin(p0, p1), p2), mx = dmax(dmax(p0, p1), p2);
      double r = (h[0] * fabs(ax[0]) + h[1] * fabs(ax[1])) + h[2] * fabs(ax[2]);
      if (mn > r || mx < -r) return 0;
    }
  }
  return 1;
}

/* Voxel i of a grid over [lo, hi] (one axis), dilated by eps on both sides.
   Reading: the paper gives no robustness rule; the dilation eps absorbs the
   float error of the traversal's clipped segment and cell quantisation, so
   that an object bit is set for every cell within eps of the triangle. */
static void voxel_bounds(double lo, double hi, int R, int i, double eps,
                         double* b0, double* b1) {
  double ext = hi - lo;
  *b0 = (lo + (ext * (double)i) / (double)R) - eps;
  *b1 = (lo + (ext * (double)(i + 1)) / (double)R) + eps;
}

/* Object mask of one triangle in the R^3 grid of box [lo, hi]: every voxel
   the triangle overlaps (Sec. 3.1.1, conservative voxelization).  Plain loop
   over all R^3 voxels; ORs into mask. */
void or_voxelize(const float* tri9, const float* lo, const float* hi, int R,
                 double eps, uint32_t* mask) {
  double t[9];
  for (int i = 0; i < 9; ++i) t[i] = (double)tri9[i];
  for (int z = 0; z < R; ++z)
    for (int y = 0; y < R; ++y)
      for (int x = 0; x < R; ++x) {
        int idx[3] = {x, y, z};
        double bmin[3], bmax[3];
        for (int k = 0; k < 3; ++k)
          voxel_bounds((double)lo[k], (double)hi[k], R, idx[k], eps, &bmin[k],
                       &bmax[k]);
        if (or_tri_box(t, bmin, bmax)) bit_set(mask, cell_bit(R, x, y, z));
      }
}

/* Parent-grid index of a position (one axis), Alg. 2:
   min(floor(R * (border - pLower) / pExtent), R - 1), plus a clamp at 0
   (a child border can only be below pLower by rounding, or by the eps
   dilation).  A flat parent axis (pExtent == 0) has all its R layers at the
   same place, so the whole range [0, R-1] is filled. */
static int parent_index(double pos, double plo, double pext, int R) {
  double q = ((double)R * (pos - plo)) / pext;
  q = floor(q);
  if (q < 0.0) q = 0.0;
  if (q > (double)(R - 1)) q = (double)(R - 1);
  return (int)q;
}

/*
 * Alg. 2 (fillByApproximatedOccupancy): every occupied voxel of the child
 * mask fills, in the parent grid, the box pattern spanned by the parent
 * indices of its min and max vertices.  The six-dimensional pattern table of
 * the paper is the product of three per-axis ranges; here it is evaluated
 * directly.  Reading: the child voxel stands for triangles within eps of it,
 * so its min vertex is projected from (border - eps) and its max vertex from
 * (border + eps); with eps = 0 this is Alg. 2 exactly.
 */
void or_fill(uint32_t* mask, const float* plo, const float* phi,
             const uint32_t* cmask, const float* clo, const float* chi, int R,
             double eps) {
  int lo_idx[3][17], hi_idx[3][17];
  for (int k = 0; k < 3; ++k) {
    double cl = (double)clo[k], cext = (double)chi[k] - (double)clo[k];
    double pl = (double)plo[k], pext = (double)phi[k] - (double)plo[k];
    for (int i = 0; i <= R; ++i) {
      double border = cl + (cext * (double)i) / (double)R;
      if (pext > 0.0) {
        lo_idx[k][i] = parent_index(border - eps, pl, pext, R);
        hi_idx[k][i] = parent_index(border + eps, pl, pext, R);
      } else {
        lo_idx[k][i] = 0;
        hi_idx[k][i] = R - 1;
      }
    }
  }
  for (int z = 0; z < R; ++z)
    for (int y = 0; y < R; ++y)
      for (int x = 0; x < R; ++x) {
        if (!bit_get(cmask, cell_bit(R, x, y, z))) continue;
        for (int pz = lo_idx[2][z]; pz <= hi_idx[2][z + 1]; ++pz)
          for (int py = lo_idx[1][y]; py <= hi_idx[1][y + 1]; ++py)
            for (int px = lo_idx[0][x]; px <= hi_idx[0][x + 1]; ++px)
              bit_set(mask, cell_bit(R, px, py, pz));
      }
}

/* ------------------------------------ compression LUT (Sec. 3.2.2/3) --- */

typedef struct {
  const uint32_t* m;
  double imp;
  int pop;
} Cand;

static int W_sort; /* mask words for the comparators below */

/* mask value as a big unsigned integer, most significant word first */
static int cmp_value(const uint32_t* a, const uint32_t* b, int W) {
  for (int w = W - 1; w >= 0; --w) {
    if (a[w] < b[w]) return -1;
    if (a[w] > b[w]) return 1;
  }
  return 0;
}
static int cmp_by_value(const void* pa, const void* pb) {
  const Cand* a = (const Cand*)pa;
  const Cand* b = (const Cand*)pb;
  return cmp_value(a->m, b->m, W_sort);
}
/* importance descending, then value ascending */
static int cmp_by_importance(const void* pa, const void* pb) {
  const Cand* a = (const Cand*)pa;
  const Cand* b = (const Cand*)pb;
  if (a->imp > b->imp) return -1;
  if (a->imp < b->imp) return 1;
  return cmp_value(a->m, b->m, W_sort);
}
/* popcount ascending, importance descending, value ascending */
static int cmp_by_popcount(const void* pa, const void* pb) {
  const Cand* a = (const Cand*)pa;
  const Cand* b = (const Cand*)pb;
  if (a->pop != b->pop) return a->pop < b->pop ? -1 : 1;
  return cmp_by_importance(pa, pb);
}

static double box_area(const float* box6) {
  double dx = (double)box6[3] - (double)box6[0];
  double dy = (double)box6[4] - (double)box6[1];
  double dz = (double)box6[5] - (double)box6[2];
  return 2.0 * ((dx * dy + dy * dz) + dz * dx);
}

/*
 * Compression LUT (Sec. 3.2.2): the importance of an object mask is
 * SA(N) * O_m(N) / R^3 (the per-node term of Eq. 2); the K most important
 * masks form the table.  Readings where the paper is silent: a mask used by
 * several slots has the sum of their importances (slot order); ties are
 * broken by the mask value; an all-ones mask is always kept (it is the only
 * mask guaranteed to be a superset of every mask, so every mask has a
 * conservative entry); the table is sorted by popcount ascending (Sec.
 * 3.2.3), ties by importance descending, then value.  Returns the number of
 * entries (<= K).
 */
int or_clut_build(const uint32_t* masks, const float* boxes, int64_t nslots,
                  int R, int K, uint32_t* clut, double* importance) {
  int W = or_mask_words(R), R3 = R * R * R;
  W_sort = W;
  /* all-ones mask */
  uint32_t* ones = (uint32_t*)calloc((size_t)W, sizeof(uint32_t));
  for (int i = 0; i < R3; ++i) bit_set(ones, i);
  /* distinct masks with summed importance, accumulated in slot order */
  Cand* c = (Cand*)malloc(sizeof(Cand) * (size_t)(nslots + 1));
  for (int64_t s = 0; s < nslots; ++s) {
    c[s].m = masks + (size_t)s * W;
    c[s].pop = popcount_mask(c[s].m, W);
    c[s].imp = 0.0;
  }
  /* sort a copy by value to find duplicates; keep the first slot's order for
     summation by summing in a second pass over slots */
  Cand* byv = (Cand*)malloc(sizeof(Cand) * (size_t)(nslots + 1));
  memcpy(byv, c, sizeof(Cand) * (size_t)nslots);
  qsort(byv, (size_t)nslots, sizeof(Cand), cmp_by_value);
  int64_t nd = 0;
  for (int64_t i = 0; i < nslots; ++i)
    if (nd == 0 || cmp_value(byv[nd - 1].m, byv[i].m, W) != 0) byv[nd++] = byv[i];
  for (int64_t s = 0; s < nslots; ++s) {
    /* binary search for the distinct entry of slot s */
    int64_t lo = 0, hi = nd - 1;
    while (lo < hi) {
      int64_t mid = (lo + hi) / 2;
      if (cmp_value(byv[mid].m, c[s].m, W) < 0) lo = mid + 1; else hi = mid;
    }
    byv[lo].imp += (box_area(boxes + 6 * s) * (double)c[s].pop) / (double)R3;
  }
  qsort(byv, (size_t)nd, sizeof(Cand), cmp_by_importance);
  int has_ones = 0;
  int64_t take = nd < K ? nd : K;
  for (int64_t i = 0; i < take; ++i)
    if (cmp_value(byv[i].m, ones, W) == 0) has_ones = 1;
  if (!has_ones) {
    double ones_imp = 0.0;
    for (int64_t i = take; i < nd; ++i)
      if (cmp_value(byv[i].m, ones, W) == 0) ones_imp = byv[i].imp;
    if (take == K) take = K - 1;
    byv[take].m = ones;
    byv[take].pop = R3;
    byv[take].imp = ones_imp;
    ++take;
  }
  qsort(byv, (size_t)take, sizeof(Cand), cmp_by_popcount);
  for (int64_t i = 0; i < take; ++i) {
    memcpy(clut + (size_t)i * W, byv[i].m, sizeof(uint32_t) * (size_t)W);
    if (importance) importance[i] = byv[i].imp;
  }
  int k = (int)take;
  free(byv);
  free(c);
  free(ones);
  return k;
}

/* b bits of a mask starting at bit position `at` (zero past R^3). */
static unsigned read_bits(const uint32_t* m, int R3, int at, int b) {
  unsigned v = 0;
  for (int j = 0; j < b; ++j) {
    int bit = at + j;
    if (bit < R3 && bit_get(m, bit)) v |= 1u << j;
  }
  return v;
}

/*
 * Requirement LUTs (Sec. 3.2.3, Fig. 8): for chunk i (bits [i*b, i*b+b)) and
 * each b-bit pattern p, the set of table entries j whose chunk i contains
 * every bit of p, as a 256-bit list (8 words).
 */
void or_req_luts(const uint32_t* clut, int K, int R, int b, uint32_t* req) {
  int R3 = R * R * R, W = or_mask_words(R);
  int nchunk = (R3 + b - 1) / b, np = 1 << b;
  memset(req, 0, sizeof(uint32_t) * (size_t)nchunk * (size_t)np * 8);
  for (int i = 0; i < nchunk; ++i)
    for (int p = 0; p < np; ++p)
      for (int j = 0; j < K; ++j) {
        unsigned cj = read_bits(clut + (size_t)j * W, R3, i * b, b);
        if ((cj & (unsigned)p) == (unsigned)p)
          bit_set(req + ((size_t)i * np + p) * 8, j);
      }
}

/* Alg. 3 (indexOfOptimalMask): AND the per-chunk requirement lists and
   return the least significant set bit, the tightest conservative entry
   because the table is sorted by popcount. */
int or_encode(const uint32_t* mask, const uint32_t* req, int R, int b) {
  int R3 = R * R * R, nchunk = (R3 + b - 1) / b, np = 1 << b;
  uint32_t list[8];
  for (int w = 0; w < 8; ++w) list[w] = 0xFFFFFFFFu;
  for (int i = 0; i < nchunk; ++i) {
    unsigned bits = read_bits(mask, R3, i * b, b);
    const uint32_t* r = req + ((size_t)i * np + bits) * 8;
    for (int w = 0; w < 8; ++w) list[w] &= r[w];
  }
  for (int j = 0; j < 256; ++j)
    if ((list[j >> 5] >> (j & 31)) & 1u) return j;
  return -1;
}

/* The paper's naive comparator (Table 3): first table entry, in popcount
   order, that contains every bit of the mask. */
int or_encode_naive(const uint32_t* mask, const uint32_t* clut, int K, int R) {
  int W = or_mask_words(R);
  for (int j = 0; j < K; ++j) {
    const uint32_t* c = clut + (size_t)j * W;
    int ok = 1;
    for (int w = 0; w < W; ++w)
      if ((c[w] & mask[w]) != mask[w]) ok = 0;
    if (ok) return j;
  }
  return -1;
}

/* ------------------------------------------- binned SAH BVH2 (Sec. 4) --- */
/*
 * The paper builds its BVH with binned SAH (Sec. 4); this path uses a binary
 * BVH.  Canonical rules (the paper gives none beyond "binned SAH"):
 *  - triangle box = float min/max of its vertices; centroid (double) =
 *    0.5*(lo + hi);
 *  - a range of n <= max_leaf triangles is a leaf;
 *  - otherwise, per axis with centroid extent > 0, bin index =
 *    min(bins-1, (int)((c - cmin) * (bins / extent))); each split plane
 *    between bins i and i+1 costs SA(L)*|L| + SA(R)*|R| (Eq. 1's greedy
 *    form, double); the cheapest non-empty split wins, ties to the lower
 *    axis then the lower plane;
 *  - no valid split (all centroids equal): the first n/2 go left;
 *  - the partition is stable; nodes are numbered in pre-order.
 */
struct OrBvh {
  int64_t ntri, nnodes, cap;
  int32_t root_child, root_count;
  float root_box[6];
  int32_t* child; /* [nn][2] */
  int32_t* count; /* [nn][2] */
  float* box;     /* [nn][2][6] */
  int32_t* perm;  /* [ntri] */
  int32_t* ndepth; /* [nn] depth of the slot each node fills (root node 0) */
  int max_depth;
  /* masks */
  int R, L, W;
  double eps;
  uint32_t* masks; /* [nn][2][W] */
  /* compression */
  int K, bits;
  uint32_t* clut;  /* [K][W] */
  uint8_t* cidx;   /* [nn][2] */
  uint32_t* raylut;
  int ideal; /* 1: culling tests use the exact ray mask (ideal_ray_mask) */
  const uint32_t* raylut2r; /* R_ray = 2R table (caller-owned), or NULL */
  int cellform; /* Alg. 1 cell form: 0 as written (default), 1 fused (or_cell_t) */
  /* 4-wide view (or_bvh_wide): per 4-wide node its child slots as (binary
     parent node, child index), and the 4-wide node of each inner child */
  int64_t nn4;
  int32_t* w4n;     /* [nn4] number of children (2..4) */
  int64_t* w4p;     /* [nn4][4] */
  int32_t* w4c;     /* [nn4][4] */
  int64_t* w4next;  /* [nn4][4] 4-wide node of an inner child, -1 for a leaf */
  int w4depth;      /* deepest 4-wide node (root 0) */
};

typedef struct {
  float lo[3], hi[3];
  double c[3];
} TriRec;

static void box_empty(float* b) {
  b[0] = b[1] = b[2] = INFINITY;
  b[3] = b[4] = b[5] = -INFINITY;
}
static void box_grow(float* b, const float* lo, const float* hi) {
  for (int k = 0; k < 3; ++k) {
    b[k] = fminf(b[k], lo[k]);
    b[3 + k] = fmaxf(b[3 + k], hi[k]);
  }
}

typedef struct {
  OrBvh* b;
  const TriRec* rec;
  int32_t* tmp;
  int max_leaf, bins;
} BuildCtx;

static int bin_of(double c, double cmin, double ext, int bins) {
  int i = (int)((c - cmin) * ((double)bins / ext));
  if (i > bins - 1) i = bins - 1;
  if (i < 0) i = 0;
  return i;
}

static int64_t new_node(OrBvh* b) {
  if (b->nnodes == b->cap) {
    b->cap = b->cap ? 2 * b->cap : 64;
    b->child = (int32_t*)realloc(b->child, sizeof(int32_t) * 2 * b->cap);
    b->count = (int32_t*)realloc(b->count, sizeof(int32_t) * 2 * b->cap);
    b->box = (float*)realloc(b->box, sizeof(float) * 12 * b->cap);
    b->ndepth = (int32_t*)realloc(b->ndepth, sizeof(int32_t) * b->cap);
  }
  return b->nnodes++;
}

/* The box of perm[begin, end) into s_box, and, for a range of more than
   max_leaf triangles, its binned-SAH split: the range is partitioned in
   place and the position of the split is returned; -1 for a leaf. */
static int64_t split_range(BuildCtx* x, int64_t begin, int64_t end, int depth, float* s_box) {
  OrBvh* b = x->b;
  int64_t n = end - begin;
  box_empty(s_box);
  for (int64_t i = begin; i < end; ++i)
    box_grow(s_box, x->rec[b->perm[i]].lo, x->rec[b->perm[i]].hi);
  if (depth > b->max_depth) b->max_depth = depth;
  if (n <= x->max_leaf) return -1;
  double cmin[3] = {INFINITY, INFINITY, INFINITY};
  double cmax[3] = {-INFINITY, -INFINITY, -INFINITY};
  for (int64_t i = begin; i < end; ++i)
    for (int k = 0; k < 3; ++k) {
      double c = x->rec[b->perm[i]].c[k];
      cmin[k] = dmin(cmin[k], c);
      cmax[k] = dmax(cmax[k], c);
    }
  int best_axis = -1, best_plane = -1;
  double best_cost = INFINITY;
  int nb = x->bins;
  int64_t* cnt = (int64_t*)malloc(sizeof(int64_t) * nb);
  float* bb = (float*)malloc(sizeof(float) * 6 * nb);
  int64_t* lcnt = (int64_t*)malloc(sizeof(int64_t) * nb);
  double* larea = (double*)malloc(sizeof(double) * nb);
  for (int k = 0; k < 3; ++k) {
    double ext = cmax[k] - cmin[k];
    if (!(ext > 0.0)) continue;
    for (int i = 0; i < nb; ++i) {
      cnt[i] = 0;
      box_empty(bb + 6 * i);
    }
    for (int64_t i = begin; i < end; ++i) {
      const TriRec* t = &x->rec[b->perm[i]];
      int bi = bin_of(t->c[k], cmin[k], ext, nb);
      cnt[bi] += 1;
      box_grow(bb + 6 * bi, t->lo, t->hi);
    }
    float acc[6];
    box_empty(acc);
    int64_t ac = 0;
    for (int i = 0; i < nb - 1; ++i) {
      ac += cnt[i];
      box_grow(acc, bb + 6 * i, bb + 6 * i + 3);
      lcnt[i] = ac;
      larea[i] = ac > 0 ? box_area(acc) : 0.0;
    }
    /* evaluate planes in ascending order for the tie rule */
    {
      double* rarea = (double*)malloc(sizeof(double) * nb);
      int64_t* rcnt = (int64_t*)malloc(sizeof(int64_t) * nb);
      box_empty(acc);
      ac = 0;
      for (int i = nb - 1; i >= 1; --i) {
        ac += cnt[i];
        box_grow(acc, bb + 6 * i, bb + 6 * i + 3);
        rcnt[i - 1] = ac;
        rarea[i - 1] = ac > 0 ? box_area(acc) : 0.0;
      }
      for (int plane = 0; plane < nb - 1; ++plane) {
        int64_t nl = lcnt[plane], nr = rcnt[plane];
        if (nl == 0 || nr == 0) continue;
        double cost = larea[plane] * (double)nl + rarea[plane] * (double)nr;
        if (cost < best_cost) {
          best_cost = cost;
          best_axis = k;
          best_plane = plane;
        }
      }
      free(rarea);
      free(rcnt);
    }
  }
  free(cnt);
  free(bb);
  free(lcnt);
  free(larea);
  int64_t mid;
  if (best_axis >= 0) {
    double ext = cmax[best_axis] - cmin[best_axis];
    int64_t nl = 0, nr = 0;
    for (int64_t i = begin; i < end; ++i) {
      int32_t t = b->perm[i];
      if (bin_of(x->rec[t].c[best_axis], cmin[best_axis], ext, nb) <= best_plane)
        b->perm[begin + nl++] = t;
      else
        x->tmp[nr++] = t;
    }
    memcpy(b->perm + begin + nl, x->tmp, sizeof(int32_t) * (size_t)nr);
    mid = begin + nl;
  } else {
    mid = begin + n / 2;
  }
  return mid;
}

/* Builds the subtree for perm[begin, end) and returns its slot. */
static void build_range(BuildCtx* x, int64_t begin, int64_t end, int depth,
                        int32_t* s_child, int32_t* s_count, float* s_box) {
  OrBvh* b = x->b;
  int64_t mid = split_range(x, begin, end, depth, s_box);
  if (mid < 0) {
    *s_child = (int32_t)begin;
    *s_count = (int32_t)(end - begin);
    return;
  }
  int64_t node = new_node(b);
  b->ndepth[node] = depth;
  *s_child = (int32_t)node;
  *s_count = 0;
  int32_t c0, n0, c1, n1;
  float b0[6], b1[6];
  build_range(x, begin, mid, depth + 1, &c0, &n0, b0);
  build_range(x, mid, end, depth + 1, &c1, &n1, b1);
  b->child[2 * node] = c0;
  b->count[2 * node] = n0;
  b->child[2 * node + 1] = c1;
  b->count[2 * node + 1] = n1;
  memcpy(b->box + 12 * node, b0, sizeof(b0));
  memcpy(b->box + 12 * node + 6, b1, sizeof(b1));
}

/* ---- the same build with independent subtrees on several threads.  The
   top of the tree is split serially (build_top) down to ranges of at most
   `task` triangles; each such range is a task that build_range turns into a
   subtree in its own node arrays (its perm range is disjoint from every
   other's); then every node gets the number the serial pre-order recursion
   gives it: a top node before its left subtree, a task's nodes as one
   block in their own pre-order. */
typedef struct {
  int64_t begin, end;
  int depth;
  int64_t parent; /* top node holding the slot, -1 for the root slot */
  int c;
  OrBvh sub;      /* the task's nodes (perm shared with the tree) */
  int32_t child, count;
  float box[6];
  const TriRec* rec;
  int max_leaf, bins;
} Task;

typedef struct {
  Task* t;
  int64_t n, cap;
} TaskList;

static void build_top(BuildCtx* x, TaskList* tl, int64_t task, int64_t begin, int64_t end,
                      int depth, int64_t parent, int c, int32_t* s_child, int32_t* s_count,
                      float* s_box) {
  OrBvh* b = x->b;
  int64_t n = end - begin;
  if (n > x->max_leaf && n <= task) {
    if (tl->n == tl->cap) {
      tl->cap = tl->cap ? 2 * tl->cap : 64;
      tl->t = (Task*)realloc(tl->t, sizeof(Task) * (size_t)tl->cap);
    }
    Task* t = &tl->t[tl->n];
    memset(t, 0, sizeof(*t));
    t->begin = begin;
    t->end = end;
    t->depth = depth;
    t->parent = parent;
    t->c = c;
    *s_child = (int32_t)tl->n++;
    *s_count = -1; /* filled in after the tasks ran */
    return;
  }
  /* as build_range, with the recursion below going to build_top */
  int64_t mid = split_range(x, begin, end, depth, s_box);
  if (mid < 0) {
    *s_child = (int32_t)begin;
    *s_count = (int32_t)n;
    return;
  }
  int64_t node = new_node(b);
  b->ndepth[node] = depth;
  *s_child = (int32_t)node;
  *s_count = 0;
  int32_t c0, n0, c1, n1;
  float b0[6], b1[6];
  build_top(x, tl, task, begin, mid, depth + 1, node, 0, &c0, &n0, b0);
  build_top(x, tl, task, mid, end, depth + 1, node, 1, &c1, &n1, b1);
  b->child[2 * node] = c0;
  b->count[2 * node] = n0;
  b->child[2 * node + 1] = c1;
  b->count[2 * node + 1] = n1;
  memcpy(b->box + 12 * node, b0, sizeof(b0));
  memcpy(b->box + 12 * node + 6, b1, sizeof(b1));
}

static void task_job(void* ctx, int64_t i) {
  Task* t = &((TaskList*)ctx)->t[i];
  BuildCtx x = {&t->sub, t->rec, (int32_t*)malloc(sizeof(int32_t) * (size_t)(t->end - t->begin)),
                t->max_leaf, t->bins};
  build_range(&x, t->begin, t->end, t->depth, &t->child, &t->count, t->box);
  free(x.tmp);
}

/* Pre-order numbers: map[top node] and base[task]. */
static void number_top(const OrBvh* b, const TaskList* tl, int64_t node, int64_t* next,
                       int64_t* map, int64_t* base) {
  map[node] = (*next)++;
  for (int c = 0; c < 2; ++c) {
    int32_t ch = b->child[2 * node + c], cn = b->count[2 * node + c];
    if (cn == -1) {
      base[ch] = *next;
      *next += tl->t[ch].sub.nnodes;
    } else if (cn == 0) {
      number_top(b, tl, ch, next, map, base);
    }
  }
}

static void build_threaded(BuildCtx* x, int64_t n, int64_t task) {
  OrBvh* b = x->b;
  TaskList tl = {NULL, 0, 0};
  build_top(x, &tl, task, 0, n, 0, -1, 0, &b->root_child, &b->root_count, b->root_box);
  for (int64_t k = 0; k < tl.n; ++k) {
    Task* t = &tl.t[k];
    t->sub.perm = b->perm;
    t->rec = x->rec;
    t->max_leaf = x->max_leaf;
    t->bins = x->bins;
  }
  run_jobs(task_job, &tl, tl.n, 1);
  int64_t ntop = b->nnodes, next = 0;
  int64_t* map = (int64_t*)malloc(sizeof(int64_t) * (size_t)(ntop > 0 ? ntop : 1));
  int64_t* base = (int64_t*)malloc(sizeof(int64_t) * (size_t)(tl.n > 0 ? tl.n : 1));
  if (b->root_count == -1) {
    base[b->root_child] = 0;
    next = tl.t[b->root_child].sub.nnodes;
  } else if (b->root_count == 0) {
    number_top(b, &tl, b->root_child, &next, map, base);
  }
  OrBvh f;
  memset(&f, 0, sizeof(f));
  f.cap = next > 0 ? next : 1;
  f.nnodes = next;
  f.child = (int32_t*)malloc(sizeof(int32_t) * 2 * (size_t)f.cap);
  f.count = (int32_t*)malloc(sizeof(int32_t) * 2 * (size_t)f.cap);
  f.box = (float*)malloc(sizeof(float) * 12 * (size_t)f.cap);
  f.ndepth = (int32_t*)malloc(sizeof(int32_t) * (size_t)f.cap);
  int max_depth = b->max_depth;
  /* a slot word (child, count) in the final numbering; a task's root is an
     inner node (the task has more than max_leaf triangles) */
  for (int64_t k = 0; k < tl.n; ++k) {
    Task* t = &tl.t[k];
    for (int64_t i = 0; i < t->sub.nnodes; ++i) {
      int64_t d = base[k] + i;
      for (int c = 0; c < 2; ++c) {
        int32_t ch = t->sub.child[2 * i + c], cn = t->sub.count[2 * i + c];
        f.child[2 * d + c] = cn > 0 ? ch : (int32_t)(base[k] + ch);
        f.count[2 * d + c] = cn;
      }
      memcpy(f.box + 12 * d, t->sub.box + 12 * i, sizeof(float) * 12);
      f.ndepth[d] = t->sub.ndepth[i];
    }
    if (t->sub.max_depth > max_depth) max_depth = t->sub.max_depth;
    if (t->parent >= 0) {
      memcpy(b->box + 12 * t->parent + 6 * t->c, t->box, sizeof(float) * 6);
    } else {
      memcpy(b->root_box, t->box, sizeof(float) * 6);
    }
  }
  for (int64_t i = 0; i < ntop; ++i) {
    int64_t d = map[i];
    for (int c = 0; c < 2; ++c) {
      int32_t ch = b->child[2 * i + c], cn = b->count[2 * i + c];
      if (cn == -1) {
        f.child[2 * d + c] = (int32_t)base[ch];
        f.count[2 * d + c] = 0;
      } else {
        f.child[2 * d + c] = cn > 0 ? ch : (int32_t)map[ch];
        f.count[2 * d + c] = cn;
      }
    }
    memcpy(f.box + 12 * d, b->box + 12 * i, sizeof(float) * 12);
    f.ndepth[d] = b->ndepth[i];
  }
  if (b->root_count == -1) {
    b->root_child = 0;
    b->root_count = 0;
  } else if (b->root_count == 0) {
    b->root_child = (int32_t)map[b->root_child];
  }
  free(b->child);
  free(b->count);
  free(b->box);
  free(b->ndepth);
  b->child = f.child;
  b->count = f.count;
  b->box = f.box;
  b->ndepth = f.ndepth;
  b->nnodes = f.nnodes;
  b->cap = f.cap;
  b->max_depth = max_depth;
  for (int64_t k = 0; k < tl.n; ++k) {
    free(tl.t[k].sub.child);
    free(tl.t[k].sub.count);
    free(tl.t[k].sub.box);
    free(tl.t[k].sub.ndepth);
  }
  free(tl.t);
  free(map);
  free(base);
}

OrBvh* or_bvh_build(const float* tris, int64_t n, int max_leaf, int bins) {
  OrBvh* b = (OrBvh*)calloc(1, sizeof(OrBvh));
  b->ntri = n;
  b->perm = (int32_t*)malloc(sizeof(int32_t) * (size_t)(n > 0 ? n : 1));
  TriRec* rec = (TriRec*)malloc(sizeof(TriRec) * (size_t)(n > 0 ? n : 1));
  for (int64_t i = 0; i < n; ++i) {
    const float* t = tris + 9 * i;
    for (int k = 0; k < 3; ++k) {
      rec[i].lo[k] = fminf(fminf(t[k], t[3 + k]), t[6 + k]);
      rec[i].hi[k] = fmaxf(fmaxf(t[k], t[3 + k]), t[6 + k]);
      rec[i].c[k] = 0.5 * ((double)rec[i].lo[k] + (double)rec[i].hi[k]);
    }
    b->perm[i] = (int32_t)i;
  }
  if (n == 0) {
    b->root_child = -1;
    b->root_count = 0;
    box_empty(b->root_box);
    free(rec);
    return b;
  }
  BuildCtx x = {b, rec, (int32_t*)malloc(sizeof(int32_t) * (size_t)n),
                max_leaf, bins};
  int th = num_threads();
  int64_t task = g_task_tris > 0 ? g_task_tris : n / (16 * (int64_t)th);
  if (task < 4096) task = 4096;
  if (th > 1 && n > task && max_leaf >= 1) {
    build_threaded(&x, n, task);
  } else {
    build_range(&x, 0, n, 0, &b->root_child, &b->root_count, b->root_box);
  }
  free(x.tmp);
  free(rec);
  return b;
}

void or_bvh_set_ideal(OrBvh* b, int ideal) { b->ideal = ideal; }
void or_bvh_set_cellform(OrBvh* b, int form) { b->cellform = form == 1 ? 1 : 0; }

/* Refit for moved triangles (dynamic scenes, which the paper leaves to
   future work): the tree's topology and triangle order stay; every child
   slot's box becomes the union of the boxes of the triangles below it, each
   triangle's box taken from `tris` (new positions, input order) exactly as
   the build takes it.  Object masks and compression indices are then
   recomputed by the caller (or_bvh_masks, or_bvh_reencode). */
static void refit_slot(OrBvh* b, const float* tris, int32_t child, int32_t count,
                       float* box) {
  box_empty(box);
  if (count > 0) {
    for (int32_t i = 0; i < count; ++i) {
      const float* t = tris + 9 * (size_t)b->perm[child + i];
      float lo[3], hi[3];
      for (int k = 0; k < 3; ++k) {
        lo[k] = fminf(fminf(t[k], t[3 + k]), t[6 + k]);
        hi[k] = fmaxf(fmaxf(t[k], t[3 + k]), t[6 + k]);
      }
      box_grow(box, lo, hi);
    }
    return;
  }
  for (int c = 0; c < 2; ++c) {
    float* cb = b->box + 12 * (size_t)child + 6 * c;
    refit_slot(b, tris, b->child[2 * (size_t)child + c], b->count[2 * (size_t)child + c], cb);
    box_grow(box, cb, cb + 3);
  }
}

int or_bvh_refit(OrBvh* b, const float* tris) {
  if (b->ntri == 0) return 0;
  refit_slot(b, tris, b->root_child, b->root_count, b->root_box);
  return 0;
}

/* Alg. 3 again for every slot against the LUT already chosen (after the
   masks changed); the LUT itself is kept. */
int or_bvh_reencode(OrBvh* b) {
  if (!b->clut || !b->masks) return -1;
  int W = b->W, R = b->R;
  int64_t ns = b->nnodes * 2;
  int nchunk = (R * R * R + b->bits - 1) / b->bits;
  uint32_t* req = (uint32_t*)malloc(sizeof(uint32_t) * (size_t)nchunk * (1u << b->bits) * 8);
  or_req_luts(b->clut, b->K, R, b->bits, req);
  for (int64_t s = 0; s < ns; ++s)
    b->cidx[s] = (uint8_t)or_encode(b->masks + (size_t)s * W, req, R, b->bits);
  free(req);
  return 0;
}

void or_bvh_set_raylut2r(OrBvh* b, const uint32_t* lut2r) { b->raylut2r = lut2r; }

void or_bvh_free(OrBvh* b) {
  if (!b) return;
  free(b->child);
  free(b->count);
  free(b->box);
  free(b->perm);
  free(b->masks);
  free(b->clut);
  free(b->cidx);
  free(b->raylut);
  free(b->ndepth);
  free(b->w4n);
  free(b->w4p);
  free(b->w4c);
  free(b->w4next);
  free(b);
}

int64_t or_bvh_num_nodes(const OrBvh* b) { return b->nnodes; }
int or_bvh_max_depth(const OrBvh* b) { return b->max_depth; }
void or_bvh_root(const OrBvh* b, int32_t* child, int32_t* count, float* box6) {
  *child = b->root_child;
  *count = b->root_count;
  memcpy(box6, b->root_box, sizeof(float) * 6);
}
void or_bvh_nodes(const OrBvh* b, int32_t* child, int32_t* count, float* box) {
  memcpy(child, b->child, sizeof(int32_t) * 2 * (size_t)b->nnodes);
  memcpy(count, b->count, sizeof(int32_t) * 2 * (size_t)b->nnodes);
  memcpy(box, b->box, sizeof(float) * 12 * (size_t)b->nnodes);
}
void or_bvh_perm(const OrBvh* b, int32_t* perm) {
  memcpy(perm, b->perm, sizeof(int32_t) * (size_t)b->ntri);
}

/* SAH cost of the tree (Eq. 1): (C_T * sum over inner nodes SA + C_I * sum
   over leaves SA * |N_l|) / SA(root). */
double or_bvh_sah(const OrBvh* b, double ct, double ci) {
  if (b->ntri == 0) return 0.0;
  double sroot = box_area(b->root_box);
  double inner = 0.0, leaf = 0.0;
  if (b->root_count > 0) leaf += sroot * (double)b->root_count;
  else inner += sroot;
  for (int64_t nidx = 0; nidx < b->nnodes; ++nidx)
    for (int c = 0; c < 2; ++c) {
      double a = box_area(b->box + 12 * nidx + 6 * c);
      if (b->count[2 * nidx + c] > 0) leaf += a * (double)b->count[2 * nidx + c];
      else inner += a;
    }
  return (ct * inner + ci * leaf) / sroot;
}

/* ------------------------------------- object masks for the BVH (3.2.1) --- */

/* eps = eps_rel * max(1, max |vertex coordinate|) */
double or_scene_eps(const float* tris, int64_t n, double eps_rel) {
  double s = 1.0;
  for (int64_t i = 0; i < 9 * n; ++i) s = dmax(s, fabs((double)tris[i]));
  return eps_rel * s;
}

typedef struct {
  OrBvh* b;
  const float* tris;
} MaskCtx;

static void voxelize_leaf(MaskCtx* x, int32_t start, int32_t count,
                          const float* gbox, uint32_t* out) {
  OrBvh* b = x->b;
  for (int32_t i = 0; i < count; ++i)
    or_voxelize(x->tris + 9 * (size_t)b->perm[start + i], gbox, gbox + 3, b->R,
                b->eps, out);
}

/* Gathers into `out` (grid = gbox) the occupancy of inner node m, which is
   `depth - 1` levels below the slot being built: descendants exactly L
   levels below contribute their own masks through Alg. 2; leaves reached
   earlier contribute their triangles directly. */
static void collect(MaskCtx* x, int64_t m, int depth, const float* gbox,
                    uint32_t* out) {
  OrBvh* b = x->b;
  for (int c = 0; c < 2; ++c) {
    int32_t ch = b->child[2 * m + c], cn = b->count[2 * m + c];
    const float* cbox = b->box + 12 * m + 6 * c;
    if (depth == b->L) {
      or_fill(out, gbox, gbox + 3, b->masks + ((size_t)m * 2 + c) * b->W, cbox,
              cbox + 3, b->R, b->eps);
    } else if (cn > 0) {
      voxelize_leaf(x, ch, cn, gbox, out);
    } else {
      collect(x, ch, depth + 1, gbox, out);
    }
  }
}

/*
 * Object masks of every child slot (Sec. 3.2.1).  Reading of "compute object
 * masks from the node L levels below": the mask of a slot is the OR of
 *   - the direct voxelization of the triangles of every leaf fewer than L
 *     levels below the slot's node, and
 *   - Alg. 2 applied to the mask of every descendant exactly L levels below.
 * L = 1 uses the direct children only; a very large L voxelizes every
 * triangle below the slot (the exact mask).  Leaf slots are voxelized
 * directly.  Nodes are visited in decreasing index order, so (pre-order
 * numbering) every descendant's mask exists before it is used.
 */
static int masks_fill_all(OrBvh* b, const float* tris);

int or_bvh_masks(OrBvh* b, const float* tris, int R, int L, double eps) {
  if (R < 1 || R > 16 || L < 1) return -1;
  b->R = R;
  b->L = L;
  b->W = or_mask_words(R);
  b->eps = eps;
  free(b->masks);
  b->masks = (uint32_t*)calloc((size_t)(b->nnodes > 0 ? b->nnodes : 1) * 2 * b->W,
                               sizeof(uint32_t));
  free(b->raylut);
  b->raylut = NULL;
  return masks_fill_all(b, tris);
}

/* The two slot masks of node nidx. */
static void node_masks(MaskCtx* x, int64_t nidx) {
  OrBvh* b = x->b;
  for (int c = 0; c < 2; ++c) {
    uint32_t* out = b->masks + ((size_t)nidx * 2 + c) * b->W;
    const float* gbox = b->box + 12 * nidx + 6 * c;
    int32_t ch = b->child[2 * nidx + c], cn = b->count[2 * nidx + c];
    memset(out, 0, sizeof(uint32_t) * b->W);
    if (cn > 0) voxelize_leaf(x, ch, cn, gbox, out);
    else collect(x, ch, 1, gbox, out);
  }
}

typedef struct {
  MaskCtx* x;
  const int64_t* nodes;
} LevelJob;

static void level_job(void* ctx, int64_t i) {
  LevelJob* j = (LevelJob*)ctx;
  node_masks(j->x, j->nodes[i]);
}

/* A slot's mask reads only the masks of slots deeper than itself, so the
   nodes are processed one depth level at a time, deepest first, and the
   nodes of one level independently (on several threads). */
static int masks_fill_all(OrBvh* b, const float* tris) {
  MaskCtx x = {b, tris};
  int64_t nn = b->nnodes;
  if (nn == 0) return 0;
  int D = 0;
  for (int64_t i = 0; i < nn; ++i)
    if (b->ndepth[i] > D) D = b->ndepth[i];
  int64_t* start = (int64_t*)calloc((size_t)D + 2, sizeof(int64_t));
  int64_t* order = (int64_t*)malloc(sizeof(int64_t) * (size_t)nn);
  for (int64_t i = 0; i < nn; ++i) start[b->ndepth[i] + 1] += 1;
  for (int d = 0; d <= D; ++d) start[d + 1] += start[d];
  int64_t* fill = (int64_t*)malloc(sizeof(int64_t) * ((size_t)D + 1));
  for (int d = 0; d <= D; ++d) fill[d] = start[d];
  for (int64_t i = 0; i < nn; ++i) order[fill[b->ndepth[i]]++] = i;
  for (int d = D; d >= 0; --d) {
    LevelJob j = {&x, order + start[d]};
    run_jobs(level_job, &j, start[d + 1] - start[d], 64);
  }
  free(fill);
  free(order);
  free(start);
  return 0;
}

void or_bvh_get_masks(const OrBvh* b, uint32_t* masks) {
  memcpy(masks, b->masks, sizeof(uint32_t) * (size_t)b->nnodes * 2 * b->W);
}

typedef struct {
  OrBvh* b;
  const uint32_t* req;
} EncodeJob;

static void encode_job(void* ctx, int64_t s) {
  EncodeJob* j = (EncodeJob*)ctx;
  j->b->cidx[s] = (uint8_t)or_encode(j->b->masks + (size_t)s * j->b->W, j->req, j->b->R, j->b->bits);
}

int or_bvh_compress(OrBvh* b, int K, int bits) {
  if (!b->masks || K < 1 || K > 256 || bits < 1 || bits > 16) return -1;
  int W = b->W, R = b->R;
  int64_t ns = b->nnodes * 2;
  free(b->clut);
  free(b->cidx);
  b->clut = (uint32_t*)calloc((size_t)K * W, sizeof(uint32_t));
  b->cidx = (uint8_t*)calloc((size_t)(ns > 0 ? ns : 1), 1);
  b->K = or_clut_build(b->masks, b->box, ns, R, K, b->clut, NULL);
  b->bits = bits;
  int nchunk = (R * R * R + bits - 1) / bits;
  uint32_t* req = (uint32_t*)malloc(sizeof(uint32_t) * (size_t)nchunk * (1u << bits) * 8);
  or_req_luts(b->clut, b->K, R, bits, req);
  EncodeJob j = {b, req};
  run_jobs(encode_job, &j, ns, 4096);
  free(req);
  return b->K;
}

void or_bvh_get_clut(const OrBvh* b, uint32_t* clut, uint8_t* idx) {
  if (clut) memcpy(clut, b->clut, sizeof(uint32_t) * (size_t)b->K * b->W);
  if (idx) memcpy(idx, b->cidx, (size_t)b->nnodes * 2);
}

/* --------------------------------------------- traversal (Alg. 1 + 4) --- */

/* Slab test: entry/exit distances of the ray with a box, clipped to
   [tmin, tcur]; the hit test widens the exit by 1 + 2*gamma_3 (rounded up
   to a float), after Ize, "Robust BVH Ray Traversal" (JCGT 2013), so that
   rounding never loses a box the ray touches.  The paper reuses these two
   distances as the segment ends p0, p1 for culling (Sec. 3.1.2). */
static const float ROBUST = 1.00000047683715820f; /* 1 + 4 * 2^-23 */

typedef struct {
  float o[3], d[3], inv[3], tmin, tmax;
} ORay;

static void load_ray(const float* r8, ORay* r) {
  for (int k = 0; k < 3; ++k) {
    r->o[k] = r8[k];
    r->d[k] = r8[4 + k];
    r->inv[k] = 1.0f / r8[4 + k];
  }
  r->tmin = r8[3];
  r->tmax = r8[7];
}

static int slab_test(const ORay* r, const float* bx, float tcur, float* tn_o,
                     float* tf_o) {
  float t0[3], t1[3];
  for (int k = 0; k < 3; ++k) {
    t0[k] = (bx[k] - r->o[k]) * r->inv[k];
    t1[k] = (bx[3 + k] - r->o[k]) * r->inv[k];
  }
  float tn = fmaxf(fmaxf(fminf(t0[0], t1[0]), fminf(t0[1], t1[1])),
                   fmaxf(fminf(t0[2], t1[2]), r->tmin));
  float tf = fminf(fminf(fmaxf(t0[0], t1[0]), fmaxf(t0[1], t1[1])),
                   fminf(fmaxf(t0[2], t1[2]), tcur));
  *tn_o = tn;
  *tf_o = tf;
  return tn <= tf * ROBUST;
}

int or_slab(const float* ray8, const float* box6, float tcur, float* tn,
            float* tf) {
  ORay r;
  load_ray(ray8, &r);
  return slab_test(&r, box6, tcur, tn, tf);
}

/* Alg. 1 cell index on one axis: min(floor(R/extent * (p - lower)), R-1),
   written as (p - lower) * (R / extent).  Additions (the paper is silent):
   a clamp at 0 (rounding can put p slightly below `lower`), and a floor of
   1e-30 on the extent for flat boxes. */
int or_cell(float p, float lo, float hi, int R) {
  float ext = hi - lo;
  float s = (float)R / fmaxf(ext, 1e-30f);
  float q = (p - lo) * s;
  q = fminf(fmaxf(q, -1.0f), (float)R);
  int i = (int)floorf(q);
  if (i < 0) i = 0;
  if (i > R - 1) i = R - 1;
  return i;
}

/* Moeller-Trumbore on (v0, e1 = v1 - v0, e2 = v2 - v0); the paper leaves the
   triangle test open (Alg. 4).  No epsilon on the determinant (thin slivers
   have tiny determinants); inclusive edges; accept tmin < t < tcur. */
static int mt_test(const ORay* r, const float* tri9, float tcur, float* t_o,
                   float* u_o, float* v_o) {
  float v0[3], e1[3], e2[3];
  for (int k = 0; k < 3; ++k) {
    v0[k] = tri9[k];
    e1[k] = tri9[3 + k] - tri9[k];
    e2[k] = tri9[6 + k] - tri9[k];
  }
  float p[3] = {r->d[1] * e2[2] - r->d[2] * e2[1], r->d[2] * e2[0] - r->d[0] * e2[2],
                r->d[0] * e2[1] - r->d[1] * e2[0]};
  float det = (e1[0] * p[0] + e1[1] * p[1]) + e1[2] * p[2];
  if (det == 0.0f) return 0;
  float inv = 1.0f / det;
  float s[3] = {r->o[0] - v0[0], r->o[1] - v0[1], r->o[2] - v0[2]};
  float u = ((s[0] * p[0] + s[1] * p[1]) + s[2] * p[2]) * inv;
  if (u < 0.0f || u > 1.0f) return 0;
  float q[3] = {s[1] * e1[2] - s[2] * e1[1], s[2] * e1[0] - s[0] * e1[2],
                s[0] * e1[1] - s[1] * e1[0]};
  float v = ((r->d[0] * q[0] + r->d[1] * q[1]) + r->d[2] * q[2]) * inv;
  if (v < 0.0f || u + v > 1.0f) return 0;
  float t = ((e2[0] * q[0] + e2[1] * q[1]) + e2[2] * q[2]) * inv;
  if (!(t > r->tmin && t < tcur)) return 0;
  *t_o = t;
  *u_o = u;
  *v_o = v;
  return 1;
}

int or_ray_tri(const float* ray8, const float* tri9, float tcur, float* t,
               float* u, float* v) {
  ORay r;
  load_ray(ray8, &r);
  return mt_test(&r, tri9, tcur, t, u, v);
}

/* Cell of the point at parameter t on one axis, Alg. 1 as written: the
   point p = o + t d (a product, then a sum: two roundings, no fused
   multiply-add), then floor(R/extent * (p - lower)) by or_cell, clamped to
   [0, R-1].  This is the traversal's default. */
int or_cell_at(float t, float o, float d, float lo, float hi, int R) {
  float p = o + t * d;
  return or_cell(p, lo, hi, R);
}

/* The same cell evaluated in the ray parameter instead (an option of the
   traversal, not the paper's order): q(t) = s (o - lower) + t (s d) with
   s = R / extent, as one fused multiply-add, fmaf(t, s*d, s*(o - lower)).
   It can differ from Alg. 1 only where q lies within rounding of a cell
   border; the eps dilation of the object masks keeps culling conservative
   either way.  Clamped to [0, R-1] like or_cell. */
int or_cell_t(float t, float o, float d, float lo, float hi, int R) {
  float ext = hi - lo;
  float s = (float)R / fmaxf(ext, 1e-30f);
  float q = fmaf(t, d * s, (o - lo) * s);
  q = fminf(fmaxf(q, -1.0f), (float)R);
  int i = (int)floorf(q);
  if (i < 0) i = 0;
  if (i > R - 1) i = R - 1;
  return i;
}

/* "Ideal" ray mask (the paper's Sec. 4.1 reference, which creates the ray
   mask by grid traversal): every cell whose closed box the segment [t0, t1]
   of the ray meets, in double.  Per axis k the ray's cell coordinate is
   u_k(t) = (o_k - lo_k) * s_k + t * d_k * s_k with s_k = R / extent; cell j
   spans [j, j+1] (the first and last cells extend to -inf / +inf, since the
   lookup path clamps the same way), and a cell is met iff the t-intervals
   of its three axes and [t0, t1] share a point.  A flat axis (extent 0)
   puts the segment in every cell along it. */
static void ideal_ray_mask(const ORay* r, const float* bx, float tn, float tf, int R,
                           uint32_t* m) {
  const int W = or_mask_words(R);
  const double t0 = tn, t1 = tf > tn ? tf : tn;
  double lo[3][8], hi[3][8];
  for (int k = 0; k < 3; ++k) {
    const double ext = (double)bx[3 + k] - (double)bx[k];
    for (int j = 0; j < R; ++j) {
      lo[k][j] = t0;
      hi[k][j] = t1;
    }
    if (!(ext > 0.0)) continue; /* flat: every cell along k */
    const double sk = (double)R / ext;
    const double a = ((double)r->o[k] - (double)bx[k]) * sk;
    const double bb = (double)r->d[k] * sk;
    for (int j = 0; j < R; ++j) {
      const double ulo = j == 0 ? -INFINITY : (double)j;
      const double uhi = j == R - 1 ? INFINITY : (double)(j + 1);
      if (bb == 0.0) {
        if (!(a >= ulo && a <= uhi)) { lo[k][j] = 1.0; hi[k][j] = 0.0; }
        continue;
      }
      double ta = (ulo - a) / bb, tb = (uhi - a) / bb;
      if (ta > tb) { const double x = ta; ta = tb; tb = x; }
      if (ta > lo[k][j]) lo[k][j] = ta;
      if (tb < hi[k][j]) hi[k][j] = tb;
    }
  }
  memset(m, 0, sizeof(uint32_t) * (size_t)W);
  for (int z = 0; z < R; ++z)
    for (int y = 0; y < R; ++y)
      for (int x = 0; x < R; ++x) {
        double l = lo[0][x], h = hi[0][x];
        if (lo[1][y] > l) l = lo[1][y];
        if (lo[2][z] > l) l = lo[2][z];
        if (hi[1][y] < h) h = hi[1][y];
        if (hi[2][z] < h) h = hi[2][z];
        /* a relative slack of 2^-40 keeps touching cells despite rounding */
        if (l <= h + 1e-12 * (1.0 + fabs(h))) {
          const int bit = cell_bit(R, x, y, z);
          m[bit >> 5] |= 1u << (bit & 31);
        }
      }
}

/* Cell of the point at parameter t on the 2R grid (R_ray = 2R, Sec. 4.2):
   twice the R-grid coordinate q, rounded down and clamped to [0, 2R-1].
   Doubling is exact, so the enclosing R cell is the Alg. 1 cell.  form 0
   (default): q = R/extent * (p - lower) with p = o + t d as in or_cell_at;
   form 1: q by the fused multiply-add of or_cell_t. */
int or_cell2_at(float t, float o, float d, float lo, float hi, int R, int form) {
  float ext = hi - lo;
  float s = (float)R / fmaxf(ext, 1e-30f);
  float q;
  if (form == 1) {
    q = fmaf(t, d * s, (o - lo) * s);
  } else {
    float p = o + t * d;
    q = (p - lo) * s;
  }
  q = 2.0f * q;
  q = fminf(fmaxf(q, -1.0f), (float)(2 * R));
  int i = (int)floorf(q);
  if (i < 0) i = 0;
  if (i > 2 * R - 1) i = 2 * R - 1;
  return i;
}

int or_cell2_t(float t, float o, float d, float lo, float hi, int R) {
  return or_cell2_at(t, o, d, lo, hi, R, 1);
}

/* Culling test of one child (Sec. 3.1.2 and the red part of Alg. 4): the
   ends of the clipped segment, at tn and tf, are turned into cells (Alg. 1:
   or_cell_at, or or_cell_t when the BVH's cell form is 1), the ray mask of
   the (begin, end) pair is looked up, and the child survives iff its AND
   with the object mask is non-zero. */
static int cell_of(const OrBvh* b, float t, float o, float d, float lo, float hi) {
  return b->cellform == 1 ? or_cell_t(t, o, d, lo, hi, b->R) : or_cell_at(t, o, d, lo, hi, b->R);
}

static int cull_pass(const OrBvh* b, const ORay* r, const float* bx, float tn,
                     float tf, const uint32_t* objmask) {
  int R = b->R, W = b->W, R3 = R * R * R;
  if (b->ideal) {
    uint32_t rm[16];
    ideal_ray_mask(r, bx, tn, tf, R, rm);
    for (int w = 0; w < W; ++w)
      if (rm[w] & objmask[w]) return 1;
    return 0;
  }
  if (b->raylut2r) {
    const int R2 = 2 * R, R23 = R2 * R2 * R2;
    int b2[3], e2[3];
    for (int k = 0; k < 3; ++k) {
      b2[k] = or_cell2_at(tn, r->o[k], r->d[k], bx[k], bx[3 + k], R, b->cellform);
      e2[k] = or_cell2_at(tf, r->o[k], r->d[k], bx[k], bx[3 + k], R, b->cellform);
    }
    const int beg = b2[0] + R2 * b2[1] + R2 * R2 * b2[2];
    const int end = e2[0] + R2 * e2[1] + R2 * R2 * e2[2];
    const uint32_t* rm = b->raylut2r + ((size_t)beg * R23 + end) * W;
    for (int w = 0; w < W; ++w)
      if (rm[w] & objmask[w]) return 1;
    return 0;
  }
  int cb[3], ce[3];
  for (int k = 0; k < 3; ++k) {
    cb[k] = cell_of(b, tn, r->o[k], r->d[k], bx[k], bx[3 + k]);
    ce[k] = cell_of(b, tf, r->o[k], r->d[k], bx[k], bx[3 + k]);
  }
  int beg = cell_bit(R, cb[0], cb[1], cb[2]);
  int end = cell_bit(R, ce[0], ce[1], ce[2]);
  const uint32_t* rm = b->raylut + ((size_t)beg * R3 + end) * W;
  for (int w = 0; w < W; ++w)
    if (rm[w] & objmask[w]) return 1;
  return 0;
}

typedef struct {
  int32_t child, count;
  float tn;
} StackEntry;

/* Seed of the second phase of a seeded traversal: the slot (child, count)
   whose subtree the first phase traced in full, and that phase's hit
   (id < 0: none). */
typedef struct {
  int32_t child, count;
  float t, u, v;
  int32_t id;
} Seed;

/*
 * Alg. 4 for one ray.  Readings where the paper is silent (it gives neither
 * child order nor pop rule): the root box is not tested; visiting an inner
 * node costs two slab tests (node_tests += 2); if both children survive, the
 * one with the smaller entry distance is visited next (tie: child 0) and the
 * other is pushed with its entry distance; a popped entry is dropped
 * without a test unless it would still pass the (widened) slab test, i.e.
 * unless tn <= tcur * (1 + 2 gamma_3) -- the same bound the slab test uses,
 * so a child is kept or dropped the same way whether it is reached directly
 * or through the stack; leaf
 * triangles are tested in order (tri_tests += 1 each).  Any-hit stops at the
 * first accepted triangle.  A child whose object mask has at least skip_bits
 * bits set is kept without a test (skip_bits = R^3: only an all-ones mask,
 * whose test cannot fail -- the paper's method exactly; smaller values skip
 * dense masks, which rarely cull), and an inner child at depth d is tested
 * only when d is a multiple of `stride` (1: every level, the paper's
 * method); a leaf child holding fewer than leaf_min triangles is kept
 * untested (0 or 1: every leaf is tested, the paper's method).  Skipping a
 * test only keeps a child, so hits are the same for every setting.
 */
static void trace_one(const OrBvh* b, const float* tris, const float* ray8,
                      int mode, int cull, int skip_bits, int stride, int leaf_min,
                      StackEntry* stack,
                      float* hit_t,
                      int32_t* hit_id, float* hit_uv, uint32_t* counts,
                      uint32_t* mtests, const Seed* seed) {
  ORay r;
  load_ray(ray8, &r);
  float tcur = r.tmax, bu = 0.0f, bv = 0.0f, bt = INFINITY;
  int32_t bid = -1;
  uint32_t ntest = 0, ttest = 0, mtest = 0;
  int sp = 0, have = b->ntri > 0, done = 0;
  int32_t cur_child = b->root_child, cur_count = b->root_count;
  /* seeded second phase: the seed hit is provisional, with t_max just
     above it, until the traversal reaches the seed slot in its own order */
  int prov = 0;
  if (seed && seed->id >= 0) {
    bt = seed->t; bid = seed->id; bu = seed->u; bv = seed->v;
    tcur = nextafterf(seed->t, INFINITY);
    prov = 1;
  }
  while (!done) {
    if (have) {
      if (seed && cur_child == seed->child && cur_count == seed->count) {
        if (prov) tcur = bt; /* the seed now counts as found here */
        have = 0;
        continue;
      } else if (cur_count > 0) {
        for (int32_t i = 0; i < cur_count; ++i) {
          int32_t tid = b->perm[cur_child + i];
          float t, u, v;
          ++ttest;
          if (mt_test(&r, tris + 9 * (size_t)tid, tcur, &t, &u, &v)) {
            bt = t; bid = tid; bu = u; bv = v;
            prov = 0;
            if (mode == 1) { done = 1; break; }
            tcur = t;
          }
        }
        have = 0;
        continue;
      }
      int64_t m = cur_child;
      float tn[2], tf[2];
      int hit[2];
      ntest += 2;
      for (int c = 0; c < 2; ++c)
        hit[c] = slab_test(&r, b->box + 12 * m + 6 * c, tcur, &tn[c], &tf[c]);
      if (cull) {
        for (int c = 0; c < 2; ++c) {
          if (!hit[c]) continue;
          const uint32_t* om =
              cull == 2 ? b->clut + (size_t)b->cidx[2 * m + c] * b->W
                        : b->masks + ((size_t)m * 2 + c) * b->W;
          if (popcount_mask(om, b->W) >= skip_bits) continue; /* kept untested */
          if (b->count[2 * m + c] == 0 && (b->ndepth[m] + 1) % stride != 0) continue;
          if (b->count[2 * m + c] > 0 && b->count[2 * m + c] < leaf_min) continue;
          ++mtest;
          hit[c] = cull_pass(b, &r, b->box + 12 * m + 6 * c, tn[c], tf[c], om);
        }
      }
      if (hit[0] && hit[1]) {
        int nr = tn[1] < tn[0] ? 1 : 0, fr = 1 - nr;
        stack[sp].child = b->child[2 * m + fr];
        stack[sp].count = b->count[2 * m + fr];
        stack[sp].tn = tn[fr];
        ++sp;
        cur_child = b->child[2 * m + nr];
        cur_count = b->count[2 * m + nr];
      } else if (hit[0] || hit[1]) {
        int c = hit[0] ? 0 : 1;
        cur_child = b->child[2 * m + c];
        cur_count = b->count[2 * m + c];
      } else {
        have = 0;
      }
      continue;
    }
    while (sp > 0) {
      --sp;
      if (stack[sp].tn > tcur * ROBUST) continue;
      cur_child = stack[sp].child;
      cur_count = stack[sp].count;
      have = 1;
      break;
    }
    if (!have) done = 1;
  }
  *hit_t = bt;
  *hit_id = bid;
  hit_uv[0] = bu;
  hit_uv[1] = bv;
  counts[0] = ntest;
  counts[1] = ttest;
  if (mtests) *mtests = mtest;
}

/* ------------------------------------------------------- 4-wide nodes --- */
/*
 * 4-wide BVH (the paper's node layout is 4-wide, Sec. 3.2.4 / Fig. 5),
 * made from the binary tree.  The 4-wide node made from binary node n takes,
 * in order, for each child slot c of n: the two child slots of c when c is
 * an inner node, else slot c itself -- 2 to 4 slots, each a slot (p, c) of
 * the binary tree, so it keeps that slot's box, object mask and LUT index.
 * An inner child slot (p, c) is the 4-wide node made from binary node
 * child[p][c].  4-wide nodes are numbered in pre-order (root node 0).
 */
static int64_t wide_rec(OrBvh* b, int64_t n, int depth) {
  int64_t q = b->nn4++;
  int k = 0;
  if (depth > b->w4depth) b->w4depth = depth;
  for (int c = 0; c < 2; ++c) {
    if (b->count[2 * n + c] == 0) {
      int64_t m = b->child[2 * n + c];
      for (int g = 0; g < 2; ++g) {
        b->w4p[4 * q + k] = m;
        b->w4c[4 * q + k] = g;
        ++k;
      }
    } else {
      b->w4p[4 * q + k] = n;
      b->w4c[4 * q + k] = c;
      ++k;
    }
  }
  b->w4n[q] = k;
  for (int i = 0; i < k; ++i) {
    int64_t p = b->w4p[4 * q + i];
    int c = b->w4c[4 * q + i];
    b->w4next[4 * q + i] =
        b->count[2 * p + c] == 0 ? wide_rec(b, b->child[2 * p + c], depth + 1) : -1;
  }
  return q;
}

int64_t or_bvh_wide(OrBvh* b) {
  if (b->w4n) return b->nn4;
  size_t cap = (size_t)(b->nnodes > 0 ? b->nnodes : 1);
  b->w4n = (int32_t*)calloc(cap, sizeof(int32_t));
  b->w4p = (int64_t*)calloc(4 * cap, sizeof(int64_t));
  b->w4c = (int32_t*)calloc(4 * cap, sizeof(int32_t));
  b->w4next = (int64_t*)calloc(4 * cap, sizeof(int64_t));
  b->nn4 = 0;
  b->w4depth = 0;
  if (b->ntri > 0 && b->root_count == 0) wide_rec(b, b->root_child, 0);
  return b->nn4;
}

void or_bvh_wide_export(const OrBvh* b, int32_t* n, int64_t* p, int32_t* c, int64_t* next) {
  if (n) memcpy(n, b->w4n, sizeof(int32_t) * (size_t)b->nn4);
  if (p) memcpy(p, b->w4p, sizeof(int64_t) * 4 * (size_t)b->nn4);
  if (c) memcpy(c, b->w4c, sizeof(int32_t) * 4 * (size_t)b->nn4);
  if (next) memcpy(next, b->w4next, sizeof(int64_t) * 4 * (size_t)b->nn4);
}

typedef struct {
  int64_t q;              /* 4-wide node, or -1: a leaf */
  int32_t first, count;   /* the leaf */
  float tn;
} Stack4;

/*
 * Alg. 4 on the 4-wide tree, with the readings of trace_one: the root is
 * not tested; a visited 4-wide node costs one slab test per child
 * (node_tests += its 2..4 children); the slab-passing children (after
 * their culling tests, eager, as in Alg. 4) are ordered by entry distance,
 * ties by position in the node; the nearest is visited next and the others
 * are pushed farthest first, so the second nearest is popped first; the
 * pop rule and the leaf tests are trace_one's.
 */
static void trace4_one(const OrBvh* b, const float* tris, const float* ray8, int mode,
                       int cull, int skip_bits, int stride, int leaf_min, Stack4* stack,
                       float* hit_t, int32_t* hit_id, float* hit_uv, uint32_t* counts,
                       uint32_t* mtests) {
  ORay r;
  load_ray(ray8, &r);
  float tcur = r.tmax, bu = 0.0f, bv = 0.0f, bt = INFINITY;
  int32_t bid = -1;
  uint32_t ntest = 0, ttest = 0, mtest = 0;
  int sp = 0, have = b->ntri > 0, done = 0;
  int64_t q = b->root_count == 0 ? 0 : -1;
  int32_t lf = b->root_child, lc = b->root_count;
  while (!done) {
    if (have) {
      if (q < 0) {
        for (int32_t i = 0; i < lc; ++i) {
          int32_t tid = b->perm[lf + i];
          float t, u, v;
          ++ttest;
          if (mt_test(&r, tris + 9 * (size_t)tid, tcur, &t, &u, &v)) {
            bt = t; bid = tid; bu = u; bv = v;
            if (mode == 1) { done = 1; break; }
            tcur = t;
          }
        }
        have = 0;
        continue;
      }
      const int k = b->w4n[q];
      float tn[4], tf[4];
      int hit[4], ord[4], nh = 0;
      ntest += (uint32_t)k;
      for (int i = 0; i < k; ++i) {
        const int64_t p = b->w4p[4 * q + i];
        const int c = b->w4c[4 * q + i];
        hit[i] = slab_test(&r, b->box + 12 * p + 6 * c, tcur, &tn[i], &tf[i]);
        if (hit[i] && cull) {
          const uint32_t* om = cull == 2 ? b->clut + (size_t)b->cidx[2 * p + c] * b->W
                                         : b->masks + ((size_t)p * 2 + c) * b->W;
          const int32_t cnt = b->count[2 * p + c];
          int test = popcount_mask(om, b->W) < skip_bits;
          if (cnt == 0 && (b->ndepth[p] + 1) % stride != 0) test = 0;
          if (cnt > 0 && cnt < leaf_min) test = 0;
          if (test) {
            ++mtest;
            hit[i] = cull_pass(b, &r, b->box + 12 * p + 6 * c, tn[i], tf[i], om);
          }
        }
        if (hit[i]) {
          /* insertion by (tn, position) */
          int j = nh++;
          while (j > 0 && tn[ord[j - 1]] > tn[i]) {
            ord[j] = ord[j - 1];
            --j;
          }
          ord[j] = i;
        }
      }
      if (nh == 0) {
        have = 0;
        continue;
      }
      for (int j = nh - 1; j >= 1; --j) {
        const int i = ord[j];
        const int64_t p = b->w4p[4 * q + i];
        const int c = b->w4c[4 * q + i];
        stack[sp].q = b->w4next[4 * q + i];
        stack[sp].first = b->child[2 * p + c];
        stack[sp].count = b->count[2 * p + c];
        stack[sp].tn = tn[i];
        ++sp;
      }
      {
        const int i = ord[0];
        const int64_t p = b->w4p[4 * q + i];
        const int c = b->w4c[4 * q + i];
        const int64_t nq = b->w4next[4 * q + i];
        lf = b->child[2 * p + c];
        lc = b->count[2 * p + c];
        q = nq;
      }
      continue;
    }
    while (sp > 0) {
      --sp;
      if (stack[sp].tn > tcur * ROBUST) continue;
      q = stack[sp].q;
      lf = stack[sp].first;
      lc = stack[sp].count;
      have = 1;
      break;
    }
    if (!have) done = 1;
  }
  *hit_t = bt;
  *hit_id = bid;
  hit_uv[0] = bu;
  hit_uv[1] = bv;
  counts[0] = ntest;
  counts[1] = ttest;
  if (mtests) *mtests = mtest;
}

int or_trace4_range(OrBvh* b, const float* tris, const float* rays, int64_t r_begin,
                    int64_t r_end, int mode, int cull, int skip_bits, int stride, int leaf_min,
                    float* hit_t, int32_t* hit_id, float* hit_uv, uint32_t* counts,
                    uint32_t* mask_tests) {
  if (stride < 1) return -3;
  if (cull && !b->masks) return -1;
  if (cull == 2 && !b->clut) return -2;
  if (cull && !b->raylut) {
    int R3 = b->R * b->R * b->R;
    uint32_t* lut = (uint32_t*)malloc(sizeof(uint32_t) * (size_t)R3 * R3 * b->W);
    or_raylut(b->R, lut);
    b->raylut = lut;
  }
  or_bvh_wide(b);
  Stack4* stack = (Stack4*)malloc(sizeof(Stack4) * (size_t)(3 * (b->w4depth + 2) + 4));
  for (int64_t i = r_begin; i < r_end; ++i)
    trace4_one(b, tris, rays + 8 * i, mode, cull, skip_bits, stride, leaf_min, stack,
               hit_t + i, hit_id + i, hit_uv + 2 * i, counts + 2 * i,
               mask_tests ? mask_tests + i : NULL);
  free(stack);
  return 0;
}

int or_trace_range(const OrBvh* b, const float* tris, const float* rays,
                   int64_t r_begin, int64_t r_end, int mode, int cull,
                   int skip_bits, int stride, int leaf_min, float* hit_t, int32_t* hit_id,
                   float* hit_uv,
                   uint32_t* counts, uint32_t* mask_tests) {
  if (stride < 1) return -3;
  if (cull && !b->masks) return -1;
  if (cull == 2 && !b->clut) return -2;
  if (cull && !b->raylut) {
    /* the ray-mask table is built once per resolution, on first use */
    int R3 = b->R * b->R * b->R;
    uint32_t* lut = (uint32_t*)malloc(sizeof(uint32_t) * (size_t)R3 * R3 * b->W);
    or_raylut(b->R, lut);
    ((OrBvh*)b)->raylut = lut;
  }
  StackEntry* stack =
      (StackEntry*)malloc(sizeof(StackEntry) * (size_t)(b->max_depth + 4));
  for (int64_t i = r_begin; i < r_end; ++i)
    trace_one(b, tris, rays + 8 * i, mode, cull, skip_bits, stride, leaf_min, stack, hit_t + i,
              hit_id + i,
              hit_uv + 2 * i, counts + 2 * i, mask_tests ? mask_tests + i : NULL, NULL);
  free(stack);
  return 0;
}

int or_trace(const OrBvh* b, const float* tris, const float* rays, int64_t n,
             int mode, int cull, float* hit_t, int32_t* hit_id, float* hit_uv,
             uint32_t* counts, uint32_t* mask_tests) {
  int R3 = b->R * b->R * b->R;
  return or_trace_range(b, tris, rays, 0, n, mode, cull, R3, 1, 0, hit_t, hit_id, hit_uv,
                        counts, mask_tests);
}

/* Closest (or any) hit by testing every triangle, lowest index first. */
void or_brute(const float* tris, int64_t ntri, const float* rays, int64_t n,
              int mode, float* hit_t, int32_t* hit_id, float* t2) {
  for (int64_t i = 0; i < n; ++i) {
    ORay r;
    load_ray(rays + 8 * i, &r);
    float best = INFINITY, second = INFINITY;
    int32_t bid = -1;
    for (int64_t j = 0; j < ntri; ++j) {
      float t, u, v;
      if (!mt_test(&r, tris + 9 * j, r.tmax, &t, &u, &v)) continue;
      if (t < best) {
        second = best;
        best = t;
        bid = (int32_t)j;
        if (mode == 1) break;
      } else if (t < second) {
        second = t;
      }
    }
    hit_t[i] = best;
    hit_id[i] = bid;
    if (t2) t2[i] = second;
  }
}

/* --------------------------------------------- diffuse bounce rays (waves) --- */
/*
 * Not part of the paper (its path tracer is unspecified beyond "path tracing
 * with 16 samples per pixel", Sec. 4): the wave workloads spawn one
 * cosine-weighted diffuse bounce per hit.  Random numbers come from a
 * counter-based hash, the PCG-based hash of Jarzynski & Olano, "Hash
 * Functions for GPU Rendering" (JCGT 9(3), 2020), restated from its
 * definition: state = v * 747796405 + 2891336453; word = ((state >>
 * ((state >> 28) + 4)) ^ state) * 277803737; result = (word >> 22) ^ word.
 */
uint32_t or_pcg_hash(uint32_t v) {
  uint32_t state = v * 747796405u + 2891336453u;
  uint32_t word = ((state >> ((state >> 28u) + 4u)) ^ state) * 277803737u;
  return (word >> 22u) ^ word;
}

uint32_t or_bounce_hash(uint32_t seed, uint32_t rid, uint32_t bounce, uint32_t k) {
  return or_pcg_hash(or_pcg_hash(or_pcg_hash(seed ^ (bounce << 24)) + rid) + k);
}

/*
 * Bounce ray from a hit: origin o + t*d; geometric normal cross(e1, e2)
 * turned against d and normalised; an orthonormal frame from cross products;
 * a point of the unit disk by rejection (at most 64 tries, else the centre)
 * lifted to the hemisphere (Malley's method gives a cosine-weighted
 * direction); tmin = 1e-4, tmax = +inf.  Float ops only, each correctly
 * rounded (sqrt included), so the GPU produces the same bits.  Returns 0 for
 * a degenerate triangle (no bounce).
 */
int or_bounce(const float* ray8, float t, const float* tri9, uint32_t seed,
              uint32_t rid, uint32_t bounce, float* out8) {
  float o[3] = {ray8[0], ray8[1], ray8[2]}, d[3] = {ray8[4], ray8[5], ray8[6]};
  float p[3], e1[3], e2[3], n[3];
  for (int k = 0; k < 3; ++k) {
    p[k] = o[k] + t * d[k];
    e1[k] = tri9[3 + k] - tri9[k];
    e2[k] = tri9[6 + k] - tri9[k];
  }
  n[0] = e1[1] * e2[2] - e1[2] * e2[1];
  n[1] = e1[2] * e2[0] - e1[0] * e2[2];
  n[2] = e1[0] * e2[1] - e1[1] * e2[0];
  if ((n[0] * d[0] + n[1] * d[1]) + n[2] * d[2] > 0.0f) {
    n[0] = -n[0]; n[1] = -n[1]; n[2] = -n[2];
  }
  float l2 = (n[0] * n[0] + n[1] * n[1]) + n[2] * n[2];
  if (!(l2 > 0.0f)) return 0;
  float l = sqrtf(l2);
  for (int k = 0; k < 3; ++k) n[k] = n[k] / l;
  float a[3] = {0.0f, 0.0f, 0.0f};
  if (fabsf(n[0]) > 0.9f) a[1] = 1.0f; else a[0] = 1.0f;
  float t1[3] = {a[1] * n[2] - a[2] * n[1], a[2] * n[0] - a[0] * n[2],
                 a[0] * n[1] - a[1] * n[0]};
  float m = sqrtf((t1[0] * t1[0] + t1[1] * t1[1]) + t1[2] * t1[2]);
  for (int k = 0; k < 3; ++k) t1[k] = t1[k] / m;
  float t2[3] = {n[1] * t1[2] - n[2] * t1[1], n[2] * t1[0] - n[0] * t1[2],
                 n[0] * t1[1] - n[1] * t1[0]};
  float x = 0.0f, y = 0.0f, r2 = 0.0f;
  for (uint32_t k = 0; k < 64; ++k) {
    float u1 = (float)(or_bounce_hash(seed, rid, bounce, 2 * k) >> 8) * 5.9604644775390625e-08f;
    float u2 = (float)(or_bounce_hash(seed, rid, bounce, 2 * k + 1) >> 8) * 5.9604644775390625e-08f;
    float xx = 2.0f * u1 - 1.0f, yy = 2.0f * u2 - 1.0f;
    float rr = xx * xx + yy * yy;
    if (rr < 1.0f) { x = xx; y = yy; r2 = rr; break; }
  }
  float z = sqrtf(1.0f - r2);
  for (int k = 0; k < 3; ++k) {
    out8[k] = p[k];
    out8[4 + k] = (x * t1[k] + y * t2[k]) + z * n[k];
  }
  out8[3] = 1e-4f;
  out8[7] = INFINITY;
  return 1;
}

/* ------------------------------------------------ learned-proposal seeds --- */
/* Not in the paper.  Frontier of depth D: the slots at depth D below the
   root (root slot depth 0) and leaf slots reached earlier, in pre-order
   (left child first), with the box each slot's parent stores for it (the
   root box for the root slot).  Returns their number; class_of_tri (or
   NULL) gets the frontier index of every triangle id. */
static void frontier_rec(const OrBvh* b, int32_t child, int32_t count, const float* box,
                         int depth, int D, int32_t* fc, int32_t* fn, float* fbox, int* n,
                         uint8_t* cls) {
  if (count > 0 || depth == D) {
    fc[*n] = child;
    fn[*n] = count;
    if (fbox) memcpy(fbox + 6 * *n, box, 6 * sizeof(float));
    if (cls) {
      /* every triangle below this slot */
      int32_t stack_c[128], stack_n[128];
      int sp = 0;
      stack_c[sp] = child; stack_n[sp] = count; ++sp;
      while (sp > 0) {
        --sp;
        int32_t c = stack_c[sp], k = stack_n[sp];
        if (k > 0) {
          for (int32_t i = 0; i < k; ++i) cls[b->perm[c + i]] = (uint8_t)*n;
        } else {
          stack_c[sp] = b->child[2 * c]; stack_n[sp] = b->count[2 * c]; ++sp;
          stack_c[sp] = b->child[2 * c + 1]; stack_n[sp] = b->count[2 * c + 1]; ++sp;
        }
      }
    }
    ++*n;
    return;
  }
  for (int c = 0; c < 2; ++c)
    frontier_rec(b, b->child[2 * child + c], b->count[2 * child + c],
                 b->box + 12 * (size_t)child + 6 * c, depth + 1, D, fc, fn, fbox, n, cls);
}

int or_bvh_frontier(const OrBvh* b, int D, int32_t* fchild, int32_t* fcount, float* fbox,
                    uint8_t* cls) {
  int n = 0;
  if (b->ntri == 0) return 0;
  frontier_rec(b, b->root_child, b->root_count, b->root_box, 0, D, fchild, fcount, fbox, &n,
               cls);
  return n;
}

/* Seeded closest-hit traversal.  A class outside [0, nf) means no seed:
   the plain traversal.  Otherwise the seed slot's box is slab-tested with
   the ray's tmax (one node test); if the ray enters it, phase 1 traverses
   that subtree with the ray's tmax.  Phase 2 traverses from the root,
   skipping the seed slot (phase 1 covered it, or the ray misses its box):
   if phase 1 hit at t_s, phase 2 starts with that hit, held provisionally
   with tmax = nextafterf(t_s, +inf) so that an equally distant triangle
   met earlier in traversal order replaces it, and lowers tmax to t_s when
   it reaches the seed slot; else it starts with the ray's tmax.  The
   result is the plain traversal's closest hit; counts sum both phases. */
int or_trace_seeded(const OrBvh* b, const float* tris, const float* rays, int64_t n,
                    int cull, int skip_bits, int stride, int leaf_min, const int32_t* cls,
                    const int32_t* fchild, const int32_t* fcount, const float* fbox, int nf,
                    float* hit_t, int32_t* hit_id, float* hit_uv, uint32_t* counts) {
  if (stride < 1) return -3;
  if (cull && !b->masks) return -1;
  if (cull == 2 && !b->clut) return -2;
  if (cull && !b->raylut) {
    int R3 = b->R * b->R * b->R;
    uint32_t* lut = (uint32_t*)malloc(sizeof(uint32_t) * (size_t)R3 * R3 * b->W);
    or_raylut(b->R, lut);
    ((OrBvh*)b)->raylut = lut;
  }
  StackEntry* stack = (StackEntry*)malloc(sizeof(StackEntry) * (size_t)(b->max_depth + 4));
  OrBvh sub = *b; /* a view whose root is the seed slot */
  for (int64_t i = 0; i < n; ++i) {
    const float* r8 = rays + 8 * i;
    float t1 = INFINITY, uv1[2] = {0.0f, 0.0f}, t2, uv2[2];
    int32_t id1 = -1, id2;
    uint32_t c1[2] = {0, 0}, c2[2], mt;
    int k = cls[i];
    if (k < 0 || k >= nf) {
      trace_one(b, tris, r8, 0, cull, skip_bits, stride, leaf_min, stack, &t2, &id2, uv2, c2,
                &mt, NULL);
    } else {
      ORay r;
      float tn, tf;
      load_ray(r8, &r);
      c1[0] = 1;
      if (slab_test(&r, fbox + 6 * (size_t)k, r.tmax, &tn, &tf)) {
        uint32_t cs[2];
        sub.root_child = fchild[k];
        sub.root_count = fcount[k];
        trace_one(&sub, tris, r8, 0, cull, skip_bits, stride, leaf_min, stack, &t1, &id1, uv1,
                  cs, &mt,
                  NULL);
        c1[0] += cs[0];
        c1[1] += cs[1];
      }
      Seed sd;
      sd.child = fchild[k];
      sd.count = fcount[k];
      sd.t = t1; sd.u = uv1[0]; sd.v = uv1[1]; sd.id = id1;
      trace_one(b, tris, r8, 0, cull, skip_bits, stride, leaf_min, stack, &t2, &id2, uv2, c2,
                &mt, &sd);
    }
    hit_t[i] = t2;
    hit_id[i] = id2;
    if (hit_uv) { hit_uv[2 * i] = uv2[0]; hit_uv[2 * i + 1] = uv2[1]; }
    counts[2 * i] = c1[0] + c2[0];
    counts[2 * i + 1] = c1[1] + c2[1];
  }
  free(stack);
  return 0;
}
