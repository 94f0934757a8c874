/*
 * scenegen.h — seeded synthetic inputs (triangles and rays).
 *
 * This module produces the *inputs* of the traversal path and holds none of
 * the method's arithmetic: no boxes, masks, lookup tables or intersection
 * tests.  It is compiled into the product library (behind sc_scene_generate /
 * sc_rays_generate) and, separately, into a stand-alone library that the CPU
 * oracle's tests use, so both sides consume byte-identical buffers.
 *
 * Determinism: every value is computed in IEEE double with correctly rounded
 * + - * / sqrt only (built with -ffp-contract=off), then rounded once to
 * float.  sin/cos/exp are evaluated by this module's own series so that x86
 * and Arm hosts produce the same bits (no libm in the data path).
 *
 * Random numbers: SplitMix64 derives the stream seeds of a PCG32 generator
 * (O'Neill, "PCG: A Family of Simple Fast Space-Efficient Statistically Good
 * Algorithms for Random Number Generation", 2014, pcg32 XSH-RR); a uniform
 * double is (u32 >> 8) * 2^-24.
 *
 * Layouts:
 *   triangles: float[n][9] = v0.xyz, v1.xyz, v2.xyz; the triangle id is its
 *              index in this array.
 *   rays:      float[n][8] = o.xyz, tmin, d.xyz, tmax.
 */
#ifndef SUBCULL_SCENEGEN_H
#define SUBCULL_SCENEGEN_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Number of triangles of the hair scene: strands * segs * 2, plus 2 for the
   ground quad when ground != 0. */
int64_t sg_hair_count(int64_t strands, int segs, int ground);

/* Curly-hair scene.  Strand s (0 <= s < strands) has its root uniform on the
   unit sphere (outward normal n), and follows a helix of radius 0.02 and
   pitch 0.05 for an axial length 0.5 along n, sampled at segs+1 points; each
   segment is a ribbon quad of width 1e-3 split into two triangles.
   Triangle index of (strand s, segment k, half j) = 2*(s*segs + k) + j.
   Writes strands [s_begin, s_end) only (so callers may split the work); the
   ground quad (y = -1.2, x,z in [-4,4]) occupies the last two triangles and
   is written by the call whose s_end == strands when ground != 0. */
void sg_hair(uint64_t seed, int64_t strands, int segs, int ground,
             int64_t s_begin, int64_t s_end, float* tris);

/* Triangle soup in the unit cube: alternate triangles are thin slivers
   (aspect 1:1000, long axis uniform on the sphere) and axis-aligned right
   triangles ("slabs"); edge length log-uniform in [1e-4, 1e-1].
   Writes triangles [i_begin, i_end). */
void sg_soup(uint64_t seed, int64_t i_begin, int64_t i_end, float* tris);

/* Pinhole camera: eye (0,0,3) looking at the origin, up +y, vertical field
   of view 40 degrees, pixel centres.  Rays are emitted in 8x4-pixel tile
   order (tiles row-major, pixels row-major inside a tile), which keeps each
   32-ray group spatially coherent.  tmin = 0, tmax = +inf.
   If pix != NULL, pix[r] = row * W + column of ray r.
   jitter_seed != 0 replaces the pixel centre by a uniform sub-pixel sample
   drawn from stream (jitter_seed, pixel). */
void sg_rays_pinhole(int W, int H, uint64_t jitter_seed, float* rays,
                     int32_t* pix);

/* Random rays: origin uniform in [0,1]^3, direction uniform on the sphere,
   tmin = 0, tmax = +inf.  Writes rays [r_begin, r_end). */
void sg_rays_random(uint64_t seed, int64_t r_begin, int64_t r_end,
                    float* rays);

/* Uniform double in [0,1) from stream (seed, stream), draw k (k >= 0):
   exposed so tests can check the generator against its definition. */
double sg_uniform(uint64_t seed, uint64_t stream, int k);

/* This module's own sin/cos/exp (double). */
void sg_sincos(double x, double* s, double* c);
double sg_exp(double x);

#ifdef __cplusplus
}
#endif
#endif
