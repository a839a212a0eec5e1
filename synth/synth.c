/*
 * Seeded synthetic particle sets for the short-range P3M force.
 *
 * This module only draws random numbers and places particles; it holds none
 * of the force, sort, rung or kick arithmetic, so that the CUDA path and the
 * CPU oracle can both be fed from it without sharing any of the method.
 *
 * Workload shape (stand-in for the cosmological snapshots of Section 3, which
 * are not available here): a fraction of the particles is uniform in the unit
 * box, the rest is spread over Plummer spheres (the density profile implied
 * by the Plummer shape of Section 2.1.1), with per-sphere scale b either fixed
 * or log-uniform in [b_lo, b_hi].  Radii are drawn by inverting the Plummer
 * mass profile M(<r) = r^3 / (r^2 + b^2)^{3/2}; draws beyond r_max are redrawn.
 *
 * Random numbers: every particle (and every sphere) owns an independent
 * xoshiro256** stream whose 256-bit state is filled by SplitMix64 from
 * (seed, stream id).  Particle i uses stream i, sphere k uses stream n + k.
 * The result is therefore independent of the number of threads.
 */
#include <stdint.h>
#include <math.h>

typedef struct { uint64_t s[4]; } rng_t;

static uint64_t splitmix64(uint64_t* z) {
  uint64_t r = (*z += 0x9E3779B97F4A7C15ULL);
  r = (r ^ (r >> 30)) * 0xBF58476D1CE4E5B9ULL;
  r = (r ^ (r >> 27)) * 0x94D049BB133111EBULL;
  return r ^ (r >> 31);
}

static void rng_seed(rng_t* g, uint64_t seed, uint64_t stream) {
  uint64_t z = seed * 0xD1B54A32D192ED03ULL ^ (stream + 1) * 0xAEF17502108EF2D9ULL;
  for (int k = 0; k < 4; ++k) g->s[k] = splitmix64(&z);
}

static inline uint64_t rotl(uint64_t x, int k) { return (x << k) | (x >> (64 - k)); }

static uint64_t rng_next(rng_t* g) {
  uint64_t* s = g->s;
  const uint64_t result = rotl(s[1] * 5, 7) * 9;
  const uint64_t t = s[1] << 17;
  s[2] ^= s[0]; s[3] ^= s[1]; s[1] ^= s[2]; s[0] ^= s[3];
  s[2] ^= t; s[3] = rotl(s[3], 45);
  return result;
}

/* uniform double in [0, 1) with 53 random bits */
static double u01(rng_t* g) { return (double)(rng_next(g) >> 11) * 0x1.0p-53; }
/* uniform double in (0, 1] */
static double u01_open0(rng_t* g) { return (double)((rng_next(g) >> 11) + 1) * 0x1.0p-53; }

static double wrap01(double v) {
  double w = v - floor(v);
  return (w >= 1.0 || w < 0.0) ? 0.0 : w;
}

/* Sphere k: centre (3 uniforms) and scale b (log-uniform in [b_lo, b_hi]). */
static void sphere_params(uint64_t seed, int64_t n, int64_t k, double b_lo, double b_hi,
                          double* c, double* b) {
  rng_t g; rng_seed(&g, seed, (uint64_t)(n + k));
  c[0] = u01(&g); c[1] = u01(&g); c[2] = u01(&g);
  double u = u01(&g);
  *b = (b_hi > b_lo) ? exp(log(b_lo) + u * (log(b_hi) - log(b_lo))) : b_lo;
}

/*
 * Fill x, y, z (each n doubles, structure of arrays) with positions in [0,1).
 * Particles 0 .. n_u-1 (n_u = llround(frac_uniform * n)) are uniform; the rest
 * belong to n_spheres Plummer spheres.  Returns the number of uniform particles.
 */
int64_t synth_positions(int64_t n, uint64_t seed, double frac_uniform, int64_t n_spheres,
                        double b_lo, double b_hi, double r_max,
                        double* x, double* y, double* z) {
  int64_t n_u = llround(frac_uniform * (double)n);
  if (n_spheres <= 0) n_u = n;
  const double two_pi = 6.283185307179586476925286766559;
#pragma omp parallel for schedule(static)
  for (int64_t i = 0; i < n; ++i) {
    rng_t g; rng_seed(&g, seed, (uint64_t)i);
    if (i < n_u) {
      x[i] = u01(&g); y[i] = u01(&g); z[i] = u01(&g);
      continue;
    }
    int64_t k = (int64_t)(u01(&g) * (double)n_spheres);
    if (k >= n_spheres) k = n_spheres - 1;
    double c[3], b;
    sphere_params(seed, n, k, b_lo, b_hi, c, &b);
    double r;
    for (;;) {
      double U = u01_open0(&g);
      double d = pow(U, -2.0 / 3.0) - 1.0;
      r = (d > 0.0) ? b / sqrt(d) : INFINITY;
      if (r <= r_max) break;
    }
    double cz = 2.0 * u01(&g) - 1.0;
    double ph = two_pi * u01(&g);
    double st = sqrt(fmax(0.0, 1.0 - cz * cz));
    x[i] = wrap01(c[0] + r * st * cos(ph));
    y[i] = wrap01(c[1] + r * st * sin(ph));
    z[i] = wrap01(c[2] + r * cz);
  }
  return n_u;
}

/* n doubles uniform in [lo, hi) from stream (stream_base + i). */
void synth_uniform(int64_t n, uint64_t seed, uint64_t stream_base, double lo, double hi, double* out) {
#pragma omp parallel for schedule(static)
  for (int64_t i = 0; i < n; ++i) {
    rng_t g; rng_seed(&g, seed, stream_base + (uint64_t)i);
    out[i] = lo + (hi - lo) * u01(&g);
  }
}

/* n small integers uniform in [0, m) from stream (stream_base + i). */
void synth_uniform_int8(int64_t n, uint64_t seed, uint64_t stream_base, int m, int8_t* out) {
#pragma omp parallel for schedule(static)
  for (int64_t i = 0; i < n; ++i) {
    rng_t g; rng_seed(&g, seed, stream_base + (uint64_t)i);
    int v = (int)(u01(&g) * (double)m);
    out[i] = (int8_t)(v >= m ? m - 1 : v);
  }
}
