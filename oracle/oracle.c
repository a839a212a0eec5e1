/*
 * CPU oracle for the short-range P3M particle-particle force.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product library calls, links or
 * loads this file; only the tests, the smoke check and the benchmark's CPU
 * baseline leg do.  It shares no code, header, table or constant generator with
 * the CUDA path: every formula below is written out again from the paper.
 *
 * Everything is IEEE double precision, compiled with -ffp-contract=off so that
 * the integer decisions (subtile ids, rungs) follow the exact operation order
 * written here.
 *
 * What is computed (Section 2.1.3, Eq. p3m_gravity, lower "short-range" half):
 *
 *   a_i = -G m  sum_{j != i, |x_ij| < x_r}  B(|x_ij|) x_ij ,
 *
 *   B(r) = erfc(u)/r^3 + exp(-u^2)/(sqrt(pi) x_s r^2) + ( |x|^{-3}_shape - r^{-3} ),
 *   u = r / (2 x_s),
 *
 * with x_ij the nearest periodic image of x_i - x_j (Section 2.1.3: only the
 * nearest image n' contributes since x_r < L/2).  Accelerations a_i = f_i / m
 * are returned (units L = 1 by default, G m = G_m passed in).
 *
 * Softening shapes (Section 2.1.1):
 *   0  point particles   |x|^{-3}_delta = r^{-3}                    (Eq. force)
 *   1  Plummer           |x|^{-3}_P = (r^2 + eps^2)^{-3/2}          (Eq. plummer_shape)
 *   2  B-spline          |x|^{-3}_B piecewise in x_B = r / eps_B,   (Eq. bspline_force)
 *                        eps_B = 2.8 eps, zero softening for r >= eps_B.
 *
 * Where the plain formula cancels catastrophically (r much smaller than the
 * softening length, where erfc(u)/r^3 and -r^{-3} are both huge), the oracle
 * uses the exact identity
 *
 *   erfc(u) + 2u/sqrt(pi) e^{-u^2} - 1 = -u^3 h(u),
 *   h(u) = [erf(u) - 2u/sqrt(pi) e^{-u^2}] / u^3
 *        = (2/sqrt(pi)) sum_{n>=1} (-1)^{n+1} 2n / (n! (2n+1)) u^{2n-2},
 *
 * so that B(r) = |x|^{-3}_shape - h(u) / (2 x_s)^3.  The series follows from
 * the Taylor series of erf(u) and of u e^{-u^2}, subtracted term by term.
 * This rewrite is used for r < r_sw, where r_sw = eps_B (B-spline) or 2.8 eps
 * (Plummer); point particles always use the plain formula.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define ORACLE_PI 3.14159265358979323846264338327950288

/* ------------------------------------------------------------------------- */
/* Softening shapes |x|^{-3}_shape and their r-derivatives (Section 2.1.1).   */
/* ------------------------------------------------------------------------- */

/* Eq. bspline_force: |x|^{-3}_B for x_B = r/eps_B < 1 (caller handles >= 1). */
static double bspline_inv3(double r, double eps_B) {
  double xb = r / eps_B;
  double c = 32.0 / (eps_B * eps_B * eps_B);
  if (xb < 0.5) return c * (xb * xb * xb - 1.2 * xb * xb + 1.0 / 3.0);
  return c * (-xb * xb * xb / 3.0 + 1.2 * xb * xb - 1.5 * xb + 2.0 / 3.0
              - 1.0 / (480.0 * xb * xb * xb));
}

/* d/dr of Eq. bspline_force for r < eps_B. */
static double bspline_inv3_dr(double r, double eps_B) {
  double xb = r / eps_B;
  double c = 32.0 / (eps_B * eps_B * eps_B * eps_B);
  if (xb < 0.5) return c * (3.0 * xb * xb - 2.4 * xb);
  return c * (-xb * xb + 2.4 * xb - 1.5 + 1.0 / (160.0 * xb * xb * xb * xb));
}

/* Eq. plummer_shape cubed: (r^2 + eps^2)^{-3/2}. */
static double plummer_inv3(double r, double eps) {
  double s = r * r + eps * eps;
  return 1.0 / (s * sqrt(s));
}

static double plummer_inv3_dr(double r, double eps) {
  double s = r * r + eps * eps;
  return -3.0 * r / (s * s * sqrt(s));
}

/* ------------------------------------------------------------------------- */
/* h(u) = [erf(u) - 2u/sqrt(pi) exp(-u^2)] / u^3 and h'(u).                   */
/* ------------------------------------------------------------------------- */

static double h_series(double u) {
  /* (2/sqrt(pi)) sum_{n>=1} (-1)^{n+1} 2n/(n!(2n+1)) u^{2n-2} */
  double u2 = u * u, term_pow = 1.0, fact = 1.0, sum = 0.0;
  for (int n = 1; n <= 30; ++n) {
    fact *= (double)n;
    double c = ((n & 1) ? 1.0 : -1.0) * (2.0 * n) / (fact * (2.0 * n + 1.0));
    sum += c * term_pow;
    term_pow *= u2;
  }
  return 2.0 / sqrt(ORACLE_PI) * sum;
}

static double h_series_du(double u) {
  double u2 = u * u, fact = 1.0, sum = 0.0;
  double upow = u; /* u^{2n-3} for n = 2 */
  fact = 1.0;
  for (int n = 1; n <= 30; ++n) {
    fact *= (double)n;
    if (n >= 2) {
      double c = ((n & 1) ? 1.0 : -1.0) * (2.0 * n) / (fact * (2.0 * n + 1.0));
      sum += c * (2.0 * n - 2.0) * upow;
      upow *= u2;
    }
  }
  return 2.0 / sqrt(ORACLE_PI) * sum;
}

/* h(u) for any u >= 0: the series where it converges quickly, else the plain
 * expression (no cancellation once u is of order one). */
static double h_of_u(double u) {
  if (u < 0.5) return h_series(u);
  return (erf(u) - 2.0 * u / sqrt(ORACLE_PI) * exp(-u * u)) / (u * u * u);
}

static double h_of_u_du(double u) {
  if (u < 0.5) return h_series_du(u);
  /* d/du [N(u)/u^3] with N = erf(u) - 2u/sqrt(pi) e^{-u^2}, N' = 4u^2/sqrt(pi) e^{-u^2} */
  double N = erf(u) - 2.0 * u / sqrt(ORACLE_PI) * exp(-u * u);
  double dN = 4.0 * u * u / sqrt(ORACLE_PI) * exp(-u * u);
  return dN / (u * u * u) - 3.0 * N / (u * u * u * u);
}

/* ------------------------------------------------------------------------- */
/* The bracket B(r) of Eq. p3m_gravity and its derivative.                    */
/* ------------------------------------------------------------------------- */

static double switch_radius(int softening, double eps) {
  if (softening == 2 || softening == 1) return 2.8 * eps;
  return 0.0;
}

static double shape_inv3(double r, int softening, double eps) {
  if (softening == 1) return plummer_inv3(r, eps);
  if (softening == 2) {
    double eps_B = 2.8 * eps;
    return (r < eps_B) ? bspline_inv3(r, eps_B) : 1.0 / (r * r * r);
  }
  return 1.0 / (r * r * r);
}

static double shape_inv3_dr(double r, int softening, double eps) {
  if (softening == 1) return plummer_inv3_dr(r, eps);
  if (softening == 2) {
    double eps_B = 2.8 * eps;
    return (r < eps_B) ? bspline_inv3_dr(r, eps_B) : -3.0 / (r * r * r * r);
  }
  return -3.0 / (r * r * r * r);
}

/* B(r) (without the -G m factor).  r > 0 unless the shape is softened. */
double oracle_bracket(double r, double x_s, int softening, double eps) {
  double u = r / (2.0 * x_s);
  if (r < switch_radius(softening, eps)) {
    double w = 2.0 * x_s;
    return shape_inv3(r, softening, eps) - h_of_u(u) / (w * w * w);
  }
  double r3 = r * r * r;
  double plain = erfc(u) / r3 + exp(-u * u) / (sqrt(ORACLE_PI) * x_s * r * r);
  if (softening == 0) return plain;
  return plain + (shape_inv3(r, softening, eps) - 1.0 / r3);
}

/* dB/dr. */
double oracle_bracket_dr(double r, double x_s, int softening, double eps) {
  double u = r / (2.0 * x_s);
  if (r < switch_radius(softening, eps)) {
    double w = 2.0 * x_s;
    return shape_inv3_dr(r, softening, eps) - h_of_u_du(u) / (w * w * w * w);
  }
  /* g(r) = [erfc(u) + 2u/sqrt(pi) e^{-u^2}] / r^3,
   * g'(r) = -3 g / r - (2 u^2 / (sqrt(pi) x_s)) e^{-u^2} / r^3 */
  double r3 = r * r * r;
  double g = (erfc(u) + 2.0 * u / sqrt(ORACLE_PI) * exp(-u * u)) / r3;
  double dg = -3.0 * g / r - 2.0 * u * u / (sqrt(ORACLE_PI) * x_s) * exp(-u * u) / r3;
  if (softening == 0) return dg;
  return dg + shape_inv3_dr(r, softening, eps) + 3.0 / (r3 * r);
}

/* ------------------------------------------------------------------------- */
/* Cell lists (the oracle's own; cell side >= x_r) and the neighbour walk.    */
/* ------------------------------------------------------------------------- */

typedef struct {
  int nc;            /* cells per dimension = floor(L / x_r) */
  int64_t* head;     /* nc^3 heads, -1 terminated */
  int64_t* next;     /* n links */
} cells_t;

static int cell_coord(double v, double box, int nc) {
  int c = (int)floor(v / box * (double)nc);
  if (c < 0) c = 0;
  if (c >= nc) c = nc - 1;
  return c;
}

static int cells_build(cells_t* cl, int64_t n, const double* x, const double* y, const double* z,
                       double box, double x_r) {
  int nc = (int)floor(box / x_r);
  if (nc < 3) return -1;
  cl->nc = nc;
  int64_t ncell = (int64_t)nc * nc * nc;
  cl->head = (int64_t*)malloc(sizeof(int64_t) * ncell);
  cl->next = (int64_t*)malloc(sizeof(int64_t) * (n > 0 ? n : 1));
  if (!cl->head || !cl->next) return -2;
  for (int64_t c = 0; c < ncell; ++c) cl->head[c] = -1;
  /* insert in reverse so each list is in increasing index order */
  for (int64_t i = n - 1; i >= 0; --i) {
    int cx = cell_coord(x[i], box, nc), cy = cell_coord(y[i], box, nc), cz = cell_coord(z[i], box, nc);
    int64_t c = ((int64_t)cx * nc + cy) * nc + cz;
    cl->next[i] = cl->head[c];
    cl->head[c] = i;
  }
  return 0;
}

static void cells_free(cells_t* cl) { free(cl->head); free(cl->next); }

static double min_image(double d, double box) { return d - box * round(d / box); }

/* Neumaier-compensated accumulator. */
typedef struct { double s, c; } acc_t;
static void acc_add(acc_t* a, double v) {
  double t = a->s + v;
  if (fabs(a->s) >= fabs(v)) a->c += (a->s - t) + v; else a->c += (v - t) + a->s;
  a->s = t;
}

/* Short-range acceleration on one receiver i by walking the 27 cells around it. */
static void accel_one(int64_t i, int64_t n, const double* x, const double* y, const double* z,
                      const cells_t* cl, double box, double x_s, double x_r, double G_m,
                      int softening, double eps, double* out, int64_t* npairs) {
  (void)n;
  int nc = cl->nc;
  int cx = cell_coord(x[i], box, nc), cy = cell_coord(y[i], box, nc), cz = cell_coord(z[i], box, nc);
  acc_t ax = {0, 0}, ay = {0, 0}, az = {0, 0};
  int64_t pairs = 0;
  double xr2 = x_r * x_r;
  for (int dx = -1; dx <= 1; ++dx)
    for (int dy = -1; dy <= 1; ++dy)
      for (int dz = -1; dz <= 1; ++dz) {
        int ox = (cx + dx + nc) % nc, oy = (cy + dy + nc) % nc, oz = (cz + dz + nc) % nc;
        int64_t c = ((int64_t)ox * nc + oy) * nc + oz;
        for (int64_t j = cl->head[c]; j >= 0; j = cl->next[j]) {
          if (j == i) continue;
          double rx = min_image(x[i] - x[j], box);
          double ry = min_image(y[i] - y[j], box);
          double rz = min_image(z[i] - z[j], box);
          double r2 = rx * rx + ry * ry + rz * rz;
          if (!(r2 < xr2)) continue;
          ++pairs;
          if (r2 == 0.0) continue; /* coincident: zero contribution by convention */
          double B = oracle_bracket(sqrt(r2), x_s, softening, eps);
          acc_add(&ax, -G_m * B * rx);
          acc_add(&ay, -G_m * B * ry);
          acc_add(&az, -G_m * B * rz);
        }
      }
  out[0] = ax.s + ax.c; out[1] = ay.s + ay.c; out[2] = az.s + az.c;
  *npairs = pairs;
}

/*
 * Short-range accelerations (Eq. p3m_gravity, short-range part) for every
 * receiver i with rung[i] >= rung_min (rung may be NULL: all active).
 * Inactive rows of acc are left untouched.  pos is 3 x n SoA.
 * Returns the number of interacting ordered pairs, or -1 on bad geometry.
 */
int64_t oracle_sr_accel(int64_t n, const double* pos, const int8_t* rung, int rung_min,
                        double box, double x_s, double x_r, double G_m, int softening, double eps,
                        double* acc) {
  const double *x = pos, *y = pos + n, *z = pos + 2 * n;
  cells_t cl;
  if (cells_build(&cl, n, x, y, z, box, x_r) != 0) { cells_free(&cl); return -1; }
  int64_t total = 0;
#pragma omp parallel for schedule(dynamic, 256) reduction(+ : total)
  for (int64_t i = 0; i < n; ++i) {
    if (rung && rung[i] < rung_min) continue;
    double a[3]; int64_t p;
    accel_one(i, n, x, y, z, &cl, box, x_s, x_r, G_m, softening, eps, a, &p);
    acc[i] = a[0]; acc[n + i] = a[1]; acc[2 * n + i] = a[2];
    total += p;
  }
  cells_free(&cl);
  return total;
}

/* Same sum for an explicit list of receivers (subsampling of large sets).
 * acc_sub is 3 x n_sub SoA; pairs_sub (nullable) gets per-receiver counts. */
int64_t oracle_sr_accel_subset(int64_t n, const double* pos, int64_t n_sub, const int64_t* recv,
                               double box, double x_s, double x_r, double G_m, int softening,
                               double eps, double* acc_sub, int64_t* pairs_sub) {
  const double *x = pos, *y = pos + n, *z = pos + 2 * n;
  cells_t cl;
  if (cells_build(&cl, n, x, y, z, box, x_r) != 0) { cells_free(&cl); return -1; }
  int64_t total = 0;
#pragma omp parallel for schedule(dynamic, 64) reduction(+ : total)
  for (int64_t k = 0; k < n_sub; ++k) {
    double a[3]; int64_t p;
    accel_one(recv[k], n, x, y, z, &cl, box, x_s, x_r, G_m, softening, eps, a, &p);
    acc_sub[k] = a[0]; acc_sub[n_sub + k] = a[1]; acc_sub[2 * n_sub + k] = a[2];
    if (pairs_sub) pairs_sub[k] = p;
    total += p;
  }
  cells_free(&cl);
  return total;
}

/* O(N^2) brute force over all j with the minimum image: the plain definition. */
int64_t oracle_sr_accel_brute(int64_t n, const double* pos, const int8_t* rung, int rung_min,
                              double box, double x_s, double x_r, double G_m, int softening,
                              double eps, double* acc) {
  const double *x = pos, *y = pos + n, *z = pos + 2 * n;
  double xr2 = x_r * x_r;
  int64_t total = 0;
#pragma omp parallel for schedule(dynamic, 16) reduction(+ : total)
  for (int64_t i = 0; i < n; ++i) {
    if (rung && rung[i] < rung_min) continue;
    acc_t ax = {0, 0}, ay = {0, 0}, az = {0, 0};
    for (int64_t j = 0; j < n; ++j) {
      if (j == i) continue;
      double rx = min_image(x[i] - x[j], box);
      double ry = min_image(y[i] - y[j], box);
      double rz = min_image(z[i] - z[j], box);
      double r2 = rx * rx + ry * ry + rz * rz;
      if (!(r2 < xr2)) continue;
      ++total;
      if (r2 == 0.0) continue;
      double B = oracle_bracket(sqrt(r2), x_s, softening, eps);
      acc_add(&ax, -G_m * B * rx);
      acc_add(&ay, -G_m * B * ry);
      acc_add(&az, -G_m * B * rz);
    }
    acc[i] = ax.s + ax.c; acc[n + i] = ay.s + ay.c; acc[2 * n + i] = az.s + az.c;
  }
  return total;
}

/*
 * Vector-Jacobian product of the short-range accelerations with respect to
 * positions (derived from Eq. p3m_gravity):
 *
 *   xbar_k = sum_{j != k, r_kj < x_r} J_kj ( abar_k [k active] - abar_j [j active] ),
 *   J_kj  = phi(r) I + (phi'(r)/r) x_kj x_kj^T ,   phi = -G m B .
 *
 * Every particle k receives a gradient (inactive particles still act as
 * suppliers).  abar and xbar are 3 x n SoA.
 */
int64_t oracle_sr_vjp(int64_t n, const double* pos, const int8_t* rung, int rung_min,
                      double box, double x_s, double x_r, double G_m, int softening, double eps,
                      const double* abar, double* xbar) {
  const double *x = pos, *y = pos + n, *z = pos + 2 * n;
  cells_t cl;
  if (cells_build(&cl, n, x, y, z, box, x_r) != 0) { cells_free(&cl); return -1; }
  int nc = cl.nc;
  double xr2 = x_r * x_r;
  int64_t total = 0;
#pragma omp parallel for schedule(dynamic, 256) reduction(+ : total)
  for (int64_t k = 0; k < n; ++k) {
    int act_k = (!rung || rung[k] >= rung_min);
    int cx = cell_coord(x[k], box, nc), cy = cell_coord(y[k], box, nc), cz = cell_coord(z[k], box, nc);
    acc_t gx = {0, 0}, gy = {0, 0}, gz = {0, 0};
    for (int dx = -1; dx <= 1; ++dx)
      for (int dy = -1; dy <= 1; ++dy)
        for (int dz = -1; dz <= 1; ++dz) {
          int ox = (cx + dx + nc) % nc, oy = (cy + dy + nc) % nc, oz = (cz + dz + nc) % nc;
          int64_t c = ((int64_t)ox * nc + oy) * nc + oz;
          for (int64_t j = cl.head[c]; j >= 0; j = cl.next[j]) {
            if (j == k) continue;
            double rx = min_image(x[k] - x[j], box);
            double ry = min_image(y[k] - y[j], box);
            double rz = min_image(z[k] - z[j], box);
            double r2 = rx * rx + ry * ry + rz * rz;
            if (!(r2 < xr2)) continue;
            ++total;
            int act_j = (!rung || rung[j] >= rung_min);
            double vx = 0, vy = 0, vz = 0;
            if (act_k) { vx += abar[k]; vy += abar[n + k]; vz += abar[2 * n + k]; }
            if (act_j) { vx -= abar[j]; vy -= abar[n + j]; vz -= abar[2 * n + j]; }
            if (r2 == 0.0) {
              if (softening == 0) continue;
              double phi0 = -G_m * oracle_bracket(0.0, x_s, softening, eps);
              acc_add(&gx, phi0 * vx); acc_add(&gy, phi0 * vy); acc_add(&gz, phi0 * vz);
              continue;
            }
            double r = sqrt(r2);
            double phi = -G_m * oracle_bracket(r, x_s, softening, eps);
            double dphi = -G_m * oracle_bracket_dr(r, x_s, softening, eps);
            double xv = rx * vx + ry * vy + rz * vz;
            double c2 = dphi / r * xv;
            acc_add(&gx, phi * vx + c2 * rx);
            acc_add(&gy, phi * vy + c2 * ry);
            acc_add(&gz, phi * vz + c2 * rz);
          }
        }
    xbar[k] = gx.s + gx.c; xbar[n + k] = gy.s + gy.c; xbar[2 * n + k] = gz.s + gz.c;
  }
  cells_free(&cl);
  return total;
}

/* ------------------------------------------------------------------------- */
/* Integer decisions: subtile ids and rungs (bit-exact definitions).          */
/* ------------------------------------------------------------------------- */

/*
 * Subtile id of each particle (Section 2.1.3, "Tiles" / "Subtiles"; walk order
 * tile -> subtile -> particle).  The box holds n_t tiles per dimension, each
 * split into n_s subtiles per dimension, M = n_t n_s subtiles per dimension:
 *   g_d = min(floor(x_d * M), M - 1)      (one correctly rounded multiply)
 *   tile_d = g_d / n_s, sub_d = g_d mod n_s
 *   id = ((tx n_t + ty) n_t + tz) n_s^3 + (sx n_s + sy) n_s + sz.
 * Positions are in [0, 1) (unit box).
 */
void oracle_subtile_ids(int64_t n, const double* pos, int n_t, int n_s, int32_t* id) {
  const double *x = pos, *y = pos + n, *z = pos + 2 * n;
  int M = n_t * n_s;
  double Md = (double)M;
  for (int64_t i = 0; i < n; ++i) {
    int g[3];
    const double v[3] = {x[i], y[i], z[i]};
    for (int d = 0; d < 3; ++d) {
      double p = v[d] * Md;
      int q = (int)floor(p);
      if (q > M - 1) q = M - 1;
      if (q < 0) q = 0;
      g[d] = q;
    }
    int64_t tile = ((int64_t)(g[0] / n_s) * n_t + g[1] / n_s) * n_t + g[2] / n_s;
    int sub = ((g[0] % n_s) * n_s + g[1] % n_s) * n_s + g[2] % n_s;
    id[i] = (int32_t)(tile * n_s * n_s * n_s + sub);
  }
}

/*
 * Rung of each particle (Section 2.2.2, Eq. rung):
 *   l = max(0, ceil(log2(dt sqrt(|a| / (2 eta eps))))), clamped to n_rung - 1.
 * Written without log2/sqrt: with q = dt^2 / (2 eta eps) and
 * s = q^2 (a_x^2 + a_y^2 + a_z^2), l is the smallest l >= 0 with s <= 16^l.
 * Returns the number of non-finite accelerations met (their rung is set to 0).
 */
int64_t oracle_rungs(int64_t n, const double* acc, double dt, double eta, double eps, int n_rung,
                     int8_t* rung) {
  double t1 = dt * dt;
  double t2 = 2.0 * eta;
  double t3 = t2 * eps;
  double q = t1 / t3;
  double qq = q * q;
  int64_t bad = 0;
  for (int64_t i = 0; i < n; ++i) {
    double ax = acc[i], ay = acc[n + i], az = acc[2 * n + i];
    double a2 = ax * ax;
    a2 = a2 + ay * ay;
    a2 = a2 + az * az;
    double s = qq * a2;
    if (!(s == s) || isinf(s)) { rung[i] = 0; ++bad; continue; }
    int l = 0;
    double p = 1.0;
    while (l < n_rung - 1 && s > p) { p *= 16.0; ++l; }
    rung[i] = (int8_t)l;
  }
  return bad;
}

/* ------------------------------------------------------------------------- */
/* Kick and drift (Section 2.2.2, operators K and D; static a = 1).           */
/* ------------------------------------------------------------------------- */

/* q_i += a_i * K[rung_i] for active i (rung >= rung_min). */
void oracle_kick(int64_t n, double* mom, const double* acc, const int8_t* rung, int rung_min,
                 const double* kick_factor) {
  for (int64_t i = 0; i < n; ++i) {
    int l = rung ? rung[i] : 0;
    if (rung && l < rung_min) continue;
    double k = kick_factor[l];
    for (int d = 0; d < 3; ++d) mom[d * n + i] = mom[d * n + i] + acc[d * n + i] * k;
  }
}

/* x_i += q_i * D, then wrap into [0, box). */
void oracle_drift(int64_t n, double* pos, const double* mom, double factor, double box) {
  for (int64_t i = 0; i < n; ++i)
    for (int d = 0; d < 3; ++d) {
      double v = pos[d * n + i] + mom[d * n + i] * factor;
      v = v - box * floor(v / box);
      if (v >= box || v < 0.0) v = 0.0;
      pos[d * n + i] = v;
    }
}

/*
 * One kick of the rung-based leapfrog (Section 2.2.2, time-stepping figure and
 * text).  Rung-l momenta are kicked every dt/2^l; this kick happens at time
 * k dt / 2^(n_rung-1) after the last synchronisation and touches the particles
 * with rung >= rung_min.  A particle's kick is f dt / 2^l with f = 1 normally,
 * 1/2 after a jump to a finer rung and 3/4 after a jump to a coarser one; with
 * sync the kick stops at the synchronisation time (f - 1/2).  After a normal
 * kick the rung of Eq. rung (oracle_rungs) decides: finer -> l+1 (next kick
 * 1/2); coarser -> l-1 (next kick 3/4), but only when k dt/2^(n_rung-1) is an
 * odd multiple of dt/2^l ("every other kick"); else unchanged.
 * state: 0 (f = 1), 1 (f = 1/2), 2 (f = 3/4).  Returns non-finite count.
 */
int64_t oracle_rung_kick(int64_t n, double* mom, const double* acc, int8_t* rung, int8_t* state, int rung_min,
                         long long k, int n_rung, double dt, double eta, double eps, int sync) {
  double t1 = dt * dt;
  double t2 = 2.0 * eta;
  double t3 = t2 * eps;
  double q = t1 / t3;
  double qq = q * q;
  int64_t bad = 0;
  for (int64_t i = 0; i < n; ++i) {
    int l = rung[i];
    if (l < rung_min) continue;
    double f = state[i] == 0 ? 1.0 : (state[i] == 1 ? 0.5 : 0.75);
    double fac = sync ? f - 0.5 : f;
    double K = ldexp(dt * fac, -l);
    double a[3];
    for (int d = 0; d < 3; ++d) {
      a[d] = acc[d * n + i];
      mom[d * n + i] = mom[d * n + i] + a[d] * K;
    }
    if (sync) { state[i] = 0; continue; }
    double a2 = a[0] * a[0];
    a2 = a2 + a[1] * a[1];
    a2 = a2 + a[2] * a[2];
    double s = qq * a2;
    int lnew = 0;
    if (!(s == s) || isinf(s)) {
      ++bad;
    } else {
      double p = 1.0;
      while (lnew < n_rung - 1 && s > p) { p *= 16.0; ++lnew; }
    }
    if (lnew > l) { rung[i] = (int8_t)(l + 1); state[i] = 1; }
    else if (lnew < l && ((k >> (n_rung - 1 - l)) & 1LL)) { rung[i] = (int8_t)(l - 1); state[i] = 2; }
    else state[i] = 0;
  }
  return bad;
}

int oracle_num_threads(void) {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}

/* Threads of the following parallel loops (timing of the single-threaded oracle). */
void oracle_set_num_threads(int k) {
#ifdef _OPENMP
  if (k > 0) omp_set_num_threads(k);
#else
  (void)k;
#endif
}
