// Internal declarations shared by the CUDA translation units of the library.
// Nothing here is part of the C ABI (include/p3m_sr.h is).
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

#include "../../include/p3m_sr.h"

namespace p3m {

constexpr int kWarp = 32;
constexpr int kMaxDrifts = 64;  // drifts of the sorted positions allowed between two sorts
constexpr int kChunk = 32;  // receivers per chunk (one warp lane each)
constexpr int kPartItems = 32768;  // work items of split chunks that the partial-sum buffer holds
constexpr int kMaxParts = 8;       // parts a chunk is split into at most

// Device-side error bits, latched in a device word by the kernels.
enum : int {
  kErrPosition = 1,      // non-finite or out-of-box position at binning
  kErrNonfiniteAcc = 2,  // non-finite acceleration at rung assignment
  kErrRungState = 4,     // rung outside [0, n_rung) or kick state outside {0, 1, 2} at a rung kick
  kErrDrift = 8,         // positions drifted so far since the sort that the traversal cannot cover them
};

// Tile/subtile geometry of the periodic box (Section 2.1.3).
struct Geometry {
  int n_t;            // tiles per dimension, floor(L / x_r)
  int ns[3];          // subtiles per tile per dimension
  int M[3];           // subtiles per dimension, n_t * ns[d]
  int nsub3;          // subtiles per tile
  int R[3];           // reach of x_r in subtiles, ceil(x_r / side_d)
  int64_t S;          // number of subtiles
  double box;
  double scale64[3];  // M[d] / L, for binning
  float inv_ns[3];    // 1 / ns[d], for quotients of small integers (see quot_small)
  double side64[3];   // L / M[d]
  float side32[3];    // (float) side64
  // multipliers of quot_magic for nsub3, n_t^2, n_t, ns[1] ns[2] and ns[2]
  unsigned long long mg_nsub3, mg_nt2, mg_nt, mg_s12, mg_s2;
  const double* org = nullptr;  // device table of subtile origins i * side64[d]: x at [0, M[0]), then y, then z
};

// Constants of the pair force (Eq. p3m_gravity, short-range bracket).
struct ForceConsts {
  int softening;
  double x_s, x_r, G_m, eps;
  double eps_b;        // B-spline length 2.8 eps
  double r_sw;         // below r_sw the softened form B = shape - h(u)/(2x_s)^3 is used
  // FP32 path
  float xr2_f;         // x_r^2
  float rsw2_f;        // r_sw^2 (tiny for no softening: only r = 0 takes that branch)
  float ce_f;          // -log2(e) / (4 x_s^2): exp(-u^2) = ex2(ce * r^2)
  float kc_f;          // K / (2 x_s): t = 1 / (1 + K u)
  float k2_f;          // 1 / (sqrt(pi) x_s)
  float k3_f;          // 1 / (2 sqrt(pi) x_s^3), for dB/dr
  float c_f[6];        // erfcx fit coefficients
  float inv2xs_f;      // 1 / (2 x_s)
  float hscale_f;      // 1 / (2 x_s)^3
  float epsb_f, inv_epsb_f, bnorm_f;  // B-spline: eps_B, 1/eps_B, 32 / eps_B^3
  float eps2_f;        // Plummer eps^2
  float margin2_f;     // conservative x_r^2 for box pruning
  // FP64 path
  double xr2_d, rsw2_d;
};

// One receiver chunk: up to 32 consecutive receivers of one tile.
struct Chunk {
  int start;  // index into the receiver list (or the sorted particle index)
  int count;  // 1..32
};

// ---- small device helpers -------------------------------------------------

// floor(a / d) for 0 <= a < 2^31 and 1 <= d < 2^33 from m = magic_u64(d): the high
// word of a * m (division by an invariant integer through multiplication,
// Granlund and Montgomery 1994).  With m = ceil(2^64 / d) the product overshoots
// a / d by less than a 2^-64 < 1 / d, which never reaches the next integer; d = 1
// has no 64-bit multiplier and is passed through.
__device__ __forceinline__ int quot_magic(int a, int d, unsigned long long m) {
  return d == 1 ? a : (int)__umul64hi((unsigned long long)a, m);
}

__device__ __forceinline__ void decode_subtile(const Geometry& g, int id, int& gx, int& gy, int& gz) {
  const int tile = quot_magic(id, g.nsub3, g.mg_nsub3);
  const int sub = id - tile * g.nsub3;
  const int nt2 = g.n_t * g.n_t;
  const int tx = quot_magic(tile, nt2, g.mg_nt2);
  const int rem = tile - tx * nt2;
  const int ty = quot_magic(rem, g.n_t, g.mg_nt);
  const int tz = rem - ty * g.n_t;
  const int s12 = g.ns[1] * g.ns[2];
  const int sx = quot_magic(sub, s12, g.mg_s12);
  const int srem = sub - sx * s12;
  const int sy = quot_magic(srem, g.ns[2], g.mg_s2);
  const int sz = srem - sy * g.ns[2];
  gx = tx * g.ns[0] + sx;
  gy = ty * g.ns[1] + sy;
  gz = tz * g.ns[2] + sz;
}

// q = floor(a / b) for 0 <= a < 2^22 and 1 <= b < 2^10, with inv ~ 1/b in FP32: the
// float estimate is within one of q (its relative error is a few 2^-24) and one
// correction each way makes it exact; cheaper than an integer division by a value
// known only at run time.
__device__ __forceinline__ int quot_small(int a, int b, float inv) {
  int q = (int)(((float)a + 0.5f) * inv);
  q -= (q * b > a) ? 1 : 0;
  q += ((q + 1) * b <= a) ? 1 : 0;
  return q;
}

// encode_subtile for 0 <= g < M with the quotients by n_sub from quot_small.
__device__ __forceinline__ int encode_subtile_fast(const Geometry& g, int gx, int gy, int gz) {
  const int tx = quot_small(gx, g.ns[0], g.inv_ns[0]), sx = gx - tx * g.ns[0];
  const int ty = quot_small(gy, g.ns[1], g.inv_ns[1]), sy = gy - ty * g.ns[1];
  const int tz = quot_small(gz, g.ns[2], g.inv_ns[2]), sz = gz - tz * g.ns[2];
  const int tile = (tx * g.n_t + ty) * g.n_t + tz;
  return tile * g.nsub3 + (sx * g.ns[1] + sy) * g.ns[2] + sz;
}

__device__ __forceinline__ int encode_subtile(const Geometry& g, int gx, int gy, int gz) {
  int tx = gx / g.ns[0], sx = gx - tx * g.ns[0];
  int ty = gy / g.ns[1], sy = gy - ty * g.ns[1];
  int tz = gz / g.ns[2], sz = gz - tz * g.ns[2];
  int tile = (tx * g.n_t + ty) * g.n_t + tz;
  return tile * g.nsub3 + (sx * g.ns[1] + sy) * g.ns[2] + sz;
}

// FP32 coordinates of (x, y, z) relative to the origin of subtile (gx, gy, gz):
// per axis one FP64 subtraction of the tabulated origin (g.org) and one
// conversion.  On this part the FP64 pipe is the scarce resource of every
// per-particle pass, so the origin is read, not computed, and no FP64 comparison
// is made.
__device__ __forceinline__ void rel_to_subtile(const Geometry& g, double x, double y, double z, int gx, int gy,
                                               int gz, double r[3]) {
  r[0] = __dsub_rn(x, __ldg(g.org + gx));
  r[1] = __dsub_rn(y, __ldg(g.org + g.M[0] + gy));
  r[2] = __dsub_rn(z, __ldg(g.org + g.M[0] + g.M[1] + gz));
}

// Subtile origins i * side64[d] for the table g.org (M[0] + M[1] + M[2] entries).
__global__ void k_fill_origins(Geometry g, double* __restrict__ org);

// ---- kernels of sort.cu launched from other translation units ---------------
constexpr int kRadixThreadsPublic = 256;
#ifndef P3M_RADIX_STEPS
#define P3M_RADIX_STEPS 8  // radix items per lane (8: 2048-item tiles, 7% faster than 4096 at 128^3, 26% at 512^3)
#endif
constexpr int kRadixTilePublic = kRadixThreadsPublic * P3M_RADIX_STEPS;  // items per radix block
__global__ void k_bin(const double* __restrict__ pos, int64_t n, Geometry g, int* __restrict__ keys,
                      int* __restrict__ vals, int* __restrict__ counts, int* __restrict__ err);
__global__ void k_radix_hist(const int* __restrict__ keys, int64_t n, int shift, int bits, int* __restrict__ hist,
                             int nblocks);
__global__ void k_radix_scatter(const int* __restrict__ keys_in, const int* __restrict__ vals_in,
                                int* __restrict__ keys_out, int* __restrict__ vals_out, int64_t n, int shift,
                                int bits, const int* __restrict__ hist, int nblocks, int* __restrict__ hist_next,
                                int shift_next, int bits_next);
__global__ void k_gather_pos(const double* __restrict__ src, const int* __restrict__ perm, int64_t n,
                             double* __restrict__ dst);

// ---- launch helpers (host) --------------------------------------------------

// Exclusive scan of n int32 values (in may equal out).  Returns cudaError.
// scratch: scratch_ints >= scan_scratch_ints(n) ints whose last int is zero before
// the first scan (and is left zero).  Adds the number of kernels it launched to
// *launches.
cudaError_t scan_exclusive_i32(const int* in, int* out, int64_t n, int* scratch, int64_t scratch_ints, cudaStream_t s,
                               int64_t* launches);
// Scratch (ints) needed by scan_exclusive_i32 for n elements.
int64_t scan_scratch_ints(int64_t n);

}  // namespace p3m
