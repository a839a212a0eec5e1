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

__device__ __forceinline__ void decode_subtile(const Geometry& g, int id, int& gx, int& gy, int& gz) {
  int tile = id / g.nsub3;
  int sub = id - tile * g.nsub3;
  int nt2 = g.n_t * g.n_t;
  int tx = tile / nt2;
  int rem = tile - tx * nt2;
  int ty = rem / g.n_t;
  int tz = rem - ty * g.n_t;
  int s12 = g.ns[1] * g.ns[2];
  int sx = sub / s12;
  int srem = sub - sx * s12;
  int sy = srem / g.ns[2];
  int sz = srem - sy * g.ns[2];
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

// ---- kernels of sort.cu launched from other translation units ---------------
constexpr int kRadixThreadsPublic = 256;
constexpr int kRadixTilePublic = 4096;  // items per radix block
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
