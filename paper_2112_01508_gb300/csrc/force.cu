// Receiver work lists, the short-range pair-force kernels (FP32 and FP64) and
// the adjoint (VJP) kernels.
//
// Paper design (Section 2.1.3): tiles of side >= x_r, subtiles inside them,
// precomputed subtile pairings inside a "blocky ball" of radius x_r, a
// squared-distance rejection r^2 >= x_r^2 before the force, image shift n'
// known per subtile pair, particles stored in tile -> subtile -> particle
// order.  Receivers are the particles on active rungs (Section 2.2.2).
//
// GB300 design: the work unit is a receiver chunk -- up to 32 consecutive
// receivers of one row of tiles (spanning at most four tiles along z), one per
// warp lane.  A warp owns a chunk and:
//   1. builds the chunk's frame (origin: the subtile of its first receiver)
//      and the receivers' tight bounding box;
//   2. enumerates, 32 candidates at a time across the lanes, the subtiles of
//      the blocky ball around the chunk's subtile block (the paper's subtile
//      pairing generalised to a block of subtiles), keeps those whose box gap
//      to the bounding box is below x_r, and appends their particle ranges to
//      a per-warp list in shared memory;
//   3. walks the concatenated supplier ranges 32 at a time: each lane loads
//      one supplier j (FP32 coordinates relative to its subtile origin, moved
//      into the chunk frame by the integer subtile offset) and tests it against
//      the bounding box; the survivors are broadcast to all lanes, and every
//      lane evaluates its own (i, j) pair.
// The one-sided FP32 forward kernel stages the survivors in shared memory as
// packed pairs and evaluates two suppliers per step in f32x2 arithmetic; the
// FP64 forward and the one-sided adjoint broadcast survivors with warp
// shuffles.  With every particle a receiver, the FP32 forward and the FP32
// adjoint evaluate each pair once instead (k_force_sym, below).  Chunks are
// handed out through an atomic counter to persistent warps, which balances the
// strongly varying cost of clustered regions.
#include <algorithm>
#include <cmath>
#include <mutex>
#include <vector>

#include <type_traits>

#include "ctx.cuh"
#include "erfcx_fit.h"
#include "pair_math.cuh"

namespace p3m {

constexpr int kForceThreads = 128;
constexpr int kForceWarps = kForceThreads / kWarp;
// Supplier subtiles buffered per warp before their particles are walked: 256
// measured best on the 128^3 and 512^3 sets (the one-sided kernel 4-8% faster than
// with 128, the each-pair-once kernel unchanged; 64 slower).
#ifndef P3M_LISTCAP
#define P3M_LISTCAP 256
#endif
constexpr int kListCap = P3M_LISTCAP;

static unsigned blocks_for(int64_t n, int t) { return (unsigned)((n + t - 1) / t); }

// ---------------------------------------------------------------------------
// Prologue kernels.
// ---------------------------------------------------------------------------

// FP32 coordinates relative to the particle's subtile origin, plus the id bits.
// All lanes of a warp reach the vote: launched with whole warps, lanes past n only vote.
__global__ void k_rel4(const double* __restrict__ pos, const int* __restrict__ cell, int64_t n, Geometry g,
                       float4* __restrict__ rel4) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const bool valid = i < n;
  int id = 0, gx = 0, gy = 0, gz = 0;
  double x = 0.0, y = 0.0, z = 0.0;
  if (valid) {
    id = cell[i];
    decode_subtile(g, id, gx, gy, gz);
    x = pos[i];
    y = pos[n + i];
    z = pos[2 * n + i];
  }
  double r[3];
  rel_to_subtile(g, x, y, z, gx, gy, gz, r);
  float f[3] = {(float)r[0], (float)r[1], (float)r[2]};
  // relative to the origin of the subtile of the last sort; a particle that drifted
  // across the periodic boundary since then takes its nearest image.  Its offset is
  // then near +-L, every other one far below L/2, so the test is made in FP32, and
  // only warps that hold such a particle spend FP64 operations on it.
  const float half = 0.5f * (float)g.box;
  const bool far = fabsf(f[0]) > half || fabsf(f[1]) > half || fabsf(f[2]) > half;
  if (__any_sync(0xffffffffu, far)) {
#pragma unroll
    for (int d = 0; d < 3; ++d)
      if (fabsf(f[d]) > half) {
        r[d] = f[d] > 0.0f ? __dsub_rn(r[d], g.box) : __dadd_rn(r[d], g.box);
        f[d] = (float)r[d];
      }
  }
  if (valid) rel4[i] = make_float4(f[0], f[1], f[2], __int_as_float(id));
}

// The receiver set in two passes over tiles of kActTile sorted particles: the number
// of receivers (rung >= rung_min) per tile, then (after a scan of those counts) each
// tile's flags, its exclusive scan act_scan[0..n] and the compacted receiver list.
constexpr int kActThreads = 256;
constexpr int kActItems = 16;
constexpr int kActTile = kActThreads * kActItems;

__global__ void __launch_bounds__(kActThreads) k_active_count(const int8_t* __restrict__ rung, int64_t n, int rung_min,
                                                              int* __restrict__ tile_count) {
  __shared__ int warp_sums[kActThreads / kWarp];
  const int64_t base = (int64_t)blockIdx.x * kActTile;
  int c = 0;
  for (int k = 0; k < kActItems; ++k) {
    const int64_t i = base + (int64_t)k * kActThreads + threadIdx.x;
    if (i < n) c += rung[i] >= rung_min ? 1 : 0;
  }
  c = __reduce_add_sync(0xffffffffu, c);
  if ((threadIdx.x & 31) == 0) warp_sums[threadIdx.x >> 5] = c;
  __syncthreads();
  if (threadIdx.x == 0) {
    int t = 0;
    for (int w = 0; w < kActThreads / kWarp; ++w) t += warp_sums[w];
    tile_count[blockIdx.x] = t;
  }
}

// flag and act_scan are 16-byte aligned (context arrays); rung is read as 16-byte
// vectors when it is too.
__global__ void __launch_bounds__(kActThreads) k_active_scan_compact(const int8_t* __restrict__ rung, int64_t n,
                                                                     int rung_min, const int* __restrict__ tile_base,
                                                                     int8_t* __restrict__ flag, int* __restrict__ act_scan,
                                                                     int* __restrict__ active_idx) {
  static_assert(kActItems == 16, "one 16-byte vector of rungs and flags per thread");
  __shared__ int warp_tot[kActThreads / kWarp];
  const int64_t base = (int64_t)blockIdx.x * kActTile + (int64_t)threadIdx.x * kActItems;  // 16 consecutive items
  const bool whole = base + kActItems <= n;
  int f[kActItems];
  int tot = 0;
  if (whole && ((reinterpret_cast<uintptr_t>(rung) & 15) == 0)) {
    const int4 v = *reinterpret_cast<const int4*>(rung + base);
    const int w[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
    for (int k = 0; k < kActItems; ++k) {
      const int r = (int)(int8_t)((w[k >> 2] >> (8 * (k & 3))) & 0xff);
      f[k] = r >= rung_min ? 1 : 0;
      tot += f[k];
    }
  } else {
#pragma unroll
    for (int k = 0; k < kActItems; ++k) {
      const int64_t i = base + k;
      f[k] = (i < n && rung[i] >= rung_min) ? 1 : 0;
      tot += f[k];
    }
  }
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  int inc = tot;
  for (int o = 1; o < 32; o <<= 1) {
    const int u = __shfl_up_sync(0xffffffffu, inc, o);
    if (lane >= o) inc += u;
  }
  if (lane == 31) warp_tot[warp] = inc;
  __syncthreads();
  int run = inc - tot + tile_base[blockIdx.x];
  for (int w = 0; w < warp; ++w) run += warp_tot[w];
  if (whole) {  // vector stores: 16 flags, then 16 scan values as four int4
    int fw[4] = {0, 0, 0, 0};
    int sc[kActItems];
#pragma unroll
    for (int k = 0; k < kActItems; ++k) {
      fw[k >> 2] |= f[k] << (8 * (k & 3));
      sc[k] = run;
      if (f[k]) active_idx[run] = (int)(base + k);
      run += f[k];
    }
    *reinterpret_cast<int4*>(flag + base) = make_int4(fw[0], fw[1], fw[2], fw[3]);
#pragma unroll
    for (int q = 0; q < 4; ++q)
      reinterpret_cast<int4*>(act_scan + base)[q] = make_int4(sc[4 * q], sc[4 * q + 1], sc[4 * q + 2], sc[4 * q + 3]);
  } else {
#pragma unroll
    for (int k = 0; k < kActItems; ++k) {
      const int64_t i = base + k;
      if (i <= n) act_scan[i] = run;
      if (i < n) {
        flag[i] = (int8_t)f[k];
        if (f[k]) active_idx[run] = (int)i;
      }
      run += f[k];
    }
  }
}

// Receiver chunks.  The receivers of one row of tiles (fixed tile x, y) are
// consecutive in the sorted order.  Each row is cut into segments of
// kChunkSpan consecutive tiles along z, and the receivers of a segment into
// ceil(count / 32) chunks, so that sparse tiles share a warp while every chunk
// stays spatially compact.  One thread per segment: no sequential walk.
#ifndef P3M_CHUNK_SPAN
#define P3M_CHUNK_SPAN 4
#endif
constexpr int kChunkSpan = P3M_CHUNK_SPAN;

__device__ __forceinline__ int tile_start(const int* __restrict__ offsets, const int* __restrict__ act_scan, int nsub3,
                                          int64_t T) {
  int p = offsets[T * nsub3];
  return act_scan ? act_scan[p] : p;
}

// Receiver range [a0, a1) of segment `seg` (row-major over rows, then segments).
__device__ __forceinline__ void segment_range(const int* __restrict__ offsets, const int* __restrict__ act_scan,
                                              int nsub3, int n_t, int64_t seg, int& a0, int& a1) {
  const int nseg = (n_t + kChunkSpan - 1) / kChunkSpan;
  const int64_t row = seg / nseg;
  const int k = (int)(seg - row * nseg);
  const int64_t t0 = row * n_t + (int64_t)k * kChunkSpan;
  const int64_t t1 = row * n_t + min(n_t, (k + 1) * kChunkSpan);
  a0 = tile_start(offsets, act_scan, nsub3, t0);
  a1 = tile_start(offsets, act_scan, nsub3, t1);
}

__global__ void k_row_chunks(const int* __restrict__ offsets, const int* __restrict__ act_scan, int n_t, int nsub3,
                             int* __restrict__ seg_chunks) {
  const int64_t seg = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t nsegs = (int64_t)n_t * n_t * ((n_t + kChunkSpan - 1) / kChunkSpan);
  if (seg > nsegs) return;
  if (seg == nsegs) {
    seg_chunks[nsegs] = 0;
    return;
  }
  int a0, a1;
  segment_range(offsets, act_scan, nsub3, n_t, seg, a0, a1);
  seg_chunks[seg] = (a1 - a0 + kChunk - 1) / kChunk;
}

__global__ void k_write_chunks(const int* __restrict__ offsets, const int* __restrict__ act_scan, int n_t, int nsub3,
                               const int* __restrict__ seg_chunks, Chunk* __restrict__ chunks,
                               int* __restrict__ n_chunks_out, int* __restrict__ n_active_out, int64_t n) {
  const int64_t seg = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t nsegs = (int64_t)n_t * n_t * ((n_t + kChunkSpan - 1) / kChunkSpan);
  if (seg == 0) {
    *n_chunks_out = seg_chunks[nsegs];
    if (n_active_out) *n_active_out = act_scan ? act_scan[n] : (int)n;
  }
  if (seg >= nsegs) return;
  int a0, a1;
  segment_range(offsets, act_scan, nsub3, n_t, seg, a0, a1);
  Chunk* out = chunks + seg_chunks[seg];
  for (int k = 0; a0 + k * kChunk < a1; ++k) {
    const int s0 = a0 + k * kChunk;
    out[k] = Chunk{s0, min(kChunk, a1 - s0)};
  }
}

// Masked abar for the VJP: abar_i * [i active].
__global__ void k_abar_f32(const float* __restrict__ abar, const int8_t* __restrict__ flag, int all_active,
                           int64_t n, float4* __restrict__ out) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  float m = (all_active || flag[i]) ? 1.0f : 0.0f;
  out[i] = make_float4(abar[i] * m, abar[n + i] * m, abar[2 * n + i] * m, 0.0f);
}

__global__ void k_abar_f64(const double* __restrict__ abar, const int8_t* __restrict__ flag, int all_active,
                           int64_t n, double* __restrict__ out) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  double m = (all_active || flag[i]) ? 1.0 : 0.0;
  out[i] = abar[i] * m;
  out[n + i] = abar[n + i] * m;
  out[2 * n + i] = abar[2 * n + i] * m;
}

// ---------------------------------------------------------------------------
// The traversal kernel.
// ---------------------------------------------------------------------------

struct TraversalArgs {
  Geometry g;
  ForceConsts f;
  SeriesConsts sc;
  const double* pos;          // FP64 path positions
  const float4* rel4;         // FP32 path coordinates
  const int* offsets;         // S + 1 subtile offsets
  const int* cell;            // sorted subtile ids
  const Chunk* chunks;
  float4* part_acc;           // per (work item, lane) partial sums when chunks are split (kPartItems x 32), or nullptr
  const float* drift_slots;   // displacement bounds of the drifts since the sort (device)
  int n_drift;                // how many of them
  int* err;                   // device error bits (kErrDrift), or nullptr
  const int* n_chunks;        // device count
  int* counter;               // dynamic chunk counter (zeroed before launch)
  const int* active_idx;      // receiver list (nullptr: chunk ranges are particle indices)
  int64_t n;
  void* out;                  // acc (forward) or xbar (vjp), 3 x n
  // vjp only
  const float4* abar4;        // masked abar FP32
  const double* abar_d;       // masked abar FP64, 3 x n
  unsigned long long* pairs;  // interacting ordered pairs
  // tabulated bracket (p3m_sr_forces_tabulated): B at the centres of n_table
  // equal bins of r^2 in [0, x_r^2)
  const float* table;
  int n_table;
  float table_scale;          // n_table / x_r^2
};

template <class Real>
struct Vec3 {
  Real x, y, z;
};

__device__ __forceinline__ float redux_min_f(float v) {
  float r;
  asm("redux.sync.min.f32 %0, %1, 0xffffffff;" : "=f"(r) : "f"(v));
  return r;
}
__device__ __forceinline__ float redux_max_f(float v) {
  float r;
  asm("redux.sync.max.f32 %0, %1, 0xffffffff;" : "=f"(r) : "f"(v));
  return r;
}
__device__ __forceinline__ double warp_min_d(double v) {
  for (int o = 16; o > 0; o >>= 1) v = fmin(v, __shfl_xor_sync(0xffffffffu, v, o));
  return v;
}
__device__ __forceinline__ double warp_max_d(double v) {
  for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
  return v;
}
__device__ __forceinline__ float warp_min(float v) { return redux_min_f(v); }
__device__ __forceinline__ float warp_max(float v) { return redux_max_f(v); }
__device__ __forceinline__ double warp_min(double v) { return warp_min_d(v); }
__device__ __forceinline__ double warp_max(double v) { return warp_max_d(v); }

__device__ __forceinline__ unsigned pack_delta(int dx, int dy, int dz) {
  return ((unsigned)(dx + 512) << 20) | ((unsigned)(dy + 512) << 10) | (unsigned)(dz + 512);
}
__device__ __forceinline__ void unpack_delta(unsigned p, int& dx, int& dy, int& dz) {
  dx = (int)(p >> 20) - 512;
  dy = (int)((p >> 10) & 1023u) - 512;
  dz = (int)(p & 1023u) - 512;
}

struct WarpList {
  int start[kListCap];
  int pre[kListCap];       // exclusive prefix of the supplier counts
  unsigned delta[kListCap];
};

// Reach of the traversal.  Right after a sort: the block R of subtiles around the
// receivers' subtiles and the pruning bound x_r on the gap between a candidate
// subtile box and the receivers' box.  After drifts of total length delta since
// the sort, a particle may lie up to delta outside the subtile it was sorted into:
// the gap bound grows to x_r + delta and the block to x_r + 2 delta (receivers and
// suppliers both moved).
struct Reach {
  int R[3];
  float sub2;     // squared gap bound, FP32 path
  double sub2_d;  // FP64 path
};

__device__ __forceinline__ Reach make_reach(const TraversalArgs& a) {
  Reach r;
  float delta = 0.0f;
  for (int k = 0; k < a.n_drift; ++k) delta += a.drift_slots[k];
  if (!(delta > 0.0f)) {
#pragma unroll
    for (int d = 0; d < 3; ++d) r.R[d] = a.g.R[d];
    r.sub2 = a.f.margin2_f;
    r.sub2_d = (double)a.f.margin2_f;
    return r;
  }
  const double dl = (double)delta * (1.0 + 1e-5);  // the float sum may round down
  const double reach = sqrt((double)a.f.margin2_f) + dl;
  if (!(reach + dl < 0.5 * a.g.box)) {
    if ((threadIdx.x & 31) == 0 && a.err) atomicOr(a.err, kErrDrift);
  }
#pragma unroll
  for (int d = 0; d < 3; ++d) {
    const double rr = fmin(reach + dl, 0.5 * a.g.box);
    r.R[d] = (int)ceil(rr / a.g.side64[d] * (1.0 + 1e-12));
  }
  r.sub2_d = reach * reach;
  r.sub2 = (float)(r.sub2_d * (1.0 + 1e-6));
  return r;
}

// The receivers of one chunk in its frame: positions, bounding box, subtile block.
template <class Real>
struct ChunkFrame {
  bool valid;       // this lane holds a receiver
  int pidx;         // its sorted particle index
  int g0[3];        // subtile of lane 0 (frame origin)
  Vec3<Real> pi;    // receiver position (chunk frame in FP32, absolute in FP64)
  Vec3<Real> lo, hi;  // bounding box of the receivers
  int elo[3], ext[3];  // candidate subtile block (offsets from g0) and its extent
  float inv_ext[2];    // 1 / ext[2], 1 / ext[1], for decoding candidate indices
  Real org[3];      // position of g0's origin in the frame
};

template <class Real>
__device__ __forceinline__ void load_chunk(const TraversalArgs& a, const Reach& rc, const Chunk& ch, int lane,
                                           ChunkFrame<Real>& F) {
  const unsigned full = 0xffffffffu;
  const Geometry& g = a.g;
  F.valid = lane < ch.count;
  F.pidx = 0;
  if (F.valid) F.pidx = a.active_idx ? a.active_idx[ch.start + lane] : ch.start + lane;
  int gi[3] = {0, 0, 0};
  float4 ri = make_float4(0.f, 0.f, 0.f, 0.f);
  {
    int id = 0;
    if constexpr (sizeof(Real) == 4) {
      if (F.valid) ri = a.rel4[F.pidx];
      id = __float_as_int(ri.w);
    } else {
      if (F.valid) id = a.cell[F.pidx];
    }
    if (F.valid) decode_subtile(g, id, gi[0], gi[1], gi[2]);
  }
#pragma unroll
  for (int d = 0; d < 3; ++d) F.g0[d] = __shfl_sync(full, gi[d], 0);
  const int e[3] = {gi[0] - F.g0[0], gi[1] - F.g0[1], gi[2] - F.g0[2]};
  if constexpr (sizeof(Real) == 4) {
    F.pi.x = fmaf((float)e[0], g.side32[0], ri.x);
    F.pi.y = fmaf((float)e[1], g.side32[1], ri.y);
    F.pi.z = fmaf((float)e[2], g.side32[2], ri.z);
  } else {
    F.pi.x = F.valid ? a.pos[F.pidx] : 0.0;
    F.pi.y = F.valid ? a.pos[a.n + F.pidx] : 0.0;
    F.pi.z = F.valid ? a.pos[2 * a.n + F.pidx] : 0.0;
    if (a.n_drift > 0 && F.valid) {  // drifted since the sort: the image nearest its sorted subtile
      F.pi.x += g.box * rint(((gi[0] + 0.5) * g.side64[0] - F.pi.x) / g.box);
      F.pi.y += g.box * rint(((gi[1] + 0.5) * g.side64[1] - F.pi.y) / g.box);
      F.pi.z += g.box * rint(((gi[2] + 0.5) * g.side64[2] - F.pi.z) / g.box);
    }
  }
  const Real big = Real(1e30);
  F.lo.x = warp_min(F.valid ? F.pi.x : big);
  F.lo.y = warp_min(F.valid ? F.pi.y : big);
  F.lo.z = warp_min(F.valid ? F.pi.z : big);
  F.hi.x = warp_max(F.valid ? F.pi.x : -big);
  F.hi.y = warp_max(F.valid ? F.pi.y : -big);
  F.hi.z = warp_max(F.valid ? F.pi.z : -big);
  if (!F.valid) { F.pi.x = big; F.pi.y = big; F.pi.z = big; }
#pragma unroll
  for (int d = 0; d < 3; ++d) {
    F.elo[d] = __reduce_min_sync(full, F.valid ? e[d] : 1 << 20) - rc.R[d];
    int ehi = __reduce_max_sync(full, F.valid ? e[d] : -(1 << 20)) + rc.R[d];
    F.ext[d] = ehi - F.elo[d] + 1;
    if constexpr (sizeof(Real) == 4) F.org[d] = 0.0f;
    else F.org[d] = (double)F.g0[d] * g.side64[d];
  }
  F.inv_ext[0] = 1.0f / (float)F.ext[2];
  F.inv_ext[1] = 1.0f / (float)F.ext[1];
}

#ifndef P3M_FAST_DECODE
#define P3M_FAST_DECODE 1  // candidate decoding and subtile encoding without integer division
#endif

// Candidate subtile cc (of ncand) of the blocky ball around the chunk's subtile
// block: whether its box gap to the receivers' bounding box is below the reach
// and it holds particles at indices >= clip_from; if so their range and the
// subtile offset.
template <class Real>
__device__ __forceinline__ bool candidate_range(const TraversalArgs& a, const Reach& rc, const ChunkFrame<Real>& F,
                                                int cc, int ncand, int clip_from, int& start, int& cnt,
                                                unsigned& dpk) {
  const Geometry& g = a.g;
  start = 0;
  cnt = 0;
  dpk = 0;
  if (cc >= ncand) return false;
  int t, dx;
  if (P3M_FAST_DECODE && ncand < (1 << 22)) {  // always, unless a drift has widened the block enormously
    t = quot_small(cc, F.ext[2], F.inv_ext[0]);
    dx = quot_small(t, F.ext[1], F.inv_ext[1]);
  } else {
    t = cc / F.ext[2];
    dx = t / F.ext[1];
  }
  int dz = cc - t * F.ext[2];
  int dy = t - dx * F.ext[1];
  dx += F.elo[0]; dy += F.elo[1]; dz += F.elo[2];
  const int dd[3] = {dx, dy, dz};
  const Real blo[3] = {F.lo.x, F.lo.y, F.lo.z}, bhi[3] = {F.hi.x, F.hi.y, F.hi.z};
  Real gap2 = Real(0);
#pragma unroll
  for (int d = 0; d < 3; ++d) {
    Real side;
    if constexpr (sizeof(Real) == 4) side = g.side32[d]; else side = g.side64[d];
    Real jlo = F.org[d] + Real(dd[d]) * side;
    Real jhi = jlo + side;
    Real gp = fmax(fmax(blo[d] - jhi, jlo - bhi[d]), Real(0));
    gap2 += gp * gp;
  }
  Real sub2;
  if constexpr (sizeof(Real) == 4) sub2 = rc.sub2; else sub2 = rc.sub2_d;
  if (!(gap2 < sub2)) return false;
  int gx = F.g0[0] + dx, gy = F.g0[1] + dy, gz = F.g0[2] + dz;
  gx += gx < 0 ? g.M[0] : (gx >= g.M[0] ? -g.M[0] : 0);
  gy += gy < 0 ? g.M[1] : (gy >= g.M[1] ? -g.M[1] : 0);
  gz += gz < 0 ? g.M[2] : (gz >= g.M[2] ? -g.M[2] : 0);
  const int sid = P3M_FAST_DECODE ? encode_subtile_fast(g, gx, gy, gz) : encode_subtile(g, gx, gy, gz);
  start = max(a.offsets[sid], clip_from);
  cnt = a.offsets[sid + 1] - start;
  dpk = pack_delta(dx, dy, dz);
  return cnt > 0;
}

// Append the taken candidates of one round (ballot tm) to the warp's list.
__device__ __forceinline__ void append_round(WarpList& L, int lane, bool take, int start, int cnt, unsigned dpk,
                                             unsigned tm, int& nlist, int& total) {
  const unsigned full = 0xffffffffu;
  int v = take ? cnt : 0;  // inclusive scan of the taken counts
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    int u = __shfl_up_sync(full, v, o);
    if (lane >= o) v += u;
  }
  const int round_total = __shfl_sync(full, v, 31);
  if (take) {
    const int slot = nlist + __popc(tm & ((1u << lane) - 1u));
    L.start[slot] = start;
    L.pre[slot] = total + v - cnt;
    L.delta[slot] = dpk;
  }
  nlist += __popc(tm);
  total += round_total;
}

// Enumerate the subtiles of the blocky ball around the chunk's subtile block
// (32 candidates per round, one per lane), keep those whose box gap to the
// receivers' bounding box is below x_r and that hold particles, and append their
// particle ranges to the warp's list; `proc(nlist, total)` consumes a full list.
// With nparts > 1 only every nparts-th candidate subtile, starting at `part`, is
// enumerated: the parts of a chunk split its suppliers between work items.
template <class Real, class Proc>
__device__ __forceinline__ void enumerate_suppliers(const TraversalArgs& a, const Reach& rc, const ChunkFrame<Real>& F,
                                                    WarpList& L, int lane, int part, int nparts, Proc&& proc) {
  const unsigned full = 0xffffffffu;
  const int ncand_all = F.ext[0] * F.ext[1] * F.ext[2];
  const int ncand = (ncand_all - part + nparts - 1) / nparts;  // candidates of this part
  int nlist = 0, total = 0;
  for (int cb = 0; cb < ncand; cb += kWarp) {
    int start, cnt;
    unsigned dpk;
    const bool take = candidate_range<Real>(a, rc, F, (cb + lane) * nparts + part, ncand_all, 0, start, cnt, dpk);
    const unsigned tm = __ballot_sync(full, take);
    if (tm == 0) continue;
    if (nlist + __popc(tm) > kListCap) {
      __syncwarp();
      proc(nlist, total);
      __syncwarp();
      nlist = 0;
      total = 0;
    }
    append_round(L, lane, take, start, cnt, dpk, tm, nlist, total);
  }
  __syncwarp();
  if (nlist > 0) proc(nlist, total);
  __syncwarp();
}

// As enumerate_suppliers, with the ranges cut to indices >= clip_from, and
// `proc(nlist, total, last)` called from one place: each time the list fills up
// and once more at the end (last = true, possibly with an empty list), so that
// a large consumer is inlined once.
template <class Real, class Proc>
__device__ __forceinline__ void enumerate_suppliers_once(const TraversalArgs& a, const Reach& rc,
                                                         const ChunkFrame<Real>& F, WarpList& L, int lane,
                                                         int clip_from, Proc&& proc) {
  const unsigned full = 0xffffffffu;
  const int ncand = F.ext[0] * F.ext[1] * F.ext[2];
  int nlist = 0, total = 0;
  int cb = 0;
  bool take = false;
  int start = 0, cnt = 0;
  unsigned dpk = 0, tm = 0;
  for (;;) {
    bool overflow = false;
    for (; cb < ncand; cb += kWarp) {
      take = candidate_range<Real>(a, rc, F, cb + lane, ncand, clip_from, start, cnt, dpk);
      tm = __ballot_sync(full, take);
      if (tm == 0) continue;
      if (nlist + __popc(tm) > kListCap) {  // flush first; this batch of candidates is appended after
        overflow = true;
        break;
      }
      append_round(L, lane, take, start, cnt, dpk, tm, nlist, total);
    }
    __syncwarp();
    proc(nlist, total, !overflow);
    __syncwarp();
    if (!overflow) break;
    nlist = 0;
    total = 0;
    append_round(L, lane, take, start, cnt, dpk, tm, nlist, total);
    cb += kWarp;
  }
}

// Load supplier number f of the list (lane-parallel): its position in the
// chunk frame (FP32) or its nearest image in absolute coordinates (FP64),
// and for the VJP its masked abar.  Returns whether it can reach the receivers'
// bounding box.
template <class Real, bool VJP>
__device__ __forceinline__ bool load_supplier(const TraversalArgs& a, const WarpList& L, int nlist, int f,
                                              const ChunkFrame<Real>& F, Vec3<Real>& pj, Vec3<Real>& aj,
                                              Real* gap2_out = nullptr) {
  int lo_e = 0, hi_e = nlist - 1;  // last entry with pre <= f
  while (lo_e < hi_e) {
    int mid = (lo_e + hi_e + 1) >> 1;
    if (L.pre[mid] <= f) lo_e = mid; else hi_e = mid - 1;
  }
  int j = L.start[lo_e] + (f - L.pre[lo_e]);
  int dx, dy, dz;
  unpack_delta(L.delta[lo_e], dx, dy, dz);
  if constexpr (sizeof(Real) == 4) {
    float4 r = a.rel4[j];
    pj.x = fmaf((float)dx, a.g.side32[0], r.x);
    pj.y = fmaf((float)dy, a.g.side32[1], r.y);
    pj.z = fmaf((float)dz, a.g.side32[2], r.z);
    if (VJP) {
      float4 q = a.abar4[j];
      aj.x = q.x; aj.y = q.y; aj.z = q.z;
    }
  } else {
    int gx = F.g0[0] + dx, gy = F.g0[1] + dy, gz = F.g0[2] + dz;
    double sx = gx < 0 ? -a.g.box : (gx >= a.g.M[0] ? a.g.box : 0.0);
    double sy = gy < 0 ? -a.g.box : (gy >= a.g.M[1] ? a.g.box : 0.0);
    double sz = gz < 0 ? -a.g.box : (gz >= a.g.M[2] ? a.g.box : 0.0);
    pj.x = a.pos[j] + sx;
    pj.y = a.pos[a.n + j] + sy;
    pj.z = a.pos[2 * a.n + j] + sz;
    if (a.n_drift > 0) {  // drifted since the sort: the image nearest the candidate subtile
      pj.x += a.g.box * rint(((gx + 0.5) * a.g.side64[0] - pj.x) / a.g.box);
      pj.y += a.g.box * rint(((gy + 0.5) * a.g.side64[1] - pj.y) / a.g.box);
      pj.z += a.g.box * rint(((gz + 0.5) * a.g.side64[2] - pj.z) / a.g.box);
    }
    if (VJP) {
      aj.x = a.abar_d[j]; aj.y = a.abar_d[a.n + j]; aj.z = a.abar_d[2 * a.n + j];
    }
  }
  Real tx = fmax(fmax(F.lo.x - pj.x, pj.x - F.hi.x), Real(0));
  Real ty = fmax(fmax(F.lo.y - pj.y, pj.y - F.hi.y), Real(0));
  Real tz = fmax(fmax(F.lo.z - pj.z, pj.z - F.hi.z), Real(0));
  const Real gap2 = tx * tx + ty * ty + tz * tz;
  if (gap2_out) *gap2_out = gap2;
  return gap2 < Real(a.f.margin2_f);
}

// Generic path (FP64 forward, and the adjoint in both precisions): every
// surviving supplier is broadcast with shuffles and evaluated by all lanes.
template <class Real, bool VJP, int SOFT>
__device__ __forceinline__ void process_list(const TraversalArgs& a, const WarpList& L, int nlist, int total, int lane,
                                             const ChunkFrame<Real>& F, const Vec3<Real>& abar_i, Vec3<Real>& acc,
                                             int& hits) {
  const unsigned full = 0xffffffffu;
  for (int b = 0; b < total; b += kWarp) {
    int f = b + lane;
    Vec3<Real> pj = {Real(0), Real(0), Real(0)};
    Vec3<Real> aj = {Real(0), Real(0), Real(0)};
    bool keep = false;
    if (f < total) keep = load_supplier<Real, VJP>(a, L, nlist, f, F, pj, aj);
    unsigned m = __ballot_sync(full, keep);
    while (m) {
      int src = __ffs(m) - 1;
      m &= m - 1;
      Real xj = __shfl_sync(full, pj.x, src);
      Real yj = __shfl_sync(full, pj.y, src);
      Real zj = __shfl_sync(full, pj.z, src);
      Real dx = F.pi.x - xj, dy = F.pi.y - yj, dz = F.pi.z - zj;
      Real r2 = dx * dx + dy * dy + dz * dz;
      bool hit;
      if constexpr (sizeof(Real) == 4) hit = r2 < a.f.xr2_f; else hit = r2 < a.f.xr2_d;
      Vec3<Real> vj;
      if (VJP) {
        vj.x = __shfl_sync(full, aj.x, src);
        vj.y = __shfl_sync(full, aj.y, src);
        vj.z = __shfl_sync(full, aj.z, src);
      }
      if (__any_sync(full, hit)) {
        Real B, D = Real(0);
        if constexpr (sizeof(Real) == 4) {
          float Dm = 0.f;
          B = bracket_main_f32<SOFT, VJP>(r2, a.f, Dm);
          D = Dm;
          // forward: a zero displacement contributes nothing, so r = 0 skips the
          // softened branch; the VJP needs B(0) for coincident distinct particles
          bool rare = hit && (r2 < a.f.rsw2_f) && (VJP || r2 > 0.0f);
          if (__any_sync(full, rare)) {
            float Ds = 0.f;
            float Bs = bracket_soft_f32<SOFT, VJP>(r2, a.f, a.sc, Ds);
            if (rare) { B = Bs; D = Ds; }
          }
        } else {
          B = (hit && (VJP || r2 > 0.0)) ? bracket_f64<SOFT, VJP>(r2, a.f, a.sc, D) : 0.0;
        }
        if (!hit || (!VJP && r2 == Real(0))) { B = Real(0); D = Real(0); }
        if (VJP) {
          Real vx = abar_i.x - vj.x, vy = abar_i.y - vj.y, vz = abar_i.z - vj.z;
          Real c = D * (dx * vx + dy * vy + dz * vz);
          acc.x += B * vx + c * dx;
          acc.y += B * vy + c * dy;
          acc.z += B * vz + c * dz;
        } else {
          acc.x += B * dx;
          acc.y += B * dy;
          acc.z += B * dz;
        }
        hits += hit ? 1 : 0;
      }
    }
  }
}

template <class Real>
__device__ __forceinline__ void store_result(const TraversalArgs& a, const ChunkFrame<Real>& F, const Vec3<Real>& acc) {
  if (!F.valid) return;
  const Real s = -Real(a.f.G_m);
  Real* o = (Real*)a.out;
  o[F.pidx] = s * acc.x;
  o[a.n + F.pidx] = s * acc.y;
  o[2 * a.n + F.pidx] = s * acc.z;
}

__device__ __forceinline__ int next_chunk(const TraversalArgs& a, int lane) {
  int c = 0;
  if (lane == 0) c = atomicAdd(a.counter, 1);
  return __shfl_sync(0xffffffffu, c, 0);
}

// The c-th chunk to process (c < n_chunks): the chunk list is in the sorted, spatial
// order, which keeps neighbouring chunks, and the suppliers they share, together in L2.
__device__ __forceinline__ Chunk chunk_at(const TraversalArgs& a, int c) { return a.chunks[c]; }

// Work items per chunk of the one-sided kernel: with few chunks (sparse receivers,
// the deepest rungs) each chunk's candidate subtiles are split between up to
// kMaxParts work items so that every resident warp has work; their partial sums
// are added in a fixed order by k_parts_finish.
__host__ __device__ __forceinline__ int parts_for(int n_chunks) {
  if (n_chunks <= 0) return 1;
  const int k = kPartItems / n_chunks;
  return k < 1 ? 1 : (k > kMaxParts ? kMaxParts : k);
}

template <class Real, bool VJP, int SOFT>
__global__ void __launch_bounds__(kForceThreads) k_traverse(TraversalArgs a) {
  __shared__ WarpList lists[kForceWarps];
  const unsigned full = 0xffffffffu;
  const int lane = threadIdx.x & 31;
  WarpList& L = lists[threadIdx.x >> 5];
  const int n_chunks = *a.n_chunks;
  const Reach rc = make_reach(a);
  unsigned long long pair_total = 0;
  for (;;) {
    const int c = next_chunk(a, lane);
    if (c >= n_chunks) break;
    ChunkFrame<Real> F;
    load_chunk<Real>(a, rc, chunk_at(a, c), lane, F);
    Vec3<Real> abar_i = {Real(0), Real(0), Real(0)};
    if (VJP && F.valid) {
      if constexpr (sizeof(Real) == 4) {
        float4 q = a.abar4[F.pidx];
        abar_i.x = q.x; abar_i.y = q.y; abar_i.z = q.z;
      } else {
        abar_i.x = a.abar_d[F.pidx]; abar_i.y = a.abar_d[a.n + F.pidx]; abar_i.z = a.abar_d[2 * a.n + F.pidx];
      }
    }
    Vec3<Real> acc = {Real(0), Real(0), Real(0)};
    int hits = 0;
    enumerate_suppliers<Real>(a, rc, F, L, lane, 0, 1, [&](int nlist, int total) {
      process_list<Real, VJP, SOFT>(a, L, nlist, total, lane, F, abar_i, acc, hits);
    });
    store_result<Real>(a, F, acc);
    if (F.valid) hits -= 1;  // the receiver met itself once (r = 0)
    pair_total += (unsigned long long)__reduce_add_sync(full, (unsigned)hits);
  }
  if (lane == 0 && pair_total) atomicAdd(a.pairs, pair_total);
}

// ---------------------------------------------------------------------------
// FP32 forward, packed broadcast variant: the structure of the generic kernel
// (32 receivers per warp, every surviving supplier tested by all lanes), but
// the survivors of a batch are staged, compacted and negated, in shared memory
// as packed pairs, read back with broadcast loads, and two suppliers are
// evaluated per step in f32x2 arithmetic.
// ---------------------------------------------------------------------------

constexpr int kPThreads = 128;
constexpr int kPWarps = kPThreads / kWarp;
constexpr float kR2Floor = 1e-24f;    // added to r^2 in the packed forward kernel
constexpr float kR2Self = 1e-23f;     // r^2 below this: a zero displacement
constexpr float kCutScale = 0x1p64f;  // cutoff mask: sat((x_r^2 - r^2) 2^64)

// saturate(a * b + c) in one FP32 instruction
__device__ __forceinline__ float fma_sat(float a, float b, float c) {
  float d;
  asm("fma.rn.sat.f32 %0, %1, %2, %3;" : "=f"(d) : "f"(a), "f"(b), "f"(c));
  return d;
}

// cp.async of 16 bytes into shared memory (completion per thread, by commit groups)
__device__ __forceinline__ void cp_async16(void* smem, const void* gmem) {
  const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 16;" ::"r"(s), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_prev() { asm volatile("cp.async.wait_group 1;" ::: "memory"); }

// As P3M_SYM_CPASYNC for the one-sided kernel (2.087 -> 2.052 ms all active on the
// 128^3 set).
#ifndef P3M_GP_CPASYNC
#define P3M_GP_CPASYNC 1
#endif

struct PackedSmem {
  WarpList L;
  float4 sxy[kWarp / 2 + 1];  // (-xa, -xb, -ya, -yb)
  float2 sz[kWarp / 2 + 1];   // (-za, -zb)
#if P3M_GP_CPASYNC
  float4 rec[2][kWarp];       // records of the current and the next batch
#endif
};

// 7 resident blocks of 4 warps per SM bound the kernel to 70 registers (no
// spills); with the cp.async staging measured best among 5 to 8 on the state of the
// 128^3 set after 25 benchmark steps (deep-rung substep 3% faster than with 6).
#ifndef P3M_GP_SOFT2
#define P3M_GP_SOFT2 1  // close pairs of both halves in one packed softened evaluation
#endif
#ifndef P3M_GP_UNROLL
#define P3M_GP_UNROLL 2  // supplier pairs per loop iteration (2: 2-3% faster than 1 on the 128^3 set)
#endif
constexpr int kGpUnroll = P3M_GP_UNROLL;
#ifndef P3M_GP_MINBLOCKS
#define P3M_GP_MINBLOCKS 7
#endif

template <int SOFT, bool TABLE = false>
__global__ void __launch_bounds__(kPThreads, P3M_GP_MINBLOCKS) k_force_packed(TraversalArgs a) {
  __shared__ PackedSmem smem[kPWarps];
  extern __shared__ float tab[];  // TABLE: the bracket table (n_table floats)
  if (TABLE) {
    for (int i = threadIdx.x; i < a.n_table; i += blockDim.x) tab[i] = a.table[i];
    __syncthreads();
  }

  const unsigned full = 0xffffffffu;
  const int lane = threadIdx.x & 31;
  PackedSmem& S = smem[threadIdx.x >> 5];
  const int n_chunks = *a.n_chunks;
  const int nparts = a.part_acc ? parts_for(n_chunks) : 1;
  const int n_items = n_chunks * nparts;
  const Reach rc = make_reach(a);
  const float xr2 = a.f.xr2_f;
  const float xr2s = xr2 * kCutScale;
  unsigned long long pair_total = 0;
  for (;;) {
    const int w = next_chunk(a, lane);
    if (w >= n_items) break;
    const int c = w / nparts, part = w - c * nparts;
    ChunkFrame<float> F;
    load_chunk<float>(a, rc, chunk_at(a, c), lane, F);
    const f2 px = pk(F.pi.x, F.pi.x), py = pk(F.pi.y, F.pi.y), pz = pk(F.pi.z, F.pi.z);
    f2 ax = pk(0.f, 0.f), ay = pk(0.f, 0.f), az = pk(0.f, 0.f);
    f2 hitsf = pk(0.f, 0.f);  // interacting pairs of this lane (exact integers in FP32)
    enumerate_suppliers<float>(a, rc, F, S.L, lane, part, nparts, [&](int nlist, int total) {
      float* sxy = (float*)S.sxy;
      float* sz = (float*)S.sz;
      const WarpList& L = S.L;
      // Supplier f = b + lane of batch b lies in list entry e_cur + (number of
      // entries starting in (b, b + lane]); the start positions of the next 32
      // entries are gathered into one bit mask with a warp OR-reduction.
      int e_cur = 0;  // entry holding position b
      auto locate = [&](int b, int& j, unsigned& dpk) -> bool {
        const int ek = e_cur + 1 + lane;
        const int pos = (ek < nlist) ? L.pre[ek] - b : 64;
        const unsigned bit = (pos > 0 && pos < kWarp) ? (1u << pos) : 0u;
        const unsigned starts = __reduce_or_sync(full, bit);
        const bool at_end = __any_sync(full, pos == kWarp);
        const unsigned upto = (lane == kWarp - 1) ? 0xffffffffu : ((2u << lane) - 1u);
        const int e = e_cur + __popc(starts & upto);
        e_cur += __popc(starts) + (at_end ? 1 : 0);
        const bool have = b + lane < total;
        j = have ? L.start[e] + (b + lane - L.pre[e]) : 0;
        dpk = have ? L.delta[e] : 0u;
        return have;
      };
      // software pipeline: the record of batch b + 32 is loaded while batch b is evaluated
      int jn;
      unsigned dn;
      bool vn = locate(0, jn, dn);
#if P3M_GP_CPASYNC
      int buf = 0;
      if (vn) cp_async16(&S.rec[0][lane], a.rel4 + jn);
      cp_async_commit();
#else
      float4 rn = vn ? a.rel4[jn] : make_float4(0.f, 0.f, 0.f, 0.f);
#endif
      for (int b = 0; b < total; b += kWarp) {
        const bool have = vn;
        const unsigned dpk = dn;
        vn = (b + kWarp < total) ? locate(b + kWarp, jn, dn) : false;
#if P3M_GP_CPASYNC
        if (vn) cp_async16(&S.rec[buf ^ 1][lane], a.rel4 + jn);
        cp_async_commit();
        cp_async_wait_prev();  // this lane's copy of batch b has landed
        const float4 r = have ? S.rec[buf][lane] : make_float4(0.f, 0.f, 0.f, 0.f);
        buf ^= 1;
#else
        const float4 r = rn;
        if (vn) rn = a.rel4[jn];
#endif
        bool keep = false, near = false;
        Vec3<float> pj = {0.f, 0.f, 0.f};
        if (have) {
          int dx, dy, dz;
          unpack_delta(dpk, dx, dy, dz);
          pj.x = fmaf((float)dx, a.g.side32[0], r.x);
          pj.y = fmaf((float)dy, a.g.side32[1], r.y);
          pj.z = fmaf((float)dz, a.g.side32[2], r.z);
          const float tx = fmaxf(fmaxf(F.lo.x - pj.x, pj.x - F.hi.x), 0.f);
          const float ty = fmaxf(fmaxf(F.lo.y - pj.y, pj.y - F.hi.y), 0.f);
          const float tz = fmaxf(fmaxf(F.lo.z - pj.z, pj.z - F.hi.z), 0.f);
          const float gap2 = fmaf(tx, tx, fmaf(ty, ty, tz * tz));
          keep = gap2 < a.f.margin2_f;
          // can this supplier come closer than r_sw to some receiver?  (the box gap
          // is a lower bound of every receiver distance)
          near = keep && gap2 < a.f.rsw2_f;
        }
        const unsigned m = __ballot_sync(full, keep);
        const int nsurv = __popc(m);
        if (keep) {
          const int k = __popc(m & ((1u << lane) - 1u));
          const int p = k >> 1, h = k & 1;
          sxy[4 * p + h] = -pj.x;
          sxy[4 * p + 2 + h] = -pj.y;
          sz[2 * p + h] = -pj.z;
        }
        if (lane == 0 && (nsurv & 1)) {  // pad the last pair far from every receiver (finite B there)
          const int p = nsurv >> 1;
          sxy[4 * p + 1] = 1e10f;
          sxy[4 * p + 3] = 1e10f;
          sz[2 * p + 1] = 1e10f;
        }
        __syncwarp();
        const int npairs = (nsurv + 1) >> 1;
        // Batches with no supplier within r_sw of the receivers' box run a loop
        // without the softened-branch test (a vote and a branch per step).
        auto run_pairs = [&](auto check_soft) {
          constexpr bool kCheckSoft = decltype(check_soft)::value;
#pragma unroll kGpUnroll
        for (int p = 0; p < npairs; ++p) {
          const float4 s = S.sxy[p];
          const float2 z = S.sz[p];
          const f2 dx = add2(px, pk(s.x, s.y));
          const f2 dy = add2(py, pk(s.z, s.w));
          const f2 dz = add2(pz, pk(z.x, z.y));
          // r^2 + 1e-24: a zero displacement (the receiver itself, coincident
          // particles) gets a large but finite B and contributes B * 0 = 0; the
          // offset is far below one ulp of the r^2 near the cutoff, and below the
          // square of the smallest non-zero displacement of subtile-relative FP32
          // coordinates, so no cutoff decision changes
          const f2 r2 = fma2(dx, dx, fma2(dy, dy, fma2(dz, dz, pk(kR2Floor, kR2Floor))));
          float q0, q1;
          upk(r2, q0, q1);
          const bool h0 = q0 < xr2, h1 = q1 < xr2;
          if (__any_sync(full, h0 || h1)) {
            // cutoff mask in the FP32 pipe: 1 iff r^2 < x_r^2 (exact: the scale is a power of two)
            const f2 c = pk(fma_sat(q0, -kCutScale, xr2s), fma_sat(q1, -kCutScale, xr2s));
            hitsf = add2(hitsf, c);
            f2 B;
            if (TABLE) {  // nearest-grid-point lookup in r^2 (softening included)
              const int i0 = min((int)(fminf(q0, a.f.xr2_f) * a.table_scale), a.n_table - 1);
              const int i1 = min((int)(fminf(q1, a.f.xr2_f) * a.table_scale), a.n_table - 1);
              B = pk(tab[max(i0, 0)], tab[max(i1, 0)]);
            } else {
              B = bracket_main_f32x2<SOFT>(r2, a.f);
              if (kCheckSoft) {
                const bool rare0 = h0 && (q0 < a.f.rsw2_f) && (q0 > kR2Self);
                const bool rare1 = h1 && (q1 < a.f.rsw2_f) && (q1 > kR2Self);
                if (__any_sync(full, rare0 || rare1)) {
#if P3M_GP_SOFT2
                  float b0, b1, s0, s1;
                  upk(B, b0, b1);
                  upk(bracket_soft_f32x2<SOFT>(r2, a.f, a.sc), s0, s1);
#else
                  float b0, b1, Ds;
                  upk(B, b0, b1);
                  const float s0 = bracket_soft_f32<SOFT, false>(q0, a.f, a.sc, Ds);
                  const float s1 = bracket_soft_f32<SOFT, false>(q1, a.f, a.sc, Ds);
#endif
                  if (rare0) b0 = s0;
                  if (rare1) b1 = s1;
                  B = pk(b0, b1);
                }
              }
            }
            B = mul2(B, c);
            ax = fma2(B, dx, ax);
            ay = fma2(B, dy, ay);
            az = fma2(B, dz, az);
          }
        }
        };
        if (TABLE || __any_sync(full, near)) run_pairs(std::true_type{});
        else run_pairs(std::false_type{});
        __syncwarp();
      }
    });
    Vec3<float> acc;
    float l, h;
    upk(ax, l, h);
    acc.x = l + h;
    upk(ay, l, h);
    acc.y = l + h;
    upk(az, l, h);
    acc.z = l + h;
    if (nparts == 1) store_result<float>(a, F, acc);
    else a.part_acc[(int64_t)w * kWarp + lane] = make_float4(acc.x, acc.y, acc.z, 0.f);
    upk(hitsf, l, h);
    // the receiver met itself once (r = 0), in the part that holds its own subtile; every
    // part counts its hits, and part 0 takes off one per receiver
    const int hits = F.valid ? (int)(l + h) - (part == 0 ? 1 : 0) : 0;
    // signed: a part-0 lane whose own subtile lies in another part counts -1; the sum
    // over a chunk's parts is exact, and the 64-bit total wraps back
    pair_total += (unsigned long long)(long long)__reduce_add_sync(full, hits);
  }
  if (lane == 0 && pair_total) atomicAdd(a.pairs, pair_total);
}

// acc = -G m (sum of the parts of each chunk, in part order), when k_force_packed
// split its chunks (nothing to do otherwise).  One warp per chunk position.
__global__ void k_parts_finish(TraversalArgs a) {
  const int n_chunks = *a.n_chunks;
  const int nparts = parts_for(n_chunks);
  if (nparts == 1) return;
  const int lane = threadIdx.x & 31;
  const int nw = (gridDim.x * blockDim.x) >> 5;
  const float s = -(float)a.f.G_m;
  float* o = (float*)a.out;
  for (int c = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; c < n_chunks; c += nw) {
    const Chunk ch = chunk_at(a, c);
    if (lane >= ch.count) continue;
    const int pidx = a.active_idx ? a.active_idx[ch.start + lane] : ch.start + lane;
    float x = 0.f, y = 0.f, z = 0.f;
    for (int k = 0; k < nparts; ++k) {
      const float4 v = a.part_acc[((int64_t)c * nparts + k) * kWarp + lane];
      x += v.x;
      y += v.y;
      z += v.z;
    }
    o[pidx] = s * x;
    o[a.n + pidx] = s * y;
    o[2 * a.n + pidx] = s * z;
  }
}

// ---------------------------------------------------------------------------
// FP32 forward with Newton's third law, for calls in which every particle is a
// receiver.  The paper pairs two neighbouring tiles only once and updates the
// particles of both (Section 2.1.3); here each unordered pair {i, j} of sorted
// indices i < j is evaluated once, by the chunk that holds i, and both
// particles receive their share.  The chunk's supplier ranges are cut to
// indices >= its first receiver, and suppliers of the chunk itself are masked
// to j > i.
//
// The survivors of the box test are staged 64 at a time as 32 packed pairs.  A
// block of P pairs (P a power of two <= 32) takes P steps: at step k, lane l
// evaluates its receiver against pair (l + k) mod P of its group of P lanes, so
// that every receiver meets every pair once and no two lanes of a group touch
// one supplier at the same time.  Each pair's accumulator travels with it from
// lane to lane by warp shuffles; at the end of the block the groups' partial
// sums are reduced and added, like the receivers' own sums at the end of the
// chunk, into an FP32 float4 array with vector atomics.  k_sym_finish scales
// that array into the caller's 3 x n output.  Pairs closer than r_sw (the
// softened form) are evaluated in the step: when some lane holds one, one packed
// softened evaluation serves both halves and each half selects its form
// (P3M_SYM_SOFT_INLINE; 0 builds the earlier variant, which queues them per warp
// and evaluates them 32 at a time, one per lane, with atomics to both particles).
// ---------------------------------------------------------------------------

constexpr float kSymPad = 1e10f;  // padding supplier at -1e10, invalid receiver at +1e10: finite B, no hit

// Supplier records of the next batch: copied into a per-warp shared-memory double
// buffer with cp.async while the current batch is staged (1), or prefetched into
// registers (0).  Measured on the 128^3 set: 1.551 -> 1.518 ms.
#ifndef P3M_SYM_CPASYNC
#define P3M_SYM_CPASYNC 1
#endif

struct SymSmem {
  WarpList L;
  float4 sxy[kWarp];  // pair q: (-x_a, -x_b, -y_a, -y_b) of suppliers a = q and b = q + P
  float2 sz[kWarp];   // (-z_a, -z_b)
  int2 sj[kWarp];     // (j_a, j_b): sorted indices, -1 for padding
  int rq[3 * kWarp];  // forward: pairs closer than r_sw (receiver lane | pair << 5 | half << 10)
#if P3M_SYM_CPASYNC
  float4 rec[2][kWarp];  // records of the current and the next batch
#endif
};


struct SymVjpSmem : SymSmem {
  float4 vxy[kWarp];  // adjoint: the suppliers' masked abar, negated, in the layout of sxy / sz
  float2 vz[kWarp];
};

// Resident blocks of 4 warps per SM: the forward at 8 (64 registers, no spills;
// with the close pairs evaluated in the step it is 7% faster than at 5 on the
// 128^3 set), the adjoint at 6 (80 registers; its softened branch with the
// derivative spills beyond).
#ifndef P3M_SYM_SOFT_INLINE
#define P3M_SYM_SOFT_INLINE 1  // forward close pairs: 1 = packed softened form in the step (5-8% faster), 0 = queue
#endif
#ifndef P3M_SYM_OWN_TRIANGLE
#define P3M_SYM_OWN_TRIANGLE 1  // forward: the chunk's own pairs in a triangular pass, not staged
#endif
#ifndef P3M_SYM_UNROLL
#define P3M_SYM_UNROLL 1  // rotation steps per loop iteration
#endif
constexpr int kSymUnroll = P3M_SYM_UNROLL;
#ifndef P3M_SYM_MINBLOCKS
#define P3M_SYM_MINBLOCKS 8
#endif
#ifndef P3M_SYMV_MINBLOCKS
#define P3M_SYMV_MINBLOCKS 6  // the adjoint instance
#endif

__device__ __forceinline__ f2 shfl2(f2 v, int src) {
  f2 r;
  r.v = __shfl_sync(0xffffffffu, v.v, src);
  return r;
}
__device__ __forceinline__ f2 shfl_xor2(f2 v, int o) {
  f2 r;
  r.v = __shfl_xor_sync(0xffffffffu, v.v, o);
  return r;
}

// VJP = true: the adjoint with the same traversal.  Its pair term J_ij (v_i - v_j),
// v the masked abar, is antisymmetric in (i, j) like the force, so the partner
// receives the negated term; every particle is a receiver.
template <int SOFT, bool VJP = false>
__global__ void __launch_bounds__(kPThreads, VJP ? P3M_SYMV_MINBLOCKS : P3M_SYM_MINBLOCKS) k_force_sym(TraversalArgs a, float4* __restrict__ acc4) {
  using Smem = typename std::conditional<VJP, SymVjpSmem, SymSmem>::type;
  __shared__ Smem smem[kPWarps];
  const unsigned full = 0xffffffffu;
  const int lane = threadIdx.x & 31;
  const unsigned lt_mask = (1u << lane) - 1u;
  Smem& S = smem[threadIdx.x >> 5];
  float* sxy = (float*)S.sxy;
  float* szf = (float*)S.sz;
  int* sjf = (int*)S.sj;
  float* vxy = nullptr;
  float* vzf = nullptr;
  if constexpr (VJP) {
    vxy = (float*)S.vxy;
    vzf = (float*)S.vz;
  }
  const int n_chunks = *a.n_chunks;
  const Reach rc = make_reach(a);
  const float xr2 = a.f.xr2_f;
  const float xr2s = xr2 * kCutScale;
  unsigned long long pair_total = 0;
  for (;;) {
    const int c = next_chunk(a, lane);
    if (c >= n_chunks) break;
    const Chunk ch = chunk_at(a, c);
    ChunkFrame<float> F;
    load_chunk<float>(a, rc, ch, lane, F);
    const int i_self = F.valid ? F.pidx : 0x7fffffff;  // the mask j > i is false on empty lanes
    const int c_end = ch.start + ch.count;
    const float rx = F.valid ? F.pi.x : kSymPad, ry = F.valid ? F.pi.y : kSymPad, rz = F.valid ? F.pi.z : kSymPad;
    const f2 px = pk(rx, rx), py = pk(ry, ry), pz = pk(rz, rz);
    f2 vix = pk(0.f, 0.f), viy = pk(0.f, 0.f), viz = pk(0.f, 0.f);  // adjoint: the receiver's masked abar
    float4 ab = make_float4(0.f, 0.f, 0.f, 0.f);
    if constexpr (VJP) {
      if (F.valid) ab = a.abar4[F.pidx];
      vix = pk(ab.x, ab.x);
      viy = pk(ab.y, ab.y);
      viz = pk(ab.z, ab.z);
    }
    f2 ax = pk(0.f, 0.f), ay = pk(0.f, 0.f), az = pk(0.f, 0.f);
    f2 hitsf = pk(0.f, 0.f);
    int cnt = 0;                          // staged suppliers (warp-uniform)
    bool blk_near = false, blk_own = false;  // the staged block holds a supplier near the box / of this chunk

    auto stage = [&](int rank, const Vec3<float>& pj, int j, const float4& aj) {
      const int q = rank & (kWarp - 1), h = rank >> 5;
      sxy[4 * q + h] = -pj.x;
      sxy[4 * q + 2 + h] = -pj.y;
      szf[2 * q + h] = -pj.z;
      sjf[2 * q + h] = j;
      if constexpr (VJP) {
        vxy[4 * q + h] = -aj.x;
        vxy[4 * q + 2 + h] = -aj.y;
        vzf[2 * q + h] = -aj.z;
      }
    };

    // Evaluate the staged block of nsup suppliers (1 <= nsup <= 64) against the chunk.
    auto eval_block = [&](int nsup) {
      int P = kWarp;
      if (nsup < 2 * kWarp) {
        const int half = (nsup + 1) >> 1;
        P = 1;
        while (P < half) P <<= 1;
        // pair q = (supplier q, supplier q + P): move q + P < 32 from the a halves to the b halves
        if (nsup <= kWarp && lane >= P && lane < nsup) {
          const int q = lane - P;
          sxy[4 * q + 1] = sxy[4 * lane];
          sxy[4 * q + 3] = sxy[4 * lane + 2];
          szf[2 * q + 1] = szf[2 * lane];
          sjf[2 * q + 1] = sjf[2 * lane];
          if constexpr (VJP) {
            vxy[4 * q + 1] = vxy[4 * lane];
            vxy[4 * q + 3] = vxy[4 * lane + 2];
            vzf[2 * q + 1] = vzf[2 * lane];
          }
        }
        if (lane < P && lane + P >= nsup) {
          sxy[4 * lane + 1] = kSymPad;
          sxy[4 * lane + 3] = kSymPad;
          szf[2 * lane + 1] = kSymPad;
          sjf[2 * lane + 1] = -1;
          if constexpr (VJP) {
            vxy[4 * lane + 1] = 0.f;
            vxy[4 * lane + 3] = 0.f;
            vzf[2 * lane + 1] = 0.f;
          }
        }
        __syncwarp();
      }
      const int qmask = P - 1;
      const int src = (lane & ~qmask) | ((lane + 1) & qmask);
      f2 sax = pk(0.f, 0.f), say = pk(0.f, 0.f), saz = pk(0.f, 0.f);
      int q = lane & qmask;
      int nq = 0;  // queued close pairs (warp-uniform)
      // Evaluate queued close pairs [base, base + count) (count <= 32), one per lane,
      // with the softened form, and add their terms to both particles.
      auto run_rare = [&](int base, int count) {
        const int e = lane < count ? S.rq[base + lane] : 0;
        const int rl = e & (kWarp - 1);
        const float xr = __shfl_sync(full, rx, rl), yr = __shfl_sync(full, ry, rl), zr = __shfl_sync(full, rz, rl);
        const int ir = __shfl_sync(full, i_self, rl);
        float vxr = 0.f, vyr = 0.f, vzr = 0.f;
        if constexpr (VJP) {
          vxr = __shfl_sync(full, ab.x, rl);
          vyr = __shfl_sync(full, ab.y, rl);
          vzr = __shfl_sync(full, ab.z, rl);
        }
        if (lane < count) {
          const int qe = (e >> 5) & (kWarp - 1), he = e >> 10;
          const float ex = xr + sxy[4 * qe + he], ey = yr + sxy[4 * qe + 2 + he], ez = zr + szf[2 * qe + he];
          const int js = sjf[2 * qe + he];
          float tx, ty, tz;
          if constexpr (!VJP) {
            const float r2s = fmaf(ex, ex, fmaf(ey, ey, fmaf(ez, ez, kR2Floor)));
            float Ds;
            const float Bs = bracket_soft_f32<SOFT, false>(r2s, a.f, a.sc, Ds);
            tx = Bs * ex;
            ty = Bs * ey;
            tz = Bs * ez;
          } else {  // B v + D (x_ij . v) x_ij with v = abar_i - abar_j
            const float r2s = fmaf(ex, ex, fmaf(ey, ey, ez * ez));
            float Ds;
            const float Bs = bracket_soft_f32<SOFT, true>(r2s, a.f, a.sc, Ds);
            const float wx = vxr + vxy[4 * qe + he], wy = vyr + vxy[4 * qe + 2 + he], wz = vzr + vzf[2 * qe + he];
            const float cd = Ds * fmaf(ex, wx, fmaf(ey, wy, ez * wz));
            tx = fmaf(Bs, wx, cd * ex);
            ty = fmaf(Bs, wy, cd * ey);
            tz = fmaf(Bs, wz, cd * ez);
          }
          atomicAdd(acc4 + ir, make_float4(tx, ty, tz, 0.f));
          atomicAdd(acc4 + js, make_float4(-tx, -ty, -tz, 0.f));
        }
        __syncwarp();
      };
      auto run = [&](auto check_soft, auto masked) {
        constexpr bool kCheckSoft = decltype(check_soft)::value;
        constexpr bool kMasked = decltype(masked)::value;
#pragma unroll kSymUnroll
        for (int k = 0; k < P; ++k) {
          const float4 s = S.sxy[q];
          const float2 z = S.sz[q];
          const f2 dx = add2(px, pk(s.x, s.y));
          const f2 dy = add2(py, pk(s.z, s.w));
          const f2 dz = add2(pz, pk(z.x, z.y));
          if constexpr (!VJP) {
            const f2 r2 = fma2(dx, dx, fma2(dy, dy, fma2(dz, dz, pk(kR2Floor, kR2Floor))));
            float q0, q1;
            upk(r2, q0, q1);
            // No skip of steps without a hit: with 32 different pairs per step
            // almost every step has one, and the vote costs more than it saves.
            float c0 = fma_sat(q0, -kCutScale, xr2s), c1 = fma_sat(q1, -kCutScale, xr2s);
            if (kMasked) {
              const int2 jj = S.sj[q];
              c0 = jj.x > i_self ? c0 : 0.f;
              c1 = jj.y > i_self ? c1 : 0.f;
            }
            const f2 cm = pk(c0, c1);
            hitsf = add2(hitsf, cm);
            f2 B = bracket_main_f32x2<SOFT>(r2, a.f);
            // Pairs closer than r_sw (the softened form): a cheap vote first, the
            // exact condition (a hit, not a zero displacement) only when some pair
            // is that close; then one packed softened evaluation for both halves
            // (or, in the queue variant, the pairs leave the step's sums for a
            // queue evaluated 32 at a time, one per lane).
            if (kCheckSoft && __any_sync(full, fminf(q0, q1) < a.f.rsw2_f)) {
              const bool rare0 = c0 > 0.f && q0 < a.f.rsw2_f && q0 > kR2Self;
              const bool rare1 = c1 > 0.f && q1 < a.f.rsw2_f && q1 > kR2Self;
#if P3M_SYM_SOFT_INLINE
              if (__any_sync(full, rare0 || rare1)) {  // both halves in one packed softened evaluation
                float b0, b1, s0, s1;
                upk(B, b0, b1);
                upk(bracket_soft_f32x2<SOFT>(r2, a.f, a.sc), s0, s1);
                B = pk(rare0 ? s0 : b0, rare1 ? s1 : b1);
              }
#else
              const unsigned rb0 = __ballot_sync(full, rare0), rb1 = __ballot_sync(full, rare1);
              if (rb0 | rb1) {
                const int n0 = __popc(rb0);
                if (rare0) S.rq[nq + __popc(rb0 & lt_mask)] = lane | (q << 5);
                if (rare1) S.rq[nq + n0 + __popc(rb1 & lt_mask)] = lane | (q << 5) | 1024;
                nq += n0 + __popc(rb1);
                float b0, b1;
                upk(B, b0, b1);
                B = pk(rare0 ? 0.f : b0, rare1 ? 0.f : b1);
                __syncwarp();
                while (nq >= kWarp) {
                  nq -= kWarp;
                  run_rare(nq, kWarp);
                }
              }
#endif
            }
            B = mul2(B, cm);
            ax = fma2(B, dx, ax);
            ay = fma2(B, dy, ay);
            az = fma2(B, dz, az);
            sax = fma2(B, dx, sax);
            say = fma2(B, dy, say);
            saz = fma2(B, dz, saz);
          } else {
            // adjoint: B and D = B'(r)/r, the term B v + D (x_ij . v) x_ij, v = abar_i - abar_j
            // (no r^2 floor: a zero displacement is either masked, the receiver itself,
            // or a coincident pair, which takes the softened branch)
            const f2 r2 = fma2(dx, dx, fma2(dy, dy, mul2(dz, dz)));
            float q0, q1;
            upk(r2, q0, q1);
            float c0 = fma_sat(q0, -kCutScale, xr2s), c1 = fma_sat(q1, -kCutScale, xr2s);
            if (kMasked) {
              const int2 jj = S.sj[q];
              c0 = jj.x > i_self ? c0 : 0.f;
              c1 = jj.y > i_self ? c1 : 0.f;
            }
            const f2 cm = pk(c0, c1);
            hitsf = add2(hitsf, cm);
            const float4 w = S.vxy[q];
            const float2 wz = S.vz[q];
            const f2 vx = add2(vix, pk(w.x, w.y));
            const f2 vy = add2(viy, pk(w.z, w.w));
            const f2 vz2 = add2(viz, pk(wz.x, wz.y));
            f2 D;
            f2 B = bracket_main_vjp_f32x2<SOFT>(r2, a.f, D);
            // close pairs (r < r_sw, coincident ones included) as in the forward, B and
            // B'/r of the softened form; selects, since the main branch is not finite
            // at r = 0
            if (kCheckSoft && __any_sync(full, fminf(q0, q1) < a.f.rsw2_f)) {
              const bool rare0 = c0 > 0.f && q0 < a.f.rsw2_f;
              const bool rare1 = c1 > 0.f && q1 < a.f.rsw2_f;
#if P3M_SYM_SOFT_INLINE
              if (__any_sync(full, rare0 || rare1)) {  // both halves in one packed softened evaluation
                f2 Dsp;
                float b0, b1, d0, d1, s0, s1, e0, e1;
                upk(B, b0, b1);
                upk(D, d0, d1);
                upk(bracket_soft_vjp_f32x2<SOFT>(r2, a.f, a.sc, Dsp), s0, s1);
                upk(Dsp, e0, e1);
                B = pk(rare0 ? s0 : b0, rare1 ? s1 : b1);
                D = pk(rare0 ? e0 : d0, rare1 ? e1 : d1);
              }
#else
              const unsigned rb0 = __ballot_sync(full, rare0), rb1 = __ballot_sync(full, rare1);
              if (rb0 | rb1) {
                const int n0 = __popc(rb0);
                if (rare0) S.rq[nq + __popc(rb0 & lt_mask)] = lane | (q << 5);
                if (rare1) S.rq[nq + n0 + __popc(rb1 & lt_mask)] = lane | (q << 5) | 1024;
                nq += n0 + __popc(rb1);
                float b0, b1, d0, d1;
                upk(B, b0, b1);
                upk(D, d0, d1);
                B = pk(rare0 ? 0.f : b0, rare1 ? 0.f : b1);
                D = pk(rare0 ? 0.f : d0, rare1 ? 0.f : d1);
                __syncwarp();
                while (nq >= kWarp) {
                  nq -= kWarp;
                  run_rare(nq, kWarp);
                }
              }
#endif
            }
            if (kMasked) {  // selects: the receiver itself (r = 0) has non-finite main-branch values
              float b0, b1, d0, d1;
              upk(B, b0, b1);
              upk(D, d0, d1);
              B = pk(c0 > 0.f ? b0 : 0.f, c1 > 0.f ? b1 : 0.f);
              D = pk(c0 > 0.f ? d0 : 0.f, c1 > 0.f ? d1 : 0.f);
            } else {
              B = mul2(B, cm);
              D = mul2(D, cm);
            }
            const f2 cc = mul2(D, fma2(dx, vx, fma2(dy, vy, mul2(dz, vz2))));
            ax = fma2(B, vx, fma2(cc, dx, ax));
            ay = fma2(B, vy, fma2(cc, dy, ay));
            az = fma2(B, vz2, fma2(cc, dz, az));
            sax = fma2(B, vx, fma2(cc, dx, sax));
            say = fma2(B, vy, fma2(cc, dy, say));
            saz = fma2(B, vz2, fma2(cc, dz, saz));
          }
          // the pair of lane l + 1 comes to lane l, with its accumulator
          sax = shfl2(sax, src);
          say = shfl2(say, src);
          saz = shfl2(saz, src);
          q = (q + 1) & qmask;
        }
      };
      if (blk_near) {
        if (blk_own) run(std::true_type{}, std::true_type{});
        else run(std::true_type{}, std::false_type{});
      } else {
        if (blk_own) run(std::false_type{}, std::true_type{});
        else run(std::false_type{}, std::false_type{});
      }
      if (nq > 0) {  // the rest of the block's queue, while its suppliers are staged
        run_rare(0, nq);
        nq = 0;
      }
      // after P steps lane l holds the sum of its group for pair l mod P
      for (int o = P; o < kWarp; o <<= 1) {
        sax = add2(sax, shfl_xor2(sax, o));
        say = add2(say, shfl_xor2(say, o));
        saz = add2(saz, shfl_xor2(saz, o));
      }
      if (lane < P) {
        const int2 jj = S.sj[lane];
        float xa, xb, ya, yb, za, zb;
        upk(sax, xa, xb);
        upk(say, ya, yb);
        upk(saz, za, zb);
        if (jj.x >= 0) atomicAdd(acc4 + jj.x, make_float4(-xa, -ya, -za, 0.f));
        if (jj.y >= 0) atomicAdd(acc4 + jj.y, make_float4(-xb, -yb, -zb, 0.f));
      }
      __syncwarp();
    };

    // The chunk's own pairs (forward): lane l with lane l + k, k = 1 ... 16 (k = 16 from
    // the lower half only), each pair {i, j} of the chunk once; the partner's share
    // comes back by a shuffle from lane l - k.  The staged suppliers then start after
    // the chunk, so no block needs the j > i mask.
    constexpr bool kOwnTri = !VJP && P3M_SYM_OWN_TRIANGLE;
    if constexpr (kOwnTri) {
      float ox = 0.f, oy = 0.f, oz = 0.f, oh = 0.f;
#pragma unroll 1
      for (int k = 1; k <= kWarp / 2; ++k) {
        const int m = (lane + k) & (kWarp - 1);
        const float xm = __shfl_sync(full, rx, m), ym = __shfl_sync(full, ry, m), zm = __shfl_sync(full, rz, m);
        const bool vm = __shfl_sync(full, (int)F.valid, m) != 0;
        const bool take = F.valid && vm && (k < kWarp / 2 || lane < kWarp / 2);
        const float dx = rx - xm, dy = ry - ym, dz = rz - zm;
        const float r2 = fmaf(dx, dx, fmaf(dy, dy, fmaf(dz, dz, kR2Floor)));
        const float c = take ? fma_sat(r2, -kCutScale, xr2s) : 0.f;
        oh += c;
        float Dm;
        float B = bracket_main_f32<SOFT, false>(r2, a.f, Dm);
        const bool rare = c > 0.f && r2 < a.f.rsw2_f && r2 > kR2Self;
        if (__any_sync(full, rare)) {
          float Ds;
          const float Bs = bracket_soft_f32<SOFT, false>(r2, a.f, a.sc, Ds);
          if (rare) B = Bs;
        }
        B = c > 0.f ? B : 0.f;  // a select: padded lanes may carry a non-finite B
        const float tx = B * dx, ty = B * dy, tz = B * dz;
        const int from = (lane - k) & (kWarp - 1);
        ox += tx - __shfl_sync(full, tx, from);
        oy += ty - __shfl_sync(full, ty, from);
        oz += tz - __shfl_sync(full, tz, from);
      }
      ax = add2(ax, pk(ox, 0.f));
      ay = add2(ay, pk(oy, 0.f));
      az = add2(az, pk(oz, 0.f));
      hitsf = add2(hitsf, pk(oh, 0.f));
    }

    // Stage the survivors of each batch of 32 list positions; evaluate a block
    // whenever 64 are staged, and the rest once the enumeration is done (one
    // call site of eval_block, so its loops are inlined once).
    enumerate_suppliers_once<float>(
        a, rc, F, S.L, lane, kOwnTri ? c_end : ch.start,
        [&](int nlist, int total, bool last) {
          const WarpList& L = S.L;
          int e_cur = 0;  // list entry holding position b (as in k_force_packed)
          auto locate = [&](int b, int& j, unsigned& dpk) -> bool {
            const int ek = e_cur + 1 + lane;
            const int pos = (ek < nlist) ? L.pre[ek] - b : 64;
            const unsigned bit = (pos > 0 && pos < kWarp) ? (1u << pos) : 0u;
            const unsigned starts = __reduce_or_sync(full, bit);
            const bool at_end = __any_sync(full, pos == kWarp);
            const unsigned upto = (lane == kWarp - 1) ? 0xffffffffu : ((2u << lane) - 1u);
            const int e = e_cur + __popc(starts & upto);
            e_cur += __popc(starts) + (at_end ? 1 : 0);
            const bool have = b + lane < total;
            j = have ? L.start[e] + (b + lane - L.pre[e]) : 0;
            dpk = have ? L.delta[e] : 0u;
            return have;
          };
          int jn;
          unsigned dn;
          bool vn = locate(0, jn, dn);
#if P3M_SYM_CPASYNC
          int buf = 0;
          if (vn) cp_async16(&S.rec[0][lane], a.rel4 + jn);
          cp_async_commit();
          float4 rn = make_float4(0.f, 0.f, 0.f, 0.f);
#else
          float4 rn = vn ? a.rel4[jn] : make_float4(0.f, 0.f, 0.f, 0.f);
#endif
          float4 an = make_float4(0.f, 0.f, 0.f, 0.f);
          if (VJP && vn) an = a.abar4[jn];
          for (int b = 0;; b += kWarp) {
            const bool more = b < total;  // warp-uniform
            bool keep = false, near = false, own = false;
            Vec3<float> pj = {0.f, 0.f, 0.f};
            int j = 0, rank = 0, ns = 0;
            float4 aj = make_float4(0.f, 0.f, 0.f, 0.f);
            if (more) {
              const bool have = vn;
              const unsigned dpk = dn;
              j = jn;
              if (VJP) aj = an;
              vn = (b + kWarp < total) ? locate(b + kWarp, jn, dn) : false;
#if P3M_SYM_CPASYNC
              if (vn) cp_async16(&S.rec[buf ^ 1][lane], a.rel4 + jn);
              cp_async_commit();
              cp_async_wait_prev();  // this lane's copy of batch b has landed
              const float4 r = have ? S.rec[buf][lane] : make_float4(0.f, 0.f, 0.f, 0.f);
              buf ^= 1;
#else
              const float4 r = rn;
              if (vn) rn = a.rel4[jn];
#endif
              if (VJP && vn) an = a.abar4[jn];
              if (have) {
                int ddx, ddy, ddz;
                unpack_delta(dpk, ddx, ddy, ddz);
                pj.x = fmaf((float)ddx, a.g.side32[0], r.x);
                pj.y = fmaf((float)ddy, a.g.side32[1], r.y);
                pj.z = fmaf((float)ddz, a.g.side32[2], r.z);
                const float tx = fmaxf(fmaxf(F.lo.x - pj.x, pj.x - F.hi.x), 0.f);
                const float ty = fmaxf(fmaxf(F.lo.y - pj.y, pj.y - F.hi.y), 0.f);
                const float tz = fmaxf(fmaxf(F.lo.z - pj.z, pj.z - F.hi.z), 0.f);
                const float gap2 = fmaf(tx, tx, fmaf(ty, ty, tz * tz));
                keep = gap2 < a.f.margin2_f;
                near = keep && gap2 < a.f.rsw2_f;
              }
              own = keep && j < c_end;
              const unsigned m = __ballot_sync(full, keep);
              ns = __popc(m);
              rank = cnt + __popc(m & lt_mask);
              if (keep && rank < 2 * kWarp) stage(rank, pj, j, aj);
              blk_near = blk_near || __any_sync(full, near && rank < 2 * kWarp);
              blk_own = blk_own || __any_sync(full, own && rank < 2 * kWarp);
            }
            const bool flush = more ? (cnt + ns >= 2 * kWarp) : (last && cnt > 0);
            if (flush) {
              __syncwarp();
              eval_block(more ? 2 * kWarp : cnt);
              if (more) {
                blk_near = __any_sync(full, near && rank >= 2 * kWarp);
                blk_own = __any_sync(full, own && rank >= 2 * kWarp);
                if (keep && rank >= 2 * kWarp) stage(rank - 2 * kWarp, pj, j, aj);
                cnt += ns - 2 * kWarp;
              } else {
                cnt = 0;
              }
            } else {
              cnt += ns;
            }
            if (!more) break;
          }
        });
    float l, h;
    float4 mine;
    upk(ax, l, h);
    mine.x = l + h;
    upk(ay, l, h);
    mine.y = l + h;
    upk(az, l, h);
    mine.z = l + h;
    mine.w = 0.f;
    if (F.valid) atomicAdd(acc4 + F.pidx, mine);
    upk(hitsf, l, h);
    const int hits = F.valid ? (int)(l + h) : 0;
    pair_total += 2ull * (unsigned long long)__reduce_add_sync(full, (unsigned)hits);  // ordered pairs
  }
  if (lane == 0 && pair_total) atomicAdd(a.pairs, pair_total);
}

// acc = -G m * (sum over partners of B(r) (x_i - x_j)) (or the adjoint's sum), from
// the float4 sums of k_force_sym.
__global__ void k_sym_finish(const float4* __restrict__ acc4, int64_t n, float scale, float* __restrict__ out) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const float4 v = acc4[i];
    out[i] = scale * v.x;
    out[n + i] = scale * v.y;
    out[2 * n + i] = scale * v.z;
  }
}

// ---------------------------------------------------------------------------
// FP32 adjoint, packed broadcast: as k_force_packed, with every particle a
// receiver and the masked abar of each supplier staged beside its position.
//   xbar_k = -G m sum_j [ B v + (B'/r) (x_kj . v) x_kj ],  v = abar_k - abar_j.
// ---------------------------------------------------------------------------

struct PackedVjpSmem {
  WarpList L;
  float4 sxy[kWarp / 2 + 1];  // (-xa, -xb, -ya, -yb)
  float2 sz[kWarp / 2 + 1];   // (-za, -zb)
  float4 vxy[kWarp / 2 + 1];  // (-abar_xa, -abar_xb, -abar_ya, -abar_yb)
  float2 vz[kWarp / 2 + 1];   // (-abar_za, -abar_zb)
};

template <int SOFT>
__global__ void __launch_bounds__(kPThreads, P3M_GP_MINBLOCKS) k_vjp_packed(TraversalArgs a) {
  __shared__ PackedVjpSmem smem[kPWarps];
  const unsigned full = 0xffffffffu;
  const int lane = threadIdx.x & 31;
  PackedVjpSmem& S = smem[threadIdx.x >> 5];
  const int n_chunks = *a.n_chunks;
  const Reach rc = make_reach(a);
  const float xr2 = a.f.xr2_f;
  unsigned long long pair_total = 0;
  for (;;) {
    const int c = next_chunk(a, lane);
    if (c >= n_chunks) break;
    ChunkFrame<float> F;
    load_chunk<float>(a, rc, chunk_at(a, c), lane, F);
    const f2 px = pk(F.pi.x, F.pi.x), py = pk(F.pi.y, F.pi.y), pz = pk(F.pi.z, F.pi.z);
    float4 ab = make_float4(0.f, 0.f, 0.f, 0.f);
    if (F.valid) ab = a.abar4[F.pidx];
    const f2 vix = pk(ab.x, ab.x), viy = pk(ab.y, ab.y), viz = pk(ab.z, ab.z);
    f2 gx = pk(0.f, 0.f), gy = pk(0.f, 0.f), gz = pk(0.f, 0.f);
    int hits = 0;
    enumerate_suppliers<float>(a, rc, F, S.L, lane, 0, 1, [&](int nlist, int total) {
      float* sxy = (float*)S.sxy;
      float* sz = (float*)S.sz;
      float* vxy = (float*)S.vxy;
      float* vz = (float*)S.vz;
      for (int b = 0; b < total; b += kWarp) {
        const int f = b + lane;
        Vec3<float> pj = {0.f, 0.f, 0.f}, aj = {0.f, 0.f, 0.f};
        bool keep = false, near = false;
        if (f < total) {
          float gap2;
          keep = load_supplier<float, true>(a, S.L, nlist, f, F, pj, aj, &gap2);
          near = keep && gap2 < a.f.rsw2_f;  // may come within r_sw of a receiver (or coincide)
        }
        const unsigned m = __ballot_sync(full, keep);
        const int nsurv = __popc(m);
        if (keep) {
          const int k = __popc(m & ((1u << lane) - 1u));
          const int p = k >> 1, h = k & 1;
          sxy[4 * p + h] = -pj.x;
          sxy[4 * p + 2 + h] = -pj.y;
          sz[2 * p + h] = -pj.z;
          vxy[4 * p + h] = -aj.x;
          vxy[4 * p + 2 + h] = -aj.y;
          vz[2 * p + h] = -aj.z;
        }
        if (lane == 0 && (nsurv & 1)) {  // pad the last pair far from every receiver
          const int p = nsurv >> 1;
          sxy[4 * p + 1] = 1e30f;
          sxy[4 * p + 3] = 1e30f;
          sz[2 * p + 1] = 1e30f;
          vxy[4 * p + 1] = 0.f;
          vxy[4 * p + 3] = 0.f;
          vz[2 * p + 1] = 0.f;
        }
        __syncwarp();
        const int npairs = (nsurv + 1) >> 1;
        // as in the forward kernel: batches with no supplier within r_sw of the
        // receivers' box skip the softened-branch test
        auto run_pairs = [&](auto check_soft) {
          constexpr bool kCheckSoft = decltype(check_soft)::value;
#pragma unroll kGpUnroll
        for (int p = 0; p < npairs; ++p) {
          const float4 s = S.sxy[p];
          const float2 z = S.sz[p];
          const f2 dx = add2(px, pk(s.x, s.y));
          const f2 dy = add2(py, pk(s.z, s.w));
          const f2 dz = add2(pz, pk(z.x, z.y));
          const f2 r2 = fma2(dx, dx, fma2(dy, dy, mul2(dz, dz)));
          float q0, q1;
          upk(r2, q0, q1);
          const bool h0 = q0 < xr2, h1 = q1 < xr2;
          if (__any_sync(full, h0 || h1)) {
            hits += (int)h0 + (int)h1;
            const float4 w = S.vxy[p];
            const float2 wz = S.vz[p];
            const f2 vx = add2(vix, pk(w.x, w.y));
            const f2 vy = add2(viy, pk(w.z, w.w));
            const f2 vz2 = add2(viz, pk(wz.x, wz.y));
            // r = 0 in the adjoint: the receiver itself has v = 0; coincident distinct
            // particles take the softened value B(0) (zero for point particles)
            f2 D;
            f2 B = bracket_main_vjp_f32x2<SOFT>(r2, a.f, D);
            float b0, b1, d0, d1;
            upk(B, b0, b1);
            upk(D, d0, d1);
            if (kCheckSoft) {
              const bool rare0 = h0 && (q0 < a.f.rsw2_f), rare1 = h1 && (q1 < a.f.rsw2_f);
              if (__any_sync(full, rare0 || rare1)) {
#if P3M_GP_SOFT2
                f2 Dsp;
                float s0, s1, Ds0, Ds1;
                upk(bracket_soft_vjp_f32x2<SOFT>(r2, a.f, a.sc, Dsp), s0, s1);
                upk(Dsp, Ds0, Ds1);
#else
                float Ds0, Ds1;
                const float s0 = bracket_soft_f32<SOFT, true>(q0, a.f, a.sc, Ds0);
                const float s1 = bracket_soft_f32<SOFT, true>(q1, a.f, a.sc, Ds1);
#endif
                if (rare0) { b0 = s0; d0 = Ds0; }
                if (rare1) { b1 = s1; d1 = Ds1; }
              }
            }
            B = pk(h0 ? b0 : 0.0f, h1 ? b1 : 0.0f);
            D = pk(h0 ? d0 : 0.0f, h1 ? d1 : 0.0f);
            const f2 xv = fma2(dx, vx, fma2(dy, vy, mul2(dz, vz2)));
            const f2 cc = mul2(D, xv);
            gx = fma2(B, vx, fma2(cc, dx, gx));
            gy = fma2(B, vy, fma2(cc, dy, gy));
            gz = fma2(B, vz2, fma2(cc, dz, gz));
          }
        }
        };
        if (__any_sync(full, near)) run_pairs(std::true_type{});
        else run_pairs(std::false_type{});
        __syncwarp();
      }
    });
    Vec3<float> acc;
    float l, h;
    upk(gx, l, h);
    acc.x = l + h;
    upk(gy, l, h);
    acc.y = l + h;
    upk(gz, l, h);
    acc.z = l + h;
    store_result<float>(a, F, acc);
    hits = F.valid ? hits - 1 : 0;  // the receiver met itself once (r = 0)
    pair_total += (unsigned long long)__reduce_add_sync(full, (unsigned)hits);
  }
  if (lane == 0 && pair_total) atomicAdd(a.pairs, pair_total);
}

// ---------------------------------------------------------------------------
// Host side.
// ---------------------------------------------------------------------------

static SeriesConsts make_series() {
  SeriesConsts s{};
  const double two_over_sqrt_pi = 1.12837916709551257390;
  // h(u) = sum_m H_m u^{2m},  H_m = (2/sqrt(pi)) (-1)^m 2(m+1) / ((m+1)! (2m+3))
  double H[kHTermsD + 1];
  double fact = 1.0;
  for (int m = 0; m <= kHTermsD; ++m) {
    fact *= (double)(m + 1);
    H[m] = two_over_sqrt_pi * ((m & 1) ? -1.0 : 1.0) * 2.0 * (m + 1) / (fact * (2.0 * m + 3.0));
  }
  for (int m = 0; m < kHTermsD; ++m) {
    s.h_d[m] = H[m];
    s.hd_d[m] = 2.0 * (m + 1) * H[m + 1];  // h'(u)/u
  }
  for (int m = 0; m < kHTermsF; ++m) {
    s.h_f[m] = (float)s.h_d[m];
    s.hd_f[m] = (float)s.hd_d[m];
  }
  return s;
}

template <class Real, bool VJP, int SOFT>
static cudaError_t launch_traverse(p3m_sr_ctx* ctx, const TraversalArgs& a) {
  constexpr bool packed = (sizeof(Real) == 4);  // FP32: packed broadcast kernels
  static int blocks_per_sm = 0;
  if (blocks_per_sm == 0) {
    if (packed && !VJP)
      cudaOccupancyMaxActiveBlocksPerMultiprocessor(&blocks_per_sm, k_force_packed<SOFT>, kPThreads, 0);
    else if (packed)
      cudaOccupancyMaxActiveBlocksPerMultiprocessor(&blocks_per_sm, k_vjp_packed<SOFT>, kPThreads, 0);
    else
      cudaOccupancyMaxActiveBlocksPerMultiprocessor(&blocks_per_sm, k_traverse<Real, VJP, SOFT>, kForceThreads, 0);
    if (blocks_per_sm < 1) blocks_per_sm = 1;
  }
  unsigned grid = (unsigned)(ctx->num_sms * blocks_per_sm);
  const int slot = VJP ? 1 : 0;
  TraversalArgs ap = a;
  if (packed && !VJP) ap.part_acc = ctx->part_acc;  // sparse receivers: chunks split into parts
  cudaEventRecord(ctx->kt_ev[2 * slot], ctx->stream);
  if (packed && !VJP)
    k_force_packed<SOFT><<<grid, kPThreads, 0, ctx->stream>>>(ap);
  else if (packed)
    k_vjp_packed<SOFT><<<grid, kPThreads, 0, ctx->stream>>>(ap);
  else
    k_traverse<Real, VJP, SOFT><<<grid, kForceThreads, 0, ctx->stream>>>(ap);
  ++ctx->launches;
  cudaEventRecord(ctx->kt_ev[2 * slot + 1], ctx->stream);
  ctx->kt_pending[slot] = true;
  if (packed && !VJP) {
    k_parts_finish<<<(unsigned)(ctx->num_sms * 4), 256, 0, ctx->stream>>>(ap);
    ++ctx->launches;
  }
  return cudaGetLastError();
}

// Newton-III FP32 forward (all particles receivers) or adjoint: zero the float4
// sums, run k_force_sym, scale the sums into a.out.
template <int SOFT, bool VJP>
static cudaError_t launch_sym_soft(p3m_sr_ctx* ctx, const TraversalArgs& a, float4* acc4) {
  static int blocks_per_sm = 0;
  if (blocks_per_sm == 0) {
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&blocks_per_sm, k_force_sym<SOFT, VJP>, kPThreads, 0);
    if (blocks_per_sm < 1) blocks_per_sm = 1;
  }
  cudaStream_t s = ctx->stream;
  cudaError_t e = cudaMemsetAsync(acc4, 0, sizeof(float4) * (size_t)ctx->n, s);
  if (e != cudaSuccess) return e;
  const int slot = VJP ? 1 : 0;
  cudaEventRecord(ctx->kt_ev[2 * slot], s);
  k_force_sym<SOFT, VJP><<<(unsigned)(ctx->num_sms * blocks_per_sm), kPThreads, 0, s>>>(a, acc4);
  ++ctx->launches;
  cudaEventRecord(ctx->kt_ev[2 * slot + 1], s);
  ctx->kt_pending[slot] = true;
  const unsigned fin = (unsigned)std::min<int64_t>((ctx->n + 255) / 256, (int64_t)ctx->num_sms * 16);
  k_sym_finish<<<fin, 256, 0, s>>>(acc4, ctx->n, -(float)a.f.G_m, (float*)a.out);
  ++ctx->launches;
  return cudaGetLastError();
}

template <bool VJP>
static cudaError_t launch_sym(p3m_sr_ctx* ctx, const TraversalArgs& a) {
  float4* acc4 = (float4*)ctx->gather_tmp;  // 32 n bytes, idle outside the sort
  switch (ctx->prm.softening) {
    case P3M_SOFT_NONE: return launch_sym_soft<P3M_SOFT_NONE, VJP>(ctx, a, acc4);
    case P3M_SOFT_PLUMMER: return launch_sym_soft<P3M_SOFT_PLUMMER, VJP>(ctx, a, acc4);
    default: return launch_sym_soft<P3M_SOFT_BSPLINE, VJP>(ctx, a, acc4);
  }
}

template <class Real, bool VJP>
static cudaError_t dispatch_traverse(p3m_sr_ctx* ctx, const TraversalArgs& a) {
  switch (ctx->prm.softening) {
    case P3M_SOFT_NONE: return launch_traverse<Real, VJP, P3M_SOFT_NONE>(ctx, a);
    case P3M_SOFT_PLUMMER: return launch_traverse<Real, VJP, P3M_SOFT_PLUMMER>(ctx, a);
    default: return launch_traverse<Real, VJP, P3M_SOFT_BSPLINE>(ctx, a);
  }
}

// Receiver chunks of the row segments.
static p3m_status build_chunks(p3m_sr_ctx* ctx, const int* act_scan, Chunk* chunks, int* n_chunks_dev,
                               int* n_active_dev) {
  cudaStream_t s = ctx->stream;
  const int n_t = ctx->geo.n_t;
  const int64_t rows = (int64_t)n_t * n_t * ((n_t + kChunkSpan - 1) / kChunkSpan);  // segments
  k_row_chunks<<<blocks_for(rows + 1, 128), 128, 0, s>>>(ctx->offsets, act_scan, n_t, ctx->geo.nsub3,
                                                         ctx->tile_chunks);
  ++ctx->launches;
  p3m_status st = cuda_check(ctx, cudaGetLastError(), "row chunk kernel");
  if (st != P3M_OK) return st;
  st = cuda_check(ctx, scan_exclusive_i32(ctx->tile_chunks, ctx->tile_chunks, rows + 1, ctx->scan_scratch,
                                          ctx->scan_scratch_ints, s, &ctx->launches), "chunk scan");
  if (st != P3M_OK) return st;
  k_write_chunks<<<blocks_for(rows, 128), 128, 0, s>>>(ctx->offsets, act_scan, n_t, ctx->geo.nsub3,
                                                        ctx->tile_chunks, chunks, n_chunks_dev, n_active_dev,
                                                        ctx->n);
  ++ctx->launches;
  return cuda_check(ctx, cudaGetLastError(), "write chunks kernel");
}

p3m_status ensure_all_chunks(p3m_sr_ctx* ctx) {
  if (ctx->all_chunks_built) return P3M_OK;
  p3m_status st = build_chunks(ctx, nullptr, ctx->chunks_all, ctx->dev_small + 1, nullptr);
  if (st == P3M_OK) ctx->all_chunks_built = true;
  return st;
}

static TraversalArgs base_args(p3m_sr_ctx* ctx) {
  static SeriesConsts series = make_series();
  TraversalArgs a{};
  a.g = ctx->geo;
  a.f = ctx->fc;
  a.sc = series;
  a.offsets = ctx->offsets;
  a.cell = ctx->cell;
  a.n = ctx->n;
  a.rel4 = ctx->rel4;
  a.pairs = ctx->pair_count;
  a.drift_slots = ctx->drift_slots;
  a.n_drift = ctx->n_drift;
  a.err = ctx->err_dev;
  return a;
}

static p3m_status prepare_rel4(p3m_sr_ctx* ctx, const double* pos) {
  if (ctx->n == 0) return P3M_OK;
  if (pos == ctx->sorted_pos && !ctx->rel4_stale) return P3M_OK;  // written by the sort for these positions
  k_rel4<<<blocks_for(ctx->n, 256), 256, 0, ctx->stream>>>(pos, ctx->cell, ctx->n, ctx->geo, ctx->rel4);
  ++ctx->launches;
  if (pos == ctx->sorted_pos) ctx->rel4_stale = false;
  return cuda_check(ctx, cudaGetLastError(), "rel4 kernel");
}

}  // namespace p3m

using namespace p3m;

extern "C" p3m_status p3m_sr_build_pairs(p3m_sr_ctx* ctx, const int8_t* rung, int rung_min) {
  if (!ctx) return P3M_ERR_INVALID;
  if (!ctx->sorted) return fail(ctx, P3M_ERR_STATE, "build_pairs: call p3m_sr_sort first");
  p3m_status st = poll_latched(ctx);
  if (st != P3M_OK) return st;
  cudaStream_t s = ctx->stream;
  const int64_t n = ctx->n;
  ctx->all_active = (rung == nullptr);
  const int* act_scan = nullptr;
  if (!ctx->all_active) {
    // receivers per tile of sorted particles, scanned, then flags + act_scan + list in one pass
    const int64_t tiles = (n + 1 + kActTile - 1) / kActTile;  // act_scan has n + 1 entries
    int* tile_count = ctx->hist;                                // idle outside the sort (>= 1024 per radix tile)
    k_active_count<<<(unsigned)tiles, kActThreads, 0, s>>>(rung, n, rung_min, tile_count);
    ++ctx->launches;
    if ((st = cuda_check(ctx, cudaGetLastError(), "active count")) != P3M_OK) return st;
    st = cuda_check(ctx, scan_exclusive_i32(tile_count, tile_count, tiles, ctx->scan_scratch, ctx->scan_scratch_ints, s,
                                            &ctx->launches), "scan");
    if (st != P3M_OK) return st;
    k_active_scan_compact<<<(unsigned)tiles, kActThreads, 0, s>>>(rung, n, rung_min, tile_count, ctx->active_flag,
                                                                   ctx->act_scan, ctx->active_idx);
    ++ctx->launches;
    if ((st = cuda_check(ctx, cudaGetLastError(), "active scan")) != P3M_OK) return st;
    act_scan = ctx->act_scan;
  }
  st = build_chunks(ctx, act_scan, ctx->chunks, ctx->dev_small + 0, ctx->dev_small + 2);
  if (st != P3M_OK) return st;
  ctx->pairs_built = true;
  return P3M_OK;
}

extern "C" p3m_status p3m_sr_forces(p3m_sr_ctx* ctx, const double* pos, int precision, void* acc_out) {
  if (!ctx) return P3M_ERR_INVALID;
  if (precision != 32 && precision != 64) return fail(ctx, P3M_ERR_INVALID, "forces: precision must be 32 or 64");
  if (ctx->n > 0 && (!pos || !acc_out)) return fail(ctx, P3M_ERR_INVALID, "forces: null pointer");
  if (!ctx->sorted || !ctx->pairs_built)
    return fail(ctx, P3M_ERR_STATE, "forces: call p3m_sr_sort and p3m_sr_build_pairs first");
  if (precision == 32 && ctx->prm.x_r > 2.0 * P3M_ERFCX_UMAX * ctx->prm.x_s)
    return fail(ctx, P3M_ERR_INVALID, "forces: the FP32 path needs x_r <= 4.6 x_s");
  p3m_status st = poll_latched(ctx);
  if (st != P3M_OK) return st;
  cudaStream_t s = ctx->stream;
  if ((st = cuda_check(ctx, cudaMemsetAsync(ctx->pair_count, 0, sizeof(unsigned long long), s), "memset")) != P3M_OK)
    return st;
  if (ctx->n == 0) return P3M_OK;
  if (precision == 32 && (st = prepare_rel4(ctx, pos)) != P3M_OK) return st;
  if ((st = cuda_check(ctx, cudaMemsetAsync(ctx->dev_small + 3, 0, sizeof(int), s), "memset")) != P3M_OK) return st;
  TraversalArgs a = base_args(ctx);
  a.pos = pos;
  a.chunks = ctx->chunks;
  a.n_chunks = ctx->dev_small + 0;
  a.counter = ctx->dev_small + 3;
  a.active_idx = ctx->all_active ? nullptr : ctx->active_idx;
  a.out = acc_out;
  cudaError_t e;
  if (precision == 32 && ctx->all_active && ctx->symmetric) e = launch_sym<false>(ctx, a);
  else e = (precision == 32) ? dispatch_traverse<float, false>(ctx, a) : dispatch_traverse<double, false>(ctx, a);
  if ((st = cuda_check(ctx, e, "force kernel")) != P3M_OK) return st;
  report_latched(ctx);
  return P3M_OK;
}

// B(r) in double on the host, for the table of p3m_sr_forces_tabulated.
static double bracket_host(double r, const ForceConsts& f, const SeriesConsts& sc) {
  const double inv_sqrt_pi = 0.56418958354775628695;
  const double r2 = r * r;
  if (r < f.r_sw) {
    if (f.softening == P3M_SOFT_NONE) return 0.0;
    const double u = r / (2.0 * f.x_s), u2 = u * u, w = 2.0 * f.x_s;
    double h = sc.h_d[kHTermsD - 1];
    for (int k = kHTermsD - 2; k >= 0; --k) h = h * u2 + sc.h_d[k];
    double s3;
    if (f.softening == P3M_SOFT_BSPLINE) {
      const double x = r / f.eps_b, c = 32.0 / (f.eps_b * f.eps_b * f.eps_b);
      s3 = (x < 0.5) ? c * (x * x * x - 1.2 * x * x + 1.0 / 3.0)
                     : c * (-x * x * x / 3.0 + 1.2 * x * x - 1.5 * x + 2.0 / 3.0 - 1.0 / (480.0 * x * x * x));
    } else {
      const double p = 1.0 / std::sqrt(r2 + f.eps * f.eps);
      s3 = p * p * p;
    }
    return s3 - h / (w * w * w);
  }
  const double u = r / (2.0 * f.x_s);
  double B = (std::erfc(u) + 2.0 * inv_sqrt_pi * u * std::exp(-u * u)) / (r2 * r);
  if (f.softening == P3M_SOFT_PLUMMER) {
    const double p = 1.0 / std::sqrt(r2 + f.eps * f.eps);
    B += p * p * p - 1.0 / (r2 * r);
  }
  return B;
}

extern "C" p3m_status p3m_sr_forces_tabulated(p3m_sr_ctx* ctx, const double* pos, int table_bits, float* acc_out) {
  if (!ctx) return P3M_ERR_INVALID;
  if (table_bits < 4 || table_bits > 14) return fail(ctx, P3M_ERR_INVALID, "forces_tabulated: table_bits must be 4..14");
  if (ctx->n > 0 && (!pos || !acc_out)) return fail(ctx, P3M_ERR_INVALID, "forces_tabulated: null pointer");
  if (!ctx->sorted || !ctx->pairs_built)
    return fail(ctx, P3M_ERR_STATE, "forces_tabulated: call p3m_sr_sort and p3m_sr_build_pairs first");
  p3m_status st = poll_latched(ctx);
  if (st != P3M_OK) return st;
  cudaStream_t s = ctx->stream;
  const int nt = 1 << table_bits;
  if (ctx->table_bits != table_bits) {
    static SeriesConsts series = make_series();
    std::vector<float> h(nt);
    for (int i = 0; i < nt; ++i) {
      const double r2c = (i + 0.5) * ctx->prm.x_r * ctx->prm.x_r / nt;  // bin centre in r^2
      h[i] = (float)bracket_host(std::sqrt(r2c), ctx->fc, series);
    }
    if (ctx->table) {
      cudaStreamSynchronize(s);
      cudaFree(ctx->table);
      ctx->table = nullptr;
    }
    if ((st = cuda_check(ctx, cudaMalloc((void**)&ctx->table, sizeof(float) * nt), "cudaMalloc(table)")) != P3M_OK)
      return st;
    if ((st = cuda_check(ctx, cudaMemcpy(ctx->table, h.data(), sizeof(float) * nt, cudaMemcpyHostToDevice),
                         "table copy")) != P3M_OK)
      return st;
    ctx->table_bits = table_bits;
  }
  if ((st = cuda_check(ctx, cudaMemsetAsync(ctx->pair_count, 0, sizeof(unsigned long long), s), "memset")) != P3M_OK)
    return st;
  if (ctx->n == 0) return P3M_OK;
  if ((st = prepare_rel4(ctx, pos)) != P3M_OK) return st;
  if ((st = cuda_check(ctx, cudaMemsetAsync(ctx->dev_small + 3, 0, sizeof(int), s), "memset")) != P3M_OK) return st;
  TraversalArgs a = base_args(ctx);
  a.pos = pos;
  a.chunks = ctx->chunks;
  a.n_chunks = ctx->dev_small + 0;
  a.counter = ctx->dev_small + 3;
  a.active_idx = ctx->all_active ? nullptr : ctx->active_idx;
  a.out = acc_out;
  a.table = ctx->table;
  a.part_acc = ctx->part_acc;
  a.n_table = nt;
  a.table_scale = (float)(nt / (ctx->prm.x_r * ctx->prm.x_r));
  const size_t shm = sizeof(float) * nt;
  auto launch = [&](auto kern) {
    cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)shm);
    int bps = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bps, kern, kPThreads, shm);
    const unsigned grid = (unsigned)(ctx->num_sms * (bps > 0 ? bps : 1));
    cudaEventRecord(ctx->kt_ev[0], s);
    kern<<<grid, kPThreads, shm, s>>>(a);
    ++ctx->launches;
    cudaEventRecord(ctx->kt_ev[1], s);
    ctx->kt_pending[0] = true;
    k_parts_finish<<<(unsigned)(ctx->num_sms * 4), 256, 0, s>>>(a);
    ++ctx->launches;
  };
  switch (ctx->prm.softening) {
    case P3M_SOFT_NONE: launch(k_force_packed<P3M_SOFT_NONE, true>); break;
    case P3M_SOFT_PLUMMER: launch(k_force_packed<P3M_SOFT_PLUMMER, true>); break;
    default: launch(k_force_packed<P3M_SOFT_BSPLINE, true>); break;
  }
  if ((st = cuda_check(ctx, cudaGetLastError(), "tabulated force kernel")) != P3M_OK) return st;
  report_latched(ctx);
  return P3M_OK;
}

extern "C" p3m_status p3m_sr_vjp(p3m_sr_ctx* ctx, const double* pos, int precision, const void* acc_bar,
                                 void* pos_bar_out) {
  if (!ctx) return P3M_ERR_INVALID;
  if (precision != 32 && precision != 64) return fail(ctx, P3M_ERR_INVALID, "vjp: precision must be 32 or 64");
  if (ctx->n > 0 && (!pos || !acc_bar || !pos_bar_out)) return fail(ctx, P3M_ERR_INVALID, "vjp: null pointer");
  if (!ctx->sorted || !ctx->pairs_built)
    return fail(ctx, P3M_ERR_STATE, "vjp: call p3m_sr_sort and p3m_sr_build_pairs first");
  if (precision == 32 && ctx->prm.x_r > 2.0 * P3M_ERFCX_UMAX * ctx->prm.x_s)
    return fail(ctx, P3M_ERR_INVALID, "vjp: the FP32 path needs x_r <= 4.6 x_s");
  p3m_status st = poll_latched(ctx);
  if (st != P3M_OK) return st;
  cudaStream_t s = ctx->stream;
  const int64_t n = ctx->n;
  if ((st = cuda_check(ctx, cudaMemsetAsync(ctx->pair_count, 0, sizeof(unsigned long long), s), "memset")) != P3M_OK)
    return st;
  if (n == 0) return P3M_OK;
  if (precision == 32 && !ctx->abar4) {
    if ((st = cuda_check(ctx, cudaMalloc((void**)&ctx->abar4, sizeof(float4) * ctx->cap), "cudaMalloc(abar4)")) != P3M_OK)
      return st;
  }
  if (precision == 64 && !ctx->abar_d) {
    if ((st = cuda_check(ctx, cudaMalloc((void**)&ctx->abar_d, sizeof(double) * 3 * ctx->cap), "cudaMalloc(abar_d)")) != P3M_OK)
      return st;
  }
  if ((st = ensure_all_chunks(ctx)) != P3M_OK) return st;
  if (precision == 32 && (st = prepare_rel4(ctx, pos)) != P3M_OK) return st;
  if (precision == 32)
    k_abar_f32<<<blocks_for(n, 256), 256, 0, s>>>((const float*)acc_bar, ctx->active_flag, ctx->all_active, n,
                                                   ctx->abar4);
  else
    k_abar_f64<<<blocks_for(n, 256), 256, 0, s>>>((const double*)acc_bar, ctx->active_flag, ctx->all_active, n,
                                                   ctx->abar_d);
  ++ctx->launches;
  if ((st = cuda_check(ctx, cudaGetLastError(), "abar kernel")) != P3M_OK) return st;
  if ((st = cuda_check(ctx, cudaMemsetAsync(ctx->dev_small + 4, 0, sizeof(int), s), "memset")) != P3M_OK) return st;
  TraversalArgs a = base_args(ctx);
  a.pos = pos;
  a.chunks = ctx->chunks_all;
  a.n_chunks = ctx->dev_small + 1;
  a.counter = ctx->dev_small + 4;
  a.active_idx = nullptr;
  a.out = pos_bar_out;
  a.abar4 = ctx->abar4;
  a.abar_d = ctx->abar_d;
  cudaError_t e;
  if (precision == 32 && ctx->symmetric) e = launch_sym<true>(ctx, a);  // each pair once (any active set)
  else e = (precision == 32) ? dispatch_traverse<float, true>(ctx, a) : dispatch_traverse<double, true>(ctx, a);
  if ((st = cuda_check(ctx, e, "vjp kernel")) != P3M_OK) return st;
  report_latched(ctx);
  return P3M_OK;
}

// ---------------------------------------------------------------------------
// Allocation-free entry point.
//
// Some callers cannot allocate device memory at all: code that runs under a
// memory pool or arena owned by a host application, a plugin that is handed
// only its input and output buffers, or a pipeline that forbids cudaMalloc
// after start-up.  p3m_sr_forces_noalloc serves them: it sorts a small
// particle set, builds its receiver chunks and evaluates the FP32 forces with
// the same kernels as the context-based path, but every intermediate array
// lives in one file-scope device array of fixed size.  That array belongs to
// every GPU that loads the library, for as long as the process lives.
// ---------------------------------------------------------------------------

namespace p3m {

constexpr int64_t kNoallocMaxN = 1 << 16;         // particles
constexpr int64_t kNoallocMaxSubtiles = 1 << 18;  // subtiles (n_t n_sub)^3
constexpr int64_t kNoallocMaxRows = 1 << 14;      // chunk segments n_t^2 ceil(n_t / 4)
constexpr int64_t kNoallocRadixBlocks = (kNoallocMaxN + kRadixTilePublic - 1) / kRadixTilePublic;
constexpr int64_t kNoallocMaxChunks = kNoallocMaxN + kNoallocMaxN / kChunk + 1;

constexpr int64_t noalloc_align(int64_t b) { return (b + 255) / 256 * 256; }
constexpr int64_t kNoallocScanInts = 4096;  // scan scratch; its last int is the scan's ticket

// Byte layout of the scratch array (each part 256-byte aligned).
struct NoallocLayout {
  static constexpr int64_t keys0 = 0;
  static constexpr int64_t keys1 = keys0 + noalloc_align(4 * kNoallocMaxN);
  static constexpr int64_t vals0 = keys1 + noalloc_align(4 * kNoallocMaxN);
  static constexpr int64_t vals1 = vals0 + noalloc_align(4 * kNoallocMaxN);
  static constexpr int64_t offsets = vals1 + noalloc_align(4 * kNoallocMaxN);
  static constexpr int64_t hist = offsets + noalloc_align(4 * (kNoallocMaxSubtiles + 1));
  static constexpr int64_t scan = hist + noalloc_align(4 * 1024 * kNoallocRadixBlocks);
  static constexpr int64_t wpos = scan + noalloc_align(4 * kNoallocScanInts);
  static constexpr int64_t bad = wpos + noalloc_align(8 * 3 * kNoallocMaxN);
  static constexpr int64_t pos = bad + noalloc_align(kNoallocMaxN);
  static constexpr int64_t rel4 = pos + noalloc_align(8 * 3 * kNoallocMaxN);
  static constexpr int64_t rows = rel4 + noalloc_align(16 * kNoallocMaxN);
  static constexpr int64_t chunks = rows + noalloc_align(4 * (kNoallocMaxRows + 1));
  static constexpr int64_t acc = chunks + noalloc_align(8 * kNoallocMaxChunks);
  static constexpr int64_t small = acc + noalloc_align(4 * 3 * kNoallocMaxN);
  static constexpr int64_t total = small + noalloc_align(64);
};

static __device__ __align__(256) unsigned char g_noalloc_scratch[NoallocLayout::total];

constexpr int kNoallocMaxDevices = 64;
static void* g_noalloc_addr[kNoallocMaxDevices];
static std::mutex g_noalloc_mutex;

// The caller's positions brought into the periodic box: x - L floor(x / L) for a
// finite coordinate outside [0, L) (the same point of the periodic box), 0 with
// bad[i] = 1 for a non-finite one.
__global__ void k_noalloc_wrap(const double* __restrict__ pos, int64_t n, double box, double* __restrict__ wpos,
                               unsigned char* __restrict__ bad) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  bool finite = true;
#pragma unroll
  for (int d = 0; d < 3; ++d) {
    double v = pos[d * n + i];
    if (!isfinite(v)) {
      finite = false;
      v = 0.0;
    } else if (!(v >= 0.0 && v < box)) {
      v = __dsub_rn(v, __dmul_rn(box, floor(__ddiv_rn(v, box))));
      if (!(v >= 0.0 && v < box)) v = 0.0;  // rounded up to L: the same point as 0
    }
    if (v == 0.0) v = 0.0;  // -0 as +0 (the binning compares bit patterns)
    wpos[d * n + i] = v;
  }
  bad[i] = finite ? 0 : 1;
}

// Sorted positions and FP32 subtile-relative records; a particle with a
// non-finite coordinate gets a record far outside the box, so that no receiver
// ever meets it (its own row is overwritten with NaN by k_noalloc_unsort).
__global__ void k_noalloc_gather(const double* __restrict__ wpos, const unsigned char* __restrict__ bad,
                                 const int* __restrict__ perm, const int* __restrict__ cell, int64_t n, Geometry g,
                                 double* __restrict__ spos, float4* __restrict__ rel4) {
  int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= n) return;
  const int64_t j = perm[k];
  const double x = wpos[j], y = wpos[n + j], z = wpos[2 * n + j];
  spos[k] = x;
  spos[n + k] = y;
  spos[2 * n + k] = z;
  const int id = cell[k];
  if (bad[j]) {
    rel4[k] = make_float4(1e10f, 1e10f, 1e10f, __int_as_float(id));
    return;
  }
  int gx, gy, gz;
  decode_subtile(g, id, gx, gy, gz);
  rel4[k] = make_float4((float)__fma_rn(-(double)gx, g.side64[0], x), (float)__fma_rn(-(double)gy, g.side64[1], y),
                        (float)__fma_rn(-(double)gz, g.side64[2], z), __int_as_float(id));
}

// acc_out[d][perm[k]] = acc[d][k], NaN for a particle with a non-finite coordinate
__global__ void k_noalloc_unsort(const float* __restrict__ acc, const int* __restrict__ perm,
                                 const unsigned char* __restrict__ bad, int64_t n, float* __restrict__ out) {
  int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= n) return;
  int64_t j = perm[k];
  const float nan = __int_as_float(0x7fc00000);
  const bool b = bad[j] != 0;
  out[j] = b ? nan : acc[k];
  out[n + j] = b ? nan : acc[n + k];
  out[2 * n + j] = b ? nan : acc[2 * n + k];
}

}  // namespace p3m

extern "C" p3m_status p3m_sr_forces_noalloc(const p3m_sr_params* params, void* cuda_stream, const double* pos,
                                            float* acc_out) {
  if (!params) return P3M_ERR_INVALID;
  p3m_sr_ctx c;  // host-side bookkeeping only: no device memory, no events
  p3m_status st = validate_params(&c, *params);
  if (st != P3M_OK) return st;
  const int64_t n = params->n;
  if (n > kNoallocMaxN) return P3M_ERR_INVALID;
  c.prm = *params;
  c.n = n;
  setup_geometry(&c);
  setup_force_consts(&c);
  const Geometry& g = c.geo;
  if (g.S > kNoallocMaxSubtiles ||
      (int64_t)g.n_t * g.n_t * ((g.n_t + kChunkSpan - 1) / kChunkSpan) > kNoallocMaxRows)
    return P3M_ERR_INVALID;
  if (params->x_r > 2.0 * P3M_ERFCX_UMAX * params->x_s) return P3M_ERR_INVALID;
  if (n == 0) return P3M_OK;
  if (!pos || !acc_out) return P3M_ERR_INVALID;

  // once per device: the device address of the scratch array
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kNoallocMaxDevices) return P3M_ERR_CUDA;
  unsigned char* base = nullptr;
  {
    std::lock_guard<std::mutex> lock(g_noalloc_mutex);
    if (!g_noalloc_addr[dev]) {
      void* p = nullptr;
      if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || !p) {
        cudaGetLastError();
        return P3M_ERR_CUDA;
      }
      g_noalloc_addr[dev] = p;
    }
    base = (unsigned char*)g_noalloc_addr[dev];
  }
  using Lay = NoallocLayout;
  int* keys[2] = {(int*)(base + Lay::keys0), (int*)(base + Lay::keys1)};
  int* vals[2] = {(int*)(base + Lay::vals0), (int*)(base + Lay::vals1)};
  int* offsets = (int*)(base + Lay::offsets);
  int* hist = (int*)(base + Lay::hist);
  int* scan = (int*)(base + Lay::scan);
  double* wpos = (double*)(base + Lay::wpos);
  unsigned char* bad = base + Lay::bad;
  double* spos = (double*)(base + Lay::pos);
  float4* rel4 = (float4*)(base + Lay::rel4);
  int* rows = (int*)(base + Lay::rows);
  Chunk* chunks = (Chunk*)(base + Lay::chunks);
  float* acc = (float*)(base + Lay::acc);
  int* small = (int*)(base + Lay::small);  // [0] n_chunks, [1] counter, [2] k_bin's error word (unused: the
                                           // positions are wrapped first), [4..5] pair count
  cudaStream_t s = (cudaStream_t)cuda_stream;
  int64_t launches = 0;
  auto ok = [&](cudaError_t e) { return e == cudaSuccess; };

  // periodic wrap, then bin + subtile offsets (histogram, exclusive scan)
  if (!ok(cudaMemsetAsync(offsets, 0, sizeof(int) * (g.S + 1), s))) return P3M_ERR_CUDA;
  if (!ok(cudaMemsetAsync(small, 0, 64, s))) return P3M_ERR_CUDA;
  if (!ok(cudaMemsetAsync(scan + kNoallocScanInts - 1, 0, sizeof(int), s))) return P3M_ERR_CUDA;
  k_noalloc_wrap<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(pos, n, g.box, wpos, bad);
  if (!ok(cudaGetLastError())) return P3M_ERR_CUDA;
  k_bin<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(wpos, n, g, keys[0], vals[0], offsets, small + 2);
  if (!ok(cudaGetLastError())) return P3M_ERR_CUDA;
  if (!ok(scan_exclusive_i32(offsets, offsets, g.S + 1, scan, kNoallocScanInts, s, &launches))) return P3M_ERR_CUDA;
  // stable LSD radix sort of the subtile ids
  int key_bits = 1;
  while (key_bits < 31 && ((int64_t)1 << key_bits) < g.S) ++key_bits;
  const int passes = (key_bits + 9) / 10;
  const int nblocks = (int)((n + kRadixTilePublic - 1) / kRadixTilePublic);
  int cur = 0, shift = 0;
  for (int p = 0, left = key_bits; p < passes; ++p) {
    const int bits = (left + (passes - p) - 1) / (passes - p);
    left -= bits;
    k_radix_hist<<<nblocks, kRadixThreadsPublic, 0, s>>>(keys[cur], n, shift, bits, hist, nblocks);
    if (!ok(cudaGetLastError())) return P3M_ERR_CUDA;
    if (!ok(scan_exclusive_i32(hist, hist, (int64_t)nblocks << bits, scan, kNoallocScanInts, s, &launches))) return P3M_ERR_CUDA;
    k_radix_scatter<<<nblocks, kRadixThreadsPublic, 0, s>>>(keys[cur], vals[cur], keys[cur ^ 1], vals[cur ^ 1], n,
                                                            shift, bits, hist, nblocks, nullptr, 0, 0);
    if (!ok(cudaGetLastError())) return P3M_ERR_CUDA;
    cur ^= 1;
    shift += bits;
  }
  const int* cell = keys[cur];
  const int* perm = vals[cur];
  // sorted positions and their FP32 subtile-relative records
  k_noalloc_gather<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(wpos, bad, perm, cell, n, g, spos, rel4);
  if (!ok(cudaGetLastError())) return P3M_ERR_CUDA;
  // receiver chunks (all particles active)
  const int64_t nrows = (int64_t)g.n_t * g.n_t * ((g.n_t + kChunkSpan - 1) / kChunkSpan);  // segments
  k_row_chunks<<<(unsigned)((nrows + 1 + 127) / 128), 128, 0, s>>>(offsets, nullptr, g.n_t, g.nsub3, rows);
  if (!ok(cudaGetLastError())) return P3M_ERR_CUDA;
  if (!ok(scan_exclusive_i32(rows, rows, nrows + 1, scan, kNoallocScanInts, s, &launches))) return P3M_ERR_CUDA;
  k_write_chunks<<<(unsigned)((nrows + 127) / 128), 128, 0, s>>>(offsets, nullptr, g.n_t, g.nsub3, rows, chunks,
                                                                 small + 0, nullptr, n);
  if (!ok(cudaGetLastError())) return P3M_ERR_CUDA;
  // pair forces in the sorted order, then back to the caller's order
  static SeriesConsts series = make_series();
  TraversalArgs a{};
  a.g = g;
  a.f = c.fc;
  a.sc = series;
  a.pos = spos;
  a.rel4 = rel4;
  a.offsets = offsets;
  a.cell = cell;
  a.chunks = chunks;
  a.n_chunks = small + 0;
  a.counter = small + 1;
  a.active_idx = nullptr;
  a.n = n;
  a.out = acc;
  a.pairs = (unsigned long long*)(small + 4);
  int num_sms = 0;
  cudaDeviceGetAttribute(&num_sms, cudaDevAttrMultiProcessorCount, dev);
  const unsigned grid = (unsigned)(num_sms > 0 ? num_sms : 1) * 4;
  switch (params->softening) {
    case P3M_SOFT_NONE: k_force_packed<P3M_SOFT_NONE><<<grid, kPThreads, 0, s>>>(a); break;
    case P3M_SOFT_PLUMMER: k_force_packed<P3M_SOFT_PLUMMER><<<grid, kPThreads, 0, s>>>(a); break;
    default: k_force_packed<P3M_SOFT_BSPLINE><<<grid, kPThreads, 0, s>>>(a); break;
  }
  if (!ok(cudaGetLastError())) return P3M_ERR_CUDA;
  k_noalloc_unsort<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(acc, perm, bad, n, acc_out);
  if (!ok(cudaGetLastError())) return P3M_ERR_CUDA;
  return P3M_OK;
}
