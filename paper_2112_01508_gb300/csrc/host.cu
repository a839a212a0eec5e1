// Context creation, parameter validation, error latch and the shared int32 scan.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <new>

#include "ctx.cuh"
#include "erfcx_fit.h"

namespace p3m {

p3m_status fail(p3m_sr_ctx* ctx, p3m_status st, const std::string& msg) {
  if (ctx) ctx->last_error = msg;
  return st;
}

p3m_status cuda_check(p3m_sr_ctx* ctx, cudaError_t e, const char* what) {
  if (e == cudaSuccess) return P3M_OK;
  std::string m = std::string(what) + ": " + cudaGetErrorString(e);
  if (e == cudaErrorMemoryAllocation) return fail(ctx, P3M_ERR_OOM, m);
  return fail(ctx, P3M_ERR_CUDA, m);
}

static p3m_status status_from_bits(p3m_sr_ctx* ctx, int bits) {
  if (bits & kErrPosition)
    return fail(ctx, P3M_ERR_NONFINITE, "a position was non-finite or outside [0, L) when binned");
  if (bits & kErrNonfiniteAcc)
    return fail(ctx, P3M_ERR_NONFINITE, "a non-finite acceleration was met by the rung assignment");
  if (bits & kErrDrift)
    return fail(ctx, P3M_ERR_STATE, "positions drifted too far since the last sort (x_r + 2 drift >= L/2): sort again");
  if (bits & kErrRungState)
    return fail(ctx, P3M_ERR_STATE, "a rung kick met a rung outside [0, n_rung) or a kick state outside {0, 1, 2}");
  return P3M_OK;
}

p3m_status poll_latched(p3m_sr_ctx* ctx) {
  if (ctx->err_event_pending && cudaEventQuery(ctx->err_event) == cudaSuccess) {
    ctx->err_event_pending = false;
  }
  if (!ctx->err_event_pending && *ctx->err_host) return status_from_bits(ctx, *ctx->err_host);
  return P3M_OK;
}

void report_latched(p3m_sr_ctx* ctx) {
  if (ctx->err_event_pending) return;  // the previous report is still in flight
  cudaMemcpyAsync(ctx->err_host, ctx->err_dev, sizeof(int), cudaMemcpyDeviceToHost, ctx->stream);
  cudaEventRecord(ctx->err_event, ctx->stream);
  ctx->err_event_pending = true;
}

// ---------------------------------------------------------------------------
// Exclusive scan of int32 (tiles of 4096 per block, recursive over tile sums).
// ---------------------------------------------------------------------------

constexpr int kScanThreads = 256;
constexpr int kScanItems = 16;
constexpr int kScanTile = kScanThreads * kScanItems;

__device__ __forceinline__ int smem_pad(int i) { return i + (i >> 5); }

__global__ void k_scan_reduce(const int* __restrict__ in, int64_t n, int* __restrict__ sums) {
  __shared__ int warp_sums[kScanThreads / kWarp];
  int64_t base = (int64_t)blockIdx.x * kScanTile;
  int s = 0;
  for (int k = 0; k < kScanItems; ++k) {
    int64_t i = base + (int64_t)k * kScanThreads + threadIdx.x;
    if (i < n) s += in[i];
  }
  for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
  if ((threadIdx.x & 31) == 0) warp_sums[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x < 32) {
    int v = threadIdx.x < kScanThreads / kWarp ? warp_sums[threadIdx.x] : 0;
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    if (threadIdx.x == 0) sums[blockIdx.x] = v;
  }
}

__global__ void k_scan_tile(const int* in, int* out, int64_t n, const int* __restrict__ offs) {
  __shared__ int tile[kScanTile + kScanTile / 32];
  __shared__ int warp_tot[kScanThreads / kWarp];
  int64_t base = (int64_t)blockIdx.x * kScanTile;
  for (int k = 0; k < kScanItems; ++k) {
    int li = k * kScanThreads + threadIdx.x;
    int64_t i = base + li;
    tile[smem_pad(li)] = i < n ? in[i] : 0;
  }
  __syncthreads();
  int vals[kScanItems];
  int tot = 0;
#pragma unroll
  for (int k = 0; k < kScanItems; ++k) {
    vals[k] = tile[smem_pad(threadIdx.x * kScanItems + k)];
    tot += vals[k];
  }
  // exclusive scan of per-thread totals across the block
  int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  int inc = tot;
  for (int o = 1; o < 32; o <<= 1) {
    int t = __shfl_up_sync(0xffffffffu, inc, o);
    if (lane >= o) inc += t;
  }
  if (lane == 31) warp_tot[warp] = inc;
  __syncthreads();
  int wpre = 0;
  for (int w = 0; w < warp; ++w) wpre += warp_tot[w];
  int run = wpre + inc - tot + (offs ? offs[blockIdx.x] : 0);
#pragma unroll
  for (int k = 0; k < kScanItems; ++k) {
    tile[smem_pad(threadIdx.x * kScanItems + k)] = run;
    run += vals[k];
  }
  __syncthreads();
  for (int k = 0; k < kScanItems; ++k) {
    int li = k * kScanThreads + threadIdx.x;
    int64_t i = base + li;
    if (i < n) out[i] = tile[smem_pad(li)];
  }
}

// Exclusive scan of the nb <= kScanTile values of v in place, by one block.
__device__ __forceinline__ void block_scan_small(volatile int* v, int nb) {
  __shared__ int warp_tot[kScanThreads / kWarp];
  const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
  int vals[kScanItems];
  int tot = 0;
#pragma unroll
  for (int k = 0; k < kScanItems; ++k) {
    const int i = t * kScanItems + k;
    vals[k] = i < nb ? v[i] : 0;
    tot += vals[k];
  }
  int inc = tot;
  for (int o = 1; o < 32; o <<= 1) {
    const int u = __shfl_up_sync(0xffffffffu, inc, o);
    if (lane >= o) inc += u;
  }
  if (lane == 31) warp_tot[warp] = inc;
  __syncthreads();
  int run = inc - tot;
  for (int w = 0; w < warp; ++w) run += warp_tot[w];
#pragma unroll
  for (int k = 0; k < kScanItems; ++k) {
    const int i = t * kScanItems + k;
    if (i < nb) v[i] = run;
    run += vals[k];
  }
}

// Tile sums, and in the same launch their exclusive scan by the block that finishes
// last (an atomic ticket; no block waits for another).  *ticket is 0 on entry and
// is reset to 0 by the last block.
__global__ void k_scan_reduce_last(const int* __restrict__ in, int64_t n, int* sums, int* ticket) {
  __shared__ int warp_sums[kScanThreads / kWarp];
  __shared__ bool last;
  int64_t base = (int64_t)blockIdx.x * kScanTile;
  int s = 0;
  for (int k = 0; k < kScanItems; ++k) {
    int64_t i = base + (int64_t)k * kScanThreads + threadIdx.x;
    if (i < n) s += in[i];
  }
  for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
  if ((threadIdx.x & 31) == 0) warp_sums[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    int v = 0;
    for (int w = 0; w < kScanThreads / kWarp; ++w) v += warp_sums[w];
    sums[blockIdx.x] = v;
    __threadfence();
    last = atomicAdd(ticket, 1) == (int)gridDim.x - 1;
  }
  __syncthreads();
  if (last) {
    __threadfence();
    block_scan_small(sums, (int)gridDim.x);
    if (threadIdx.x == 0) *ticket = 0;
  }
}

int64_t scan_scratch_ints(int64_t n) {
  int64_t total = 0;
  int64_t m = n;
  while (m > kScanTile) {
    m = (m + kScanTile - 1) / kScanTile;
    total += m;
  }
  return total + 2;  // + the ticket of k_scan_reduce_last
}

// The ticket lives in the last int of the scratch that scan_scratch_ints(n) sized.
static cudaError_t scan_rec(const int* in, int* out, int64_t n, int* scratch, int* ticket, cudaStream_t s,
                            int64_t* launches) {
  if (n <= 0) return cudaSuccess;
  int64_t nb = (n + kScanTile - 1) / kScanTile;
  if (nb == 1) {
    k_scan_tile<<<1, kScanThreads, 0, s>>>(in, out, n, nullptr);
    ++*launches;
    return cudaGetLastError();
  }
  int* sums = scratch;
  if (nb <= kScanTile) {  // two launches: tile sums scanned by the last block, then the tiles
    k_scan_reduce_last<<<(unsigned)nb, kScanThreads, 0, s>>>(in, n, sums, ticket);
    ++*launches;
  } else {
    k_scan_reduce<<<(unsigned)nb, kScanThreads, 0, s>>>(in, n, sums);
    ++*launches;
    cudaError_t e = scan_rec(sums, sums, nb, scratch + nb, ticket, s, launches);
    if (e != cudaSuccess) return e;
  }
  k_scan_tile<<<(unsigned)nb, kScanThreads, 0, s>>>(in, out, n, sums);
  ++*launches;
  return cudaGetLastError();
}

cudaError_t scan_exclusive_i32(const int* in, int* out, int64_t n, int* scratch, int64_t scratch_ints, cudaStream_t s,
                               int64_t* launches) {
  return scan_rec(in, out, n, scratch, scratch + scratch_ints - 1, s, launches);
}

}  // namespace p3m

using namespace p3m;

// ---------------------------------------------------------------------------
// Parameter validation and constants.
// ---------------------------------------------------------------------------

p3m_status validate_params(p3m_sr_ctx* ctx, const p3m_sr_params& p) {
  if (p.n < 0 || p.n > 0x7fffffffLL - 64) return fail(ctx, P3M_ERR_INVALID, "n must be in [0, 2^31 - 64)");
  if (!(p.box > 0.0) || !std::isfinite(p.box)) return fail(ctx, P3M_ERR_INVALID, "box must be positive");
  if (!(p.x_s > 0.0) || !std::isfinite(p.x_s)) return fail(ctx, P3M_ERR_INVALID, "x_s must be positive");
  if (!(p.x_r > 0.0) || !std::isfinite(p.x_r)) return fail(ctx, P3M_ERR_INVALID, "x_r must be positive");
  if (!std::isfinite(p.G_m)) return fail(ctx, P3M_ERR_INVALID, "G_m must be finite");
  if (p.softening < 0 || p.softening > 2) return fail(ctx, P3M_ERR_INVALID, "softening must be 0, 1 or 2");
  if (p.softening != 0 && !(p.eps > 0.0)) return fail(ctx, P3M_ERR_INVALID, "eps must be positive when softened");
  for (int d = 0; d < 3; ++d)
    if (p.n_sub[d] < 1 || p.n_sub[d] > 16) return fail(ctx, P3M_ERR_INVALID, "n_sub must be in 1..16");
  if (p.n_rung < 1 || p.n_rung > 8) return fail(ctx, P3M_ERR_INVALID, "n_rung must be in 1..8");
  double nt = std::floor(p.box / p.x_r);
  if (nt < 4.0) return fail(ctx, P3M_ERR_TOO_FEW_TILES, "need at least 4 tiles per dimension (x_r <= L/4)");
  double r_sw = (p.softening == 0) ? 0.0 : 2.8 * p.eps;
  if (r_sw / (2.0 * p.x_s) > 1.0)
    return fail(ctx, P3M_ERR_INVALID, "softening length too large for the split scale (2.8 eps > 2 x_s)");
  if (r_sw > p.x_r) return fail(ctx, P3M_ERR_INVALID, "softening length exceeds the cutoff");
  return P3M_OK;
}

// ceil(2^64 / d) for d >= 2 (0 for d = 1, which quot_magic passes through).
static unsigned long long magic_u64(int64_t d) {
  return d <= 1 ? 0ULL : ~0ULL / (unsigned long long)d + 1ULL;
}

void setup_geometry(p3m_sr_ctx* ctx) {
  const p3m_sr_params& p = ctx->prm;
  Geometry& g = ctx->geo;
  g.n_t = (int)std::floor(p.box / p.x_r);
  g.nsub3 = 1;
  g.S = 1;
  g.box = p.box;
  for (int d = 0; d < 3; ++d) {
    g.ns[d] = p.n_sub[d];
    g.M[d] = g.n_t * g.ns[d];
    g.nsub3 *= g.ns[d];
    g.S *= g.M[d];
    g.scale64[d] = (double)g.M[d] / p.box;
    g.side64[d] = p.box / (double)g.M[d];
    g.side32[d] = (float)g.side64[d];
    g.R[d] = (int)std::ceil(p.x_r / g.side64[d] * (1.0 + 1e-12));
    g.inv_ns[d] = 1.0f / (float)g.ns[d];
  }
  ctx->n_tiles = (int64_t)g.n_t * g.n_t * g.n_t;
  g.mg_nsub3 = magic_u64(g.nsub3);
  g.mg_nt2 = magic_u64((int64_t)g.n_t * g.n_t);
  g.mg_nt = magic_u64(g.n_t);
  g.mg_s12 = magic_u64((int64_t)g.ns[1] * g.ns[2]);
  g.mg_s2 = magic_u64(g.ns[2]);
}

static int64_t origin_count(const Geometry& g) { return (int64_t)g.M[0] + g.M[1] + g.M[2]; }

// Fill the subtile-origin table of the current geometry (stream-ordered: work
// queued before still reads the previous values).
static p3m_status fill_origins(p3m_sr_ctx* ctx) {
  ctx->geo.org = ctx->org;
  const int64_t m = origin_count(ctx->geo);
  k_fill_origins<<<(unsigned)((m + 255) / 256), 256, 0, ctx->stream>>>(ctx->geo, ctx->org);
  ++ctx->launches;
  return cuda_check(ctx, cudaGetLastError(), "origin table kernel");
}

void setup_force_consts(p3m_sr_ctx* ctx) {
  const p3m_sr_params& p = ctx->prm;
  ForceConsts& f = ctx->fc;
  const double pi = 3.14159265358979323846;
  const double log2e = 1.44269504088896340736;
  f.softening = p.softening;
  f.x_s = p.x_s;
  f.x_r = p.x_r;
  f.G_m = p.G_m;
  f.eps = p.eps;
  f.eps_b = 2.8 * p.eps;
  f.r_sw = (p.softening == 0) ? 0.0 : 2.8 * p.eps;
  f.xr2_f = (float)(p.x_r * p.x_r);
  f.rsw2_f = (p.softening == 0) ? 1e-37f : (float)(f.r_sw * f.r_sw);
  f.ce_f = (float)(-log2e / (4.0 * p.x_s * p.x_s));
  f.kc_f = (float)(P3M_ERFCX_K / (2.0 * p.x_s));
  f.k2_f = (float)(1.0 / (std::sqrt(pi) * p.x_s));
  f.k3_f = (float)(1.0 / (2.0 * std::sqrt(pi) * p.x_s * p.x_s * p.x_s));
  const double c[6] = {P3M_ERFCX_C0, P3M_ERFCX_C1, P3M_ERFCX_C2, P3M_ERFCX_C3, P3M_ERFCX_C4, P3M_ERFCX_C5};
  for (int k = 0; k < 6; ++k) f.c_f[k] = (float)c[k];
  f.inv2xs_f = (float)(1.0 / (2.0 * p.x_s));
  f.hscale_f = (float)(1.0 / (8.0 * p.x_s * p.x_s * p.x_s));
  f.epsb_f = (float)f.eps_b;
  f.inv_epsb_f = f.eps_b > 0 ? (float)(1.0 / f.eps_b) : 0.f;
  f.bnorm_f = f.eps_b > 0 ? (float)(32.0 / (f.eps_b * f.eps_b * f.eps_b)) : 0.f;
  f.eps2_f = (float)(p.eps * p.eps);
  f.margin2_f = (float)(p.x_r * p.x_r * (1.0 + 1e-4));
  f.xr2_d = p.x_r * p.x_r;
  f.rsw2_d = (p.softening == 0) ? 0.0 : f.r_sw * f.r_sw;
}

// radix passes over ceil(log2(S)) key bits, at most 10 bits each
static void setup_radix(p3m_sr_ctx* ctx) {
  int key_bits = 1;
  while (key_bits < 31 && ((int64_t)1 << key_bits) < ctx->geo.S) ++key_bits;
  ctx->radix_passes = (key_bits + 9) / 10;
  for (int k = 0, left = key_bits; k < ctx->radix_passes; ++k) {
    int b = (left + (ctx->radix_passes - k) - 1) / (ctx->radix_passes - k);
    ctx->radix_bits[k] = b;
    left -= b;
  }
}

// longest array the exclusive scan is applied to
static int64_t scan_length(const p3m_sr_ctx* ctx) {
  return std::max<int64_t>(std::max<int64_t>(ctx->geo.S + 1, ctx->cap + 1),
                           std::max<int64_t>(ctx->hist_ints, ctx->n_tiles + 1));
}

template <class T>
static p3m_status alloc(p3m_sr_ctx* ctx, T** ptr, int64_t count, const char* what) {
  size_t bytes = (size_t)(count > 0 ? count : 1) * sizeof(T);
  cudaError_t e = cudaMalloc((void**)ptr, bytes);
  if (e != cudaSuccess) {
    *ptr = nullptr;
    cudaGetLastError();
    return fail(ctx, e == cudaErrorMemoryAllocation ? P3M_ERR_OOM : P3M_ERR_CUDA,
                std::string("cudaMalloc(") + what + ") failed: " + cudaGetErrorString(e));
  }
  return P3M_OK;
}

extern "C" p3m_status p3m_sr_create(const p3m_sr_params* params, void* cuda_stream, p3m_sr_ctx** out) {
  if (!out) return P3M_ERR_INVALID;
  *out = nullptr;
  if (!params) return P3M_ERR_INVALID;
  p3m_sr_ctx* ctx = new (std::nothrow) p3m_sr_ctx();
  if (!ctx) return P3M_ERR_OOM;
  p3m_status st = validate_params(ctx, *params);
  if (st != P3M_OK) {
    delete ctx;
    return st;
  }
  ctx->prm = *params;
  ctx->n = params->n;
  ctx->cap = params->n;
  ctx->stream = (cudaStream_t)cuda_stream;
  setup_geometry(ctx);
  setup_force_consts(ctx);
  if (ctx->geo.S > 0x7fffffffLL - 2) {
    delete ctx;
    return P3M_ERR_INVALID;
  }
  cudaGetDevice(&ctx->device);
  cudaDeviceGetAttribute(&ctx->num_sms, cudaDevAttrMultiProcessorCount, ctx->device);

  const int64_t n = ctx->n;
  const int64_t S = ctx->geo.S;
  setup_radix(ctx);
  int64_t radix_blocks = (n + kRadixTilePublic - 1) / kRadixTilePublic;
  ctx->hist_ints = 1024 * (radix_blocks > 0 ? radix_blocks : 1);
  ctx->scan_scratch_ints = scan_scratch_ints(scan_length(ctx));
  ctx->offsets_cap = S + 1;
  ctx->max_chunks = std::min<int64_t>(n, ctx->n_tiles) + (n + kChunk - 1) / kChunk + 1;

#define P3M_ALLOC(ptr, count) \
  if ((st = alloc(ctx, &(ptr), (count), #ptr)) != P3M_OK) goto fail_alloc;
  P3M_ALLOC(ctx->keys[0], n);
  P3M_ALLOC(ctx->keys[1], n);
  P3M_ALLOC(ctx->vals[0], n);
  P3M_ALLOC(ctx->vals[1], n);
  P3M_ALLOC(ctx->offsets, S + 1);
  P3M_ALLOC(ctx->hist, 2 * ctx->hist_ints);  // this radix pass's digit counts and the next pass's
  P3M_ALLOC(ctx->scan_scratch, ctx->scan_scratch_ints);
  {
    char* gt = nullptr;
    P3M_ALLOC(gt, 32 * n);
    ctx->gather_tmp = gt;
  }
  P3M_ALLOC(ctx->active_flag, n);
  P3M_ALLOC(ctx->act_scan, n + 1);
  P3M_ALLOC(ctx->active_idx, n);
  P3M_ALLOC(ctx->tile_chunks, ctx->n_tiles + 1);
  P3M_ALLOC(ctx->part_acc, std::min<int64_t>(kPartItems, ctx->max_chunks * kMaxParts) * kChunk);
  P3M_ALLOC(ctx->chunks, ctx->max_chunks);
  P3M_ALLOC(ctx->chunks_all, ctx->max_chunks);
  P3M_ALLOC(ctx->dev_small, 16);
  P3M_ALLOC(ctx->pair_count, 2);
  P3M_ALLOC(ctx->rel4, n);
  P3M_ALLOC(ctx->org, origin_count(ctx->geo));
  ctx->org_cap = origin_count(ctx->geo);
  P3M_ALLOC(ctx->err_dev, 1);
  P3M_ALLOC(ctx->drift_slots, kMaxDrifts);
#undef P3M_ALLOC
  if (cudaMallocHost((void**)&ctx->err_host, sizeof(int)) != cudaSuccess) {
    st = fail(ctx, P3M_ERR_OOM, "cudaMallocHost failed");
    goto fail_alloc;
  }
  *ctx->err_host = 0;
  if (cudaEventCreateWithFlags(&ctx->err_event, cudaEventDisableTiming) != cudaSuccess) {
    st = fail(ctx, P3M_ERR_CUDA, "cudaEventCreate failed");
    goto fail_alloc;
  }
  for (int k = 0; k < 4; ++k)
    if (cudaEventCreate(&ctx->kt_ev[k]) != cudaSuccess) {
      st = fail(ctx, P3M_ERR_CUDA, "cudaEventCreate failed");
      goto fail_alloc;
    }
  if ((st = cuda_check(ctx, cudaMemsetAsync(ctx->err_dev, 0, sizeof(int), ctx->stream), "memset")) != P3M_OK)
    goto fail_alloc;
  if ((st = cuda_check(ctx, cudaMemsetAsync(ctx->scan_scratch, 0, sizeof(int) * ctx->scan_scratch_ints, ctx->stream),
                       "memset")) != P3M_OK)
    goto fail_alloc;
  if ((st = cuda_check(ctx, cudaMemsetAsync(ctx->drift_slots, 0, sizeof(float) * kMaxDrifts, ctx->stream),
                       "memset")) != P3M_OK)
    goto fail_alloc;
  if ((st = cuda_check(ctx, cudaMemsetAsync(ctx->dev_small, 0, 16 * sizeof(int), ctx->stream), "memset")) != P3M_OK)
    goto fail_alloc;
  if ((st = cuda_check(ctx, cudaMemsetAsync(ctx->pair_count, 0, 2 * sizeof(unsigned long long), ctx->stream),
                       "memset")) != P3M_OK)
    goto fail_alloc;
  if ((st = fill_origins(ctx)) != P3M_OK) goto fail_alloc;
  *out = ctx;
  return P3M_OK;
fail_alloc:
  p3m_sr_destroy(ctx);
  return st;
}

extern "C" p3m_status p3m_sr_set_count(p3m_sr_ctx* ctx, int64_t n) {
  if (!ctx) return P3M_ERR_INVALID;
  if (n < 0 || n > ctx->cap)
    return fail(ctx, P3M_ERR_INVALID, "set_count: n must be in [0, the count given to p3m_sr_create]");
  ctx->n = n;
  ctx->prm.n = n;
  ctx->sorted = false;
  ctx->sorted_pos = nullptr;
  ctx->pairs_built = false;
  ctx->all_chunks_built = false;
  ctx->perm = nullptr;
  return P3M_OK;
}

extern "C" p3m_status p3m_sr_set_symmetric(p3m_sr_ctx* ctx, int enable) {
  if (!ctx) return P3M_ERR_INVALID;
  ctx->symmetric = enable != 0;
  return P3M_OK;
}

extern "C" p3m_status p3m_sr_set_subtiles(p3m_sr_ctx* ctx, const int* n_sub) {
  if (!ctx) return P3M_ERR_INVALID;
  if (!n_sub) return fail(ctx, P3M_ERR_INVALID, "set_subtiles: null n_sub");
  p3m_sr_params p = ctx->prm;
  for (int d = 0; d < 3; ++d) p.n_sub[d] = n_sub[d];
  p3m_status st = validate_params(ctx, p);
  if (st != P3M_OK) return st;
  int64_t S = (int64_t)std::floor(p.box / p.x_r);
  S = S * p.n_sub[0] * S * p.n_sub[1] * S * p.n_sub[2];
  if (S > 0x7fffffffLL - 2) return fail(ctx, P3M_ERR_INVALID, "set_subtiles: too many subtiles");
  if ((st = poll_latched(ctx)) != P3M_OK) return st;
  const p3m_sr_params old_prm = ctx->prm;
  const Geometry old_geo = ctx->geo;
  ctx->prm = p;
  setup_geometry(ctx);
  // per-subtile offsets and the scan scratch grow with S; cudaFree waits for queued work
  int64_t scan_ints = scan_scratch_ints(scan_length(ctx));
  int* new_offsets = nullptr;
  int* new_scan = nullptr;
  double* new_org = nullptr;
  const int64_t n_org = origin_count(ctx->geo);
  if (S + 1 > ctx->offsets_cap && (st = alloc(ctx, &new_offsets, S + 1, "offsets")) != P3M_OK) goto restore;
  if (scan_ints > ctx->scan_scratch_ints && (st = alloc(ctx, &new_scan, scan_ints, "scan_scratch")) != P3M_OK) {
    cudaFree(new_offsets);
    goto restore;
  }
  if (n_org > ctx->org_cap && (st = alloc(ctx, &new_org, n_org, "org")) != P3M_OK) {
    cudaFree(new_offsets);
    cudaFree(new_scan);
    goto restore;
  }
  if (new_org) {
    cudaFree(ctx->org);
    ctx->org = new_org;
    ctx->org_cap = n_org;
  }
  if (new_offsets) {
    cudaFree(ctx->offsets);
    ctx->offsets = new_offsets;
    ctx->offsets_cap = S + 1;
  }
  if (new_scan) {
    cudaFree(ctx->scan_scratch);
    ctx->scan_scratch = new_scan;
    ctx->scan_scratch_ints = scan_ints;
    if ((st = cuda_check(ctx, cudaMemsetAsync(new_scan, 0, sizeof(int) * scan_ints, ctx->stream), "memset")) != P3M_OK)
      return st;
  }
  if ((st = fill_origins(ctx)) != P3M_OK) return st;
  setup_radix(ctx);
  ctx->sorted = false;
  ctx->sorted_pos = nullptr;
  ctx->pairs_built = false;
  ctx->all_chunks_built = false;
  return P3M_OK;
restore:
  ctx->prm = old_prm;
  ctx->geo = old_geo;
  return st;
}

extern "C" void p3m_sr_destroy(p3m_sr_ctx* ctx) {
  if (!ctx) return;
  if (ctx->stream || true) cudaStreamSynchronize(ctx->stream);
  void* ptrs[] = {ctx->keys[0], ctx->keys[1], ctx->vals[0], ctx->vals[1], ctx->offsets, ctx->hist,
                  ctx->scan_scratch, ctx->gather_tmp, ctx->active_flag, ctx->act_scan, ctx->active_idx,
                  ctx->tile_chunks, ctx->part_acc,
                  ctx->chunks, ctx->chunks_all, ctx->dev_small, ctx->pair_count,
                  ctx->rel4, ctx->org, ctx->abar4, ctx->abar_d, ctx->table, ctx->err_dev, ctx->drift_slots};
  for (void* p : ptrs)
    if (p) cudaFree(p);
  if (ctx->err_host) cudaFreeHost(ctx->err_host);
  if (ctx->err_event) cudaEventDestroy(ctx->err_event);
  for (int k = 0; k < 4; ++k)
    if (ctx->kt_ev[k]) cudaEventDestroy(ctx->kt_ev[k]);
  delete ctx;
}

extern "C" const char* p3m_sr_last_error(const p3m_sr_ctx* ctx) {
  if (!ctx) return "null context";
  return ctx->last_error.c_str();
}

extern "C" p3m_status p3m_sr_sync(p3m_sr_ctx* ctx) {
  if (!ctx) return P3M_ERR_INVALID;
  p3m_status st = cuda_check(ctx, cudaStreamSynchronize(ctx->stream), "cudaStreamSynchronize");
  if (st != P3M_OK) return st;
  int bits = 0;
  st = cuda_check(ctx, cudaMemcpy(&bits, ctx->err_dev, sizeof(int), cudaMemcpyDeviceToHost), "cudaMemcpy");
  if (st != P3M_OK) return st;
  ctx->err_event_pending = false;
  *ctx->err_host = bits;
  return status_from_bits(ctx, bits);
}

extern "C" p3m_status p3m_sr_stats(p3m_sr_ctx* ctx, p3m_sr_stats_t* out) {
  if (!ctx || !out) return P3M_ERR_INVALID;
  p3m_status st = p3m_sr_sync(ctx);
  std::memset(out, 0, sizeof(*out));
  out->n_tile = ctx->geo.n_t;
  for (int d = 0; d < 3; ++d) out->n_sub[d] = ctx->geo.ns[d];
  out->n_subtiles = ctx->geo.S;
  int small[3] = {0, 0, 0};
  unsigned long long pc = 0;
  cudaMemcpy(small, ctx->dev_small, sizeof(small), cudaMemcpyDeviceToHost);
  cudaMemcpy(&pc, ctx->pair_count, sizeof(pc), cudaMemcpyDeviceToHost);
  out->n_chunks = ctx->pairs_built ? small[0] : 0;
  out->n_active = ctx->pairs_built ? small[2] : 0;
  out->pairs_last = (int64_t)pc;
  for (int k = 0; k < 2; ++k) {
    if (ctx->kt_pending[k]) {
      float ms = 0.f;
      if (cudaEventElapsedTime(&ms, ctx->kt_ev[2 * k], ctx->kt_ev[2 * k + 1]) == cudaSuccess) ctx->kt_ms[k] = ms;
      ctx->kt_pending[k] = false;
    }
  }
  out->force_kernel_ms = ctx->kt_ms[0];
  out->vjp_kernel_ms = ctx->kt_ms[1];
  out->kernel_launches = ctx->launches;
  return st;
}
