// Sorting particles into tiles and subtiles (Section 2.1.3, "Tiles": an O(N)
// sort into the box tiling, with the particles reordered in memory in the
// tile -> subtile -> particle walk order of the short-range computation).
//
// GPU design: one pass bins every particle (subtile id from one correctly
// rounded multiply per dimension) and builds the subtile histogram; an
// exclusive scan turns it into the subtile offsets.  The permutation itself
// comes from a stable LSD radix sort of the subtile ids (8-bit digits at
// most, warp-level ranking with match.any so that equal ids keep their input
// order), after which positions and any carried arrays are gathered.
#include <string>

#include "ctx.cuh"

namespace p3m {

constexpr int kRadixThreads = 256;
constexpr int kRadixWarps = kRadixThreads / kWarp;
constexpr int kRadixSteps = P3M_RADIX_STEPS;              // items per lane
constexpr int kRadixTile = kRadixThreads * kRadixSteps;   // items per block
static_assert(kRadixThreads == kRadixThreadsPublic && kRadixTile == kRadixTilePublic, "radix tiling");

// Subtile id of particle i: g_d = min(floor(x_d M_d / L), M_d - 1) with one correctly
// rounded multiply; a coordinate outside [0, L) (or NaN) is binned as 0 and sets *bad.
__device__ __forceinline__ int bin_one(const double* __restrict__ pos, int64_t n, int64_t i, const Geometry& g,
                                       bool& bad) {
  int gc[3];
  const long long box_bits = __double_as_longlong(g.box);
#pragma unroll
  for (int d = 0; d < 3; ++d) {
    double v = pos[d * n + i];
    // 0 <= v < L on the bit patterns (non-negative doubles order like integers;
    // NaN, negative values and v >= L all fail)
    const long long vb = __double_as_longlong(v);
    bool ok = (vb >= 0) && (vb < box_bits);
    bad |= !ok;
    double p = __dmul_rn(ok ? v : 0.0, g.scale64[d]);
    // floor(p) for 0 <= p < 2^31 from the exponent and mantissa bits
    const long long pb = __double_as_longlong(p);
    const int e = (int)(pb >> 52) - 1023;
    int q = 0;
    if (e >= 0) q = (int)((((pb & 0xfffffffffffffLL) | (1LL << 52)) >> (52 - e)));
    gc[d] = q < g.M[d] - 1 ? q : g.M[d] - 1;
  }
  return encode_subtile_fast(g, gc[0], gc[1], gc[2]);  // 0 <= gc < M < 2^22
}

__global__ void k_bin(const double* __restrict__ pos, int64_t n, Geometry g, int* __restrict__ keys,
                      int* __restrict__ vals, int* __restrict__ counts, int* __restrict__ err) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const bool valid = i < n;  // every lane stays for the warp-wide match below
  int id = 0;
  if (valid) {
    bool bad = false;
    id = bin_one(pos, n, i, g, bad);
    if (bad) atomicOr(err, kErrPosition);
    keys[i] = id;
    vals[i] = (int)i;
  }
  // one atomic per distinct subtile in the warp (sorted input repeats ids)
  const int lane = threadIdx.x & 31;
  const unsigned peers = __match_any_sync(0xffffffffu, valid ? id : -1 - lane);
  if (valid && lane == __ffs(peers) - 1) atomicAdd(&counts[id], __popc(peers));
}

// k_bin over radix tiles of kRadixTile particles, which also counts the digits of
// the first radix pass (bits low bits of the id) per tile: hist[d nblocks + tile].
__global__ void __launch_bounds__(256) k_bin_tile(const double* __restrict__ pos, int64_t n, Geometry g,
                                                  int* __restrict__ keys, int* __restrict__ vals,
                                                  int* __restrict__ counts, int* __restrict__ err,
                                                  int* __restrict__ hist, int bits, int nblocks) {
  __shared__ int cnt[1024];
  const int radix = 1 << bits, mask = radix - 1;
  for (int d = threadIdx.x; d < radix; d += blockDim.x) cnt[d] = 0;
  __syncthreads();
  const int lane = threadIdx.x & 31;
  const int64_t base = (int64_t)blockIdx.x * kRadixTile;
  bool any_bad = false;
  for (int k = 0; k < kRadixSteps; ++k) {
    const int64_t i = base + (int64_t)k * kRadixThreads + threadIdx.x;
    const bool valid = i < n;
    int id = 0;
    if (valid) {
      id = bin_one(pos, n, i, g, any_bad);
      keys[i] = id;
      vals[i] = (int)i;
      atomicAdd(&cnt[id & mask], 1);
    }
    const unsigned peers = __match_any_sync(0xffffffffu, valid ? id : -1 - lane);
    if (valid && lane == __ffs(peers) - 1) atomicAdd(&counts[id], __popc(peers));
  }
  if (any_bad) atomicOr(err, kErrPosition);
  __syncthreads();
  for (int d = threadIdx.x; d < radix; d += blockDim.x) hist[(int64_t)d * nblocks + blockIdx.x] = cnt[d];
}

constexpr int kMaxRadix = 1024;  // digits of at most 10 bits

__global__ void k_radix_hist(const int* __restrict__ keys, int64_t n, int shift, int bits,
                             int* __restrict__ hist, int nblocks) {
  __shared__ int cnt[kMaxRadix];
  const int radix = 1 << bits;
  for (int d = threadIdx.x; d < radix; d += blockDim.x) cnt[d] = 0;
  __syncthreads();
  int64_t base = (int64_t)blockIdx.x * kRadixTile;
  const int mask = radix - 1;
  for (int k = 0; k < kRadixSteps; ++k) {
    int64_t i = base + (int64_t)k * kRadixThreads + threadIdx.x;
    if (i < n) atomicAdd(&cnt[(keys[i] >> shift) & mask], 1);
  }
  __syncthreads();
  for (int d = threadIdx.x; d < radix; d += blockDim.x) hist[(int64_t)d * nblocks + blockIdx.x] = cnt[d];
}

// Stable scatter of one radix pass.  Warp w of a block owns the contiguous
// items [w*512, (w+1)*512) of the block's tile and walks them in 16 steps of
// 32 consecutive items, so ranks follow the input order.  The block then puts
// its tile in digit order in shared memory and writes it out from there, so that
// consecutive threads write consecutive positions of each digit's run.
// hist_next (nullable, zeroed before the launch): the digit counts of the next pass
// (bits_next bits from shift_next) per output tile, accumulated here with one atomic
// per distinct (digit, tile) of each warp, so that pass needs no histogram kernel.
__global__ void __launch_bounds__(kRadixThreads) k_radix_scatter(
    const int* __restrict__ keys_in, const int* __restrict__ vals_in, int* __restrict__ keys_out,
    int* __restrict__ vals_out, int64_t n, int shift, int bits, const int* __restrict__ hist, int nblocks,
    int* __restrict__ hist_next, int shift_next, int bits_next) {
  __shared__ int wcnt[kRadixWarps][kMaxRadix];  // per-warp digit counts; later the staged tile
  __shared__ int bstart[kMaxRadix];             // first position of each digit in the block's tile
  __shared__ int wtot[kRadixWarps];
  static_assert(kRadixWarps * kMaxRadix >= 2 * kRadixTile, "staging area");
  const int radix = 1 << bits;
  const int mask = radix - 1;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int d = lane; d < radix; d += 32) wcnt[warp][d] = 0;
  __syncwarp();
  const int64_t tile0 = (int64_t)blockIdx.x * kRadixTile;
  const int64_t wbase = tile0 + (int64_t)warp * (kRadixSteps * kWarp);
  const unsigned lt = (1u << lane) - 1u;
  int key[kRadixSteps], val[kRadixSteps], rank[kRadixSteps];
#pragma unroll
  for (int k = 0; k < kRadixSteps; ++k) {
    int64_t i = wbase + k * kWarp + lane;
    bool valid = i < n;
    key[k] = valid ? keys_in[i] : 0;
    val[k] = valid ? vals_in[i] : 0;
    int d = (key[k] >> shift) & mask;
    int tag = valid ? d : -1 - lane;  // invalid lanes match nobody
    unsigned peers = __match_any_sync(0xffffffffu, tag);
    int r = __popc(peers & lt);
    int base = valid ? wcnt[warp][d] : 0;
    __syncwarp();
    if (valid && r == 0) wcnt[warp][d] = base + __popc(peers);
    __syncwarp();
    rank[k] = base + r;
  }
  __syncthreads();
  // exclusive prefix over the warps of the block, per digit; the digit totals
  for (int d = threadIdx.x; d < radix; d += blockDim.x) {
    int run = 0;
#pragma unroll
    for (int w = 0; w < kRadixWarps; ++w) {
      int t = wcnt[w][d];
      wcnt[w][d] = run;
      run += t;
    }
    bstart[d] = run;
  }
  __syncthreads();
  // exclusive scan of the digit totals: thread t holds digits [4t, 4t + 4)
  {
    int v[4], tot = 0;
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int d = 4 * threadIdx.x + q;
      v[q] = d < radix ? bstart[d] : 0;
      tot += v[q];
    }
    int inc = tot;
    for (int o = 1; o < 32; o <<= 1) {
      const int u = __shfl_up_sync(0xffffffffu, inc, o);
      if (lane >= o) inc += u;
    }
    if (lane == 31) wtot[warp] = inc;
    __syncthreads();
    int run = inc - tot;
    for (int w = 0; w < warp; ++w) run += wtot[w];
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int d = 4 * threadIdx.x + q;
      if (d < radix) bstart[d] = run;
      run += v[q];
    }
  }
  __syncthreads();
  int lp[kRadixSteps];  // position of each item in the block's digit-ordered tile
#pragma unroll
  for (int k = 0; k < kRadixSteps; ++k) {
    const int d = (key[k] >> shift) & mask;
    lp[k] = bstart[d] + wcnt[warp][d] + rank[k];
  }
  __syncthreads();  // every warp has read wcnt
  int* sk = &wcnt[0][0];
  int* sv = sk + kRadixTile;
  const int64_t left = n - tile0;
  const int nvalid = left < kRadixTile ? (int)left : kRadixTile;
#pragma unroll
  for (int k = 0; k < kRadixSteps; ++k) {
    if (wbase + k * kWarp + lane < n) {
      sk[lp[k]] = key[k];
      sv[lp[k]] = val[k];
    }
  }
  __syncthreads();
  const int mask_next = (1 << bits_next) - 1;
  for (int p = threadIdx.x; p < kRadixTile; p += kRadixThreads) {
    const bool valid = p < nvalid;
    int tag = -1 - lane;
    if (valid) {
      const int kk = sk[p];
      const int d = (kk >> shift) & mask;
      const int64_t dst = (int64_t)hist[(int64_t)d * nblocks + blockIdx.x] + (p - bstart[d]);
      keys_out[dst] = kk;
      vals_out[dst] = sv[p];
      tag = ((kk >> shift_next) & mask_next) * nblocks + (int)(dst / kRadixTile);
    }
    if (hist_next) {  // uniform over the launch
      const unsigned peers = __match_any_sync(0xffffffffu, tag);
      if (valid && lane == __ffs(peers) - 1) atomicAdd(&hist_next[tag], __popc(peers));
    }
  }
}

__global__ void k_gather_pos(const double* __restrict__ src, const int* __restrict__ perm, int64_t n,
                             double* __restrict__ dst) {
  int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= n) return;
  int64_t j = perm[k];
  dst[k] = src[j];
  dst[n + k] = src[n + j];
  dst[2 * n + k] = src[2 * n + j];
}

// Gather the positions into walk order and write the FP32 record of each
// particle: its coordinates relative to the origin of its subtile and the id.
__global__ void k_gather_pos_rel4(const double* __restrict__ src, const int* __restrict__ perm,
                                  const int* __restrict__ cell, int64_t n, Geometry g, double* __restrict__ dst,
                                  float4* __restrict__ rel4) {
  int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= n) return;
  int64_t j = perm[k];
  const double x = src[j], y = src[n + j], z = src[2 * n + j];
  dst[k] = x;
  dst[n + k] = y;
  dst[2 * n + k] = z;
  const int id = cell[k];
  int gx, gy, gz;
  decode_subtile(g, id, gx, gy, gz);
  double r[3];
  rel_to_subtile(g, x, y, z, gx, gy, gz, r);
  rel4[k] = make_float4((float)r[0], (float)r[1], (float)r[2], __int_as_float(id));
}

// Carried arrays of an out-of-place sort: element bytes as `words` words of
// `wbytes` (8, 4, 2 or 1) bytes, chosen from the size and alignment.
constexpr int kMaxCarry = 8;
struct CarrySet {
  const void* src[kMaxCarry];
  void* dst[kMaxCarry];
  int words[kMaxCarry];
  int wbytes[kMaxCarry];
  int count;
};

template <class T>
__device__ __forceinline__ void copy_words(const void* src, void* dst, int64_t j, int64_t k, int words) {
  const T* s = (const T*)src + j * words;
  T* d = (T*)dst + k * words;
  for (int w = 0; w < words; ++w) d[w] = s[w];
}

// The sorted positions, their FP32 records and every carried array in one pass:
// element k of each output is element perm[k] of the input.
__global__ void k_gather_all(const double* __restrict__ src, const int* __restrict__ perm,
                             const int* __restrict__ cell, int64_t n, Geometry g, double* __restrict__ dst,
                             float4* __restrict__ rel4, CarrySet cs) {
  const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= n) return;
  const int64_t j = perm[k];
  const double x = src[j], y = src[n + j], z = src[2 * n + j];
  dst[k] = x;
  dst[n + k] = y;
  dst[2 * n + k] = z;
  const int id = cell[k];
  int gx, gy, gz;
  decode_subtile(g, id, gx, gy, gz);
  double r[3];
  rel_to_subtile(g, x, y, z, gx, gy, gz, r);
  rel4[k] = make_float4((float)r[0], (float)r[1], (float)r[2], __int_as_float(id));
  for (int c = 0; c < cs.count; ++c) {
    switch (cs.wbytes[c]) {
      case 8: copy_words<unsigned long long>(cs.src[c], cs.dst[c], j, k, cs.words[c]); break;
      case 4: copy_words<unsigned>(cs.src[c], cs.dst[c], j, k, cs.words[c]); break;
      case 2: copy_words<unsigned short>(cs.src[c], cs.dst[c], j, k, cs.words[c]); break;
      default: copy_words<unsigned char>(cs.src[c], cs.dst[c], j, k, cs.words[c]); break;
    }
  }
}

template <class T>
__global__ void k_gather_words(const T* __restrict__ src, const int* __restrict__ perm, int64_t n, int words,
                               T* __restrict__ dst) {
  int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= n) return;
  int64_t j = perm[k];
  for (int w = 0; w < words; ++w) dst[k * words + w] = src[j * words + w];
}

__global__ void k_fill_origins(Geometry g, double* __restrict__ org) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const int d = i < g.M[0] ? 0 : (i < g.M[0] + g.M[1] ? 1 : 2);
  const int j = i - (d > 0 ? g.M[0] : 0) - (d > 1 ? g.M[1] : 0);
  if (d == 2 && j >= g.M[2]) return;
  org[i] = __dmul_rn((double)j, g.side64[d]);
}

static unsigned blocks_for(int64_t n, int t) { return (unsigned)((n + t - 1) / t); }

// dst[r n + k] = src[r n + perm[k]] (to sorted order) or dst[r n + perm[k]] = src[r n + k] (back).
template <class T>
__global__ void k_permute_rows(const T* __restrict__ src, T* __restrict__ dst, const int* __restrict__ perm, int64_t n,
                               int rows, int to_sorted) {
  int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= n) return;
  int64_t j = perm[k];
  for (int r = 0; r < rows; ++r) {
    if (to_sorted) dst[(int64_t)r * n + k] = src[(int64_t)r * n + j];
    else dst[(int64_t)r * n + j] = src[(int64_t)r * n + k];
  }
}

static p3m_status gather_carry(p3m_sr_ctx* ctx, void* arr, int bytes) {
  const int64_t n = ctx->n;
  const int t = 256;
  cudaStream_t s = ctx->stream;
  uintptr_t a = (uintptr_t)arr;
  if (bytes % 8 == 0 && a % 8 == 0)
    k_gather_words<uint64_t><<<blocks_for(n, t), t, 0, s>>>((const uint64_t*)arr, ctx->perm, n, bytes / 8,
                                                             (uint64_t*)ctx->gather_tmp);
  else if (bytes % 4 == 0 && a % 4 == 0)
    k_gather_words<uint32_t><<<blocks_for(n, t), t, 0, s>>>((const uint32_t*)arr, ctx->perm, n, bytes / 4,
                                                             (uint32_t*)ctx->gather_tmp);
  else if (bytes % 2 == 0 && a % 2 == 0)
    k_gather_words<uint16_t><<<blocks_for(n, t), t, 0, s>>>((const uint16_t*)arr, ctx->perm, n, bytes / 2,
                                                             (uint16_t*)ctx->gather_tmp);
  else
    k_gather_words<uint8_t><<<blocks_for(n, t), t, 0, s>>>((const uint8_t*)arr, ctx->perm, n, bytes,
                                                            (uint8_t*)ctx->gather_tmp);
  ++ctx->launches;
  p3m_status st = cuda_check(ctx, cudaGetLastError(), "gather kernel");
  if (st != P3M_OK) return st;
  return cuda_check(ctx, cudaMemcpyAsync(arr, ctx->gather_tmp, (size_t)bytes * n, cudaMemcpyDeviceToDevice, s),
                    "carry copy");
}

}  // namespace p3m

using namespace p3m;

// Bin the particles of pos and sort their subtile ids (Section 2.1.3: an O(N)
// sort into tiles): fills the subtile offsets, ctx->cell (sorted ids) and
// ctx->perm (sorted -> input index).  The first radix pass's digit histogram is
// counted by the binning kernel and each later pass's by the scatter before it.
static p3m_status bin_and_sort_ids(p3m_sr_ctx* ctx, const double* pos) {
  const int64_t n = ctx->n;
  cudaStream_t s = ctx->stream;
  const Geometry& g = ctx->geo;
  p3m_status st = cuda_check(ctx, cudaMemsetAsync(ctx->offsets, 0, sizeof(int) * (g.S + 1), s), "memset offsets");
  if (st != P3M_OK) return st;
  const int nblocks = (int)((n + kRadixTile - 1) / kRadixTile);
  int* hist[2] = {ctx->hist, ctx->hist + ctx->hist_ints};  // this pass's and the next pass's digit counts
  if (n > 0) {
    k_bin_tile<<<nblocks, kRadixThreads, 0, s>>>(pos, n, g, ctx->keys[0], ctx->vals[0], ctx->offsets, ctx->err_dev,
                                                 hist[0], ctx->radix_bits[0], nblocks);
    ++ctx->launches;
    if ((st = cuda_check(ctx, cudaGetLastError(), "bin kernel")) != P3M_OK) return st;
  }
  st = cuda_check(ctx, scan_exclusive_i32(ctx->offsets, ctx->offsets, g.S + 1, ctx->scan_scratch,
                                          ctx->scan_scratch_ints, s, &ctx->launches),
                  "scan");
  if (st != P3M_OK) return st;
  int cur = 0;
  if (n > 0) {
    int shift = 0;
    for (int p = 0; p < ctx->radix_passes; ++p) {
      const int bits = ctx->radix_bits[p];
      const bool more = p + 1 < ctx->radix_passes;
      st = cuda_check(ctx, scan_exclusive_i32(hist[p & 1], hist[p & 1], (int64_t)nblocks << bits, ctx->scan_scratch,
                                              ctx->scan_scratch_ints, s,
                                              &ctx->launches), "radix scan");
      if (st != P3M_OK) return st;
      int* next = more ? hist[(p + 1) & 1] : nullptr;
      if (more && (st = cuda_check(ctx, cudaMemsetAsync(next, 0, sizeof(int) * ((int64_t)nblocks << ctx->radix_bits[p + 1]), s),
                                   "memset hist")) != P3M_OK)
        return st;
      k_radix_scatter<<<nblocks, kRadixThreads, 0, s>>>(ctx->keys[cur], ctx->vals[cur], ctx->keys[cur ^ 1],
                                                          ctx->vals[cur ^ 1], n, shift, bits, hist[p & 1], nblocks, next,
                                                          shift + bits, more ? ctx->radix_bits[p + 1] : 0);
      ++ctx->launches;
      if ((st = cuda_check(ctx, cudaGetLastError(), "radix scatter")) != P3M_OK) return st;
      cur ^= 1;
      shift += bits;
    }
  }
  ctx->cell = ctx->keys[cur];
  ctx->perm = ctx->vals[cur];
  return P3M_OK;
}

static p3m_status sort_outputs(p3m_sr_ctx* ctx, int32_t* perm_out, int32_t* subtile_id_out) {
  const int64_t n = ctx->n;
  p3m_status st = P3M_OK;
  if (n > 0 && perm_out)
    if ((st = cuda_check(ctx, cudaMemcpyAsync(perm_out, ctx->perm, sizeof(int) * n, cudaMemcpyDeviceToDevice,
                                              ctx->stream), "perm copy")) != P3M_OK)
      return st;
  if (n > 0 && subtile_id_out)
    if ((st = cuda_check(ctx, cudaMemcpyAsync(subtile_id_out, ctx->cell, sizeof(int) * n, cudaMemcpyDeviceToDevice,
                                              ctx->stream), "id copy")) != P3M_OK)
      return st;
  return P3M_OK;
}

static p3m_status sort_done(p3m_sr_ctx* ctx, const double* sorted_pos) {
  report_latched(ctx);
  ctx->sorted = true;
  ctx->sorted_pos = sorted_pos;  // the FP32 records in ctx->rel4 describe these positions
  ctx->n_drift = 0;              // no displacement since this sort
  ctx->rel4_stale = false;
  return cuda_check(ctx, cudaMemsetAsync(ctx->drift_slots, 0, sizeof(float) * kMaxDrifts, ctx->stream), "memset");
}

static p3m_status check_carry(p3m_sr_ctx* ctx, void* const* carry, const int* carry_bytes, int n_carry,
                              const char* name) {
  if (n_carry < 0 || (n_carry > 0 && (!carry || !carry_bytes)))
    return fail(ctx, P3M_ERR_INVALID, std::string(name) + ": bad carry arguments");
  for (int c = 0; c < n_carry; ++c) {
    if (carry_bytes[c] < 1 || carry_bytes[c] > 32)
      return fail(ctx, P3M_ERR_INVALID, std::string(name) + ": carry_bytes must be 1..32");
    if (!carry[c] && ctx->n > 0) return fail(ctx, P3M_ERR_INVALID, std::string(name) + ": null carry array");
  }
  return P3M_OK;
}

extern "C" p3m_status p3m_sr_sort(p3m_sr_ctx* ctx, double* pos, void* const* carry, const int* carry_bytes,
                                  int n_carry, int32_t* perm_out, int32_t* subtile_id_out) {
  if (!ctx) return P3M_ERR_INVALID;
  const int64_t n = ctx->n;
  p3m_status st = check_carry(ctx, carry, carry_bytes, n_carry, "sort");
  if (st != P3M_OK) return st;
  if (!pos && n > 0) return fail(ctx, P3M_ERR_INVALID, "sort: null positions");
  if ((st = poll_latched(ctx)) != P3M_OK) return st;
  cudaStream_t s = ctx->stream;
  ctx->pairs_built = false;
  ctx->all_chunks_built = false;
  if ((st = bin_and_sort_ids(ctx, pos)) != P3M_OK) return st;
  if (n > 0) {
    double* tmp = (double*)ctx->gather_tmp;
    k_gather_pos_rel4<<<blocks_for(n, 256), 256, 0, s>>>(pos, ctx->perm, ctx->cell, n, ctx->geo, tmp, ctx->rel4);
    ++ctx->launches;
    if ((st = cuda_check(ctx, cudaGetLastError(), "gather positions")) != P3M_OK) return st;
    st = cuda_check(ctx, cudaMemcpyAsync(pos, tmp, sizeof(double) * 3 * n, cudaMemcpyDeviceToDevice, s), "copy");
    if (st != P3M_OK) return st;
    for (int c = 0; c < n_carry; ++c)
      if ((st = gather_carry(ctx, carry[c], carry_bytes[c])) != P3M_OK) return st;
  }
  if ((st = sort_outputs(ctx, perm_out, subtile_id_out)) != P3M_OK) return st;
  return sort_done(ctx, pos);
}

extern "C" p3m_status p3m_sr_sort_into(p3m_sr_ctx* ctx, const double* pos_in, double* pos_out,
                                       const void* const* carry_in, void* const* carry_out, const int* carry_bytes,
                                       int n_carry, int32_t* perm_out, int32_t* subtile_id_out) {
  if (!ctx) return P3M_ERR_INVALID;
  const int64_t n = ctx->n;
  if (n_carry > kMaxCarry) return fail(ctx, P3M_ERR_INVALID, "sort_into: at most 8 carried arrays");
  p3m_status st = check_carry(ctx, carry_out, carry_bytes, n_carry, "sort_into");
  if (st != P3M_OK) return st;
  if (n > 0 && (!pos_in || !pos_out)) return fail(ctx, P3M_ERR_INVALID, "sort_into: null positions");
  if (n > 0 && pos_in == pos_out) return fail(ctx, P3M_ERR_INVALID, "sort_into: pos_in and pos_out must differ");
  CarrySet cs{};
  cs.count = n_carry;
  for (int c = 0; c < n_carry; ++c) {
    if (n > 0 && (!carry_in || !carry_in[c] || carry_in[c] == carry_out[c]))
      return fail(ctx, P3M_ERR_INVALID, "sort_into: carried inputs must be non-null and differ from the outputs");
    const int b = carry_bytes[c];
    const uintptr_t al = (uintptr_t)(n > 0 ? carry_in[c] : nullptr) | (uintptr_t)carry_out[c];
    const int wb = (b % 8 == 0 && al % 8 == 0) ? 8 : (b % 4 == 0 && al % 4 == 0) ? 4 : (b % 2 == 0 && al % 2 == 0) ? 2 : 1;
    cs.src[c] = n > 0 ? carry_in[c] : nullptr;
    cs.dst[c] = carry_out[c];
    cs.wbytes[c] = wb;
    cs.words[c] = b / wb;
  }
  if ((st = poll_latched(ctx)) != P3M_OK) return st;
  ctx->pairs_built = false;
  ctx->all_chunks_built = false;
  if ((st = bin_and_sort_ids(ctx, pos_in)) != P3M_OK) return st;
  if (n > 0) {
    k_gather_all<<<blocks_for(n, 256), 256, 0, ctx->stream>>>(pos_in, ctx->perm, ctx->cell, n, ctx->geo, pos_out,
                                                             ctx->rel4, cs);
    ++ctx->launches;
    if ((st = cuda_check(ctx, cudaGetLastError(), "gather kernel")) != P3M_OK) return st;
  }
  if ((st = sort_outputs(ctx, perm_out, subtile_id_out)) != P3M_OK) return st;
  return sort_done(ctx, pos_out);
}

// out[T] = first sorted index of tile T (T = (t_x n_t + t_y) n_t + t_z), out[n_tiles] = n.
__global__ void k_tile_offsets(const int* __restrict__ offsets, int64_t n_tiles, int nsub3, int* __restrict__ out) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t <= n_tiles) out[t] = offsets[t * nsub3];
}

extern "C" p3m_status p3m_sr_tile_offsets(p3m_sr_ctx* ctx, int32_t* offsets_out) {
  if (!ctx) return P3M_ERR_INVALID;
  if (!offsets_out) return fail(ctx, P3M_ERR_INVALID, "tile_offsets: null output");
  if (!ctx->sorted) return fail(ctx, P3M_ERR_STATE, "tile_offsets: call p3m_sr_sort first");
  const int64_t nt = ctx->n_tiles;
  k_tile_offsets<<<blocks_for(nt + 1, 256), 256, 0, ctx->stream>>>(ctx->offsets, nt, ctx->geo.nsub3, offsets_out);
  ++ctx->launches;
  return cuda_check(ctx, cudaGetLastError(), "tile offsets kernel");
}

static p3m_status permute_rows(p3m_sr_ctx* ctx, const void* src, void* dst, int elem_bytes, int rows, int to_sorted,
                               const char* name) {
  if (!ctx) return P3M_ERR_INVALID;
  if (!ctx->sorted && !ctx->perm) return fail(ctx, P3M_ERR_STATE, std::string(name) + ": call p3m_sr_sort first");
  if (!ctx->perm) return fail(ctx, P3M_ERR_STATE, std::string(name) + ": call p3m_sr_sort first");
  if (rows < 1 || (elem_bytes != 1 && elem_bytes != 2 && elem_bytes != 4 && elem_bytes != 8))
    return fail(ctx, P3M_ERR_INVALID, std::string(name) + ": elem_bytes must be 1, 2, 4 or 8 and rows >= 1");
  const int64_t n = ctx->n;
  if (n == 0) return P3M_OK;
  if (!src || !dst || src == dst) return fail(ctx, P3M_ERR_INVALID, std::string(name) + ": need distinct non-null arrays");
  const unsigned b = blocks_for(n, 256);
  cudaStream_t s = ctx->stream;
  switch (elem_bytes) {
    case 1: k_permute_rows<uint8_t><<<b, 256, 0, s>>>((const uint8_t*)src, (uint8_t*)dst, ctx->perm, n, rows, to_sorted); break;
    case 2: k_permute_rows<uint16_t><<<b, 256, 0, s>>>((const uint16_t*)src, (uint16_t*)dst, ctx->perm, n, rows, to_sorted); break;
    case 4: k_permute_rows<uint32_t><<<b, 256, 0, s>>>((const uint32_t*)src, (uint32_t*)dst, ctx->perm, n, rows, to_sorted); break;
    default: k_permute_rows<uint64_t><<<b, 256, 0, s>>>((const uint64_t*)src, (uint64_t*)dst, ctx->perm, n, rows, to_sorted); break;
  }
  ++ctx->launches;
  return cuda_check(ctx, cudaGetLastError(), name);
}

extern "C" p3m_status p3m_sr_permute(p3m_sr_ctx* ctx, const void* src, void* dst, int elem_bytes, int rows) {
  return permute_rows(ctx, src, dst, elem_bytes, rows, 1, "permute");
}

extern "C" p3m_status p3m_sr_unpermute(p3m_sr_ctx* ctx, const void* src, void* dst, int elem_bytes, int rows) {
  return permute_rows(ctx, src, dst, elem_bytes, rows, 0, "unpermute");
}
