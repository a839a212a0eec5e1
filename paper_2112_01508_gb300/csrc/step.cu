// Rung assignment (Section 2.2.2, Eq. rung), kick and drift (Section 2.2.2,
// operators K and D with a static scale factor a = 1).  All three are
// elementwise and HBM-bound; the arithmetic is IEEE double with explicit
// round-to-nearest intrinsics so that the integer rung decision and the
// updated momenta/positions are reproducible bit for bit.
#include <algorithm>
#include <cmath>

#include <type_traits>

#include "ctx.cuh"

namespace p3m {

static unsigned blocks_for(int64_t n, int t) { return (unsigned)((n + t - 1) / t); }

#ifndef P3M_KD_MINBLOCKS
#define P3M_KD_MINBLOCKS 4  // resident blocks of 256 asked of the drift kernels (64 registers; 10% faster than 72)
#endif
constexpr int kKdMinBlocks = P3M_KD_MINBLOCKS;

// Eq. rung for the acceleration (ax, ay, az): the smallest l >= 0 with
// s = qq |a|^2 <= 16^l, s = qq ((ax^2 + ay^2) + az^2) with each FP64 operation
// correctly rounded, clamped to n_rung - 1; a non-finite s latches
// kErrNonfiniteAcc and gives 0.
//
// FP32 accelerations take an FP32 first pass: they are exact in FP64, and with
// qqf = fl32(qq) the FP32 s has a relative error below 7 x 2^-24.  The rung changes
// only where s crosses a power of 16; unless the FP32 s lies within 64 ulps of one,
// the FP64 s is on the same side of every boundary and gives the same rung.  Near
// a boundary, or out of the FP32 normal range (qqf = 0 when qq is), the FP64 rule
// decides.
template <class A>
__device__ __forceinline__ int rung_rule(A ax, A ay, A az, double qq, float qqf, int n_rung, int* err) {
  if constexpr (std::is_same<A, float>::value) {
    if (qqf > 0.0f) {
      const float a2f = __fadd_rn(__fadd_rn(__fmul_rn(ax, ax), __fmul_rn(ay, ay)), __fmul_rn(az, az));
      const float sf = __fmul_rn(qqf, a2f);
      if (a2f >= 1e-30f && sf <= 1e30f) {  // false for NaN and infinity too
        const int b = __float_as_int(sf);
        const int e = ((b >> 23) & 0xff) - 127;
        const int m = b & 0x7fffff;
        const bool near = ((e & 3) == 0 && m < 64) || ((e & 3) == 3 && m > 0x7fffff - 64);
        if (!near) return sf > 1.0f ? min((e + (m != 0 ? 1 : 0) + 3) >> 2, n_rung - 1) : 0;
      }
    }
  }
  const double x = (double)ax, y = (double)ay, z = (double)az;
  const double a2 = __dadd_rn(__dadd_rn(__dmul_rn(x, x), __dmul_rn(y, y)), __dmul_rn(z, z));
  const double s = __dmul_rn(qq, a2);
  int l = 0;
  if (isnan(s) || isinf(s)) {
    atomicOr(err, kErrNonfiniteAcc);
  } else if (s > 1.0) {
    // smallest k with s <= 2^k from the exponent bits (s = m 2^e, m in [1, 2)):
    // k = e if s is a power of two, else e + 1; then l = ceil(k / 4)
    long long b = __double_as_longlong(s);
    int e = (int)((b >> 52) & 0x7ff) - 1023;
    int k = e + (((b & 0xfffffffffffffLL) != 0) ? 1 : 0);
    l = (k + 3) >> 2;
    if (l > n_rung - 1) l = n_rung - 1;
  }
  return l;
}

// qqf: fl32(qq) for the FP32 first pass of rung_rule, or 0 to skip it.
__host__ inline float rung_qqf(double qq) { return (qq >= 1e-30 && qq <= 1e30) ? (float)qq : 0.0f; }

template <class A>
__global__ void k_rungs(const A* __restrict__ acc, int64_t n, double qq, float qqf, int n_rung,
                        int8_t* __restrict__ rung, int* __restrict__ err) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  rung[i] = (int8_t)rung_rule<A>(acc[i], acc[n + i], acc[2 * n + i], qq, qqf, n_rung, err);
}

struct KickFactors {
  double k[8];
};

template <class M, class A>
__global__ void k_kick(M* __restrict__ mom, const A* __restrict__ acc, const int8_t* __restrict__ rung, int rung_min,
                       int64_t n, KickFactors kf) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  double k = kf.k[0];
  if (rung) {
    int l = rung[i];
    if (l < rung_min) return;
    k = kf.k[l < 0 ? 0 : (l > 7 ? 7 : l)];
  }
#pragma unroll
  for (int d = 0; d < 3; ++d) {
    double q = (double)mom[d * n + i];
    double v = __dadd_rn(q, __dmul_rn((double)acc[d * n + i], k));
    mom[d * n + i] = (M)v;
  }
}

// disp (optional): receives, by atomic max, an upper bound of the largest
// displacement |q| |factor| of this drift (non-negative floats order as
// integers), one atomic per block.
template <class M>
__global__ void __launch_bounds__(256, kKdMinBlocks) k_drift(double* __restrict__ pos, const M* __restrict__ mom, int64_t n,
                                               double factor, double box, float* __restrict__ disp) {
  __shared__ unsigned warp_max[8];
  float my = 0.0f;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    float q2 = 0.0f;
#pragma unroll
    for (int d = 0; d < 3; ++d) {
      const double q = (double)mom[d * n + i];
      const float qf = (float)q;
      q2 = fmaf(qf, qf, q2);
      double v = __dadd_rn(pos[d * n + i], __dmul_rn(q, factor));
      const long long vb = __double_as_longlong(v);
      if (!(vb >= 0 && vb < __double_as_longlong(box))) {  // v - L floor(v / L); floor is 0 inside the box
        v = __dsub_rn(v, __dmul_rn(box, floor(__ddiv_rn(v, box))));
        if (v >= box || v < 0.0) v = 0.0;
      }
      pos[d * n + i] = v;
    }
    // FP32 with a relative margin far above its rounding (a few ulps)
    float di = sqrtf(q2) * (float)fabs(factor) * 1.0001f;
    if (!(di < 3.0e38f)) di = 3.0e38f;  // non-finite or huge momenta: the bound saturates
    my = fmaxf(my, di);
  }
  if (disp) {
    const unsigned m = __reduce_max_sync(0xffffffffu, __float_as_uint(my));
    if ((threadIdx.x & 31) == 0) warp_max[threadIdx.x >> 5] = m;
    __syncthreads();
    if (threadIdx.x == 0) {
      unsigned b = 0;
      for (int w = 0; w < (int)(blockDim.x >> 5); ++w) b = max(b, warp_max[w]);
      if (b) atomicMax((unsigned*)disp, b);
    }
  }
}

// Rungs (Eq. rung), kick and drift in one pass over the particle arrays: the
// arithmetic of k_rungs, k_kick (rung_min 0) and k_drift in that order, so the
// results are those of the three kernels bit for bit.  disp as in k_drift.
template <class M, class A>
__global__ void __launch_bounds__(256, kKdMinBlocks) k_kick_drift(double* __restrict__ pos, M* __restrict__ mom,
                                                    const A* __restrict__ acc, int8_t* __restrict__ rung, int64_t n,
                                                    double qq, float qqf, int n_rung, KickFactors kf, double factor,
                                                    double box, float* __restrict__ disp, int* __restrict__ err) {
  __shared__ unsigned warp_max[8];
  float my = 0.0f;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const A av[3] = {acc[i], acc[n + i], acc[2 * n + i]};
    const int l = rung_rule<A>(av[0], av[1], av[2], qq, qqf, n_rung, err);
    rung[i] = (int8_t)l;
    const double k = kf.k[l];
    float q2 = 0.0f;
#pragma unroll
    for (int d = 0; d < 3; ++d) {
      const M qm = (M)__dadd_rn((double)mom[d * n + i], __dmul_rn((double)av[d], k));
      mom[d * n + i] = qm;
      const double q = (double)qm;
      const float qf = (float)q;
      q2 = fmaf(qf, qf, q2);
      double v = __dadd_rn(pos[d * n + i], __dmul_rn(q, factor));
      const long long vb = __double_as_longlong(v);
      if (!(vb >= 0 && vb < __double_as_longlong(box))) {
        v = __dsub_rn(v, __dmul_rn(box, floor(__ddiv_rn(v, box))));
        if (v >= box || v < 0.0) v = 0.0;
      }
      pos[d * n + i] = v;
    }
    float di = sqrtf(q2) * (float)fabs(factor) * 1.0001f;
    if (!(di < 3.0e38f)) di = 3.0e38f;
    my = fmaxf(my, di);
  }
  if (disp) {
    const unsigned m = __reduce_max_sync(0xffffffffu, __float_as_uint(my));
    if ((threadIdx.x & 31) == 0) warp_max[threadIdx.x >> 5] = m;
    __syncthreads();
    if (threadIdx.x == 0) {
      unsigned b = 0;
      for (int w = 0; w < (int)(blockDim.x >> 5); ++w) b = max(b, warp_max[w]);
      if (b) atomicMax((unsigned*)disp, b);
    }
  }
}

// One kick of the rung-based leapfrog with the rung update (see p3m_sr_rung_kick) for
// particle i.
template <class M, class A>
__device__ __forceinline__ void rung_kick_one(M* __restrict__ mom, const A* __restrict__ acc, int8_t* __restrict__ rung,
                                              int8_t* __restrict__ state, int64_t n, int64_t i, int rung_min,
                                              long long k, int log2_sub, double dt, double qq, float qqf, int n_rung,
                                              int sync, int* __restrict__ err) {
  const int l = rung[i];
  if (l < rung_min) return;
  const int st = state[i];
  if (l >= n_rung || st < 0 || st > 2) {  // corrupted rung or state: leave the particle alone
    atomicOr(err, kErrRungState);
    return;
  }
  const double f = st == 0 ? 1.0 : (st == 1 ? 0.5 : 0.75);
  const double fac = sync ? f - 0.5 : f;
  const double K = ldexp(__dmul_rn(dt, fac), -l);  // fac dt / 2^l (the scaling is exact)
  A av[3];
#pragma unroll
  for (int d = 0; d < 3; ++d) {
    av[d] = acc[d * n + i];
    mom[d * n + i] = (M)__dadd_rn((double)mom[d * n + i], __dmul_rn((double)av[d], K));
  }
  if (sync) {
    state[i] = 0;
    return;
  }
  // Eq. rung on the acceleration of this kick (the rule of k_rungs)
  const int lnew = rung_rule<A>(av[0], av[1], av[2], qq, qqf, n_rung, err);
  int out = l, ost = 0;
  if (lnew > l) {
    out = l + 1;  // next kick: half of the finer rung's usual kick
    ost = 1;
  } else if (lnew < l && ((k >> (log2_sub - l)) & 1LL)) {
    out = l - 1;  // only at every other kick of rung l; next kick: 3/4 of the coarser rung's
    ost = 2;
  }
  rung[i] = (int8_t)out;
  state[i] = (int8_t)ost;
}

template <class M, class A>
__global__ void k_rung_kick(M* __restrict__ mom, const A* __restrict__ acc, int8_t* __restrict__ rung,
                            int8_t* __restrict__ state, int64_t n, int rung_min, long long k, int log2_sub, double dt,
                            double qq, float qqf, int n_rung, int sync, int* __restrict__ err) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  rung_kick_one<M, A>(mom, acc, rung, state, n, i, rung_min, k, log2_sub, dt, qq, qqf, n_rung, sync, err);
}

// A rung kick followed by the drift of every particle, in one pass (the results of
// k_rung_kick then k_drift, bit for bit; disp as in k_drift).
template <class M, class A>
__global__ void __launch_bounds__(256, kKdMinBlocks) k_rung_kick_drift(M* __restrict__ mom, const A* __restrict__ acc,
                                                         int8_t* __restrict__ rung, int8_t* __restrict__ state,
                                                         int64_t n, int rung_min, long long k, int log2_sub, double dt,
                                                         double qq, float qqf, int n_rung, int* __restrict__ err,
                                                         double* __restrict__ pos, double factor, double box,
                                                         float* __restrict__ disp) {
  __shared__ unsigned warp_max[8];
  float my = 0.0f;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    rung_kick_one<M, A>(mom, acc, rung, state, n, i, rung_min, k, log2_sub, dt, qq, qqf, n_rung, 0, err);
    float q2 = 0.0f;
#pragma unroll
    for (int d = 0; d < 3; ++d) {
      const double q = (double)mom[d * n + i];
      const float qf = (float)q;
      q2 = fmaf(qf, qf, q2);
      double v = __dadd_rn(pos[d * n + i], __dmul_rn(q, factor));
      const long long vb = __double_as_longlong(v);
      if (!(vb >= 0 && vb < __double_as_longlong(box))) {
        v = __dsub_rn(v, __dmul_rn(box, floor(__ddiv_rn(v, box))));
        if (v >= box || v < 0.0) v = 0.0;
      }
      pos[d * n + i] = v;
    }
    float di = sqrtf(q2) * (float)fabs(factor) * 1.0001f;
    if (!(di < 3.0e38f)) di = 3.0e38f;
    my = fmaxf(my, di);
  }
  if (disp) {
    const unsigned m = __reduce_max_sync(0xffffffffu, __float_as_uint(my));
    if ((threadIdx.x & 31) == 0) warp_max[threadIdx.x >> 5] = m;
    __syncthreads();
    if (threadIdx.x == 0) {
      unsigned b = 0;
      for (int w = 0; w < (int)(blockDim.x >> 5); ++w) b = max(b, warp_max[w]);
      if (b) atomicMax((unsigned*)disp, b);
    }
  }
}

// Drifting the sorted positions keeps the sort usable: the displacement bound of
// each drift is recorded and the pair traversal widens its reach by their sum,
// until kMaxDrifts drifts, after which a new sort is required.  Returns the slot
// that receives this drift's bound (nullptr when pos is not the sorted array).
static float* drift_slot(p3m_sr_ctx* ctx, const double* pos) {
  float* slot = nullptr;
  if (ctx->sorted && pos == ctx->sorted_pos) {
    if (ctx->n_drift < kMaxDrifts) {
      slot = ctx->drift_slots + ctx->n_drift++;
      ctx->rel4_stale = true;
    } else {
      ctx->sorted = false;
      ctx->pairs_built = false;
      ctx->sorted_pos = nullptr;
    }
  }
  return slot;
}

// q = dt^2 / (2 eta eps) in this order in IEEE double, then qq = q^2 (Eq. rung)
static double rung_qq(double dt, double eta, double eps) {
  volatile double t1 = dt * dt;
  volatile double t2 = 2.0 * eta;
  volatile double t3 = t2 * eps;
  volatile double q = t1 / t3;
  return q * q;
}

}  // namespace p3m

using namespace p3m;

extern "C" p3m_status p3m_sr_kick_drift(p3m_sr_ctx* ctx, double* pos, void* mom, int mom_precision, const void* acc,
                                       int acc_precision, int8_t* rung_out, double dt, double eta, double eps,
                                       const double* kick_factor, double drift_factor) {
  if (!ctx) return P3M_ERR_INVALID;
  if ((mom_precision != 32 && mom_precision != 64) || (acc_precision != 32 && acc_precision != 64))
    return fail(ctx, P3M_ERR_INVALID, "kick_drift: precision must be 32 or 64");
  if (!kick_factor) return fail(ctx, P3M_ERR_INVALID, "kick_drift: null kick_factor");
  if (ctx->n > 0 && (!pos || !mom || !acc || !rung_out)) return fail(ctx, P3M_ERR_INVALID, "kick_drift: null pointer");
  if (!(dt >= 0.0) || !(eta > 0.0) || !(eps > 0.0))
    return fail(ctx, P3M_ERR_INVALID, "kick_drift: need dt >= 0, eta > 0, eps > 0");
  if (!std::isfinite(drift_factor)) return fail(ctx, P3M_ERR_INVALID, "kick_drift: drift_factor must be finite");
  p3m_status st = poll_latched(ctx);
  if (st != P3M_OK) return st;
  if (ctx->n == 0) return P3M_OK;
  const double qq = rung_qq(dt, eta, eps);
  KickFactors kf{};
  for (int l = 0; l < ctx->prm.n_rung; ++l) kf.k[l] = kick_factor[l];
  float* slot = drift_slot(ctx, pos);
  const int t = 256;
  const int64_t n = ctx->n;
  const unsigned b = (unsigned)std::min<int64_t>(blocks_for(n, t), (int64_t)ctx->num_sms * 8);
  cudaStream_t s = ctx->stream;
  const int nr = ctx->prm.n_rung;
  const double L = ctx->prm.box;
  const float qqf = rung_qqf(qq);
  if (mom_precision == 64 && acc_precision == 32)
    k_kick_drift<double, float><<<b, t, 0, s>>>(pos, (double*)mom, (const float*)acc, rung_out, n, qq, qqf, nr, kf,
                                                drift_factor, L, slot, ctx->err_dev);
  else if (mom_precision == 64 && acc_precision == 64)
    k_kick_drift<double, double><<<b, t, 0, s>>>(pos, (double*)mom, (const double*)acc, rung_out, n, qq, qqf, nr, kf,
                                                 drift_factor, L, slot, ctx->err_dev);
  else if (mom_precision == 32 && acc_precision == 32)
    k_kick_drift<float, float><<<b, t, 0, s>>>(pos, (float*)mom, (const float*)acc, rung_out, n, qq, qqf, nr, kf,
                                               drift_factor, L, slot, ctx->err_dev);
  else
    k_kick_drift<float, double><<<b, t, 0, s>>>(pos, (float*)mom, (const double*)acc, rung_out, n, qq, qqf, nr, kf,
                                                drift_factor, L, slot, ctx->err_dev);
  ++ctx->launches;
  if ((st = cuda_check(ctx, cudaGetLastError(), "kick-drift kernel")) != P3M_OK) return st;
  report_latched(ctx);
  return P3M_OK;
}

extern "C" p3m_status p3m_sr_assign_rungs(p3m_sr_ctx* ctx, const void* acc, int acc_precision, double dt, double eta,
                                          double eps, int8_t* rung_out) {
  if (!ctx) return P3M_ERR_INVALID;
  if (acc_precision != 32 && acc_precision != 64) return fail(ctx, P3M_ERR_INVALID, "assign_rungs: bad precision");
  if (ctx->n > 0 && (!acc || !rung_out)) return fail(ctx, P3M_ERR_INVALID, "assign_rungs: null pointer");
  if (!(dt >= 0.0) || !(eta > 0.0) || !(eps > 0.0))
    return fail(ctx, P3M_ERR_INVALID, "assign_rungs: need dt >= 0, eta > 0, eps > 0");
  p3m_status st = poll_latched(ctx);
  if (st != P3M_OK) return st;
  if (ctx->n == 0) return P3M_OK;
  // q = dt^2 / (2 eta eps), evaluated in this order in IEEE double
  volatile double t1 = dt * dt;
  volatile double t2 = 2.0 * eta;
  volatile double t3 = t2 * eps;
  volatile double q = t1 / t3;
  double qq = q * q;
  const float qqf = rung_qqf(qq);
  const int t = 256;
  if (acc_precision == 64)
    { k_rungs<double><<<blocks_for(ctx->n, t), t, 0, ctx->stream>>>((const double*)acc, ctx->n, qq, qqf,
                                                                   ctx->prm.n_rung, rung_out, ctx->err_dev);
      ++ctx->launches; }
  else
    { k_rungs<float><<<blocks_for(ctx->n, t), t, 0, ctx->stream>>>((const float*)acc, ctx->n, qq, qqf,
                                                                  ctx->prm.n_rung, rung_out, ctx->err_dev);
      ++ctx->launches; }
  if ((st = cuda_check(ctx, cudaGetLastError(), "rung kernel")) != P3M_OK) return st;
  report_latched(ctx);
  return P3M_OK;
}

extern "C" p3m_status p3m_sr_kick(p3m_sr_ctx* ctx, void* mom, int mom_precision, const void* acc, int acc_precision,
                                  const int8_t* rung, int rung_min, const double* kick_factor) {
  if (!ctx) return P3M_ERR_INVALID;
  if ((mom_precision != 32 && mom_precision != 64) || (acc_precision != 32 && acc_precision != 64))
    return fail(ctx, P3M_ERR_INVALID, "kick: precision must be 32 or 64");
  if (!kick_factor) return fail(ctx, P3M_ERR_INVALID, "kick: null kick_factor");
  if (ctx->n > 0 && (!mom || !acc)) return fail(ctx, P3M_ERR_INVALID, "kick: null pointer");
  p3m_status st = poll_latched(ctx);
  if (st != P3M_OK) return st;
  if (ctx->n == 0) return P3M_OK;
  KickFactors kf{};
  for (int l = 0; l < ctx->prm.n_rung; ++l) kf.k[l] = kick_factor[l];
  const int t = 256;
  const unsigned b = blocks_for(ctx->n, t);
  cudaStream_t s = ctx->stream;
  const int64_t n = ctx->n;
  if (mom_precision == 64 && acc_precision == 32)
    { k_kick<double, float><<<b, t, 0, s>>>((double*)mom, (const float*)acc, rung, rung_min, n, kf); ++ctx->launches; }
  else if (mom_precision == 64 && acc_precision == 64)
    { k_kick<double, double><<<b, t, 0, s>>>((double*)mom, (const double*)acc, rung, rung_min, n, kf); ++ctx->launches; }
  else if (mom_precision == 32 && acc_precision == 32)
    { k_kick<float, float><<<b, t, 0, s>>>((float*)mom, (const float*)acc, rung, rung_min, n, kf); ++ctx->launches; }
  else
    { k_kick<float, double><<<b, t, 0, s>>>((float*)mom, (const double*)acc, rung, rung_min, n, kf); ++ctx->launches; }
  return cuda_check(ctx, cudaGetLastError(), "kick kernel");
}

extern "C" p3m_status p3m_sr_drift(p3m_sr_ctx* ctx, double* pos, const void* mom, int mom_precision, double factor) {
  if (!ctx) return P3M_ERR_INVALID;
  if (mom_precision != 32 && mom_precision != 64) return fail(ctx, P3M_ERR_INVALID, "drift: bad precision");
  if (ctx->n > 0 && (!pos || !mom)) return fail(ctx, P3M_ERR_INVALID, "drift: null pointer");
  if (!std::isfinite(factor)) return fail(ctx, P3M_ERR_INVALID, "drift: factor must be finite");
  p3m_status st = poll_latched(ctx);
  if (st != P3M_OK) return st;
  if (ctx->n == 0) return P3M_OK;
  float* slot = drift_slot(ctx, pos);
  const int t = 256;
  const unsigned b = blocks_for(ctx->n, t);
  if (mom_precision == 64)
    { k_drift<double><<<b, t, 0, ctx->stream>>>(pos, (const double*)mom, ctx->n, factor, ctx->prm.box, slot);
      ++ctx->launches; }
  else
    { k_drift<float><<<b, t, 0, ctx->stream>>>(pos, (const float*)mom, ctx->n, factor, ctx->prm.box, slot);
      ++ctx->launches; }
  return cuda_check(ctx, cudaGetLastError(), "drift kernel");
}

static p3m_status rung_kick_impl(p3m_sr_ctx* ctx, void* mom, int mom_precision, const void* acc, int acc_precision,
                                 int8_t* rung, int8_t* kick_state, int rung_min, long long substep, double dt,
                                 double eta, double eps, int synchronize, double* pos, double drift_factor);

extern "C" p3m_status p3m_sr_rung_kick(p3m_sr_ctx* ctx, void* mom, int mom_precision, const void* acc,
                                       int acc_precision, int8_t* rung, int8_t* kick_state, int rung_min,
                                       long long substep, double dt, double eta, double eps, int synchronize) {
  return rung_kick_impl(ctx, mom, mom_precision, acc, acc_precision, rung, kick_state, rung_min, substep, dt, eta, eps,
                        synchronize, nullptr, 0.0);
}

extern "C" p3m_status p3m_sr_rung_kick_drift(p3m_sr_ctx* ctx, void* mom, int mom_precision, const void* acc,
                                             int acc_precision, int8_t* rung, int8_t* kick_state, int rung_min,
                                             long long substep, double dt, double eta, double eps, double* pos,
                                             double drift_factor) {
  if (!ctx) return P3M_ERR_INVALID;
  if (ctx->n > 0 && !pos) return fail(ctx, P3M_ERR_INVALID, "rung_kick_drift: null positions");
  if (!std::isfinite(drift_factor)) return fail(ctx, P3M_ERR_INVALID, "rung_kick_drift: drift_factor must be finite");
  return rung_kick_impl(ctx, mom, mom_precision, acc, acc_precision, rung, kick_state, rung_min, substep, dt, eta, eps,
                        0, pos, drift_factor);
}

static p3m_status rung_kick_impl(p3m_sr_ctx* ctx, void* mom, int mom_precision, const void* acc, int acc_precision,
                                 int8_t* rung, int8_t* kick_state, int rung_min, long long substep, double dt,
                                 double eta, double eps, int synchronize, double* pos, double drift_factor) {
  if (!ctx) return P3M_ERR_INVALID;
  if ((mom_precision != 32 && mom_precision != 64) || (acc_precision != 32 && acc_precision != 64))
    return fail(ctx, P3M_ERR_INVALID, "rung_kick: precision must be 32 or 64");
  if (ctx->n > 0 && (!mom || !acc || !rung || !kick_state)) return fail(ctx, P3M_ERR_INVALID, "rung_kick: null pointer");
  if (!(dt >= 0.0) || !(eta > 0.0) || !(eps > 0.0) || substep < 1)
    return fail(ctx, P3M_ERR_INVALID, "rung_kick: need dt >= 0, eta > 0, eps > 0, substep >= 1");
  const int log2_sub = ctx->prm.n_rung - 1;
  const long long period = 1LL << log2_sub;
  int tz = 0;
  while (tz < log2_sub && ((substep >> tz) & 1LL) == 0) ++tz;
  if (rung_min != log2_sub - tz) return fail(ctx, P3M_ERR_INVALID, "rung_kick: rung_min does not match the substep");
  if (synchronize && (substep % period) != 0)
    return fail(ctx, P3M_ERR_INVALID, "rung_kick: synchronisation only at the end of a global step");
  p3m_status st = poll_latched(ctx);
  if (st != P3M_OK) return st;
  if (ctx->n == 0) return P3M_OK;
  volatile double t1 = dt * dt;
  volatile double t2 = 2.0 * eta;
  volatile double t3 = t2 * eps;
  volatile double q = t1 / t3;
  const double qq = q * q;
  const int t = 256;
  const unsigned b = blocks_for(ctx->n, t);
  cudaStream_t s = ctx->stream;
  const int64_t n = ctx->n;
  const int nr = ctx->prm.n_rung;
  const int sy = synchronize ? 1 : 0;
  if (pos) {  // the kick, then the drift of every particle, in one pass
    float* slot = drift_slot(ctx, pos);
    const unsigned bd = (unsigned)std::min<int64_t>(b, (int64_t)ctx->num_sms * 8);
    const float qqf = rung_qqf(qq);
    const double L = ctx->prm.box;
    if (mom_precision == 64 && acc_precision == 32)
      k_rung_kick_drift<double, float><<<bd, t, 0, s>>>((double*)mom, (const float*)acc, rung, kick_state, n, rung_min,
                                                        substep, log2_sub, dt, qq, qqf, nr, ctx->err_dev, pos,
                                                        drift_factor, L, slot);
    else if (mom_precision == 64 && acc_precision == 64)
      k_rung_kick_drift<double, double><<<bd, t, 0, s>>>((double*)mom, (const double*)acc, rung, kick_state, n,
                                                         rung_min, substep, log2_sub, dt, qq, qqf, nr, ctx->err_dev,
                                                         pos, drift_factor, L, slot);
    else if (mom_precision == 32 && acc_precision == 32)
      k_rung_kick_drift<float, float><<<bd, t, 0, s>>>((float*)mom, (const float*)acc, rung, kick_state, n, rung_min,
                                                       substep, log2_sub, dt, qq, qqf, nr, ctx->err_dev, pos,
                                                       drift_factor, L, slot);
    else
      k_rung_kick_drift<float, double><<<bd, t, 0, s>>>((float*)mom, (const double*)acc, rung, kick_state, n, rung_min,
                                                        substep, log2_sub, dt, qq, qqf, nr, ctx->err_dev, pos,
                                                        drift_factor, L, slot);
    ++ctx->launches;
    if ((st = cuda_check(ctx, cudaGetLastError(), "rung kick-drift kernel")) != P3M_OK) return st;
    report_latched(ctx);
    return P3M_OK;
  }
  if (mom_precision == 64 && acc_precision == 32)
    k_rung_kick<double, float><<<b, t, 0, s>>>((double*)mom, (const float*)acc, rung, kick_state, n, rung_min, substep,
                                               log2_sub, dt, qq, rung_qqf(qq), nr, sy, ctx->err_dev);
  else if (mom_precision == 64 && acc_precision == 64)
    k_rung_kick<double, double><<<b, t, 0, s>>>((double*)mom, (const double*)acc, rung, kick_state, n, rung_min,
                                                substep, log2_sub, dt, qq, rung_qqf(qq), nr, sy, ctx->err_dev);
  else if (mom_precision == 32 && acc_precision == 32)
    k_rung_kick<float, float><<<b, t, 0, s>>>((float*)mom, (const float*)acc, rung, kick_state, n, rung_min, substep,
                                              log2_sub, dt, qq, rung_qqf(qq), nr, sy, ctx->err_dev);
  else
    k_rung_kick<float, double><<<b, t, 0, s>>>((float*)mom, (const double*)acc, rung, kick_state, n, rung_min,
                                               substep, log2_sub, dt, qq, rung_qqf(qq), nr, sy, ctx->err_dev);
  ++ctx->launches;
  if ((st = cuda_check(ctx, cudaGetLastError(), "rung kick kernel")) != P3M_OK) return st;
  report_latched(ctx);
  return P3M_OK;
}
