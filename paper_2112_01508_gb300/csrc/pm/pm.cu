// Long-range (particle-mesh) half of the P3M gravity on one GPU: the C ABI of
// include/p3m_pm.h (Section 2.1.2 Eq. pm_method; Section 2.1.3 Eq. p3m_gravity,
// upper half, with the long-range kernel exp(-x_s^2 k^2)/k^2).
//
// Pipeline per call, all on the context's stream:
//   k_assign   particles -> mesh with W_p (one thread per particle, atomics into
//              the padded in-place mesh; particles sorted by tile give locality)
//   cuFFT      real -> complex, in place
//   k_green    multiply by G(k) = deconvolution^2 x kernel x 4 pi G m / L_phi^4 / n_phi^3
//              (one warp per (k_x, k_y) row; per-dimension factors from tables)
//   cuFFT      complex -> real, in place
//   k_interp   D_pd and mesh -> particle interpolation fused: per dimension the
//              p_i interpolation weights and the p_d difference weights combine
//              into one 1-D stencil of p_i + p_d points, so a particle reads
//              3 p_i^2 (p_i + p_d) mesh values and no force mesh is stored.
#include <cuda_runtime.h>
#include <cufft.h>

#include <cmath>
#include <cstring>
#include <new>
#include <string>

#include "../../../include/p3m_pm.h"

namespace {

constexpr int kErrBadPosition = 1;

template <class T>
struct Cplx;
template <>
struct Cplx<float> {
  using type = cufftComplex;
};
template <>
struct Cplx<double> {
  using type = cufftDoubleComplex;
};

// Symmetric difference weights c_q, q = 1 .. p_d/2 (c_{-q} = -c_q, c_0 = 0), the
// values of Eqs. symmetric_diff_2 ... symmetric_diff_8.
struct DiffCoef {
  double c[5];  // c[1..4]
};

DiffCoef diff_coef(int p_d) {
  DiffCoef d{};
  switch (p_d) {
    case 2: d.c[1] = 1.0 / 2.0; break;
    case 4: d.c[1] = 8.0 / 12.0; d.c[2] = -1.0 / 12.0; break;
    case 6: d.c[1] = 45.0 / 60.0; d.c[2] = -9.0 / 60.0; d.c[3] = 1.0 / 60.0; break;
    default: d.c[1] = 672.0 / 840.0; d.c[2] = -168.0 / 840.0; d.c[3] = 32.0 / 840.0; d.c[4] = -3.0 / 840.0; break;
  }
  return d;
}

// W_p(t) of Eqs. W_NGP ... W_PCS at t = |x - x_m| / L_phi, for t inside the support
// of the cell it is evaluated on (NGP: the one cell, weight 1).
template <int P, class T>
__device__ __forceinline__ T weight(T t) {
  if (P == 1) return T(1);
  if (P == 2) return T(1) - t;
  if (P == 3) return t < T(0.5) ? T(0.75) - t * t : (T(2) * t - T(3)) * (T(2) * t - T(3)) * T(0.125);
  // P == 4
  if (t < T(1)) return (T(3) * t * t * t - T(6) * t * t + T(4)) * (T(1) / T(6));
  const T u = T(2) - t;
  return u * u * u * (T(1) / T(6));
}

// First mesh cell of the W_p stencil of coordinate x (s = x / L_phi - 1/2 in cell
// units) and the p weights.  Odd orders centre on the nearest cell floor(s + 1/2)
// (a particle exactly on a cell face goes to the upper cell); even orders start
// p/2 - 1 cells below floor(s).
template <int P, class T>
__device__ __forceinline__ long long stencil_1d(double s, T (&w)[P]) {
  const double c = (P & 1) ? floor(s + 0.5) : floor(s);
  constexpr int off = (P & 1) ? (P - 1) / 2 : P / 2 - 1;
  const long long first = (long long)c - off;
  // cell first + a lies at (a - off) - f from the particle, f = s - c (exact in FP64):
  // one FP64 subtraction per coordinate, the weights in T
  const T f = (T)(s - c);
#pragma unroll
  for (int a = 0; a < P; ++a) {
    const T d = (T)(a - off) - f;
    w[a] = weight<P, T>(d < T(0) ? -d : d);
  }
  return first;
}

// m mod n for -n <= m < 2n: every stencil index lies within 8 cells of the mesh
// (first cell >= -6, last <= n + 6), and n_phi >= 8.
__device__ __forceinline__ int wrap(long long m, long long n) {
  int r = (int)m;
  const int nn = (int)n;
  r += r < 0 ? nn : 0;
  r -= r >= nn ? nn : 0;
  return r;
}

__device__ __forceinline__ bool position_ok(double x, double box) { return x >= 0.0 && x < box; }

// rho[(X n + Y) pad + Z] += prod_d W_p for the p^3 cells of every particle.
template <int P, class T>
__global__ void k_assign(const double* __restrict__ pos, long long n, long long nphi, long long pad, double scale,
                         double box, T* __restrict__ rho, int* __restrict__ err) {
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    const double x = pos[i], y = pos[n + i], z = pos[2 * n + i];
    if (!(position_ok(x, box) && position_ok(y, box) && position_ok(z, box))) {
      atomicOr(err, kErrBadPosition);
      continue;
    }
    T wx[P], wy[P], wz[P];
    const long long fx = stencil_1d<P, T>(x * scale - 0.5, wx);
    const long long fy = stencil_1d<P, T>(y * scale - 0.5, wy);
    const long long fz = stencil_1d<P, T>(z * scale - 0.5, wz);
    int iz[P];
#pragma unroll
    for (int c = 0; c < P; ++c) iz[c] = wrap(fz + c, nphi);
#pragma unroll
    for (int a = 0; a < P; ++a) {
      const long long row_a = (long long)wrap(fx + a, nphi) * nphi;
#pragma unroll
      for (int b = 0; b < P; ++b) {
        const long long row = (row_a + wrap(fy + b, nphi)) * pad;
        const T wab = wx[a] * wy[b];
#pragma unroll
        for (int c = 0; c < P; ++c) atomicAdd(rho + row + iz[c], wab * wz[c]);
      }
    }
  }
}

// Multiply the half spectrum by G(k).  f[j] = sinc^(-2p)(L_phi k_j / 2) exp(-x_s^2 k_j^2) and
// k2[j] = k_j^2 for mesh index j (both even in k, so one table serves the full x, y
// and the half z index ranges); pref folds in 4 pi G m / L_phi^4 and 1 / n_phi^3.
template <class T>
__global__ void k_green(typename Cplx<T>::type* __restrict__ mesh, const T* __restrict__ f, const T* __restrict__ k2,
                        long long nphi, long long nz, T pref) {
  const int lane = threadIdx.x & 31;
  const long long warps = (long long)gridDim.x * (blockDim.x >> 5);
  for (long long row = (long long)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); row < nphi * nphi;
       row += warps) {
    const long long jx = row / nphi, jy = row - jx * nphi;
    const T fxy = f[jx] * f[jy] * pref;
    const T kxy = k2[jx] + k2[jy];
    typename Cplx<T>::type* r = mesh + row * nz;
    for (long long jz = lane; jz < nz; jz += 32) {
      const T kk = kxy + k2[jz];
      T g = kk > T(0) ? fxy * f[jz] / kk : T(0);
      typename Cplx<T>::type v = r[jz];
      v.x *= g;
      v.y *= g;
      r[jz] = v;
    }
  }
}

// a_i = sum over the stencil of W_p x D_pd phi, per dimension through one combined
// 1-D stencil e_j = sum_a w_a c_{j - H - a} (j = 0 .. P + PD - 1, H = PD / 2).
template <int P, int PD, class T>
__global__ void k_interp(const double* __restrict__ pos, long long n, long long nphi, long long pad, double scale,
                         double box, const T* __restrict__ phi, DiffCoef dc, T* __restrict__ acc, int accumulate,
                         int* __restrict__ err) {
  constexpr int H = PD / 2;
  constexpr int E = P + PD;
  T c[2 * H + 1];
#pragma unroll
  for (int q = -H; q <= H; ++q) c[q + H] = q == 0 ? T(0) : (q > 0 ? (T)dc.c[q] : -(T)dc.c[-q]);
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    const double x = pos[i], y = pos[n + i], z = pos[2 * n + i];
    T g[3] = {T(0), T(0), T(0)};
    if (position_ok(x, box) && position_ok(y, box) && position_ok(z, box)) {
      T w[3][P];
      long long first[3];
      first[0] = stencil_1d<P, T>(x * scale - 0.5, w[0]);
      first[1] = stencil_1d<P, T>(y * scale - 0.5, w[1]);
      first[2] = stencil_1d<P, T>(z * scale - 0.5, w[2]);
      // wrapped mesh indices of cells first - H ... first + P - 1 + H, and the combined stencils
      int idx[3][E];
      T e[3][E];
#pragma unroll
      for (int d = 0; d < 3; ++d) {
#pragma unroll
        for (int j = 0; j < E; ++j) {
          idx[d][j] = wrap(first[d] - H + j, nphi);
          T s = T(0);
#pragma unroll
          for (int a = 0; a < P; ++a) {
            const int q = j - H - a;
            if (q >= -H && q <= H) s += w[d][a] * c[q + H];
          }
          e[d][j] = s;
        }
      }
      // x: difference along x, weights along y and z
#pragma unroll
      for (int b = 0; b < P; ++b) {
#pragma unroll
        for (int cc = 0; cc < P; ++cc) {
          const T wyz = w[1][b] * w[2][cc];
          const long long yz = (long long)idx[1][b + H] * pad + idx[2][cc + H];
          T s = T(0);
#pragma unroll
          for (int j = 0; j < E; ++j) s += e[0][j] * __ldg(phi + (long long)idx[0][j] * nphi * pad + yz);
          g[0] += wyz * s;
        }
      }
      // y
#pragma unroll
      for (int a = 0; a < P; ++a) {
#pragma unroll
        for (int cc = 0; cc < P; ++cc) {
          const T wxz = w[0][a] * w[2][cc];
          const long long xz = (long long)idx[0][a + H] * nphi * pad + idx[2][cc + H];
          T s = T(0);
#pragma unroll
          for (int j = 0; j < E; ++j) s += e[1][j] * __ldg(phi + xz + (long long)idx[1][j] * pad);
          g[1] += wxz * s;
        }
      }
      // z (contiguous in memory)
#pragma unroll
      for (int a = 0; a < P; ++a) {
#pragma unroll
        for (int b = 0; b < P; ++b) {
          const T wxy = w[0][a] * w[1][b];
          const T* row = phi + ((long long)idx[0][a + H] * nphi + idx[1][b + H]) * pad;
          T s = T(0);
#pragma unroll
          for (int j = 0; j < E; ++j) s += e[2][j] * __ldg(row + idx[2][j]);
          g[2] += wxy * s;
        }
      }
    } else {
      atomicOr(err, kErrBadPosition);
    }
#pragma unroll
    for (int d = 0; d < 3; ++d) {
      T* o = acc + d * n + i;
      *o = accumulate ? *o + g[d] : g[d];
    }
  }
}

}  // namespace

struct p3m_pm_ctx {
  p3m_pm_params prm{};
  cudaStream_t stream = nullptr;
  int device = 0;
  int num_sms = 0;
  long long nphi = 0, pad = 0, nz = 0;
  size_t elem = 0;                 // bytes per real
  void* mesh = nullptr;            // nphi * nphi * pad reals (in-place FFT)
  void* f_tab = nullptr;           // nphi entries of the precision's type
  void* k2_tab = nullptr;
  void* work = nullptr;            // shared cuFFT work area
  size_t work_bytes = 0;
  cufftHandle fwd = 0, inv = 0;
  bool fwd_made = false, inv_made = false;
  DiffCoef dc{};
  double pref = 0.0;
  int* err_dev = nullptr;
  int* err_host = nullptr;
  cudaEvent_t ev[6] = {};
  bool timed = false;
  bool have_potential = false;
  long long launches = 0;
  std::string last_error;
};

namespace {

p3m_status pm_fail(p3m_pm_ctx* ctx, p3m_status st, const std::string& msg) {
  if (ctx) ctx->last_error = msg;
  return st;
}

p3m_status pm_cuda(p3m_pm_ctx* ctx, cudaError_t e, const char* what) {
  if (e == cudaSuccess) return P3M_OK;
  cudaGetLastError();
  return pm_fail(ctx, e == cudaErrorMemoryAllocation ? P3M_ERR_OOM : P3M_ERR_CUDA,
                 std::string(what) + ": " + cudaGetErrorString(e));
}

p3m_status pm_cufft(p3m_pm_ctx* ctx, cufftResult r, const char* what) {
  if (r == CUFFT_SUCCESS) return P3M_OK;
  return pm_fail(ctx, r == CUFFT_ALLOC_FAILED ? P3M_ERR_OOM : P3M_ERR_CUDA,
                 std::string(what) + ": cuFFT error " + std::to_string((int)r));
}

p3m_status validate(p3m_pm_ctx* ctx, const p3m_pm_params& p) {
  if (p.n < 0 || p.n > (1LL << 40)) return pm_fail(ctx, P3M_ERR_INVALID, "n out of range");
  if (!(p.box > 0.0) || !std::isfinite(p.box)) return pm_fail(ctx, P3M_ERR_INVALID, "box must be positive");
  if (p.n_phi < 8 || p.n_phi > 4096 || (p.n_phi & 1))
    return pm_fail(ctx, P3M_ERR_INVALID, "n_phi must be even and in 8..4096");
  if (!(p.x_s >= 0.0) || !std::isfinite(p.x_s)) return pm_fail(ctx, P3M_ERR_INVALID, "x_s must be >= 0");
  if (!std::isfinite(p.G_m)) return pm_fail(ctx, P3M_ERR_INVALID, "G_m must be finite");
  if (p.p_i < 1 || p.p_i > 4) return pm_fail(ctx, P3M_ERR_INVALID, "p_i must be 1..4");
  if (p.p_d != 2 && p.p_d != 4 && p.p_d != 6 && p.p_d != 8)
    return pm_fail(ctx, P3M_ERR_INVALID, "p_d must be 2, 4, 6 or 8");
  if (p.precision != 32 && p.precision != 64) return pm_fail(ctx, P3M_ERR_INVALID, "precision must be 32 or 64");
  return P3M_OK;
}

// Per-dimension factors of G(k), in double on the host: k_j = 2 pi h / L with h = j
// (j <= n/2) or j - n; f = sinc^(-2 p_i)(L_phi k / 2) exp(-x_s^2 k^2).
template <class T>
p3m_status upload_tables(p3m_pm_ctx* ctx) {
  const long long n = ctx->nphi;
  T* f = new (std::nothrow) T[n];
  T* k2 = new (std::nothrow) T[n];
  if (!f || !k2) {
    delete[] f;
    delete[] k2;
    return pm_fail(ctx, P3M_ERR_OOM, "host tables");
  }
  const double pi = 3.14159265358979323846;
  const double L = ctx->prm.box, L_phi = L / (double)n;
  for (long long j = 0; j < n; ++j) {
    const double h = (double)(j <= n / 2 ? j : j - n);
    const double k = 2.0 * pi * h / L;
    const double t = 0.5 * L_phi * k;
    const double sinc = (t == 0.0) ? 1.0 : std::sin(t) / t;
    f[j] = (T)(std::pow(sinc, -2.0 * ctx->prm.p_i) * std::exp(-ctx->prm.x_s * ctx->prm.x_s * k * k));
    k2[j] = (T)(k * k);
  }
  p3m_status st = pm_cuda(ctx, cudaMemcpy(ctx->f_tab, f, sizeof(T) * n, cudaMemcpyHostToDevice), "table upload");
  if (st == P3M_OK)
    st = pm_cuda(ctx, cudaMemcpy(ctx->k2_tab, k2, sizeof(T) * n, cudaMemcpyHostToDevice), "table upload");
  delete[] f;
  delete[] k2;
  return st;
}

template <class T>
p3m_status launch_assign(p3m_pm_ctx* ctx, const double* pos, T* rho, long long pad) {
  const long long n = ctx->prm.n;
  if (n == 0) return P3M_OK;
  const double scale = (double)ctx->nphi / ctx->prm.box;
  const int threads = 256;
  long long blocks = (n + threads - 1) / threads;
  if (blocks > (long long)ctx->num_sms * 64) blocks = (long long)ctx->num_sms * 64;
  const unsigned b = (unsigned)(blocks > 0 ? blocks : 1);
  switch (ctx->prm.p_i) {
    case 1: k_assign<1, T><<<b, threads, 0, ctx->stream>>>(pos, n, ctx->nphi, pad, scale, ctx->prm.box, rho, ctx->err_dev); break;
    case 2: k_assign<2, T><<<b, threads, 0, ctx->stream>>>(pos, n, ctx->nphi, pad, scale, ctx->prm.box, rho, ctx->err_dev); break;
    case 3: k_assign<3, T><<<b, threads, 0, ctx->stream>>>(pos, n, ctx->nphi, pad, scale, ctx->prm.box, rho, ctx->err_dev); break;
    default: k_assign<4, T><<<b, threads, 0, ctx->stream>>>(pos, n, ctx->nphi, pad, scale, ctx->prm.box, rho, ctx->err_dev); break;
  }
  ++ctx->launches;
  return pm_cuda(ctx, cudaGetLastError(), "assign kernel");
}

template <int P, class T>
void interp_pd(p3m_pm_ctx* ctx, unsigned b, const double* pos, T* acc, int accumulate) {
  const long long n = ctx->prm.n;
  const double scale = (double)ctx->nphi / ctx->prm.box;
  const T* phi = (const T*)ctx->mesh;
  switch (ctx->prm.p_d) {
    case 2: k_interp<P, 2, T><<<b, 256, 0, ctx->stream>>>(pos, n, ctx->nphi, ctx->pad, scale, ctx->prm.box, phi, ctx->dc, acc, accumulate, ctx->err_dev); break;
    case 4: k_interp<P, 4, T><<<b, 256, 0, ctx->stream>>>(pos, n, ctx->nphi, ctx->pad, scale, ctx->prm.box, phi, ctx->dc, acc, accumulate, ctx->err_dev); break;
    case 6: k_interp<P, 6, T><<<b, 256, 0, ctx->stream>>>(pos, n, ctx->nphi, ctx->pad, scale, ctx->prm.box, phi, ctx->dc, acc, accumulate, ctx->err_dev); break;
    default: k_interp<P, 8, T><<<b, 256, 0, ctx->stream>>>(pos, n, ctx->nphi, ctx->pad, scale, ctx->prm.box, phi, ctx->dc, acc, accumulate, ctx->err_dev); break;
  }
}

template <class T>
p3m_status run_accel(p3m_pm_ctx* ctx, const double* pos, T* acc, int accumulate) {
  cudaStream_t s = ctx->stream;
  p3m_status st;
  const size_t mesh_bytes = (size_t)ctx->nphi * ctx->nphi * ctx->pad * sizeof(T);
  cudaEventRecord(ctx->ev[0], s);
  if ((st = pm_cuda(ctx, cudaMemsetAsync(ctx->mesh, 0, mesh_bytes, s), "mesh clear")) != P3M_OK) return st;
  if ((st = launch_assign<T>(ctx, pos, (T*)ctx->mesh, ctx->pad)) != P3M_OK) return st;
  cudaEventRecord(ctx->ev[1], s);
  if (sizeof(T) == 4)
    st = pm_cufft(ctx, cufftExecR2C(ctx->fwd, (cufftReal*)ctx->mesh, (cufftComplex*)ctx->mesh), "forward FFT");
  else
    st = pm_cufft(ctx, cufftExecD2Z(ctx->fwd, (cufftDoubleReal*)ctx->mesh, (cufftDoubleComplex*)ctx->mesh),
                  "forward FFT");
  if (st != P3M_OK) return st;
  cudaEventRecord(ctx->ev[2], s);
  {
    const long long rows = ctx->nphi * ctx->nphi;
    long long blocks = (rows + 7) / 8;
    if (blocks > (long long)ctx->num_sms * 32) blocks = (long long)ctx->num_sms * 32;
    k_green<T><<<(unsigned)blocks, 256, 0, s>>>((typename Cplx<T>::type*)ctx->mesh, (const T*)ctx->f_tab,
                                                 (const T*)ctx->k2_tab, ctx->nphi, ctx->nz, (T)ctx->pref);
    ++ctx->launches;
    if ((st = pm_cuda(ctx, cudaGetLastError(), "green kernel")) != P3M_OK) return st;
  }
  cudaEventRecord(ctx->ev[3], s);
  if (sizeof(T) == 4)
    st = pm_cufft(ctx, cufftExecC2R(ctx->inv, (cufftComplex*)ctx->mesh, (cufftReal*)ctx->mesh), "inverse FFT");
  else
    st = pm_cufft(ctx, cufftExecZ2D(ctx->inv, (cufftDoubleComplex*)ctx->mesh, (cufftDoubleReal*)ctx->mesh),
                  "inverse FFT");
  if (st != P3M_OK) return st;
  cudaEventRecord(ctx->ev[4], s);
  const long long n = ctx->prm.n;
  if (n > 0) {
    long long blocks = (n + 255) / 256;
    if (blocks > (long long)ctx->num_sms * 64) blocks = (long long)ctx->num_sms * 64;
    const unsigned b = (unsigned)blocks;
    switch (ctx->prm.p_i) {
      case 1: interp_pd<1, T>(ctx, b, pos, acc, accumulate); break;
      case 2: interp_pd<2, T>(ctx, b, pos, acc, accumulate); break;
      case 3: interp_pd<3, T>(ctx, b, pos, acc, accumulate); break;
      default: interp_pd<4, T>(ctx, b, pos, acc, accumulate); break;
    }
    ++ctx->launches;
    if ((st = pm_cuda(ctx, cudaGetLastError(), "interpolation kernel")) != P3M_OK) return st;
  }
  cudaEventRecord(ctx->ev[5], s);
  ctx->timed = true;
  ctx->have_potential = true;
  return P3M_OK;
}

}  // namespace

extern "C" p3m_status p3m_pm_create(const p3m_pm_params* params, void* cuda_stream, p3m_pm_ctx** out) {
  if (!out) return P3M_ERR_INVALID;
  *out = nullptr;
  if (!params) return P3M_ERR_INVALID;
  p3m_pm_ctx* ctx = new (std::nothrow) p3m_pm_ctx();
  if (!ctx) return P3M_ERR_OOM;
  p3m_status st = validate(ctx, *params);
  if (st != P3M_OK) {
    delete ctx;
    return st;
  }
  ctx->prm = *params;
  ctx->stream = (cudaStream_t)cuda_stream;
  ctx->nphi = params->n_phi;
  ctx->nz = ctx->nphi / 2 + 1;
  ctx->pad = 2 * ctx->nz;
  ctx->elem = params->precision == 32 ? sizeof(float) : sizeof(double);
  ctx->dc = diff_coef(params->p_d);
  {
    const double pi = 3.14159265358979323846;
    const double L_phi = params->box / (double)params->n_phi;
    const double n3 = (double)ctx->nphi * (double)ctx->nphi * (double)ctx->nphi;
    ctx->pref = 4.0 * pi * params->G_m / (L_phi * L_phi * L_phi * L_phi) / n3;
  }
  cudaGetDevice(&ctx->device);
  cudaDeviceGetAttribute(&ctx->num_sms, cudaDevAttrMultiProcessorCount, ctx->device);
  if (ctx->num_sms <= 0) ctx->num_sms = 1;
  const size_t mesh_bytes = (size_t)ctx->nphi * ctx->nphi * ctx->pad * ctx->elem;
  cufftType tf = params->precision == 32 ? CUFFT_R2C : CUFFT_D2Z;
  cufftType ti = params->precision == 32 ? CUFFT_C2R : CUFFT_Z2D;
  long long dims[3] = {ctx->nphi, ctx->nphi, ctx->nphi};
  size_t wf = 0, wi = 0;
  if ((st = pm_cuda(ctx, cudaMalloc(&ctx->mesh, mesh_bytes), "mesh")) != P3M_OK) goto fail;
  if ((st = pm_cuda(ctx, cudaMalloc(&ctx->f_tab, ctx->nphi * ctx->elem), "tables")) != P3M_OK) goto fail;
  if ((st = pm_cuda(ctx, cudaMalloc(&ctx->k2_tab, ctx->nphi * ctx->elem), "tables")) != P3M_OK) goto fail;
  if ((st = pm_cuda(ctx, cudaMalloc((void**)&ctx->err_dev, sizeof(int)), "error word")) != P3M_OK) goto fail;
  if ((st = pm_cuda(ctx, cudaMemset(ctx->err_dev, 0, sizeof(int)), "error word")) != P3M_OK) goto fail;
  if ((st = pm_cuda(ctx, cudaMallocHost((void**)&ctx->err_host, sizeof(int)), "error mirror")) != P3M_OK) goto fail;
  *ctx->err_host = 0;
  for (int k = 0; k < 6; ++k)
    if ((st = pm_cuda(ctx, cudaEventCreate(&ctx->ev[k]), "event")) != P3M_OK) goto fail;
  st = params->precision == 32 ? upload_tables<float>(ctx) : upload_tables<double>(ctx);
  if (st != P3M_OK) goto fail;
  // plans with one shared work area
  if ((st = pm_cufft(ctx, cufftCreate(&ctx->fwd), "plan")) != P3M_OK) goto fail;
  ctx->fwd_made = true;
  if ((st = pm_cufft(ctx, cufftCreate(&ctx->inv), "plan")) != P3M_OK) goto fail;
  ctx->inv_made = true;
  cufftSetAutoAllocation(ctx->fwd, 0);
  cufftSetAutoAllocation(ctx->inv, 0);
  if ((st = pm_cufft(ctx, cufftMakePlanMany64(ctx->fwd, 3, dims, nullptr, 1, 0, nullptr, 1, 0, tf, 1, &wf),
                     "forward plan")) != P3M_OK)
    goto fail;
  if ((st = pm_cufft(ctx, cufftMakePlanMany64(ctx->inv, 3, dims, nullptr, 1, 0, nullptr, 1, 0, ti, 1, &wi),
                     "inverse plan")) != P3M_OK)
    goto fail;
  ctx->work_bytes = wf > wi ? wf : wi;
  if (ctx->work_bytes > 0 &&
      (st = pm_cuda(ctx, cudaMalloc(&ctx->work, ctx->work_bytes), "FFT work area")) != P3M_OK)
    goto fail;
  if ((st = pm_cufft(ctx, cufftSetWorkArea(ctx->fwd, ctx->work), "work area")) != P3M_OK) goto fail;
  if ((st = pm_cufft(ctx, cufftSetWorkArea(ctx->inv, ctx->work), "work area")) != P3M_OK) goto fail;
  if ((st = pm_cufft(ctx, cufftSetStream(ctx->fwd, ctx->stream), "stream")) != P3M_OK) goto fail;
  if ((st = pm_cufft(ctx, cufftSetStream(ctx->inv, ctx->stream), "stream")) != P3M_OK) goto fail;
  *out = ctx;
  return P3M_OK;
fail:
  p3m_pm_destroy(ctx);
  return st;
}

extern "C" void p3m_pm_destroy(p3m_pm_ctx* ctx) {
  if (!ctx) return;
  if (ctx->stream || ctx->mesh) cudaStreamSynchronize(ctx->stream);
  if (ctx->fwd_made) cufftDestroy(ctx->fwd);
  if (ctx->inv_made) cufftDestroy(ctx->inv);
  cudaFree(ctx->work);
  cudaFree(ctx->mesh);
  cudaFree(ctx->f_tab);
  cudaFree(ctx->k2_tab);
  cudaFree(ctx->err_dev);
  if (ctx->err_host) cudaFreeHost(ctx->err_host);
  for (int k = 0; k < 6; ++k)
    if (ctx->ev[k]) cudaEventDestroy(ctx->ev[k]);
  cudaGetLastError();
  delete ctx;
}

extern "C" const char* p3m_pm_last_error(const p3m_pm_ctx* ctx) {
  if (!ctx) return "null context";
  return ctx->last_error.c_str();
}

extern "C" p3m_status p3m_pm_sync(p3m_pm_ctx* ctx) {
  if (!ctx) return P3M_ERR_INVALID;
  p3m_status st = pm_cuda(ctx, cudaStreamSynchronize(ctx->stream), "stream synchronize");
  if (st != P3M_OK) return st;
  if ((st = pm_cuda(ctx, cudaMemcpy(ctx->err_host, ctx->err_dev, sizeof(int), cudaMemcpyDeviceToHost),
                    "error word")) != P3M_OK)
    return st;
  if (*ctx->err_host) {
    *ctx->err_host = 0;
    cudaMemset(ctx->err_dev, 0, sizeof(int));
    return pm_fail(ctx, P3M_ERR_NONFINITE, "a position was non-finite or outside [0, L)");
  }
  return P3M_OK;
}

extern "C" p3m_status p3m_pm_stats(p3m_pm_ctx* ctx, p3m_pm_stats_t* out) {
  if (!ctx || !out) return P3M_ERR_INVALID;
  p3m_status st = p3m_pm_sync(ctx);
  std::memset(out, 0, sizeof(*out));
  out->n_phi = (int)ctx->nphi;
  out->mesh_bytes = (int64_t)(ctx->nphi * ctx->nphi * ctx->pad * (long long)ctx->elem);
  out->fft_work_bytes = (int64_t)ctx->work_bytes;
  out->kernel_launches = ctx->launches;
  if (ctx->timed) {
    float ms[5] = {0, 0, 0, 0, 0};
    for (int k = 0; k < 5; ++k) cudaEventElapsedTime(&ms[k], ctx->ev[k], ctx->ev[k + 1]);
    out->assign_ms = ms[0];
    out->fft_ms = ms[1];
    out->kernel_ms = ms[2];
    out->ifft_ms = ms[3];
    out->interp_ms = ms[4];
  }
  return st;
}

extern "C" p3m_status p3m_pm_accel(p3m_pm_ctx* ctx, const double* pos, void* acc, int accumulate) {
  if (!ctx) return P3M_ERR_INVALID;
  if (ctx->prm.n > 0 && (!pos || !acc)) return pm_fail(ctx, P3M_ERR_INVALID, "accel: null pointer");
  if (ctx->prm.precision == 32) return run_accel<float>(ctx, pos, (float*)acc, accumulate ? 1 : 0);
  return run_accel<double>(ctx, pos, (double*)acc, accumulate ? 1 : 0);
}

extern "C" p3m_status p3m_pm_assign(p3m_pm_ctx* ctx, const double* pos, void* rho_out) {
  if (!ctx) return P3M_ERR_INVALID;
  if (!rho_out || (ctx->prm.n > 0 && !pos)) return pm_fail(ctx, P3M_ERR_INVALID, "assign: null pointer");
  const size_t bytes = (size_t)ctx->nphi * ctx->nphi * ctx->nphi * ctx->elem;
  p3m_status st = pm_cuda(ctx, cudaMemsetAsync(rho_out, 0, bytes, ctx->stream), "clear");
  if (st != P3M_OK) return st;
  if (ctx->prm.precision == 32) return launch_assign<float>(ctx, pos, (float*)rho_out, ctx->nphi);
  return launch_assign<double>(ctx, pos, (double*)rho_out, ctx->nphi);
}

extern "C" p3m_status p3m_pm_potential(p3m_pm_ctx* ctx, void* phi_out) {
  if (!ctx) return P3M_ERR_INVALID;
  if (!phi_out) return pm_fail(ctx, P3M_ERR_INVALID, "potential: null pointer");
  if (!ctx->have_potential) return pm_fail(ctx, P3M_ERR_STATE, "potential: call p3m_pm_accel first");
  const size_t row = (size_t)ctx->nphi * ctx->elem;
  return pm_cuda(ctx, cudaMemcpy2DAsync(phi_out, row, ctx->mesh, (size_t)ctx->pad * ctx->elem, row,
                                        (size_t)(ctx->nphi * ctx->nphi), cudaMemcpyDeviceToDevice, ctx->stream),
                 "potential copy");
}
