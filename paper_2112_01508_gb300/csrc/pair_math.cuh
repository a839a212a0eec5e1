// The short-range pair bracket B(r) of Eq. p3m_gravity (Section 2.1.3) and its
// derivative, in FP32 (fast path) and FP64 (parity path).
//
//   B(r) = erfc(u)/r^3 + exp(-u^2)/(sqrt(pi) x_s r^2) + ( |x|^{-3}_shape - r^{-3} ),
//   u = r / (2 x_s).
//
// Main branch (r >= r_sw): B r^3 = exp(-u^2) [erfcx(u) + 2u/sqrt(pi)], i.e.
//   B = exp(-u^2) r^{-2} [erfcx(u) r^{-1} + 1/(sqrt(pi) x_s)],
// with exp(-u^2) from one ex2 and erfcx from the fit of fit_erfcx.py.
// Softened branch (r < r_sw, rare): the exact identity
//   erfc(u) + 2u/sqrt(pi) e^{-u^2} - 1 = -u^3 h(u),  h(u) = [erf u - 2u/sqrt(pi) e^{-u^2}] / u^3,
// gives B = |x|^{-3}_shape - h(u) / (2 x_s)^3 without the cancellation of
// erfc(u)/r^3 against -r^{-3}; h is its Taylor series in u^2.
// Shapes (Section 2.1.1): Plummer (r^2+eps^2)^{-3/2} (Eq. plummer_shape) and
// the B-spline piecewise polynomial of Eq. bspline_force (eps_B = 2.8 eps).
#pragma once

#include "common.cuh"

namespace p3m {

constexpr int kHTermsF = 8;
constexpr int kHTermsD = 18;

// Series coefficients of h(u) = sum_n H_n u^{2n} and h'(u)/u = sum_n Hd_n u^{2n}.
struct SeriesConsts {
  float h_f[kHTermsF], hd_f[kHTermsF];
  double h_d[kHTermsD], hd_d[kHTermsD];
};

__device__ __forceinline__ float ex2_approx(float x) {
  float y;
  asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}
__device__ __forceinline__ float rsqrt_approx(float x) {
  float y;
  asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}
__device__ __forceinline__ float rcp_approx(float x) {
  float y;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}

// Packed pairs of floats (sm_100+ f32x2 arithmetic): one instruction issues
// two FP32 lanes' worth of work, halving the issue slots of the FP32 chain.
struct f2 {
  unsigned long long v;
};
__device__ __forceinline__ f2 pk(float lo, float hi) {
  f2 r;
  asm("mov.b64 %0, {%1, %2};" : "=l"(r.v) : "f"(lo), "f"(hi));
  return r;
}
__device__ __forceinline__ void upk(f2 a, float& lo, float& hi) {
  asm("mov.b64 {%0, %1}, %2;" : "=f"(lo), "=f"(hi) : "l"(a.v));
}
__device__ __forceinline__ f2 fma2(f2 a, f2 b, f2 c) {
  f2 r;
  asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(r.v) : "l"(a.v), "l"(b.v), "l"(c.v));
  return r;
}
__device__ __forceinline__ f2 mul2(f2 a, f2 b) {
  f2 r;
  asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(r.v) : "l"(a.v), "l"(b.v));
  return r;
}
__device__ __forceinline__ f2 add2(f2 a, f2 b) {
  f2 r;
  asm("add.rn.f32x2 %0, %1, %2;" : "=l"(r.v) : "l"(a.v), "l"(b.v));
  return r;
}

// ---------------------------------------------------------------- FP32 ----

// Main branch.  Returns B; with VJP also D = B'(r)/r.
template <int SOFT, bool VJP>
__device__ __forceinline__ float bracket_main_f32(float r2, const ForceConsts& f, float& D) {
  float rinv = rsqrt_approx(r2);
  float r = r2 * rinv;
  float e = ex2_approx(r2 * f.ce_f);
  float t = rcp_approx(fmaf(r, f.kc_f, 1.0f));
  float q = fmaf(f.c_f[5], t, f.c_f[4]);
  q = fmaf(q, t, f.c_f[3]);
  q = fmaf(q, t, f.c_f[2]);
  q = fmaf(q, t, f.c_f[1]);
  q = fmaf(q, t, f.c_f[0]);
  float ex = q * t;  // erfcx(u)
  float rinv2 = rinv * rinv;
  float er2 = e * rinv2;
  float B = er2 * fmaf(ex, rinv, f.k2_f);
  if (VJP) {
    // g'(r)/r = -r^{-2} (3 g + exp(-u^2) / (2 sqrt(pi) x_s^3))
    D = -rinv2 * fmaf(3.0f, B, e * f.k3_f);
  }
  if (SOFT == P3M_SOFT_PLUMMER) {
    float p = rsqrt_approx(r2 + f.eps2_f);
    float p3 = p * p * p;
    float rinv3 = rinv2 * rinv;
    if (VJP) D += 3.0f * (rinv3 * rinv2 - p3 * p * p);
    B += p3 - rinv3;
  }
  return B;
}

// Main branch for two pairs at once (forward only): the FP32 chain of
// bracket_main_f32 in packed f32x2 form; the SFU operations stay scalar.
template <int SOFT>
__device__ __forceinline__ f2 bracket_main_f32x2(f2 r2, const ForceConsts& f) {
  float a, b;
  upk(r2, a, b);
  const f2 rinv = pk(rsqrt_approx(a), rsqrt_approx(b));
  const f2 r = mul2(r2, rinv);
  float ea, eb;
  upk(mul2(r2, pk(f.ce_f, f.ce_f)), ea, eb);
  const f2 e = pk(ex2_approx(ea), ex2_approx(eb));
  float da, db;
  upk(fma2(r, pk(f.kc_f, f.kc_f), pk(1.0f, 1.0f)), da, db);
  const f2 t = pk(rcp_approx(da), rcp_approx(db));
  f2 q = fma2(pk(f.c_f[5], f.c_f[5]), t, pk(f.c_f[4], f.c_f[4]));
  q = fma2(q, t, pk(f.c_f[3], f.c_f[3]));
  q = fma2(q, t, pk(f.c_f[2], f.c_f[2]));
  q = fma2(q, t, pk(f.c_f[1], f.c_f[1]));
  q = fma2(q, t, pk(f.c_f[0], f.c_f[0]));
  const f2 ex = mul2(q, t);
  const f2 rinv2 = mul2(rinv, rinv);
  const f2 er2 = mul2(e, rinv2);
  f2 B = mul2(er2, fma2(ex, rinv, pk(f.k2_f, f.k2_f)));
  if (SOFT == P3M_SOFT_PLUMMER) {
    float pa, pb;
    upk(add2(r2, pk(f.eps2_f, f.eps2_f)), pa, pb);
    const f2 p = pk(rsqrt_approx(pa), rsqrt_approx(pb));
    const f2 p3 = mul2(mul2(p, p), p);
    const f2 rinv3 = mul2(rinv2, rinv);
    B = add2(B, fma2(rinv3, pk(-1.0f, -1.0f), p3));
  }
  return B;
}

// Main branch for two pairs with the derivative (adjoint): returns B and sets
// D = B'(r)/r for both halves.
template <int SOFT>
__device__ __forceinline__ f2 bracket_main_vjp_f32x2(f2 r2, const ForceConsts& f, f2& D) {
  float a, b;
  upk(r2, a, b);
  const f2 rinv = pk(rsqrt_approx(a), rsqrt_approx(b));
  const f2 r = mul2(r2, rinv);
  float ea, eb;
  upk(mul2(r2, pk(f.ce_f, f.ce_f)), ea, eb);
  const f2 e = pk(ex2_approx(ea), ex2_approx(eb));
  float da, db;
  upk(fma2(r, pk(f.kc_f, f.kc_f), pk(1.0f, 1.0f)), da, db);
  const f2 t = pk(rcp_approx(da), rcp_approx(db));
  f2 q = fma2(pk(f.c_f[5], f.c_f[5]), t, pk(f.c_f[4], f.c_f[4]));
  q = fma2(q, t, pk(f.c_f[3], f.c_f[3]));
  q = fma2(q, t, pk(f.c_f[2], f.c_f[2]));
  q = fma2(q, t, pk(f.c_f[1], f.c_f[1]));
  q = fma2(q, t, pk(f.c_f[0], f.c_f[0]));
  const f2 ex = mul2(q, t);
  const f2 rinv2 = mul2(rinv, rinv);
  const f2 er2 = mul2(e, rinv2);
  f2 B = mul2(er2, fma2(ex, rinv, pk(f.k2_f, f.k2_f)));
  // g'(r)/r = -r^{-2} (3 g + exp(-u^2) k3)
  D = mul2(mul2(rinv2, pk(-1.0f, -1.0f)), fma2(pk(3.0f, 3.0f), B, mul2(e, pk(f.k3_f, f.k3_f))));
  if (SOFT == P3M_SOFT_PLUMMER) {
    float pa, pb;
    upk(add2(r2, pk(f.eps2_f, f.eps2_f)), pa, pb);
    const f2 p = pk(rsqrt_approx(pa), rsqrt_approx(pb));
    const f2 p2 = mul2(p, p);
    const f2 p3 = mul2(p2, p);
    const f2 rinv3 = mul2(rinv2, rinv);
    // D += 3 (r^-5 - p^5),  B += p^3 - r^-3
    D = fma2(pk(3.0f, 3.0f), fma2(rinv3, rinv2, mul2(mul2(p3, p2), pk(-1.0f, -1.0f))), D);
    B = add2(B, fma2(rinv3, pk(-1.0f, -1.0f), p3));
  }
  return B;
}

// Softened branch, r^2 < r_sw^2 (and r = 0 for point particles).
template <int SOFT, bool VJP>
__device__ __forceinline__ float bracket_soft_f32(float r2, const ForceConsts& f, const SeriesConsts& sc,
                                                  float& D) {
  if (SOFT == P3M_SOFT_NONE) {  // only coincident particles arrive here: zero by convention
    D = 0.0f;
    return 0.0f;
  }
  float r = sqrtf(r2);
  float u = r * f.inv2xs_f;
  float u2 = u * u;
  float h = sc.h_f[kHTermsF - 1];
#pragma unroll
  for (int k = kHTermsF - 2; k >= 0; --k) h = fmaf(h, u2, sc.h_f[k]);
  float s3, ds;  // |x|^{-3}_shape and its r-derivative divided by r
  if (SOFT == P3M_SOFT_BSPLINE) {
    float x = r * f.inv_epsb_f;
    float c = f.bnorm_f;
    float ce = c * f.inv_epsb_f * f.inv_epsb_f;  // 32 / eps_B^5
    if (x < 0.5f) {
      s3 = c * fmaf(x * x, x - 1.2f, 1.0f / 3.0f);
      ds = ce * fmaf(3.0f, x, -2.4f);
    } else {
      float xi = 1.0f / x;
      float xi3 = xi * xi * xi;
      s3 = c * (fmaf(x * x, fmaf(-1.0f / 3.0f, x, 1.2f), fmaf(-1.5f, x, 2.0f / 3.0f)) - xi3 * (1.0f / 480.0f));
      ds = ce * (fmaf(-1.0f, x, 2.4f) - 1.5f * xi + xi3 * xi * xi * (1.0f / 160.0f));
    }
  } else {  // Plummer
    float p = rsqrt_approx(r2 + f.eps2_f);
    s3 = p * p * p;
    ds = -3.0f * s3 * p * p;
  }
  if (VJP) {
    float hd = sc.hd_f[kHTermsF - 1];
#pragma unroll
    for (int k = kHTermsF - 2; k >= 0; --k) hd = fmaf(hd, u2, sc.hd_f[k]);
    // d/dr [h(u)/(2x_s)^3] / r = h'(u)/u / (2x_s)^5
    D = ds - hd * f.hscale_f * f.inv2xs_f * f.inv2xs_f;
  }
  return s3 - h * f.hscale_f;
}

// Softened branch for two pairs at once (forward only): both B-spline pieces are
// evaluated and the piece of each half selected, so a warp whose close pairs sit
// in either half pays one packed evaluation.  r comes from r^2 times its
// reciprocal square root (r^2 > 0 here: a zero displacement never takes this
// branch), and the outer piece's 1/x from the approximate reciprocal.  A half
// that is not a close pair may overflow; the caller discards it.
template <int SOFT>
__device__ __forceinline__ f2 bracket_soft_f32x2(f2 r2, const ForceConsts& f, const SeriesConsts& sc) {
  if (SOFT == P3M_SOFT_NONE) return pk(0.0f, 0.0f);
  float a, b;
  upk(r2, a, b);
  const f2 r = mul2(r2, pk(rsqrt_approx(a), rsqrt_approx(b)));
  const f2 u = mul2(r, pk(f.inv2xs_f, f.inv2xs_f));
  const f2 u2 = mul2(u, u);
  f2 h = pk(sc.h_f[kHTermsF - 1], sc.h_f[kHTermsF - 1]);
#pragma unroll
  for (int k = kHTermsF - 2; k >= 0; --k) h = fma2(h, u2, pk(sc.h_f[k], sc.h_f[k]));
  f2 s3;
  if (SOFT == P3M_SOFT_BSPLINE) {
    const f2 x = mul2(r, pk(f.inv_epsb_f, f.inv_epsb_f));
    const f2 x2 = mul2(x, x);
    const f2 c = pk(f.bnorm_f, f.bnorm_f);
    // x < 1/2: c (x^2 (x - 6/5) + 1/3)
    const f2 s_in = mul2(c, fma2(x2, add2(x, pk(-1.2f, -1.2f)), pk(1.0f / 3.0f, 1.0f / 3.0f)));
    // 1/2 <= x < 1: c (x^2 (6/5 - x/3) + 2/3 - 3x/2 - x^-3 / 480)
    float xa, xb;
    upk(x, xa, xb);
    const f2 xi = pk(rcp_approx(xa), rcp_approx(xb));
    const f2 xi3 = mul2(mul2(xi, xi), xi);
    const f2 poly = fma2(x2, fma2(pk(-1.0f / 3.0f, -1.0f / 3.0f), x, pk(1.2f, 1.2f)),
                         fma2(pk(-1.5f, -1.5f), x, pk(2.0f / 3.0f, 2.0f / 3.0f)));
    const f2 s_out = mul2(c, fma2(xi3, pk(-1.0f / 480.0f, -1.0f / 480.0f), poly));
    float ia, ib, oa, ob;
    upk(s_in, ia, ib);
    upk(s_out, oa, ob);
    s3 = pk(xa < 0.5f ? ia : oa, xb < 0.5f ? ib : ob);
  } else {  // Plummer
    float pa, pb;
    upk(add2(r2, pk(f.eps2_f, f.eps2_f)), pa, pb);
    const f2 p = pk(rsqrt_approx(pa), rsqrt_approx(pb));
    s3 = mul2(mul2(p, p), p);
  }
  return fma2(h, pk(-f.hscale_f, -f.hscale_f), s3);
}

// Softened branch for two pairs at once with the derivative (adjoint): returns B
// and sets D = B'(r)/r for both halves.  A zero displacement (coincident
// particles) is allowed here and gives r = 0 (the inner piece's B(0) and D(0)).
template <int SOFT>
__device__ __forceinline__ f2 bracket_soft_vjp_f32x2(f2 r2, const ForceConsts& f, const SeriesConsts& sc, f2& D) {
  if (SOFT == P3M_SOFT_NONE) {
    D = pk(0.0f, 0.0f);
    return pk(0.0f, 0.0f);
  }
  float a, b;
  upk(r2, a, b);
  const f2 r = pk(a > 0.0f ? a * rsqrt_approx(a) : 0.0f, b > 0.0f ? b * rsqrt_approx(b) : 0.0f);
  const f2 u = mul2(r, pk(f.inv2xs_f, f.inv2xs_f));
  const f2 u2 = mul2(u, u);
  f2 h = pk(sc.h_f[kHTermsF - 1], sc.h_f[kHTermsF - 1]);
  f2 hd = pk(sc.hd_f[kHTermsF - 1], sc.hd_f[kHTermsF - 1]);
#pragma unroll
  for (int k = kHTermsF - 2; k >= 0; --k) {
    h = fma2(h, u2, pk(sc.h_f[k], sc.h_f[k]));
    hd = fma2(hd, u2, pk(sc.hd_f[k], sc.hd_f[k]));
  }
  f2 s3, ds;
  if (SOFT == P3M_SOFT_BSPLINE) {
    const f2 x = mul2(r, pk(f.inv_epsb_f, f.inv_epsb_f));
    const f2 x2 = mul2(x, x);
    const float ce = f.bnorm_f * f.inv_epsb_f * f.inv_epsb_f;  // 32 / eps_B^5
    const f2 c = pk(f.bnorm_f, f.bnorm_f), cc = pk(ce, ce);
    const f2 s_in = mul2(c, fma2(x2, add2(x, pk(-1.2f, -1.2f)), pk(1.0f / 3.0f, 1.0f / 3.0f)));
    const f2 d_in = mul2(cc, fma2(pk(3.0f, 3.0f), x, pk(-2.4f, -2.4f)));
    float xa, xb;
    upk(x, xa, xb);
    const f2 xi = pk(rcp_approx(xa), rcp_approx(xb));
    const f2 xi2 = mul2(xi, xi);
    const f2 xi3 = mul2(xi2, xi);
    const f2 poly = fma2(x2, fma2(pk(-1.0f / 3.0f, -1.0f / 3.0f), x, pk(1.2f, 1.2f)),
                         fma2(pk(-1.5f, -1.5f), x, pk(2.0f / 3.0f, 2.0f / 3.0f)));
    const f2 s_out = mul2(c, fma2(xi3, pk(-1.0f / 480.0f, -1.0f / 480.0f), poly));
    // ce (2.4 - x - 1.5 / x + x^-5 / 160)
    const f2 d_out = mul2(cc, fma2(mul2(xi3, xi2), pk(1.0f / 160.0f, 1.0f / 160.0f),
                                   fma2(pk(-1.5f, -1.5f), xi, add2(pk(2.4f, 2.4f), mul2(x, pk(-1.0f, -1.0f))))));
    float ia, ib, oa, ob, dia, dib, doa, dob;
    upk(s_in, ia, ib);
    upk(s_out, oa, ob);
    upk(d_in, dia, dib);
    upk(d_out, doa, dob);
    s3 = pk(xa < 0.5f ? ia : oa, xb < 0.5f ? ib : ob);
    ds = pk(xa < 0.5f ? dia : doa, xb < 0.5f ? dib : dob);
  } else {  // Plummer
    float pa, pb;
    upk(add2(r2, pk(f.eps2_f, f.eps2_f)), pa, pb);
    const f2 p = pk(rsqrt_approx(pa), rsqrt_approx(pb));
    const f2 p2 = mul2(p, p);
    s3 = mul2(p2, p);
    ds = mul2(mul2(s3, p2), pk(-3.0f, -3.0f));
  }
  const float kd = -f.hscale_f * f.inv2xs_f * f.inv2xs_f;
  D = fma2(hd, pk(kd, kd), ds);
  return fma2(h, pk(-f.hscale_f, -f.hscale_f), s3);
}

// ---------------------------------------------------------------- FP64 ----

template <int SOFT, bool VJP>
__device__ __forceinline__ double bracket_f64(double r2, const ForceConsts& f, const SeriesConsts& sc, double& D) {
  const double inv_sqrt_pi = 0.56418958354775628695;
  if (r2 < f.rsw2_d || r2 == 0.0) {
    if (SOFT == P3M_SOFT_NONE) {
      D = 0.0;
      return 0.0;
    }
    double r = sqrt(r2);
    double u = r / (2.0 * f.x_s);
    double u2 = u * u;
    double h = sc.h_d[kHTermsD - 1];
    for (int k = kHTermsD - 2; k >= 0; --k) h = fma(h, u2, sc.h_d[k]);
    double w = 2.0 * f.x_s;
    double w3 = w * w * w;
    double s3, ds;
    if (SOFT == P3M_SOFT_BSPLINE) {
      double eb = f.eps_b;
      double x = r / eb;
      double c = 32.0 / (eb * eb * eb);
      double ce = c / (eb * eb);
      if (x < 0.5) {
        s3 = c * (x * x * x - 1.2 * x * x + 1.0 / 3.0);
        ds = ce * (3.0 * x - 2.4);
      } else {
        s3 = c * (-x * x * x / 3.0 + 1.2 * x * x - 1.5 * x + 2.0 / 3.0 - 1.0 / (480.0 * x * x * x));
        ds = ce * (-x + 2.4 - 1.5 / x + 1.0 / (160.0 * x * x * x * x * x));
      }
    } else {
      double s = r2 + f.eps * f.eps;
      double p = 1.0 / sqrt(s);
      s3 = p * p * p;
      ds = -3.0 * s3 / s;
    }
    if (VJP) {
      double hd = sc.hd_d[kHTermsD - 1];
      for (int k = kHTermsD - 2; k >= 0; --k) hd = fma(hd, u2, sc.hd_d[k]);
      D = ds - hd / (w3 * w * w);
    }
    return s3 - h / w3;
  }
  double r = sqrt(r2);
  double rinv = 1.0 / r;
  double u = r / (2.0 * f.x_s);
  double e = exp(-u * u);
  double rinv3 = rinv * rinv * rinv;
  double B = (erfc(u) + 2.0 * inv_sqrt_pi * u * e) * rinv3;
  if (VJP) {
    double k3 = inv_sqrt_pi / (2.0 * f.x_s * f.x_s * f.x_s);
    D = -(3.0 * B + e * k3) * rinv * rinv;
  }
  if (SOFT == P3M_SOFT_PLUMMER) {
    double s = r2 + f.eps * f.eps;
    double p = 1.0 / sqrt(s);
    double p3 = p * p * p;
    if (VJP) D += -3.0 * p3 / s + 3.0 * rinv3 * rinv * rinv;
    B += p3 - rinv3;
  }
  return B;
}

}  // namespace p3m
