/*
 * C ABI of the long-range (particle-mesh) half of the P3M gravity of
 * CONCEPT 1.0 (arXiv:2112.01508, Section 2.1.2 Eq. pm_method and Section 2.1.3
 * Eq. p3m_gravity, upper half), for one GPU (sm_103a).
 *
 * For particles at positions x_i in the periodic box [0, L)^3 with equal masses
 * m, the long-range acceleration is
 *
 *   a_i = (4 pi G m / L_phi^4) sum_m W_p((x_i - x_m)/L_phi) D_pd F^-1{ G(k) F rho }_m
 *   rho_m = sum_j W_p((x_m - x_j)/L_phi)                       (particles -> mesh)
 *   G(k)  = [prod_d sinc^p(L_phi k_d / 2)]^-2 exp(-x_s^2 k^2) / k^2,  G(0) = 0
 *
 * on an n_phi^3 mesh with cell-centred points x_m = L_phi (m + 1/2),
 * L_phi = L / n_phi, interpolation W_p of order p_i (Eqs. W_NGP, W_CIC, W_TSC,
 * W_PCS), the symmetric difference D_pd of order p_d (Eqs. symmetric_diff_2 ...
 * symmetric_diff_8), F the discrete Fourier transform (cuFFT), F^-1 its
 * inverse normalised so that F^-1 F = 1.  With x_s = 0 the kernel is the plain
 * Poisson kernel 1/k^2 of the PM method.  These are accelerations (force / m).
 *
 * The difference is applied per particle, on the mesh values its interpolation
 * stencil needs, instead of building three force meshes first; the result is the
 * same sum up to rounding order.
 *
 * Conventions: all particle arrays are caller-owned device memory; the context
 * owns the mesh (n_phi^2 (n_phi + 2) reals, FFT in place) and the cuFFT plans and
 * work area.  Calls are asynchronous on the context's stream; errors are
 * returned, never aborted on.  Positions outside [0, L) or non-finite latch
 * P3M_ERR_NONFINITE (reported by p3m_pm_sync or the next call); such particles
 * contribute nothing and receive zero acceleration.
 */
#ifndef P3M_PM_H
#define P3M_PM_H

#include <stdint.h>

#include "p3m_sr.h" /* p3m_status */

#ifdef __cplusplus
extern "C" {
#endif

typedef struct p3m_pm_ctx p3m_pm_ctx;

typedef struct {
  int64_t n;      /* particles (>= 0)                                              */
  double box;     /* L > 0                                                         */
  int n_phi;      /* mesh points per dimension, even, 8 ... 4096                   */
  double x_s;     /* split scale (>= 0); Eq. p3m_parameters takes 1.25 L_phi        */
  double G_m;     /* G m (finite)                                                  */
  int p_i;        /* interpolation order: 1 NGP, 2 CIC, 3 TSC, 4 PCS               */
  int p_d;        /* difference order: 2, 4, 6 or 8                                */
  int precision;  /* 32: float mesh, FFT and interpolation; 64: double throughout  */
} p3m_pm_params;

typedef struct {
  int n_phi;
  int64_t mesh_bytes;       /* the padded in-place mesh                             */
  int64_t fft_work_bytes;   /* cuFFT work area (forward + inverse plans)            */
  int64_t kernel_launches;  /* kernels of this library (cuFFT's own not counted)    */
  double assign_ms;         /* device time of the phases of the last p3m_pm_accel   */
  double fft_ms;
  double kernel_ms;         /* G(k) multiplication                                  */
  double ifft_ms;
  double interp_ms;         /* difference + mesh -> particle interpolation          */
} p3m_pm_stats_t;

/*
 * Create a context: validates the parameters (P3M_ERR_INVALID), allocates the
 * mesh and builds the forward and inverse cuFFT plans on cuda_stream (NULL =
 * legacy default stream).  Allocation failure returns P3M_ERR_OOM.
 */
p3m_status p3m_pm_create(const p3m_pm_params* params, void* cuda_stream, p3m_pm_ctx** out);

/* Free the context, its mesh and plans.  NULL is ignored. */
void p3m_pm_destroy(p3m_pm_ctx* ctx);

/* Message describing the last error of this context (never NULL). */
const char* p3m_pm_last_error(const p3m_pm_ctx* ctx);

/* Wait for the context's stream; returns a latched device-side error if any. */
p3m_status p3m_pm_sync(p3m_pm_ctx* ctx);

/* Synchronise and fill *out (see p3m_pm_stats_t). */
p3m_status p3m_pm_stats(p3m_pm_ctx* ctx, p3m_pm_stats_t* out);

/*
 * Long-range accelerations of all n particles (the paper applies them to every
 * particle whenever rung 0 is kicked).
 *   pos         3 x n float64 SoA, device, any order (the tile/subtile order of
 *               p3m_sr_sort gives the best locality).
 *   acc         3 x n device, float (precision 32) or double (64), SoA.
 *   accumulate  0: acc is overwritten; 1: the long-range part is added to acc
 *               (e.g. onto the short-range accelerations of p3m_sr_forces).
 */
p3m_status p3m_pm_accel(p3m_pm_ctx* ctx, const double* pos, void* acc, int accumulate);

/*
 * The mesh steps on their own, for inspection and tests.
 * p3m_pm_assign: rho_m = sum_j W_p((x_m - x_j)/L_phi) into rho_out, a dense
 *   n_phi^3 array (x slowest, z fastest) of the context's precision, device.
 * p3m_pm_potential: the mesh left by the last p3m_pm_accel, i.e.
 *   (4 pi G m / L_phi^4) F^-1{G(k) F rho}, copied densely into phi_out
 *   (n_phi^3, same layout and type); P3M_ERR_STATE before any p3m_pm_accel.
 */
p3m_status p3m_pm_assign(p3m_pm_ctx* ctx, const double* pos, void* rho_out);
p3m_status p3m_pm_potential(p3m_pm_ctx* ctx, void* phi_out);

#ifdef __cplusplus
}
#endif

#endif /* P3M_PM_H */
