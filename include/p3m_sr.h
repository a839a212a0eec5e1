/*
 * p3m_sr.h -- C ABI of the GB300 short-range P3M gravity library.
 *
 * The library computes the short-range half of CONCEPT 1.0's P3M gravity
 * (arXiv:2112.01508, Section 2.1.3, lower half of Eq. p3m_gravity):
 *
 *   a_i = -G m  sum_{j != i, |x_ij| < x_r}  B(|x_ij|) x_ij ,
 *   B(r) = erfc(u)/r^3 + exp(-u^2)/(sqrt(pi) x_s r^2) + ( |x|^{-3}_shape - r^{-3} ),
 *   u = r/(2 x_s),  x_ij = nearest periodic image of x_i - x_j,
 *
 * over the paper's tile/subtile decomposition of the periodic box (Section
 * 2.1.3, "Tiles" and "Subtiles"), for the receivers on the active rungs of the
 * individual time-stepping (Section 2.2.2), plus the rung rule (Eq. rung), the
 * kick and drift operators (Section 2.2.2) and the vector-Jacobian product of
 * the accelerations with respect to positions.
 *
 * Conventions shared by every entry point:
 *   - Particle arrays are DEVICE pointers owned by the caller (for example the
 *     data_ptr of torch tensors).  Vectors are structure-of-arrays, 3 x n:
 *     x[0..n), then y[0..n), then z[0..n).  The library never frees them.
 *   - The context owns its scratch memory (sort buffers, offsets, chunk lists),
 *     allocated once by p3m_sr_create for the particle count given there.
 *   - Every call only enqueues work on the context's CUDA stream and returns
 *     without synchronising (except p3m_sr_sync and p3m_sr_stats).
 *   - Errors are returned, never aborted on.  Argument errors are detected on
 *     the host and returned immediately.  Errors found by kernels (non-finite
 *     or out-of-box positions, non-finite accelerations) are latched in a
 *     device word; p3m_sr_sync waits for the stream and returns the latched
 *     status, and later calls return it once the copy that reports it has
 *     landed.  p3m_sr_last_error gives a human-readable message.
 *   - "precision" arguments are 32 (float) or 64 (double).
 *   - After p3m_sr_sort, every other call assumes the particles are in the
 *     sorted (tile -> subtile -> particle) order and positions lie in [0, L).
 *     p3m_sr_drift may move the sorted positions without invalidating the sort
 *     (up to 64 drifts; see p3m_sr_drift).
 */
#ifndef P3M_SR_H
#define P3M_SR_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  P3M_OK = 0,
  P3M_ERR_INVALID = 1,        /* bad argument or parameter                          */
  P3M_ERR_TOO_FEW_TILES = 2,  /* fewer than 4 tiles per dimension (Section 2.1.3)   */
  P3M_ERR_OOM = 3,            /* device allocation failed                           */
  P3M_ERR_CUDA = 4,           /* a CUDA runtime call failed                         */
  P3M_ERR_TIMEOUT = 5,        /* reserved: a bounded device-side wait expired       */
  P3M_ERR_NONFINITE = 6,      /* non-finite or out-of-box input met by a kernel     */
  P3M_ERR_STATE = 7           /* call out of order (e.g. forces before sort), or
                                 positions drifted too far since the sort          */
} p3m_status;

typedef enum { P3M_SOFT_NONE = 0, P3M_SOFT_PLUMMER = 1, P3M_SOFT_BSPLINE = 2 } p3m_softening;

/*
 * Physical and decomposition parameters.
 *   n          number of particles (0 <= n < 2^31)
 *   box        periodic box side L (> 0)
 *   x_s, x_r   force split scale and cutoff, 0 < x_s, 0 < x_r <= L/4
 *              (paper defaults x_s = 1.25 L/n_phi, x_r = 4.5 x_s, Eq. p3m_parameters)
 *   G_m        G times the particle mass (accelerations are returned)
 *   softening  p3m_softening: none, Plummer (Eq. plummer_shape) or B-spline
 *              (Eq. bspline_force with eps_B = 2.8 eps, Section 2.1.1)
 *   eps        Plummer softening length epsilon (> 0 when softened)
 *   n_sub      subtiles per tile along x, y, z (each 1..16)
 *   n_rung     number of rungs, 1..8 (Section 2.2.2)
 * The box is split into n_t = floor(L / x_r) tiles per dimension (tiles are at
 * least x_r wide, Section 2.1.3); n_t must be at least 4.
 */
typedef struct {
  int64_t n;
  double box;
  double x_s;
  double x_r;
  double G_m;
  int softening;
  double eps;
  int n_sub[3];
  int n_rung;
} p3m_sr_params;

typedef struct p3m_sr_ctx p3m_sr_ctx;

/* Geometry and counters, filled by p3m_sr_stats. */
typedef struct {
  int n_tile;              /* tiles per dimension                               */
  int n_sub[3];            /* subtiles per tile per dimension                   */
  int64_t n_subtiles;      /* (n_tile n_sub[0]) (n_tile n_sub[1]) (n_tile n_sub[2]) */
  int64_t n_active;        /* receivers of the last p3m_sr_build_pairs          */
  int64_t n_chunks;        /* receiver chunks (<= 32 particles) of that call    */
  int64_t pairs_last;      /* interacting ordered pairs (i active, j != i,
                              r^2 < x_r^2) met by the last forces/vjp call      */
  int64_t kernel_launches; /* kernels launched by this context so far           */
  double force_kernel_ms;  /* device time of the last forward pair kernel       */
  double vjp_kernel_ms;    /* device time of the last adjoint pair kernel       */
} p3m_sr_stats_t;

/*
 * Create a context for n particles.  cuda_stream is a cudaStream_t (NULL: the
 * legacy default stream).  Validates the parameters (P3M_ERR_INVALID,
 * P3M_ERR_TOO_FEW_TILES) and allocates all scratch on the current device
 * (P3M_ERR_OOM).  *out is NULL on failure.
 */
p3m_status p3m_sr_create(const p3m_sr_params* params, void* cuda_stream, p3m_sr_ctx** out);

/* Free the context and its scratch.  NULL is ignored. */
void p3m_sr_destroy(p3m_sr_ctx* ctx);

/* Message describing the last error of this context (never NULL). */
const char* p3m_sr_last_error(const p3m_sr_ctx* ctx);

/* Wait for the context's stream; return the latched device status. */
p3m_status p3m_sr_sync(p3m_sr_ctx* ctx);

/* Synchronise and fill *out (see p3m_sr_stats_t). */
p3m_status p3m_sr_stats(p3m_sr_ctx* ctx, p3m_sr_stats_t* out);

/*
 * Change the number of particles of the following calls, for a domain whose
 * particle count changes (Section 2.1.2, "Parallelisation": particles migrate
 * between the domains of neighbouring processes as they move).
 *   n  0 <= n <= the n given to p3m_sr_create (the context's capacity: no
 *      memory is allocated or freed); larger values return P3M_ERR_INVALID.
 * Every particle array of the following calls has n rows per component (a
 * 3 x n SoA vector is x[0..n), y[0..n), z[0..n)).  The sort state is dropped:
 * the next force, build_pairs or vjp call needs a p3m_sr_sort first.
 */
p3m_status p3m_sr_set_count(p3m_sr_ctx* ctx, int64_t n);

/*
 * Tile ranges of the last p3m_sr_sort (Section 2.1.3, "Tiles": the particles
 * are stored tile by tile).  offsets_out: DEVICE array of n_t^3 + 1 int32;
 * offsets_out[T] is the sorted index of the first particle of tile
 * T = (t_x n_t + t_y) n_t + t_z and offsets_out[n_t^3] = n, so the particles of
 * the slab of tile columns [c0, c1) along x are the sorted indices
 * [offsets_out[c0 n_t^2], offsets_out[c1 n_t^2]).  Enqueued on the context's
 * stream.  P3M_ERR_STATE before any sort (or after set_count / set_subtiles).
 */
p3m_status p3m_sr_tile_offsets(p3m_sr_ctx* ctx, int32_t* offsets_out);

/*
 * Change the subtile decomposition (Section 2.1.3, "Subtiles": the number of
 * subtiles per tile is free, and the paper refines it while the simulation
 * runs by timing a force computation with one more subdivision).
 *   n_sub  HOST array of 3 ints in 1..16 (subtiles per tile per dimension).
 * Forces do not depend on it beyond rounding.  The per-subtile arrays are
 * reallocated when the subtile count grows (cudaFree/cudaMalloc, which wait for
 * queued work; not inside stream capture).  The sort state is dropped: the
 * next force, build_pairs or vjp call needs a p3m_sr_sort first
 * (P3M_ERR_STATE).  On an error the old decomposition stays in force.
 */
p3m_status p3m_sr_set_subtiles(p3m_sr_ctx* ctx, const int* n_sub);

/*
 * Sort the particles into tiles and subtiles (Section 2.1.3: O(N) sort into
 * tiles, memory reordered in tile -> subtile -> particle walk order).
 *   pos          3 x n float64 SoA, device; reordered IN PLACE.  Each position
 *                must be finite and in [0, L) (else P3M_ERR_NONFINITE is
 *                latched, the offending coordinate is binned as 0 and the
 *                forces that follow are undefined until the next good sort).
 *   carry        n_carry device arrays of n elements of carry_bytes[c] bytes
 *                each (1..32), permuted in place alongside (momenta, rungs,
 *                identifiers ...).  May be NULL when n_carry == 0.
 *   perm_out     nullable, n int32: perm_out[k] = pre-sort index of the
 *                particle now at k.
 *   subtile_id_out nullable, n int32: subtile id of the particle now at k.
 * Subtile of a particle: g_d = min(floor(x_d * (M_d / L)), M_d - 1) with
 * M_d = n_t n_sub[d] (one correctly rounded multiply), tile t_d = g_d / n_sub[d],
 * s_d = g_d mod n_sub[d];
 *   id = ((t_x n_t + t_y) n_t + t_z) (n_sub[0] n_sub[1] n_sub[2]) + (s_x n_sub[1] + s_y) n_sub[2] + s_z.
 * The sort is stable (equal ids keep their input order) and deterministic.
 */
p3m_status p3m_sr_sort(p3m_sr_ctx* ctx, double* pos, void* const* carry, const int* carry_bytes,
                       int n_carry, int32_t* perm_out, int32_t* subtile_id_out);

/*
 * Out-of-place variant of p3m_sr_sort (same binning, same stable order): the
 * sorted positions and carried arrays are written to separate output arrays in
 * one pass and the inputs are left unchanged, which halves the memory traffic of
 * the reordering (no copy back).  Callers alternate two sets of buffers.
 *   pos_in, pos_out   3 x n float64 SoA, device, distinct (each position of pos_in
 *                     finite and in [0, L), as for p3m_sr_sort).
 *   carry_in, carry_out  n_carry (at most 8) pairs of distinct device arrays of n
 *                     elements of carry_bytes[c] bytes (1..32).
 *   perm_out, subtile_id_out  as for p3m_sr_sort.
 * After the call the sort describes pos_out (drifting pos_out keeps it usable).
 */
p3m_status p3m_sr_sort_into(p3m_sr_ctx* ctx, const double* pos_in, double* pos_out, const void* const* carry_in,
                            void* const* carry_out, const int* carry_bytes, int n_carry, int32_t* perm_out,
                            int32_t* subtile_id_out);

/*
 * Move per-particle data between the caller's order and the order of the last
 * p3m_sr_sort (the tile -> subtile walk order of Section 2.1.3), for data that
 * was not carried through the sort (for example to return accelerations in the
 * caller's order, or to bring gradients into the sorted order).
 *   src, dst    distinct device arrays of `rows` rows of n elements of
 *               elem_bytes bytes (1, 2, 4 or 8); a 3 x n SoA vector has rows = 3.
 *   p3m_sr_permute:    dst[r][k] = src[r][perm[k]]   (caller order -> sorted)
 *   p3m_sr_unpermute:  dst[r][perm[k]] = src[r][k]   (sorted -> caller order)
 * with perm the permutation of the last sort (P3M_ERR_STATE before any sort).
 */
p3m_status p3m_sr_permute(p3m_sr_ctx* ctx, const void* src, void* dst, int elem_bytes, int rows);
p3m_status p3m_sr_unpermute(p3m_sr_ctx* ctx, const void* src, void* dst, int elem_bytes, int rows);

/*
 * Build the receiver set and work list for the following forces / vjp calls
 * (Section 2.1.3 "precomputed (sub)tile pairings"; Section 2.2.2: receivers are
 * the particles on rungs >= rung_min, suppliers are all particles).
 *   rung      nullable device int8 array (sorted order); NULL: all active.
 *   rung_min  current rung; particles with rung >= rung_min are receivers.
 * Must follow p3m_sr_sort (P3M_ERR_STATE otherwise).
 */
p3m_status p3m_sr_build_pairs(p3m_sr_ctx* ctx, const int8_t* rung, int rung_min);

/*
 * Short-range accelerations (Section 2.1.3, short-range half of Eq.
 * p3m_gravity) on the receivers of the last p3m_sr_build_pairs.
 *   pos        3 x n float64 SoA, device, in the sorted order, unchanged
 *              since the last p3m_sr_sort or moved only by p3m_sr_drift (the
 *              sort wrote the FP32 subtile-relative records of that array;
 *              after a drift, or for a different array, they are rebuilt
 *              here).
 *   precision  32: FP32 arithmetic and accumulation, displacements taken
 *              relative to subtile origins (positions read once in FP64);
 *              acc_out is 3 x n float.  64: FP64 throughout, acc_out 3 x n
 *              double.
 *   acc_out    receivers' rows are overwritten; other rows are untouched.
 * The FP32 path requires x_r <= 4.6 x_s (range of its erfc fit).
 * With every particle a receiver (build_pairs with rung NULL) the FP32 path
 * evaluates each pair once and updates both particles (see
 * p3m_sr_set_symmetric); its sums are then added with atomics, so the last
 * bits of the result depend on the order of execution.
 */
p3m_status p3m_sr_forces(p3m_sr_ctx* ctx, const double* pos, int precision, void* acc_out);

/*
 * Pair evaluation of the all-active FP32 forces.  enable = 1 (the default):
 * each unordered pair {i, j} is evaluated once and both particles receive their
 * share, as the paper's tile pairing does (Section 2.1.3: a supplier tile is
 * never paired again with a receiver tile it already met in the opposite
 * roles); the per-particle sums are FP32 atomics into a context buffer.
 * enable = 0: every receiver gathers its own sum over all its partners, each
 * pair being evaluated from both sides; the result is then bitwise
 * reproducible.  The FP32 vjp follows the same setting for any active set
 * (its pair term is antisymmetric in the pair too, and every particle gets a
 * gradient).  Partially active force calls, the FP64 path and the tabulated
 * variant always gather.  P3M_ERR_INVALID for a NULL context.
 */
p3m_status p3m_sr_set_symmetric(p3m_sr_ctx* ctx, int enable);

/*
 * The paper's tabulated variant of the FP32 forces (Section 2.1.3, "Other
 * optimisations": the bracket of Eq. p3m_gravity, softening included, stored in
 * a 1-D table indexed by r^2 on [0, x_r^2) and read with a nearest-grid-point
 * lookup; the paper uses 2^12 entries).  Same receivers, traversal and output
 * as p3m_sr_forces with precision 32; only B(r) comes from the table, built in
 * FP64 at the bin centres on the first call with a given table_bits (4..14).
 * Its error is far above the analytic path's (see the tests); it exists to
 * measure the paper's speed/accuracy trade-off on this hardware.
 *   acc_out  3 x n float; receivers' rows are overwritten.
 */
p3m_status p3m_sr_forces_tabulated(p3m_sr_ctx* ctx, const double* pos, int table_bits, float* acc_out);

/*
 * Rungs from accelerations (Section 2.2.2, Eq. rung):
 *   l_i = max(0, ceil(log2(dt sqrt(|a_i| / (2 eta eps))))), clamped to n_rung-1,
 * evaluated exactly as: q = dt*dt / ((2*eta)*eps); s = (q*q) * ((ax*ax + ay*ay) + az*az);
 * l = smallest l >= 0 with s <= 16^l (IEEE double, correctly rounded, no FMA).
 *   acc        3 x n SoA device, acc_precision 32 or 64 (floats are widened).
 *   rung_out   n int8 device.
 * Non-finite accelerations get rung 0 and latch P3M_ERR_NONFINITE.
 */
p3m_status p3m_sr_assign_rungs(p3m_sr_ctx* ctx, const void* acc, int acc_precision, double dt,
                               double eta, double eps, int8_t* rung_out);

/*
 * Kick (Section 2.2.2, operator K with a = 1): for particles with
 * rung >= rung_min (all when rung is NULL, using kick_factor[0]),
 *   q_i <- q_i + a_i * kick_factor[rung_i]     in double (widen, multiply, add).
 *   mom        3 x n device, mom_precision 32 or 64 (FP32 momenta are rounded
 *              once after the double update).
 *   acc        3 x n device, acc_precision 32 or 64.
 *   kick_factor HOST array of n_rung doubles (K(Delta t / 2^l)).
 */
p3m_status p3m_sr_kick(p3m_sr_ctx* ctx, void* mom, int mom_precision, const void* acc,
                       int acc_precision, const int8_t* rung, int rung_min,
                       const double* kick_factor);

/*
 * One kick of the rung-based leapfrog (Section 2.2.2, the time-stepping figure:
 * rung-l momenta are kicked every dt / 2^l, positions drift every
 * dt / 2^(n_rung-1); a particle whose rung changes jumps to a neighbouring rung
 * by making its next kick 1/2 or 3/4 as large as usual, and can move to a lower
 * rung only at every other kick).  For the particles with rung >= rung_min:
 *   q_i <- q_i + a_i f_i dt / 2^l_i,   f_i = 1, 1/2 or 3/4 by kick_state_i (0, 1, 2);
 * then, from the same a_i, the rung of Eq. rung (computed as in
 * p3m_sr_assign_rungs) decides the jump:
 *   higher than l_i -> l_i + 1, next kick 1/2 of the usual (state 1);
 *   lower than l_i and substep / 2^(n_rung-1-l_i) odd -> l_i - 1, next kick 3/4
 *   of the usual (state 2);  otherwise unchanged (state 0).
 *   substep   global substep counter k >= 1: this kick happens at k dt / 2^(n_rung-1)
 *             after the last synchronisation; rung_min must equal
 *             n_rung - 1 - (trailing zero bits of k), capped at 0 (P3M_ERR_INVALID
 *             otherwise).
 *   synchronize  non-zero at the end of a global step (k a multiple of
 *             2^(n_rung-1)): the kick stops at that time (factor f_i - 1/2), the
 *             states are reset and the rungs are left for p3m_sr_assign_rungs.
 *   mom, acc  3 x n device, precision 32 or 64; rung, kick_state  n int8 device,
 *             updated in place.  Arithmetic in IEEE double as in p3m_sr_kick.
 * A particle with rung >= n_rung or kick_state outside {0, 1, 2} is left
 * untouched and latches P3M_ERR_STATE (reported by this or a later call, or
 * by p3m_sr_sync); a non-finite acceleration latches P3M_ERR_NONFINITE.
 */
p3m_status p3m_sr_rung_kick(p3m_sr_ctx* ctx, void* mom, int mom_precision, const void* acc, int acc_precision,
                            int8_t* rung, int8_t* kick_state, int rung_min, long long substep, double dt,
                            double eta, double eps, int synchronize);

/*
 * p3m_sr_rung_kick (synchronize = 0) followed by p3m_sr_drift of every particle,
 * in one pass over the particle arrays (the kick of substep k of the rung-based
 * leapfrog and the drift that starts substep k + 1, Section 2.2.2): the results
 * equal those two calls bit for bit.
 *   pos, drift_factor  as for p3m_sr_drift (drifting the sorted array keeps the
 *                      sort usable, as p3m_sr_drift does); the other arguments as
 *                      for p3m_sr_rung_kick.
 */
p3m_status p3m_sr_rung_kick_drift(p3m_sr_ctx* ctx, void* mom, int mom_precision, const void* acc, int acc_precision,
                                  int8_t* rung, int8_t* kick_state, int rung_min, long long substep, double dt,
                                  double eta, double eps, double* pos, double drift_factor);

/*
 * Drift (Section 2.2.2, operator D with a = 1):
 *   x_i <- x_i + q_i * factor, then wrapped into [0, L): x <- x - L floor(x / L).
 *   pos  3 x n float64 device;  mom  3 x n device, mom_precision 32 or 64.
 * Drifting the array of the last p3m_sr_sort keeps that sort usable, as the
 * paper's periodic (not per-step) memory reordering does (Section 2.1.3,
 * "Other optimisations"): the drift records a bound on its largest
 * displacement, and build_pairs / forces / vjp widen the subtile reach by the
 * sum of the bounds since the sort (more candidates, same pairs).  After 64
 * such drifts the sort is dropped (P3M_ERR_STATE until the next p3m_sr_sort);
 * a total drift with x_r + 2 drift >= L/2 latches P3M_ERR_STATE in the next
 * traversal.  Drifting any other array does not touch the sort.
 */
p3m_status p3m_sr_drift(p3m_sr_ctx* ctx, double* pos, const void* mom, int mom_precision,
                        double factor);

/*
 * Rungs, kick and drift in one pass over the particle arrays (Section 2.2.2:
 * Eq. rung, then operator K, then operator D, with a = 1), for steps in which
 * every particle is kicked: for each particle,
 *   rung_i <- Eq. rung of a_i            (as p3m_sr_assign_rungs),
 *   q_i    <- q_i + a_i kick_factor[rung_i]   (as p3m_sr_kick with rung_min 0),
 *   x_i    <- wrap(x_i + q_i drift_factor)   (as p3m_sr_drift),
 * with the same IEEE double arithmetic, so the results equal those three calls
 * bit for bit while the arrays are read and written once.
 *   pos        3 x n float64 device; mom 3 x n device (mom_precision 32 or 64);
 *   acc        3 x n device (acc_precision 32 or 64); rung_out n int8 device;
 *   kick_factor HOST array of n_rung doubles; drift_factor finite.
 * Drifting the array of the last p3m_sr_sort keeps that sort usable exactly as
 * p3m_sr_drift does.  Non-finite accelerations latch P3M_ERR_NONFINITE.
 */
p3m_status p3m_sr_kick_drift(p3m_sr_ctx* ctx, double* pos, void* mom, int mom_precision, const void* acc,
                             int acc_precision, int8_t* rung_out, double dt, double eta, double eps,
                             const double* kick_factor, double drift_factor);

/*
 * Vector-Jacobian product of the short-range accelerations with respect to
 * the positions (derived from Eq. p3m_gravity):
 *   xbar_k = sum_{j != k, r_kj < x_r} J_kj (abar_k [k active] - abar_j [j active]),
 *   J_kj = phi(r) I + (phi'(r)/r) x_kj x_kj^T,   phi = -G m B.
 * Active means receiver of the last p3m_sr_build_pairs.  Every particle gets a
 * gradient (suppliers move the receivers' accelerations too).  The pair term
 * changes sign under k <-> j, so the FP32 path evaluates each pair once and
 * adds the term to both with atomics (p3m_sr_set_symmetric; its last bits then
 * depend on the order of execution).
 *   pos          3 x n float64 SoA device (sorted order)
 *   acc_bar      3 x n device, float (precision 32) or double (64)
 *   pos_bar_out  3 x n device, same type; every row is overwritten.
 */
p3m_status p3m_sr_vjp(p3m_sr_ctx* ctx, const double* pos, int precision, const void* acc_bar,
                      void* pos_bar_out);

/*
 * Allocation-free FP32 short-range accelerations for a small particle set.
 *
 * The paper has no counterpart to this entry point; it exists for callers that
 * cannot allocate device memory: code running inside a memory pool or arena
 * owned by a host application, a plugin that is handed only its input and
 * output buffers, or a pipeline that forbids cudaMalloc after start-up.  It
 * needs no context and calls no cudaMalloc, cudaFree or other allocating
 * routine.  It sorts the particles into tiles and subtiles, builds the
 * receiver chunks and evaluates the FP32 forces with the same kernels as
 * p3m_sr_sort + p3m_sr_build_pairs + p3m_sr_forces (all particles active), but
 * keeps every intermediate array in one fixed-size device array inside the
 * library (about 7.9 MB, held by every GPU that loads the library until the
 * process exits).
 *   params      as for p3m_sr_create; n <= 65536, at most 2^18 subtiles and
 *               2^14 chunk segments (n_t^2 ceil(n_t/4)), x_r <= 4.6 x_s.  Larger inputs return
 *               P3M_ERR_INVALID.
 *   cuda_stream cudaStream_t; all work is enqueued on it (nothing is waited for).
 *   pos         3 x n float64 SoA, device, any order; it is not modified.
 *               The box is periodic: a finite coordinate outside [0, L) is
 *               taken as its periodic image x - L floor(x / L).  A particle
 *               with a non-finite coordinate gets NaN accelerations and exerts
 *               no force on the others (no status reports it: the call does
 *               not wait for the GPU).
 *   acc_out     3 x n float, device: accelerations in the order of pos.
 * The first call on a device looks up the device address of the internal array
 * (cudaGetSymbolAddress, with that device current); make that first call before
 * any stream capture.  The address is kept for the life of the process: do not
 * use this entry point on a device after cudaDeviceReset (or any other
 * teardown of its primary context).  Every call uses the same internal array:
 * calls whose GPU work overlaps (other streams, other host threads) race and
 * must be serialised by the caller.
 */
p3m_status p3m_sr_forces_noalloc(const p3m_sr_params* params, void* cuda_stream, const double* pos,
                                 float* acc_out);

#ifdef __cplusplus
}
#endif

#endif /* P3M_SR_H */
