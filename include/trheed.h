/*
 * trheed.h - C ABI of the GB300 RHEED/TRHEPD rocking-curve library (libtrheed.so).
 *
 * The library computes the forward model of reflection high-energy electron diffraction (RHEED)
 * and total-reflection high-energy positron diffraction (TRHEPD) by the matrix-ODE multi-slice
 * method of Kudo, Yamamoto & Hoshi, "A fast and accurate computation method for reflective
 * diffraction simulations" (arXiv 2306.00271):
 *
 *   - the problem (Section 2.1, Eqs. sch1-sch3, vtau, vrho, bd0, bd1): a 2D-periodic surface slab
 *     z_e <= z <= 0 with lattice a1, a2; beams k_j = m1 b1 + m2 b2 (k_1 = 0); the n-beam system
 *     c'' = -(U(z) + Gamma^2) c with U_jk = u_{g_j - g_k}(z) and
 *     Gamma = diag(sqrt(gamma^2 - |b0 + k_j|^2)); incident tau(0) = e_1, no wave from below
 *     (rho(z_e) = 0);
 *   - the method (Section 3, Algorithm 1): the economical state Z = [Q; P] (2n x n, Eq. mateq2)
 *     integrated from z_e to 0 by a splitting integrator (Section 3.4), with the right-hand-side
 *     transformation Z <- Z Q^{-1} whenever the Gershgorin-based bound xi on cond(Q) exceeds a
 *     threshold (Section 3.2), and rho(0) = (Gamma + i P Q^{-1})(Gamma - i P Q^{-1})^{-1} e_1
 *     (Eq. vrhocomp);
 *   - the output (Section 2.1, below Eq. bd1): rho(0) per beam and the intensity
 *     eta_i = |rho_i|^2 sin(theta0) Gamma_1 / Gamma_i for propagating beams (0 for evanescent ones).
 *
 * Every step of that path runs in CUDA kernels for sm_103a. There is no CPU fallback: on a
 * machine without a usable GPU every compute call returns TRH_ECUDA.
 *
 * Conventions
 *   - All functions return 0 (TRH_OK) or a negative TRH_E* code; no C++ exception crosses the
 *     ABI. trh_strerror() names a code; trh_last_error() gives a message for the last failing
 *     call on this thread.
 *   - Lengths in Angstrom, energies in eV, angles in degrees.
 *   - complex128 = two consecutive doubles (re, im).
 *   - Pointers marked "host or device" may point to host memory or to device memory of the
 *     current device; the library detects which (cudaPointerGetAttributes). Host outputs are
 *     written before the call returns; device outputs are written in stream order on `stream`.
 *   - The caller owns every buffer it passes; the library never frees or retains caller memory
 *     beyond the call (trh_create copies what it needs). The library owns its context and all
 *     device scratch, allocated in trh_create / trh_set_structure and freed in trh_destroy.
 *   - A context may be used by one thread at a time.
 */
#ifndef TRHEED_H
#define TRHEED_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes ---------------------------------------------------------------------- */
#define TRH_OK            0
#define TRH_EINVAL       -1  /* bad argument: shape, k_1 != 0, h <= 0, z_e >= 0, N too large...  */
#define TRH_EGRAZING     -2  /* some Gamma_j = 0 (beam exactly on the Ewald circle)              */
#define TRH_ESINGULAR    -3  /* zero or non-finite pivot in the RHST or in the final solve       */
#define TRH_ETIMEOUT     -4  /* a device-side bounded wait expired                               */
#define TRH_ENOMEM       -5  /* device or host allocation failed                                 */
#define TRH_ECUDA        -6  /* CUDA runtime error (including: no device)                        */
#define TRH_EUNSUPPORTED -7  /* valid request this build does not implement                      */
#define TRH_ENOCONV      -8  /* the bulk boundary condition did not converge in max_periods       */

/* ---- method selection --------------------------------------------------------------------- */
enum trh_integrator {
  TRH_SP4 = 0, /* BAB splitting, SRKN_6^b coefficients (Section 3.4; 6 kicks per step with FSAL) */
  TRH_SP6 = 1, /* BAB splitting, SRKN_11^b coefficients (11 kicks per step with FSAL)            */
  TRH_RK4 = 2, /* classical Runge-Kutta (Section 3.4); FP64 path only                         */
  TRH_CONVENTIONAL = 3 /* the conventional multi-slice method (Section 2.2): per-slice
                          exponential at the slice midpoint and recursive reflection, the
                          comparison point for the others; FP64 path only; the RHST threshold
                          and RHST counts do not apply                                        */
};

enum trh_precision {
  TRH_FP64  = 0, /* every product, update and solve in IEEE binary64                            */
  TRH_MIXED = 1  /* U*Q products on the BF16 tensor cores as fixed-point digit products (four
                    8-bit digits per operand, FP32 accumulators that never round); state as
                    FP32 pairs, RHST in FP32 plus double-float, final solve in binary64 (see
                    trh_rocking_curve)                                                           */
};

/* ---- problem description ------------------------------------------------------------------ */
typedef struct trh_problem {
  int particle;          /* +1 electron (RHEED), -1 positron (TRHEPD)                            */
  double energy_ev;      /* kinetic energy E (eV), > 0                                           */
  double absorption;     /* absorptive potential as a fraction of the real one (e.g. 0.1), >= 0  */
  double a1[2], a2[2];   /* surface lattice vectors (A)                                           */
  int n_beams;           /* N >= 1                                                                */
  const int* beams;      /* [N][2] (m1, m2) host; beams[0] must be (0, 0); entries distinct       */
  int n_atoms;           /* atoms per parameter set, >= 1                                         */
  const double* atoms;   /* [n_atoms][3] x, y, z (A), z <= 0; host. Default structure.           */
  const double* dw;      /* [n_atoms] Debye-Waller B (A^2), >= 0; host                            */
  const int* species;    /* [n_atoms] species index in [0, n_species); host                      */
  int n_species;         /* >= 1                                                                  */
  const double* sf;      /* [n_species][8] scattering factor a_1..a_4 (A), b_1..b_4 (A^2), host.
                            Electron scattering factor f(s) = sum_i a_i exp(-b_i s^2),
                            s = |q| / (4 pi).                                                     */
  double z_e;            /* slab bottom (A), < 0                                                  */
  int n_steps;           /* L >= 1; step h = -z_e / L                                              */
  int integrator;        /* enum trh_integrator                                                    */
  double rhst_threshold; /* RHST threshold on xi; <= 0 selects 1000 (Algorithm 1)                 */
  int precision;         /* enum trh_precision                                                     */
} trh_problem;

typedef struct trh_ctx trh_ctx;

/* Counters of the last trh_rocking_curve call. */
typedef struct trh_stats {
  int n_sets;             /* parameter sets in the context                                        */
  int n_angles;           /* angles in the last call                                               */
  int n_beams;            /* N                                                                     */
  int n_nodes;            /* potential evaluation nodes per set (kick positions)                  */
  long long rhst_total;   /* RHST transforms summed over all (set, angle) of the last call         */
  int rhst_max;           /* largest RHST count of one (set, angle)                                */
  int n_bad;              /* (set, angle) pairs with a nonzero status                              */
  int first_bad_set;      /* -1 if none                                                            */
  int first_bad_angle;    /* -1 if none                                                            */
  int first_bad_status;   /* TRH_E* code of that pair                                              */
  int kernels_launched;   /* kernels launched by the last call                                     */
  double ms_last;         /* wall time of the last call (host clock, includes synchronisation)   */
  double ms_potential;    /* device time of the potential-table kernels of the last call (CUDA
                             events on the call's stream; 0 if the tables were current)          */
  double ms_integrate;    /* device time of the integration kernel of the last call              */
  double ms_gradient;     /* device time of the reverse sweep of the last trh_curve_jacobian /
                             trh_rfactor_grad call (0 after trh_rocking_curve)                   */
  int wide_tile;          /* tile edge the autotuner chose for the wide FP64 kernel (N > 64) of
                             the last call, 0 if that kernel did not run                         */
  int graph_replay;       /* trh_batch_run: 1 if the work was replayed from the captured graph   */
  int bulk_periods;       /* bulk periods the last bulk computation needed (largest over angles;
                             0 without a bulk or when the cached one was reused)                 */
  double ms_bulk;         /* device time of that bulk computation (0 if none ran)               */
  int column_split;       /* 1 if the last call ran two CTAs per (set, angle) pair
                             (trh_set_column_split), else 0                                    */
  int ctas_per_pair;      /* CTAs (one thread-block cluster) that integrated each pair in the
                             last call: 1 or 2 (N <= 64), ceil(N / 32) on the mixed path for
                             64 < N <= 128, ceil(N / 16) for 128 < N <= 256                   */
  int set_chunks;         /* mixed path: chunks of parameter sets the last call ran in (the
                             sets' digit images are built for one chunk at a time, at most
                             40 GiB of them; 1 when every set fits)                            */
  int tuned;              /* 1 if the launch shape of the last call (column_split, wide_tile) was
                             chosen by the autotuner: the candidate shapes timed on short
                             probes of the call's own pairs, the fastest kept per (precision, N,
                             integrator, pair count, L) for the life of the process; 0 for a fixed
                             rule (a forced split mode, more pairs than SMs, N <= 32, a mixed
                             cluster of ceil(N / 32) or ceil(N / 16) CTAs)                      */
  int sweep_split;        /* 1 if the reverse sweep of the last trh_curve_jacobian /
                             trh_rfactor_grad call ran its recompute and adjoint kernels as
                             two-CTA clusters (column split, N <= 64), else 0                  */
} trh_stats;

/* Create a context for one beam set and method. Validates and copies `p` (the caller may free
 * its arrays afterwards), allocates device tables for one parameter set (the default structure
 * p->atoms, p->dw) and builds the host-side geometry (reciprocal rods, difference map U_jk ->
 * u_{g_j - g_k}, kick positions of the integrator).
 * Errors: TRH_EINVAL (see field comments), TRH_EUNSUPPORTED (N > 256 on either path; on the
 * mixed path above 128 beams a beam set whose grid of differences (m1_j - m1_k, m2_j - m2_k)
 * has a bounding box of more than 1536 entries, or a device that cannot hold a cluster of
 * ceil(N / 16) CTAs; RK4 or the conventional method on the mixed path), TRH_ENOMEM, TRH_ECUDA.
 * On error *out is NULL. */
int trh_create(trh_ctx** out, const trh_problem* p);

/* Replace the context's parameter sets: n_sets structures sharing the beam set, species table
 * and slab. `atoms` is [n_sets][n_atoms][3] and `dw` is [n_sets][n_atoms], host or device
 * memory (both on the same side); `dw` may be NULL (every set uses the problem's dw). Host
 * inputs are validated (z <= 0, dw >= 0); device inputs are copied as given. The copies are
 * enqueued on the stream of the context's last call (the legacy default stream before the
 * first), after that call's work, without synchronising; the next call's stream waits for them.
 * A device input must therefore be ready in that stream's order. Builds nothing yet: the potential
 * tables are rebuilt by the next trh_rocking_curve (Section 3.4: one U(z) serves every angle
 * of a set), so calling this with unchanged data forces a rebuild.
 * Errors: TRH_EINVAL (n_sets < 1, z > 0, dw < 0), TRH_ENOMEM, TRH_ECUDA. */
int trh_set_structure(trh_ctx* ctx, int n_sets, const double* atoms, const double* dw);

/* Rocking curves of every parameter set at n_angles incident directions (Section 2.1: eta as a
 * function of theta0 and theta1).
 *   theta0, theta1 : [n_angles] glancing angle and azimuth (from a1), degrees; host or device.
 *   rho_out        : [n_sets][n_angles][N] complex128 rho(0); host or device; may be NULL.
 *   eta_out        : [n_sets][n_angles][N] float64 intensities; host or device; may be NULL.
 *   stream         : cudaStream_t (NULL = legacy default stream).
 * Steps per set: potential table at every kick position (one kernel), then one kernel that
 * integrates every (set, angle) pair from z_e to 0 with the RHST and assembles rho and eta.
 * TRH_FP64 computes everything in binary64. TRH_MIXED computes U*Q on the tensor cores (four
 * 8-bit fixed-point digits per operand in BF16, FP32 accumulators that never round), keeps Q and
 * P in double-float (pairs of FP32, about 48 significant bits), inverts Q for the RHST in FP32
 * and applies the inverse in double-float, and assembles rho in binary64 with one step of
 * iterative refinement.
 * Errors: TRH_EINVAL (n_angles < 1, theta0 outside (0, 90)), TRH_EGRAZING, TRH_ESINGULAR (the
 * outputs of the failing pairs are NaN; trh_query names the first one), TRH_ETIMEOUT,
 * TRH_ECUDA. */
int trh_rocking_curve(trh_ctx* ctx, int n_angles, const double* theta0, const double* theta1,
                      void* rho_out, double* eta_out, void* stream);

/* ---- bulk layer ---------------------------------------------------------------------------
 * Section 2.2 (end): below the surface region the crystal is an ideal bulk whose reflection
 * converges quickly with depth; it is computed once, the computation stopping when it has
 * converged, and reused. Here the bulk is periodic in z with period `period` (A) below z_e; one
 * period's atoms are given with z relative to the top of the period, in (-period, 0]. Its
 * boundary condition at z_e is X = P Q^{-1} of the solutions that belong in the bulk (c' = X c),
 * the fixed point of one period's map (integrate [I; X] over the period with the context's
 * splitting scheme, `steps_per_period` steps, and normalise), iterated from X = i Gamma until the
 * largest entry changes by less than `tol` (<= 0 selects 1e-12) relative to the largest entry,
 * at most `max_periods` times. The potential of a period includes the images of its atoms
 * within 8 A. Slab integrations then start from [I; X] instead of [I; i Gamma]; the slab's own
 * atoms (set by trh_create / trh_set_structure) should include the bulk atoms near z_e whose
 * potential reaches into the slab. X is computed on the binary64 path (N <= 64) once per set of
 * directions and reused while the directions stay the same (every path, the reverse sweep and
 * batches use it). n_atoms = 0 removes the bulk.
 * Errors: TRH_EINVAL, TRH_EUNSUPPORTED (N > 64, RK4 or the conventional integrator); a later call
 * returns TRH_ENOCONV if some direction did not converge. */
int trh_set_bulk(trh_ctx* ctx, int n_atoms, const double* atoms, const double* dw,
                 const int* species, double period, int steps_per_period, int max_periods,
                 double tol);

/* ---- CTAs per (set, angle) pair --------------------------------------------------------------
 * The kick and the drift act column by column (W_c = U Q_c, Section 3.4), so on the mixed path
 * and on the FP64 path (N <= 64, SP4/SP6) the columns of one pair can be shared by the two CTAs
 * of a thread-block cluster, 32 each. They exchange the Varah row sums once per step, the column
 * halves of Q and P at every RHST (Section 3.2: both CTAs hold the whole [Q; P] for it) and at
 * the end (CTA 0 assembles rho). This shortens a pair's critical path but takes two SMs per pair:
 * TRH_SPLIT_AUTO (the default) lets the autotuner choose when N > 32 and the call has at most
 * as many pairs as SMs (both forms timed on probes of the call's pairs at 2 and 12 steps, their
 * times at the call's L extrapolated, the faster kept for that shape; trh_stats.tuned), TRH_SPLIT_OFF never splits, TRH_SPLIT_ON whenever N > 32
 * (trh_curve_jacobian's forward splits when its pairs fit on half the SMs, and so do its reverse
 * sweep's recompute and adjoint kernels: trh_stats.sweep_split). Results are identical either way:
 * every column sees the same arithmetic, and the row sums are added in the same fixed order, so
 * the RHST decisions coincide. Batches (trh_batch_*) always run one CTA per pair. A wait for the
 * other CTA that runs out (about 2 s) ends the pair with TRH_ETIMEOUT.
 * Errors: TRH_EINVAL (mode not one of the three). */
enum trh_split_mode { TRH_SPLIT_AUTO = 0, TRH_SPLIT_OFF = 1, TRH_SPLIT_ON = 2 };
int trh_set_column_split(trh_ctx* ctx, int mode);

/* ---- asynchronous calls ------------------------------------------------------------------------
 * Not a step of the method (the paper's program is synchronous): a host-side convenience. With
 * on != 0, trh_rocking_curve returns as soon as its work is enqueued on `stream` instead of
 * waiting for it to read the per-pair status words, so that back-to-back calls queue on the
 * device without a host stall per call. Outputs in device memory, or in pinned host memory
 * (copied with cudaMemcpyAsync), are ready in stream order; outputs in pageable host memory still
 * make the call wait for its copies. The per-pair counters of trh_stats (rhst_total, n_bad,
 * first_bad_*), and ms_potential and ms_integrate, belong to the last call and are completed by
 * trh_query, which waits for that call's work; a failing pair is then reported only there
 * (n_bad, first_bad_status, and trh_last_error()), not by the call's return code, which covers
 * argument and enqueue errors. A later call replaces the counters of an earlier one that was not
 * queried. on = 0 (the default) restores the synchronous behaviour: the call waits and returns
 * the first failing pair's code. The gradient calls are synchronous in either mode.
 * Errors: TRH_EINVAL (NULL context), TRH_ECUDA. */
int trh_set_async(trh_ctx* ctx, int on);

/* ---- device memory of the mixed path ---------------------------------------------------------
 * The mixed path multiplies by U(tau) on the tensor cores from fixed-point digit images of U at
 * every kick position, built once per parameter set from the binary64 potential table (Section
 * 3.4: one U(z) serves every angle) and read by every angle's integration: 131.6 KB per node at
 * N = 61 (1.58 GB per set at 2000 slices), 512 KB per node at N = 121 (6.1 GB per set). The
 * images of at most `bytes` (0 selects the default, 40 GiB) are kept at once: a call whose sets
 * need more builds them for a chunk of sets, integrates those sets, then moves to the next chunk
 * (trh_stats.set_chunks). Results do not depend on the chunking. At least one set is always
 * taken, whatever the budget.
 * Errors: TRH_EINVAL (ctx is NULL). */
int trh_set_image_budget(trh_ctx* ctx, size_t bytes);

/* ---- reverse analysis ---------------------------------------------------------------------
 * The paper's motivation (Section 1) is the reverse analysis of measured curves: a structure
 * x* = argmin_x |d - F(x)|^2 over structural parameters x. The calls below give the gradient of
 * that objective with respect to atomic z coordinates and Debye-Waller factors, by the adjoint
 * (reverse sweep) of Algorithm 1 on the binary64 path, so that gradient-based searches can use
 * it. The objective (the paper prints none) is the R-factor of the specular curve:
 *   eta~(theta) = eta_1(theta) / sum_theta' eta_1(theta'),   R = sum_theta (eta~ - t~)^2,
 * with t~ the target curve normalised the same way. The RHST matrices are constants of the
 * reverse map (rho is invariant under Z -> Z T, Section 3.2). Memory is bounded by
 * checkpoints: the forward pass stores [Q; P] every `ckpt_every` steps and the reverse sweep
 * recomputes one segment at a time, up to two segments ahead of the adjoint (three segment
 * slots, or one per segment when there are fewer). Device scratch per (set, angle) pair, in bytes:
 *   16 N^2 (2 (L / C + 1) + 3 (2 (s C + 1) + 2 C) + 2) + 12 C,   C = ckpt_every,
 * s = kicks per step, about 164 MB at N = 61, L = 2000, C = 64 (sp4, s = 6); for 64 < N <= 256
 * (the wide reverse sweep, state in global memory)
 *   16 N^2 (2 (L / C + 1) + (s C + 1) + 2 C + 6) + 4 C.
 * N <= 64: on a TRH_FP64 context everything runs on the binary64 path; on a TRH_MIXED context
 * the forward pass (curve, R and the checkpoints, binary64 values of its double-float state)
 * runs on the mixed path and every segment is recomputed on the binary64 path from its
 * checkpoint, so the reverse map differentiates the trajectory it recomputes; the adjoint is
 * binary64 too, and only the contraction Ubar = -c Pbar Q^H (summed into the gradient, not
 * carried) runs on the tensor cores as four-digit BF16 products, each entry to FP32 precision.
 * The gradient then carries a relative error of ~1e-7 (the 1e-5 bar of the tests with margin). 64 < N <= 256: the forward pass, the recompute
 * and the adjoint all run on the binary64 wide kernels for either precision (the beam set's
 * distinct differences must fit shared memory twice: about 2000 at most). */

/* Declare the fit parameters: the z coordinates of atoms free_atoms[0..n_free-1] (distinct
 * indices into the context's atoms) and n_classes Debye-Waller classes, dw_class[a] in
 * [0, n_classes) for an atom whose B is the class's parameter, -1 for a fixed B (dw_class is
 * [n_atoms], host; may be NULL when n_classes = 0). Every class needs at least one atom; at most
 * 64 atoms may carry a parameter. ckpt_every <= 0 selects 64 steps per checkpoint.
 * Errors: TRH_EINVAL, TRH_EUNSUPPORTED (more than 64 atoms), TRH_ENOMEM, TRH_ECUDA. */
int trh_set_fit(trh_ctx* ctx, int n_free, const int* free_atoms, int n_classes,
                const int* dw_class, int ckpt_every);

/* Jacobian of the specular intensity eta_1 with respect to the fit parameters, for every
 * parameter set and angle.
 *   theta0, theta1 : [n_angles] degrees; host or device.
 *   eta_out        : [n_sets][n_angles][N] float64 intensities; host or device; may be NULL.
 *   jac_out        : [n_sets][n_angles][n_free + n_classes] float64: d eta_1 / d z of each free
 *                    atom (1/A), then d eta_1 / d B of each class (1/A^2); host or device.
 *   stream         : cudaStream_t (NULL = legacy default stream); synchronised before return.
 * Errors: as trh_rocking_curve, TRH_EINVAL before trh_set_fit, TRH_EUNSUPPORTED (RK4 or the
 * conventional integrator; above 64 beams, too many distinct differences). */
int trh_curve_jacobian(trh_ctx* ctx, int n_angles, const double* theta0, const double* theta1,
                       double* eta_out, double* jac_out, void* stream);

/* R-factor of each parameter set's specular curve against `target` ([n_angles] float64, >= 0,
 * not all zero; host or device; shared by all sets) and its gradient.
 *   R_out  : [n_sets]; host or device; may be NULL.
 *   dR_dz  : [n_sets][n_free] dR/dz of the free atoms (1/A); host or device.
 *   dR_dB  : [n_sets][n_classes] dR/dB of the classes (1/A^2); host or device.
 * Errors: as trh_curve_jacobian, and TRH_EINVAL for a negative or all-zero host target. */
int trh_rfactor_grad(trh_ctx* ctx, int n_angles, const double* theta0, const double* theta1,
                     const double* target, double* R_out, double* dR_dz, double* dR_dB,
                     void* stream);

/* ---- batches ----------------------------------------------------------------------------------
 * Many rocking curves of different beam sets (one context each, any N) and parameter sets in as
 * few launches as possible (Section 3.4's parallelisation over angles, extended across problems):
 * all binary64 work items (context, set, angle) with N <= 64 go to one persistent kernel and all
 * with 64 < N <= 256 (and all RK4 items) to a second one, and all TRH_MIXED items to a third;
 * each persistent CTA takes items from an atomic counter in decreasing-cost order (N^3 L,
 * longest first), so uneven beam counts balance across the SMs. The first trh_batch_run executes eagerly
 * and captures the same launch sequence in a CUDA graph; later runs replay the graph (the
 * potential tables of contexts whose structure changed are rebuilt before the replay, and the
 * plan and graph are rebuilt when a context's device tables moved). The wide kernel's tile edge
 * comes from the autotuner (trh_stats.wide_tile). */
typedef struct trh_batch trh_batch;

/* Empty batch. Errors: TRH_EINVAL (out is NULL). */
int trh_batch_create(trh_batch** out);

/* Queue all parameter sets of `ctx` at n_angles directions. theta0, theta1 ([n_angles], degrees),
 * rho_out ([n_sets][n_angles][N] complex128) and eta_out ([n_sets][n_angles][N] float64) must be
 * DEVICE memory; the batch keeps the pointers (not the data) and the context, which must outlive
 * the batch. Angle values may change between runs; their count may not.
 * Errors: TRH_EINVAL (NULL, n_angles < 1, host pointers). */
int trh_batch_add(trh_batch* batch, trh_ctx* ctx, int n_angles, const double* theta0,
                  const double* theta1, void* rho_out, double* eta_out);

/* Run every queued job on `stream` (cudaStream_t, NULL = legacy default stream) and synchronise.
 * Outputs and errors as trh_rocking_curve; trh_batch_query then reports the batch's counters
 * (first_bad_set = job index and first_bad_angle = pair index within that job). */
int trh_batch_run(trh_batch* batch, void* stream);

/* Counters of the last trh_batch_run. Errors: TRH_EINVAL (NULL arguments). */
int trh_batch_query(const trh_batch* batch, trh_stats* out);

/* Free the batch (not its contexts). NULL is accepted. Synchronises the device. */
void trh_batch_destroy(trh_batch* batch);

/* Counters of the last call (see trh_stats); after an asynchronous call (trh_set_async) this
 * waits for that call's work and completes its per-pair counters. Errors: TRH_EINVAL (NULL
 * arguments), TRH_ECUDA. */
int trh_query(const trh_ctx* ctx, trh_stats* out);

/* Static string naming a status code; never NULL. */
const char* trh_strerror(int status);

/* Message of the last failing call on the calling thread ("" if none); valid until the next
 * call on this thread. */
const char* trh_last_error(void);

/* Free the context and its device memory. NULL is accepted. Synchronises the device. */
void trh_destroy(trh_ctx* ctx);

/* Rocking curve of one structure on the binary64 path without any device allocation.
 *
 * The paper has no counterpart: this entry exists for callers that cannot call cudaMalloc when
 * they need a curve: code that runs under a fixed device-memory budget which must not grow,
 * plug-ins whose host application owns and hands out all device memory itself, and loops where
 * cudaMalloc's implicit device synchronisation is not acceptable. The caller passes device
 * buffers for the angles and the outputs; the potential table,
 * scattering factors, geometry tables and status words live in one fixed-size device array of
 * 16 MiB inside this library, which every GPU that loads the library keeps until process exit.
 *   p              : problem as for trh_create (host memory); precision must be TRH_FP64,
 *                    integrator TRH_SP4 or TRH_SP6, N <= 64, at most 256 atoms.
 *   theta0, theta1 : [n_angles] degrees, DEVICE memory.
 *   rho_out        : [n_angles][N] complex128, DEVICE memory.
 *   eta_out        : [n_angles][N] float64, DEVICE memory.
 *   stream         : cudaStream_t (NULL = legacy default stream); the work is enqueued on it and
 *                    the call returns without synchronising.
 * The first call on each device looks up the array's device address (cudaGetSymbolAddress); make
 * that first call before any stream capture on the device. No call allocates or frees device
 * memory. All calls share the array and it keeps the last call's contents (nothing in it needs
 * to start at zero), so calls whose work overlaps on the GPU race: serialise them on one stream.
 * Results equal those of trh_rocking_curve with TRH_FP64 for the same problem and angles; a
 * (set, angle) whose RHST or final solve hits a singular pivot yields NaN outputs.
 * Errors: TRH_EINVAL (bad arguments, or a problem whose tables exceed the 16 MiB array: the
 * message from trh_last_error() states the bytes needed), TRH_ECUDA. */
int trh_rocking_curve_noalloc(const trh_problem* p, int n_angles, const double* theta0,
                              const double* theta1, void* rho_out, double* eta_out, void* stream);

#ifdef __cplusplus
}
#endif
#endif /* TRHEED_H */
