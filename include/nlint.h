/*
 * nlint — free-space Coulomb / dipole-dipole convolution on a uniform grid by the
 * phase-space quadrature + NUFFT method of Jiang, Greengard & Bao (arXiv 1311.4120,
 * Algorithm 1, Section 3.2), on one NVIDIA GB300 (sm_103a).
 *
 * What the library computes (eq. gpe, eq. gpe2, eq. 3.2, eq. 3.7, Remark 3.3):
 *   grid      x_i = -L/2 + i h, h = L/n, i = 0..n-1 on every axis (d = 2 or 3),
 *             arrays in C order, last index fastest: (i_z, i_y, i_x) or (i_y, i_x);
 *   nodes     k_j = r (sin t cos p, sin t sin p, cos t) in 3D, r (cos p, sin p) in 2D, with
 *             r Gauss-Legendre on [0, P], t Gauss-Legendre on [0, pi], p = 2 pi l / N_phi;
 *   weights   W_j = (2 pi)^{-d} w_r w_t sin(t) w_p |k_j|^{d-1} U_hat(k_j)     (eq. 3.7)
 *             U_hat = 1/|k|^2 (3D Coulomb), 1/|k| (2.5D Coulomb),
 *             -(m.n) + 3 (n.k)(m.k)/|k|^2 (3D dipole, eq. dipkerneldF; m = n: dipkernelF),
 *             -alpha + 3 [(n_p.k)(m_p.k) - n_3 m_3 |k|^2] / (2|k|) (2.5D dipole,
 *             eq. dipkernelF2dd; n_p = (n_1, n_2); m = n: dipkernelF2d)   (table int3dd)
 *   type 2    rho_hat_j = h^d sum_i rho_i exp(-i k_j . x_i)                  (eq. 3.2)
 *   type 1    u_i = Re sum_j W_j rho_hat_j exp(+i k_j . x_i)                 (eq. 3.7)
 *   energy    E = (lambda / 2) h^d sum_i u_i rho_i                    (Remark 3.3)
 * Both sums are evaluated by NUFFTs (Section 2) to the plan's tolerance.
 *
 * Canonical node order (used by nlint_type2 / nlint_type1): j = (a N_theta + b) N_phi + c
 * in 3D and j = a N_phi + c in 2D (a radial, b polar, c azimuthal index).
 *
 * Conventions for every entry point:
 *   - Device pointers are CUDA device (or managed) addresses on the plan's device, owned by
 *     the caller, in the plan's precision (float or double; complex values interleaved).
 *     They must stay valid until the work queued on `stream` has finished.
 *   - `stream` is a cudaStream_t passed as void* (NULL = the legacy default stream).  Work
 *     is queued on it; nothing synchronises the host unless a host output is requested.
 *     An Algorithm 1 plan clears its spreading grid on an internal stream while the
 *     interpolation runs: that work is forked from `stream` (after everything queued on it)
 *     and joined back before the spreading, by events, so the evaluation stays ordered on
 *     `stream` and can be captured into a CUDA graph.
 *   - Return value: NLINT_OK or a negative status; nlint_last_error() then returns a
 *     message for the calling thread.  No C++ exception crosses this interface.
 *   - A plan is not re-entrant: one evaluation at a time per plan (its workspaces are
 *     reused).  Different plans may run concurrently on different streams.
 */
#ifndef NLINT_H
#define NLINT_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct nlint_plan_s *nlint_plan;
typedef struct nlint_batch_s *nlint_batch;

enum { NLINT_COULOMB = 0, NLINT_DIPOLE = 1 };
enum { NLINT_FP32 = 0, NLINT_FP64 = 1 };
enum {
    NLINT_OK = 0,
    NLINT_EINVAL = -1,       /* bad argument (message says which)                  */
    NLINT_ENOMEM = -2,       /* device or host allocation failed                    */
    NLINT_ECUDA = -3,        /* a CUDA call failed (message carries CUDA's string)  */
    NLINT_ETIMEOUT = -4,     /* a bounded device-side wait gave up                  */
    NLINT_EUNSUPPORTED = -5  /* valid request outside what this build implements    */
};

/* Full set of plan parameters.  nlint_params_default() fills every field; zero in an
 * optional field means "choose from the other fields". */
typedef struct nlint_params {
    int d;               /* 2 or 3                                                      */
    int64_t n;           /* grid points per axis, even, >= 8                            */
    double L;            /* box side; the box is [-L/2, L/2)^d                          */
    int kernel;          /* NLINT_COULOMB or NLINT_DIPOLE (3D only)                     */
    double axis[3];      /* dipole axis n (normalised internally); ignored for Coulomb  */
    int64_t n_r, n_theta, n_phi; /* node counts; 0 = default for n (n_theta ignored in 2D) */
    double P;            /* radial cutoff; 0 = pi / h (the Nyquist radius of the grid)   */
    double eps;          /* NUFFT tolerance; picks the precision and spreading width     */
    int precision;       /* -1 = from eps (eps >= 1e-7 -> FP32), else NLINT_FP32/FP64     */
    int w;               /* spreading width in fine cells; 0 = from eps                  */
    double sigma;        /* oversampling factor of the fine grid; 0 = 2                  */
    int device;          /* CUDA device ordinal; -1 = current device                     */
    double axis2[3];     /* second dipole orientation m (eq. dipkerneldF, dipkernelF2dd);
                            zero = same as axis (one orientation)                        */
    double alpha;        /* 2.5D dipole constant alpha (eq. dipkernelF2d); 0 in 3D         */
    int max_sub;         /* nodes per interpolation/spreading CTA; 0 = 1024 (FP32), 512 (FP64) */
    int crowd_min;       /* bins above this many nodes sum their tiles in FP64; 0 = 4096    */
    /* Algorithm 2 (Section 3.3): algorithm = 2 evaluates u = I_1 + I_2 (eq. 3.9) with the
     * partition p_3(k) = exp(-|k|^2/a) (eq. 3.10, 3D) or p_2(k) = erfc(12 (|k| - (R0+R1)/2) /
     * (R1-R0)) / 2 (eq. 3.12, 2D): I_1 by the zero-padded FFT on the fine grid (n_fine >= 2n)
     * with the multiplier U_hat (1 - p) on |k| <= P, I_2 by the NUFFT path on nodes of radius P2
     * with weights W_j p(k_j).  n_r, n_theta, n_phi are then I_2's node counts (0 = 32x32x64 /
     * 40x40x80 in 3D, 48x96 / 64x128 in 2D for FP32 / FP64).                                 */
    int algorithm;       /* 1 (default, also for 0) or 2                                      */
    double pu_a;         /* 3D: a of p_3; 0 = (11.8 / L)^2                                    */
    double pu_r0, pu_r1; /* 2D: R0 < R1 of p_2; 0 = 12 / L and 160 / L                        */
    double P2;           /* radius of I_2's nodes; 0 = min(P, 6.1 sqrt(a)) (3D), min(P, R1) (2D) */
    /* Bins of stencil-origin cells that one interpolation / spreading CTA covers with a
     * shared-memory tile of bin + w - 1 cells per axis.  0 = automatic; 3D: 1 = 8x8x8,
     * 2 = 4x8x8 (FP64 only), 3 = 8x16x16 (FP32 only), 4 = 16x16x16 (FP32 only); 2D: 1 =
     * 16x16.  A shape whose tile does not fit in shared memory at the plan's width is
     * NLINT_EUNSUPPORTED (automatic: the smallest shape is taken instead).                  */
    int bin_shape;
    /* FFT pass schedules (FP32 plans; ignored in FP64): bit set = the two-stage radix schedule
     * (radix 2^ceil(a/2) x 2^floor(a/2) on lines of 2^a >= 128 points, one exchange through
     * shared memory per line instead of two) for, bit 0: the column passes, 1: the row passes,
     * 2: the first inverse row pass (fold), 3: the real-data column passes along the slowest
     * axis; other lines have one schedule.  0..15; 0 = default.                              */
    int fft_sched;
} nlint_params;

/* Read-only description of a plan. */
typedef struct nlint_info {
    int d, precision, w, kernel;
    int64_t n, n_fine, n_nodes, n_half_nodes;
    int64_t n_r, n_theta, n_phi;
    double L, h, P, sigma, beta;
    size_t workspace_bytes; /* device bytes owned by the plan */
    int64_t n_bins;         /* non-empty bins of the sorted half node set              */
    int64_t n_subproblems;  /* CTAs of one interpolation / spreading launch             */
    int64_t n_crowd_bins;   /* bins whose tiles are summed in FP64 (FP32 plans)         */
    int bin[3];             /* bin extent per array axis, in fine cells                 */
    int device;             /* CUDA device ordinal the plan lives on                    */
    int algorithm;          /* 1 or 2; for 2 the node fields describe I_2's nodes       */
    double pu_a, pu_r0, pu_r1, P2; /* Algorithm 2's partition parameters (0 if unused)  */
    int toeplitz;           /* 1 once nlint_plan_toeplitz has precomputed K_hat          */
    int bin_shape;          /* the bin shape in use (see nlint_params.bin_shape)         */
    int fft_sched;          /* the FFT pass schedules in use (nlint_params.fft_sched)    */
} nlint_info;

/* Fill *p with defaults (d = 3, Coulomb, eps = 1e-6, everything else automatic). */
void nlint_params_default(nlint_params *p);

/* Build a plan: nodes and weights in FP64 on the host, sorted into fine-grid tiles, uploaded
 * once; device workspaces allocated.  Algorithm 1 steps 1-3 (Section 3.2).
 * dipole_axis: 3 doubles for NLINT_DIPOLE (must be non-zero; normalised), NULL for Coulomb;
 * one orientation, alpha = 0.  nlint_plan_create_ex also takes a second orientation (axis2)
 * and the 2.5D constant alpha.
 * Errors: NLINT_EINVAL (d not 2/3, n odd or < 8, L <= 0, zero axis), NLINT_EUNSUPPORTED
 *         (fine grid above 2048 per axis), NLINT_ENOMEM, NLINT_ECUDA. */
int nlint_plan_create(int d, int64_t n, double L, int kernel, const double *dipole_axis,
                      double eps, nlint_plan *out);
int nlint_plan_create_ex(const nlint_params *p, nlint_plan *out);
int nlint_plan_info(nlint_plan plan, nlint_info *info);
/* Device-side waits of the plan's kernels (the interpolation's wait for its TMA tile load) give
 * up after a bounded number of polls and set a status word instead of hanging.  This call
 * synchronises the plan's device, reads and clears that word: NLINT_ETIMEOUT if a wait ran out
 * since the last check (the evaluation that saw it produced invalid results), else NLINT_OK.
 * Errors: NLINT_EINVAL (NULL plan), NLINT_ECUDA. */
int nlint_plan_check(nlint_plan plan);
void nlint_plan_destroy(nlint_plan plan); /* NULL is a no-op; waits for the plan's work */

/* u = U * rho on the grid (Algorithm 1 steps 4-5: type-2 NUFFT, multiply by W_j, type-1
 * NUFFT; for an Algorithm 2 plan, u = I_1 + I_2 of eq. 3.9).  rho_dev, u_dev: n^d reals in the
 * plan precision; they may not alias. */
int nlint_eval(nlint_plan plan, const void *rho_dev, void *u_dev, void *stream);

/* nlint_eval followed by the energy (lambda/2) h^d sum u rho, written as one double to
 * E_dev (device).  The sum is taken in FP64 with compensated (Neumaier) partial sums in a
 * fixed order, so repeated calls give identical results. */
int nlint_eval_energy(nlint_plan plan, const void *rho_dev, void *u_dev, double lambda,
                      double *E_dev, void *stream);

/* E = (lambda/2) h^d sum u rho for caller-supplied rho and u (Remark 3.3).  E_dev (device
 * double) and/or E_host may be NULL; a non-NULL E_host synchronises `stream`. */
int nlint_energy(nlint_plan plan, const void *rho_dev, const void *u_dev, double lambda,
                 double *E_dev, double *E_host, void *stream);

/* Energy without the potential: E = (lambda/2) sum_j W_j |rho_hat_j|^2 (eq. 3.7 substituted
 * into the trapezoidal energy of Remark 3.3; for the discrete operator this equals
 * (lambda/2) h^d sum_i u_i rho_i up to the NUFFT tolerance).  Runs the type-2 half of the path
 * only (forward FFT passes and interpolation), about half the work of nlint_eval_energy.
 * E_dev (device double) and/or E_host may be NULL; a non-NULL E_host synchronises `stream`.
 * The sum is compensated and taken in a fixed order. */
int nlint_energy_only(nlint_plan plan, const void *rho_dev, double lambda, double *E_dev,
                      double *E_host, void *stream);

/* Precomputed Toeplitz form of the same discrete operator.  u = K rho with the translation-
 * invariant kernel K(dx) = h^d Re sum_j W_j exp(i k_j . dx) (eq. 3.2 substituted into eq. 3.7).
 * nlint_plan_toeplitz computes K on dx in [-N, N)^d cells with 2^d type-1 NUFFTs of the plan
 * itself, and its DFT K_hat on the plan's oversampled grid (n_fine >= 2N, so the circular
 * convolution equals the linear one on the grid); it allocates K_hat (real, Hermitian half) and
 * synchronises `stream`.  nlint_eval_toeplitz then computes u (and E if E_dev != NULL) with the
 * FFT passes only: zero-padded forward FFT of rho, multiply by K_hat (between the forward and
 * inverse transforms along x, in one row pass), inverse FFT, crop.  The result equals nlint_eval_energy's to the NUFFT
 * tolerance; no interpolation or spreading runs per evaluation.  This form is not in the paper:
 * it follows from the operator's Toeplitz structure. */
/* Both return NLINT_EUNSUPPORTED for an Algorithm 2 plan (whose I_1 part already is an FFT
 * convolution).  nlint_energy_only does the same. */
int nlint_plan_toeplitz(nlint_plan plan, void *stream);
int nlint_eval_toeplitz(nlint_plan plan, const void *rho_dev, void *u_dev, double lambda,
                        double *E_dev, void *stream);

/* End-to-end form with HOST buffers: copies rho_host to the device, evaluates u and E,
 * copies u back to u_host and E to *E_host (E_host may be NULL), and synchronises
 * `stream`.  Pinned host memory gives the fastest copies. */
int nlint_eval_host(nlint_plan plan, const void *rho_host, void *u_host, double lambda,
                    double *E_host, void *stream);

/* Streaming form of nlint_eval_host for many densities: evaluates rho_host[k] -> u_host[k]
 * and E_host[k] for k < count (each array n^d values of the plan's precision in host memory;
 * E_host may be NULL: no energies), overlapping the copies with the evaluations.  The copy of
 * density k+1 to the device and the copy of u_{k-1} back to the host run on two plan-owned
 * streams while density k is evaluated on `stream`, through two device staging buffers each
 * way; events order every copy against the evaluations that use its buffer.  The copies are
 * forked from `stream` after the work already queued on it, and the call returns after every
 * copy has finished (it synchronises `stream`).  Pinned host memory lets the copies overlap;
 * pageable memory gives the same results with serialised copies.  Each u_host[k], E_host[k]
 * equals what nlint_eval_host gives for rho_host[k].  The paper has no counterpart: it is the
 * serving form of the same evaluation.  Errors: NLINT_EINVAL (count <= 0, NULL arrays or
 * entries), NLINT_ECUDA (including a failed allocation of the staging buffers, which are
 * allocated on the first call and kept by the plan). */
int nlint_eval_host_many(nlint_plan plan, int count, const void *const *rho_host,
                         void *const *u_host, double lambda, double *E_host, void *stream);

/* Stage entry points.  nlint_type2: rho (n^d reals) -> rho_hat_dev (n_nodes complex, the
 * canonical node order, eq. 3.2).  nlint_type1: c_dev (n_nodes complex, canonical order)
 * -> u_dev = Re sum_j c_j exp(+i k_j . x) (eq. 3.7 with c_j in place of W_j rho_hat_j).
 * For an Algorithm 2 plan the nodes are I_2's (and nlint_plan_nodes' W includes p(k_j)). */
int nlint_type2(nlint_plan plan, const void *rho_dev, void *rho_hat_dev, void *stream);
int nlint_type1(nlint_plan plan, const void *c_dev, void *u_dev, void *stream);

/* Node data in canonical order, FP64, for inspection: k_host (n_nodes x d, (k_x,k_y[,k_z]))
 * and W_host (n_nodes); either may be NULL. */
int nlint_plan_nodes(nlint_plan plan, double *k_host, double *W_host);

/* Per-stage timing: when enabled, each evaluation records CUDA events between its stages
 * on the evaluation stream; nlint_stage_times returns the milliseconds of the last
 * evaluation (synchronising on its final event) and the stage names. */
int nlint_set_stage_timing(nlint_plan plan, int enable);
int nlint_stage_times(nlint_plan plan, float *ms, const char **names, int max_stages,
                      int *n_stages);

/* Autotuner.  For the plan described by *in and a target relative L-inf error `tol` of u,
 * picks (1) the smallest spreading width w whose error, measured on the device against an FP64
 * plan with the widest stencil (same grid, nodes, cutoff and kernel) on a seeded probe
 * density with content up to the grid's Nyquist radius, is at most tol/2, (2) of that width and
 * the next one the fastest, each with its fastest bin shape among those compiled for the
 * precision and dimension whose tile fits in shared memory (evaluation time by CUDA events),
 * (3) for that width and shape the fastest subproblem size (max_sub) among 256..2048, and (4)
 * for FP32 plans the FFT pass schedules (nlint_params.fft_sched), one pass class at a time,
 * each kept when the evaluation's FFT stages (its stage events) measured at least 1 % faster.
 * *out = *in with w, bin_shape, max_sub, fft_sched and the precision (from tol when
 * in->precision is -1) filled in; rep (may be NULL) reports the choice, its measured error
 * and time.  The choice is cached as one JSON object per line in
 * cache_path (NULL: $NLINT_TUNE_CACHE; neither: no cache); a cached key skips measurement.
 * Synchronous; creates and destroys several plans (NLINT_ENOMEM etc. pass through). */
typedef struct nlint_tune_report {
    int w, max_sub;
    double err;      /* measured relative L-inf error of the chosen width on the probe */
    double ms;       /* median evaluation time of the choice                           */
    int from_cache;  /* 1: read from the cache, nothing measured                      */
    int bin_shape;   /* chosen bin shape (nlint_params.bin_shape)                      */
    int w_alt;       /* the other width timed in (2), also within tol/2 (0: none)      */
    double err_alt;  /* its measured error                                             */
    int fft_sched;   /* chosen FFT pass schedules (nlint_params.fft_sched), step (4)    */
} nlint_tune_report;
int nlint_autotune(const nlint_params *in, double tol, const char *cache_path, nlint_params *out,
                   nlint_tune_report *rep);

/* Batch autotuner, for `count` densities evaluated together by nlint_batch_*: members with the
 * same geometry, kernel and precision form a class (dipoles of any orientation share one: the
 * width's error does not depend on it), each class is tuned once by nlint_autotune on its first
 * member (its width for `tol`, and its own fastest bin shape and subproblem size when evaluated alone),
 * and the whole batch graph (nlint_batch_create with `branches`, on each member's probe density)
 * is then timed with three parameter sets: (0) every class at its own fastest decomposition and
 * width, (1) every class at the default decomposition (bin_shape 0, max_sub 0) and its tuned
 * width, (2) the default decomposition at each class's other timed width (w_alt, also within
 * the tolerance).  Evaluated alone a small grid gains from many small subproblems (and a width
 * from its lane layout), but in a batch the GPU is already filled by the other members and those
 * extra CTAs only add tile work, so the batch keeps whichever set measured fastest.
 * out[i] = in[i] with w, bin_shape, max_sub and precision filled in; member_reps (may be NULL)
 * holds count per-member reports of the chosen parameters (err from the class tuning, ms the
 * class's own time); rep (may be NULL) the batch choice and both times.  The class tunings use
 * the cache as nlint_autotune does; the batch timing is not cached.  Synchronous; creates and
 * destroys plans, a batch and count density/potential buffers on in[0]'s device.  Errors:
 * NLINT_EINVAL (count < 1, NULL in/out, members on different devices), and those of
 * nlint_autotune, nlint_plan_create_ex and nlint_batch_create. */
typedef struct nlint_batch_tune_report {
    int choice;     /* 0, 1 or 2: the parameter set kept (see above)                     */
    int classes;    /* distinct (geometry, kernel, precision) classes tuned              */
    double ms[3];   /* median batch evaluation time of each set (ms; 0: not timed, when  */
                    /* no class has another width, set 2 equals set 1)                   */
} nlint_batch_tune_report;
int nlint_autotune_batch(int count, const nlint_params *in, double tol, const char *cache_path,
                         int branches, nlint_params *out, nlint_tune_report *member_reps,
                         nlint_batch_tune_report *rep);

/* Batched evaluation of independent densities (Algorithm 1 applied to each), e.g. grids of
 * mixed sizes, kernels and precisions.  A plan whose Toeplitz kernel has been precomputed
 * (nlint_plan_toeplitz) before the batch graph is captured is evaluated in that form (the same
 * operator to the NUFFT tolerance, FFT passes only); the others by nlint_eval_energy.  nlint_batch_create: `count` plans (not owned: they
 * must outlive the batch), all on one device; `branches` concurrent streams inside the batch's
 * CUDA graph (0 = min(16, count)); plans are dealt to branches by a cost model.
 * nlint_batch_eval: rho[i], u[i] are plan i's device arrays (its n^d reals, its precision);
 * E_dev (may be NULL) receives count device doubles E_i = (lambda/2) h_i^d sum u_i rho_i.  The
 * first call, and any call whose pointers or lambda differ from the previous one, captures a
 * CUDA graph of all evaluations (one fork, one branch per stream, one join); every call then
 * launches that graph on `stream` (no host synchronisation).  Each u_i equals what
 * nlint_eval_energy gives for plan i alone, up to the order of the spreading's atomic
 * additions.  One batch evaluation at a time; the plans must not be used concurrently.
 * Errors: NLINT_EINVAL (NULL arguments, invalid plans, plans on different devices, a plan
 * listed more than once: its workspaces cannot serve two concurrent evaluations),
 * NLINT_ECUDA. */
int nlint_batch_create(int count, const nlint_plan *plans, int branches, nlint_batch *out);
int nlint_batch_eval(nlint_batch batch, const void *const *rho_dev, void *const *u_dev,
                     double lambda, double *E_dev, void *stream);
int nlint_batch_info(nlint_batch batch, int *count, int *branches, int64_t *kernels_per_eval);
void nlint_batch_destroy(nlint_batch batch); /* NULL is a no-op; waits for the device */

/* Energy E = (lambda/2) h^d sum_i u_i rho_i (h = L/n) of caller-owned device arrays, written
 * to the device double E_dev, for callers that cannot allocate device memory when they need
 * it (a framework that owns the whole device through its own pool, a thread that must not
 * call cudaMalloc/cudaFree because they synchronise the device, a fixed memory budget).  The
 * paper has no counterpart: it is a deployment variant of nlint_energy that needs no plan.
 *   d = 2 or 3; n points per axis; precision NLINT_FP32 (float arrays) or NLINT_FP64;
 *   rho_dev, u_dev: n^d values each on the current device; E_dev: one device double.
 * It allocates nothing: its scratch is a 1 MiB array in the library's device memory, held on
 * every device that loads the library until the process exits.  The first call on a device
 * looks up that array's device address (cudaGetSymbolAddress) with the device current; make
 * that first call before any stream capture.  The address is cached per device and CUDA
 * context: a call under another context of the device (after cudaDeviceReset, or with a
 * non-primary context current) looks it up again, so that call too belongs before capture.  Grids above 268435456 points (65536 partial
 * sums of 4096 points) are rejected with NLINT_EINVAL.  Every call reuses the same scratch:
 * calls that overlap on the GPU (other streams or host threads) race; serialise them.
 * Summation order is fixed by the inputs (deterministic), partial sums compensated in FP64. */
int nlint_energy_noalloc(int d, int64_t n, double L, int precision, const void *rho_dev,
                         const void *u_dev, double lambda, double *E_dev, void *stream);

/* Number of CUDA kernels this plan has launched so far, over all entry points (memsets and
 * copies are not counted).  Host-side counter; no synchronisation. */
int nlint_launch_count(nlint_plan plan, int64_t *count);

/* Thread-local message for the last failed call on this thread ("" if none). */
const char *nlint_last_error(void);

#ifdef __cplusplus
}
#endif
#endif /* NLINT_H */
