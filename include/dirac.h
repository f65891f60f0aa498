/*
 * dirac.h -- C ABI of the GB300 Dirac Lanczos propagator.
 *
 * The library advances a two-component spinor field on a uniform 2D grid by
 * the Lanczos (Krylov) approximation of the time-evolution operator of the
 * discretised Dirac equation (Beerwerth & Bauke, "Krylov subspace methods for
 * the Dirac equation"):
 *
 *   H = c sigma.(p - qA) + sigma_z m c^2 + V          (Sec. 3, Eq. 12; q = -1)
 *   psi(t+dt) = exp(-i H dt) psi ~ ||psi|| Q exp(-i T dt) e_1   (Sec. 4, Eq. 17)
 *
 * with Q, T from the Lanczos recurrence (Sec. 2, Fig. 1 with the modified
 * Gram-Schmidt alpha of Eq. 4) and the error estimate of Eq. 18.
 *
 * Conventions shared by every call:
 *  - a spinor field is complex128 laid out [ny][nx][2] (x fastest, then the
 *    upper and lower component of one site adjacent): 32 bytes per site,
 *    row-major, no padding.  Device pointers must be 32-byte aligned.
 *  - site (j, l) sits at x = (j - nx/2) dx, y = (l - ny/2) dy (atomic units).
 *  - all work is enqueued on the context's CUDA stream and is asynchronous
 *    unless a call says it synchronises.
 *  - no call aborts or throws; each returns a dirac_status.  Device-side
 *    failures (non-finite values: DIRAC_ENONFINITE; a timed-out grid barrier
 *    of the one-launch step: DIRAC_ECUDA) are recorded on the device and
 *    returned by the next call that synchronises (an info request,
 *    dirac_sync); psi is left unchanged and the context stays usable.
 *  - the caller owns every buffer it passes; the library owns the context
 *    and its workspace (the Krylov basis lives in device memory).
 */
#ifndef DIRAC_GB300_H
#define DIRAC_GB300_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    DIRAC_OK = 0,
    DIRAC_EINVAL = 1,      /* an argument is out of range (see dirac_last_error) */
    DIRAC_ENOMEM = 2,      /* device or pinned host allocation failed */
    DIRAC_ECUDA = 3,       /* a CUDA runtime call failed */
    DIRAC_ENONFINITE = 4,  /* NaN/Inf met in a reduction; psi left unchanged */
    DIRAC_ESTATE = 5       /* call out of order (e.g. step before set_fields) */
} dirac_status;

enum { DIRAC_PERIODIC = 0, DIRAC_DIRICHLET = 1 };
enum { DIRAC_FP64 = 0, DIRAC_MIXED = 1 };

/* Largest Krylov dimension m one step may use. */
#define DIRAC_KRYLOV_MAX 32

typedef struct dirac_ctx dirac_ctx;

/* Diagnostics of the most recent step (Sec. 4 and Sec. 6). */
typedef struct {
    int k_used;        /* Krylov dimension used (< m after breakdown or tol) */
    int breakdown;     /* 1 if the recurrence stopped on beta_k ~ 0 */
    double err_est;    /* Eq. 18: dt beta_k ||psi|| |e_k^T exp(-i T dt) e_1| */
    double cum_err;    /* sum of err_est since create (Sec. 6, cumulative bound) */
    double norm;       /* ||psi|| before the step (sum over sites, no dx dy) */
    double energy;     /* <psi|H|psi>/<psi|psi> before the step (hartree) */
    double alpha[DIRAC_KRYLOV_MAX];  /* T diagonal, of H - energy_shift (hartree) */
    double beta[DIRAC_KRYLOV_MAX];   /* beta[i] couples i, i+1; beta[k-1] = beta_k */
    double kappa_max;  /* largest ||y^||^2 / (||y^||^2 - P^2/X) of a pass since create:
                          the cancellation in the fused beta estimate */
} dirac_step_info;

/*
 * Create a propagator for an nx-by-ny grid with spacings dx, dy (bohr),
 * particle mass and speed of light c (atomic units), central finite
 * differences of stencil_order 2 or 4 (Sec. 7: finite differences; the
 * central form keeps H Hermitian), DIRAC_PERIODIC or DIRAC_DIRICHLET
 * boundaries, precision DIRAC_FP64 or DIRAC_MIXED, and Krylov dimension up
 * to m_max (1..DIRAC_KRYLOV_MAX).  DIRAC_FP64 computes everything in FP64.
 * DIRAC_MIXED keeps the state psi in complex128 but stores the Krylov basis
 * in complex64 and applies H in FP32 (every coefficient as an FP32 value
 * plus its remainder, the diagonal plus V by an exact two-sum), while the
 * inner products are summed in FP64 across warps and the scalars alpha,
 * beta, the small exponential and the recombination coefficients stay FP64;
 * the recombination adds C_1 psi in FP64 and the other terms as compensated
 * FP32 sums.  Energies are best given relative to m c^2 on this path
 * (energy_shift of dirac_set_fields).  Allocates the workspace: (m_max + 1) device fields of nx*ny
 * sites (32 B per site for FP64, 16 B for MIXED).  cuda_stream is a cudaStream_t (NULL: the legacy default
 * stream).  On success *out owns the context.
 * Errors: DIRAC_EINVAL (nx, ny < 1; dx, dy, c <= 0; mass < 0; bad order,
 * boundary, precision or m_max), DIRAC_ENOMEM, DIRAC_ECUDA.
 */
dirac_status dirac_create(dirac_ctx** out, int nx, int ny, double dx, double dy,
                          double mass, double c, int stencil_order, int boundary,
                          int precision, int m_max, void* cuda_stream);

/* Free the context and its workspace (synchronises its stream). NULL is a no-op. */
void dirac_destroy(dirac_ctx* ctx);

/* Change the stream later work is enqueued on. */
dirac_status dirac_set_stream(dirac_ctx* ctx, void* cuda_stream);

/*
 * Set the fields of Eq. 12 for the following steps.  V_dev: device float64
 * [ny][nx] potential energy q*phi in hartree (copied into the context, the
 * caller keeps its buffer), or NULL for V = 0.  A_x, A_y: the spatially
 * uniform vector potential for the next step -- for a time-dependent field
 * the caller passes the mean of A over the step (the first Magnus term,
 * Eq. 16; dirac_pulse_sin2_mean computes it for a sin^2 pulse).
 * energy_shift s: the recurrence runs on H - s and the step multiplies by
 * exp(-i s dt) -- exact in exact arithmetic; reported alpha are of H - s.
 * Errors: DIRAC_EINVAL (non-finite scalars), DIRAC_ECUDA.
 */
dirac_status dirac_set_fields(dirac_ctx* ctx, const double* V_dev, double A_x, double A_y,
                              double energy_shift);

/* Update only the uniform vector potential (cheap; keeps V and the shift). */
dirac_status dirac_set_vector_potential(dirac_ctx* ctx, double A_x, double A_y);

/*
 * One time step, in place: psi_dev <- exp(-i H dt) psi_dev by Eq. 17 with a
 * Krylov space of dimension m (1..m_max).  tol > 0 stops the recurrence at the
 * first k whose Eq. 18 estimate is <= tol * ||psi||; tol = 0 always uses m
 * (unless the recurrence breaks down, beta_k <= 1e-12 times the largest
 * |alpha_j + s| or beta_j so far).  A zero psi stays zero (k_used = 1,
 * norm 0, no error).  psi_dev: device complex128 [ny][nx][2],
 * 32-byte aligned, owned by the caller.  If info is non-NULL the call
 * synchronises the stream and fills it; otherwise it returns after enqueueing.
 * dt < 0 steps backwards in time, psi <- exp(+i H |dt|) psi (T is real, so
 * the small exponential is the conjugate of the forward one).
 * Errors: DIRAC_EINVAL (m out of range, dt = 0 or non-finite, tol < 0,
 * misaligned psi, dt too large for the small exponential: |dt| ||H|| > 90),
 * DIRAC_ESTATE (no set_fields yet), DIRAC_ENONFINITE (only with info),
 * DIRAC_ECUDA (a CUDA call failed, or -- only with info -- a grid barrier
 * of the one-launch step timed out).
 */
dirac_status dirac_lanczos_step(dirac_ctx* ctx, void* psi_dev, double dt, int m, double tol,
                                dirac_step_info* info);

/*
 * nsteps steps in place, the vector potential of step n being
 * (A_xy_host[2n], A_xy_host[2n+1]) (host array of 2*nsteps doubles), or the
 * current one for every step if A_xy_host is NULL.  info (optional) describes
 * the last step and synchronises.  Errors as dirac_lanczos_step.
 */
dirac_status dirac_lanczos_steps(dirac_ctx* ctx, void* psi_dev, int nsteps, double dt, int m,
                                 double tol, const double* A_xy_host, dirac_step_info* info);

/*
 * As dirac_lanczos_steps, but psi_host is a HOST complex128 [ny][nx][2]
 * buffer: the call copies it to a device buffer owned by the context, runs
 * the steps, copies the result back and synchronises.  Pinned host memory
 * makes the copies asynchronous DMA; pageable memory also works.
 */
dirac_status dirac_propagate_host(dirac_ctx* ctx, void* psi_host, int nsteps, double dt, int m,
                                  double tol, const double* A_xy_host, dirac_step_info* info);

/* Wait for the context's stream; returns a pending device error if any. */
dirac_status dirac_sync(dirac_ctx* ctx);

/*
 * Checkpoint and resume.  Between steps a context carries, besides psi, a
 * small device block of scalars from step to step (the next step's stencil
 * shift, the cumulative Eq. 18 estimate, ...).  dirac_export_state copies it
 * to a host buffer of dirac_state_bytes(ctx) bytes (synchronises; DIRAC_ESTATE
 * before the first step); dirac_import_state loads it into a context created
 * with the same arguments by the same library build, after its
 * dirac_set_fields (which otherwise re-derives the shift from psi).  With the
 * same fields and psi, the resumed context then computes bitwise what the
 * original would have.  The block is opaque.  Errors: DIRAC_EINVAL (sizes, a block not
 * exported between steps), DIRAC_ECUDA.
 */
size_t dirac_state_bytes(const dirac_ctx* ctx);
dirac_status dirac_export_state(dirac_ctx* ctx, void* host, size_t bytes);
dirac_status dirac_import_state(dirac_ctx* ctx, const void* host, size_t bytes);

/* Mean of A_x(t) = a0 sin^2(pi t/T) sin(omega t) (zero outside [0, T]) over
 * [t0, t0 + dt], in closed form: the first Magnus term of Eq. 16. */
double dirac_pulse_sin2_mean(double t0, double dt, double a0, double omega, double duration);

/* Step means of the sine basis of a pulse, A_x(t) = sum_k a_k sin((k+1) pi t/T)
 * on [0, T]: W[n * n_coef + k] = (1/dt) integral over [n dt, (n+1) dt] of
 * sin((k+1) pi t/T) dt, in closed form (Eq. 16's first Magnus term for each
 * basis function), so that the step means are W a.  W: host array of
 * nsteps * n_coef doubles.  Errors: DIRAC_EINVAL. */
dirac_status dirac_pulse_sine_basis_means(int nsteps, double dt, int n_coef, double duration, double* W);

/* Number of kernels the library launched on this context so far. */
long long dirac_kernel_launches(const dirac_ctx* ctx);

/*
 * Per-kernel device timing with CUDA events, for tracing and benchmarks.
 * While enabled, the context records an event on its stream before every
 * kernel it launches and after every time step.  dirac_profile_read waits
 * for the last recorded event and returns, per kernel kind, the device time
 * (ms) between each kernel's event and the next one, and the number of
 * launches, accumulated since the previous read; it then clears the record.
 * Kinds: 0 = Lanczos pass (stencil + reductions), 1 = recombination,
 * 2 = one-launch time step (all passes and the recombination, see
 * dirac_set_step_mode).
 * ms and launches point to DIRAC_KERNEL_KINDS elements each.
 */
#define DIRAC_KERNEL_KINDS 3
dirac_status dirac_profile_enable(dirac_ctx* ctx, int enable);
dirac_status dirac_profile_read(dirac_ctx* ctx, double* ms, long long* launches);

/* Static description of a status code. */
const char* dirac_status_string(dirac_status s);

/* Message of the last error raised on the calling thread ("" if none). */
const char* dirac_last_error(void);

/*
 * Batches: many independent propagations advanced together (one launch per
 * Lanczos iteration covers every problem of the batch, so the per-launch
 * costs are shared).  All problems share mass, c, stencil order, boundary,
 * precision, m_max, dt, m and tol; each has its own grid (nx[b] x ny[b],
 * spacings dx[b], dy[b]), state, potential, shift and vector potential.
 * The semantics per problem are those of the single-problem calls above.
 * Errors as dirac_create / dirac_lanczos_steps.
 */
typedef struct dirac_batch dirac_batch;

dirac_status dirac_batch_create(dirac_batch** out, int n_problems, const int* nx, const int* ny,
                                const double* dx, const double* dy, double mass, double c,
                                int stencil_order, int boundary, int precision, int m_max,
                                void* cuda_stream);
void dirac_batch_destroy(dirac_batch* batch);

/* As dirac_set_fields, for problem `problem` (0-based). */
dirac_status dirac_batch_set_fields(dirac_batch* batch, int problem, const double* V_dev,
                                    double A_x, double A_y, double energy_shift);

/*
 * Launch shape of the Lanczos passes: tile height 32 or 16 sites and a cap
 * on resident CTAs per SM (0: no cap).  Without a call the tile height is
 * chosen per run (FP64: from the tile count per SM; mixed: 16).  Used by the
 * autotuner; results do not depend on it beyond the order of floating-point
 * sums.
 */
dirac_status dirac_batch_set_launch_shape(dirac_batch* batch, int tile_height, int ctas_per_sm);

/*
 * nsteps steps of every problem, in place.  psi_dev: n_problems device
 * pointers (complex128 [ny[b]][nx[b]][2], 32-byte aligned).  A_xy_host:
 * host array [nsteps][n_problems][2] of per-step vector potentials, or NULL
 * to keep each problem's current one.  info: n_problems entries or NULL
 * (synchronises when given).
 */
dirac_status dirac_batch_steps(dirac_batch* batch, void* const* psi_dev, int nsteps, double dt,
                               int m, double tol, const double* A_xy_host, dirac_step_info* info);

/* Wait for the batch's stream and fill info (n_problems entries, may be NULL). */
dirac_status dirac_batch_sync(dirac_batch* batch, dirac_step_info* info);

/*
 * Autotuner of the launch shape: times every candidate (tile height x
 * CTAs per SM) over `steps` steps of the batch on scratch copies of the
 * states psi_dev (the states themselves and the scalar blocks are left
 * unchanged), keeps the fastest, and, when the environment variable
 * DIRAC_AUTOTUNE_CACHE names a file, records the choice there by a
 * signature of the problem set (precision, stencil, boundary, sizes, m,
 * GPU) and reuses it on later calls.  A_xy_host: as for dirac_batch_steps
 * (for `steps` steps) or NULL.  Allocates scratch (the states' size).
 */
typedef struct {
    int tile_height, ctas_per_sm;   /* the chosen shape */
    double ms_per_step;             /* its measured time */
    int from_cache;                 /* 1: taken from the cache file */
    int candidates;                 /* shapes timed */
} dirac_tune_result;

dirac_status dirac_batch_autotune(dirac_batch* batch, void* const* psi_dev, double dt, int m,
                                  const double* A_xy_host, int steps, dirac_tune_result* out);

/*
 * Replay of a captured CUDA graph per step (default on; off: direct
 * launches).  The kernels and their order are the same either way.
 */
dirac_status dirac_batch_use_graphs(dirac_batch* batch, int enable);
dirac_status dirac_use_graphs(dirac_ctx* ctx, int enable);

/*
 * How the time steps of a context are launched.
 *   DIRAC_STEP_PASSES: one launch per Lanczos pass and one for the
 *     recombination (replayed as a CUDA graph); the last CTA of each pass
 *     updates the scalars.
 *   DIRAC_STEP_ONE_LAUNCH: the whole step as one cooperative launch (every
 *     CTA resident), the passes separated by grid-wide barriers; after each
 *     barrier every CTA sums all CTA partials in the same order and updates
 *     its own copy of the scalars.  Each barrier wait is bounded: a timeout
 *     ends the launch and the next read of the state reports DIRAC_ECUDA.
 *     On the mixed path the tiles are staged by tensor copies into a
 *     shared-memory ring by a producer warp, and batches run every problem
 *     in the same launch.
 *   DIRAC_STEP_AUTO (default): one launch per step on the FP64 path (one
 *     CTA per SM), per-pass launches on the mixed path (eight CTAs per SM;
 *     measured faster there than the one-launch form).
 * Results agree to rounding: the partial sums are added in another order.
 */
#define DIRAC_STEP_AUTO 0
#define DIRAC_STEP_PASSES 1
#define DIRAC_STEP_ONE_LAUNCH 2
dirac_status dirac_set_step_mode(dirac_ctx* ctx, int mode);

/*
 * The same choice for a batch (mixed precision: DIRAC_STEP_ONE_LAUNCH runs
 * every pass of every problem and the recombination as one cooperative
 * launch per step; FP64 batches always use per-pass launches).
 * Errors: DIRAC_EINVAL (null batch, unknown mode).
 */
dirac_status dirac_batch_set_step_mode(dirac_batch* batch, int mode);

/*
 * Test of the failure path of the one-launch step: runs one step whose grid
 * barriers wait for one CTA more than the launch has, so that every bounded
 * wait runs out (about a second); no fault, no hang.  Returns the status the
 * context reports afterwards -- DIRAC_ECUDA, psi_dev (complex128 [ny][nx][2],
 * device) untouched -- and leaves the context usable.  DIRAC_ESTATE on a
 * context without the one-launch step (fields not set: DIRAC_ESTATE too).
 */
dirac_status dirac_debug_barrier_timeout(dirac_ctx* ctx, void* psi_dev, double dt, int m);

/* dirac_profile_enable / dirac_profile_read / dirac_kernel_launches for a batch. */
dirac_status dirac_batch_profile_enable(dirac_batch* batch, int enable);
dirac_status dirac_batch_profile_read(dirac_batch* batch, double* ms, long long* launches);
long long dirac_batch_kernel_launches(const dirac_batch* batch);

/*
 * Allocation-free single step.  The paper has no counterpart: this entry
 * point exists for callers that must not allocate device memory -- a host
 * framework that owns all device allocations and forbids libraries from
 * calling cudaMalloc, a memory budget fixed up front, or a per-step loop in
 * which an allocation's latency or failure is not acceptable.
 *
 * It performs one FP64 time step, in place on psi_dev, as dirac_lanczos_step
 * would for an FP64 context created with the same problem (dirac_problem
 * below) and launched one pass at a time, dt < 0 stepping backwards as
 * there, but keeps its whole workspace in one static device array of
 * dirac_noalloc_scratch_bytes() bytes (8 MiB) per device, and calls no
 * cudaMalloc, cudaFree or other allocating routine.  Problems whose
 * workspace, about (m + 1) * nx * ny * 32 bytes, does not fit are rejected
 * with DIRAC_EINVAL.  The per-call tables reach the device as kernel
 * arguments; no host buffer is read after the call returns.
 *  - The first call on each device looks up the array's device address
 *    (cudaGetSymbolAddress) with that device current and keeps it for the
 *    life of the process; make that first call before any stream capture.
 *    cudaDeviceReset unloads the array: do not call this entry point on a
 *    device after resetting it.
 *  - Every call in the process shares the one array, and the array keeps the
 *    previous call's contents (the call clears what must start at zero).
 *    Calls whose work overlaps on the GPU -- on different streams, or from
 *    different threads -- race on it: serialise them.
 *  - With V_dev non-NULL the call reads two doubles back (the range of V)
 *    and so synchronises the stream.  With info non-NULL it synchronises and
 *    fills info (cum_err is this step's estimate); device-side errors
 *    (DIRAC_ENONFINITE) are only reported when info is requested.
 * psi_dev, V_dev: device buffers owned by the caller, laid out as for
 * dirac_lanczos_step / dirac_set_fields.  cuda_stream: a cudaStream_t.
 * Errors: DIRAC_EINVAL (the problem's sizes, spacings, order, boundary or
 * scalars as for dirac_create / dirac_set_fields; m outside
 * 1..DIRAC_KRYLOV_MAX; dt = 0 or non-finite; tol < 0; misaligned psi; a
 * workspace beyond the scratch; V with non-finite entries), DIRAC_ENONFINITE
 * (only with info), DIRAC_ECUDA.
 */
typedef struct {
    int nx, ny;
    double dx, dy, mass, c;
    int stencil_order, boundary;
    const double* V_dev;          /* [ny][nx] potential energy or NULL */
    double A_x, A_y, energy_shift;
} dirac_problem;

dirac_status dirac_lanczos_step_noalloc(const dirac_problem* problem, void* psi_dev, double dt,
                                        int m, double tol, void* cuda_stream,
                                        dirac_step_info* info);

/* Size in bytes of the static scratch array used by dirac_lanczos_step_noalloc. */
size_t dirac_noalloc_scratch_bytes(void);

/* ------------------------------------------------------------------------
 * Hamiltonian product and eigenvalue mode (Sec. 2, Sec. 5)
 * ------------------------------------------------------------------------ */

/*
 * out = (H - s) in for the context's operator and fields (Eq. 12 with the
 * V, A and energy shift s of dirac_set_fields), in FP64 whatever the
 * context's precision.  in, out: complex128 [ny][nx][2] device fields,
 * 32-byte aligned, not aliased.  Asynchronous on the context stream.
 * Errors: DIRAC_EINVAL (null, unaligned or aliased pointers), DIRAC_ESTATE
 * (fields not set), DIRAC_ECUDA.
 */
dirac_status dirac_apply_hamiltonian(dirac_ctx* ctx, const void* in_dev, void* out_dev);

/* Most Ritz values examined per convergence check (and so largest n_want). */
#define DIRAC_EIG_RITZ_MAX 256
/* Largest Lanczos iteration count of the eigenvalue mode. */
#define DIRAC_EIG_ITER_MAX 8192

typedef struct {
    int iterations;    /* Lanczos iterations k run (size of T_k at the end) */
    int n_found;       /* values written to eigs_out */
    int n_in_window;   /* Ritz values of T_k in the window (folded: k) */
    int n_converged;   /* of those examined, with bound <= tol * max(1, |theta|) */
    int breakdown;     /* 1: beta_k fell below 1e-12 * scale, T_k's spectrum is exact */
    long long launches;  /* kernels launched by the call */
    /* device time (ms) per kernel kind, measured with CUDA events while
       dirac_profile_enable is on (else 0): the stencil product, the
       Gram-Schmidt inner products, the Gram-Schmidt updates, everything else
       (coefficient sums, Ritz values and vectors) */
    double ms_apply, ms_dot, ms_update, ms_other;
} dirac_eig_info;

/*
 * Eigenvalues of H - s near the bottom of the band gap, by the Lanczos
 * algorithm with full reorthogonalisation (classical Gram-Schmidt applied
 * twice, Sec. 2; reorth = 0: the plain three-term recurrence of Fig. 1).
 *
 * The recurrence runs on A = H - s (fold = 0) or on A = (H - s - sigma)^2
 * (fold = 1), starting from start_dev (complex128 [ny][nx][2], any nonzero
 * norm; not modified).  Every check_every iterations and at max_iter the Ritz
 * values theta of T_k and their Eq. 9 bounds |beta_k t_i^k| are computed on
 * the device; theta counts as converged when its bound is
 * <= tol * max(1, |theta|).
 *   fold = 0: stops when n_want converged Ritz values lie in the open window
 *     (e_lo, e_hi) (energies of H - s; the bound states of a potential that
 *     vanishes at infinity lie in (-s, mc^2 - s), Sec. 5).  Returns the lowest
 *     n_want converged ones, ascending, with their bounds.
 *   fold = 1: stops when the n_want smallest Ritz values of A are converged;
 *     each gives lambda = sigma + sign(rho) sqrt(theta), rho the Rayleigh
 *     quotient of its Ritz vector with H - s - sigma, bound
 *     min(sqrt(r), r / sqrt(theta)) from the Eq. 9 bound r; returned
 *     ascending in lambda.  e_lo, e_hi are not used.
 * At a breakdown (invariant subspace) the recurrence stops and T_k's spectrum
 * is exact.  On a DIRAC_MIXED context the off-diagonal part of the stencil
 * products (differences, vector potential) runs in FP32 on complex64 copies
 * of the vectors and the diagonal (+-m c^2 + V - s) in FP64; the Lanczos
 * combination, the Gram-Schmidt passes, T and the Ritz values and
 * vectors stay FP64.  At most DIRAC_EIG_RITZ_MAX Ritz values (the lowest in the window)
 * are examined per check.
 *
 * eigs_out, bounds_out: host arrays of n_want doubles; the first
 * info->n_found entries are written.  vecs_dev: NULL, or room for n_want
 * device fields (complex128 [ny][nx][2] each, consecutive, 32-byte aligned)
 * that receive the unit-norm Ritz vectors Q t_i (Eq. 8) of the returned
 * values.  info may be NULL.
 *
 * Device memory: (max_iter + 1) fields for the basis (plus 1 + n_want with
 * fold = 1), allocated for the call and freed before it returns; the call
 * synchronises the context stream at every check.
 * Errors: DIRAC_EINVAL (n_want outside 1..DIRAC_EIG_RITZ_MAX, max_iter
 * outside 1..DIRAC_EIG_ITER_MAX, check_every < 1, tol < 0, e_lo >= e_hi,
 * null outputs, unaligned pointers), DIRAC_ESTATE (fields not set),
 * DIRAC_ENOMEM (the basis does not fit), DIRAC_ENONFINITE (NaN/Inf met, or a
 * zero start vector), DIRAC_ECUDA.
 */
dirac_status dirac_lanczos_eigs(dirac_ctx* ctx, const void* start_dev, int n_want, int max_iter,
                                int check_every, double tol, double e_lo, double e_hi, int reorth,
                                int fold, double sigma, double* eigs_out, double* bounds_out,
                                void* vecs_dev, dirac_eig_info* info);

/* ------------------------------------------------------------------------
 * Gradients through the propagation (adjoint of the time-discrete map)
 * ------------------------------------------------------------------------ */

enum { DIRAC_OBS_PX = 0, DIRAC_OBS_PROJ = 1 };

typedef struct {
    int observable;        /* DIRAC_OBS_PX: L = dx dy Re <psi_N, p_x psi_N>, p_x = -i D_x
                              (the Hamiltonian's central difference);
                              DIRAC_OBS_PROJ: L = |dx dy <phi, psi_N>|^2 */
    const void* phi_dev;   /* PROJ: the fixed state phi (complex128 [ny][nx][2]) */
    int checkpoint_every;  /* forward states kept every this many steps (>= 1) */
    int block_x, block_y;  /* dV_dev receives dL/dV summed over blocks of
                              block_x x block_y sites (1, 1: per site) */
    int n_coef;            /* with W_host: A_x of step n = sum_k W[n][k] a_k */
    const double* W_host;  /* nsteps x n_coef, row-major (host), or NULL */
} dirac_adjoint_opts;

typedef struct {
    double ms_forward;     /* device time of the forward sweep and the observable */
    double ms_backward;    /* of the backward sweep (recomputation included) */
    int quadrature_nodes;  /* Gauss-Legendre nodes of the Frechet integral */
    int checkpoints;       /* stored forward states */
    long long launches;    /* kernels launched by the call (both contexts) */
    double ms_contract;    /* device time of the per-site contraction kernels, measured
                              with CUDA events while dirac_profile_enable is on (else 0) */
} dirac_adjoint_info;

/*
 * Gradient of a real observable of the final state psi_N of nsteps time
 * steps psi_{n+1} = exp(-i H_n dt) psi_n (Sec. 4, Eq. 17, Krylov dimension
 * m, the context's V and energy shift, H_n with the vector potential
 * (A_xy_host[2n], A_xy_host[2n+1]) -- the step means of Eq. 16) with respect
 * to the potential V at every site and to the step-mean vector potential of
 * every step.  The paper has no counterpart; the map differentiated is the
 * time-discrete propagation itself (its Krylov error, Eq. 18, is taken as
 * negligible).
 *
 * Method: reverse (adjoint) sweep, lambda_N = dL/d conj(psi_N),
 * lambda_n = exp(+i H_n dt) lambda_{n+1}; each step contributes
 * dL/dtheta = 2 dt Im int_0^1 <exp(+i H_n dt s) lambda_{n+1}, dH_n/dtheta
 * exp(-i H_n dt (1 - s)) psi_n> ds (the Frechet derivative of the
 * exponential), evaluated exactly in the two Krylov spaces with a
 * Gauss-Legendre rule in s.  Forward states are kept every checkpoint_every
 * steps and recomputed segment by segment.
 *
 * psi0_dev: initial state (device, not modified).  loss_out: L (host).
 * psiN_dev: NULL or receives psi_N.  dV_dev: NULL or a device array of
 * (ny / block_y) x (nx / block_x) doubles receiving dL/dV summed over blocks
 * (V is the potential energy).  dA_host: NULL or host nsteps x 2 doubles
 * receiving dL/dA_x, dL/dA_y of every step.  da_host: NULL or host n_coef
 * doubles receiving dL/da_k = sum_n W[n][k] dL/dA_x(n).  With all three
 * NULL only the forward sweep and L are computed.  info may be NULL.
 * The context must be FP64 with fields set; a second context with the same
 * operator is created for the adjoint.  Device memory: about
 * (nsteps / checkpoint_every + checkpoint_every + 3) fields plus one Krylov
 * basis.  Synchronises.
 * Errors: DIRAC_EINVAL (arguments, mixed-precision context, blocks that do not
 * tile the grid, dt * ||H|| too large for the quadrature), DIRAC_ESTATE,
 * DIRAC_ENOMEM, DIRAC_ENONFINITE, DIRAC_ECUDA.
 */
dirac_status dirac_adjoint_gradient(dirac_ctx* ctx, const void* psi0_dev, int nsteps, double dt, int m,
                                    const double* A_xy_host, const dirac_adjoint_opts* opts,
                                    double* loss_out, void* psiN_dev, void* dV_dev, double* dA_host,
                                    double* da_host, dirac_adjoint_info* info);

/*
 * Measured arithmetic peak of the current GPU, the denominator of the
 * roofline of the kernels that are bound by arithmetic rather than memory
 * (the FP64 path).  The paper has no counterpart: it is a measurement
 * utility.  kind DIRAC_PEAK_FP64 or DIRAC_PEAK_FP32: every SM's resident
 * threads run eight independent fused multiply-add chains each; *tflops
 * receives 2 x (FMAs) / (best CUDA-event time of three launches after one
 * warm-up), in TFLOP/s.  Runs on a private stream, allocates a few bytes,
 * synchronises; takes about a quarter of a second.
 * Errors: DIRAC_EINVAL (kind, null output), DIRAC_ECUDA.
 */
#define DIRAC_PEAK_FP64 0
#define DIRAC_PEAK_FP32 1
dirac_status dirac_measure_peak(int kind, double* tflops);

/*
 * Test hook for the device small-matrix exponential: v = exp(-i T dt) e_1 for
 * the k-by-k tridiagonal T (alpha[0..k-1] diagonal, beta[0..k-2] off
 * diagonal), whose spectrum must lie in [lo, hi], computed by the same device
 * routine the propagator uses.  Host arrays in and out (v_re, v_im: k each);
 * synchronises.  Errors: DIRAC_EINVAL (k out of 1..DIRAC_KRYLOV_MAX, lo > hi,
 * dt * (hi - lo) / 2 > 90), DIRAC_ECUDA.
 */
dirac_status dirac_debug_tridiag_expm(const double* alpha, const double* beta, int k, double dt,
                                      double lo, double hi, double* v_re, double* v_im);

#ifdef __cplusplus
}
#endif
#endif /* DIRAC_GB300_H */
