/*
 * lbm.h — C ABI of the GB300 (sm_103a) quasi-incompressible phase-field
 * lattice Boltzmann solver of Yang & Guo (arXiv 1507.03521), D2Q9.
 *
 * The method: two coupled lattice Boltzmann equations advanced together
 * each time step (Sec. 3):
 *   - f_i, the FLOW population (Eq. 22), relaxed with tau_f (viscosity
 *     nu = cs2 (tau_f - 1/2), Eq. 33), whose moments give the pressure p
 *     (Eq. 32) and the velocity u (Eq. 31);
 *   - g_i, the PHASE-FIELD population (Eq. 23), relaxed with tau_g
 *     (mobility lambda = cs2 (tau_g - 1/2) alpha, Eq. 33), whose zeroth
 *     moment is the order parameter phi (Eq. 30).
 * Naming follows the paper: f is flow, g is phase.
 *
 * Conventions (all entry points):
 *   - Every call returns lbm_status; LBM_OK is 0, errors are negative.
 *     After an error, lbm_last_error(sim) holds a one-line message.
 *   - Fields are row-major [ny][nx], x fastest; y is the wall and gravity
 *     direction.  The field element type is double for LBM_F64 and float
 *     for every other dtype ("field type" below).
 *   - Device work is asynchronous on the stream given to lbm_create (a
 *     cudaStream_t, NULL for the legacy default stream).  Calls that hand
 *     results to the host (lbm_mass, lbm_laplace, and any *_host variant)
 *     synchronise that stream.  Asynchronous CUDA errors surface at the
 *     next synchronising call as LBM_ERR_CUDA.
 *   - The library allocates no device memory of its own for a simulation:
 *     the caller allocates the two buffers sized by lbm_buffer_sizes and
 *     binds them with lbm_bind_buffers.  They must stay valid until
 *     lbm_destroy; the library never frees them.
 *   - A handle is not thread-safe; distinct handles are independent.
 */
#ifndef LBM_H
#define LBM_H

#include <stddef.h>
#include <stdint.h>

#if defined(__GNUC__)
#define LBM_API __attribute__((visibility("default")))
#else
#define LBM_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

typedef struct lbm_sim lbm_sim; /* opaque handle, owned by the caller */

typedef enum {
    LBM_OK = 0,
    LBM_ERR_ARG = -1,       /* invalid argument or parameter set */
    LBM_ERR_CUDA = -2,      /* a CUDA runtime call failed */
    LBM_ERR_NONFINITE = -3, /* a reduction met NaN or Inf in the state */
    LBM_ERR_TIMEOUT = -4,   /* reserved: a bounded device wait ran out */
    LBM_ERR_STATE = -5,     /* call out of order (e.g. step before init) */
    LBM_ERR_NOMEM = -6      /* a bound buffer is too small */
} lbm_status;

typedef enum {
    LBM_F64 = 0,  /* populations and arithmetic in FP64 */
    LBM_F32 = 1,  /* populations and arithmetic in FP32 */
    LBM_F16S = 2, /* FP32 arithmetic; f_0..8 and g_1..8 stored as scaled FP16, g_0 in FP32 */
    LBM_BF16S = 3, /* FP32 arithmetic; f_0..8 and g_1..8 stored as BF16, g_0 in FP32 */
    /* FP32 arithmetic; f_0..8 and g_1..8 stored as their deviations from the
     * rest equilibrium of the cell they sit on (Eqs. 24-27 at u = 0:
     * w_i p and w_i alpha mu, with p and alpha mu of that cell's previous
     * time level, cut to 16 bits and stored beside the populations), in
     * scaled FP16 (LBM_F16D) or BF16 (LBM_BF16D); g_0 in FP32.  Single
     * domains with nx a multiple of 8 only (not batches, slabs, the lagged
     * variant or the adjoint). */
    LBM_F16D = 4,
    LBM_BF16D = 5
} lbm_dtype;

typedef enum { LBM_PERIODIC = 0, LBM_WALL = 1 } lbm_bc;

/* Physical and lattice parameters of one domain, in lattice units
 * (dx = dt = 1, D2Q9, cs2 = 1/3; Sec. 3).
 *   nx, ny          grid size, each >= 5
 *   rho_A, rho_B    densities of fluids A and B (> 0)
 *   phi_A, phi_B    bulk order parameters of A and B (distinct)
 *   sigma, W        surface tension and interface width; they fix
 *                   kappa = 3 sigma W / (2 dphi^2) and
 *                   beta = 12 sigma / (W dphi^4), dphi = phi_A - phi_B
 *                   (Eqs. 3-4 solved for kappa and beta)
 *   M               mobility lambda of the Cahn-Hilliard equation (Eq. 7)
 *   tau_f, tau_g    relaxation times of f (flow) and g (phase), > 1/2
 *   gravity, rho_ref body force F_b = (0, -(rho - rho_ref) gravity)
 *                   (the form of Sec. 4.3 with rho_A replaced by rho_ref)
 *   bc_x            LBM_PERIODIC only
 *   bc_y            LBM_PERIODIC, or LBM_WALL: no-slip walls at y = -1/2
 *                   and y = ny - 1/2 (halfway bounce-back)
 *   u_wall_bottom, u_wall_top  x-velocity of the walls (LBM_WALL only)
 *   dtype           an lbm_dtype
 *   gradp_lag       0: the paper's synchronous step (default).  1: the
 *                   lagged-grad-p variant, not in the paper: G_i of Eq. 29
 *                   takes grad p from the previous step's pressure (0
 *                   before the first step), which each level then stores
 *                   in one more slot.  Single domains with nx a multiple of
 *                   8 only (not batches, slabs or the adjoint). */
typedef struct {
    int nx, ny;
    double rho_A, rho_B, phi_A, phi_B;
    double sigma, W, M, tau_f, tau_g;
    double gravity, rho_ref;
    int bc_x, bc_y;
    double u_wall_bottom, u_wall_top;
    int dtype;
    int gradp_lag;
} lbm_params;

/* Library ABI version (this header: 1). */
LBM_API int lbm_version(void);

/* Bytes the caller must allocate on the device for one domain:
 * *state_bytes for the populations (two time levels, ping-pong) and
 * *work_bytes for field staging and reduction partials.  Both are
 * multiples of 256.  Returns LBM_ERR_ARG for an invalid parameter set. */
LBM_API lbm_status lbm_buffer_sizes(const lbm_params *prm, size_t *state_bytes, size_t *work_bytes);

/* Validate prm and create a handle bound to `stream` (a cudaStream_t) on
 * the current CUDA device.  Host memory only.  *out is NULL on error. */
LBM_API lbm_status lbm_create(const lbm_params *prm, void *stream, lbm_sim **out);

/* Bind caller-owned device buffers (>= the sizes of lbm_buffer_sizes,
 * 256-byte aligned).  LBM_ERR_NOMEM if either is too small. */
LBM_API lbm_status lbm_bind_buffers(lbm_sim *sim, void *state, size_t state_bytes, void *work,
                            size_t work_bytes);

/* Initial state (Secs. 4.1-4.2: "at equilibrium"): p = 0, u = (ux, uy)
 * (zero where a pointer is NULL), mu from phi (Eq. 5), f = f^eq (Eq. 24),
 * g = g^eq (Eq. 25).  phi, ux, uy: nx*ny elements of the field type, on
 * the device (on_host = 0) or in host memory (on_host = 1, copied in on
 * the stream, which is then synchronised).  Resets the step counter. */
LBM_API lbm_status lbm_init_phi(lbm_sim *sim, const void *phi, const void *ux, const void *uy,
                        int on_host);

/* Advance n >= 0 time steps (Eqs. 22-23 with Eqs. 24-32, streaming,
 * bounce-back).  Asynchronous; one kernel launch per step. */
LBM_API lbm_status lbm_step(lbm_sim *sim, int64_t n);

/* Macroscopic fields of the current time level: phi (Eq. 30), rho
 * (Eq. 11), p (Eq. 32), ux and uy (Eq. 31), mu (Eq. 5).  Each output is
 * nx*ny elements of the field type or NULL; device pointers for
 * on_host = 0, host pointers for on_host = 1 (the stream is then
 * synchronised before return). */
LBM_API lbm_status lbm_fields(lbm_sim *sim, void *phi, void *rho, void *p, void *ux, void *uy, void *mu,
                      int on_host);

/* Total mass sum(rho) and total order parameter sum(phi) over the grid,
 * accumulated in FP64 in a fixed order (bitwise reproducible).
 * Synchronises the stream.  LBM_ERR_NONFINITE if either is NaN or Inf. */
LBM_API lbm_status lbm_mass(lbm_sim *sim, double *mass, double *phi_total);

/* Laplace-law diagnostic of Sec. 4.2 for a droplet centred at (xc, yc)
 * with nominal radius R: *dP = mean total pressure
 * P = p0 - kappa phi lap(phi) + kappa |grad phi|^2 / 2 + p, p0 = phi psi' - psi,
 * over r < R - 2W minus its mean over r > R + 2W (nearest periodic image);
 * *R_eff = sqrt(A / pi), A = sum (phi - phi_B) / (phi_A - phi_B).
 * FP64 accumulation.  Synchronises the stream. */
LBM_API lbm_status lbm_laplace(lbm_sim *sim, double xc, double yc, double R, double *dP, double *R_eff);

/* Bytes of one time level of populations (what get/set_state copy). */
LBM_API size_t lbm_state_bytes(const lbm_sim *sim);

/* Copy the current populations out (dst) or in (src), device pointers for
 * on_host = 0 and host pointers for on_host = 1.  The layout is the
 * library's storage layout for the dtype; a state written by get_state
 * and read back by set_state resumes bit-identically.  set_state also
 * sets the step counter. */
LBM_API lbm_status lbm_get_state(lbm_sim *sim, void *dst, int on_host, int64_t *step);
LBM_API lbm_status lbm_set_state(lbm_sim *sim, const void *src, int on_host, int64_t step);

/* Number of time steps taken since lbm_init_phi / lbm_set_state. */
LBM_API int64_t lbm_step_count(const lbm_sim *sim);

/* Last error message of this handle ("" if none).  Valid until the next
 * call on the handle. */
LBM_API const char *lbm_last_error(const lbm_sim *sim);

/* Message of the last lbm_create / lbm_buffer_sizes / lbm_batch_create /
 * lbm_batch_buffer_sizes / lbm_mass_noalloc failure in this thread (those
 * calls have no handle to store it in). */
LBM_API const char *lbm_create_error(void);

/* Free the handle's host state.  Bound buffers stay the caller's. */
LBM_API void lbm_destroy(lbm_sim *sim);

/* Test hook of the timeout path; the paper has no counterpart.  FP32
 * single domains stage population rows by TMA tile loads, and every wait
 * for one is bounded (about one second).  With on != 0 the tile loads of
 * the following steps announce 16 bytes more than they bring, so their
 * waits run out: the kernel sets the handle's error word and its CTAs
 * return, and the next lbm_mass or lbm_laplace returns LBM_ERR_TIMEOUT.
 * The state is then not a valid time level (re-initialise it).  on = 0
 * restores normal loads.  Errors: LBM_ERR_ARG for a NULL handle. */
LBM_API lbm_status lbm_test_unfinished_tiles(lbm_sim *sim, int on);

/* ------------------------------------------------------------------ adjoint
 * Hand-written discrete adjoint (vector-Jacobian product) of the step, for
 * LBM_F64 and LBM_F32 handles.  With s_t the populations after t steps
 * (one level, the layout lbm_get_state writes) and lambda_t = dL/ds_t for
 * the loss L = sum_x (phi_T(x) - phi_target(x))^2:
 *   lbm_adj_seed   lambda_T from s_T and phi_target (and L itself);
 *   lbm_adj_step   lambda_t from s_t and lambda_{t+1}, adding the step's
 *                  contributions to dL/dM and dL/dsigma;
 *   lbm_adj_init   dL/dphi0 from lambda_0 (adjoint of lbm_init_phi with
 *                  u = 0), adding its (M, sigma) contributions;
 *   lbm_adj_grads  read the accumulated dL/dM, dL/dsigma.
 * M is the mobility lambda (alpha = M / (cs2 (tau_g - 1/2))), sigma the
 * surface tension (kappa and beta proportional to it).  All pointers are
 * device pointers; state and lambda buffers are lbm_state_bytes() each and
 * lam_next must differ from lam_t.  `work` is a caller-owned device buffer
 * of lbm_adj_work_bytes() bytes, 256-byte aligned, holding scratch fields,
 * the running totals and a counter of the reverse-step kernels; call
 * lbm_adj_reset (which zeroes both) before a buffer's first use.  Asynchronous on the
 * handle's stream except lbm_adj_grads and a seed that returns the loss.
 * The step being differentiated is the synchronous step of Eqs. 22-32
 * (Sec. 3) with its moment, stencil and wall rules; the paper itself has
 * no adjoint.
 * Errors (every call): LBM_ERR_ARG for a NULL handle, a handle that is not
 * LBM_F64 or LBM_F32, a lagged-grad-p handle (gradp_lag != 0), a NULL or
 * not 256-byte aligned work buffer, a NULL state/lambda/field pointer, or
 * lam_next == lam_t; LBM_ERR_CUDA for a failed launch or copy (message in
 * lbm_last_error).  lbm_adj_work_bytes returns LBM_ERR_ARG for a NULL
 * output or an unsupported handle; lbm_adj_grads synchronises the stream
 * and leaves a NULL output unwritten. */
LBM_API lbm_status lbm_adj_work_bytes(const lbm_sim *sim, size_t *bytes);
LBM_API lbm_status lbm_adj_reset(lbm_sim *sim, void *work);
LBM_API lbm_status lbm_adj_seed(lbm_sim *sim, const void *state_T, const void *phi_target,
                                void *lam_T, void *work, double *loss);
LBM_API lbm_status lbm_adj_step(lbm_sim *sim, const void *state_t, const void *lam_next,
                                void *lam_t, void *work);
LBM_API lbm_status lbm_adj_init(lbm_sim *sim, const void *phi0, const void *lam_0,
                                void *phi0_bar, void *work);
LBM_API lbm_status lbm_adj_grads(lbm_sim *sim, void *work, double *dM, double *dsigma);

/* One checkpoint segment of the reverse sweep in one call: the recompute
 * of the segment's states and its n reverse steps, the sequence that
 * checkpoint-and-recompute repeats for every segment.  The step is the one
 * of Eqs. 22-32 (Sec. 3); the paper itself has no adjoint.
 *   n             steps in the segment (>= 1), t0 .. t0+n-1
 *   states        device buffer of n levels, `level_stride` bytes apart
 *                 (>= lbm_state_bytes, 256-byte aligned, as is `states`):
 *                 level 0 holds s_{t0} (the checkpoint) on entry; levels
 *                 1 .. n-1 are overwritten with s_{t0+1} .. s_{t0+n-1},
 *                 computed by the forward step
 *   lam           lambda_{t0+n} on entry, lambda_{t0} on return
 *   lam_tmp       a second lambda buffer (scratch), not lam
 *   work          the adjoint work buffer; the segment's dL/dM, dL/dsigma
 *                 contributions are added to its running totals
 * Same result, bit for bit, as n - 1 calls of lbm_step's kernel followed
 * by n calls of lbm_adj_step.  Asynchronous on the handle's stream; the
 * handle's own state and step count are untouched.  With
 * lbm_adj_set_graph(sim, 1) the launch sequence is captured in a CUDA graph
 * on the first call and replayed by later calls with the same n, buffers
 * and stride (a call with others captures again); graph replay needs a
 * stream other than the default stream.  Errors: as lbm_adj_step, plus
 * LBM_ERR_ARG for n < 1, lam == lam_tmp, a NULL buffer or a bad stride or
 * alignment, and for lbm_adj_set_graph(sim, 1) on the default stream. */
LBM_API lbm_status lbm_adj_segment(lbm_sim *sim, int64_t n, void *states, size_t level_stride,
                                   void *lam, void *lam_tmp, void *work);
LBM_API lbm_status lbm_adj_set_graph(lbm_sim *sim, int on);

/* The same sweep with the recompute of each segment overlapped with the
 * reverse steps of the one after it, for a caller that alternates two
 * state buffers of K levels:
 *   lbm_adj_recompute        levels 1 .. n-1 of `states` from level 0 (the
 *                            recompute half of lbm_adj_segment), on the
 *                            handle's stream;
 *   lbm_adj_reverse_overlap  the n reverse steps of `states` (levels 0 ..
 *                            n-1 already recomputed; lam, lam_tmp, work as
 *                            lbm_adj_segment) on the handle's stream, while
 *                            a second stream recomputes levels 1 .. n_next-1
 *                            of `next_states` (a different buffer, same
 *                            stride) from its level 0, which the caller has
 *                            filled with the next segment's checkpoint by
 *                            work issued before this call on the handle's
 *                            stream.  n_next = 0 (or 1): nothing to
 *                            recompute.  Work issued after the call on the
 *                            handle's stream runs after both halves.
 * Per segment the results equal lbm_adj_segment's bit for bit.  The second
 * stream and its two events are created on the current device by the first
 * call with n_next > 1 and live as long as the handle.  With
 * lbm_adj_set_graph(sim, 1) each call is captured as one CUDA graph (both
 * streams) and replayed by later calls with the same sizes and buffers; the
 * graphs of the last two distinct calls are kept.  Errors: as
 * lbm_adj_segment (for both buffers), plus LBM_ERR_ARG for n_next < 0 or
 * next_states == states. */
LBM_API lbm_status lbm_adj_recompute(lbm_sim *sim, int64_t n, void *states, size_t level_stride);
LBM_API lbm_status lbm_adj_reverse_overlap(lbm_sim *sim, int64_t n, void *states,
                                           size_t level_stride, void *lam, void *lam_tmp,
                                           void *work, int64_t n_next, void *next_states);

/* ------------------------------------------------------------------ batches
 * The batched form: n independent domains, each with its own size and
 * parameters (one dtype for the whole batch; every nx a multiple of 8; not
 * the deviation storage), advanced together by one persistent kernel
 * launch per time step.  The launch works through one list of (domain,
 * strip, row segment) items, its CTAs claiming items from a counter in the
 * work buffer: 128-column strips (FP64: 64-column), the strips with more
 * than 64 active columns first, each group by decreasing cost.  A batch
 * whose strips all have at most 64 active columns (f32, f16s, bf16s) runs
 * a kernel of 64-column CTAs instead.  Per-domain results equal (bit for
 * bit in FP64 and the 16-bit forms; to FP32 rounding in FP32, where each
 * kernel may contract multiply-adds differently) those of
 * stepping each domain alone with lbm_step.  Fields and phi are
 * concatenated in domain order, each domain row-major [ny][nx] in the
 * field type.
 */
typedef struct lbm_batch lbm_batch; /* opaque handle, owned by the caller */

/* Device bytes for the populations (two levels per domain) and the work
 * buffer (domain and item tables, field staging, reduction partials). */
LBM_API lbm_status lbm_batch_buffer_sizes(const lbm_params *prms, int n, size_t *state_bytes,
                                          size_t *work_bytes);
/* Validate every domain (as lbm_create) and create the handle; `stream`
 * must be a non-default stream if graph replay is wanted. */
LBM_API lbm_status lbm_batch_create(const lbm_params *prms, int n, void *stream,
                                    lbm_batch **out);
/* Bind caller-owned device buffers and upload the domain and item tables
 * (synchronises the stream). */
LBM_API lbm_status lbm_batch_bind_buffers(lbm_batch *b, void *state, size_t state_bytes,
                                          void *work, size_t work_bytes);
/* Equilibrium initial state of every domain from the concatenated phi
 * (u = 0), device or host memory (on_host). */
LBM_API lbm_status lbm_batch_init_phi(lbm_batch *b, const void *phi, int on_host);
/* Advance every domain n steps: per step one launch of the strip kernel,
 * plus one of the narrow-strip kernel when some strips have at most 64
 * active columns (forms that have one: f32, f16s, bf16s); with graph replay
 * on, two steps per replay of a captured CUDA graph. */
LBM_API lbm_status lbm_batch_step(lbm_batch *b, int64_t n);
/* Work items of one step: *wide for the strip kernel, *narrow for the
 * narrow-strip kernel (0 when that launch is skipped).  Either pointer may
 * be NULL.  Errors: LBM_ERR_ARG (null handle), LBM_ERR_STATE (no buffers
 * bound yet). */
LBM_API lbm_status lbm_batch_work_items(const lbm_batch *b, int *wide, int *narrow);
/* Switch CUDA-graph replay of lbm_batch_step on (1) or off (0). */
LBM_API lbm_status lbm_batch_set_graph(lbm_batch *b, int use_graph);
/* Rows per work item (>= 16; default 64): the tile shape of the batch. */
LBM_API lbm_status lbm_batch_set_segment(lbm_batch *b, int seg_h);
/* Time candidate segment heights (16 .. 256) over `steps` steps each on the
 * current state and keep the fastest.  The state advances by the timed
 * steps; re-initialise afterwards if that matters. */
LBM_API lbm_status lbm_batch_autotune(lbm_batch *b, int steps, int *seg_h_out, double *ms_out);
/* Concatenated phi, ux, uy, p of the current time level (any may be NULL),
 * device or host pointers (on_host; the stream is then synchronised). */
LBM_API lbm_status lbm_batch_fields(lbm_batch *b, void *phi, void *ux, void *uy, void *p,
                                    int on_host);
/* Per-domain sum(rho) and sum(phi) (n doubles each, host), FP64. */
LBM_API lbm_status lbm_batch_mass(lbm_batch *b, double *mass, double *phi_total);
/* Total cells, steps taken, current segment height. */
LBM_API int64_t lbm_batch_cells(const lbm_batch *b);
LBM_API int64_t lbm_batch_step_count(const lbm_batch *b);
LBM_API int lbm_batch_segment(const lbm_batch *b);
LBM_API const char *lbm_batch_last_error(const lbm_batch *b);
LBM_API void lbm_batch_destroy(lbm_batch *b);

/* ------------------------------------------------------------------ y-slabs
 * One domain decomposed into n y-slabs that are stepped separately and
 * exchange ghost rows: the domain decomposition of the step (Eqs. 22-32 act
 * within 3 rows: grad p <- p <- lap mu <- lap phi), with every slab on the
 * handle's device and device-to-device copies.  Slab i owns global rows
 * a_i .. b_i - 1 and holds 3 ghost rows on each side (across the wrap when
 * periodic in y; ghost rows past a wall are not used).  A step is
 *   1. the strip kernel on each slab's own rows: the n launches run side by
 *      side, slab i > 0 on a side stream forked from the handle's stream
 *      (the handle creates n - 1 streams and n events at bind and destroys
 *      them with itself), each sized for 1/n of the GPU,
 *   2. one copy launch moving the populations pushed across each slab edge
 *      (f and g slots 2, 5, 6 upward; 4, 7, 8 downward) to the slab that
 *      owns their row,
 *   3. one copy launch refreshing every ghost row (all 18 slots).
 * Every cell runs the same kernel body as lbm_step, so the gathered state
 * equals stepping the whole domain: bit for bit in FP64 and the 16-bit
 * forms, to FP32 rounding in FP32 (the slab kernel and the whole-domain
 * kernel are compiled separately and may contract multiply-adds
 * differently).  Requirements: nx a
 * multiple of 8; every slab >= 3 rows.  `row_starts` (n entries, the first
 * 0, increasing) gives a_i; NULL splits ny evenly.  States are levels in
 * the layout of lbm_get_state for the whole domain (device memory).
 */
typedef struct lbm_slabs lbm_slabs; /* opaque handle, owned by the caller */

/* Device bytes of the slabs' populations (two levels each) and of the work
 * buffer (the copy tables).  Errors: LBM_ERR_ARG (message in
 * lbm_create_error). */
LBM_API lbm_status lbm_slabs_buffer_sizes(const lbm_params *prm, int n_slabs,
                                          const int *row_starts, size_t *state_bytes,
                                          size_t *work_bytes);
/* Validate (as lbm_create plus the slab requirements) and create. */
LBM_API lbm_status lbm_slabs_create(const lbm_params *prm, int n_slabs, const int *row_starts,
                                    void *stream, lbm_slabs **out);
/* Bind caller-owned, 256-byte aligned device buffers and upload the copy
 * tables (synchronises the stream). */
LBM_API lbm_status lbm_slabs_bind_buffers(lbm_slabs *s, void *state, size_t state_bytes,
                                          void *work, size_t work_bytes);
/* Load a whole-domain level (device) into the slabs, ghost rows included,
 * and set the step counter. */
LBM_API lbm_status lbm_slabs_scatter(lbm_slabs *s, const void *level, int64_t step);
/* Write the slabs' current state as a whole-domain level (device). */
LBM_API lbm_status lbm_slabs_gather(lbm_slabs *s, void *level, int64_t *step);
/* Advance n steps (asynchronous on the handle's stream, which waits for
 * the side streams before the copies; n + 2 launches per step). */
LBM_API lbm_status lbm_slabs_step(lbm_slabs *s, int64_t n);
/* Rows a_i .. b_i - 1 owned by slab i. */
LBM_API lbm_status lbm_slabs_rows(const lbm_slabs *s, int i, int *a, int *b);
LBM_API int64_t lbm_slabs_step_count(const lbm_slabs *s);
LBM_API const char *lbm_slabs_last_error(const lbm_slabs *s);
LBM_API void lbm_slabs_destroy(lbm_slabs *s);

/* ------------------------------------------------------------------ 3-D
 * The same step on D3Q19 (Sec. 3 says the scheme carries over to other
 * lattices; the paper works in 2-D): every formula of Eqs. 22-32 with
 * three-component vectors, weights 1/3 (rest), 1/18 (6 axis directions),
 * 1/36 (12 edge diagonals), c_s^2 = 1/3, the isotropic stencils built from
 * those weights, body force F_b = (0, -(rho - rho_ref) gravity, 0).
 * Periodic in x, y and z; LBM_F32 or LBM_F64; nx * ny * nz < 2^31 and
 * ny, nz <= 65535.
 * prm->bc_y must be LBM_PERIODIC and prm->gradp_lag 0.  Fields are
 * [nz][ny][nx], x fastest, in the field type, on the device.  A step is
 * four launches: phi, mu, p (each into the work buffer), then the
 * collision and push into the other level (populations f_0..18, g_0..18,
 * 2 x 152 B per cell in FP32).
 */
typedef struct lbm3_sim lbm3_sim; /* opaque handle, owned by the caller */

/* Device bytes of the two population levels and of the work buffer
 * (phi, mu, p fields and reduction partials).  Errors: LBM_ERR_ARG. */
LBM_API lbm_status lbm3_buffer_sizes(const lbm_params *prm, int nz, size_t *state_bytes,
                                     size_t *work_bytes);
LBM_API lbm_status lbm3_create(const lbm_params *prm, int nz, void *stream, lbm3_sim **out);
/* Caller-owned, 256-byte aligned device buffers. */
LBM_API lbm_status lbm3_bind_buffers(lbm3_sim *s, void *state, size_t state_bytes, void *work,
                                     size_t work_bytes);
/* Equilibrium initial state from phi (p = 0, u = (ux, uy, uz), NULL = 0);
 * device pointers of the field type. */
LBM_API lbm_status lbm3_init_phi(lbm3_sim *s, const void *phi, const void *ux, const void *uy,
                                 const void *uz);
/* Advance n >= 0 steps (asynchronous). */
LBM_API lbm_status lbm3_step(lbm3_sim *s, int64_t n);
/* phi, rho, p, u, mu of the current level (device pointers or NULL). */
LBM_API lbm_status lbm3_fields(lbm3_sim *s, void *phi, void *rho, void *p, void *ux, void *uy,
                               void *uz, void *mu);
/* sum rho and sum phi in FP64, fixed order; synchronises the stream. */
LBM_API lbm_status lbm3_mass(lbm3_sim *s, double *mass, double *phi_total);
/* Laplace diagnostic of a droplet centred at (xc, yc, zc), nominal radius R:
 * total pressure of Sec. 4.2 averaged over r < R - 2W minus over
 * r > R + 2W; R_eff = (3 V / 4 pi)^(1/3) from the volume of fluid A. */
LBM_API lbm_status lbm3_laplace(lbm3_sim *s, double xc, double yc, double zc, double R,
                                double *dP, double *R_eff);
LBM_API int64_t lbm3_step_count(const lbm3_sim *s);
LBM_API const char *lbm3_last_error(const lbm3_sim *s);
LBM_API void lbm3_destroy(lbm3_sim *s);

/* The mass diagnostic of lbm_mass for callers that cannot allocate device
 * memory.  The paper has no counterpart: this is a library convenience.
 *
 * lbm_mass keeps its reduction partials in the work buffer the caller binds
 * to a handle.  Callers whose device memory is a fixed budget owned by
 * someone else, plug-ins that must not grow the process's device footprint,
 * and loops that cannot take cudaMalloc's implicit device-wide
 * synchronisation have no such buffer to give.  This entry point needs none
 * and no handle: its scratch is a static 64 KB device array inside the
 * library (every GPU that loads the library holds it until the process
 * exits), and it calls no allocating routine.
 *
 *   prm        parameters of the domain (validated as by lbm_buffer_sizes)
 *   level      device pointer to ONE time level of populations in the
 *              library's layout for prm->dtype, e.g. what lbm_get_state
 *              writes (read only)
 *   stream     cudaStream_t to run on; it is synchronised before return
 *   mass, phi_total  host outputs (either may be NULL): sum rho and sum phi,
 *              accumulated in FP64 in a fixed order
 *
 * Limits and errors: grids of at most 2^28 cells (16384 x 16384); larger
 * grids return LBM_ERR_NOMEM without touching the GPU.  LBM_ERR_ARG for
 * invalid parameters or a NULL level, LBM_ERR_NONFINITE for NaN/Inf sums,
 * LBM_ERR_CUDA for a failed CUDA call; lbm_create_error() gives the
 * message.  Every call looks up the scratch array's device address on the
 * current device (cudaGetSymbolAddress) and synchronises `stream`, so it
 * cannot be part of a stream capture.  All calls in the process share the one scratch array,
 * which keeps the last call's contents (each call writes every slot it
 * reads, so nothing needs clearing): calls that overlap on the GPU, from
 * any thread or stream, race with each other. */
LBM_API lbm_status lbm_mass_noalloc(const lbm_params *prm, const void *level, void *stream,
                                    double *mass, double *phi_total);

/* ---------------------------------------------------------- ALU ceiling
 * Measured FMA throughput of the current device, the arithmetic ceiling
 * the step kernels are compared with.  The paper has no counterpart: it
 * measures the GPU, not the method.
 *   kind       0: FP32 scalar FMA, 1: FP32 FMA on packed pairs (f32x2),
 *              2: FP64 FMA
 *   fma_per_s  host output: FMA operations per second (FLOP/s = 2x)
 * Launches a warm-up and a timed kernel (8 independent FMA chains per
 * thread, 16 CTAs of 256 threads per SM) on a stream of its own and
 * synchronises it; about 10-50 ms.  Allocates and frees 2 KB of device
 * memory.  Errors: LBM_ERR_ARG (kind out of range, NULL output),
 * LBM_ERR_CUDA (a failed CUDA call). */
LBM_API lbm_status lbm_alu_peak(int kind, double *fma_per_s);

#ifdef __cplusplus
}
#endif

#endif /* LBM_H */
