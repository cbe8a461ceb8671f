/*
 * libvd -- B300-native non-rigid lattice solve of VolumeDeform (arXiv 1603.08161).
 *
 * One lattice G of nx x ny x nz grid points (node i = x + nx (y + ny z), x fastest;
 * canonical position t^_i = origin + spacing * (x, y, z)) carries a displacement
 * u_i = t_i - t^_i and a rotation R_i per node (Sec. 4).  Each frame, vd_solve runs
 * the flip-flop Gauss-Newton minimisation of
 *     E_total = w_s E_sparse + w_d E_dense + w_r E_reg                 (Eq. 1)
 * with the point-to-plane term (Eq. 2), the feature term (Eq. 3) and the ARAP prior
 * (Eq. 4): positions by Jacobi-preconditioned CG on the normal equations with the
 * rotations fixed, then rotations by per-node Procrustes with positions fixed
 * (Sec. 7.1).  Every step runs in this library's own CUDA kernels (sm_103a).
 *
 * Conventions shared by every call:
 *   - Arrays at the boundary are row-major AoS float32: points and displacements
 *     n x 3, rotations n x 9 (row-major 3x3), depth H x W (row v, column u), in metres.
 *   - `mem` says where a pointer lives: VD_MEM_HOST (pageable or pinned host memory)
 *     or VD_MEM_DEVICE (device memory of the current CUDA device, e.g. from torch).
 *     The caller keeps ownership of every pointer it passes; the library copies what
 *     it needs before the call returns (inputs) or writes outputs before it returns.
 *   - Every call returns a vd_status and never throws.  On an error the lattice state
 *     is unchanged, except after VD_ERR_NUMERIC / VD_ERR_TIMEOUT from a solve, which
 *     leave the warp of the last completed Gauss-Newton iteration.  vd_last_error()
 *     gives a one-line reason.
 *   - One handle is used by one host thread at a time.  Work is ordered on the
 *     lattice's CUDA stream.
 */
#ifndef VD_H
#define VD_H

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    VD_OK = 0,
    VD_ERR_INVALID_ARG = 1, /* bad pointer, size or parameter */
    VD_ERR_OOM = 2,         /* device or host allocation failed */
    VD_ERR_CUDA = 3,        /* a CUDA runtime call failed (message in vd_last_error) */
    VD_ERR_STATE = 4,       /* call out of order, e.g. vd_solve before vd_set_frame */
    VD_ERR_NUMERIC = 5,     /* non-finite energy */
    VD_ERR_TIMEOUT = 6      /* a bounded device-side wait gave up */
} vd_status;

enum { VD_ACTIVE_SURFACE = 0, VD_ACTIVE_ALL = 1 };
enum { VD_PREC_FP32 = 0, VD_PREC_MIXED = 1 };
enum { VD_MEM_HOST = 0, VD_MEM_DEVICE = 1 };
enum { VD_INIT_PREV = 0, VD_INIT_ZERO = 1 };

typedef struct vd_lattice vd_lattice; /* opaque; owned by the library */

typedef struct {
    int nx, ny, nz;     /* nodes per axis, each >= 2 */
    float origin[3];    /* canonical position of node (0, 0, 0), metres */
    float spacing;      /* lattice spacing h > 0, metres */
    int active_mode;    /* VD_ACTIVE_SURFACE: M = cells holding a sample or a sparse
                           point plus their one-ring (Sec. 6-7); VD_ACTIVE_ALL: every node */
    int precision;      /* VD_PREC_FP32 (FP32 storage and arithmetic, FP64 reductions)
                           or VD_PREC_MIXED (BF16 storage of per-sample records and normals) */
    void *cuda_stream;  /* cudaStream_t to order work on; NULL = a stream of the library's own */
} vd_lattice_desc;

typedef struct {
    float w_sparse, w_dense, w_reg; /* w_s, w_d, w_r of Eq. 1 */
    float eps_d, eps_n, eps_v;      /* pruning thresholds of Sec. 5.1, Phi_r(x) = 1 - x / eps_r */
    int gn_iters;                   /* flip-flop (Gauss-Newton) iterations, >= 1 */
    int cg_iters;                   /* PCG iterations per position step, >= 0 */
    double cg_tol;                  /* stop PCG once r.z <= cg_tol^2 * r0.z0 (0: run all) */
    int fixed_association;          /* 1: associate once, at the first iteration */
    int init;                       /* VD_INIT_PREV: start from the current warp;
                                       VD_INIT_ZERO: from u = 0, R = I */
} vd_solve_params;

typedef struct {
    double e_total, e_dense, e_sparse, e_reg; /* Eq. 1-4 after the last iteration, under its association */
    int gn_done;          /* Gauss-Newton iterations completed */
    int cg_done;          /* PCG iterations of the last position step */
    int n_valid_corr;     /* dense correspondences with w_c > 0 (last association) */
    int n_degenerate_rot; /* nodes whose best rotation was not unique (last rotation step) */
    int n_refined;        /* association decisions re-taken in FP64 (last association) */
    int status;           /* vd_status of the solve */
} vd_solve_report;

/* Create a lattice (all u = 0, R = I).  Allocates device memory for the lattice state.
 * VD_ERR_INVALID_ARG for dims < 2 or spacing <= 0. */
vd_status vd_create_lattice(const vd_lattice_desc *desc, vd_lattice **out);

/* Free the lattice and all its device memory.  NULL is accepted. */
vd_status vd_destroy_lattice(vd_lattice *lat);

/* Input of one frame (Sec. 5.1): the depth map D_t (W x H, 0 = invalid), intrinsics
 * K = (fx, fy, cx, cy), the global pose (R | t) of Sec. 4 as 12 floats (row-major R,
 * then t; NULL = identity) -- K and pose are always host pointers, whatever `mem`
 * says -- and the n_src source samples p^_c with normals n^_c in
 * canonical coordinates (the samples of the rasterised model).  Computes the target
 * normal map, bins the samples by lattice cell and builds the active set M.
 * Samples whose cell is not inside the lattice, or whose position or normal is not
 * finite, get w_c = 0; a depth that is not a positive finite number (0, negative, NaN,
 * infinite) marks an invalid pixel.  Synchronous. */
vd_status vd_set_frame(vd_lattice *lat, const float *depth, int W, int H, const float K[4],
                       const float pose[12], const float *src_pts, const float *src_nrm, int n_src,
                       int mem);

/* The S sparse feature pairs of Eq. 3: canonical positions f^_s and observed
 * positions f_s (S x 3 each).  Pairs outside the lattice (or with a non-finite
 * canonical position) are ignored; an observed position that is not finite makes the
 * energy non-finite, and the next solve returns VD_ERR_NUMERIC.  Applies to the
 * next vd_set_frame / vd_solve; S = 0 clears them.  Synchronous. */
vd_status vd_set_correspondences(vd_lattice *lat, const float *canon, const float *target, int S,
                                 int mem);

/* Per-frame flip-flop solve (Sec. 7.1): gn_iters x (associate, position step by PCG,
 * rotation step, energy).  Replays a captured CUDA graph of the whole schedule.
 * Synchronous: returns after the solve finished and fills `out` (may be NULL). */
vd_status vd_solve(vd_lattice *lat, const vd_solve_params *params, vd_solve_report *out);

/* Enqueue the same solve on the lattice's stream and return at once; vd_get_report
 * waits for it.  Inputs must not change until then. */
vd_status vd_solve_async(vd_lattice *lat, const vd_solve_params *params);

/* Wait for the last enqueued solve and return its report. */
vd_status vd_get_report(vd_lattice *lat, vd_solve_report *out);

/* Copy the warp out: disp = u (nx*ny*nz x 3), rot = R (nx*ny*nz x 9, may be NULL). */
vd_status vd_get_warp(const vd_lattice *lat, float *disp, float *rot, int mem);

/* The same read without waiting for it: on the lattice's stream the warp (after the work
 * enqueued before, e.g. vd_solve_async) is converted into a readback buffer of the
 * lattice's own (allocated on the first call), and a second stream of the lattice copies
 * it to disp / rot (either may be NULL), so that the copy overlaps what the caller
 * enqueues next (the next frame's vd_set_frame and vd_solve_async, which no longer wait
 * for it).  mem: VD_MEM_HOST (page-locked buffers, for the copy to run asynchronously)
 * or VD_MEM_DEVICE.  The buffers hold the warp once vd_get_warp_wait returns; a later
 * vd_get_warp_async waits on the GPU for the previous copy to finish before it reuses the
 * readback buffer.  VD_ERR_INVALID_ARG for another mem; VD_ERR_CUDA if a copy cannot be
 * enqueued. */
vd_status vd_get_warp_async(vd_lattice *lat, float *disp, float *rot, int mem);

/* Wait until the copies of the last vd_get_warp_async have landed. */
vd_status vd_get_warp_wait(vd_lattice *lat);

/* Replace the warp (warm start, or resume a sequence): disp may be NULL (u = 0),
 * rot may be NULL (R = I). */
vd_status vd_set_warp(vd_lattice *lat, const float *disp, const float *rot, int mem);

/* One-line description of the last error on this lattice ("" if none). */
const char *vd_last_error(const vd_lattice *lat);

/* ---- step API: the individual stages of one Gauss-Newton iteration, for callers
 * ---- that drive their own schedule (and for per-stage checks). */

/* Number of nodes in the active set M of the current frame. */
vd_status vd_num_active(const vd_lattice *lat, int *n_active);

/* Active-set mask (nx*ny*nz bytes, 1 = in M). */
vd_status vd_get_active(const vd_lattice *lat, unsigned char *mask, int mem);

/* Target normal map n^a of the current frame (H x W x 3; zero where invalid):
 * central differences of the back-projected depth, oriented towards the camera. */
vd_status vd_get_target_normals(const vd_lattice *lat, float *nrm, int mem);

/* Projective association (Sec. 5.1) of every source sample at the current warp. */
vd_status vd_step_associate(vd_lattice *lat, const vd_solve_params *params);

/* Result of the last association in the caller's sample order: target pixel
 * (py * W + px, or -1), confidence w_c, and the dense residual
 * sqrt(w_d w_c) n^a . (S(p^_c) - p^a) at the current warp.  Any pointer may be NULL. */
vd_status vd_get_association(vd_lattice *lat, const vd_solve_params *params, int *pix, float *w,
                             float *r, int mem);

/* Right-hand side b = -J^T r and Jacobi diagonal diag(J^T J) of the position step at
 * the current warp and association (nx*ny*nz x 3 each; 0 outside M; may be NULL). */
vd_status vd_step_rhs(vd_lattice *lat, const vd_solve_params *params, float *b, float *diag, int mem);

/* Ap = J^T J p for a full-lattice vector p (nx*ny*nz x 3; entries outside M ignored);
 * p_Ap (may be NULL) receives p.Ap accumulated in FP64. */
vd_status vd_step_apply(vd_lattice *lat, const vd_solve_params *params, const float *p, float *Ap,
                        double *p_Ap, int mem);

/* Position step: PCG on J^T J delta = -J^T r from delta = 0.  Writes delta
 * (nx*ny*nz x 3, may be NULL) and the iterations done; with `apply` != 0 also adds
 * delta to u. */
vd_status vd_step_pcg(vd_lattice *lat, const vd_solve_params *params, float *delta, int *iters,
                      int apply, int mem);

/* Rotation step (Sec. 7.1): per-node Procrustes fit of R_i to the current positions. */
vd_status vd_step_fit_rotations(vd_lattice *lat, int *n_degenerate);

/* E_total, E_dense, E_sparse, E_reg (Eq. 1-4) at the current warp under the last
 * association. */
vd_status vd_step_energy(vd_lattice *lat, const vd_solve_params *params, double out[4]);

/* ---- global rigid pose (Sec. 6: "dense projective ICP") ----
 *
 * Estimates the frame's global pose (R_g, t_g) with the lattice warp held fixed:
 * `iters` Gauss-Newton steps of the point-to-plane energy of the dense samples,
 *     sum_c w_c (n^a_c . (R_g q_c + t_g - p^a_c))^2,   q_c = p^_c + sum_k alpha_k u_k,
 * each after a projective association at the current pose (Sec. 5.1: nearest pixel,
 * Phi_d, Phi_n, Phi_v and w_c, with the thresholds of `params`), over the perturbation
 * R_g <- exp([omega]x) R_g, t_g <- t_g + tau (6 x 6 normal equations, Cholesky in FP64,
 * the pose kept in FP64 between steps).  Starts from the pose of the last vd_set_frame;
 * the result becomes the frame's pose for the following solves and is written to
 * pose_out (12 floats, row-major R_g then t_g, host; may be NULL).  steps (may be NULL)
 * gets the steps taken: fewer than iters when the normal matrix stopped being positive
 * definite (too few correspondences), the pose then being the last one reached.
 * e_hist (host, iters doubles, may be NULL) gets the energy before each step.  Runs on
 * the lattice's stream and waits for it.  iters in [0, 64]. */
vd_status vd_estimate_pose(vd_lattice *lat, const vd_solve_params *params, int iters, float pose_out[12],
                           int *steps, double *e_hist);

/* ---- cached B^T B (Sec. 7.1) ----
 *
 * The paper precomputes and caches B^T B (the data constraints' part of the normal
 * matrix) before the PCG iterations, because a cell may hold thousands of constraints.
 * With VD_APPLY_CACHED the dense samples' part of J^T J is built once per association as
 * one 24 x 24 block per occupied lattice cell (w_d sum_j (alpha_j (x) g_j)(alpha_j (x)
 * g_j)^T over the cell's samples, 2,304 bytes per cell) and every PCG iteration applies
 * the blocks; the sparse pairs and the ARAP stencil stay matrix-free.  The result is
 * the same matrix as the matrix-free apply (VD_APPLY_MATRIX_FREE, the default, which
 * reads each sample's record every iteration), in a different summation order.
 * VD_APPLY_AUTO takes the cached blocks when the frame has at least 32 samples per
 * occupied cell (the coarse levels of a hierarchy start in this mode). */
enum { VD_APPLY_MATRIX_FREE = 0, VD_APPLY_CACHED = 1, VD_APPLY_AUTO = 2 };

/* Select how the samples' J^T J p is applied (takes effect from the next solve or
 * step call; may allocate the blocks).  VD_ERR_INVALID_ARG for an unknown mode. */
vd_status vd_set_apply_mode(vd_lattice *lat, int mode);

/* The selected mode and whether the current frame uses the cached blocks (either may be
 * NULL). */
vd_status vd_get_apply_mode(const vd_lattice *lat, int *mode, int *cached_now);

/* Autotune the apply for this frame and these parameters: time two solves with each of
 * VD_APPLY_MATRIX_FREE and VD_APPLY_CACHED (after one warm-up solve each), keep the
 * faster.  ms_out (may be NULL) gets the time per solve of each (ms).  Runs the solve
 * six times, so the warp changes (VD_INIT_PREV) -- save and restore it around the call
 * if it matters. */
vd_status vd_tune_apply(vd_lattice *lat, const vd_solve_params *params, int *mode_out, float ms_out[2]);

/* ---- measurement support ---- */

/* Kernel classes that vd_profile can time inside the captured solve graph. */
enum {
    VD_KC_ASSOCIATE = 0, VD_KC_RHS = 1, VD_KC_APPLY_STENCIL = 2, VD_KC_APPLY_SAMPLES = 3,
    VD_KC_UPDATE_X = 4, VD_KC_UPDATE_P = 5, VD_KC_ROTATION = 6, VD_KC_ENERGY = 7,
    VD_KC_PCG = 8, /* the persistent position step (one cooperative launch per step) */
    VD_KC_COUNT = 9
};

/* Select one kernel class (or -1 for none) to bracket with CUDA events inside the
 * solve graph; the graph is re-captured on the next solve. */
vd_status vd_profile_select(vd_lattice *lat, int kernel_class);

/* Total device time (ms) and launch count of the selected class over the solves
 * since the last call (the counters are then reset). */
vd_status vd_profile_read(vd_lattice *lat, double *total_ms, int *launches);

/* Number of kernel launches of one vd_solve with the given parameters, and of one
 * vd_set_frame. */
vd_status vd_launch_counts(vd_lattice *lat, const vd_solve_params *params, int *per_solve,
                           int *per_frame);

/* The partition of the persistent position step (Sec. 7.1) that vd_solve uses for this
 * lattice (any pointer may be NULL): CTAs and slots per CTA (0, 0 when the position step
 * is streamed instead), and for an all-nodes lattice the brick of by x bz x-rows that each
 * CTA owns (0 x 0: contiguous slot ranges); padded = 1 when the bricks' rows are padded
 * to a multiple of 4 slots or the far bricks are ragged (nx % 4 != 0, or ny, nz not
 * multiples of by, bz). */
vd_status vd_pcg_plan(vd_lattice *lat, int *ctas, int *chunk, int *by, int *bz, int *padded);

/* ---- batched solve: many independent lattices in one graph launch ---- */

typedef struct vd_batch vd_batch; /* opaque; references the lattices, owns no lattice data */

/* Group `count` lattices (each with its frame and correspondences set, all on the
 * current device) for batched solves.  The lattices must outlive the batch. */
vd_status vd_batch_create(vd_lattice *const *lattices, int count, vd_batch **out);

/* Free the batch (not the lattices).  NULL is accepted. */
vd_status vd_batch_destroy(vd_batch *batch);

/* Solve every lattice of the batch with the same parameters (the flip-flop of Sec. 7.1
 * per lattice, exactly as vd_solve): one captured CUDA graph, launched on the first
 * lattice's stream, in which the lattices at or above a size threshold (chosen by
 * vd_batch_tune; none by default) run first, one after another, each with its
 * persistent position step, and every other lattice's schedule is a branch on one of
 * several concurrent streams.  `out` (may be NULL) receives `count` reports.
 * Synchronous. */
vd_status vd_batch_solve(vd_batch *batch, const vd_solve_params *params, vd_solve_report *out);

/* Enqueue the batched solve and return; vd_batch_get_reports waits for it. */
vd_status vd_batch_solve_async(vd_batch *batch, const vd_solve_params *params);
vd_status vd_batch_get_reports(vd_batch *batch, vd_solve_report *out);

/* Autotune the batch for these parameters: time the solve for each candidate number
 * of concurrent branches (1, 2, 4, ... up to the batch size) and branch order (largest
 * lattice first, or as given), then for the fastest of those each size threshold
 * (2^19, 2^17, 2^15, 2^13 active nodes) above which lattices run ahead with their
 * persistent position step, then the waves of the shared-memory position step
 * (VD_BATCH_WAVES) with 8 / 16 branches and 2^20 (no sample bound) / 4096 / 1024
 * samples per CTA (vd_batch_set_wave_share), then the persistent form with vectors in
 * global memory (VD_BATCH_GLOBAL) for 256 / 512 threads, 1 / 2 / 4 CTAs per SM, sample
 * weights 1 / 4 and 8 / 16 branches; keep the fastest.  Runs the solve several times (the
 * lattices' warps change).  Reports the number of branches and the time per batched
 * solve (ms). */
vd_status vd_batch_tune(vd_batch *batch, const vd_solve_params *params, int *streams, float *ms);

/* Set the batch's schedule directly instead of by vd_batch_tune: `streams` concurrent
 * branches (1..64), branch order (largest_first != 0: by active nodes, descending;
 * else as given), and the size from which lattices run ahead, one after another, with
 * their persistent position step (active nodes >= run_ahead_nodes; a value above any
 * lattice's size, e.g. 2^31 - 1, disables it; 0 makes every lattice run ahead).
 * VD_ERR_INVALID_ARG for NULL or out-of-range values. */
vd_status vd_batch_set_plan(vd_batch *batch, int streams, int largest_first, long long run_ahead_nodes);

/* Forms of a batch's position steps (the `form` of vd_batch_set_persistent). */
#define VD_BATCH_BRANCHES 0 /* every lattice's schedule as a branch of the graph */
#define VD_BATCH_GLOBAL 1   /* one cooperative kernel over all lattices, vectors in global memory */
#define VD_BATCH_WAVES 2    /* one cooperative kernel, lattices in waves of the shared-memory step */

/* Run the batch's position steps as one persistent cooperative kernel per Gauss-Newton
 * iteration, the other stages of the iteration as per-lattice branches between these
 * launches.  form = VD_BATCH_GLOBAL: the CTAs, ctas_per_sm per SM, each of `threads`
 * threads (256 or 512), are split among the lattices in proportion to (active nodes +
 * sample_weight x samples), at least one each; each lattice's group runs its PCG (the
 * recurrence of vd_solve, vectors in global memory) with its own barriers and
 * reductions.  form = VD_BATCH_WAVES (threads, ctas_per_sm and sample_weight are then
 * not used): one CTA per SM; each lattice takes the fewest CTAs whose slots fit in
 * shared memory and runs the position step of vd_solve on them (vectors in shared and
 * tensor memory, its own barriers); the lattices' CTA groups are packed into waves of
 * at most one CTA per SM (largest first, first fit), and each CTA runs its groups wave
 * after wave within the one launch.  Every lattice must fit on the SMs: at most
 * SMs x 6,144 active nodes (909,312 on a 148-SM B300, e.g. a 96^3 lattice).  form =
 * VD_BATCH_BRANCHES returns to the graph of per-lattice schedules.  VD_ERR_INVALID_ARG
 * for another form, other thread counts, ctas_per_sm outside [1, 8] or a negative
 * weight; a setting the device cannot hold (the CTAs must all be resident) fails at the
 * next solve. */
vd_status vd_batch_set_persistent(vd_batch *batch, int form, int threads, int ctas_per_sm, float sample_weight);

/* VD_BATCH_WAVES: a lattice's CTA group holds at most `samples_per_cta` of its samples
 * per CTA (beside the shared-memory bound on its nodes), up to one CTA per SM; a CTA's
 * sample warps take their share of the samples' J^T J p while its stencil warps run.
 * Default 2^20 (in effect no sample bound); vd_batch_tune searches it.
 * VD_ERR_INVALID_ARG below 32. */
vd_status vd_batch_set_wave_share(vd_batch *batch, int samples_per_cta);

/* The batch's current plan (any pointer may be NULL): the form of its position steps
 * (VD_BATCH_*), the threads, CTAs per SM and sample weight of VD_BATCH_GLOBAL, and the
 * number of concurrent branches. */
vd_status vd_batch_get_plan(const vd_batch *batch, int *persistent, int *threads, int *ctas_per_sm,
                            float *sample_weight, int *streams);

/* Kernel launches in one batched solve (after the first solve or tune). */
vd_status vd_batch_launch_count(const vd_batch *batch, int *launches);

/* The CTA groups of the last persistent build (VD_BATCH_GLOBAL or VD_BATCH_WAVES):
 * `ctas` (may be NULL; room for the batch's lattice count) receives each lattice's CTAs,
 * `waves` (may be NULL) the number of waves over all launch sets (0 for
 * VD_BATCH_GLOBAL).  Both are zero before the first such build. */
vd_status vd_batch_get_groups(const vd_batch *batch, int *ctas, int *waves);

/* One-line description of the batch's last error. */
const char *vd_batch_last_error(const vd_batch *batch);

/* Convenience: create a batch, solve once, destroy it (re-captures every call). */
vd_status vd_solve_batch(vd_lattice *const *lattices, int count, const vd_solve_params *params,
                         vd_solve_report *out);

/* ---- allocation-free variant ----
 *
 * The paper has no counterpart to this entry point; it exists for callers that cannot
 * let the library allocate device memory: programs that reserve their whole device
 * memory budget up front (real-time pipelines, embedded deployments) and processes
 * whose device memory belongs to another allocator (a framework's caching allocator),
 * where a cudaMalloc from inside the library could fail or fragment the pool.
 *
 * vd_fit_rotations_noalloc runs the rotation step of vd_step_fit_rotations on a lattice
 * in which every node is active, reading and writing only the caller's device arrays:
 *   disp    u, nx*ny*nz x 3 floats (node i = x + nx (y + ny z)), device memory
 *   rot_in  R before the step, nx*ny*nz x 9 floats (row-major 3x3), device memory
 *   rot_out R after the step, same layout, device memory (may equal rot_in)
 *   e_reg   (may be NULL) device double: E_reg (Eq. 4) with the new rotations
 *   n_degenerate (may be NULL) device int: nodes whose rotation was kept
 * It calls no cudaMalloc, cudaFree or allocating library routine.  Its scratch is one
 * fixed array in device memory of this library (VD_NOALLOC_MAX_NODES x 12 floats plus
 * 256 bytes, about 3 MB), which every device that loads the library keeps until the
 * process exits; lattices of more than VD_NOALLOC_MAX_NODES nodes return
 * VD_ERR_INVALID_ARG.  All calls share that scratch and each one clears the part that
 * must start at zero; calls that overlap on the GPU (different streams, or different
 * host threads) race on it, so serialise them.  The work is enqueued on cuda_stream
 * (NULL = the legacy default stream) and the function returns without waiting.  The
 * first call on a device looks up the scratch address on that device (with it
 * current); make that first call before any stream capture.  Errors: VD_ERR_INVALID_ARG
 * for bad sizes (any dimension, or their product, above VD_NOALLOC_MAX_NODES) or NULL
 * arrays; VD_ERR_CUDA if a CUDA call fails (there is no handle, so no vd_last_error
 * message), and also, before anything is enqueued, when a CUDA error from earlier work
 * of the calling thread is still pending: that error is left in place for the caller
 * to read with cudaGetLastError. */
#define VD_NOALLOC_MAX_NODES 65536
vd_status vd_fit_rotations_noalloc(int nx, int ny, int nz, float spacing, const float *disp,
                                   const float *rot_in, float *rot_out, double *e_reg,
                                   int *n_degenerate, void *cuda_stream);

/* ---- source samples on the GPU (Sec. 4: marching cubes; Sec. 5.1: rasterisation) ----
 *
 * The paper extracts the canonical iso-surface with data-parallel marching cubes (one
 * thread per cell, a prefix sum to compact the triangles) and rasterises the mesh,
 * deformed by the current warp, to obtain the sample points S(p^_c).  A renderer holds
 * one canonical mesh and a W x H z-buffer.
 *
 * Marching cubes: corner k of a cell is at (k & 1, (k >> 1) & 1, (k >> 2) & 1) and is
 * inside when its value is below the iso value; the case table is generated from a face
 * rule (walking each face counter-clockwise as seen from outside the cell, an edge
 * crossed from outside to inside opens a segment that closes at the next crossed edge;
 * the segments form loops, each cut into a fan from its lowest edge, edges numbered 4 A
 * + b + 2 c for the edge along axis A whose lower corner has the other two coordinates
 * (b, c)), which separates diagonal inside corners of a face the same way from both
 * cells and gives watertight, consistently oriented surfaces (normals toward values
 * above the iso value).  A vertex sits on its edge at t = (iso - g_a) / (g_b - g_a) from
 * the lower corner; its normal is the grid's central-difference gradient interpolated
 * the same way, normalised.  Triangles are ordered by cell (x fastest), then by the
 * table.
 *
 * Rasterisation: each vertex p^ becomes S(p^) = R_g (p^ + sum alpha_k u_k) + t_g with
 * the lattice's displacements (u = 0 outside the lattice, or everywhere when lat is
 * NULL) and the given pose, and projects to (f_x X / Z + c_x, f_y Y / Z + c_y), pixel
 * centres at integer coordinates.  A pixel centre with all three barycentric
 * coordinates >= 0 is covered (triangles with a vertex at Z <= 1e-3 are skipped); the
 * covering triangle of smallest depth 1 / sum(lambda_i / Z_i) wins, ties to the lower
 * index.  Its sample is the perspective-correct interpolation of the canonical vertices
 * and normals (normal renormalised). */
typedef struct vd_renderer vd_renderer; /* opaque; owned by the library */

/* A renderer for meshes of at most max_triangles triangles and W x H images. */
vd_status vd_renderer_create(int max_triangles, int W, int H, vd_renderer **out);
vd_status vd_renderer_destroy(vd_renderer *r);
const char *vd_renderer_last_error(const vd_renderer *r);

/* Marching cubes of the sx x sy x sz grid `sdf` (x fastest; `mem` says where it lives)
 * at origin (host, 3 floats) and spacing into the renderer's canonical mesh.
 * n_triangles (may be NULL) gets the surface's triangle count; VD_ERR_INVALID_ARG if it
 * exceeds max_triangles (the mesh then holds the first max_triangles).  Synchronous. */
vd_status vd_marching_cubes(vd_renderer *r, const float *sdf, int sx, int sy, int sz, const float origin[3],
                            float spacing, float iso, int mem, int *n_triangles);

/* The marching-cubes case table: the triangles of case cs (bit k set: corner k inside),
 * as edge triples written to edges (up to 30 ints, may be NULL); returns the triangle
 * count, or -1 for cs outside [0, 255].  Host only. */
int vd_mc_case(int cs, int *edges);

/* The canonical mesh: n_triangles x 9 vertex positions and normals (either may be NULL). */
vd_status vd_get_mesh(vd_renderer *r, float *tri, float *nrm, int mem);

/* Rasterise the mesh deformed by lat's warp (NULL: none) and `pose` (12 floats, host;
 * NULL: identity) with intrinsics K (host), and write the samples of the covered pixels
 * whose column and row are multiples of `stride`, in pixel order: canonical points and
 * normals (cap x 3 floats each) and (pix, may be NULL) their pixel indices v W + u.
 * count gets the number of such pixels (only the first cap are written).  Uses lat's
 * stream when lat is given (after its pending work), else the renderer's.  Synchronous. */
vd_status vd_render_samples(vd_renderer *r, const vd_lattice *lat, const float K[4], const float pose[12],
                            int stride, float *pts, float *nrm, int *pix, int cap, int *count, int mem);

/* ---- hierarchical coarse-to-fine solve (Sec. 7.2) ----
 *
 * A hierarchy nests levels - 1 coarse lattices on a lattice (level 0): level l has
 * n_{l-1} / 2 + 1 nodes per axis (integer division; node X of level l sits on node 2X of
 * level l - 1, one spacing past its end when n_{l-1} - 1 is odd), spacing 2^l h, the
 * same origin, active-set mode, precision and CUDA stream.  Every coarse cell is the
 * parent voxel of 2 x 2 x 2 cells of the level below; a coarse level gathers all the
 * constraints of level 0 (the dense samples and sparse pairs whose cell exists on level
 * 0) and expresses each trilinearly in its own nodes.  Each level's energy is Eq. 1-4 on
 * its own lattice with the same weights.  The hierarchy owns the coarse lattices; level
 * 0 stays the caller's and must outlive it. */
typedef struct vd_hierarchy vd_hierarchy; /* opaque; owned by the library */

/* levels >= 1 (1: level 0 alone), at most 8.  Allocates the coarse lattices. */
vd_status vd_hierarchy_create(vd_lattice *fine, int levels, vd_hierarchy **out);
vd_status vd_hierarchy_destroy(vd_hierarchy *h);

/* The lattice of one level (0 = the caller's), for vd_get_warp, vd_get_association and
 * the other per-lattice calls; coarse lattices belong to the hierarchy (do not destroy). */
vd_status vd_hierarchy_level(vd_hierarchy *h, int level, vd_lattice **out);

/* Coarse-to-fine solve of level 0's current frame.  params[k] is the schedule of level
 * levels - 1 - k (coarsest first, level 0 last); only the last entry's init is used
 * (VD_INIT_ZERO resets level 0's warp first).  Steps, on level 0's stream: the state of
 * every coarse level is restricted from the level below (displacement and rotation of
 * the coinciding node; along an axis past the end of the level below, the displacement
 * extrapolated linearly from its last two nodes); then from the coarsest level up: its
 * flip-flop solve (as vd_solve, starting from the restricted state), the trilinear
 * prolongation of its displacement increment to every node of the level below, and one
 * rotation step (Sec. 7.1) there; finally level 0's flip-flop solve.  A coarse level's
 * frame is copied from level 0 on the first solve after vd_set_frame or
 * vd_set_correspondences on level 0.  `out` (may be NULL) gets `levels` reports,
 * coarsest first.  Synchronous; the _async form enqueues and returns,
 * vd_hierarchy_get_reports waits.  An energy target set with vd_set_energy_target on a
 * level's lattice gates that level's iterations. */
vd_status vd_hierarchy_solve(vd_hierarchy *h, const vd_solve_params *params, vd_solve_report *out);
vd_status vd_hierarchy_solve_async(vd_hierarchy *h, const vd_solve_params *params);
vd_status vd_hierarchy_get_reports(vd_hierarchy *h, vd_solve_report *out);

/* One-line description of the hierarchy's last error. */
const char *vd_hierarchy_last_error(const vd_hierarchy *h);

/* ---- Gauss-Newton early stop ----
 *
 * With a target set, every later solve of this lattice ends its flip-flop loop after
 * the first iteration whose E_total (Eq. 1) is <= e_target; the report's gn_done counts
 * the iterations run.  A negative (or NaN) e_target removes the target.  The value is
 * stored on the device in stream order, so it may change between queued solves without
 * a new graph capture (setting or removing the target re-captures once). */
vd_status vd_set_energy_target(vd_lattice *lat, double e_target);

/* ---- failure injection (tests; the paper has no counterpart) ----
 *
 * With on != 0, every later persistent position step of this lattice waits at its first
 * grid barrier for one more arrival than it has CTAs.  No CTA can supply it, so the
 * bounded wait runs out (about 2e9 SM cycles, one second at 2 GHz), the kernel sets its
 * error word and returns, and the solve reports VD_ERR_TIMEOUT with the warp of the
 * last completed iteration (each Gauss-Newton iteration's step waits once).  The CUDA
 * context stays usable; on = 0 restores normal solves.  Solves that stream the position
 * step (no cooperative launch) are unaffected.  Returns VD_ERR_INVALID_ARG for NULL. */
vd_status vd_test_stall_barrier(vd_lattice *lat, int on);

/* ---- check of the position step's grid reduction (tests; the paper has no counterpart) ----
 *
 * Runs `rounds` reductions of G per-CTA FP64 partials (parts: rounds x G, host) through
 * the barrier reduction of the persistent position step, in a cooperative launch of G
 * CTAs (G <= the SM count), round k using round k-1's sum as the scale of its
 * fixed-point path (as the position step uses the previous p.Ap or r.z); out (host,
 * 2 x rounds doubles) gets per round the barrier's sum and the FP64 sum of the partials
 * in CTA order.  The barrier's sum agrees with the row sum to FP64 rounding when the
 * round takes the row path (no positive previous sum, a partial too large, or a sum below
 * 1/16 of the scale, as after a sharp drop), and to 3e-7 relative on the fixed-point path.  Allocates and frees its own
 * device memory; VD_ERR_INVALID_ARG without cooperative launches or for bad sizes. */
vd_status vd_test_grid_reduce(const double *parts, int G, int rounds, double *out);

/* ---- learned warm start (the paper has no counterpart: Sec. 7.1 starts each frame from
 * the previous frame's warp) ----
 *
 * A 3-level 3D U-Net (16 / 32 / 64 channels, 3x3x3 convolutions, 2x2x2 average pooling,
 * nearest up-sampling, skip concatenations) over the lattice grid, in BF16 with FP32
 * accumulation on the tensor cores.  Input per node (6 floats, node-major, node i =
 * x + nx (y + ny z)): u_i / h and the data-term gradient scaled by one Jacobi step,
 * b_i / (h (diag_i + 2 w_r |N_i|)) with b = -J_data^T r; output per node (3 floats): the
 * predicted change of u in units of h.  Training minimises the mean squared error to
 * solver increments (u_f - u_{f-1}) / h with Adam (beta 0.9 / 0.999, eps 1e-8).
 * Arrays passed to the network calls are device memory; a handle's buffers are shared
 * by its calls, so calls on one handle must not overlap on the GPU. */
typedef struct vd_unet vd_unet; /* opaque; owned by the library */

/* Network for an nx x ny x nz grid (each a multiple of 4); parameters drawn from a
 * seeded He-normal initialisation (the output layer scaled by 0.01), Adam moments 0. */
vd_status vd_unet_create(int nx, int ny, int nz, unsigned long long seed, vd_unet **out);
vd_status vd_unet_destroy(vd_unet *net);
vd_status vd_unet_dims(const vd_unet *net, int *nx, int *ny, int *nz);
/* Number of FP32 parameters: per layer, weights [27][Cin][Cout] (tap = 9 dz + 3 dy + dx
 * over offsets -1..1) then bias [Cout], layers in the order a1 b1 a2 b2 a3 b3 c2 d2 c1 d1
 * head. */
vd_status vd_unet_num_params(const vd_unet *net, int *n);
vd_status vd_unet_get_params(vd_unet *net, float *host, int n);
vd_status vd_unet_set_params(vd_unet *net, const float *host, int n);
/* Gradients of the loss of the last vd_unet_train_step, same layout (host array). */
vd_status vd_unet_get_grads(vd_unet *net, float *host, int n);
/* out3 = net(in6) (the output layer in FP32); synchronous / enqueued on cuda_stream
 * (NULL = the handle's stream). */
vd_status vd_unet_forward(vd_unet *net, const float *in6, float *out3);
vd_status vd_unet_forward_async(vd_unet *net, const float *in6, float *out3, void *cuda_stream);
/* One Adam step with learning rate lr (lr = 0: loss and gradients only) on
 *     loss = sum_i w_i |net(in6)_i - target3_i|^2 / (3 n),
 * w_i = 1 + surface_weight (>= 0) at nodes whose gradient input (channels 3-5) is not
 * all zero, else 1; `loss` (host, may be NULL) gets the loss before the step. */
vd_status vd_unet_train_step(vd_unet *net, const float *in6, const float *target3,
                             float surface_weight, float lr, double *loss);
/* Parameters to / from a file: "VDUNET01", int32 layer count, int32 Cin[], int32 Cout[],
 * int32 parameter count, FP32 parameters, all little-endian.  A file whose shapes do
 * not match gives VD_ERR_INVALID_ARG. */
vd_status vd_unet_save(vd_unet *net, const char *path);
vd_status vd_unet_load(vd_unet *net, const char *path);

/* Test support: an intermediate tensor of the last vd_unet_forward / vd_unet_train_step
 * (activations after the forward pass; gradients with respect to them after the
 * backward pass, in their final state: ReLU masks applied, the skip and pooling
 * contributions summed) as dense floats converted from the stored BF16, layout
 * D x H x W x C (channels fastest, x, then y, then z), C the stored channel count
 * (padded to a multiple of 16; padding channels are zero).  dims (may be NULL) gets
 * D, H, W, C; host may be NULL to query dims only, else it needs n >= D H W C floats.
 * Synchronises the handle's stream.  VD_ERR_INVALID_ARG for a bad id or a short n. */
enum {
    VD_UNET_T_X = 0, VD_UNET_T_E1A, VD_UNET_T_E1, VD_UNET_T_P1, VD_UNET_T_E2A, VD_UNET_T_E2, VD_UNET_T_P2,
    VD_UNET_T_E3A, VD_UNET_T_E3, VD_UNET_T_CAT2, VD_UNET_T_D2A, VD_UNET_T_D2, VD_UNET_T_CAT1, VD_UNET_T_D1A,
    VD_UNET_T_D1, VD_UNET_T_GOUT, VD_UNET_T_GD1, VD_UNET_T_GD1A, VD_UNET_T_GCAT1, VD_UNET_T_GD2,
    VD_UNET_T_GD2A, VD_UNET_T_GCAT2, VD_UNET_T_GE3, VD_UNET_T_GE3A, VD_UNET_T_GP2, VD_UNET_T_GE2,
    VD_UNET_T_GE2A, VD_UNET_T_GP1, VD_UNET_T_GE1, VD_UNET_T_GE1A, VD_UNET_T_COUNT
};
vd_status vd_unet_get_tensor(vd_unet *net, int id, float *host, long long n, int dims[4]);

typedef struct {
    double e_start;      /* E_total (Eq. 1) of the warp before the call, under its association */
    double e_predicted;  /* E_total of the predicted warp (rotations refitted), its association */
    int used_prediction; /* 1 if the prediction was kept (finite and lower energy) */
    int status;
} vd_warm_report;

/* The network input for the current frame at the current warp (nx*ny*nz x 6 floats,
 * zero at inactive nodes), written to in6 (`mem` as elsewhere).  Synchronous. */
vd_status vd_warm_features(vd_lattice *lat, const vd_solve_params *params, float *in6, int mem);

/* Learned warm start of the current frame: features, network, candidate warp u + h net
 * (with the rotations refitted to it), kept only if its energy is below the current
 * warp's; then call vd_solve with init = VD_INIT_PREV.  The network's grid must equal the
 * lattice's.  Enqueued on the lattice's stream; with `out` non-NULL it waits and fills
 * it, else vd_get_warm_report does. */
vd_status vd_warm_start(vd_lattice *lat, vd_unet *net, const vd_solve_params *params,
                        vd_warm_report *out);
vd_status vd_get_warm_report(vd_lattice *lat, vd_warm_report *out);

#ifdef __cplusplus
}
#endif
#endif /* VD_H */
