/*
 * ba.h -- C ABI of the GB300 local bundle-adjustment library.
 *
 * The library runs the Levenberg-Marquardt iteration of a local (cluster)
 * bundle adjustment on one GPU: per-observation reprojection residuals and
 * Jacobians, Schur-complement assembly of the reduced camera system, a damped
 * Cholesky solve, point back-substitution, and the cost / gain-ratio test.
 *
 * Problem statement it follows (arXiv 2511.06152, Sec. 3.2):
 *   - a cluster C_l = {I_k1 ... I_kM} of M images, each with an initial pose
 *     (R_k, T_k) from GNSS/IMU in local ENU coordinates;
 *   - observations p_kj of points X_j, Eq. 5: p_kj = pi(K R_k^T (X_j - T_k)),
 *     R_k camera->world, T_k the camera centre, pi(x,y,z) = (x/z, y/z);
 *     K carries one focal length f, the principal point (cx, cy) and Brown
 *     radial (k1, k2) and tangential (p1, p2) terms on normalised coordinates;
 *   - the robust cost of Eq. 7, E = sum_k sum_j rho(||p_kj - pi(...)||^2), with
 *     rho = Huber of threshold huber_delta_px acting on the squared 2-D norm,
 *     residuals whitened by sigma_px; GNSS position and IMU attitude priors
 *     whitened by sigma_gnss_m / sigma_imu_rad are added for every free camera;
 *   - overlap images carried over from the previous cluster may be held fixed.
 * The cost the library minimises is
 *   F = 1/2 sum rho(s)/sigma_px^2 + 1/2 sum_free(|T - T_gnss|^2/sigma_gnss^2
 *       + |Log(R_imu^T R)|^2 / sigma_imu^2).
 * The optimiser (the paper names none) is LM with Marquardt scaling
 * D = clamp(diag(J^T J), 1e-6, 1e32), pred = 1/2 d^T (mu D d + g), gain =
 * (F - F(x+d)) / pred, accept when gain > 0, and Nielsen's mu/nu update.
 * Parameters move by R <- R Exp(dtheta), T <- T + dT, X <- X + dX.
 *
 * Conventions for every entry point:
 *   - Arrays are row-major.  Doubles are IEEE binary64, int32_t / uint8_t as
 *     named.  A rotation is 9 doubles (3x3, camera->world).
 *   - Pointers in ba_cluster_desc are host pointers when ptr_kind is
 *     BA_PTR_HOST and device pointers (current device) when BA_PTR_DEVICE.
 *     The library copies every input into device memory it owns before
 *     ba_create_cluster returns; the caller may free its buffers afterwards.
 *   - Output buffers are caller-owned and written before the call returns
 *     (ba_get_state, ba_solve_step, ba_run, ba_solve_batch, ba_poll).
 *   - Return codes only; nothing is thrown across the ABI.  A numerical
 *     failure (a reduced camera system that is not positive definite) is
 *     reported in the per-step status and handled as a rejected LM step.
 *   - Solves run on the stream given in ba_config; ba_create_cluster uploads
 *     on a stream of its own and the serving scheduler runs on its own.  Any
 *     entry point may be called from any thread: the context serialises its
 *     bookkeeping with one lock, which is not held during a cluster's host
 *     presort, a serving round or the device run of ba_solve_batch.
 *   - Reductions are deterministic: every sum runs in a fixed order that
 *     depends only on the cluster, never on the batch it runs in, so a
 *     cluster's result is bit-identical alone and in any batch.
 */
#ifndef BA_GB300_H
#define BA_GB300_H

#include <stddef.h>
#include <stdint.h>

#if defined(__GNUC__)
#define BA_API __attribute__((visibility("default")))
#else
#define BA_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

typedef int32_t ba_status;
#define BA_OK 0
#define BA_PENDING 1
#define BA_ERR_INVALID (-1)   /* malformed argument or problem data */
#define BA_ERR_BUDGET (-2)    /* would exceed hbm_budget_bytes or slots: retry later */
#define BA_ERR_NOT_PD (-3)    /* damped reduced camera system not positive definite */
#define BA_ERR_TIMEOUT (-4)   /* a bounded wait expired */
#define BA_ERR_CUDA (-5)      /* a CUDA runtime call failed */
#define BA_ERR_NOT_FOUND (-6) /* unknown cluster id or ticket */

#define BA_FP64 0  /* every step in binary64 */
#define BA_MIXED 1 /* per-observation work in binary32, solve and cost in binary64 */

#define BA_PTR_HOST 0
#define BA_PTR_DEVICE 1

#define BA_MAX_TRACK 32 /* observations of one point in one cluster */

typedef struct ba_ctx ba_ctx;
typedef uint64_t ba_cluster_id; /* 0 is never a valid id */
typedef uint64_t ba_ticket;     /* 0 is never a valid ticket */

typedef struct {
  int32_t device;            /* CUDA device ordinal */
  void* stream;              /* cudaStream_t to run on; NULL: the library creates one */
  uint64_t hbm_budget_bytes; /* device memory the context may hold; 0 = unlimited */
  int32_t precision;         /* BA_FP64 or BA_MIXED */
  int32_t n_slots;           /* clusters the serving scheduler runs at once (ba_submit); 0 = 64 */
  int32_t refine_steps;      /* iterative-refinement passes against the binary64 S after the Cholesky
                                solve; <0 = the default: 1 in BA_FP64, 0 in BA_MIXED (whose system
                                carries binary32 rounding from the per-observation terms, far above
                                the double-float factor's) */
  int32_t flags;             /* BA_FLAG_* */
  const char* tune_table;    /* NULL, or the path of a tuning table (ba_tune_table_lookup): the
                                entry for this GPU and precision, if any, is applied at ba_init */
} ba_config;

#define BA_FLAG_KERNEL_TIMING 1 /* bracket every kernel with CUDA events (also inside graphs) */
/* Failure injection, for tests of the failure handling only: in mixed
 * precision, the linearise+Schur kernel waits for each CTA's first staged
 * chunk on a barrier that nothing completes, gives up after 1 ms, and takes
 * the path of an expired copy wait (the copies it issued are waited for, the
 * clusters of its chunks get BA_ERR_TIMEOUT in their step status and the
 * step is rejected; nothing faults or hangs).  No effect in BA_FP64. */
#define BA_FLAG_INJECT_COPY_TIMEOUT 2
/* Reduced camera systems of more than 32 free images are factored on the
 * tensor cores by default: the factor kept as double-float (binary32 pairs),
 * its dense products computed exactly from 8-bit digit matrices on the bf16
 * tensor cores (Ozaki's error-free splitting), the solution refined against
 * S in binary64 by the configured refinement passes.  This flag selects the
 * binary64 CUDA-core factorisation instead (same envelope, same refinement),
 * for comparisons. */
#define BA_FLAG_BIG_FP64_FACTOR 4
/* Reduced camera systems of up to 32 free images are factored in shared
 * memory by one CTA: in binary64 in BA_FP64, in double-float on the binary32
 * pipe in BA_MIXED (the system equilibrated by powers of two), then the
 * configured refinement passes against the binary64 S.  This flag selects
 * the double-float factorisation in BA_FP64 too, for comparisons (no effect
 * in BA_MIXED). */
#define BA_FLAG_SMALL_DF_FACTOR 8

/* Kernel kinds reported by ba_kernel_stats, in this order. */
#define BA_KERNEL_LIN_SCHUR 0      /* per chunk: residuals, Jacobians, point blocks, Schur partial sums */
#define BA_KERNEL_PARTIAL_REDUCE 1 /* chunk partial sums -> per-camera / per-pair sums */
#define BA_KERNEL_FACTOR 2         /* assembly, Cholesky, solve, refinement, candidate poses */
#define BA_KERNEL_BACKSUB 3        /* point back-substitution and candidate cost */
#define BA_KERNEL_LM_UPDATE 4      /* gain ratio, accept/reject, damping update */
#define BA_KERNEL_COST_TILES 5     /* cost at the current state (per tile) */
#define BA_KERNEL_COST_INIT 6      /* cost at the current state (per cluster) */
#define BA_KERNEL_OTHER 7          /* arm, reset, gather, camera copies, diagnostics */
#define BA_KERNEL_KINDS 8

typedef struct {
  int32_t n_cams, n_pts, n_obs;
  int32_t ptr_kind;             /* BA_PTR_HOST or BA_PTR_DEVICE */
  const double* intr;           /* [n_cams][7]: f, cx, cy, k1, k2, p1, p2 */
  const double* R;              /* [n_cams][9]: initial rotations, camera->world */
  const double* T;              /* [n_cams][3]: initial centres, metres */
  const double* X;              /* [n_pts][3]: initial points, metres */
  const double* R_prior;        /* [n_cams][9]: IMU attitude */
  const double* T_prior;        /* [n_cams][3]: GNSS position */
  const uint8_t* fixed;         /* [n_cams]: 1 = pose held fixed; NULL = none fixed */
  const int32_t* obs_cam;       /* [n_obs] camera of each observation */
  const int32_t* obs_pt;        /* [n_obs] point of each observation */
  const double* obs_uv;         /* [n_obs][2] pixel measurement */
  double sigma_px;              /* pixel standard deviation (> 0) */
  double huber_delta_px;        /* Huber threshold in pixels (> 0) */
  double sigma_gnss_m;          /* GNSS sigma; 0 switches the position prior off */
  double sigma_imu_rad;         /* IMU sigma; 0 switches the attitude prior off */
  double mu0;                   /* initial damping; <= 0 means 1e-4 */
  ba_cluster_id warm_from;      /* 0, or a live cluster whose state seeds this one */
  const int32_t* warm_cam_map;  /* [n_cams] camera index in warm_from, or -1 (host pointer) */
  const int32_t* warm_pt_map;   /* [n_pts] point index in warm_from, or -1 (host pointer) */
} ba_cluster_desc;

typedef struct {
  double cost;     /* F(x) at the current state */
  double grad_inf; /* max |g| over free-camera and point coordinates */
  int32_t n_free;  /* free cameras */
  int32_t reserved;
} ba_lin_info;

typedef struct {
  int32_t accepted;
  int32_t status;   /* BA_OK or BA_ERR_NOT_PD */
  double F_before;  /* F(x) */
  double F_after;   /* F(x + d) */
  double predicted; /* pred = 1/2 d^T (mu D d + g) */
  double gain;      /* (F_before - F_after) / pred */
  double mu_used;   /* damping of this step */
  double mu;        /* damping after the update */
  double nu;
} ba_step_info;

typedef struct {
  int32_t max_iters; /* LM iterations at most (accepted and rejected both count) */
  int32_t reserved;
  double ftol;       /* 0: run max_iters.  > 0: the cluster also stops after an accepted
                        step, other than its first iteration, that lowered F by no more
                        than ftol * F (F before that step).  Finite and >= 0. */
} ba_solve_opts;

typedef struct {
  int32_t status;     /* BA_OK, or the last step's error */
  int32_t iters;      /* iterations run by this call (or ticket) */
  int32_t accepted;   /* accepted steps: all of the cluster's, since its creation or reset */
  int32_t reserved;
  double initial_cost; /* F before the first iteration: ba_solve_batch with a trace that holds
                          every iteration; 0 otherwise (ba_poll included) */
  double final_cost;
  double latency_ms;  /* submit -> completion seen by the scheduler (ba_poll) */
} ba_result;

/* Create a context on cfg->device: the device-side home of the clusters a
 * flight produces one after another (Sec. 3.2: BA runs on each cluster C_l
 * as it fills, on the same platform, in real time; Sec. 1, Eq. 1 gives the
 * per-image time budget it serves).  cfg (host, caller-owned, read during the
 * call only): device ordinal, stream, device-memory budget, precision,
 * serving slots, refinement passes, flags.  *out (host) receives the handle,
 * which the caller releases with ba_shutdown.  BA_ERR_INVALID for a NULL
 * argument or an unknown precision; BA_ERR_CUDA when the device cannot be
 * used (no GPU, or a runtime call failed). */
BA_API ba_status ba_init(ba_ctx** out, const ba_config* cfg);

/* Copy a cluster to the device and presort its observation index
 * (point-major and camera-major orders, camera-pair table).  The cluster is
 * the unit of the paper's local BA (Sec. 3.2): M images C_l = {I_k1 .. I_kM},
 * including images of adjacent strips, each with its GNSS/IMU pose as the
 * initial value (R, T) and as the prior (R_prior, T_prior); the tracks of
 * the points matched inside the cluster (obs_cam, obs_pt, obs_uv: the
 * observations p_kj of Eq. 5 and Eq. 6); and the overlap images carried over
 * from the previous cluster, the first half of which are held fixed
 * (`fixed`).  d (host, caller-owned) and the arrays it points to (host or
 * device memory by d->ptr_kind) are read during the call only.  *out (host)
 * receives the id; the cluster lives until ba_destroy_cluster or
 * ba_shutdown.  Fails with BA_ERR_INVALID on indices out of range, repeated
 * (camera, point) pairs, more than BA_MAX_TRACK observations of one point,
 * non-finite input, or no free camera; with BA_ERR_BUDGET when the device
 * memory it needs would exceed the context's budget (retry once other
 * clusters are freed); BA_ERR_CUDA when an upload fails. */
BA_API ba_status ba_create_cluster(ba_ctx* ctx, const ba_cluster_desc* d, ba_cluster_id* out);

/* Sizes and self-check of the presorted tables (ba_presort_host). */
typedef struct {
  int32_t n_free, n_tiles, n_chunks, n_pairs; /* free images, tiles, chunks, co-visible free pairs */
  int32_t n_cam_jobs, n_pair_jobs;            /* image and pair reduction jobs over all chunks */
  int32_t max_lanes;                          /* most lanes one chunk's jobs use (<= 256) */
  int32_t fallback_chunks;                    /* chunks with more jobs than threads (one lane per job) */
  int32_t tiles_per_chunk;                    /* of this precision */
  int32_t checks_failed;                      /* 0 when every table invariant holds */
  int64_t n_free_obs, n_pair_entries;         /* observations of free images; co-visible observation pairs */
  uint64_t digest;                            /* FNV-1a of the tables' bytes */
  char message[128];                          /* first failed check, or why the call failed */
} ba_presort_info;

/* Host only: the presort ba_create_cluster runs (validation, point order,
 * point-major order, tiles, chunks, reduction jobs and their lanes, pair
 * table, elimination order and envelope) on a cluster in host memory
 * (d->ptr_kind = BA_PTR_HOST; warm-start fields ignored), for the tables of
 * `precision`, with no context and no device: nothing is uploaded.  The
 * tables are then checked against what the observations alone imply, rebuilt
 * by brute force: every observation once in point-major order, tiles of whole
 * points, each chunk's image and pair jobs holding exactly the observations
 * and co-visible observation pairs of its points in order, counts
 * non-increasing, lanes inside the CTA, the envelope holding every pair.
 * threads > 0 builds the chunk tables on exactly that many threads (the
 * tables must not depend on it; compare digests), 0 lets the library choose.
 * Fails like ba_create_cluster on invalid input (BA_ERR_INVALID, reason in
 * out->message); a failed table check is reported in out->checks_failed. */
BA_API ba_status ba_presort_host(const ba_cluster_desc* d, int32_t precision, int32_t threads, ba_presort_info* out);

/* Warm start an existing cluster from a live one (the cluster transition of
 * Sec. 3.2: a new window reuses the optimised overlap images and their
 * points).  cam_map[dst n_cams] / pt_map[dst n_pts] (host arrays) give, for
 * each camera / point of dst, its index in src or -1.  The current state of
 * the mapped cameras and points of src is copied on the device into dst
 * (also into the state ba_reset restores), and so is src's damping state:
 * dst starts from src's current mu and nu (the LM state stays resident on
 * the device from one window to the next), which ba_reset also restores.  Neither cluster may be queued or
 * running in the serving scheduler.  Enqueued on the context's stream; this
 * split from ba_create_cluster lets a caller presort a window while the
 * previous one is still being solved. */
BA_API ba_status ba_warm_start(ba_ctx* ctx, ba_cluster_id dst, ba_cluster_id src, const int32_t* cam_map,
                               const int32_t* pt_map);

/* Cluster transition (Sec. 3.2, Eq. 8).  For every image of cluster dst that
 * is free in dst and mapped to an image of src (cam_map[dst n_cams], host
 * array: its index in src or -1), its current pose in dst is replaced by the
 * weighted average of its current poses in src and in dst, the weights being
 * its numbers of observations in src and in dst: the position is the weighted
 * mean; the orientation is the point at fraction w_dst / (w_src + w_dst) on
 * the geodesic from the src orientation to the dst orientation (the weighted
 * mean on SO(3) of two rotations).  Images fixed in dst keep their pose (they
 * hold the optimised pose of src already).  Typically called once dst has
 * been solved.  Neither cluster may be queued or running in the serving
 * scheduler.  Enqueued on the context's stream.  BA_ERR_NOT_FOUND for an
 * unknown id, BA_ERR_INVALID for a null map or an index out of range. */
BA_API ba_status ba_transition(ba_ctx* ctx, ba_cluster_id dst, ba_cluster_id src, const int32_t* cam_map);

/* ---- Cluster formation: image footprints and their overlaps ----
 *
 * Sec. 3.1 projects each image's four corners onto a digital surface model
 * (the image's footprint, a ground quadrilateral) and detects the overlap
 * between new images and images of neighbouring strips by comparing
 * footprints; Sec. 3.2 brings those adjacent-strip images into the cluster. */

/* DSM raster, host memory: heights h[iy * nx + ix] (metres, same frame as
 * the poses) at (x0 + ix * dx, y0 + iy * dy); nx, ny >= 2; bilinear between
 * nodes, positions outside clamped to the raster. */
typedef struct ba_dsm {
  int32_t nx, ny;
  double x0, y0, dx, dy;
  const double* h;
} ba_dsm;

/* Footprints of n images (host arrays): intr[n][7], R[n][9] (camera->world),
 * T[n][3]; images of width x height pixels.  corners[n][4][3] (host, output):
 * the first surface point of the rays through pixels (0,0), (w,0), (w,h),
 * (0,h) (lens distortion not applied; the ray is sampled at most half a
 * raster cell apart from where it enters the DSM's height range, then the
 * bracketed hit is bisected 60 times).  A corner whose ray does not point
 * down is NaN.  BA_ERR_INVALID for bad sizes or null pointers. */
BA_API ba_status ba_footprints(ba_ctx* ctx, int32_t n, const double* intr, double width, double height,
                               const double* R, const double* T, const ba_dsm* dsm, double* corners);

/* Areas of intersection, in the ground plane, of every footprint of qa[na]
 * with every footprint of qb[nb] (host arrays of [4][3] corners as written by
 * ba_footprints; convex quadrilaterals, either orientation): area[na][nb]
 * (host, output).  Sutherland-Hodgman clipping; binary64. */
BA_API ba_status ba_footprint_overlaps(ba_ctx* ctx, int32_t na, const double* qa, int32_t nb, const double* qb,
                                       double* area);

/* Patch transfer through the poses (Sec. 3.1, Eq. 3): the centres p0[n][2]
 * (pixels) of patches of image 0 (intrinsics intr0[7], pose R0[9] camera->
 * world, T0[3]) moved to the m images of intr[m][7], R[m][9], T[m][3]: the
 * point at depth lambda along image 0's optical axis through each centre,
 * projected into image k with the pinhole part (f, cx, cy) of its
 * intrinsics (Eq. 3 has no distortion term).  p[m][n][2] (host, output;
 * target-major; NaN where the point is behind image k) and inside[m][n]
 * (host, output, may be NULL): 1 where the transferred centre lies in
 * [0, width) x [0, height), the patch-keyed correspondences.  Binary64.
 * BA_ERR_INVALID for bad sizes, null pointers or a non-finite lambda. */
BA_API ba_status ba_patch_transfer_poses(ba_ctx* ctx, int32_t n, const double* p0, const double* intr0,
                                         const double* R0, const double* T0, double lambda, int32_t m,
                                         const double* intr, const double* R, const double* T, double width,
                                         double height, double* p, uint8_t* inside);

/* Patch transfer by the footprints (Sec. 3.1, Eq. 4): patch centres
 * q0[n][2] of image 0 in a ground frame, moved to each of m images by the
 * in-plane rotation theta[k] (radians, R = [cos -sin; sin cos]) about the
 * patch-grid centre c[2] and the displacement g[k] - g0 of the image centres
 * (g[m][2], g0[2]): q[m][n][2] (host, output; target-major).  Binary64.
 * BA_ERR_INVALID for bad sizes or null pointers. */
BA_API ba_status ba_patch_transfer_planar(ba_ctx* ctx, int32_t n, const double* q0, const double* c,
                                          const double* g0, int32_t m, const double* theta, const double* g,
                                          double* q);

/* The robust cost F(x) of Eq. 7 at the current state (Huber on each
 * squared pixel residual over sigma_px^2, halved, plus half the squared
 * whitened GNSS/IMU prior residuals of the free images) and the infinity norm
 * of its gradient over the free images' 6-vectors and the points' 3-vectors,
 * from one linearisation (Sec. 3.2).  out (host, caller-owned) must not be
 * NULL.  Blocking.  BA_ERR_NOT_FOUND for an unknown id, BA_ERR_INVALID for a
 * NULL out or a cluster in service. */
BA_API ba_status ba_linearize(ba_ctx* ctx, ba_cluster_id id, ba_lin_info* out);

/* One Levenberg-Marquardt iteration of the local BA of Sec. 3.2 (Eq. 7) on
 * one cluster: linearise, eliminate the points (Schur complement), damp,
 * factor and solve the reduced camera system (BA_FP64: binary64 with one
 * refinement pass; BA_MIXED: double-float), back-substitute the points,
 * evaluate F at the candidate, accept or reject it and update the damping.
 * Blocking; *out (host, may be NULL)
 * receives the step record.  A reduced or point system that is not positive
 * definite is a rejected step with status BA_ERR_NOT_PD in the record, not a
 * failed call.  BA_ERR_NOT_FOUND for an unknown id, BA_ERR_INVALID for a
 * cluster in service. */
BA_API ba_status ba_solve_step(ba_ctx* ctx, ba_cluster_id id, ba_step_info* out);

/* iters (>= 0) iterations of ba_solve_step on one cluster in one device-side
 * sequence (one CUDA-graph launch, no host round trip between iterations).
 * trace (host, caller-owned, may be NULL) receives [iters] step records; the
 * device keeps the last 256, so for iters > 256 the earlier records are
 * zero.  Blocking.  Errors as ba_solve_step; BA_ERR_INVALID for iters < 0. */
BA_API ba_status ba_run(ba_ctx* ctx, ba_cluster_id id, int32_t iters, ba_step_info* trace);

/* iters LM iterations on n clusters at once: the clusters are dealt to
 * batch_chains (ba_tune) concurrent launch chains, every kernel of an
 * iteration is one launch over a chain's clusters, and the whole sequence is
 * one CUDA-graph launch.  Each cluster's result equals its ba_run result bit
 * for bit, for any number of chains.
 * results[n] may be NULL; trace may be NULL or [n][iters].  While the device
 * runs the batch the context stays open to other threads (creating, reading
 * or solving other clusters); the batch's own clusters are in service until
 * the call returns: calls that write or free them fail with BA_ERR_INVALID
 * ("cluster is in service"), and reads (ba_get_state,
 * ba_reprojection_errors) are queued behind the batch on the context's
 * stream, so they return its final state. */
BA_API ba_status ba_solve_batch(ba_ctx* ctx, const ba_cluster_id* ids, int32_t n, int32_t iters,
                         ba_result* results, ba_step_info* trace);

/* Restore a cluster's initial state (the one given at create, or the one a
 * warm start wrote), its initial damping (mu0 and nu = 2 from create, or the
 * mu and nu a warm start carried over) and clear its LM counters.  Enqueued on the context's
 * stream.  BA_ERR_NOT_FOUND for an unknown id, BA_ERR_INVALID for a cluster
 * in service. */
BA_API ba_status ba_reset(ba_ctx* ctx, ba_cluster_id id);

/* ba_reset on n clusters in one launch (enqueued on the context's stream;
 * returns without waiting). */
BA_API ba_status ba_reset_batch(ba_ctx* ctx, const ba_cluster_id* ids, int32_t n);

/* Queue a cluster for the serving scheduler (non-blocking): the sliding
 * clusters of Sec. 3.2 solved as they arrive.  The scheduler admits queued
 * clusters into free slots between LM iterations, so work submitted while
 * others run joins the running batch; each iteration is the arithmetic of
 * ba_solve_step.  Work the caller queued on the context's stream before the
 * call (creation, warm start, reset) is ordered before the cluster's first
 * iteration.  The cluster is in service until its ticket completes.  *out
 * receives a ticket for ba_poll.  BA_ERR_NOT_FOUND for an unknown id;
 * BA_ERR_INVALID for NULL opts or out, max_iters <= 0, a negative or
 * non-finite ftol, a cluster of more than 32 free images, or a cluster
 * already submitted. */
BA_API ba_status ba_submit(ba_ctx* ctx, ba_cluster_id id, const ba_solve_opts* opts, ba_ticket* out);

/* BA_PENDING while the ticket's cluster is queued or running; BA_OK with
 * *out (host, may be NULL) filled once it has finished, which consumes the
 * ticket.  BA_ERR_NOT_FOUND for an unknown or consumed ticket.  Thread-safe. */
BA_API ba_status ba_poll(ba_ctx* ctx, ba_ticket t, ba_result* out);

/* Copy the current state out in binary64 (double-float states rounded):
 * the refined exterior orientations (R_k, T_k) of the cluster's images and
 * the refined points X_j, the unknowns of Eq. 7 (Sec. 3.2) that the cluster
 * transition hands on to the next cluster.  R[n_cams][9] (row-major,
 * camera->world), T[n_cams][3], X[n_pts][3] in the caller's camera and point
 * order.  Caller-owned buffers: host pointers when
 * ptr_kind is BA_PTR_HOST, device pointers when BA_PTR_DEVICE; any may be
 * NULL.  Blocking (ordered behind the work on the context's stream).
 * BA_ERR_NOT_FOUND for an unknown id. */
BA_API ba_status ba_get_state(ba_ctx* ctx, ba_cluster_id id, double* R, double* T, double* X, int32_t ptr_kind);

/* The current states of n clusters at once, each as ba_get_state returns it
 * (binary64, caller's point order), into host memory: R[i], T[i], X[i] are
 * the host destinations of cluster ids[i] ([nc][9], [nc][3], [np][3]; an
 * entry, or a whole array, may be NULL).  The clusters go in groups of at
 * most 32 MiB of state: per group one device export per cluster into one
 * block, one copy to the host through pinned memory the context keeps, one
 * wait.  The clusters are in service during the call, which does not hold
 * the context's lock meanwhile (other threads may create or solve other
 * clusters).  BA_ERR_NOT_FOUND if an id is unknown, BA_ERR_INVALID if one is
 * in service (nothing is written then). */
BA_API ba_status ba_get_state_batch(ba_ctx* ctx, const ba_cluster_id* ids, int32_t n, double* const* R,
                                    double* const* T, double* const* X);

/* Per-observation reprojection error norms |pi(K R^T (X - T)) - p| in pixels
 * (the model of Eq. 5, the residual of Eq. 6) at the current state, in the
 * caller's observation order, into err[n_obs] (host, caller-owned).
 * BA_ERR_INVALID for a NULL err, BA_ERR_NOT_FOUND for an unknown id. */
BA_API ba_status ba_reprojection_errors(ba_ctx* ctx, ba_cluster_id id, double* err);

/* Sizes of a cluster's presorted tables: the units the kernels of one LM
 * iteration process (used to state work per launch, and to plan capacity).
 * Observations and points count as after validation; pair entries are the
 * (observation, observation) pairs of one point whose two images are both
 * free, i.e. the terms of sum_j Z_kj Z_lj^T in the Schur complement. */
typedef struct ba_cluster_info {
  int32_t n_cams, n_free, n_pts, n_obs;
  int32_t n_tiles;       /* warp tiles of whole points, at most 32 observations each */
  int32_t n_chunks;      /* CTA chunks of consecutive tiles */
  int32_t n_cam_slots;   /* per-chunk partial sums of free cameras */
  int32_t n_pair_slots;  /* per-chunk partial sums of co-visible free-camera pairs */
  int32_t n_pairs;       /* co-visible free-camera pairs (off-diagonal blocks of S) */
  int32_t reserved;
  int64_t n_free_obs;    /* observations by free cameras */
  int64_t n_pair_entries;
  int64_t arena_bytes;   /* device memory held by the cluster */
  double presort_ms;     /* ba_create_cluster: host validation, presort and staging (wall clock) */
  double upload_ms;      /* ba_create_cluster: device allocation, upload and camera records */
} ba_cluster_info;

/* Fill *out for cluster id (host pointer).  BA_ERR_NOT_FOUND for an unknown
 * id.  Reads host-side records only: no device work. */
BA_API ba_status ba_get_cluster_info(ba_ctx* ctx, ba_cluster_id id, ba_cluster_info* out);

/* Device memory the context holds now, in bytes (clusters, plans, serving
 * slots; the budget of ba_config.hbm_budget_bytes counts the same). */
BA_API ba_status ba_memory_in_use(ba_ctx* ctx, uint64_t* bytes);

/* Kernels this context has launched so far (kernel nodes of graph launches
 * included). */
BA_API ba_status ba_launch_count(ba_ctx* ctx, uint64_t* out);

/* Per-kernel-kind device time (ms) and launch counts accumulated since the
 * context was created or last reset (reset != 0 clears after reading).
 * ms[n] and launches[n] are host arrays, n <= BA_KERNEL_KINDS; times are only
 * collected when the context was created with BA_FLAG_KERNEL_TIMING. */
BA_API ba_status ba_kernel_stats(ba_ctx* ctx, double* ms, uint64_t* launches, int32_t n, int32_t reset);

/* Robust cost F(x) of a cluster given entirely in caller-owned device memory,
 * computed without allocating anything.  The paper has no counterpart: this
 * entry point exists for callers that cannot allocate once running, such as
 * onboard flight software that reserves all its memory at start-up, or a
 * process whose device memory belongs to another allocator.
 *   d       every pointer a device pointer (d->ptr_kind must be
 *           BA_PTR_DEVICE); R, T, X are the state at which F is evaluated;
 *           fixed may be NULL; mu0, warm_* are ignored.  Observations may be
 *           in any order.  Indices are not checked on the host: an
 *           out-of-range index makes *F_out NaN (never a fault).
 *   stream  cudaStream_t to run on (NULL = the legacy default stream); the
 *           call enqueues two kernels and returns without waiting.
 *   F_out   device pointer to one double, written when the kernels finish.
 * Scratch is a 512 KiB file-scope device array that every GPU loading the
 * library holds until exit, so n_obs may be at most 67,108,864; larger
 * problems are rejected with BA_ERR_INVALID.  The array is shared by all
 * calls: calls that overlap on the GPU race, and must be ordered (one
 * stream, or events).  The first call on a device looks up the array's
 * device address; make that first call before any stream capture.  No
 * cudaMalloc, cudaFree or other allocating routine is called. */
BA_API ba_status ba_cost_noalloc(const ba_cluster_desc* d, void* stream, double* F_out);

/* ---- Autotuning of the launch shapes ----
 *
 * Launch and presort parameters of the LM iteration.  None changes what is
 * computed; chunk_tiles and factor_nb change the order of some sums (every
 * configuration is deterministic: alone = in a batch, bit for bit).
 * Values: chunk_tiles 0 (the precision's maximum: 16 mixed, 8 FP64) or
 * 4 .. that maximum; lin_ctas_per_sm and back_ctas_per_sm 1 .. 32;
 * factor_nb 2 .. 32; factor_threads 256, 384 or 512; big_panel_w 1, 2, 4, 8,
 * 16 or 32; batch_chains 1 .. 8.  ms_default / ms_tuned: what ba_autotune measured (device time
 * of one solve of its batch with the defaults and with the chosen values;
 * 0 when not measured). */
typedef struct {
  int32_t chunk_tiles;      /* observations per linearise+Schur CTA, in tiles of up to 32 (whole points) */
  int32_t lin_ctas_per_sm;  /* linearise+Schur grid: CTAs per SM before it strides */
  int32_t back_ctas_per_sm; /* back-substitution grid: CTAs per SM before it strides */
  int32_t factor_nb;        /* panel width of the shared-memory Cholesky (clusters of <= 32 free images) */
  int32_t factor_threads;   /* threads of its CTA */
  int32_t big_panel_w;      /* column-block width of the tensor-core solver's diagonal factorisation */
  int32_t batch_chains;     /* a batch's LM iterations as this many concurrent launch chains over disjoint
                               parts of the batch (clusters dealt by decreasing size); 1: one chain */
  double ms_default;
  double ms_tuned;
} ba_tune;

/* The context's current parameters (defaults, the tuning table's entry,
 * ba_set_tune's or ba_autotune's choice). */
BA_API ba_status ba_get_tune(ba_ctx* ctx, ba_tune* out);

/* Set the parameters (t host, read during the call; ms fields ignored).
 * chunk_tiles applies to clusters created afterwards, the rest to every
 * later launch.  BA_ERR_INVALID for a value out of range, or while a
 * cluster is in service (a batch on the device, or serving). */
BA_API ba_status ba_set_tune(ba_ctx* ctx, const ba_tune* t);

/* Choose the parameters by measurement: the n clusters of descs (host
 * arrays, as for ba_create_cluster) are created in this context, solved
 * iters LM iterations at a time as one batch (ba_solve_batch, from their
 * initial state), and timed with CUDA events on the context's stream, the
 * fastest of three solves per candidate; one parameter at a time, each over
 * a few candidates around the current choice, in the order above (a
 * coordinate descent from the defaults; big_panel_w only when a cluster has
 * more than 32 free images).  The choice is kept in the context and written
 * to *out with both timings; the tuning clusters are destroyed.  Blocking;
 * takes seconds (chunk_tiles candidates re-create the clusters).
 * BA_ERR_INVALID for bad arguments or while a cluster is in service; errors
 * of cluster creation are returned as they come. */
BA_API ba_status ba_autotune(ba_ctx* ctx, const ba_cluster_desc* descs, int32_t n, int32_t iters, ba_tune* out);

/* Host only: the entry of a tuning table (a text file) for a GPU and a
 * precision.  One entry per line, '#' starts a comment:
 *   <gpu name, spaces as '_'> <SM count> <fp64|mixed> chunk_tiles=.. lin_ctas_per_sm=..
 *   back_ctas_per_sm=.. factor_nb=.. factor_threads=.. big_panel_w=.. batch_chains=..
 *   [ms_default=.. ms_tuned=..]
 * Missing keys keep their defaults; the last matching line wins.
 * BA_ERR_NOT_FOUND when the file has no such entry or cannot be read,
 * BA_ERR_INVALID for a malformed matching entry or out-of-range values. */
BA_API ba_status ba_tune_table_lookup(const char* path, const char* gpu_name, int32_t sm_count, int32_t precision,
                                      ba_tune* out);

/* Free a cluster: the end of a sliding cluster's life (Sec. 3.2: once the
 * next cluster has taken over its overlap images, its state is no longer
 * needed).  Its device arena is released stream-ordered (after the work
 * already queued on the context's stream), without waiting; batch plans that
 * hold it are dropped.  BA_ERR_NOT_FOUND for an unknown id,
 * BA_ERR_INVALID for a cluster in service. */
BA_API ba_status ba_destroy_cluster(ba_ctx* ctx, ba_cluster_id id);

/* Stop the serving scheduler once every submitted cluster has finished, wait
 * for the device, free every cluster, plan and buffer of the context and the
 * context itself.  Results not yet polled are dropped.  ctx is invalid
 * afterwards. */
BA_API ba_status ba_shutdown(ba_ctx* ctx);

/* Measure this GPU's binary32 fused multiply-add rate (the denominator of
 * the roofline of the binary32-bound kernels): one launch of ctas_per_sm x
 * SMs CTAs of 512 threads, each thread running 16 independent FMA chains
 * for `iters` steps, timed with CUDA events on the context's stream after
 * one warm-up launch.  *tflops = 2 x 16 x iters x threads / time; *ms = the
 * launch's time.  Blocking.  BA_ERR_INVALID for NULL outputs or sizes < 1. */
BA_API ba_status ba_probe_fp32_fma(ba_ctx* ctx, int32_t ctas_per_sm, int32_t iters, double* tflops, double* ms);

/* Static text of a status code (never NULL). */
BA_API const char* ba_status_string(ba_status s);

/* Human-readable reason of the last error a call on the calling thread
 * returned (thread-local: the API is called from several threads, the
 * scheduler among them); valid until that thread's next failing call. */
BA_API const char* ba_last_error(ba_ctx* ctx);

#ifdef __cplusplus
}
#endif
#endif /* BA_GB300_H */
