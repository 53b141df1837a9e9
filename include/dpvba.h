/*
 * dpvba.h -- C ABI of a single-GPU (B300, sm_103a) Gauss-Newton bundle
 * adjustment over the DPVO patch graph (arxiv 2408.01654).
 *
 * The operation (Sec. 3.1, Eq. 2 and Eq. 3): every edge (i,k,j) reprojects
 * patch k of frame i into frame j,
 *     P'_ikj = Pi[ G_j^-1 G_i Pi^-1(P_ik) ],
 * and one Gauss-Newton iteration minimises
 *     sum_(i,k,j) || P'_ikj - I_ikj ||^2_{diag(w_ikj)}
 * over the free camera poses and the per-patch inverse depths, with the
 * inverse depths Schur-eliminated and the dense pose system Cholesky-solved
 * (Sec. 3.2 "Efficient Global Optimization"; the appendix "Bundle-Adjustment
 * Efficiency" names that pose-block Cholesky as the bottleneck).
 *
 * Conventions used by every call:
 *   - poses  : float64 [N,7] (tx,ty,tz,qx,qy,qz,qw), world->camera (the
 *              inverse of the paper's G_i); perturbed on the left,
 *              T <- Exp(xi) T, xi = (rho, phi), translation first.
 *   - patches: float32 [P,3,3,3], channels (x, y, inverse depth) over a 3x3
 *              pixel patch (Eq. 1 with p = 3).  The residual uses the centre
 *              pixel [k][:][1][1]; the nine pixels share one inverse depth.
 *   - ii, jj, kk : int32 [E]; edge e is patch kk[e] of frame ii[e] observed in
 *              frame jj[e].  All edges of one patch must have the same ii.
 *   - targets: float32 [E,2] pixels (the paper's I_ikj); weights: float32
 *              [E,2] (w_ikj); residual r = target - proj, cost sum w_c r_c^2.
 *   - intrinsics: float32 [4] (fx, fy, cx, cy), host or device memory.
 *   - an edge with i == j, or whose point lies less than z_min (metres) in
 *     front of frame j, contributes nothing.
 *
 * Memory and streams: every pointer argument is DEVICE memory unless stated.
 * The handle owns its workspace; it BORROWS poses, patches, targets and
 * weights, which must stay allocated until the next ba_set_graph or
 * ba_destroy.  All work is ordered on the handle's stream; calls return as
 * soon as the work is queued.
 *
 * Errors: arguments a host can check (null pointers, non-positive sizes,
 * fixed_poses out of range, a call out of order) return an error at once and
 * queue nothing.  Errors the GPU detects (an index out of range, a patch with
 * two source frames, a pose system that is not positive definite, a window
 * wider than the kernels support) are written to a device status word; the
 * kernels that follow skip their work, the poses and depths stay at the last
 * completed iteration, and ba_sync returns the first such error.
 */
#ifndef DPVBA_H
#define DPVBA_H

#if defined(__GNUC__)
#define DPVBA_API __attribute__((visibility("default")))
#else
#define DPVBA_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

typedef struct ba_handle_s* ba_handle_t;

typedef enum {
  BA_OK = 0,
  BA_ERR_INVALID_ARG = 1, /* bad argument, or an invalid edge index found on the GPU */
  BA_ERR_CUDA = 2,        /* a CUDA runtime call failed                             */
  BA_ERR_OOM = 3,         /* workspace allocation failed                            */
  BA_ERR_NOT_SPD = 4,     /* reduced pose system not positive definite              */
  BA_ERR_TIMEOUT = 5,     /* a bounded device-side wait ran out                     */
  BA_ERR_STATE = 6,       /* call out of order (e.g. ba_step before ba_set_graph)   */
  BA_ERR_UNSUPPORTED = 7  /* graph shape beyond the kernels' limits                 */
} ba_status_t;

typedef enum {
  BA_FP32 = 0, /* FP32 linearisation with compensated sums, FP32 factorisation with
                  compensated-FP32 refinement; FP64 retraction                       */
  BA_MIXED = 1 /* the linearisation (reprojection, Jacobians, block products, Schur
                  complement, back-substitution) in double-float arithmetic (pairs
                  of FP32, ~48 bits), the FP32/TF32 factorisation with FP64
                  refinement (one-CTA systems) or preconditioned conjugate
                  gradients on a double-float copy of S (larger systems): the step
                  of an FP64 Gauss-Newton to ~1e-9 on ill-conditioned loop-closure
                  systems                                                           */
} ba_precision_t;

typedef struct {
  int precision;           /* ba_precision_t                                     */
  float lambda_pose;       /* added to every free-pose diagonal (default 1e-4)    */
  float lambda_depth;      /* added to every inverse-depth diagonal (1e-4)        */
  float z_min;             /* minimum depth in frame j, metres (0.1)              */
  float d_min;             /* lower clamp of inverse depth after a step (1e-3)    */
  int patches_per_group;   /* patches per reduction group; 0 = automatic; at most
                              64 (BA_FP32) or 32 (BA_MIXED)                      */
  int max_refine;          /* FP64 refinement sweeps in BA_MIXED (default 3) for
                              systems <= 256 unknowns; larger systems run up to
                              max(8, max_refine) conjugate-gradient iterations
                              preconditioned by the factor; all stop once the
                              estimated error left in the step is < 1e-7 of it
                              (BA_FP32) or < 1e-10 of it (BA_MIXED)             */
  long long timeout_cycles;/* bound on any device-side wait (default 2e9 cycles)  */
  void* stream;            /* cudaStream_t for all work; NULL = legacy stream      */
  int residual_pixels;     /* residual rows per edge: 1 = the patch centre (2-D,
                              default); 9 = every pixel of the 3x3 patch (18-D,
                              Eq. 3 summed over the patch): the targets passed to
                              ba_set_graph* are then float32 [E,9,2] (row-major
                              pixel order), the weights stay [E,2] and are shared
                              by the edge's nine residuals; ba_backward's target
                              cotangents take the targets' layout                  */
  int dense_policy;        /* ba_dense_policy_t: the dense or the block-sparse form
                              of an iteration (default BA_DENSE_AUTO)              */
} ba_options_t;

/* The two forms of a Gauss-Newton iteration (the appendix "Bundle-Adjustment
 * Efficiency" compares DPVO's dense bundle adjustment with the block-sparse
 * one and switches between them on the fly by graph size).  The dense form
 * scatters every edge's products into dense arrays (the pose system, the
 * pose-depth matrix E with one column per patch, C and w) and forms
 * S = B - E Ct^-1 E^T as one dense product; the block-sparse form reduces
 * each (source, target) run and each patch group's window and adds only the
 * window blocks to S.  The dense form applies to one problem bound by
 * ba_set_graph with BA_FP32, residual_pixels = 1, 6 to 256 pose unknowns and
 * no tape being recorded (the adjoint runs on the block-sparse form); in any
 * other case the block-sparse form runs. */
typedef enum {
  BA_DENSE_AUTO = 0,   /* dense where it applies and the graph has at most the
                          measured crossover number of edges; on B300 the
                          block-sparse form measured faster at every size (8
                          to 44 keyframes), so this selects block-sparse       */
  BA_DENSE_ALWAYS = 1, /* dense wherever it applies                             */
  BA_DENSE_NEVER = 2   /* block-sparse always                                   */
} ba_dense_policy_t;

/* Fill *opt with the defaults above. */
DPVBA_API ba_status_t ba_default_options(ba_options_t* opt);

/* Create a handle on the current CUDA device.  opt == NULL means defaults.
 * *out receives the handle.  Allocates only a small fixed workspace. */
DPVBA_API ba_status_t ba_create(ba_handle_t* out, const ba_options_t* opt);

/* Release the handle and its workspace (synchronises its stream first). */
DPVBA_API ba_status_t ba_destroy(ba_handle_t h);

/* Change the stream used by later calls. */
DPVBA_API ba_status_t ba_set_stream(ba_handle_t h, void* stream);

/* Bind a patch graph (Sec. 3.1 "The patch graph").  Validates the indices on
 * the GPU, sorts the edges into reduction groups and builds the group windows,
 * edge->block slot maps and run tables; grows the workspace if needed (the
 * only call that may allocate).  poses and patches are updated in place by
 * ba_step; targets and weights are read on every ba_step, so the caller may
 * refresh their contents between steps without calling ba_set_graph again.
 * ii, jj, kk are read only during this call's queued work.
 * N >= 1, P >= 1, E >= 0.  intrinsics may be host or device memory and is
 * copied. */
DPVBA_API ba_status_t ba_set_graph(ba_handle_t h, int N, int P, int E, double* poses, float* patches,
                         const int* ii, const int* jj, const int* kk, const float* targets,
                         const float* weights, const float* intrinsics);

/* Bind B independent problems to one handle, solved together (batched
 * execution of many uneven bundle adjustments, e.g. one per map segment or
 * per sequence).  The paper solves one problem at a time; this binding runs
 * every kernel once over all problems: one preprocessing pass, one assembly
 * launch, the pose systems in batched solver launches, one back-substitution.
 *   frame_off, patch_off, edge_off : HOST int64 [B+1], non-decreasing from 0;
 *       problem b owns frames [frame_off[b], frame_off[b+1]) of `poses`,
 *       patches [patch_off[b], patch_off[b+1]) of `patches`, and edges
 *       [edge_off[b], edge_off[b+1]) of ii, jj, kk, targets, weights;
 *       every problem has at least one frame and one patch.
 *   poses [N,7] f64, patches [P,3,3,3] f32 : device, concatenated, updated by
 *       ba_step as for ba_set_graph;
 *   ii, jj, kk : device int32 [E], indices LOCAL to the edge's problem;
 *   targets, weights : device f32 [E,2], 8-byte aligned;
 *   intrinsics : host or device f32 [B,4] (fx, fy, cx, cy per problem).
 * ba_step's fixed_poses applies to each problem (its first fixed_poses
 * frames) and must not exceed the smallest frame count.  When a problem's
 * patch count is not a multiple of the reduction group size the library
 * works on a padded copy of `patches`, read at each ba_step and written back
 * at its end.  Errors: BA_ERR_INVALID_ARG for bad offsets or pointers (host
 * checked) and, through ba_sync, for local indices out of range; the
 * debug exports of S and of the block keys are single-problem only
 * (BA_ERR_UNSUPPORTED). */
DPVBA_API ba_status_t ba_set_graph_batched(ba_handle_t h, int B, const long long* frame_off,
                                           const long long* patch_off, const long long* edge_off, double* poses,
                                           float* patches, const int* ii, const int* jj, const int* kk,
                                           const float* targets, const float* weights, const float* intrinsics);

/* Run `iters` Gauss-Newton iterations of Eq. 3 in place (Sec. 3.1-3.2):
 * linearise every edge, reduce into the block system, eliminate the inverse
 * depths, factor and solve the pose system, back-substitute the depths,
 * retract the poses.  Poses [0, fixed_poses) are held constant (gauge).
 * 0 <= fixed_poses <= N, iters >= 0.  fixed_poses = N holds every pose: the
 * iterations then solve for the inverse depths alone (structure-only BA,
 * Sec. 3.3, e.g. to triangulate patches for known cameras). */
DPVBA_API ba_status_t ba_step(ba_handle_t h, int iters, int fixed_poses);

/* ---- batched execution patterns ------------------------------------------
 *
 * on != 0: replay ba_step, and the device work of ba_set_graph /
 * ba_set_graph_batched (validation, sort, grouping), from captured CUDA
 * graphs.  The first call for a configuration (binding pointers, sizes and
 * offsets, workspace allocation, iters, fixed_poses, profiling on/off,
 * stream) runs eagerly and sizes the workspace; the second captures the work
 * on a private stream; later calls launch the graph on the handle's stream
 * (one graph launch per call).  Rebinding the same buffers with the same
 * sizes (new contents) keeps both graphs; the intrinsics are copied outside
 * the graph on every binding.  Steps that record a tape (ba_set_record) run
 * eagerly.  Work the runtime cannot capture keeps running eagerly for its
 * configuration (ba_debug_info reports captures and replays).  With
 * profiling on, each replay's event times are read before the next replay of
 * the same graph, which then waits on the host for the previous one to
 * finish.  on == 0 releases the graphs (synchronises). */
DPVBA_API ba_status_t ba_set_capture(ba_handle_t h, int on);

/* Autotune the patch-group size (patches reduced by one CTA of the assembly
 * kernel) on the bound graph: for each candidate size in {8, 16, 24, 32, 48,
 * 64} rebind the graph (its pointers are BORROWED again for this call: ii,
 * jj, kk must still hold the bound edges), run one warm-up ba_step (two with
 * graph replay), then time `reps` >= 1 calls of ba_step(iters, fixed_poses)
 * with CUDA events on the handle's stream, restoring the caller's poses and
 * patches (device copies) before every step; the median is the candidate's
 * time.  A size the kernels cannot run on this graph (a group touching more
 * than 64 frames) is infeasible (time -1).  The fastest feasible size is
 * bound on return and recorded in a process-wide table under the binding's
 * shape class (device, single or batched, patch and edge counts in
 * half-octaves, precision), which the automatic choice (patches_per_group = 0)
 * consults from then on; a handle created with an explicit size keeps the
 * best one instead.  The poses and patches are left as they were.
 * Outputs (host): *best_group; cand_group[i], cand_ms[i] for the first
 * max_cand candidates (may be null when max_cand = 0); *n_cand (may be null)
 * the number of candidates tried.  Synchronises; allocates temporaries.
 * Errors: BA_ERR_STATE without a graph, BA_ERR_INVALID_ARG for bad
 * arguments, BA_ERR_UNSUPPORTED if no candidate is feasible. */
DPVBA_API ba_status_t ba_autotune(ba_handle_t h, int iters, int fixed_poses, int reps, int max_cand,
                                  int* cand_group, float* cand_ms, int* n_cand, int* best_group);

/* Forget every group size recorded by ba_autotune (the automatic choice goes
 * back to its fixed rule).  Bound handles keep their current size. */
DPVBA_API ba_status_t ba_autotune_clear(void);

/* Wait for the handle's stream; return the first device-detected error. */
DPVBA_API ba_status_t ba_sync(ba_handle_t h);

/* Text of the last error on this handle (never NULL). */
DPVBA_API const char* ba_last_error(ba_handle_t h);

/* Name of a status code (never NULL). */
DPVBA_API const char* ba_status_string(ba_status_t s);

/* ---- inspection (tests and profiling; not needed to run a step) --------- */

/* Build the reduced pose system at the current state without solving:
 * afterwards BA_EXPORT_S / _Y / _CT / _W hold S, y, C+lambda_depth and w. */
DPVBA_API ba_status_t ba_linearize(ba_handle_t h, int fixed_poses);

enum {
  BA_EXPORT_S = 0,      /* float64 [n,n] dense, lower triangle (upper zero), n = 6 (N - fixed) */
  BA_EXPORT_Y = 1,      /* float64 [n]        reduced right-hand side                         */
  BA_EXPORT_DX = 2,     /* float64 [n]        last pose step                                  */
  BA_EXPORT_DD = 3,     /* float32 [P]        last inverse-depth step                         */
  BA_EXPORT_CT = 4,     /* float32 [P]        C + lambda_depth                                */
  BA_EXPORT_W = 5,      /* float32 [P]        depth gradient w                                */
  BA_EXPORT_PERM = 6,   /* int32 [E]          sorted position -> input edge                   */
  BA_EXPORT_SLOTS = 7,  /* uint32 [E]         slot_i | slot_j << 8 | patch-in-group << 16     */
  BA_EXPORT_GPTR = 8,   /* int32 [groups+1]   edge range of each group                        */
  BA_EXPORT_WIN = 9,    /* int32 [groups, 64] window frames of each group (-1 padded)          */
  BA_EXPORT_COST = 10,  /* float64 [iters]    cost sum w r^2 at each iteration's linearisation point */
  BA_EXPORT_PMPOS = 11, /* int32 [E]          sorted position -> patch-major position          */
  BA_EXPORT_PPTR = 12   /* int32 [P+1]        patch-major edge range of each patch             */
};

/* Copy an internal array into `dst` (device memory, `bytes` long; fails if
 * too small).  Synchronises the stream. */
DPVBA_API ba_status_t ba_debug_export(ba_handle_t h, int what, void* dst, long long bytes);

/* Host integers describing the bound graph:
 * info[0..14] = N, P, E, patches_per_group, groups, n (last fixed), tile size, runs,
 * kernels launched by the handle so far; then for the CUDA graphs of
 * ba_set_capture: ba_step captures, replays, kernels in one replay, and the
 * same three for the binding's device work (ba_set_graph*); info[15] = 1 if
 * the last ba_step ran the dense form (ba_dense_policy_t), else 0. */
DPVBA_API ba_status_t ba_debug_info(ba_handle_t h, long long* info, int cap);

/* The row envelope of every pose system above 256 unknowns, as the last
 * factorisation found it (the block-sparse structure of the reduced system,
 * Sec. 3.2): out (host) receives the number of such systems B, then per
 * system its tile count T (64-row tiles) followed by T integers env[a] = the
 * first tile column holding a nonzero in tile row a of S (env[a] <= a; the
 * factor L is zero left of it, and the factorisation and the solves visit
 * only the tiles of the envelope).  cap: integers available at out;
 * *count (host) receives the integers needed; a smaller cap writes nothing
 * (BA_ERR_INVALID_ARG).  BA_ERR_STATE before the bound systems were first
 * factored.  Synchronises the handle's stream. */
DPVBA_API ba_status_t ba_debug_envelope(ba_handle_t h, int* out, long long cap, long long* count);

/* Canonical pose-pose block keys of the B part of the system, computed on the
 * GPU: sorted unique (a,b), a <= b, over (i,i), (j,j), (min,max) of each
 * non-self edge with both poses free.  keys_out: device int32 [cap,2];
 * *n_out (host) receives the count.  Synchronises; allocates temporaries. */
DPVBA_API ba_status_t ba_debug_keys(ba_handle_t h, int fixed_poses, int* keys_out, int cap, int* n_out);

/* ---- timing (CUDA events recorded on the handle's stream) --------------- */

enum {
  BA_KERNEL_PREPROCESS = 0, /* every kernel of ba_set_graph                     */
  BA_KERNEL_INIT = 1,       /* clearing the pose system                          */
  BA_KERNEL_ASSEMBLE = 2,   /* linearisation + block reduction + Schur complement */
  BA_KERNEL_SOLVE = 3,      /* pose-system solves except the large factorisation */
  BA_KERNEL_BACKSUB = 4,    /* inverse-depth back-substitution                   */
  BA_KERNEL_RETRACT = 5,    /* SE(3) retraction                                  */
  BA_KERNEL_ADJOINT = 6,    /* adjoint-only kernels of ba_backward               */
  BA_KERNEL_FACTOR = 7,     /* the persistent factorisation of systems > 256 unknowns */
  BA_KERNEL_PROXIMITY = 8,  /* ba_proximity_edges                                */
  BA_KERNEL_CORRELATION = 9,/* ba_patch_correlation                              */
  BA_KERNEL_PGO = 10,       /* ba_pgo_lm, its pose-system solves included        */
  BA_KERNEL_CLASSES = 11
};

/* on != 0: from now on record a CUDA event pair around every launch of each
 * kernel class above (and clear earlier records); on == 0: stop recording. */
DPVBA_API ba_status_t ba_profile_enable(ba_handle_t h, int on);

/* As ba_profile_enable, for the kernel classes whose bits are set in `mask`
 * (bit k = the class BA_KERNEL_* numbered k above; 0 stops recording).
 * Launches of the other classes run without event records, so a captured
 * step keeps their programmatic (early-launch) dependencies; a changed mask
 * re-captures the step's graph on the next call.  BA_ERR_INVALID_ARG for a
 * bit at or above BA_KERNEL_CLASSES. */
DPVBA_API ba_status_t ba_profile_classes(ba_handle_t h, unsigned mask);

/* Synchronise, then report for kernel class `kind` the summed event time of
 * its recorded launches (*total_ms) and their number (*launches). */
DPVBA_API ba_status_t ba_profile_read(ba_handle_t h, int kind, double* total_ms, long long* launches);

/* ---- adjoint (reverse mode through the iterations) ----------------------
 *
 * The bundle adjustment is a differentiable layer (Sec. 3.1: the update
 * operator's targets and confidence weights are trained through the unrolled
 * Gauss-Newton iterations of Eq. 3).  ba_backward gives the derivative of a
 * scalar loss L(poses_final, depths_final) with respect to the targets and
 * weights of the last recorded ba_step call, by reverse mode through each
 * iteration: the retraction, the damped normal equations H Delta = g (solved
 * with the same Schur/Cholesky path as the forward step, H being symmetric)
 * and the per-edge linearisation (Eq. 2).  The depth clamp at d_min passes
 * the cotangent only where it did not clamp; masked edges (i = j, or the point
 * less than z_min in front of frame j) contribute nothing; fixed poses have no
 * cotangent. */

/* on != 0: every following ba_step call records its iterations (copies of
 * the state before each iteration and of each step, ~(56 N + 120 P + 8 n)
 * bytes per iteration, owned by the handle) and becomes the tape of
 * ba_backward, replacing the previous tape.  on == 0: stop recording (the
 * last tape stays usable).  ba_set_graph discards the tape. */
DPVBA_API ba_status_t ba_set_record(ba_handle_t h, int on);

/* Reverse-mode pass over the tape, stream-ordered on the handle's stream.
 * Inputs (device, may be null = zero):
 *   grad_poses  : float64 [N,7], dL/d(t, q) of the final poses (the layout of
 *                 `poses`; only the component tangent to the unit quaternion
 *                 matters, and rows of fixed poses are ignored);
 *   grad_depths : float32 [P], dL/d(inverse depth) of the final patches.
 * Outputs (device, may be null = not wanted):
 *   grad_targets, grad_weights : float32 [E,2] in input edge order,
 *                 8-byte aligned, overwritten (grad_targets [E,9,2] when
 *                 the handle's residual_pixels is 9);
 *   grad_tangent0 : float64 [N,6], dL/dxi of the initial poses under the left
 *                 perturbation T <- Exp(xi) T, xi = (rho, phi) (0 for fixed);
 *   grad_depths0  : float32 [P], dL/d(initial inverse depth).
 * The bound targets/weights buffers must hold the values the tape was
 * recorded with; the poses/patches buffers are not read.  A handle bound by
 * ba_set_graph_batched is differentiated over all its problems at once (the
 * arrays above are the concatenated ones).  Errors: BA_ERR_STATE without a
 * tape, BA_ERR_INVALID_ARG for misaligned outputs, BA_ERR_UNSUPPORTED for a
 * batched binding that works on a padded patch copy (a problem's patch count
 * not a multiple of the group size), BA_ERR_OOM; device-detected errors
 * (BA_ERR_NOT_SPD) come from ba_sync. */
DPVBA_API ba_status_t ba_backward(ba_handle_t h, const double* grad_poses, const float* grad_depths,
                                  float* grad_targets, float* grad_weights, double* grad_tangent0,
                                  float* grad_depths0);

/* ---- proximity loop edges ----------------------------------------------- */

/* Loop-closure edges from camera proximity (Sec. 3.2 "Proximity Loop Closure"
 * and "Constructing the Patch Graph"): a loop is detected when the camera
 * comes close to where an older frame was, and it is closed with
 * uni-directional edges from that old frame's stored patches to the recent
 * frame (so only recent frames need dense features).  For every query frame
 * b in [b0, b1):
 *   - the candidates are the frames a with b - a > gap;
 *   - the selected frame is the candidate whose camera centre c = -R^T t is
 *     nearest to frame b's (lowest index among equal distances), if the
 *     squared distance is < radius^2 (FP64);
 *   - its patches m = 0..M-1 (patch index k = a*M + m) become edges
 *     (ii, jj, kk) = (a, b, k) if the centre pixel reprojects by Eq. 2, at
 *     the patch's current inverse depth, more than the handle's z_min in
 *     front of frame b and inside [0, width) x [0, height) (FP64).
 * Edges are written in the order (b, m), at most `cap` of them.
 *   poses      : device float64 [N,7] world->camera (as for ba_set_graph).
 *   patches    : device float32 [N*M,3,3,3]; patch a*M + m belongs to frame a.
 *   intrinsics : HOST float32 [4] (fx, fy, cx, cy), read during the call.
 *   ii, jj, kk : device int32 [cap] (may be null when cap == 0); pointing them
 *                past the local edges of a graph appends the loop edges.
 *   coords     : device float32 [cap,2], 8-byte aligned, or null: the
 *                reprojected centre pixel of each edge (FP64 rounded).
 *   match      : device int32 [b1-b0] or null: selected frame of each query,
 *                -1 if none.
 *   count      : device int32 [1]: the number of edges found (may exceed cap;
 *                only the first cap are written).
 *   n_host     : host or null.  Non-null: the call waits for its work and
 *                stores the count; returns BA_ERR_INVALID_ARG if it exceeds
 *                cap (the first cap edges are still written).  Null: the
 *                call only queues work and may be captured into a CUDA graph
 *                once a first call of the same or larger size has sized the
 *                handle's scratch.
 * Limits: 1 <= M <= 1024, N*M < 2^31, 0 <= b0 <= b1 <= N, gap >= 0,
 * 0 <= radius < inf, width, height > 0; anything else returns
 * BA_ERR_INVALID_ARG at once and queues nothing.  cap >= (b1-b0)*M always
 * suffices.  Uses the handle's stream and scratch; needs no bound graph. */
DPVBA_API ba_status_t ba_proximity_edges(ba_handle_t h, int N, int M, const double* poses, const float* patches,
                                         const float* intrinsics, int b0, int b1, int gap, double radius,
                                         double width, double height, int* ii, int* jj, int* kk, float* coords,
                                         long long cap, int* match, int* count, long long* n_host);

/* ---- patch correlation --------------------------------------------------- */

/* The correlation volume of Eq. 4 (Sec. 3.1 "Patch correlation"): for every
 * edge e and pixel (v, u) of its p x p patch,
 *   out[e][v][u][a][b] = < gmap[kk[e]][v][u][:],
 *                          f_jj[e](coords[e][v][u] + (b - R, a - R)) >,
 * a, b in 0..2R, where f_j(x, y) samples fmap[j] bilinearly from the four
 * pixels around (x, y) (x0 = floor x, weight x - x0; likewise y; integer
 * coordinates are pixel centres; pixels outside the map count as zero).
 *   fmap   : device float32 [Nf, H, W, D], channels last (the dense
 *            correlation feature maps of the target frames).
 *   gmap   : device float32 [P, p, p, D] (each patch's correlation features).
 *   kk, jj : device int32 [E] (source patch, target frame of each edge).
 *   coords : device float32 [E, p, p, 2], (x, y) in feature-map pixels (the
 *            reprojected patch pixels P', Eq. 2, at the maps' resolution).
 *   out    : device float32 [E, p, p, 2R+1, 2R+1] (row offset a, column b).
 * Limits: 1 <= p <= 3, 0 <= R <= 4, D a multiple of 32, E >= 0, fmap and
 * gmap 16-byte aligned (BA_ERR_INVALID_ARG otherwise); a (2R+2)^2 block of
 * D-channel map pixels must fit the ~72 KB staging buffer (D <= 224 for
 * R = 3), and Nf <= 51,199, else BA_ERR_UNSUPPORTED.  An edge with kk or jj
 * out of range gets zeros and sets the handle's device status (ba_sync
 * returns BA_ERR_INVALID_ARG; like any device-detected error it makes the
 * next ba_step skip its work).  FP32 arithmetic; queued on the handle's
 * stream; needs no bound graph.  The handle keeps a scratch of
 * 4 (2 Nf + E + 2) bytes for ordering the edges by target frame, grown by a
 * call that needs more (not while its stream is being captured). */
DPVBA_API ba_status_t ba_patch_correlation(ba_handle_t h, int Nf, int H, int W, int D, int P, int p, int E,
                                           const float* fmap, const float* gmap, const int* kk, const int* jj,
                                           const float* coords, int radius, float* out);

/* ---- Sim(3) pose-graph optimisation -------------------------------------- */

#define BA_PGO_MAX_FRAMES 4096

/* Levenberg-Marquardt on the Sim(3) pose graph of Sec. 3.3 "Optimization"
 * (Eqs. 5-7): minimise sum_f |r_f|^2 over the similarities S_1..S_{N-1}
 * (S_0 held, fixing the gauge), with
 *   r_f = log(dS_f^-1 S_a^-1 S_b)   for a smoothness factor (loop[f] = 0, Eq. 5),
 *   r_f = log(dS_f    S_a^-1 S_b)   for a loop factor       (loop[f] = 1, Eq. 6),
 * a = fa[f], b = fb[f].  A similarity is 8 doubles (tx, ty, tz, qx, qy, qz, qw,
 * s) mapping x to s R(q) x + t; log/Exp use the tangent (rho, phi, sigma) with
 * t = W rho, W = int_0^1 exp(tau([phi]x + sigma I)) dtau.  Each iteration
 * linearises every factor by central differences of step fd_step in the
 * coordinates of S <- S Exp(d) of both endpoints, solves
 * (H + lambda diag(H)) d = -J^T r with the library's dense pose solver (the
 * handle's precision option applies), and keeps S Exp(d) if it lowers the
 * cost (lambda /= 10) or rejects it (lambda *= 10).
 *   S        : device float64 [N,8], updated in place (S[0] never changes).
 *   dS       : device float64 [F,8] measurements.
 *   fa, fb   : device int32 [F] endpoints, 0 <= fa, fb < N, fa != fb.
 *   loop     : device int32 [F], 0 (Eq. 5) or 1 (Eq. 6).
 *   cost     : device float64 [iters+1]: the cost before each iteration and
 *              after the last.
 *   accepted : device int32 [iters] or null: 1 where the step was kept.
 * Limits: 1 <= N <= BA_PGO_MAX_FRAMES, F >= 0, iters >= 0, lambda0 > 0,
 * 0 < fd_step < 1e-2, else BA_ERR_INVALID_ARG at once.  A factor with an
 * endpoint out of range, or fa == fb, sets the device status (ba_sync returns
 * BA_ERR_INVALID_ARG); a damped system that is not positive definite (a
 * similarity no factor touches) makes ba_sync return BA_ERR_NOT_SPD.  The
 * work is queued on the handle's stream with no host round trip inside the
 * iterations (the call itself uploads the system layout from the host, so it
 * is not captured into a CUDA graph); it borrows the handle's pose-system
 * buffers (the next ba_step lays its own system out again) and keeps
 * 8 (3 + 8N + F) bytes of scratch.  Needs no bound graph. */
DPVBA_API ba_status_t ba_pgo_lm(ba_handle_t h, int N, int F, double* S, const double* dS, const int* fa,
                                const int* fb, const int* loop, int iters, double lambda0, double fd_step,
                                double* cost, int* accepted);

/* ---- allocation-free pose-system solve ---------------------------------- */

/* The paper has no counterpart to this call; it exists for callers that cannot
 * allocate device memory when they need a solve -- a tracking loop with a
 * fixed per-frame time budget (cudaMalloc may synchronise the device), or a
 * host framework that owns all device allocations.  It solves S x = y for a
 * reduced pose system with the same one-CTA LDL^T solver as ba_step, without
 * a handle and without allocating.
 *   n      : 1 <= n <= 256; larger n returns BA_ERR_UNSUPPORTED at once.
 *   S      : device float64 [n,n] row-major; only the lower triangle is read.
 *   y      : device float64 [n].   x : device float64 [n] (output).
 *   refine : FP64 refinement sweeps, 0..16 (2 matches BA_MIXED).
 *   stream : cudaStream_t (NULL = legacy stream).
 * The call waits for its work and returns BA_ERR_NOT_SPD if S is not positive
 * definite.  Its working copy lives in a fixed ~0.5 MB device array inside the
 * library, held by every GPU that loads the library until the process exits.
 * Every call looks up that array's device address on the current device (a
 * lookup in the loaded module, no allocation), so the address stays right
 * after cudaDeviceReset.  All calls share the array, so calls whose GPU work
 * overlaps race. */
DPVBA_API ba_status_t ba_solve_pose_system_noalloc(int n, const double* S, const double* y, double* x, int refine,
                                                   void* stream);

#ifdef __cplusplus
}
#endif

#endif /* DPVBA_H */
