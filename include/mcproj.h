/*
 * mcproj -- batched manifold projection and collision checking on GB300.
 *
 * C ABI of libmcproj.so.  Plain pointers and sizes only.  Every batch buffer
 * is caller-owned DEVICE memory unless a function says otherwise; every call
 * is asynchronous on the given CUDA stream (0 = legacy default stream) unless
 * it says otherwise.
 *
 * The operations follow the paper "Vectorizing Projection in Manifold-
 * Constrained Motion Planning for Real-Time Whole-Body Control":
 *   - a configuration q in R^d satisfies the constraints when F(q) = 0, up to
 *     a tolerance ||F(q)|| < eps (Sec. II);
 *   - constraints are end-effector TSRs (Eq. 1), relative poses of two frames
 *     (Eq. 2), and the humanoid's stability constraint on the centre of mass
 *     (Sec. V-C), stacked into one F (Sec. IV-C);
 *   - projection is the loop ParallelProject / getDescentStep of Algorithm 2:
 *     d = F(q); stop when ||d|| < eps; otherwise
 *     q <- q - alpha J^T (J J^T + lambda I)^{-1} d, solved with a Cholesky
 *     factorisation (Sec. IV-A, "Vectorized Levenberg-Marquardt"), with a
 *     divergence exit when ||step|| > MaxDistance;
 *   - CollisionFree(q) checks the robot's link spheres against the obstacles
 *     (Sec. I, Algorithm 2).
 *
 * Batches are structure-of-arrays: element (joint j, configuration i) of a
 * batch with leading dimension ld lives at base[j * ld + i]; ld >= n.
 *
 * Return values: MCP_OK on success.  Argument errors return MCP_ERR_ARG
 * before anything is enqueued; CUDA runtime failures return MCP_ERR_CUDA.  In
 * both cases mcp_last_error() describes the failure.  No function aborts the
 * process, and no kernel traps: per-configuration failures are reported in
 * the flags array.
 *
 * Thread safety: one context is used by one host thread at a time.
 */
#ifndef MCPROJ_H_
#define MCPROJ_H_

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct mcp_ctx mcp_ctx;
typedef struct CUstream_st *mcp_stream; /* a cudaStream_t */

typedef enum {
  MCP_OK = 0,
  MCP_ERR_ARG = 1,         /* bad pointer, size, layout or descriptor */
  MCP_ERR_STATE = 2,       /* robot / constraints / obstacles not loaded */
  MCP_ERR_CUDA = 3,        /* a CUDA runtime call failed */
  MCP_ERR_OOM = 4,         /* device allocation failed */
  MCP_ERR_UNSUPPORTED = 5  /* robot / constraint combination outside the compiled set */
} mcp_status;

/* Limits of the compiled kernels. */
#define MCP_MAX_JOINTS 40
#define MCP_MAX_FRAMES 8
#define MCP_MAX_CONSTRAINTS 8
#define MCP_MAX_EQUATIONS 24
#define MCP_MAX_SPHERES 256
#define MCP_MAX_OBSTACLES 1024
#define MCP_MAX_AABBS 64

/* Per-configuration flag bits written by the projection calls. */
#define MCP_F_CONVERGED 1      /* ||F(q*)|| < tol, verified in FP64 */
#define MCP_F_CAP 2            /* iteration cap reached without convergence */
#define MCP_F_DIVERGED 4       /* ||step|| > max_step (Alg. 2 MaxDistance exit) */
#define MCP_F_NONFINITE 8      /* NaN/Inf or a singular system with lambda = 0 */
#define MCP_F_FP64_RESOLVE 16  /* at least one step was re-solved in FP64 */
#define MCP_F_ACCEPT_FAIL 32   /* FP32 residual passed but the FP64 check did not, at the cap */
#define MCP_F_OUT_OF_LIMITS 64 /* q* outside the joint limits (reported, never clamped) */

/* Constraint kinds.  k = number of equations. */
typedef enum {
  MCP_C_SPHERE = 0,     /* F = ||q|| - target[0] (configuration space), k = 1 */
  MCP_C_AXIS_ALIGN = 1, /* z-axis of frame_a parallel to world z: F = (z.x, z.y), k = 2
                           (Sec. II: "held upright" TSR; antiparallel also satisfies it) */
  MCP_C_POSE = 2,       /* Eq. 1 with B^w = 0: T_err = P^-1 T_a Q^-1, F = [t_err; log(R_err)],
                           P = T_w^0, Q = T_e^w, k = 6 */
  MCP_C_REL_POSE = 3,   /* Eq. 2: T_err = P^-1 (T_a^-1 T_b), F = [t_err; log(R_err)],
                           P = T_ref, a = left, b = right, k = 6 */
  MCP_C_COM_XY = 4,     /* Sec. V-C stability: F = x_com^xy - target[0:2], k = 2 */
  MCP_C_PLANE = 5,      /* Sec. III task constraint: origin x of frame_a on the xy-plane of the
                           task frame P: F = z of P^-1 x, k = 1 */
  MCP_C_LINE = 6,       /* Sec. III task constraint: x on the z-axis of P: F = (x, y) of P^-1 x, k = 2 */
  MCP_C_DIST = 7,       /* Sec. V-C closed linkage: F = |x_b - x_a| - target[0] for the origins of
                           frame_a and frame_b, k = 1 */
  MCP_C_POSE_BOUNDED = 8, /* Eq. 1 with bounds B^w (Sec. II TSR): e = [t_err; log(R_err)] as for POSE,
                           F_i = e_i - clamp(e_i, B[i], B[6 + i]) (zero inside the bounds), k = 6 */
  MCP_C_COM_HULL = 9    /* Sec. V-C stability as the distance to the support polygon: F = c - P(c)
                           with c the CoM xy and P(c) the polygon's nearest point (zero inside); the
                           polygon's target[0] = 3..6 vertices are B[0..], counter-clockwise, k = 2 */
} mcp_ckind;

/* Robot: a tree of 1-DoF joints in topological order (parent[j] < j, -1 = world).
 * T_j = T_parent(j) * X_j * Jnt(q_j); Jnt = Rz(q) (type 0, revolute) or a
 * translation q along z (type 1, prismatic).  3x4 transforms are 12 doubles,
 * row-major, column 3 = translation.  All arrays are HOST memory, copied by
 * mcp_load_robot; the caller keeps ownership. */
typedef struct {
  int32_t n_joints;
  const int32_t *parent;      /* [n_joints] */
  const int32_t *type;        /* [n_joints] */
  const double *X;            /* [n_joints * 12] */
  const double *lower;        /* [n_joints] joint limits (flag only) */
  const double *upper;        /* [n_joints] */
  const double *mass;         /* [n_joints] link masses (may be NULL if no CoM constraint) */
  const double *com;          /* [n_joints * 3] link CoM in its joint frame (may be NULL) */
  int32_t n_spheres;
  const int32_t *sphere_link; /* [n_spheres] joint the sphere rides on, -1 = world */
  const double *sphere;       /* [n_spheres * 4] centre xyz in that frame, radius */
  int32_t n_frames;
  const int32_t *frame_link;  /* [n_frames] */
  const double *frame_X;      /* [n_frames * 12] frame offset in its joint frame */
} mcp_robot_desc;

/* One constraint.  If q_ref != NULL (HOST, n_joints doubles) the reference is
 * taken from the robot at q_ref when loaded, in FP64 on the device:
 *   POSE, POSE_BOUNDED: P := T_a(q_ref) Q^-1          (T_err(q_ref) = I)
 *   REL_POSE: P := T_a(q_ref)^-1 T_b(q_ref)
 *   PLANE, LINE: the translation of P := origin of frame a at q_ref (P keeps
 *             its rotation: the plane / line passes through frame a)
 *   DIST:     target[0] := |x_b(q_ref) - x_a(q_ref)|
 *   COM_XY:   target := xy midpoint of frames a and b at q_ref (the centre of
 *             the support polygon of two feet).
 *   COM_HULL: the polygon := the xy box around frames a and b at q_ref grown
 *             by the margin target[1] (4 vertices).
 * B: POSE_BOUNDED: lower[6] then upper[6] of [t; log R] (+-inf allowed;
 * lower <= upper required); COM_HULL: the polygon's vertices; ignored by the
 * other kinds. */
typedef struct {
  int32_t kind;
  int32_t frame_a, frame_b;
  double P[12];
  double Q[12];
  double target[3];
  const double *q_ref;
  double B[12];
} mcp_constraint_desc;

typedef struct {
  double tol;          /* eps of Alg. 2, on the Euclidean norm of the stacked F */
  int32_t max_iters;   /* step cap (Alg. 2 has none; at most max_iters steps) */
  int32_t precision;   /* 0: FP32 steps with FP64 acceptance; 1: plain FP64 throughout */
  double lambda;       /* LM damping */
  double max_step;     /* Alg. 2 MaxDistance; <= 0 disables the exit */
  double pivot_fp64;   /* FP32 Cholesky pivot below this -> the step is re-solved in FP64 */
  int32_t cyclic;      /* 0: stacked F, one LM step per iteration; 1: cyclic getDescentStep
                          (Sec. IV-C): per iteration one LM step per constraint in stack order,
                          each at the configuration the previous one produced; the stopping test
                          and MaxDistance apply to the stacked F and to the whole sweep */
  int32_t outer;       /* 0: inner form dq = J^T (J J^T + lambda I)^-1 F (a k x k system);
                          1: outer form dq = (J^T J + lambda I)^-1 J^T F (d x d; Alg. 2 offers both;
                          for k >= d, e.g. consistent redundant constraints, where J J^T is
                          singular).  Stacked steps of problems with at most 14 joints, batch calls
                          (project_batch, project_check_batch); else MCP_ERR_UNSUPPORTED */
  double alpha;        /* step scale of Alg. 2: q <- q - alpha dq; 0 means 1; else in (0, 2] */
} mcp_project_params;

/* Context on CUDA device `device`. */
mcp_status mcp_create(int device, mcp_ctx **out);
/* Frees the context and its device memory (NULL-safe).  Synchronises the device. */
void mcp_destroy(mcp_ctx *ctx);
/* Message of the last failure on this context ("" if none); owned by the context. */
const char *mcp_last_error(const mcp_ctx *ctx);

/* Loads (replaces) the robot model (Sec. II: configuration space C in R^d and
 * the kinematics T_s^0 = FK(q) of Eq. 1).  Synchronous. */
mcp_status mcp_load_robot(mcp_ctx *ctx, const mcp_robot_desc *robot);
/* Loads (replaces) the stacked constraint list (Sec. IV-C), in order.  The
 * robot must be loaded first.  Synchronous (references are resolved on the device). */
mcp_status mcp_load_constraints(mcp_ctx *ctx, const mcp_constraint_desc *cons, int32_t n);
/* Loads (replaces) obstacle spheres [n * 4] (centre, radius) and axis-aligned
 * boxes [m * 6] (min xyz, max xyz); HOST memory, copied.  Synchronous.
 * MCP_ERR_ARG (the previous obstacles stay loaded) if a value is not finite.
 * The library keeps the spheres in its own (spatial) order; verdicts do not
 * depend on it. */
mcp_status mcp_load_obstacles(mcp_ctx *ctx, const double *spheres, int32_t n_spheres, const double *aabbs,
                              int32_t n_aabbs);
/* Returns the resolved constraint i (after q_ref handling): P, Q (12 each),
 * target (3) and B (12), into HOST buffers (each may be NULL). */
mcp_status mcp_get_constraint(const mcp_ctx *ctx, int32_t i, double *P, double *Q, double *target, double *B);

/* ParallelProject (Alg. 2) of n configurations.
 * q_in / q_out: [d * ld] float (precision 0) or double (precision 1); q_out may alias q_in.
 * flags [n] uint8 (MCP_F_*), iters [n] uint8 (steps applied), resid [n] double:
 * the FP64 Euclidean norm of F at the returned configuration.
 * On a divergence exit q_out holds the last iterate before the rejected step.
 * Precision 0: FP32 steps; a configuration is CONVERGED only when its FP64
 * residual is below tol.  If the FP32 residual passed and the FP64 one did
 * not, the configuration takes further FP32 steps while steps remain (then
 * CAP | ACCEPT_FAIL); a Cholesky pivot below pivot_fp64 hands the remaining
 * steps to FP64 (FP64_RESOLVE).  The humanoid classes' FP32 kernel takes at
 * most 2^31 - 1 configurations per call (MCP_ERR_CUDA, invalid argument,
 * beyond: its parked indices are 32-bit). */
mcp_status mcp_project_batch(mcp_ctx *ctx, const mcp_project_params *p, int64_t n, int64_t ld, const void *q_in,
                             void *q_out, uint8_t *flags, uint8_t *iters, double *resid, mcp_stream stream);

/* Projection followed by the collision check of every returned configuration
 * (Alg. 2: ParallelProject, then CollisionFree of each projected point), with
 * the results of mcp_project_batch and then mcp_check_batch(q_out, precision
 * p->precision).  For FP32 problems of the thread-per-configuration kernels the
 * two can run in one persistent launch (the check of each accepted output
 * follows its FP64 acceptance in the same warp, so the ALU-bound check
 * overlaps the FP64 acceptance of other warps); mcp_autotune or
 * mcp_set_tuning decides, the default is a second launch.  Requires loaded
 * obstacles.  in_collision [n] uint8 (DEVICE);
 * pairs_tested [n] uint32 (DEVICE) or NULL: sphere-obstacle tests performed
 * per configuration.  Errors as mcp_project_batch, plus MCP_ERR_STATE without
 * obstacles. */
mcp_status mcp_project_check_batch(mcp_ctx *ctx, const mcp_project_params *p, int64_t n, int64_t ld,
                                   const void *q_in, void *q_out, uint8_t *flags, uint8_t *iters, double *resid,
                                   uint8_t *in_collision, uint32_t *pairs_tested, mcp_stream stream);

/* ParallelConstrainedExtend (Algorithm 2), one call for n_ext extensions.
 * Extension x starts at q_s[:, x] (on the manifold, collision-free by the
 * caller's construction) towards q_t[:, x]: dist = min(|q_t - q_s|, r),
 * v = (q_t - q_s) / |q_t - q_s|, q_steer = q_s + dist v; the n particles
 * q_steer + eps[i, x] v (eps: the N(0, sigma^2) offsets of Alg. 2, drawn by
 * the caller) are projected and the one that converged after the fewest steps
 * (lowest index on ties) is q_proj, unless a particle's step exceeded
 * MaxDistance (p->max_step) earlier.  q_proj must be collision-free and within
 * 2 dist of q_s; n points interpolated between q_s and q_proj are projected,
 * no two consecutive points of q_s, x_1 .. x_n, q_proj may be more than r / n
 * apart and none may collide; then every gap above delta is bisected (the
 * midpoint projected, its two gaps no longer than the gap, collision-free),
 * level by level, until all gaps are at most delta (at most max_depth levels
 * and 128 points).  Each particle and point is projected on its own (FP32
 * steps, FP64 acceptance, p->tol / max_iters / lambda / pivot_fp64).
 * DEVICE buffers: q_s, q_t, q_proj float [d * ld]; eps float [n * ld_eps];
 * status [n_ext] uint8 (MCP_EXT_*); n_points [n_ext] int32: points projected
 * and validated (q_proj, interpolated, midpoints) before the outcome;
 * winner [n_ext] int32: the particle index (-1 if none); steps [n_ext]
 * int32 or NULL: Newton steps taken by all projections of the extension
 * (work accounting).  Requires
 * obstacles; precision 0 and the stacked step only; MCP_ERR_UNSUPPORTED for
 * problem classes without the extension kernel (the humanoid).  The first
 * call (and a call that needs more resident groups) allocates the context's
 * device scratch for the chains (2 x 128 points per resident group), which
 * synchronises the device; later calls allocate nothing. */
#define MCP_EXT_OK 0
#define MCP_EXT_DEGENERATE 1         /* q_t == q_s */
#define MCP_EXT_NO_PROJECTION 2      /* no particle converged before one diverged (or at the cap) */
#define MCP_EXT_PROJ_COLLISION 3     /* q_proj in collision */
#define MCP_EXT_TOO_FAR 4            /* |q_proj - q_s| > 2 dist */
#define MCP_EXT_INTERP_FAIL 5        /* an interpolated point or midpoint did not converge */
#define MCP_EXT_GAP 6                /* consecutive projected points too far apart */
#define MCP_EXT_INTERP_COLLISION 7   /* an interpolated point or midpoint in collision */
#define MCP_EXT_RESOLUTION 8         /* delta not reached within max_depth levels / 128 points */
typedef struct {
  double r;           /* extension range */
  double delta;       /* resolution of the validated chain */
  int32_t n;          /* particles = interpolated points, 1..32 */
  int32_t max_depth;  /* bisection levels, 0..16 */
} mcp_extend_params;
mcp_status mcp_extend_batch(mcp_ctx *ctx, const mcp_project_params *p, const mcp_extend_params *e, int64_t n_ext,
                            int64_t ld, const float *q_s, const float *q_t, const float *eps, int64_t ld_eps,
                            float *q_proj, uint8_t *status, int32_t *n_points, int32_t *winner, int32_t *steps,
                            mcp_stream stream);

/* Projection of uneven interpolation segments in one persistent launch
 * (Alg. 2: n points interpolated between q_s and q_proj are projected in
 * parallel).  Point t of segment s is start[:, s] + t * delta[:, s],
 * t = 0 .. len[s]-1; its outputs go to index off[s] + t, off = exclusive
 * prefix sum of len.  start / delta: float [d * ld_seg] (precision 0) or
 * double (precision 1); len: int32 [n_seg] (each >= 0); q_out: [d * ld_out]
 * with ld_out >= sum(len); flags / iters / resid as in mcp_project_batch.
 * The library scans len on the device into context-owned scratch.  Idle
 * lanes refill themselves from a work counter, so segments of any length mix
 * in one launch.  The scan, the counter reset and the projection kernel are
 * captured once into a CUDA graph and replayed while the arguments and the
 * loaded model stay the same (not when the caller's stream is itself being
 * captured: then the kernels are enqueued directly). */
mcp_status mcp_project_segments(mcp_ctx *ctx, const mcp_project_params *p, int64_t n_seg, int64_t ld_seg,
                                const void *start, const void *delta, const int32_t *len, int64_t total,
                                int64_t ld_out, void *q_out, uint8_t *flags, uint8_t *iters, double *resid,
                                mcp_stream stream);

/* CollisionFree (Alg. 2) of n configurations: in_collision[i] = 1 iff some
 * robot sphere overlaps some obstacle sphere (|c_s - c_o| < r_s + r_o) or box
 * (distance from c_s to the box < r_s).  q: [d * ld] float (precision 0) or
 * double (precision 1).  Each configuration stops at the first block of
 * spheres that overlaps; pairs_tested [n] (uint32, may be NULL) receives the
 * number of sphere-obstacle pairs evaluated for it (work accounting). */
mcp_status mcp_check_batch(mcp_ctx *ctx, int64_t n, int64_t ld, const void *q, int32_t precision,
                           uint8_t *in_collision, uint32_t *pairs_tested, mcp_stream stream);

/* Vector-Jacobian product of the projection at points on the manifold
 * (implicit-function theorem; the paper makes its log map differentiable "to
 * enable gradient-based optimization", Sec. IV-A):
 *   out = g - J^T (J J^T)^{-1} J g   at q_star.
 * q_star, g, out: float [d * ld]; out may alias g.  flags [n] (may be NULL):
 * MCP_F_FP64_RESOLVE if the solve fell back to FP64, MCP_F_NONFINITE if
 * J J^T is singular (out is NaN there). */
mcp_status mcp_project_vjp(mcp_ctx *ctx, int64_t n, int64_t ld, const float *q_star, const float *g, float *out,
                           uint8_t *flags, mcp_stream stream);

/* Path length L = sum_i |q_{i+1} - q_i| of n_paths paths of n_way waypoints
 * and its gradient with respect to every waypoint.  Q: float [d * ld] with
 * waypoint w of path p at column p * n_way + w; length [n_paths] (may be NULL);
 * grad [d * ld] (may be NULL).  Zero-length edges contribute no gradient. */
mcp_status mcp_path_length_grad(mcp_ctx *ctx, int64_t n_paths, int32_t n_way, int64_t ld, const float *Q,
                                float *length, float *grad, mcp_stream stream);

/* Gradient step on paths (the update of path shortening on the manifold):
 * for every interior waypoint (not the first or last of its path)
 *   Q[:, i] -= clip(eta * D[:, i]),  clip scales the step to infinity norm <= max_step (if > 0).
 * Q (in/out) and D: float [d * ld], same waypoint layout as
 * mcp_path_length_grad.  The result is off the manifold; project it again. */
mcp_status mcp_path_step(mcp_ctx *ctx, int64_t n_paths, int32_t n_way, int64_t ld, float *Q, const float *D, float eta,
                         float max_step, mcp_stream stream);

/* Sets the launch shape of the persistent FP32 projection kernel directly
 * (tpb in {64, 128, 256}, blocks_per_sm in 1..8 with tpb * blocks_per_sm <=
 * 2048, chunk in 1..64, fuse_check 0 / 1, threads_per_config 1 / 2), e.g. to
 * reproduce a tuned shape.  threads_per_config = 2 runs the two-chain classes
 * (the dual arm, Eq. 2) with one lane per chain; other classes ignore it.
 * Results of the two kernels differ only by the rounding of the Gram sums.
 * MCP_ERR_ARG outside those ranges. */
mcp_status mcp_set_tuning(mcp_ctx *ctx, int32_t tpb, int32_t blocks_per_sm, int32_t chunk, int32_t fuse_check,
                          int32_t threads_per_config);

/* Picks the launch shape of the persistent FP32 projection kernel (threads
 * per block, resident blocks per SM, configurations claimed per atomic, and
 * threads per configuration where the class has a choice) for
 * the loaded problem by timing every candidate on the caller's sample
 * q_sample (DEVICE, float [d * ld], n_sample configurations), and keeps the
 * fastest in the context for later calls.  With obstacles loaded the timed
 * step is mcp_project_check_batch, and every launch shape is timed with the
 * check inside the projection kernel and as a second launch.  Each candidate
 * is timed as the median of five bursts of four calls.  Uses temporary
 * device buffers; synchronous.  The choices are returned in tpb / blocks_per_sm /
 * chunk / fuse_check / threads_per_config (HOST, each may be NULL).  The
 * launch shape never changes results; threads per configuration changes them
 * by rounding only (see mcp_set_tuning). */
mcp_status mcp_autotune(mcp_ctx *ctx, const mcp_project_params *p, int64_t n_sample, int64_t ld, const void *q_sample,
                        int32_t *tpb, int32_t *blocks_per_sm, int32_t *chunk, int32_t *fuse_check,
                        int32_t *threads_per_config, mcp_stream stream);

/* Arithmetic-throughput probe (no counterpart in the paper: it measures the
 * denominator of the roofline the benchmark reports).  Launches 8 blocks of
 * 256 threads per SM on the context's device; every thread runs 8
 * independent fused multiply-add chains for `iters` rounds in FP32
 * (precision 0) or FP64 (precision 1).  out: DEVICE scratch of
 * one element of that type (written only in a case that does not occur).
 * *flops (HOST, may be NULL) receives the floating-point operations the
 * launch performs (an FMA counts 2); the caller times the launch on `stream`.
 * MCP_ERR_ARG for another precision, iters outside [1, 2^32] or a NULL /
 * host out. */
mcp_status mcp_fma_probe(mcp_ctx *ctx, int32_t precision, int64_t iters, void *out, int64_t *flops,
                         mcp_stream stream);

/* Number of kernels this context has launched so far (for launch accounting). */
int64_t mcp_launch_count(const mcp_ctx *ctx);

/* Number of device allocations (cudaMalloc) the library has made in this
 * process, over all contexts (for tests and accounting: a call that must not
 * allocate leaves it unchanged).
 *
 * Test hooks, read from the environment (host-side failure injection; no
 * kernel is made to fail):
 *   MCP_TEST_FAIL_ALLOC=<text>  every device allocation whose label contains
 *                               <text> fails as out of memory (MCP_ERR_OOM);
 *                               read at each allocation;
 *   MCP_TEST_FAIL_CUDA=<text>   a context created while it is set reports
 *                               MCP_ERR_CUDA from every CUDA call whose label
 *                               contains <text>, after the call has run.
 * Labels name what is allocated or launched ("obstacles", "segment offsets",
 * "project_batch launch", ...; they appear in mcp_last_error). */
int64_t mcp_alloc_count(void);

/* Bounds-check status (no counterpart in the paper; a debugging aid).  A
 * library built with -DMCP_CHECK_BOUNDS tests the index of every batch-array
 * access of its persistent projection kernels against the array's extent;
 * an access out of range is skipped and the source line of the first one is
 * recorded (nothing traps).  *enabled (HOST, may be NULL) receives 1 for such
 * a build, else 0; *first_line (HOST, may be NULL) the first line recorded
 * since the last reset (0: none; always 0 without the checks).  reset != 0
 * clears the record.  Synchronises the context's device.  MCP_ERR_ARG for a
 * NULL context, MCP_ERR_CUDA if the synchronisation fails. */
mcp_status mcp_bounds_status(const mcp_ctx *ctx, int32_t *enabled, uint32_t *first_line, int32_t reset);

/* Allocation-free segment projection.  The paper has no counterpart: this
 * entry point exists for callers that must not allocate device memory once
 * they are running -- a real-time planning or control loop where a
 * cudaMalloc would add unbounded latency (and synchronise the device), or a
 * caller whose device memory is owned by another allocator or budget.
 * mcp_project_segments allocates its segment-offset scratch on demand; this
 * variant computes exactly the same result but keeps the work counter and the
 * offsets in a fixed, file-scope device array of the library, so no call
 * allocates or frees anything (no cudaMalloc, cudaFree, or allocating
 * library routine).  Arguments, layouts and outputs are those of
 * mcp_project_segments.
 *   - n_seg may be at most MCP_NOALLOC_MAX_SEGMENTS; larger batches return
 *     MCP_ERR_ARG with a message and enqueue nothing.
 *   - The array is per device, about 512 KiB, and stays allocated on every
 *     GPU that loads the library until the process exits.
 *   - The first call on a device looks up the array's device address (once
 *     per device, with that device current); make that first call before any
 *     stream capture.  The address is kept for the life of the process: it
 *     does not survive cudaDeviceReset (after a reset the library's device
 *     code is loaded again and the array may move), so a process that resets
 *     a device must not call this entry point on it afterwards.
 *   - Every call shares the array and it keeps the last call's contents: the
 *     counter is cleared by each call, but calls that overlap on the GPU (on
 *     different streams, or from several contexts on the same device) race
 *     and must not be issued. */
#define MCP_NOALLOC_MAX_SEGMENTS 65536
mcp_status mcp_project_segments_noalloc(mcp_ctx *ctx, const mcp_project_params *p, int64_t n_seg, int64_t ld_seg,
                                        const void *start, const void *delta, const int32_t *len, int64_t total,
                                        int64_t ld_out, void *q_out, uint8_t *flags, uint8_t *iters, double *resid,
                                        mcp_stream stream);

#ifdef __cplusplus
}
#endif

#endif /* MCPROJ_H_ */
