/*
 * wbe.h -- C ABI of the GB300 whole-body evaluation library (libwbe.so).
 *
 * One whole-body evaluation of a robot configuration (Sec. 6 of the paper)
 * is, in order:
 *   1. forward kinematics over the kinematic tree (Sec. 6.1.1),
 *   2. collision-sphere placement (Sec. 6.1.1),
 *   3. self-collision signed distance over the masked sphere pairs reduced
 *      to the minimum and the worst pair (Sec. 6.2, Fig. self_collision),
 *   4. joint torques by recursive Newton-Euler inverse dynamics (Sec. 6.3,
 *      Alg. 4),
 * and the backward pass is the vector-Jacobian product of all four (Alg. 1,
 * Alg. 5, Sec. 6.3 "VJP-based backward pass").
 *
 * Conventions
 *   - All device buffers are owned by the caller, live on the robot's
 *     device, are contiguous and 16-byte aligned.  The library keeps no
 *     pointer to them after a call returns.
 *   - Every call that takes a stream enqueues its work on that stream
 *     (a cudaStream_t passed as void*; NULL = the legacy default stream),
 *     returns without synchronising, performs no device allocation and is
 *     safe to capture in a CUDA graph.
 *   - Batched per-configuration arrays use two layouts:
 *       joint-major   [d][B]     (q, qd, qdd, tau and their gradients)
 *       config-major  [B][...]   (link poses, sphere centres, pair bits)
 *     where B is the number of configurations and d the number of actuated
 *     joints.
 *   - A link pose is 12 floats: the world rotation R (row-major 3x3) then
 *     the world position p, so that x_world = R x_link + p.
 *   - Every function returns WB_OK (0) or a negative WB_E* code;
 *     wb_last_error() returns a message for the calling thread's last error.
 */
#ifndef WBE_H
#define WBE_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define WB_OK 0
#define WB_EINVAL (-1)   /* null required pointer, B < 0, misaligned buffer, non-unit axis */
#define WB_ETOPO (-2)    /* parent[k] >= k, bad joint index, bad joint type */
#define WB_ERANGE (-3)   /* pair or link index out of range, duplicate pair, i >= j */
#define WB_ETOOBIG (-4)  /* robot larger than the kernels' limits */
#define WB_EDEVICE (-5)  /* pointer not on the robot's device */
#define WB_ECUDA (-6)    /* CUDA runtime error (allocation, copy or launch) */

/* limits of the kernels (checked at load) */
#define WB_MAX_LINKS 255
#define WB_MAX_SPHERES 1020

typedef struct wb_robot wb_robot; /* opaque, owned by the library */
typedef struct wb_batch wb_batch; /* opaque, owned by the library */

/* Kinematic tree (Sec. 6.1, Fig. fk_comparison).  Host arrays, read during
 * the call only.
 *   parent[k]      -1 for the world, otherwise < k (topological order)
 *   joint_type[k]  0 fixed, 1 revolute, 2 prismatic
 *   axis[k][3]     joint axis in the link frame; |axis| must be 1 within 1e-5
 *                  (it is renormalised in double before rounding to float)
 *   T_fixed[k][12] pose of link k's joint frame in its parent frame:
 *                  rotation (row-major, orthonormal within 1e-5), translation
 *   joint_index[k] actuated joint of link k in [0, d), -1 iff fixed
 *   mimic_mult[k], mimic_offset[k]  (nullable: 1 and 0) the joint variable of
 *                  link k is mimic_mult*q[joint_index] + mimic_offset (the
 *                  mimic joints of Fig. fk_comparison(b) and Alg. 4)
 *   gravity[3]     (nullable: (0, 0, -9.81)) world gravity; it enters the
 *                  dynamics as the base acceleration -gravity            */
typedef struct {
  int32_t n_links;
  const int32_t* parent;
  const int32_t* joint_type;
  const double* axis;
  const double* T_fixed;
  const int32_t* joint_index;
  const double* mimic_mult;
  const double* mimic_offset;
  const double* gravity;
} wb_tree;

/* Collision spheres (Sec. 6.1.1): sphere s sits on link[s] at center[s] in
 * that link's frame, radius[s] >= 0. */
typedef struct {
  int32_t n_spheres;
  const int32_t* link;
  const double* center;
  const double* radius;
} wb_spheres;

/* Self-collision pair mask (Sec. 6.2).  Either an explicit list of n_pairs
 * pairs (i, j) with i < j (mask == NULL), or a dense S x S uint8 mask whose
 * strict upper triangle is read (pairs == NULL).  The library sorts the pairs
 * row-major: the pair index reported by wb_eval is the rank of (i, j) in
 * lexicographic order. */
typedef struct {
  int32_t n_pairs;
  const int32_t* pairs;
  const uint8_t* mask;
} wb_pairs;

/* Inertials (Sec. 6.3, Tab. rnea_comparison "runtime payload").  Per link:
 * mass[k], com[k][3] in the link frame, inertia[k][6] = (xx, yy, zz, xy, xz,
 * yz) about the CoM in link axes.  Optional point masses (payloads):
 * point_mass[m] kg rigidly attached to link point_link[m] at point_pos[m][3]
 * (link frame); their spatial inertia is added to the link's. */
typedef struct {
  const double* mass;
  const double* com;
  const double* inertia;
  int32_t n_points;
  const int32_t* point_link;
  const double* point_mass;
  const double* point_pos;
} wb_inertial;

/* Kernel selection and launch shape (all zero = automatic). */
#define WB_KERNEL_AUTO 0
#define WB_KERNEL_PLAIN 1 /* one thread per configuration, baseline */
#define WB_KERNEL_FUSED 2 /* one thread group per configuration, tiled */
#define WB_KERNEL_TREE 3  /* depth-first sweep kernels (one thread per configuration)
                             for FK, RNEA and the backward, plus a warp-per-
                             configuration sphere/pair kernel; needs link_pose
                             when spheres or pairs are wanted */
#define WB_KERNEL_TREE_NOCULL 4 /* TREE with the pair stage's full map-reduce: every
                                   block screened, no bounding-sphere culling (the
                                   results are identical; for comparison) */
typedef struct {
  int32_t kernel;            /* WB_KERNEL_* (AUTO: TREE when it applies, else FUSED) */
  int32_t lanes_per_config;  /* fused: 4, 8, 16 or 32 (0 = robot default);
                                tree: sweep segments 1, 2, 4 or 8 -- 1 = one thread
                                per configuration, G > 1 = G warps per 32
                                configurations, each sweeping a contiguous piece
                                of the depth-first order (not for robots where a
                                joint drives several links); 0 = the fewest that
                                give about 12 warps per SM */
  int32_t configs_per_block; /* fused: configurations per CTA; tree: threads per block
                                of the sweep kernels (32..256, up to 512 for
                                G > 1 segments); 0 = default */
  int32_t blocks_per_sm;     /* fused: grid = blocks_per_sm * SMs (0 = occupancy);
                                tree: warps per block of the pair kernel, 1..8
                                (0 = of the counts 4..8 whose per-warp
                                workspaces fit in a block's shared memory, the
                                one whose blocks keep the most warps resident
                                on an SM, the fewest on a tie: 4 for the 48-DoF
                                humanoid; fewer than 4 only for robots where
                                no more fit) */
} wb_tune;

typedef struct {
  int32_t n_links, dof, n_spheres, n_pairs, n_levels, max_level_width;
  int32_t n_pair_blocks; /* 4x4 sphere-group blocks holding the pairs */
  int32_t device;
} wb_robot_info;

/* Load and validate a robot; builds the topology cache (levels, children,
 * per-joint link lists; Sec. 6.1.2 "topology cache"), the sorted pair list
 * and its 4x4 block plan, compact float inertials, and copies them to
 * `device`.  *out receives a handle owned by the library (free with
 * wb_free_robot).  Errors: WB_EINVAL, WB_ETOPO, WB_ERANGE, WB_ETOOBIG,
 * WB_ECUDA. */
int wb_load_robot(const wb_tree* tree, const wb_spheres* spheres, const wb_pairs* pairs,
                  const wb_inertial* inertial, int device, wb_robot** out);

/* Replace the inertials (and point masses) of a loaded robot, e.g. to add a
 * payload at run time (Tab. rnea_comparison).  The upload is enqueued on
 * `stream`: work enqueued later on that stream sees the new values.  Calls
 * on other streams must be ordered by the caller.  Not graph-capturable
 * (it copies from host memory).  Errors: WB_EINVAL, WB_ERANGE, WB_ECUDA. */
int wb_set_inertials(wb_robot* robot, const wb_inertial* inertial, void* stream);

int wb_robot_info_get(const wb_robot* robot, wb_robot_info* out);

/* Validate a descriptor and plan it exactly as wb_load_robot would, without
 * touching any GPU: fills *out (device = -1) and, if sched_rounds is not
 * NULL, sched_rounds[t] = rounds of the per-lane pair-block schedule for
 * 4 << t lanes per configuration (t = 0..3).  Same errors as wb_load_robot
 * except WB_EDEVICE / WB_ECUDA. */
int wb_plan_info(const wb_tree* tree, const wb_spheres* spheres, const wb_pairs* pairs,
                 const wb_inertial* inertial, wb_robot_info* out, int32_t* sched_rounds);

/* Forward whole-body evaluation of B configurations (Sec. 6, Alg. 4).
 *   q, qd, qdd   [d][B] joint positions, velocities, accelerations
 *                (qd, qdd may be NULL only if tau == NULL)
 * Outputs (device, written fully; NULL = not wanted):
 *   link_pose    [B][n][12] world poses (NULL skips the store, not FK)
 *   sphere       [B][S][3]  world sphere centres
 *   d_min        [B]        min over masked pairs of |c_i-c_j| - r_i - r_j
 *                           (+inf when the robot has no pairs)
 *   worst_pair   [B]        index of the pair attaining d_min (smallest index
 *                           among exact float ties; -1 when no pairs).
 *                           Required when d_min is given.
 *   tau          [d][B]     joint torques (NULL skips the dynamics)
 *   pair_bits    [B][ceil(P/32)] bit p of word p/32 set iff pair p has
 *                           |c_i-c_j| < r_i + r_j (colliding, strict)
 * B == 0 is a no-op.  Errors: WB_EINVAL (null robot/q, B < 0, misaligned
 * pointer, d_min without worst_pair, tau without qd/qdd), WB_EDEVICE,
 * WB_ETOOBIG (launch shape does not fit), WB_ECUDA (launch failure). */
int wb_eval(wb_robot* robot, int64_t B, const float* q, const float* qd, const float* qdd,
            float* link_pose, float* sphere, float* d_min, int32_t* worst_pair, float* tau,
            uint32_t* pair_bits, const wb_tune* tune, void* stream);

/* Sphere placement and self-collision from given world link poses: the
 * second half of the split forward of Sec. 6.1.1 (a first kernel writes the
 * link transforms, a second reads them and places the spheres) followed by
 * the pair map-reduce of Sec. 6.2.
 *   link_pose    [B][n][12] world poses (as written by wb_eval), required
 *   sphere, d_min, worst_pair, pair_bits  as in wb_eval (nullable; d_min
 *                and worst_pair go together)
 * Errors as wb_eval. */
int wb_self_collision(wb_robot* robot, int64_t B, const float* link_pose, float* sphere,
                      float* d_min, int32_t* worst_pair, uint32_t* pair_bits, void* stream);
/* wb_self_collision with a launch choice: tune->kernel TREE (or AUTO, or a
 * NULL tune) culls 4x4 sphere-group blocks whose bounding-sphere lower bound
 * exceeds an exact upper bound on d_min (the default); TREE_NOCULL screens
 * every block.  tune->blocks_per_sm = warps per block (0 = the most, up to 8,
 * that fit in shared memory).  Same outputs,
 * same tie rule. */
int wb_self_collision_tuned(wb_robot* robot, int64_t B, const float* link_pose, float* sphere,
                            float* d_min, int32_t* worst_pair, uint32_t* pair_bits,
                            const wb_tune* tune, void* stream);

/* wb_self_collision_tuned that also writes worst_diff [B][3] (nullable;
 * needs d_min): c_i - c_j of the worst pair's sphere centres (zero when the
 * robot has no pairs), the direction of d_min's gradient on the spheres.
 * Hand it to wb_eval_backward_dir: the backward then needs no forward
 * kinematics of the worst pair's links of its own.  Errors as wb_eval. */
int wb_self_collision_dir(wb_robot* robot, int64_t B, const float* link_pose, float* sphere,
                          float* d_min, int32_t* worst_pair, float* worst_diff,
                          uint32_t* pair_bits, const wb_tune* tune, void* stream);

/* Kinematic Jacobians of chosen links and the whole-body centre of mass,
 * from world link poses [B][n][12] (from wb_eval): the second-kernel outputs
 * of the split forward kinematics (Sec. 6.1.1), columns as in Alg. 2 (a joint
 * driving several links -- mimic -- sums their contributions).
 *   jac     [B][n_targets][6][d]  per target link e, column j = d/dq_j of
 *           e's world origin (rows 0-2) and e's angular velocity (rows 3-5),
 *           world coordinates; zero for joints not on e's chain
 *   com     [B][3]                centre of mass (links + payload point masses)
 *   jac_com [B][3][d]             its Jacobian
 * targets is a HOST array of n_targets link indices (0 <= n_targets <= 64);
 * each output is nullable.  Errors: WB_EINVAL, WB_ERANGE (target out of
 * range), WB_EDEVICE, WB_ETOOBIG, WB_ECUDA. */
int wb_kinematics(wb_robot* robot, int64_t B, const float* link_pose, int32_t n_targets,
                  const int32_t* targets, float* jac, float* com, float* jac_com, void* stream);

/* All-pairs summed self-collision hinge with activation distance eta (the
 * constraint C_robot <= 0 of the paper's problem statement with a margin, as
 * a penalty over every masked pair rather than the worst one):
 *   cost[b] = w * sum_p max(0, eta - d_p),  d_p = |c_i - c_j| - r_i - r_j
 * and, in g_sphere [B][S][3], its gradient with respect to the sphere centres
 * (a pair with d_p < eta adds -w u at sphere i and +w u at sphere j,
 * u = (c_i - c_j) / |c_i - c_j|; coincident centres add nothing).  Pass
 * g_sphere to wb_eval_backward as its sphere gradient for dcost/dq.  Spheres
 * are placed from link_pose [B][n][12] (from wb_eval).  cost [B] and g_sphere
 * are each nullable.  Deterministic (no atomics).  A pair exactly at eta adds
 * nothing.  Errors: WB_EINVAL, WB_EDEVICE, WB_ETOOBIG, WB_ECUDA. */
int wb_self_collision_hinge(wb_robot* robot, int64_t B, const float* link_pose, float eta,
                            float w, float* cost, float* g_sphere, void* stream);

/* Backward pass: the gradient of
 *   L = <g_pose, link_pose> + <g_sphere, sphere> + sum_b g_dmin[b] d_min[b]
 *       + <g_tau, tau>
 * with respect to q, qd, qdd (Alg. 1 for the kinematic terms, Alg. 5 for the
 * torque terms; the d_min term flows through worst_pair only).  Link
 * transforms and the dynamics forward sweep are recomputed, not stored.
 *   q, qd, qdd   [d][B] the inputs of the forward call
 *   worst_pair   [B] from the forward call (required iff g_dmin != NULL)
 *   g_pose [B][n][12], g_sphere [B][S][3], g_dmin [B], g_tau [d][B]
 *                upstream gradients, each nullable (= zero)
 *   gq, gqd, gqdd [d][B] outputs, overwritten (not accumulated)
 * Errors as wb_eval. */
int wb_eval_backward(wb_robot* robot, int64_t B, const float* q, const float* qd,
                     const float* qdd, const int32_t* worst_pair, const float* g_pose,
                     const float* g_sphere, const float* g_dmin, const float* g_tau, float* gq,
                     float* gqd, float* gqdd, const wb_tune* tune, void* stream);

/* wb_eval / wb_eval_backward with external link wrenches (Alg. 4's f_ext):
 * f_ext [B][n][6], link coordinates, moment then force about the link
 * origin, enters every link force as f_k = I a + v x* I v - f_ext,k (it
 * changes tau only).  The backward also returns g_fext [B][n][6] =
 * dL/df_ext = -fbar_k, the adjoint of the link force (Sec. 6.3).  Both are
 * nullable; the fused kernels reject them (WB_EINVAL), the tree and plain
 * kernels take them. */
int wb_eval_ext(wb_robot* robot, int64_t B, const float* q, const float* qd, const float* qdd,
                const float* f_ext, float* link_pose, float* sphere, float* d_min,
                int32_t* worst_pair, float* tau, uint32_t* pair_bits, const wb_tune* tune,
                void* stream);
int wb_eval_backward_ext(wb_robot* robot, int64_t B, const float* q, const float* qd,
                         const float* qdd, const float* f_ext, const int32_t* worst_pair,
                         const float* g_pose, const float* g_sphere, const float* g_dmin,
                         const float* g_tau, float* gq, float* gqd, float* gqdd, float* g_fext,
                         const wb_tune* tune, void* stream);

/* wb_eval_backward_ext with the worst pair's centre difference worst_diff
 * [B][3] from wb_self_collision_dir on the same poses (nullable: the sweep
 * places the two spheres itself).  The tree kernels use it in place of the
 * forward kinematics of the pair's two links and give the same results bit
 * for bit; the fused and plain kernels ignore it.  Errors as wb_eval. */
int wb_eval_backward_dir(wb_robot* robot, int64_t B, const float* q, const float* qd,
                         const float* qdd, const float* f_ext, const int32_t* worst_pair,
                         const float* worst_diff, const float* g_pose, const float* g_sphere,
                         const float* g_dmin, const float* g_tau, float* gq, float* gqd,
                         float* gqdd, float* g_fext, const wb_tune* tune, void* stream);

/* Autotuner (a setup-time call: it allocates scratch buffers for B
 * configurations, synchronises the device and must not be captured).  Times
 * every applicable kernel family and launch shape -- depth-first sweep kernels
 * with 64 / 128 / 256 threads per block (512 and the block that deals B
 * evenly over the SMs in one wave for segmented sweeps; the latter for one
 * segment too) and 4 / 8 warps per pair block, fused
 * kernels with 4, 8, 16 and 32 lanes per configuration, the plain kernels --
 * on random states with all outputs (forward) and all upstream gradients
 * (backward; the tree kernels with the worst pair's centre difference from
 * wb_self_collision_dir, as wb_eval_backward_dir takes it), and returns the
 * fastest choice for each pass with its median
 * time (ms, nullable).  Each candidate is timed 5 times, each run after an
 * L2 flush (a memset of twice the L2 size), and ranked by the median; a
 * backward candidate runs after the flush and an untimed forward with the
 * pair stage (default launch), so that it meets the cache as a step leaves
 * it. */
int wb_autotune(wb_robot* robot, int64_t B, wb_tune* fwd, wb_tune* bwd, float* fwd_ms,
                float* bwd_ms);

void wb_free_robot(wb_robot* robot);

/* ---------------------------------------------------------------------------
 * Uneven batches (several robots, uneven horizons) in one persistent launch
 * per pass.  A problem is (robot index, horizon H); problem p owns slices of
 * packed arrays:
 *   joint-major  [d_p][H_p]       q, qd, qdd, tau, gradients (offset joint[p])
 *   poses        [H_p][n_p][12]   (offset pose[p])
 *   spheres      [H_p][S_p][3]    (offset sphere[p])
 *   per config   [H_p]            d_min, worst pair, g_dmin (offset config[p])
 * (offsets in elements, from wb_batch_offsets).  Work items are sorted by cost
 * and pulled by the warps of a persistent grid through an atomic counter held
 * by the batch object (cleared on the stream before each launch): calls on
 * one batch object must not overlap on the GPU; use one object per stream.
 * Forward and backward are graph-capturable.  Robots must stay alive while
 * the batch exists. */
typedef struct {
  int32_t robot;   /* index into the robots array of wb_batch_create */
  int32_t horizon; /* configurations of this problem, >= 0 */
} wb_problem;

typedef struct {
  int64_t joint_elems, pose_elems, sphere_elems, configs; /* packed array lengths */
  int32_t n_problems, n_robots;
} wb_batch_sizes;

int wb_batch_create(wb_robot* const* robots, int32_t n_robots, const wb_problem* problems,
                    int32_t n_problems, wb_batch** out);
int wb_batch_sizes_get(const wb_batch* batch, wb_batch_sizes* out);
/* per-problem offsets into the packed arrays (host arrays of n_problems) */
int wb_batch_offsets(const wb_batch* batch, int64_t* joint, int64_t* pose, int64_t* sphere,
                     int64_t* config);
/* link_pose is required when sphere or d_min is wanted (the pair pass reads it) */
int wb_batch_eval(wb_batch* batch, const float* q, const float* qd, const float* qdd,
                  float* link_pose, float* sphere, float* d_min, int32_t* worst_pair, float* tau,
                  void* stream);
int wb_batch_eval_backward(wb_batch* batch, const float* q, const float* qd, const float* qdd,
                           const int32_t* worst_pair, const float* g_pose, const float* g_sphere,
                           const float* g_dmin, const float* g_tau, float* gq, float* gqd,
                           float* gqdd, void* stream);
void wb_free_batch(wb_batch* batch);

/* Launch choices of an uneven batch (Sec. 7, batched evaluation: the
 * threads per configuration and the block shapes of the persistent launches,
 * chosen per robot and per batch).  Per robot and pass, the sweep takes 1 or 2
 * segments: 2 = the two warps of a pair sweep the two halves of the robot's
 * depth-first order over the same 32 configurations (robots with a
 * 2-segment plan only), 1 = each warp sweeps its own 32 configurations whole.
 * Outputs do not depend on the choice beyond float summation order (the
 * segments' shares of a shared ancestor are added in segment order). */
typedef struct {
  int32_t fwd_threads; /* threads per block of the forward sweep pass: 64, 128 or 256 (0 = 128) */
  int32_t bwd_threads; /* the same for the backward sweep pass */
  int32_t pair_warps;  /* warps per block of the pair pass, 1..8 (0 = the most that fit) */
} wb_batch_tune;

/* Set the batch's launch choices; fwd_segments and bwd_segments are host
 * arrays of n_robots values (1 or 2), each nullable (= 2 where the robot has a
 * 2-segment plan, else 1: wb_batch_create's defaults).  A set-up call: it
 * uploads the batch's work lists with a synchronous copy; do not call it while
 * the batch's work is in flight or during stream capture.  Errors: WB_EINVAL
 * (bad value, 2 segments for a robot without a plan), WB_ETOOBIG (more pair
 * warps than fit), WB_ECUDA. */
int wb_batch_set_tune(wb_batch* batch, const wb_batch_tune* tune, const int32_t* fwd_segments,
                      const int32_t* bwd_segments);
/* The batch's current choices (each output nullable; segments: n_robots). */
int wb_batch_get_tune(const wb_batch* batch, wb_batch_tune* tune, int32_t* fwd_segments,
                      int32_t* bwd_segments);
/* Autotuner of the batch (a set-up call like wb_autotune: it allocates scratch
 * buffers of the batch's packed sizes, synchronises the device and must not
 * be captured).  On deterministic states and upstream gradients it times the
 * forward and backward sweep passes for every per-robot choice of 1 or 2
 * segments (all combinations over the robots that have a 2-segment plan and a
 * problem when there are at most 4, else one pass of coordinate descent from
 * the defaults) in blocks of 64, 128 and 256 threads, and the pair pass with
 * 2, 4 and 8 warps a block (those that fit), 5 runs per candidate after an L2
 * flush (median); the fastest become the batch's choices for later calls and
 * are returned (each output nullable), with the forward (sweep + pair) and
 * backward times in ms.  Errors: WB_EINVAL, WB_ETOOBIG, WB_ECUDA. */
int wb_batch_autotune(wb_batch* batch, wb_batch_tune* tune, int32_t* fwd_segments,
                      int32_t* bwd_segments, float* fwd_ms, float* bwd_ms);

/* ---------------------------------------------------------------------------
 * Trajectory-optimisation ends of the evaluation.  These calls take no robot:
 * every buffer must live on one device (the first non-NULL buffer fixes it),
 * be 16-byte aligned and caller-owned.
 *
 * Joint states from uniform cubic B-spline control points (Sec. 4,
 * Eq. bspline-cubic): U [n_traj][d][K] control points per trajectory and
 * joint; each trajectory is sampled at T points uniformly spaced over its K-3
 * segments, t_s = s (K-3) / (T-1), segment k = min(floor(t_s), K-4),
 * alpha = t_s - k, window u_k .. u_k+3, state = T P(alpha) C window with the
 * time scaling 1/dt per derivative order.  Outputs q, qd, qdd (each nullable)
 * joint-major [d][n_traj*T], configuration b = traj*T + s.
 * Limits: 4 <= K <= 4096, 2 <= T <= 4096, dt > 0.
 * Errors: WB_EINVAL, WB_EDEVICE, WB_ECUDA. */
int wb_bspline_eval(int64_t n_traj, int32_t d, int32_t K, int32_t T, float dt, const float* U,
                    float* q, float* qd, float* qdd, void* stream);

/* Control-point gradient (Eq. backward_grad): gU [n_traj][d][K] (overwritten)
 * = sum over samples of B(alpha)^T (gq, gqd, gqdd) for the four control
 * points of each sample's window; upstream gradients [d][n_traj*T], each
 * nullable (= zero).  Deterministic (no atomics).  Errors as wb_bspline_eval. */
int wb_bspline_backward(int64_t n_traj, int32_t d, int32_t K, int32_t T, float dt,
                        const float* gq, const float* gqd, const float* gqdd, float* gU,
                        void* stream);

/* Boundary conditions (Sec. 4.2).  The spline is evaluated on an extended
 * sequence of Kx = K + 3 [start] + 3 [end_static] knots:
 *   - start (nullable) [n_traj][d][3] holds theta_0, thetadot_0, thetaddot_0
 *     per trajectory and joint; the ghost knots of Eqs. fixed_3, fixed_2,
 *     fixed_1 come first,
 *       u_-3 = th0 - a0 dt^2 / 6,  u_-2 = th0 + v0 dt + a0 dt^2 / 3,
 *       u_-1 = th0 + 2 v0 dt + 11 a0 dt^2 / 6,
 *     so the first sample is the start state carried one knot interval
 *     forward with zero jerk;
 *   - end_static != 0 repeats the last control point three more times, so the
 *     last segment holds it at rest (Eq. stop-constraint).
 * The T samples spread over the Kx - 3 segments as in wb_bspline_eval.
 * Limits: 1 <= K <= 4096 and Kx >= 4; T, dt as wb_bspline_eval.  start is a
 * caller-owned device buffer on the device of U.  With start == NULL and
 * end_static == 0 this is wb_bspline_eval.
 * Errors: WB_EINVAL, WB_EDEVICE, WB_ECUDA. */
int wb_bspline_eval_bc(int64_t n_traj, int32_t d, int32_t K, int32_t T, float dt, const float* U,
                       const float* start, int32_t end_static, float* q, float* qd, float* qdd,
                       void* stream);

/* Gradients through wb_bspline_eval_bc (Eq. backward_grad on the extended
 * sequence): gU [n_traj][d][K] (overwritten; with end_static the last
 * control point also receives the gradients of its three repeats) and, when
 * has_start != 0 and g_start != NULL, the start-state gradient g_start
 * [n_traj][d][3] (the transpose of the ghost knots' linear map applied to
 * their gradients).  Upstream gradients gq, gqd, gqdd and the additive
 * gqd_add, gqdd_add [d][n_traj*T], each nullable.  g_start without
 * has_start is an error.  Deterministic.  Errors as wb_bspline_eval_bc. */
int wb_bspline_backward_bc(int64_t n_traj, int32_t d, int32_t K, int32_t T, float dt,
                           int32_t has_start, int32_t end_static, const float* gq,
                           const float* gqd, const float* gqdd, const float* gqd_add,
                           const float* gqdd_add, float* gU, float* g_start, void* stream);

/* As wb_bspline_backward, with two more upstream gradients gqd_add and
 * gqdd_add [d][n_traj*T] (nullable) that add to gqd and gqdd before the
 * transpose: the direct state gradients of a cost (wb_trajopt_cost_ext)
 * join those of the dynamics without a separate addition pass.
 * Deterministic.  Errors as wb_bspline_eval. */
int wb_bspline_backward_ext(int64_t n_traj, int32_t d, int32_t K, int32_t T, float dt,
                            const float* gq, const float* gqd, const float* gqdd,
                            const float* gqd_add, const float* gqdd_add, float* gU,
                            void* stream);

/* Per-configuration cost of trajectory optimisation and its upstream
 * gradients:
 *   cost[b]     = sum_j max(0, tau[j][b] - tau_hi[j]) + max(0, tau_lo[j] - tau[j][b])
 *                 + w_coll * max(0, -d_min[b])
 *   g_tau[j][b] = [tau > tau_hi] - [tau < tau_lo]      (d cost / d tau)
 *   g_dmin[b]   = -w_coll * [d_min < 0]                (d cost / d d_min)
 * i.e. torque-limit hinges and the self-collision hinge on the worst pair
 * (the constraint C_robot <= 0 of the paper's problem statement turned into
 * a penalty); a kink takes the zero one-sided derivative.  tau, g_tau [d][B];
 * d_min, cost, g_dmin [B]; tau_lo, tau_hi [d] device arrays (required with
 * tau).  Any of tau / d_min may be NULL (its terms vanish); any output may be
 * NULL.  Feed g_tau and g_dmin (with the forward's worst pair) to
 * wb_eval_backward and the result to wb_bspline_backward for dL/dU.
 * Errors: WB_EINVAL, WB_EDEVICE, WB_ECUDA. */
int wb_trajopt_cost(int64_t B, int32_t d, const float* tau, const float* d_min,
                    const float* tau_lo, const float* tau_hi, float w_coll, float* cost,
                    float* g_tau, float* g_dmin, void* stream);

/* Weights of the cost terms of wb_trajopt_cost_ext. */
typedef struct {
  float collision; /* w_coll of the worst-pair hinge */
  float smooth;    /* weight of |qdd|^2 */
  float length;    /* weight of |qd|^2 */
  float energy;    /* weight of sum_j (qd_j tau_j dt)^2 */
  float dt;        /* time between consecutive samples (the energy term's dt) */
} wb_cost_weights;

/* wb_trajopt_cost with the motion terms of the problem's loss (Sec. 3,
 * Eq. cost_motion_opt: the smooth, length and energy terms):
 *   cost[b]     = (wb_trajopt_cost's terms with w_coll = w->collision)
 *                 + smooth |qdd_b|^2 + length |qd_b|^2
 *                 + energy dt^2 sum_j (qd[j][b] tau[j][b])^2
 *   g_tau[j][b] = [tau > tau_hi] - [tau < tau_lo] + 2 energy dt^2 qd^2 tau
 *   g_dmin[b]   = -w->collision [d_min < 0]
 *   g_qd[j][b]  = 2 length qd + 2 energy dt^2 qd tau^2   (direct gradient)
 *   g_qdd[j][b] = 2 smooth qdd                           (direct gradient)
 * qd, qdd, g_qd, g_qdd [d][B], each nullable (a NULL state is zero, its
 * terms vanish; a NULL output is not written).  w is a host pointer, read
 * before the call returns, all five weights finite and dt > 0.  Pass g_qd
 * and g_qdd to wb_bspline_backward_ext as gqd_add and gqdd_add.
 * Errors: WB_EINVAL, WB_EDEVICE, WB_ECUDA. */
int wb_trajopt_cost_ext(int64_t B, int32_t d, const float* tau, const float* d_min,
                        const float* qd, const float* qdd, const float* tau_lo,
                        const float* tau_hi, const wb_cost_weights* w, float* cost,
                        float* g_tau, float* g_dmin, float* g_qd, float* g_qdd, void* stream);

/* The trajectory cost folded into the backward sweep (the cost's gradients
 * formed in the sweep's prologue, without a separate cost pass).  Same
 * results, up to float summation order, as
 *   wb_trajopt_cost_ext(B, d, tau, d_min, qd, qdd, tau_lo, tau_hi, w,
 *                       cost, g_tau, g_dmin, g_qd, g_qdd)
 *   wb_eval_backward(robot, B, q, qd, qdd, worst_pair, g_pose, g_sphere,
 *                    g_dmin, g_tau, gq, gqd, gqdd)
 *   gqd += g_qd; gqdd += g_qdd
 * i.e. gq, gqd, gqdd [d][B] are the total gradients of
 *   sum_b cost_b + <g_pose, poses> + <g_sphere, sphere centres>
 * with respect to q, qd, qdd (feed them to wb_bspline_backward for dL/dU),
 * and cost [B] (nullable) is the per-configuration cost.  tau [d][B] are the
 * forward torques at (q, qd, qdd); d_min [B] (nullable: no collision term)
 * the forward's worst-pair distance with its worst_pair (then required);
 * g_pose, g_sphere nullable.  Runs in the tree kernels only (tune NULL,
 * AUTO or TREE with its segment and block choices).  The robot must drive
 * each joint with one link (no shared mimic joints).
 * Errors: WB_EINVAL (also a robot with shared mimic joints or another
 * kernel), WB_EDEVICE, WB_ETOOBIG (tree deeper than the sweep kernels take),
 * WB_ECUDA. */
int wb_eval_backward_cost(wb_robot* robot, int64_t B, const float* q, const float* qd,
                          const float* qdd, const int32_t* worst_pair, const float* g_pose,
                          const float* g_sphere, const float* tau, const float* d_min,
                          const float* tau_lo, const float* tau_hi, const wb_cost_weights* w,
                          float* cost, float* gq, float* gqd, float* gqdd, const wb_tune* tune,
                          void* stream);

/* wb_eval_backward_cost with the worst pair's centre difference worst_diff
 * [B][3] from wb_self_collision_dir on the same poses (nullable), as
 * wb_eval_backward_dir takes it: the same results, without the forward
 * kinematics of the pair's two links in the sweep. */
int wb_eval_backward_cost_dir(wb_robot* robot, int64_t B, const float* q, const float* qd,
                              const float* qdd, const int32_t* worst_pair,
                              const float* worst_diff, const float* g_pose,
                              const float* g_sphere, const float* tau, const float* d_min,
                              const float* tau_lo, const float* tau_hi, const wb_cost_weights* w,
                              float* cost, float* gq, float* gqd, float* gqdd,
                              const wb_tune* tune, void* stream);

/* The whole-body evaluation with the joint states evaluated from uniform
 * cubic B-spline control points inside the sweeps (Sec. 4, Eq.
 * bspline-cubic, fused with the evaluation): no q, qd, qdd arrays.
 * U [n_traj][d][K] control points (device, caller-owned); configuration
 * b = traj * T + s is sample s of trajectory traj, laid out as in
 * wb_bspline_eval.  Limits: 4 <= K <= 4096, 2 <= T <= 4096, dt > 0.  The
 * states are the same bits as wb_bspline_eval's, so the results equal those
 * of wb_bspline_eval followed by wb_eval (and wb_eval_backward_cost). */
typedef struct {
  const float* U;
  int64_t n_traj;
  int32_t K, T;
  float dt;
} wb_spline;

/* wb_eval on B = n_traj * T configurations from control points: link poses,
 * spheres, d_min / worst pair (each nullable; spheres and pairs need the
 * poses) and tau.  Tree kernels only (tune NULL, AUTO, TREE, TREE_NOCULL);
 * no pair bits.  Errors as wb_eval. */
int wb_eval_spline(wb_robot* robot, const wb_spline* spline, float* link_pose, float* sphere,
                   float* d_min, int32_t* worst_pair, float* tau, const wb_tune* tune,
                   void* stream);

/* wb_eval_backward_cost on the same configurations from control points: the
 * cost in the backward sweep's prologue, gq, gqd, gqdd [d][n_traj*T] (feed
 * them to wb_bspline_backward for dL/dU) and the cost [n_traj*T].  Arguments
 * and errors as wb_eval_backward_cost. */
int wb_eval_backward_spline_cost(wb_robot* robot, const wb_spline* spline,
                                 const int32_t* worst_pair, const float* g_pose,
                                 const float* g_sphere, const float* tau, const float* d_min,
                                 const float* tau_lo, const float* tau_hi,
                                 const wb_cost_weights* w, float* cost, float* gq, float* gqd,
                                 float* gqdd, const wb_tune* tune, void* stream);

/* wb_eval_backward_spline_cost with the worst pair's centre difference
 * worst_diff [n_traj*T][3] (nullable), as wb_eval_backward_cost_dir. */
int wb_eval_backward_spline_cost_dir(wb_robot* robot, const wb_spline* spline,
                                     const int32_t* worst_pair, const float* worst_diff,
                                     const float* g_pose, const float* g_sphere,
                                     const float* tau, const float* d_min, const float* tau_lo,
                                     const float* tau_hi, const wb_cost_weights* w, float* cost,
                                     float* gq, float* gqd, float* gqdd, const wb_tune* tune,
                                     void* stream);

/* Autotuner of the control-point path (a setup-time call like wb_autotune:
 * it allocates scratch buffers for n_traj * T configurations, synchronises the
 * device and must not be captured).  Times the depth-first sweep shapes
 * (1 / 2 / 4 / 8 segments as the robot's segment plans allow, and the block
 * sizes wb_autotune tries) of the two kernels this path runs -- wb_eval_spline
 * with link poses and torques (the forward sweep), and
 * wb_eval_backward_spline_cost_dir with the cost weights w (host pointer),
 * torque limits of +-30 and the worst pairs' centre differences -- on
 * deterministic control points in [-pi/2, pi/2],
 * 5 runs per candidate, each after an L2 flush (a backward candidate also
 * after an untimed forward sweep and pair stage), and returns the fastest
 * shape for each with its median time (ms, nullable).  Its choices differ from
 * wb_autotune's where the spline-cost backward kernel prefers another block
 * size than the plain backward sweep.  n_traj >= 1 and K, T, dt as
 * wb_spline.
 * Errors: WB_EINVAL (NULL argument, sizes, shared mimic joints), WB_ETOOBIG
 * (tree deeper than the sweep kernels take), WB_ECUDA. */
int wb_autotune_spline(wb_robot* robot, int64_t n_traj, int32_t K, int32_t T, float dt,
                       const wb_cost_weights* w, wb_tune* fwd, wb_tune* bwd, float* fwd_ms,
                       float* bwd_ms);

/* ---------------------------------------------------------------------------
 * Forward evaluation of an uneven batch without any device allocation.  The
 * paper has no counterpart to this entry point.
 *
 * Who needs it: a caller whose mix of problems (which robots, which horizons)
 * changes from call to call, e.g. a planner or controller that checks a fresh
 * set of candidate trajectories every cycle.  With wb_batch_create it would
 * create and free a batch object per call, and that allocates and releases
 * device memory (cudaMalloc / cudaFree), which can synchronise the whole
 * device and take unbounded time: a fixed-period control loop cannot afford
 * that, and a process whose device memory is held by another allocator (a
 * framework's caching allocator) may not be able to allocate at all.  This
 * call allocates nothing, on the device or through any library.
 *
 * Arguments and packed layouts are those of wb_batch_create + wb_batch_eval:
 * problem p's slices start at the prefix sums, in problem order, of d_p*H_p
 * (joint-major arrays), H_p*n_p*12 (poses), H_p*S_p*3 (spheres) and H_p (per
 * configuration); wb_batch_offsets of a batch built from the same problems
 * gives the same offsets.  Outputs are identical to wb_batch_eval's.
 *
 * Scratch: the work tables and counters live in one device array inside the
 * library, about 0.6 MiB per device, reserved when the library's device code
 * is loaded on that device.  Limits: at most WB_NOALLOC_MAX_ROBOTS robots,
 * WB_NOALLOC_MAX_PROBLEMS problems and WB_NOALLOC_MAX_CONFIGS configurations
 * (sum of horizons) per call; larger calls fail with WB_ETOOBIG and change
 * nothing.  Each call rebuilds the tables on `stream` (one setup kernel) before
 * the passes read them.  What must start at zero: the work counter of each
 * pass; the call clears it itself on `stream` (cudaMemsetAsync) before the
 * pass.
 *
 * Setup: the first call on a device looks up the scratch array's device
 * address (cudaGetSymbolAddress, with that device current), which may load
 * the library's device code there; make that first call on each device before
 * any stream capture begins, e.g. as a warm-up.  The address is kept for the
 * life of the process: after a cudaDeviceReset of that device it is stale,
 * and this call must not be used on that device again.
 *
 * The statement on graph capture in the conventions at the top of this file
 * does not cover this call.
 *
 * The scratch is shared by all calls on a device: calls whose GPU work may
 * overlap (different streams without ordering between them, or several host
 * threads) race on it and give wrong results.  Order them on one stream or
 * with events.  Robots must stay alive until the call's work has finished.
 *
 * Errors: WB_EINVAL (null robots or q, horizon < 0, misaligned pointer,
 * d_min without worst_pair, tau without qd/qdd, sphere or d_min without
 * link_pose), WB_ERANGE (robot index out of range), WB_EDEVICE (robots or
 * buffers on different devices), WB_ETOOBIG (a limit above exceeded, robot
 * deeper than the sweep kernels' limit), WB_ECUDA (lookup or launch failure). */
#define WB_NOALLOC_MAX_ROBOTS 8
#define WB_NOALLOC_MAX_PROBLEMS 1024
#define WB_NOALLOC_MAX_CONFIGS 65536
int wb_batch_eval_noalloc(wb_robot* const* robots, int32_t n_robots, const wb_problem* problems,
                          int32_t n_problems, const float* q, const float* qd, const float* qdd,
                          float* link_pose, float* sphere, float* d_min, int32_t* worst_pair,
                          float* tau, void* stream);

/* Message describing the calling thread's most recent error ("" if none). */
const char* wb_last_error(void);

/* Library version (major*10000 + minor*100 + patch). */
int wb_version(void);

#ifdef __cplusplus
}
#endif

#endif /* WBE_H */
