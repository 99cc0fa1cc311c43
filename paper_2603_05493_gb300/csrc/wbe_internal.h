// wbe_internal.h -- device-side robot layout shared by the host loader and
// the kernels of libwbe.so (not part of the public ABI).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace wbe {

// Device copy of a robot: everything a kernel needs, as device pointers.
// Passed to kernels by value.  All per-link arrays are indexed by link id
// (topological order, parent[k] < k).
struct DevRobot {
  int n;       // links (including fixed ones)
  int d;       // actuated joints
  int S;       // spheres
  int P;       // masked pairs
  int nlev;    // tree levels (depth 0 = links whose parent is the world)
  int maxw;    // widest level
  int Sg;      // sphere groups of 4 (S padded up to a multiple of 4)
  int nblk;    // 4x4 group blocks holding at least one pair
  float margin;              // pair filter margin (metres), see the pair stage
  float etol;                // pair filter tolerance on the squared form (m^2)
  float rmin;                // smallest sphere radius
  int all_full;              // every pair block holds all 16 pairs
  int sph_vec4;              // S % 4 == 0 and every link's spheres are runs of 4
                             // consecutive indices from a multiple of 4: a link's
                             // [B][S][3] rows load as float4 triples, and every
                             // group of 4 spheres lies on one link
  float abase[3];            // base acceleration = -gravity

  // per link
  const int16_t* parent;     // [n] -1 = world
  const int8_t* jtype;       // [n] 0 fixed, 1 revolute, 2 prismatic
  const int8_t* rot_id;      // [n] 1 if the fixed rotation is the identity
  const int16_t* jidx;       // [n] actuated joint or -1
  const float* mimic;        // [n][2] multiplier, offset
  const float* axis;         // [n][4] unit axis (xyz, pad)
  const float* Tf;           // [n][12] fixed transform R (row-major), p
  const float* inert;        // [n][10] m, h = m*c (3), Io (xx yy zz xy xz yz) about origin
  // topology cache (Sec. 6.1.2)
  const int16_t* lev_start;  // [nlev+1]
  const int16_t* lev_links;  // [n] links grouped by level
  const int2* dfs;           // [n] depth-first pre-order: link, depth
  const int2* dfs_kj;        // [n] the same positions packed for the sweeps: link |
                             //   depth << 8 | chain_start[link] << 16, (joint + 1) |
                             //   min(children, 255) << 16 | joint type << 24 | rot_id << 26
  const int* lmeta;          // [n] per link: (joint + 1) | joint type << 16 | rot_id << 24
  int maxdepth;              // deepest link depth + 1
  int mimic_shared;          // 1 if some joint drives more than one link
  const int16_t* chain_start;// [n+1] ancestor chains (Alg. 1 "linkChain")
  const int16_t* chain;      // root -> link, link included
  const int* chain_m;        // the chain's entries packed: link | (joint + 1) << 8 |
                             //   joint type << 17 | rot_id << 19
  const int16_t* dfs_pos;    // [n] DFS position of each link
  const int16_t* dfs_end;    // [n] one past the last DFS position of its subtree
  // segmented sweeps with G = 2 << t segments, t = 0, 1, 2 (tree_sweep.cuh)
  int seg_ok;                // bit t set: plan t exists
  int seg_ns[3];             // shared output slots of plan t
  int16_t seg_pos[3][9];     // first DFS position of each segment; [G] = n
  const int16_t* seg_slot;   // [3][n] shared output slot of a link, -1 = none
  const int16_t* seg_slot_link; // [3][n] link of each slot
  const int4* lvm;           // [n] per level-ordered slot: link, parent,
                             //   (jidx+1) | jtype << 16 | rot_id << 24,
                             //   child_start | child_end << 16
  const int16_t* child_start;// [n+1]
  const int16_t* children;   // [n]
  const int16_t* jl_start;   // [d+1] links driven by each joint (mimic)
  const int16_t* jl_links;   // [#driven links]
  const int16_t* ls_start;   // [n+1] spheres of each link
  const int16_t* ls_sph;     // [S]
  // spheres and pairs
  const float4* sph;         // [S] centre in link frame (xyz), radius (w)
  const int16_t* sph_link;   // [S]
  const int2* pairs;         // [P] sorted row-major
  const float4* grp_rad;     // [Sg] radii of the 4 spheres of a group (0 pad)
  const float4* grp_loc;     // [Sg] bounding sphere of a one-link group in its link frame
  const int16_t* grp_link;   // [Sg] that link, or -1 (spheres on several links)
  const int32_t* blk_pidx;   // [nblk][16] pair index of (4gi+a, 4gj+b) or -1
};

// A per-lane schedule of pair blocks for the fused kernel with G lanes per
// configuration: entry [r][l] is the block lane l processes in round r.
// x = gi | gj << 8 | mask << 16 (mask bit a*4+b = pair (4gi+a, 4gj+b) is
// masked in), y = block id (row of blk_pidx); mask 0 = no work.
struct PairSchedule {
  int G;
  int rounds;
  const uint2* ent;          // [rounds][G]
};

// The same blocks dealt to 32 lanes for the warp-per-configuration pair
// kernel, encoded with byte offsets: x = 16 gi | (16 gj) << 16 (offsets of
// the row / column group within one per-warp sphere array), y = mask << 16 |
// block id; mask 0 = no work.
struct PairSchedule32 {
  int rounds;
  const uint2* ent;          // [rounds + 1][32], the last round all null
};

// Kernel-side launch configuration of the fused kernels.
struct FusedShape {
  int G;                     // lanes per configuration (4, 8, 16, 32)
  int cpb;                   // configurations per CTA
  int grid;                  // CTAs
  size_t smem;               // dynamic shared memory per CTA
};

struct FwdArgs {
  int64_t B;
  const float* q;
  const float* qd;
  const float* qdd;
  float* pose;
  float* sph;
  float* dmin;
  int32_t* worst;
  float* tau;
  uint32_t* bits;
  const float* fext = nullptr;  // [B][n][6] external link wrenches, link coordinates
  float* wdiff = nullptr;       // [B][3] c_i - c_j of the worst pair (pair stage), or nullptr
};

// The trajectory cost folded into the backward sweep (a separate kernel
// argument of the cost variants of the sweep kernels): the sweep computes
// g_tau, g_dmin and the cost's direct qd / qdd gradients itself, adds the
// latter to its gqd / gqdd outputs and writes the cost.
struct FusedCost {
  const float* tau = nullptr;    // [d][B] forward torques
  const float* d_min = nullptr;  // [B] worst-pair distance, or nullptr (no collision term)
  const float* lo = nullptr;     // [d] torque limits
  const float* hi = nullptr;
  float w = 0.0f, smooth = 0.0f, length = 0.0f, e = 0.0f;  // e = energy dt^2
  float* cost = nullptr;         // [B] out, or nullptr
};

// Joint states from uniform cubic B-spline control points U [n_traj][d][K]:
// configuration b is sample b mod T of trajectory b / T (Sec. 4).
struct SplineArgs {
  const float* U = nullptr;
  int K = 0, T = 0;
  float dt = 0.0f;
};

struct BwdArgs {
  int64_t B;
  const float* q;
  const float* qd;
  const float* qdd;
  const int32_t* worst;
  const float* g_pose;
  const float* g_sph;
  const float* g_dmin;
  const float* g_tau;
  float* gq;
  float* gqd;
  float* gqdd;
  const float* fext = nullptr;  // [B][n][6]
  float* g_fext = nullptr;      // [B][n][6]: -Fbar_k
  const float* wdiff = nullptr; // [B][3] c_i - c_j of the worst pair from the pair stage, or
                                // nullptr: the sweep places the two spheres itself
};

// One problem of an uneven batch: robot index and horizon, and the offsets
// (in elements) of its slices of the packed arrays.
struct BatchProblemDev {
  int robot;
  int H;
  int64_t jo, po, so, co;  // joint-major, pose, sphere, per-configuration
};

struct BatchIO {
  const float* q;
  const float* qd;
  const float* qdd;
  float* pose;
  float* sph;
  float* dmin;
  int32_t* worst;
  float* tau;
  const float* g_pose;
  const float* g_sph;
  const float* g_dmin;
  const float* g_tau;
  float* gq;
  float* gqd;
  float* gqdd;
};

// Sweep items of an uneven batch: x = problem, y = first configuration,
// z = count, w = mode (0: the two warps of a pair sweep the two segments of
// the robot's 2-segment plan over <= 32 configurations, or the first warp the
// whole tree when the robot has no plan; 1: each warp of the pair sweeps its
// own 32 of <= 64 configurations whole).  ns_max: the most shared output
// slots among the robots' 2-segment plans; threads: 64, 128 or 256 (pairs of
// warps per block).
cudaError_t launch_batch_tree_fwd(const DevRobot* robots, const BatchProblemDev* probs,
                                  const int4* items, int n_items, int* counter, const BatchIO& io,
                                  int grid, int ns_max, int threads, cudaStream_t s);
cudaError_t launch_batch_tree_bwd(const DevRobot* robots, const BatchProblemDev* probs,
                                  const int4* items, int n_items, int* counter, const BatchIO& io,
                                  int grid, int ns_max, int threads, cudaStream_t s);
cudaError_t launch_batch_pair(const DevRobot* robots, const PairSchedule32* scheds,
                              const BatchProblemDev* probs, const int2* items, int n_items,
                              int* counter, const BatchIO& io, int grid, int warps, int ws_words,
                              int rad_words, cudaStream_t s);
cudaError_t batch_pair_max_blocks_per_sm(int warps, int ws_words, int rad_words, int* out);
size_t batch_pair_smem(int ws_words, int rad_words, int warps);

// Forward batch evaluation on tables in a file-scope device array
// (k_noalloc.cu).  The limits equal the public WB_NOALLOC_MAX_* values.
constexpr int NA_MAX_ROBOTS = 8;
constexpr int NA_MAX_PROBLEMS = 1024;
constexpr int NA_MAX_CONFIGS = 65536;
constexpr int NA_MAX_DEVICES = 64;
struct NoAllocPlan {  // launch parameters of the setup kernel
  int n_robots, n_problems, n_configs;
  DevRobot robots[NA_MAX_ROBOTS];
  PairSchedule32 scheds[NA_MAX_ROBOTS];
  int prob[NA_MAX_PROBLEMS];    // robot << 24 | horizon
  int tstart[NA_MAX_PROBLEMS];  // first sweep item of the problem, in cost order
  int pstart[NA_MAX_PROBLEMS];  // first pair item of the problem, in cost order
};
struct NoAllocTables {
  DevRobot* robots;
  PairSchedule32* scheds;
  BatchProblemDev* probs;
  int4* titems;
  int2* pitems;
  int* counters;
};
__host__ __device__ NoAllocTables noalloc_tables(unsigned char* base);
cudaError_t noalloc_scratch(int device, unsigned char** out);
cudaError_t launch_noalloc_setup(const NoAllocPlan& plan, unsigned char* base, int grid,
                                 cudaStream_t s);
cudaError_t batch_tree_max_blocks_per_sm(bool fwd, int ns_max, int threads, int* out);
int pair_plan_words(const DevRobot& r);

// launchers (return cudaGetLastError())
// link Jacobians and the centre of mass (k_kin.cu)
constexpr int KIN_MAX_TARGETS = 64;
struct KinArgs {
  int64_t B;
  const float* pose;  // [B][n][12]
  int nt;
  int targets[KIN_MAX_TARGETS];
  float* jac;         // [B][nt][6][d] or nullptr
  float* com;         // [B][3] or nullptr
  float* jac_com;     // [B][3][d] or nullptr
};
cudaError_t launch_kin(const DevRobot& r, const KinArgs& a, int grid, int warps, cudaStream_t s);
cudaError_t kin_max_blocks_per_sm(const DevRobot& r, int warps, int* out);
size_t kin_smem_per_warp(const DevRobot& r);

// all-pairs summed collision hinge (k_hinge.cu)
struct HingeArgs {
  int64_t B;
  const float* pose;  // [B][n][12]
  float eta, w;       // activation distance, weight
  float* cost;        // [B] or nullptr
  float* g_sph;       // [B][S][3] or nullptr
};
size_t hinge_smem_per_warp(const DevRobot& r);
size_t hinge_smem_fixed(const DevRobot& r);  // per block, besides the warps' workspaces
cudaError_t launch_hinge(const DevRobot& r, const PairSchedule32& ps, const HingeArgs& a,
                         int grid, int warps, cudaStream_t s);
cudaError_t hinge_max_blocks_per_sm(const DevRobot& r, int warps, int* out);

// trajectory-optimisation ends (k_traj.cu)
cudaError_t launch_bspline_fwd(int64_t n_traj, int d, int K, int T, float dt, const float* U,
                               const float* start, int end_static, float* q, float* qd,
                               float* qdd, cudaStream_t s);
size_t bspline_bwd_smem(int Kx, int T);
cudaError_t launch_bspline_bwd(int64_t n_traj, int d, int K, int T, float dt, int has_start,
                               int end_static, const float* gq, const float* gqd,
                               const float* gqdd, const float* gqd2, const float* gqdd2,
                               float* gU, float* gstart, cudaStream_t s);
cudaError_t launch_trajopt_cost(int64_t B, int d, const float* tau, const float* d_min,
                                const float* qd, const float* qdd, const float* lo,
                                const float* hi, float w, float smooth, float length, float e,
                                float* cost, float* g_tau, float* g_dmin, float* g_qd,
                                float* g_qdd, cudaStream_t s);

// segments: 1 = one thread per configuration; 2, 4, 8 = segmented sweep
// (requires the robot's plan for it, bit log2(segments) - 1 of seg_ok).
// threads: threads per block, a multiple of 32, at most 256 for one segment
// and 512 for a segmented sweep (its launch bounds); every sweep block also
// stages the robot's link parameters in shared memory
cudaError_t launch_tree_fwd(const DevRobot& r, const FwdArgs& a, int threads, int segments,
                            cudaStream_t s);
cudaError_t launch_tree_bwd(const DevRobot& r, const BwdArgs& a, int threads, int segments,
                            cudaStream_t s, const FusedCost* fc = nullptr);
// the sweeps with the joint states evaluated from control points
cudaError_t launch_tree_fwd_spline(const DevRobot& r, const FwdArgs& a, const SplineArgs& sp,
                                   int threads, int segments, cudaStream_t s);
cudaError_t launch_tree_bwd_spline_cost(const DevRobot& r, const BwdArgs& a, const FusedCost& fc,
                                        const SplineArgs& sp, int threads, int segments,
                                        cudaStream_t s);
size_t tree_seg_smem(const DevRobot& r, int segments, int threads, bool fwd, bool cost = false);
// the backward's per-thread gradient-row slots of a segmented block
size_t grad_slot_smem(int segments, int threads);
// shared-memory carveout hint: the smallest that holds every block of `threads`
// threads and `smem` dynamic bytes one SM can keep, leaving the rest to L1
void fit_carveout(const void* kern, int threads, size_t smem);
int tree_max_depth();
size_t pair_smem(const DevRobot& r, int warps, bool bits);
size_t pair_block_smem(const DevRobot& r, int warps, bool bits);  // the same, out of line
cudaError_t launch_pair(const DevRobot& r, const PairSchedule32& ps, const FwdArgs& a, int grid,
                        int warps, cudaStream_t s, bool cull = true);
cudaError_t pair_max_blocks_per_sm(const DevRobot& r, int warps, bool bits, int* out);
cudaError_t launch_plain_fwd(const DevRobot& r, const FwdArgs& a, int threads, cudaStream_t s);
cudaError_t launch_plain_bwd(const DevRobot& r, const BwdArgs& a, int threads, cudaStream_t s);

size_t fused_fwd_smem_per_config(const DevRobot& r, int G, bool bits);
size_t fused_bwd_smem_per_config(const DevRobot& r, int G);
size_t fused_cta_smem(const DevRobot& r);  // robot metadata cached per CTA
cudaError_t launch_fused_fwd(const DevRobot& r, const PairSchedule& ps, const FwdArgs& a,
                             const FusedShape& sh, cudaStream_t s);
cudaError_t launch_fused_bwd(const DevRobot& r, const BwdArgs& a, const FusedShape& sh,
                             cudaStream_t s);
cudaError_t fused_fwd_max_blocks_per_sm(int G, int cpb, size_t smem, int* out);
cudaError_t fused_bwd_max_blocks_per_sm(int G, int cpb, size_t smem, int* out);

}  // namespace wbe
