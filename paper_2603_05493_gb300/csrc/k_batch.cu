// k_batch.cu -- uneven batches: many problems (robot, horizon) of different
// robots evaluated by one persistent launch per pass.
//
// Each problem p owns a contiguous slice of packed arrays: joint-major
// [d_p][H_p] blocks for q, qd, qdd, tau and their gradients (offset jo_p),
// [H_p][n_p][12] link poses (po_p), [H_p][S_p][3] sphere centres (so_p) and
// [H_p] d_min / worst pair (co_p).  The host cuts the problems into work
// items and sorts them by cost, longest first; warps (pairs of warps for the
// sweeps) of a persistent grid pull items through an atomic counter (a
// 4-byte scratch word per pass, cleared on the stream before the launch)
// until the list is exhausted, and each item runs the single-robot
// per-configuration code (tree_sweep.cuh, pair_body.cuh) with its own
// robot's descriptor.  There are no waits on other blocks: a warp (pair)
// that finds the list exhausted returns.
#include "pair_body.cuh"
#include "tree_sweep.cuh"

namespace wbe {

__device__ __forceinline__ int warp_pull(int* counter, int lane) {
  int it = 0;
  if (lane == 0) it = atomicAdd(counter, 1);
  return __shfl_sync(0xffffffffu, it, 0);
}

// Tree items (x = problem, y = first configuration, z = count, w = mode) are
// taken by pairs of warps; a block holds blockDim.x / 64 pairs (1, 2 or 4,
// chosen by the batch's tune).  Mode 0 (z <= 32): the two warps of the pair
// sweep the two segments of the item's robot's 2-segment plan (the
// segmented sweeps of tree_sweep.cuh: warp g replays the ancestors of its
// first link, then sweeps its links); the outputs of links both segments
// hold go to the pair's shared-memory partials and are summed in segment
// order after the pair's barrier.  A robot without a 2-segment plan (a joint
// driving several links) is swept whole by the pair's first warp in mode 0.
// Mode 1 (z <= 64): each warp sweeps its own 32 configurations of the item
// whole (warp g takes configurations y + 32 g ...), the one-segment choice.
// The mode is per robot (the batch's tune).  The pair shares the pulled item
// through shared memory; its barriers are named barriers of 64 threads, and
// both warps leave the loop on the same item.
__device__ __forceinline__ void pair_bar(int id) {
  asm volatile("bar.sync %0, 64;" ::"r"(id) : "memory");
}

// shared memory: one item slot per pair (32 words, up to 32 pairs), then per
// pair the partials [nout][ns_max][2][32]
__host__ __device__ inline size_t batch_tree_words(int nout, int ns_max, int pairs) {
  return 32 + (size_t)pairs * nout * ns_max * 64;
}

// the configuration a lane sweeps in item w, and whether it sweeps one:
// mode 0 -- lane of the 32; the second warp only with a segment plan;
// mode 1 -- configuration 32 g + lane of the 64
__device__ __forceinline__ bool batch_lane(const int4& w, bool seg, int g, int lane, int64_t* b) {
  if (w.w == 1) {
    *b = (int64_t)w.y + 32 * g + lane;
    return 32 * g + lane < w.z;
  }
  *b = (int64_t)w.y + lane;
  return (seg || g == 0) && lane < w.z;
}

__global__ void __launch_bounds__(256) batch_tree_fwd_kernel(const DevRobot* robots,
                                                             const BatchProblemDev* probs,
                                                             const int4* items, int n_items,
                                                             int* counter, BatchIO io,
                                                             int ns_max) {
  extern __shared__ float sm[];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int pi = warp >> 1, g = warp & 1, bar = 1 + pi;
  int* slot = reinterpret_cast<int*>(sm) + pi;
  float* part = sm + 32 + (size_t)pi * ns_max * 64;
  for (;;) {
    if (g == 0 && lane == 0) *slot = atomicAdd(counter, 1);
    pair_bar(bar);
    const int it = *slot;
    if (it >= n_items) return;
    const int4 w = items[it];
    const BatchProblemDev pb = probs[w.x];
    const DevRobot& r = robots[pb.robot];
    FwdArgs A{pb.H,
              io.q + pb.jo,
              io.qd ? io.qd + pb.jo : nullptr,
              io.qdd ? io.qdd + pb.jo : nullptr,
              io.pose ? io.pose + pb.po : nullptr,
              nullptr,
              nullptr,
              nullptr,
              io.tau ? io.tau + pb.jo : nullptr,
              nullptr};
    const bool seg = w.w == 0 && (r.seg_ok & 1);
    int64_t b;
    const bool act = batch_lane(w, seg, g, lane, &b);
    const int ns = seg ? r.seg_ns[0] : 0;
    // one call site for both cases (a second inlined sweep would cost registers)
    const Seg sg = seg ? Seg{r.seg_pos[0][g], r.seg_pos[0][g + 1], g, 2, r.seg_slot, part, ns, lane}
                       : whole_sweep(r);
    for (int q = 0; q < ns; ++q) part[(q * 2 + g) * 32 + lane] = 0.0f;
    if (act) tree_fwd_seg(r, A, ArrayStates{A.q, A.qd, A.qdd, A.B, b}, b, sg);
    pair_bar(bar);
    if (lane < w.z && A.tau)
      for (int q = g; q < ns; q += 2) {
        const float acc = part[(q * 2) * 32 + lane] + part[(q * 2 + 1) * 32 + lane];
        A.tau[(int64_t)__ldg(r.jidx + __ldg(r.seg_slot_link + q)) * A.B + b] = acc;
      }
    pair_bar(bar);  // the slot and the partials are free again
  }
}

// capped at 128 registers, as the single-robot backward sweeps
__global__ void __launch_bounds__(256, 2) batch_tree_bwd_kernel(const DevRobot* robots,
                                                             const BatchProblemDev* probs,
                                                             const int4* items, int n_items,
                                                             int* counter, BatchIO io,
                                                             int ns_max) {
  extern __shared__ float sm[];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int pi = warp >> 1, g = warp & 1, bar = 1 + pi;
  int* slot = reinterpret_cast<int*>(sm) + pi;
  float* part = sm + 32 + (size_t)pi * 3 * ns_max * 64;
  // the gradient-row slots behind every pair's partials
  const GradSlot gs = grad_slot_of(sm + batch_tree_words(3, ns_max, blockDim.x / 64));
  for (;;) {
    if (g == 0 && lane == 0) *slot = atomicAdd(counter, 1);
    pair_bar(bar);
    const int it = *slot;
    if (it >= n_items) return;
    const int4 w = items[it];
    const BatchProblemDev pb = probs[w.x];
    const DevRobot& r = robots[pb.robot];
    BwdArgs A{pb.H,
              io.q + pb.jo,
              io.qd + pb.jo,
              io.qdd + pb.jo,
              io.worst ? io.worst + pb.co : nullptr,
              io.g_pose ? io.g_pose + pb.po : nullptr,
              io.g_sph ? io.g_sph + pb.so : nullptr,
              io.g_dmin ? io.g_dmin + pb.co : nullptr,
              io.g_tau ? io.g_tau + pb.jo : nullptr,
              io.gq + pb.jo,
              io.gqd + pb.jo,
              io.gqdd + pb.jo};
    const bool seg = w.w == 0 && (r.seg_ok & 1);
    int64_t b;
    const bool act = batch_lane(w, seg, g, lane, &b);
    const int ns = seg ? r.seg_ns[0] : 0;
    const size_t o = (size_t)ns * 64;  // one output's partials
    const Seg sg = seg ? Seg{r.seg_pos[0][g], r.seg_pos[0][g + 1], g, 2, r.seg_slot, part, ns, lane}
                       : whole_sweep(r);
    for (int q = 0; q < ns; ++q)
      for (int k = 0; k < 3; ++k) part[k * o + (q * 2 + g) * 32 + lane] = 0.0f;
    if (act) tree_bwd_seg<false>(r, A, FusedCost{}, ArrayStates{A.q, A.qd, A.qdd, A.B, b}, b, sg, gs);
    pair_bar(bar);
    if (lane < w.z)
      for (int q = g; q < ns; q += 2) {
        float acc[3];
        for (int k = 0; k < 3; ++k)
          acc[k] = part[k * o + (q * 2) * 32 + lane] + part[k * o + (q * 2 + 1) * 32 + lane];
        const int64_t at = (int64_t)__ldg(r.jidx + __ldg(r.seg_slot_link + q)) * A.B + b;
        A.gq[at] = acc[0];
        A.gqd[at] = acc[1];
        A.gqdd[at] = acc[2];
      }
    pair_bar(bar);  // the slot and the partials are free again
  }
}

// pair items: x = problem, y = configuration
__global__ void __launch_bounds__(256, 3) batch_pair_kernel(const DevRobot* robots,
                                                            const PairSchedule32* scheds,
                                                            const BatchProblemDev* probs,
                                                            const int2* items, int n_items,
                                                            int* counter, BatchIO io,
                                                            int ws_words, int rad_words) {
  extern __shared__ __align__(128) float smem[];
  const int lane = threadIdx.x & 31;
  const int warp = threadIdx.x >> 5;
  float4* radw = reinterpret_cast<float4*>(smem + (size_t)warp * (ws_words + rad_words));
  float* ws = smem + (size_t)warp * (ws_words + rad_words) + rad_words;
  int cur_robot = -1;
  for (;;) {
    const int it = warp_pull(counter, lane);
    if (it >= n_items) return;
    const int2 w = items[it];
    const BatchProblemDev pb = probs[w.x];
    const DevRobot& r = robots[pb.robot];
    if (pb.robot != cur_robot) {  // this warp's radius table follows its robot
      __syncwarp();
      for (int i = lane; i < r.Sg; i += 32) radw[i] = __ldg(r.grp_rad + i);
      cur_robot = pb.robot;
      __syncwarp();
    }
    FwdArgs A{pb.H,   nullptr, nullptr, nullptr, io.pose + pb.po,
              io.sph ? io.sph + pb.so : nullptr,
              io.dmin ? io.dmin + pb.co : nullptr,
              io.worst ? io.worst + pb.co : nullptr,
              nullptr, nullptr};
    if (r.all_full)
      pair_one_culled<true, false>(r, scheds[pb.robot], A, w.y, ws, radw, lane);
    else
      pair_one_culled<false, false>(r, scheds[pb.robot], A, w.y, ws, radw, lane);
  }
}

// ---------------------------------------------------------------------------
// launchers
// ---------------------------------------------------------------------------
// the backward adds each thread's gradient-row slot (GradSlot)
size_t batch_tree_smem(bool fwd, int ns_max, int threads) {
  return sizeof(float) * batch_tree_words(fwd ? 1 : 3, ns_max, threads / 64) +
         (fwd ? 0 : 16 + (size_t)kGradSlotBytes * threads);
}

cudaError_t launch_batch_tree_fwd(const DevRobot* robots, const BatchProblemDev* probs, const int4* items,
                                  int n_items, int* counter, const BatchIO& io, int grid,
                                  int ns_max, int threads, cudaStream_t s) {
  const size_t smem = batch_tree_smem(true, ns_max, threads);
  cudaError_t e = cudaFuncSetAttribute(batch_tree_fwd_kernel,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  fit_carveout((const void*)batch_tree_fwd_kernel, threads, smem);
  e = cudaMemsetAsync(counter, 0, sizeof(int), s);
  if (e != cudaSuccess) return e;
  batch_tree_fwd_kernel<<<grid, threads, smem, s>>>(robots, probs, items, n_items, counter, io,
                                                    ns_max);
  return cudaGetLastError();
}

cudaError_t launch_batch_tree_bwd(const DevRobot* robots, const BatchProblemDev* probs, const int4* items,
                                  int n_items, int* counter, const BatchIO& io, int grid,
                                  int ns_max, int threads, cudaStream_t s) {
  const size_t smem = batch_tree_smem(false, ns_max, threads);
  cudaError_t e = cudaFuncSetAttribute(batch_tree_bwd_kernel,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  fit_carveout((const void*)batch_tree_bwd_kernel, threads, smem);
  e = cudaMemsetAsync(counter, 0, sizeof(int), s);
  if (e != cudaSuccess) return e;
  batch_tree_bwd_kernel<<<grid, threads, smem, s>>>(robots, probs, items, n_items, counter, io,
                                                    ns_max);
  return cudaGetLastError();
}

size_t batch_pair_smem(int ws_words, int rad_words, int warps) {
  return sizeof(float) * (size_t)warps * (ws_words + rad_words);
}

cudaError_t launch_batch_pair(const DevRobot* robots, const PairSchedule32* scheds,
                              const BatchProblemDev* probs, const int2* items, int n_items, int* counter,
                              const BatchIO& io, int grid, int warps, int ws_words,
                              int rad_words, cudaStream_t s) {
  const size_t smem = batch_pair_smem(ws_words, rad_words, warps);
  cudaError_t e = cudaFuncSetAttribute(batch_pair_kernel,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  e = cudaMemsetAsync(counter, 0, sizeof(int), s);
  if (e != cudaSuccess) return e;
  batch_pair_kernel<<<grid, warps * 32, smem, s>>>(robots, scheds,
                                                  probs,
                                                  items, n_items, counter, io, ws_words,
                                                  rad_words);
  return cudaGetLastError();
}

cudaError_t batch_pair_max_blocks_per_sm(int warps, int ws_words, int rad_words, int* out) {
  const size_t smem = batch_pair_smem(ws_words, rad_words, warps);
  cudaError_t e = cudaFuncSetAttribute(batch_pair_kernel,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  return cudaOccupancyMaxActiveBlocksPerMultiprocessor(out, batch_pair_kernel, warps * 32, smem);
}

cudaError_t batch_tree_max_blocks_per_sm(bool fwd, int ns_max, int threads, int* out) {
  const size_t smem = batch_tree_smem(fwd, ns_max, threads);
  cudaError_t e = cudaFuncSetAttribute(fwd ? batch_tree_fwd_kernel : batch_tree_bwd_kernel,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  return fwd ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(out, batch_tree_fwd_kernel, threads,
                                                             smem)
             : cudaOccupancyMaxActiveBlocksPerMultiprocessor(out, batch_tree_bwd_kernel, threads,
                                                             smem);
}

int pair_plan_words(const DevRobot& r) { return PairPlan(r.n, r.Sg, r.P, false).total; }

}  // namespace wbe
