// k_batch.cu -- uneven batches: many problems (robot, horizon) of different
// robots evaluated by one persistent launch per pass.
//
// Each problem p owns a contiguous slice of packed arrays: joint-major
// [d_p][H_p] blocks for q, qd, qdd, tau and their gradients (offset jo_p),
// [H_p][n_p][12] link poses (po_p), [H_p][S_p][3] sphere centres (so_p) and
// [H_p] d_min / worst pair (co_p).  The host cuts the problems into work
// items and sorts them by cost, longest first; warps of a persistent grid
// pull items through an atomic counter (a 4-byte scratch word per pass,
// cleared on the stream before the launch) until the list is exhausted, and
// each item runs the single-robot per-configuration code (tree_sweep.cuh,
// pair_body.cuh) with its own robot's descriptor.  There are no waits on
// other blocks: a warp that finds the list exhausted returns.
#include "pair_body.cuh"
#include "tree_sweep.cuh"

namespace wbe {

__device__ __forceinline__ int warp_pull(int* counter, int lane) {
  int it = 0;
  if (lane == 0) it = atomicAdd(counter, 1);
  return __shfl_sync(0xffffffffu, it, 0);
}

// tree items: x = problem, y = first configuration, z = count (<= 32)
__global__ void __launch_bounds__(128) batch_tree_fwd_kernel(const DevRobot* robots,
                                                             const BatchProblemDev* probs,
                                                             const int4* items, int n_items,
                                                             int* counter, BatchIO io) {
  const int lane = threadIdx.x & 31;
  for (;;) {
    const int it = warp_pull(counter, lane);
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
    if (lane < w.z) tree_fwd_one(r, A, (int64_t)w.y + lane);
  }
}

// capped at 128 registers, as the single-robot backward sweeps
__global__ void __launch_bounds__(128, 4) batch_tree_bwd_kernel(const DevRobot* robots,
                                                             const BatchProblemDev* probs,
                                                             const int4* items, int n_items,
                                                             int* counter, BatchIO io) {
  const int lane = threadIdx.x & 31;
  for (;;) {
    const int it = warp_pull(counter, lane);
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
    if (lane < w.z) tree_bwd_one(r, A, (int64_t)w.y + lane);
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
cudaError_t launch_batch_tree_fwd(const DevRobot* robots, const BatchProblemDev* probs, const int4* items,
                                  int n_items, int* counter, const BatchIO& io, int grid,
                                  cudaStream_t s) {
  cudaError_t e = cudaMemsetAsync(counter, 0, sizeof(int), s);
  if (e != cudaSuccess) return e;
  batch_tree_fwd_kernel<<<grid, 128, 0, s>>>(
      robots, probs, items, n_items, counter, io);
  return cudaGetLastError();
}

cudaError_t launch_batch_tree_bwd(const DevRobot* robots, const BatchProblemDev* probs, const int4* items,
                                  int n_items, int* counter, const BatchIO& io, int grid,
                                  cudaStream_t s) {
  cudaError_t e = cudaMemsetAsync(counter, 0, sizeof(int), s);
  if (e != cudaSuccess) return e;
  batch_tree_bwd_kernel<<<grid, 128, 0, s>>>(
      robots, probs, items, n_items, counter, io);
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

cudaError_t batch_tree_max_blocks_per_sm(bool fwd, int* out) {
  return fwd ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(out, batch_tree_fwd_kernel, 128, 0)
             : cudaOccupancyMaxActiveBlocksPerMultiprocessor(out, batch_tree_bwd_kernel, 128, 0);
}

int pair_plan_words(const DevRobot& r) { return PairPlan(r.n, r.Sg, r.P, false).total; }

}  // namespace wbe
