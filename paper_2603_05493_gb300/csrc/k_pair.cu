// k_pair.cu -- the single-robot pair kernel: one warp per configuration,
// persistent grid; the per-configuration work is pair_one_culled (default)
// or the full map-reduce pair_one (pair_body.cuh).
#include "pair_body.cuh"

namespace wbe {

template <bool FULL, bool BITS, bool CULL>
__global__ void __launch_bounds__(256, 3) pair_kernel(DevRobot r, PairSchedule32 ps, FwdArgs A) {
  extern __shared__ __align__(128) float smem[];
  const PairPlan pl(r.n, r.Sg, r.P, BITS);
  float4* radw = reinterpret_cast<float4*>(smem);
  for (int i = threadIdx.x; i < r.Sg; i += blockDim.x) radw[i] = __ldg(r.grp_rad + i);
  __syncthreads();
  const int lane = threadIdx.x & 31;
  const int warp = threadIdx.x >> 5;
  const int wpb = blockDim.x >> 5;
  float* ws = smem + a32(4 * r.Sg) + warp * pl.total;
  for (int64_t b = (int64_t)blockIdx.x * wpb + warp; b < A.B; b += (int64_t)gridDim.x * wpb)
    if (CULL)
      pair_one_culled<FULL, BITS>(r, ps, A, b, ws, radw, lane);
    else
      pair_one<FULL, BITS>(r, ps, A, b, ws, radw, lane);
}

template <bool FULL, bool BITS, bool CULL>
static cudaError_t pair_launch_t(const DevRobot& r, const PairSchedule32& ps, const FwdArgs& a,
                                 int grid, int warps, size_t smem, cudaStream_t s, int* occ) {
  auto kern = pair_kernel<FULL, BITS, CULL>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)smem);
  if (e != cudaSuccess) return e;
  if (occ) return cudaOccupancyMaxActiveBlocksPerMultiprocessor(occ, kern, warps * 32, smem);
  kern<<<grid, warps * 32, smem, s>>>(r, ps, a);
  return cudaGetLastError();
}

template <bool CULL>
static cudaError_t pair_dispatch_t(const DevRobot& r, const PairSchedule32& ps, const FwdArgs& a,
                                   int grid, int warps, cudaStream_t s, int* occ) {
  const bool bits = a.bits != nullptr;
  const size_t smem = pair_smem(r, warps, bits);
  if (r.all_full) {
    return bits ? pair_launch_t<true, true, CULL>(r, ps, a, grid, warps, smem, s, occ)
                : pair_launch_t<true, false, CULL>(r, ps, a, grid, warps, smem, s, occ);
  }
  return bits ? pair_launch_t<false, true, CULL>(r, ps, a, grid, warps, smem, s, occ)
              : pair_launch_t<false, false, CULL>(r, ps, a, grid, warps, smem, s, occ);
}

static cudaError_t pair_dispatch(const DevRobot& r, const PairSchedule32& ps, const FwdArgs& a,
                                 int grid, int warps, cudaStream_t s, int* occ, bool cull) {
  return cull ? pair_dispatch_t<true>(r, ps, a, grid, warps, s, occ)
              : pair_dispatch_t<false>(r, ps, a, grid, warps, s, occ);
}

cudaError_t launch_pair(const DevRobot& r, const PairSchedule32& ps, const FwdArgs& a, int grid,
                        int warps, cudaStream_t s, bool cull) {
  return pair_dispatch(r, ps, a, grid, warps, s, nullptr, cull);
}

size_t pair_block_smem(const DevRobot& r, int warps, bool bits) { return pair_smem(r, warps, bits); }

cudaError_t pair_max_blocks_per_sm(const DevRobot& r, int warps, bool bits, int* out) {
  FwdArgs a{};
  a.bits = bits ? reinterpret_cast<uint32_t*>(16) : nullptr;  // only selects the variant
  return pair_dispatch(r, PairSchedule32{}, a, 0, warps, nullptr, out, true);
}

}  // namespace wbe
