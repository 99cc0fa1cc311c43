// k_tree.cu -- the single-robot depth-first sweep kernels (tree_sweep.cuh):
// one thread per configuration of a batch of B.
#include "tree_sweep.cuh"

namespace wbe {

__global__ void __launch_bounds__(256) tree_fwd_kernel(DevRobot r, FwdArgs A) {
  const int64_t b = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (b < A.B) tree_fwd_one(r, A, b);
}

__global__ void __launch_bounds__(256) tree_bwd_kernel(DevRobot r, BwdArgs A) {
  const int64_t b = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (b < A.B) tree_bwd_one(r, A, b);
}

// The sweep kernels use no shared memory: give the whole unified L1/shared
// array to L1, where the stacks live.
static void prefer_l1() {
  static bool done = false;
  if (!done) {
    cudaFuncSetAttribute(tree_fwd_kernel, cudaFuncAttributePreferredSharedMemoryCarveout, 0);
    cudaFuncSetAttribute(tree_bwd_kernel, cudaFuncAttributePreferredSharedMemoryCarveout, 0);
    done = true;
  }
}

cudaError_t launch_tree_fwd(const DevRobot& r, const FwdArgs& a, int threads, cudaStream_t s) {
  prefer_l1();
  if (threads <= 0) threads = 128;
  const int64_t grid = (a.B + threads - 1) / threads;
  tree_fwd_kernel<<<(unsigned)grid, threads, 0, s>>>(r, a);
  return cudaGetLastError();
}

cudaError_t launch_tree_bwd(const DevRobot& r, const BwdArgs& a, int threads, cudaStream_t s) {
  prefer_l1();
  if (threads <= 0) threads = 128;
  const int64_t grid = (a.B + threads - 1) / threads;
  tree_bwd_kernel<<<(unsigned)grid, threads, 0, s>>>(r, a);
  return cudaGetLastError();
}

int tree_max_depth() { return TMAXD; }

}  // namespace wbe
