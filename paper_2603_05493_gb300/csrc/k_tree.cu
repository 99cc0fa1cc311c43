// k_tree.cu -- the single-robot depth-first sweep kernels (tree_sweep.cuh):
// one thread per configuration of a batch of B, or G warps per 32
// configurations (segmented sweep).
#include "tree_sweep.cuh"

#include <algorithm>
#include <mutex>

namespace wbe {

// The sweeps read a link's fixed transform, axis, mimic factors and inertia
// at its push (and the backward again at its close).  Every sweep kernel
// stages these once per block in shared memory (kParamWords floats a link,
// behind the partials or basis rows it also keeps there), where they no
// longer compete with the depth-first stacks for L1.
constexpr int kParamWords = 28;  // Tf 12, axis 4, inertia 10, mimic 2
constexpr size_t kSegSmemMax = 227 * 1024;  // dynamic shared memory of one block
__device__ __forceinline__ DevRobot stage_params(const DevRobot& r, float* dst) {
  const int n = r.n;
  for (int i = threadIdx.x; i < 12 * n; i += blockDim.x) dst[i] = __ldg(r.Tf + i);
  for (int i = threadIdx.x; i < 4 * n; i += blockDim.x) dst[12 * n + i] = __ldg(r.axis + i);
  for (int i = threadIdx.x; i < 10 * n; i += blockDim.x) dst[16 * n + i] = __ldg(r.inert + i);
  for (int i = threadIdx.x; i < 2 * n; i += blockDim.x) dst[26 * n + i] = __ldg(r.mimic + i);
  DevRobot s = r;
  s.Tf = dst;
  s.axis = dst + 12 * n;
  s.inert = dst + 16 * n;
  s.mimic = dst + 26 * n;
  return s;
}

// the block's dynamic shared memory covers `words` floats
__device__ __forceinline__ bool smem_holds(size_t words) {
  unsigned dyn;
  asm("mov.u32 %0, %%dynamic_smem_size;" : "=r"(dyn));
  return sizeof(float) * words <= dyn;
}

// FS: the force stack in shared memory behind the link parameters, as in the
// segmented forward below
template <bool FS>
__global__ void __launch_bounds__(256) tree_fwd_kernel(const __grid_constant__ DevRobot r,
                                                       FwdArgs A) {
  extern __shared__ float prm[];
  if (FS && !smem_holds(kParamWords * (size_t)r.n + 6 * (size_t)r.maxdepth * blockDim.x)) return;
  const DevRobot rs = stage_params(r, prm);
  __syncthreads();
  const int64_t b = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (b >= A.B) return;
  Seg sg = whole_sweep(r);
  if (FS) {
    sg.fst = prm + kParamWords * (size_t)r.n + threadIdx.x;
    sg.fstr = blockDim.x;
  }
  tree_fwd_seg<ArrayStates, FS>(rs, A, ArrayStates{A.q, A.qd, A.qdd, A.B, b}, b, sg);
}

// The backward sweeps are capped at 128 registers (two 256-thread blocks per
// SM, or one 512-thread block of a segmented sweep): with the register copies
// of the stack top they would take ~165, and the occupancy lost costs more
// than the few spills (measured on the 48-DoF humanoid: 0.29 ms capped vs
// 0.36 ms uncapped at 2 segments).  The segmented sweeps take blocks of up to
// 512 threads, so that one block per SM holds the staged link parameters once
// and the shared-memory carveout stays small.
__global__ void __launch_bounds__(256, 2) tree_bwd_kernel(const __grid_constant__ DevRobot r,
                                                          BwdArgs A) {
  extern __shared__ float prm[];
  const DevRobot rs = stage_params(r, prm);
  __syncthreads();
  const int64_t b = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (b < A.B) tree_bwd_one(rs, A, b);
}

// Segmented sweeps, plan t (G = 2 << t segments).  A block holds CG groups of
// G warps; warp w sweeps segment w % G of the 32 configurations of group
// w / G.  Shared memory per group: the partial outputs [nout][ns][G][32] of
// the ns links that several segments hold, summed in segment order after the
// barrier by the group's warps (slot s by warp s % G).
__device__ __forceinline__ Seg seg_of(const DevRobot& r, int t, float* part) {
  const int G = 2 << t;
  const int w = threadIdx.x >> 5;
  const int g = w % G;
  return Seg{r.seg_pos[t][g], r.seg_pos[t][g + 1], g, G, r.seg_slot + t * r.n,
             part, r.seg_ns[t], (int)(threadIdx.x & 31)};
}

// FS: the force stack in shared memory, [maxdepth][6][threads] floats behind
// the link parameters (a link's F is stored when its first child is pushed
// and read back at that child's close; in local memory these round trips
// missed L1 61 % of the time)
template <bool FS>
__global__ void __launch_bounds__(512) tree_fwd_seg_kernel(const __grid_constant__ DevRobot r,
                                                           FwdArgs A, int t) {
  extern __shared__ float part[];
  const int G = 2 << t;
  const int CG = blockDim.x / (32 * G);
  const int cg = (threadIdx.x >> 5) / G;
  const int ns = r.seg_ns[t];
  // the launch reserves the stack for this block's threads; a block that
  // finds less shared memory than that does nothing (its outputs stay
  // unwritten) instead of indexing past it
  if (FS && !smem_holds((size_t)CG * ns * G * 32 + kParamWords * (size_t)r.n +
                        6 * (size_t)r.maxdepth * blockDim.x))
    return;
  Seg sg = seg_of(r, t, part + (size_t)cg * ns * G * 32);
  for (int s = 0; s < ns; ++s) sg.part[(s * G + sg.g) * 32 + sg.lane] = 0.0f;
  const DevRobot rs = stage_params(r, part + (size_t)CG * ns * G * 32);
  if (FS) {
    sg.fst = part + (size_t)CG * ns * G * 32 + kParamWords * (size_t)r.n + threadIdx.x;
    sg.fstr = blockDim.x;
  }
  __syncthreads();
  const int64_t b = ((int64_t)blockIdx.x * CG + cg) * 32 + sg.lane;
  if (b < A.B) tree_fwd_seg<ArrayStates, FS>(rs, A, ArrayStates{A.q, A.qd, A.qdd, A.B, b}, b, sg);
  __syncthreads();
  if (b < A.B && A.tau) {
    for (int s = sg.g; s < ns; s += G) {
      float acc = 0.0f;
      for (int h = 0; h < G; ++h) acc += sg.part[(s * G + h) * 32 + sg.lane];
      const int k = __ldg(r.seg_slot_link + t * r.n + s);
      A.tau[(int64_t)__ldg(r.jidx + k) * A.B + b] = acc;
    }
  }
}

__global__ void __launch_bounds__(512, 1) tree_bwd_seg_kernel(const __grid_constant__ DevRobot r,
                                                           BwdArgs A, int t) {
  extern __shared__ float part[];
  const int G = 2 << t;
  const int CG = blockDim.x / (32 * G);
  const int cg = (threadIdx.x >> 5) / G;
  const int ns = r.seg_ns[t];
  const size_t o = (size_t)ns * G * 32;  // one output's partials
  Seg sg = seg_of(r, t, part + (size_t)cg * 3 * o);
  for (int s = 0; s < ns; ++s)
    for (int q = 0; q < 3; ++q) sg.part[q * o + (s * G + sg.g) * 32 + sg.lane] = 0.0f;
  const DevRobot rs = stage_params(r, part + (size_t)CG * 3 * o);
  // the gradient-row slots behind the link parameters (reserved by the
  // launch when there are upstream pose or sphere gradients)
  const GradSlot gs = grad_slot_of(part + (size_t)CG * 3 * o + kParamWords * (size_t)r.n);
  __syncthreads();
  const int64_t b = ((int64_t)blockIdx.x * CG + cg) * 32 + sg.lane;
  if (b < A.B) tree_bwd_seg<false>(rs, A, FusedCost{}, ArrayStates{A.q, A.qd, A.qdd, A.B, b}, b, sg, gs);
  __syncthreads();
  if (b < A.B) {
    for (int s = sg.g; s < ns; s += G) {
      float acc[3] = {0.0f, 0.0f, 0.0f};
      for (int h = 0; h < G; ++h)
        for (int q = 0; q < 3; ++q) acc[q] += sg.part[q * o + (s * G + h) * 32 + sg.lane];
      const int k = __ldg(r.seg_slot_link + t * r.n + s);
      const int64_t at = (int64_t)__ldg(r.jidx + k) * A.B + b;
      A.gq[at] = acc[0];
      A.gqd[at] = acc[1];
      A.gqdd[at] = acc[2];
    }
  }
}

// The same sweeps with the trajectory cost in their prologue (FusedCost):
// separate kernels, so that the plain ones keep their register allocation.
// The segmented one adds each configuration's cost terms over the segments
// in segment order (deterministic) after the barrier.
__global__ void __launch_bounds__(256, 2) tree_bwd_cost_kernel(
    const __grid_constant__ DevRobot r, BwdArgs A, FusedCost fc) {
  extern __shared__ float prm[];
  const DevRobot rs = stage_params(r, prm);
  __syncthreads();
  const int64_t b = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (b < A.B) tree_bwd_cost_one(rs, A, fc, ArrayStates{A.q, A.qd, A.qdd, A.B, b}, b);
}

__global__ void __launch_bounds__(512, 1) tree_bwd_cost_seg_kernel(
    const __grid_constant__ DevRobot r, BwdArgs A, FusedCost fc, int t) {
  extern __shared__ float part[];
  const int G = 2 << t;
  const int CG = blockDim.x / (32 * G);
  const int cg = (threadIdx.x >> 5) / G;
  const int ns = r.seg_ns[t];
  const size_t o = (size_t)ns * G * 32;  // one output's partials
  Seg sg = seg_of(r, t, part + (size_t)cg * (3 * o + G * 32));
  float* cpart = sg.part + 3 * o;  // [G][32] the segments' cost terms
  for (int s = 0; s < ns; ++s)
    for (int q = 0; q < 3; ++q) sg.part[q * o + (s * G + sg.g) * 32 + sg.lane] = 0.0f;
  const DevRobot rs = stage_params(r, part + (size_t)CG * (3 * o + G * 32));
  const GradSlot gs = grad_slot_of(part + (size_t)CG * (3 * o + G * 32) + kParamWords * (size_t)r.n);
  __syncthreads();
  const int64_t b = ((int64_t)blockIdx.x * CG + cg) * 32 + sg.lane;
  float c = 0.0f;
  if (b < A.B) c = tree_bwd_seg<true>(rs, A, fc, ArrayStates{A.q, A.qd, A.qdd, A.B, b}, b, sg, gs);
  cpart[sg.g * 32 + sg.lane] = c;
  __syncthreads();
  if (b < A.B && sg.g == 0 && fc.cost) {
    float acc = 0.0f;
    for (int h = 0; h < G; ++h) acc += cpart[h * 32 + sg.lane];
    fc.cost[b] = fc.d_min ? fmaf(fc.w, fmaxf(0.0f, -__ldg(fc.d_min + b)), acc) : acc;
  }
  if (b < A.B) {
    for (int s = sg.g; s < ns; s += G) {
      float acc[3] = {0.0f, 0.0f, 0.0f};
      for (int h = 0; h < G; ++h)
        for (int q = 0; q < 3; ++q) acc[q] += sg.part[q * o + (s * G + h) * 32 + sg.lane];
      const int k = __ldg(r.seg_slot_link + t * r.n + s);
      const int64_t at = (int64_t)__ldg(r.jidx + k) * A.B + b;
      A.gq[at] = acc[0];
      A.gqd[at] = acc[1];
      A.gqdd[at] = acc[2];
    }
  }
}

// The sweeps with the joint states evaluated from B-spline control points
// where they need them (SplineStates): no state arrays are read or written.
// Each thread keeps its sample's basis rows in shared memory, in front of the
// segments' partials.
__device__ __forceinline__ SplineStates spline_states(const DevRobot& r, const SplineArgs& sp,
                                                      int64_t b, float* bs) {
  const int64_t tr = b / sp.T;
  int k;
  float al;
  bs_sample((int)(b - tr * sp.T), sp.K, sp.T, k, al);
  float Bm[3][4];
  bs_basis(al, sp.dt, Bm);
#pragma unroll
  for (int q = 0; q < 3; ++q)
#pragma unroll
    for (int l = 0; l < 4; ++l) bs[4 * q + l] = Bm[q][l];
  return SplineStates{sp.U + (tr * r.d) * sp.K + k, sp.K, bs};
}

__global__ void __launch_bounds__(256) tree_fwd_spline_kernel(const __grid_constant__ DevRobot r,
                                                              FwdArgs A, SplineArgs sp) {
  extern __shared__ float sm[];
  const DevRobot rs = stage_params(r, sm + 12 * blockDim.x);
  __syncthreads();
  const int64_t b = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (b >= A.B) return;
  const SplineStates st = spline_states(r, sp, b, sm + 12 * threadIdx.x);
  tree_fwd_seg(rs, A, st, b, whole_sweep(r));
}

// FS as for tree_fwd_seg_kernel; the force stack follows the link parameters
template <bool FS>
__global__ void __launch_bounds__(512) tree_fwd_spline_seg_kernel(
    const __grid_constant__ DevRobot r, FwdArgs A, SplineArgs sp, int t) {
  extern __shared__ float sm[];
  float* part = sm + 12 * blockDim.x;
  const int G = 2 << t;
  const int CG = blockDim.x / (32 * G);
  const int cg = (threadIdx.x >> 5) / G;
  const int ns = r.seg_ns[t];
  if (FS && !smem_holds(12 * (size_t)blockDim.x + (size_t)CG * ns * G * 32 +
                        kParamWords * (size_t)r.n + 6 * (size_t)r.maxdepth * blockDim.x))
    return;
  Seg sg = seg_of(r, t, part + (size_t)cg * ns * G * 32);
  for (int s = 0; s < ns; ++s) sg.part[(s * G + sg.g) * 32 + sg.lane] = 0.0f;
  const DevRobot rs = stage_params(r, part + (size_t)CG * ns * G * 32);
  if (FS) {
    sg.fst = part + (size_t)CG * ns * G * 32 + kParamWords * (size_t)r.n + threadIdx.x;
    sg.fstr = blockDim.x;
  }
  __syncthreads();
  const int64_t b = ((int64_t)blockIdx.x * CG + cg) * 32 + sg.lane;
  if (b < A.B)
    tree_fwd_seg<SplineStates, FS>(rs, A, spline_states(r, sp, b, sm + 12 * threadIdx.x), b, sg);
  __syncthreads();
  if (b < A.B && A.tau) {
    for (int s = sg.g; s < ns; s += G) {
      float acc = 0.0f;
      for (int h = 0; h < G; ++h) acc += sg.part[(s * G + h) * 32 + sg.lane];
      const int k = __ldg(r.seg_slot_link + t * r.n + s);
      A.tau[(int64_t)__ldg(r.jidx + k) * A.B + b] = acc;
    }
  }
}

__global__ void __launch_bounds__(256, 2) tree_bwd_spline_cost_kernel(
    const __grid_constant__ DevRobot r, BwdArgs A, FusedCost fc, SplineArgs sp) {
  extern __shared__ float sm[];
  const DevRobot rs = stage_params(r, sm + 12 * blockDim.x);
  __syncthreads();
  const int64_t b = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (b >= A.B) return;
  tree_bwd_cost_one(rs, A, fc, spline_states(r, sp, b, sm + 12 * threadIdx.x), b);
}

__global__ void __launch_bounds__(512, 1) tree_bwd_spline_cost_seg_kernel(
    const __grid_constant__ DevRobot r, BwdArgs A, FusedCost fc, SplineArgs sp, int t) {
  extern __shared__ float sm[];
  float* base = sm + 12 * blockDim.x;
  const int G = 2 << t;
  const int CG = blockDim.x / (32 * G);
  const int cg = (threadIdx.x >> 5) / G;
  const int ns = r.seg_ns[t];
  const size_t o = (size_t)ns * G * 32;  // one output's partials
  Seg sg = seg_of(r, t, base + (size_t)cg * (3 * o + G * 32));
  float* cpart = sg.part + 3 * o;  // [G][32] the segments' cost terms
  for (int s = 0; s < ns; ++s)
    for (int q = 0; q < 3; ++q) sg.part[q * o + (s * G + sg.g) * 32 + sg.lane] = 0.0f;
  const DevRobot rs = stage_params(r, base + (size_t)CG * (3 * o + G * 32));
  __syncthreads();
  const int64_t b = ((int64_t)blockIdx.x * CG + cg) * 32 + sg.lane;
  float c = 0.0f;
  if (b < A.B)
    c = tree_bwd_seg<true>(rs, A, fc, spline_states(r, sp, b, sm + 12 * threadIdx.x), b, sg);
  cpart[sg.g * 32 + sg.lane] = c;
  __syncthreads();
  if (b < A.B && sg.g == 0 && fc.cost) {
    float acc = 0.0f;
    for (int h = 0; h < G; ++h) acc += cpart[h * 32 + sg.lane];
    fc.cost[b] = fc.d_min ? fmaf(fc.w, fmaxf(0.0f, -__ldg(fc.d_min + b)), acc) : acc;
  }
  if (b < A.B) {
    for (int s = sg.g; s < ns; s += G) {
      float acc[3] = {0.0f, 0.0f, 0.0f};
      for (int h = 0; h < G; ++h)
        for (int q = 0; q < 3; ++q) acc[q] += sg.part[q * o + (s * G + h) * 32 + sg.lane];
      const int k = __ldg(r.seg_slot_link + t * r.n + s);
      const int64_t at = (int64_t)__ldg(r.jidx + k) * A.B + b;
      A.gq[at] = acc[0];
      A.gqd[at] = acc[1];
      A.gqdd[at] = acc[2];
    }
  }
}

// Shared memory and L1 are one array per SM.  Without a preference the
// driver gave the segmented sweeps, whose blocks hold 14-22 KB of partials, a
// 132 KB shared carveout (measured), and the L1 that caches their depth-first
// stacks shrank to match.  fit_carveout asks for the smallest carveout that
// still holds every block the registers, warps and block limit let one SM
// keep (a hint: the driver rounds it up to a carveout it supports).
// the SM limits fit_carveout needs, queried once per device (host threads may
// launch on several devices at once)
struct SmLimits {
  int smem_sm, regs_sm, threads_sm, blocks_sm, reserved;
};
static bool sm_limits(int dev, SmLimits* out) {
  constexpr int kDevices = 64;
  static std::mutex mu;
  static SmLimits cache[kDevices];
  static bool have[kDevices] = {};
  auto query = [](int d, SmLimits* l) {
    return cudaDeviceGetAttribute(&l->regs_sm, cudaDevAttrMaxRegistersPerMultiprocessor, d) ==
               cudaSuccess &&
           cudaDeviceGetAttribute(&l->threads_sm, cudaDevAttrMaxThreadsPerMultiProcessor, d) ==
               cudaSuccess &&
           cudaDeviceGetAttribute(&l->blocks_sm, cudaDevAttrMaxBlocksPerMultiprocessor, d) ==
               cudaSuccess &&
           cudaDeviceGetAttribute(&l->reserved, cudaDevAttrReservedSharedMemoryPerBlock, d) ==
               cudaSuccess &&
           cudaDeviceGetAttribute(&l->smem_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, d) ==
               cudaSuccess;
  };
  if (dev < 0 || dev >= kDevices) return query(dev, out);
  std::lock_guard<std::mutex> lock(mu);
  if (!have[dev]) {
    if (!query(dev, &cache[dev])) return false;
    have[dev] = true;
  }
  *out = cache[dev];
  return true;
}

void fit_carveout(const void* kern, int threads, size_t smem) {
  int dev = 0;
  SmLimits L;
  if (cudaGetDevice(&dev) != cudaSuccess || !sm_limits(dev, &L)) {
    cudaGetLastError();
    return;
  }
  cudaFuncAttributes fa;
  if (cudaFuncGetAttributes(&fa, kern) != cudaSuccess) return;
  const int warps = (threads + 31) / 32;
  const int regs_warp = ((fa.numRegs * 32 + 255) / 256) * 256;  // 256-register allocation unit
  int nb = std::min(L.threads_sm / (32 * warps), L.blocks_sm);
  if (regs_warp > 0) nb = std::min(nb, (L.regs_sm / regs_warp) / warps);
  const size_t per = smem + fa.sharedSizeBytes + (size_t)L.reserved;
  nb = std::min<int>(nb, (int)((size_t)L.smem_sm / per));
  const size_t need = (size_t)std::max(nb, 1) * per;
  const int pct = (int)std::min<size_t>(100, (need * 100 + L.smem_sm - 1) / L.smem_sm);
  cudaFuncSetAttribute(kern, cudaFuncAttributePreferredSharedMemoryCarveout, pct);
}

static size_t param_smem(const DevRobot& r) { return sizeof(float) * kParamWords * (size_t)r.n; }

static int seg_plan(int segments) { return segments == 2 ? 0 : segments == 4 ? 1 : 2; }
static int seg_groups(int segments, int threads) { return std::max(1, threads / (32 * segments)); }

// per group of G warps: the shared-slot partials of each output (tau in the
// forward; gq, gqd, gqdd in the backward), plus, for the cost variant, one
// cost term per segment; per block, the staged link parameters
size_t tree_seg_smem(const DevRobot& r, int segments, int threads, bool fwd, bool cost) {
  const int t = seg_plan(segments);
  const size_t per =
      (size_t)(fwd ? 1 : 3) * r.seg_ns[t] * segments * 32 + (cost ? segments * 32 : 0);
  return (size_t)seg_groups(segments, threads) * per * sizeof(float) + param_smem(r);
}

// a backward block's gradient-row slots (GradSlot), when it has upstream pose
// or sphere gradients to read
size_t grad_slot_smem(int segments, int threads) {
  return 16 + (size_t)kGradSlotBytes * 32 * segments * seg_groups(segments, threads);
}

template <class Args>
static cudaError_t launch_seg(void (*kern)(DevRobot, Args, int), const DevRobot& r, const Args& a,
                              int threads, int segments, bool fwd, size_t extra,
                              cudaStream_t s) {
  const int t = seg_plan(segments);
  const int CG = seg_groups(segments, threads);
  const size_t smem = tree_seg_smem(r, segments, threads, fwd, false) + extra;
  cudaError_t e =
      cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  fit_carveout((const void*)kern, 32 * segments * CG, smem);
  const int64_t groups = (a.B + 31) / 32;
  const int64_t grid = (groups + CG - 1) / CG;
  kern<<<(unsigned)grid, 32 * segments * CG, smem, s>>>(r, a, t);
  return cudaGetLastError();
}

static cudaError_t launch_cost_seg(const DevRobot& r, const BwdArgs& a, const FusedCost& fc,
                                   int threads, int segments, cudaStream_t s) {
  const int t = seg_plan(segments);
  const int CG = seg_groups(segments, threads);
  const size_t smem = tree_seg_smem(r, segments, threads, false, true) +
                      (a.g_pose || a.g_sph ? grad_slot_smem(segments, threads) : 0);
  cudaError_t e = cudaFuncSetAttribute(tree_bwd_cost_seg_kernel,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  fit_carveout((const void*)tree_bwd_cost_seg_kernel, 32 * segments * CG, smem);
  const int64_t groups = (a.B + 31) / 32;
  const int64_t grid = (groups + CG - 1) / CG;
  tree_bwd_cost_seg_kernel<<<(unsigned)grid, 32 * segments * CG, smem, s>>>(r, a, fc, t);
  return cudaGetLastError();
}

cudaError_t launch_tree_fwd(const DevRobot& r, const FwdArgs& a, int threads, int segments,
                            cudaStream_t s) {
  if (threads <= 0) threads = 128;
  if (segments > 1) {
    // the force stack in shared memory when it fits one block's limit (the
    // humanoid's 13 levels x 448 threads: 140 KB; forward 0.0835 ->
    // 0.0809 ms), else in local memory
    const size_t bt = (size_t)32 * segments * seg_groups(segments, threads);
    const size_t fs = sizeof(float) * 6 * (size_t)r.maxdepth * bt;
    if (a.tau && tree_seg_smem(r, segments, threads, true, false) + fs <= kSegSmemMax)
      return launch_seg(tree_fwd_seg_kernel<true>, r, a, threads, segments, true, fs, s);
    return launch_seg(tree_fwd_seg_kernel<false>, r, a, threads, segments, true, 0, s);
  }
  const size_t fs = sizeof(float) * 6 * (size_t)r.maxdepth * threads;  // the force stack
  const bool use_fs = a.tau && param_smem(r) + fs <= kSegSmemMax;
  const size_t smem = param_smem(r) + (use_fs ? fs : 0);
  auto kern = use_fs ? tree_fwd_kernel<true> : tree_fwd_kernel<false>;
  cudaError_t e =
      cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  fit_carveout((const void*)kern, threads, smem);
  const int64_t grid = (a.B + threads - 1) / threads;
  kern<<<(unsigned)grid, threads, smem, s>>>(r, a);
  return cudaGetLastError();
}

cudaError_t launch_tree_bwd(const DevRobot& r, const BwdArgs& a, int threads, int segments,
                            cudaStream_t s, const FusedCost* fc) {
  if (threads <= 0) threads = 128;
  if (segments > 1)
    return fc ? launch_cost_seg(r, a, *fc, threads, segments, s)
              : launch_seg(tree_bwd_seg_kernel, r, a, threads, segments, false,
                           a.g_pose || a.g_sph ? grad_slot_smem(segments, threads) : 0, s);
  const size_t smem = param_smem(r);
  fit_carveout(fc ? (const void*)tree_bwd_cost_kernel : (const void*)tree_bwd_kernel, threads,
               smem);
  const int64_t grid = (a.B + threads - 1) / threads;
  if (fc)
    tree_bwd_cost_kernel<<<(unsigned)grid, threads, smem, s>>>(r, a, *fc);
  else
    tree_bwd_kernel<<<(unsigned)grid, threads, smem, s>>>(r, a);
  return cudaGetLastError();
}

cudaError_t launch_tree_fwd_spline(const DevRobot& r, const FwdArgs& a, const SplineArgs& sp,
                                   int threads, int segments, cudaStream_t s) {
  if (threads <= 0) threads = 128;
  if (segments > 1) {
    const int t = seg_plan(segments);
    const int CG = seg_groups(segments, threads);
    const int block = 32 * segments * CG;
    const size_t base = tree_seg_smem(r, segments, threads, true, false) + 12 * sizeof(float) * block;
    const size_t fs = sizeof(float) * 6 * (size_t)r.maxdepth * block;  // the force stack
    const bool use_fs = a.tau && base + fs <= kSegSmemMax;
    const size_t smem = use_fs ? base + fs : base;
    auto kern = use_fs ? tree_fwd_spline_seg_kernel<true> : tree_fwd_spline_seg_kernel<false>;
    cudaError_t e =
        cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    fit_carveout((const void*)kern, block, smem);
    const int64_t grid = ((a.B + 31) / 32 + CG - 1) / CG;
    kern<<<(unsigned)grid, block, smem, s>>>(r, a, sp, t);
    return cudaGetLastError();
  }
  const size_t smem = 12 * sizeof(float) * threads + param_smem(r);
  fit_carveout((const void*)tree_fwd_spline_kernel, threads, smem);
  const int64_t grid = (a.B + threads - 1) / threads;
  tree_fwd_spline_kernel<<<(unsigned)grid, threads, smem, s>>>(r, a, sp);
  return cudaGetLastError();
}

cudaError_t launch_tree_bwd_spline_cost(const DevRobot& r, const BwdArgs& a, const FusedCost& fc,
                                        const SplineArgs& sp, int threads, int segments,
                                        cudaStream_t s) {
  if (threads <= 0) threads = 128;
  if (segments > 1) {
    const int t = seg_plan(segments);
    const int CG = seg_groups(segments, threads);
    const int block = 32 * segments * CG;
    const size_t smem = tree_seg_smem(r, segments, threads, false, true) + 12 * sizeof(float) * block;
    cudaError_t e = cudaFuncSetAttribute(tree_bwd_spline_cost_seg_kernel,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    fit_carveout((const void*)tree_bwd_spline_cost_seg_kernel, block, smem);
    const int64_t grid = ((a.B + 31) / 32 + CG - 1) / CG;
    tree_bwd_spline_cost_seg_kernel<<<(unsigned)grid, block, smem, s>>>(r, a, fc, sp, t);
    return cudaGetLastError();
  }
  const size_t smem = 12 * sizeof(float) * threads + param_smem(r);
  fit_carveout((const void*)tree_bwd_spline_cost_kernel, threads, smem);
  const int64_t grid = (a.B + threads - 1) / threads;
  tree_bwd_spline_cost_kernel<<<(unsigned)grid, threads, smem, s>>>(r, a, fc, sp);
  return cudaGetLastError();
}

int tree_max_depth() { return TMAXD; }

}  // namespace wbe
