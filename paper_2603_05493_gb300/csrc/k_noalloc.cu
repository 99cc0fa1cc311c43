// k_noalloc.cu -- the device side of wb_batch_eval_noalloc: forward evaluation
// of an uneven batch whose tables live in a file-scope device array instead of
// memory allocated per batch.
//
// The tables that wb_batch_create uploads once (robot descriptors, pair
// schedules, problem slices, cost-sorted work items, work counters) are here
// rebuilt on the caller's stream by a setup kernel at every call, from launch
// parameters (NoAllocPlan), so that nothing is allocated and no host buffer has
// to outlive the call.  The forward batch kernels (k_batch.cu) then run on
// those tables unchanged.
#include "wbe_internal.h"

#include <mutex>

namespace wbe {

static constexpr size_t na_up(size_t x) { return (x + 255) & ~size_t(255); }

// scratch layout, every section 256-byte aligned
static constexpr size_t NA_MAX_TITEMS = NA_MAX_CONFIGS / 32 + NA_MAX_PROBLEMS;
static constexpr size_t NA_OFF_ROBOTS = 0;
static constexpr size_t NA_OFF_SCHEDS = NA_OFF_ROBOTS + na_up(sizeof(DevRobot) * NA_MAX_ROBOTS);
static constexpr size_t NA_OFF_PROBS = NA_OFF_SCHEDS + na_up(sizeof(PairSchedule32) * NA_MAX_ROBOTS);
static constexpr size_t NA_OFF_TITEMS = NA_OFF_PROBS + na_up(sizeof(BatchProblemDev) * NA_MAX_PROBLEMS);
static constexpr size_t NA_OFF_PITEMS = NA_OFF_TITEMS + na_up(sizeof(int4) * NA_MAX_TITEMS);
static constexpr size_t NA_OFF_COUNTERS = NA_OFF_PITEMS + na_up(sizeof(int2) * NA_MAX_CONFIGS);
static constexpr size_t NA_BYTES = NA_OFF_COUNTERS + 256;

static_assert(sizeof(NoAllocPlan) + sizeof(void*) <= 32764, "setup parameters exceed the launch limit");

// the public header promises about 0.6 MiB per device (618,240 bytes with
// the present layouts)
static_assert(NA_BYTES <= 640 * 1024, "no-alloc scratch larger than the header states");

static __device__ __align__(256) unsigned char g_noalloc_scratch[NA_BYTES];

__host__ __device__ NoAllocTables noalloc_tables(unsigned char* base) {
  NoAllocTables t;
  t.robots = reinterpret_cast<DevRobot*>(base + NA_OFF_ROBOTS);
  t.scheds = reinterpret_cast<PairSchedule32*>(base + NA_OFF_SCHEDS);
  t.probs = reinterpret_cast<BatchProblemDev*>(base + NA_OFF_PROBS);
  t.titems = reinterpret_cast<int4*>(base + NA_OFF_TITEMS);
  t.pitems = reinterpret_cast<int2*>(base + NA_OFF_PITEMS);
  t.counters = reinterpret_cast<int*>(base + NA_OFF_COUNTERS);
  return t;
}

// Device address of the scratch array on `device`, which the caller has made
// current.  Looked up once per device and kept for the life of the process.
cudaError_t noalloc_scratch(int device, unsigned char** out) {
  static std::mutex mu;
  static unsigned char* addr[NA_MAX_DEVICES] = {};
  *out = nullptr;
  if (device < 0 || device >= NA_MAX_DEVICES) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lock(mu);
  if (!addr[device]) {
    unsigned char* ptr = nullptr;
    cudaError_t e = cudaGetSymbolAddress((void**)&ptr, g_noalloc_scratch);
    if (e != cudaSuccess) return e;
    addr[device] = ptr;
  }
  *out = addr[device];
  return cudaSuccess;
}

// exclusive prefix sum over the block (1024 threads); `tot` holds 32 words
__device__ long long block_excl_scan(long long v, long long* tot) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  long long x = v;
  for (int o = 1; o < 32; o <<= 1) {
    const long long y = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= o) x += y;
  }
  if (lane == 31) tot[warp] = x;
  __syncthreads();
  if (warp == 0) {
    long long w = tot[lane];
    for (int o = 1; o < 32; o <<= 1) {
      const long long y = __shfl_up_sync(0xffffffffu, w, o);
      if (lane >= o) w += y;
    }
    tot[lane] = w;
  }
  __syncthreads();
  const long long before = warp ? tot[warp - 1] : 0;
  __syncthreads();  // tot is reused by the next scan
  return before + x - v;
}

// One thread per problem for the slice offsets (every block recomputes them:
// they are 1024 values); then a grid-stride loop over configurations writes
// the work items at the cost-ordered positions the host chose.
__global__ void __launch_bounds__(1024) noalloc_setup_kernel(const __grid_constant__ NoAllocPlan plan,
                                                             unsigned char* base) {
  __shared__ long long tot[32];
  __shared__ int co_start[NA_MAX_PROBLEMS];
  const NoAllocTables T = noalloc_tables(base);
  const int p = threadIdx.x;
  int robot = 0, H = 0;
  long long v[4] = {0, 0, 0, 0};
  if (p < plan.n_problems) {
    robot = plan.prob[p] >> 24;
    H = plan.prob[p] & 0xFFFFFF;
    const DevRobot& r = plan.robots[robot];
    v[0] = (long long)r.d * H;       // joint-major block
    v[1] = (long long)H * r.n * 12;  // link poses
    v[2] = (long long)H * r.S * 3;   // sphere centres
    v[3] = H;                        // per-configuration outputs
  }
  long long off[4];
  for (int k = 0; k < 4; ++k) off[k] = block_excl_scan(v[k], tot);
  if (p < plan.n_problems) co_start[p] = (int)off[3];
  if (blockIdx.x == 0) {
    if (p < plan.n_problems) T.probs[p] = BatchProblemDev{robot, H, off[0], off[1], off[2], off[3]};
    if (p < plan.n_robots) {
      T.robots[p] = plan.robots[p];
      T.scheds[p] = plan.scheds[p];
    }
  }
  __syncthreads();
  for (int g = blockIdx.x * blockDim.x + threadIdx.x; g < plan.n_configs;
       g += gridDim.x * blockDim.x) {
    // the last problem starting at or before g holds it (empty problems
    // share their start with the next one)
    int lo = 0, hi = plan.n_problems;
    while (hi - lo > 1) {
      const int mid = (lo + hi) >> 1;
      if (co_start[mid] <= g) lo = mid;
      else hi = mid;
    }
    const int q = lo;
    const int c = g - co_start[q];
    const int qh = plan.prob[q] & 0xFFFFFF;
    T.pitems[plan.pstart[q] + c] = make_int2(q, c);
    if ((c & 31) == 0)
      T.titems[plan.tstart[q] + (c >> 5)] = make_int4(q, c, min(32, qh - c), 0);  // mode 0
  }
}

cudaError_t launch_noalloc_setup(const NoAllocPlan& plan, unsigned char* base, int grid,
                                 cudaStream_t s) {
  noalloc_setup_kernel<<<grid, 1024, 0, s>>>(plan, base);
  return cudaGetLastError();
}

}  // namespace wbe
