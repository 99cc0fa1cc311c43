// k_pair.cu -- the single-robot pair kernel: one warp per configuration,
// persistent grid; the per-configuration work is pair_one_culled (default)
// or the full map-reduce pair_one (pair_body.cuh).
#include "pair_body.cuh"

namespace wbe {

template <bool FULL, bool BITS, bool CULL>
__device__ __forceinline__ void pair_warps(const DevRobot& r, const PairSchedule32& ps,
                                           const FwdArgs& A) {
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

// The culled map-reduce is capped at 72 registers: 7 blocks of 4 warps then
// fit an SM's registers, and its shared memory holds 7 (the humanoid's culled
// pair stage: 0.162 ms at 79 registers and 6 blocks, 0.155 ms at 72 and 7,
// without spills).  The full map-reduce keeps its own allocation (it would
// spill at 72).
template <bool FULL, bool BITS>
__global__ void __maxnreg__(72) pair_kernel(DevRobot r, PairSchedule32 ps, FwdArgs A) {
  pair_warps<FULL, BITS, true>(r, ps, A);
}
template <bool FULL, bool BITS>
__global__ void __launch_bounds__(256, 3) pair_full_kernel(DevRobot r, PairSchedule32 ps,
                                                          FwdArgs A) {
  pair_warps<FULL, BITS, false>(r, ps, A);
}

// Small robots (at most kThreadMaxS spheres and kThreadMaxP pairs, e.g. a
// 7-DoF arm: 28 spheres, 240 pairs): one thread per configuration.  A warp per
// configuration leaves most lanes idle on so few blocks, and its per-
// configuration staging and reductions cost more than the pairs.  Each thread
// places its configuration's spheres from its link poses into its column of
// shared memory ([3][S][threads]: a warp reads 32 consecutive words) and
// evaluates every masked pair exactly, in index order (the column stride is
// threads + 1, so that the warp's transposed output copy, which reads one
// configuration's centres across the lanes, hits distinct banks):
//   d = sqrt(|c_i - c_j|^2) - (r_i + r_j), kept when strictly smaller,
// the same arithmetic as the warp kernel's exact path and the same tie rule
// (smallest pair index), so the results are the same bits.  The sphere and
// pair tables are staged once per block.
constexpr int kThreadMaxS = 32, kThreadMaxP = 1024, kThreadBlock = 128;
bool pair_thread_ok(const DevRobot& r) { return r.S <= kThreadMaxS && r.P <= kThreadMaxP; }
static size_t pair_thread_smem(const DevRobot& r) {
  return 16 * (size_t)r.S + 16 * (size_t)r.P + 4 * (size_t)r.S +
         sizeof(float) * 3 * (size_t)r.S * (kThreadBlock + 1);
}

template <bool BITS>
__global__ void __launch_bounds__(kThreadBlock) pair_thread_kernel(DevRobot r, FwdArgs A) {
  extern __shared__ __align__(16) float sm[];
  const int S = r.S, P = r.P, n = r.n, t = threadIdx.x;
  const int T = blockDim.x + 1;  // column stride of the centres
  float4* sp = reinterpret_cast<float4*>(sm);  // [S] centre in the link frame, radius
  // [P] pairs, row-major sorted: the two spheres' column offsets (s T) and
  // their radius sum r_i + r_j
  int4* pr = reinterpret_cast<int4*>(sp + S);
  int* sl = reinterpret_cast<int*>(pr + P);    // [S] link of each sphere
  float* cs = reinterpret_cast<float*>(sl + S);  // [3][S][T] this block's sphere centres
  for (int i = t; i < S; i += blockDim.x) {
    sp[i] = __ldg(r.sph + i);
    sl[i] = __ldg(r.sph_link + i);
  }
  for (int i = t; i < P; i += blockDim.x) {
    const int2 ij = __ldg(r.pairs + i);
    const float rr = __ldg(r.sph + ij.x).w + __ldg(r.sph + ij.y).w;
    pr[i] = make_int4(ij.x * T, ij.y * T, __float_as_int(rr), 0);
  }
  __syncthreads();
  const int64_t b = (int64_t)blockIdx.x * blockDim.x + t;
  const int lane = t & 31;
  const int64_t b0 = b - lane;  // the warp's first configuration
  const int nw = A.B - b0 < 32 ? (int)(A.B - b0) : 32;  // configurations of this warp
  if (b0 >= A.B) return;
  float* cx = cs + t;
  float* cy = cs + (size_t)S * T + t;
  float* cz = cs + 2 * (size_t)S * T + t;
  const float4* poses = reinterpret_cast<const float4*>(A.pose + b * (int64_t)n * 12);
  int cur = -1;
  float Pw[12];
  for (int s = 0; s < S && lane < nw; ++s) {
    const int l = sl[s];
    if (l != cur) {  // the spheres of a link are consecutive in most robots
      const float4 x0 = __ldg(poses + 3 * l), x1 = __ldg(poses + 3 * l + 1),
                   x2 = __ldg(poses + 3 * l + 2);
      Pw[0] = x0.x; Pw[1] = x0.y; Pw[2] = x0.z; Pw[3] = x0.w;
      Pw[4] = x1.x; Pw[5] = x1.y; Pw[6] = x1.z; Pw[7] = x1.w;
      Pw[8] = x2.x; Pw[9] = x2.y; Pw[10] = x2.z; Pw[11] = x2.w;
      cur = l;
    }
    const float4 q = sp[s];
    const float cl[3] = {q.x, q.y, q.z};
    float c[3];
    rot(Pw, cl, c);
    c[0] += Pw[9];
    c[1] += Pw[10];
    c[2] += Pw[11];
    cx[(size_t)s * T] = c[0];
    cy[(size_t)s * T] = c[1];
    cz[(size_t)s * T] = c[2];
  }
  __syncwarp();
  if (A.sph) {  // the warp's configurations are one contiguous [nw][S][3] region
    const float* cw = cs + (t - lane);  // column of the warp's first configuration
    float* o = A.sph + b0 * S * 3;
    for (int c = 0; c < nw; ++c)
      for (int e = lane; e < 3 * S; e += 32) {
        const int sph = e / 3, k = e - 3 * sph;
        o[(size_t)c * 3 * S + e] = cw[((size_t)k * S + sph) * T + c];
      }
  }
  if (lane >= nw) return;
  if (!A.dmin && !BITS) return;
  float best = __int_as_float(0x7f800000);
  int bi = -1;
  uint32_t word = 0u;
  const int W = (P + 31) >> 5;
  for (int p = 0; p < P; ++p) {
    const int4 ij = pr[p];
    const float d = sqrtf(dist2(cx[ij.x], cy[ij.x], cz[ij.x], cx[ij.y], cy[ij.y], cz[ij.y])) -
                    __int_as_float(ij.z);
    if (d < best) {
      best = d;
      bi = p;
    }
    if (BITS) {
      word |= (d < 0.0f ? 1u : 0u) << (p & 31);
      if ((p & 31) == 31 || p == P - 1) {
        A.bits[b * (int64_t)W + (p >> 5)] = word;
        word = 0u;
      }
    }
  }
  if (A.dmin) {
    A.dmin[b] = best;
    A.worst[b] = bi;
    if (A.wdiff) {
      float dd[3] = {0.0f, 0.0f, 0.0f};
      if (bi >= 0) {
        const int4 ij = pr[bi];
        dd[0] = cx[ij.x] - cx[ij.y];
        dd[1] = cy[ij.x] - cy[ij.y];
        dd[2] = cz[ij.x] - cz[ij.y];
      }
      A.wdiff[3 * b] = dd[0];
      A.wdiff[3 * b + 1] = dd[1];
      A.wdiff[3 * b + 2] = dd[2];
    }
  }
}

static cudaError_t launch_pair_thread(const DevRobot& r, const FwdArgs& a, cudaStream_t s) {
  const size_t smem = pair_thread_smem(r);
  auto kern = a.bits ? pair_thread_kernel<true> : pair_thread_kernel<false>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)smem);
  if (e != cudaSuccess) return e;
  const int64_t grid = (a.B + kThreadBlock - 1) / kThreadBlock;
  kern<<<(unsigned)grid, kThreadBlock, smem, s>>>(r, a);
  return cudaGetLastError();
}

template <bool FULL, bool BITS, bool CULL>
static cudaError_t pair_launch_t(const DevRobot& r, const PairSchedule32& ps, const FwdArgs& a,
                                 int grid, int warps, size_t smem, cudaStream_t s, int* occ) {
  auto kern = CULL ? pair_kernel<FULL, BITS> : pair_full_kernel<FULL, BITS>;
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
  if (cull && pair_thread_ok(r)) return launch_pair_thread(r, a, s);  // small robots
  return pair_dispatch(r, ps, a, grid, warps, s, nullptr, cull);
}

size_t pair_block_smem(const DevRobot& r, int warps, bool bits) { return pair_smem(r, warps, bits); }

cudaError_t pair_max_blocks_per_sm(const DevRobot& r, int warps, bool bits, int* out) {
  FwdArgs a{};
  a.bits = bits ? reinterpret_cast<uint32_t*>(16) : nullptr;  // only selects the variant
  return pair_dispatch(r, PairSchedule32{}, a, 0, warps, nullptr, out, true);
}

}  // namespace wbe
