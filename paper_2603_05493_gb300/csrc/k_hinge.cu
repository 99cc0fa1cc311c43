// k_hinge.cu -- the all-pairs summed self-collision hinge with activation
// distance eta:
//   cost_b = w sum_p max(0, eta - d_p),  d_p = |c_i - c_j| - r_i - r_j
// over every masked pair, and its gradient on the sphere centres (a pair
// with d_p < eta adds -w u to dcost/dc_i and +w u to dcost/dc_j,
// u = (c_i - c_j) / |c_i - c_j|).  Feeding that gradient to the backward
// sweep as the sphere upstream gradient gives dcost/dq.
//
// One warp per configuration (persistent grid): the warp stages the
// configuration's link poses into shared memory, places its spheres
// (Sec. 6.1.1), then each lane walks the partner lists of its spheres
// (s = lane, lane + 32, ...; partners ascending).  A sphere accumulates its
// own gradient over all its partners in list order, and the cost counts each
// pair once, at its lower sphere, in the same order, then a fixed shuffle
// tree adds the lanes: no atomics, the same result on every run.  Pairs are
// first screened without a square root, |c_i - c_j|^2 < (eta + r_i + r_j)^2
// widened by a rounding margin, and the exact distance decides.
#include "spatial.cuh"

namespace wbe {

// per warp: link poses, then one float4 (x, y, z, r) per sphere plus the
// sentinel sphere S that pads the partner lists
static __host__ __device__ int hinge_words(int n, int S) {
  const int p = (12 * n + 31) & ~31;
  return p + 4 * (((S + 1) + 7) & ~7);
}

size_t hinge_smem_per_warp(const DevRobot& r) { return sizeof(float) * hinge_words(r.n, r.S); }

__global__ void __launch_bounds__(256) hinge_kernel(DevRobot r, HingeArgs A) {
  extern __shared__ __align__(16) float smem[];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, wpb = blockDim.x >> 5;
  const int n = r.n, S = r.S;
  float* ws = smem + (size_t)warp * hinge_words(n, S);
  float* P = ws;  // link poses
  float4* cs = reinterpret_cast<float4*>(ws + ((12 * n + 31) & ~31));  // spheres
  const float eta = A.eta, w = A.w;
  for (int64_t b = (int64_t)blockIdx.x * wpb + warp; b < A.B; b += (int64_t)gridDim.x * wpb) {
    const float4* src = reinterpret_cast<const float4*>(A.pose + b * (int64_t)n * 12);
    float4* dst = reinterpret_cast<float4*>(P);
    for (int i = lane; i < 3 * n; i += 32) dst[i] = __ldg(src + i);
    __syncwarp();
    for (int s = lane; s < S; s += 32) {
      const float4 sp = __ldg(r.sph + s);
      const float* T = P + 12 * __ldg(r.sph_link + s);
      const float cl[3] = {sp.x, sp.y, sp.z};
      float c[3];
      rot(T, cl, c);
      cs[s] = make_float4(c[0] + T[9], c[1] + T[10], c[2] + T[11], sp.w);
    }
    if (lane == 0) cs[S] = make_float4(1e18f, 1e18f, 1e18f, 0.0f);  // the padding sentinel
    __syncwarp();
    float cost = 0.0f;
    for (int s = lane; s < S; s += 32) {
      const float4 me = cs[s];
      float gx = 0.0f, gy = 0.0f, gz = 0.0f;
      const int e0 = __ldg(r.adj_start + s), e1 = __ldg(r.adj_start + s + 1);
      const ushort4* a4 = reinterpret_cast<const ushort4*>(r.adj);
      for (int e = e0; e < e1; e += 4) {
        const ushort4 pq = __ldg(a4 + (e >> 2));
        const int ps[4] = {pq.x, pq.y, pq.z, pq.w};
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          const int p = ps[u];
          const float4 o = cs[p];
          const float dx = me.x - o.x, dy = me.y - o.y, dz = me.z - o.z;
          const float n2 = fmaf(dz, dz, fmaf(dy, dy, dx * dx));
          const float t = eta + me.w + o.w;
          const float tm = fmaf(t, 1e-5f, t) + 1e-6f;  // screen margin over float rounding
          if (t > -1e-6f && n2 < tm * tm) {
            const float nrm = sqrtf(n2);
            const float d = nrm - (me.w + o.w);
            if (d < eta) {
              if (nrm > 0.0f) {
                const float k = w / nrm;
                gx = fmaf(-k, dx, gx);
                gy = fmaf(-k, dy, gy);
                gz = fmaf(-k, dz, gz);
              }
              if (p > s) cost = fmaf(w, eta - d, cost);
            }
          }
        }
      }
      if (A.g_sph) {
        float* o = A.g_sph + (b * S + s) * 3;
        o[0] = gx;
        o[1] = gy;
        o[2] = gz;
      }
    }
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) cost += __shfl_xor_sync(0xffffffffu, cost, off);
    if (lane == 0 && A.cost) A.cost[b] = cost;
    __syncwarp();  // the shared arrays are reused by the next configuration
  }
}

cudaError_t launch_hinge(const DevRobot& r, const HingeArgs& a, int grid, int warps,
                         cudaStream_t s) {
  const size_t smem = hinge_smem_per_warp(r) * warps;
  cudaError_t e =
      cudaFuncSetAttribute(hinge_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  hinge_kernel<<<grid, warps * 32, smem, s>>>(r, a);
  return cudaGetLastError();
}

cudaError_t hinge_max_blocks_per_sm(const DevRobot& r, int warps, int* out) {
  const size_t smem = hinge_smem_per_warp(r) * warps;
  cudaError_t e =
      cudaFuncSetAttribute(hinge_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  return cudaOccupancyMaxActiveBlocksPerMultiprocessor(out, hinge_kernel, warps * 32, smem);
}

}  // namespace wbe
