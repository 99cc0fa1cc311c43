// k_kin.cu -- kinematic Jacobians of chosen links and the whole-body centre of
// mass with its Jacobian, from the world link poses the forward sweep wrote
// (the "second kernel" outputs of Sec. 6.1.1; the columns follow Alg. 2).
//
// One warp per configuration (persistent grid).  The warp stages the poses
// and, at every depth-first position, the link's mass moment m_k x_k =
// m_k p_k + R_k h_k (h_k = m_k c_k, payload point masses included in the
// compact inertia), kept as exclusive prefix sums over the depth-first order
// so that any subtree's moment is one difference.  A lane per joint j then walks the links the joint
// drives (connectedLinks of Alg. 2, several for a mimic joint):
//   Jacobian of target e: a driven link l contributes when it is an ancestor
//     of e or e itself -- an O(1) test on depth-first ranges (l's subtree is
//     the range [pos_l, end_l)) in place of Alg. 2's affects / linkChain
//     filters -- with m_l [w x (p_e - p_l); w] for a revolute joint
//     (w = R_l a_l) and m_l [R_l a_l; 0] for a prismatic one;
//   centre of mass: sum_k m_k x_k / M, and column j of its Jacobian
//     sum_l m_l (w x (S_l - M_l p_l)) / M (revolute) or M_l R_l a_l / M
//     (prismatic), with S_l and M_l the mass moment and mass of l's subtree:
//     the difference of the prefix sums at the ends of its contiguous
//     depth-first range.
// Rows of a link Jacobian: velocity of the world origin, then angular
// velocity, both in world coordinates.
#include "spatial.cuh"

namespace wbe {

// per warp: link poses, then the exclusive prefix sums of the mass moments
// over the depth-first order (n + 1 float4)
static __host__ __device__ int kin_words(int n) {
  return ((12 * n + 31) & ~31) + ((4 * (n + 1) + 31) & ~31);
}

__global__ void __launch_bounds__(256) kin_kernel(DevRobot r, const __grid_constant__ KinArgs A) {
  extern __shared__ __align__(16) float smem[];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, wpb = blockDim.x >> 5;
  const int n = r.n, d = r.d;
  float* P = smem + (size_t)warp * kin_words(n);       // poses
  float4* mom = reinterpret_cast<float4*>(P + ((12 * n + 31) & ~31));  // by DFS position
  for (int64_t b = (int64_t)blockIdx.x * wpb + warp; b < A.B; b += (int64_t)gridDim.x * wpb) {
    const float4* src = reinterpret_cast<const float4*>(A.pose + b * (int64_t)n * 12);
    float4* dst = reinterpret_cast<float4*>(P);
    for (int i = lane; i < 3 * n; i += 32) dst[i] = __ldg(src + i);
    __syncwarp();
    const bool want_com = A.com || A.jac_com;
    float M = 0.0f;
    if (want_com) {
      // mass moments by DFS position and their exclusive prefix sums
      // mom[pos] = sum of the first pos moments (warp scans, 32 at a time):
      // a subtree is a DFS range [pos_l, end_l), so its moment is
      // mom[end_l] - mom[pos_l], and the whole body's is mom[n]
      float4 carry = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
      if (lane == 0) mom[0] = carry;
      for (int p0 = 0; p0 < n; p0 += 32) {
        const int pos = p0 + lane;
        float4 v = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
        if (pos < n) {
          const int k = __ldg(r.dfs + pos).x;
          const float* I = r.inert + 10 * k;
          const float mk = __ldg(I), h[3] = {__ldg(I + 1), __ldg(I + 2), __ldg(I + 3)};
          const float* T = P + 12 * k;
          float Rh[3];
          rot(T, h, Rh);
          v = make_float4(fmaf(mk, T[9], Rh[0]), fmaf(mk, T[10], Rh[1]), fmaf(mk, T[11], Rh[2]),
                          mk);
        }
#pragma unroll
        for (int off = 1; off < 32; off <<= 1) {  // inclusive scan
          const float x = __shfl_up_sync(0xffffffffu, v.x, off);
          const float y = __shfl_up_sync(0xffffffffu, v.y, off);
          const float z = __shfl_up_sync(0xffffffffu, v.z, off);
          const float w = __shfl_up_sync(0xffffffffu, v.w, off);
          if (lane >= off) {
            v.x += x;
            v.y += y;
            v.z += z;
            v.w += w;
          }
        }
        if (pos < n)
          mom[pos + 1] = make_float4(carry.x + v.x, carry.y + v.y, carry.z + v.z, carry.w + v.w);
        carry.x += __shfl_sync(0xffffffffu, v.x, 31);
        carry.y += __shfl_sync(0xffffffffu, v.y, 31);
        carry.z += __shfl_sync(0xffffffffu, v.z, 31);
        carry.w += __shfl_sync(0xffffffffu, v.w, 31);
      }
      __syncwarp();
      const float4 tot = mom[n];
      M = tot.w;
      if (A.com && lane == 0) {
        const float iM = M > 0.0f ? 1.0f / M : 0.0f;
        A.com[3 * b] = tot.x * iM;
        A.com[3 * b + 1] = tot.y * iM;
        A.com[3 * b + 2] = tot.z * iM;
      }
    }
    for (int j = lane; j < d; j += 32) {
      const int l0 = __ldg(r.jl_start + j), l1 = __ldg(r.jl_start + j + 1);
      // centre-of-mass column
      if (A.jac_com) {
        float c[3] = {0.0f, 0.0f, 0.0f};
        for (int li = l0; li < l1; ++li) {
          const int l = __ldg(r.jl_links + li);
          const float* T = P + 12 * l;
          const float4 a4 = __ldg(reinterpret_cast<const float4*>(r.axis) + l);
          const float a[3] = {a4.x, a4.y, a4.z};
          float wv[3];
          rot(T, a, wv);  // R_l a_l
          const float mm = __ldg(reinterpret_cast<const float2*>(r.mimic) + l).x;
          const float4 hi = mom[__ldg(r.dfs_end + l)], lo = mom[__ldg(r.dfs_pos + l)];
          const float S[3] = {hi.x - lo.x, hi.y - lo.y, hi.z - lo.z};
          const float Ms = hi.w - lo.w;
          if (__ldg(r.jtype + l) == 1) {
            const float rel[3] = {fmaf(-Ms, T[9], S[0]), fmaf(-Ms, T[10], S[1]),
                                  fmaf(-Ms, T[11], S[2])};
            float cr[3];
            cross3(wv, rel, cr);
            for (int i = 0; i < 3; ++i) c[i] = fmaf(mm, cr[i], c[i]);
          } else if (__ldg(r.jtype + l) == 2) {
            for (int i = 0; i < 3; ++i) c[i] = fmaf(mm * Ms, wv[i], c[i]);
          }
        }
        const float iM = M > 0.0f ? 1.0f / M : 0.0f;
        for (int i = 0; i < 3; ++i) A.jac_com[(b * 3 + i) * d + j] = c[i] * iM;
      }
      // link Jacobians
      if (A.jac) {
        for (int t = 0; t < A.nt; ++t) {
          const int e = A.targets[t];
          const int pe = __ldg(r.dfs_pos + e);
          const float* Te = P + 12 * e;
          float col[6] = {0.0f, 0.0f, 0.0f, 0.0f, 0.0f, 0.0f};
          for (int li = l0; li < l1; ++li) {
            const int l = __ldg(r.jl_links + li);
            if (pe < __ldg(r.dfs_pos + l) || pe >= __ldg(r.dfs_end + l)) continue;  // not on e's chain
            const float* T = P + 12 * l;
            const float4 a4 = __ldg(reinterpret_cast<const float4*>(r.axis) + l);
            const float a[3] = {a4.x, a4.y, a4.z};
            float wv[3];
            rot(T, a, wv);
            const float mm = __ldg(reinterpret_cast<const float2*>(r.mimic) + l).x;
            if (__ldg(r.jtype + l) == 1) {
              const float rel[3] = {Te[9] - T[9], Te[10] - T[10], Te[11] - T[11]};
              float cr[3];
              cross3(wv, rel, cr);
              for (int i = 0; i < 3; ++i) {
                col[i] = fmaf(mm, cr[i], col[i]);
                col[3 + i] = fmaf(mm, wv[i], col[3 + i]);
              }
            } else if (__ldg(r.jtype + l) == 2) {
              for (int i = 0; i < 3; ++i) col[i] = fmaf(mm, wv[i], col[i]);
            }
          }
          float* o = A.jac + ((b * A.nt + t) * 6) * (int64_t)d + j;
          for (int i = 0; i < 6; ++i) o[(int64_t)i * d] = col[i];
        }
      }
    }
    __syncwarp();  // shared arrays are reused by the next configuration
  }
}

size_t kin_smem_per_warp(const DevRobot& r) { return sizeof(float) * kin_words(r.n); }

cudaError_t launch_kin(const DevRobot& r, const KinArgs& a, int grid, int warps, cudaStream_t s) {
  const size_t smem = sizeof(float) * kin_words(r.n) * warps;
  cudaError_t e =
      cudaFuncSetAttribute(kin_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  kin_kernel<<<grid, warps * 32, smem, s>>>(r, a);
  return cudaGetLastError();
}

cudaError_t kin_max_blocks_per_sm(const DevRobot& r, int warps, int* out) {
  const size_t smem = sizeof(float) * kin_words(r.n) * warps;
  cudaError_t e =
      cudaFuncSetAttribute(kin_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  return cudaOccupancyMaxActiveBlocksPerMultiprocessor(out, kin_kernel, warps * 32, smem);
}

}  // namespace wbe
