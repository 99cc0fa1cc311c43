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
// (Sec. 6.1.1) and bounds every group of 4 with a sphere (C_g, R_g) (for a
// group on one link, the host-made sphere in its link frame moved with the
// link), then each
// lane walks the partner groups of its spheres (s = lane, lane + 32, ...;
// groups ascending).  A partner group whose bound is farther than eta,
// |c_s - C_g| - r_s - R_g >= eta (every partner in it then has d >= eta),
// is skipped after one test; otherwise its partners (a 4-bit mask) are tested
// -- without a square root, |c_s - c_p|^2 < (eta + r_s + r_p)^2 widened by a
// rounding margin -- and the exact distance decides.  A sphere sums its own
// gradient over its partners in list order, the cost counts each pair once,
// at its lower sphere, in the same order, and a fixed shuffle tree adds the
// lanes: no atomics, the same result on every run.
#include "spatial.cuh"

namespace wbe {

// per warp: link poses, one float4 (x, y, z, r) per sphere (padded to whole
// groups), one float4 (C, R) per group
static __host__ __device__ int hinge_words(int n, int S) {
  const int p = (12 * n + 31) & ~31;
  const int s4 = (S + 3) & ~3;
  return p + 4 * ((s4 + 7) & ~7) + 4 * (((s4 / 4) + 7) & ~7);
}

size_t hinge_smem_per_warp(const DevRobot& r) { return sizeof(float) * hinge_words(r.n, r.S); }

__global__ void __launch_bounds__(256) hinge_kernel(DevRobot r, HingeArgs A) {
  extern __shared__ __align__(16) float smem[];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, wpb = blockDim.x >> 5;
  const int n = r.n, S = r.S;
  float* ws = smem + (size_t)warp * hinge_words(n, S);
  float* P = ws;  // link poses
  const int s4 = (S + 3) & ~3, Sg = s4 / 4;
  float4* cs = reinterpret_cast<float4*>(ws + ((12 * n + 31) & ~31));  // spheres
  float4* gb = cs + ((s4 + 7) & ~7);                                  // group bounds
  const float eta = A.eta, w = A.w;
  for (int64_t b = (int64_t)blockIdx.x * wpb + warp; b < A.B; b += (int64_t)gridDim.x * wpb) {
    const float4* src = reinterpret_cast<const float4*>(A.pose + b * (int64_t)n * 12);
    float4* dst = reinterpret_cast<float4*>(P);
    for (int i = lane; i < 3 * n; i += 32) dst[i] = __ldg(src + i);
    __syncwarp();
    for (int s = lane; s < s4; s += 32) {
      if (s < S) {
        const float4 sp = __ldg(r.sph + s);
        const float* T = P + 12 * __ldg(r.sph_link + s);
        const float cl[3] = {sp.x, sp.y, sp.z};
        float c[3];
        rot(T, cl, c);
        cs[s] = make_float4(c[0] + T[9], c[1] + T[10], c[2] + T[11], sp.w);
      } else {
        cs[s] = make_float4(0.0f, 0.0f, 0.0f, 0.0f);  // padding, never a partner
      }
    }
    __syncwarp();
    for (int g = lane; g < Sg; g += 32) {  // group bounding spheres
      const int gl = __ldg(r.grp_link + g);
      if (gl >= 0) {  // one link: its host-made bound, moved with the link
        const float4 L = __ldg(r.grp_loc + g);
        const float* T = P + 12 * gl;
        const float cl[3] = {L.x, L.y, L.z};
        float c[3];
        rot(T, cl, c);
        const float scale = fabsf(T[9]) + fabsf(T[10]) + fabsf(T[11]) + fabsf(L.x) +
                            fabsf(L.y) + fabsf(L.z);
        gb[g] = make_float4(c[0] + T[9], c[1] + T[10], c[2] + T[11],
                            fmaf(scale, 1e-6f, fmaf(L.w, 1e-6f, L.w)) + 1e-6f);
        continue;
      }
      const int s1 = min(S, 4 * g + 4);
      float cx = 0.0f, cy = 0.0f, cz = 0.0f;
      for (int s = 4 * g; s < s1; ++s) {
        cx += cs[s].x;
        cy += cs[s].y;
        cz += cs[s].z;
      }
      const float inv = 1.0f / (float)max(s1 - 4 * g, 1);
      cx *= inv;
      cy *= inv;
      cz *= inv;
      float R = 0.0f;
      for (int s = 4 * g; s < s1; ++s)
        R = fmaxf(R, sqrtf(dist2(cx, cy, cz, cs[s].x, cs[s].y, cs[s].z)) + cs[s].w);
      gb[g] = make_float4(cx, cy, cz, fmaf(R, 1e-6f, R) + 1e-6f);  // widened for rounding
    }
    __syncwarp();
    float cost = 0.0f;
    for (int s = lane; s < S; s += 32) {
      const float4 me = cs[s];
      float gx = 0.0f, gy = 0.0f, gz = 0.0f;
      const int e1 = __ldg(r.adj_start + s + 1);
      for (int e = __ldg(r.adj_start + s); e < e1; ++e) {
        const int ent = __ldg(r.adj + e);
        const int g = ent & 0xFF;
        const float4 B4 = gb[g];
        const float tg = eta + me.w + B4.w;  // skip the group when |c_s - C_g| >= tg
        const float tgm = fmaf(tg, 1e-5f, tg) + 1e-6f;
        if (tg <= -1e-6f || dist2(me.x, me.y, me.z, B4.x, B4.y, B4.z) >= tgm * tgm) continue;
        for (int m = ent >> 8; m; m &= m - 1) {
          const int p = 4 * g + __ffs(m) - 1;
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
