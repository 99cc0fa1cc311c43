// k_hinge.cu -- the all-pairs summed self-collision hinge with activation
// distance eta:
//   cost_b = w sum_p max(0, eta - d_p),  d_p = |c_i - c_j| - r_i - r_j
// over every masked pair, and its gradient on the sphere centres (a pair
// with d_p < eta adds -w u to dcost/dc_i and +w u to dcost/dc_j,
// u = (c_i - c_j) / |c_i - c_j|).  Feeding that gradient to the backward
// sweep as the sphere upstream gradient gives dcost/dq.
//
// One warp per configuration (persistent grid).  The warp stages the
// configuration's link poses into shared memory, places its spheres (Sec.
// 6.1.1) as SoA rows and bounds every group of 4 with a sphere (C_g, R_g)
// (for a group on one link, the host-made sphere in its link frame moved
// with the link), as the pair stage does.  It then walks the pair stage's
// 4x4 block schedule: a block whose bound |C_i - C_j| - R_i - R_j (widened
// for the approximate square root) is at least eta holds no active pair.
// Each lane marks its surviving blocks of 32 rounds in a bit mask, the
// survivors are queued from a warp scan of the counts and worked 32 at a
// time, one block a lane, every masked pair exactly (sqrt distance).  A
// block's lane sums its pairs' cost and each of its 8 spheres' gradient in
// pair order; the row spheres' gradients, then (a second phase) the column
// spheres', go to a slot of shared memory and are added into the per-sphere
// gradient in a fixed order -- each group's slots by the lowest lane holding
// that group, in lane order -- and the lanes' costs meet in a fixed shuffle
// tree: no atomics, the same result on every run.
#include "spatial.cuh"

namespace wbe {

// per warp, 32-bit words: link poses while the spheres are placed, then the
// 32 block slots in the same region; the sphere SoA rows x, y, z, the group
// bounds (float4), the gradient SoA rows gx, gy, gz and the queue of
// surviving schedule entries
struct HingePlan {
  int xc, yc, zc, gb, gx, gy, gz, q, total;
  __host__ __device__ HingePlan(int n, int S) {
    const int s4 = (S + 3) & ~3, m = (s4 + 31) & ~31;
    const int p0 = (12 * n + 31) & ~31, ps = (32 * kSlotWords + 31) & ~31;
    const int p = p0 > ps ? p0 : ps;
    xc = p;
    yc = xc + m;
    zc = yc + m;
    gb = zc + m;
    gx = gb + m;  // m >= 4 x groups
    gy = gx + m;
    gz = gy + m;
    q = gz + m;
    total = q + 64;
  }
  // a block's slot: the 12 gradient floats of its row spheres, then (a second
  // phase) of its column spheres (an odd stride: the lanes' writes hit
  // distinct banks)
  static constexpr int kSlotWords = 13;
};

size_t hinge_smem_per_warp(const DevRobot& r) {
  return sizeof(float) * HingePlan(r.n, r.S).total;
}
size_t hinge_smem_fixed(const DevRobot& r) { return sizeof(float) * ((4 * r.Sg + 31) & ~31); }
static size_t hinge_block_smem(const DevRobot& r, int warps) {
  return hinge_smem_fixed(r) + (size_t)warps * hinge_smem_per_warp(r);
}

__device__ __forceinline__ float4 ld4(const char* base, uint32_t off) {
  return *reinterpret_cast<const float4*>(base + off);
}
__device__ __forceinline__ float p4(const float4& v, int i) {
  return i == 0 ? v.x : (i == 1 ? v.y : (i == 2 ? v.z : v.w));
}

// Three 8-warp blocks an SM (24 warps; the slots share the pose region, so
// three blocks' workspaces fit): 80 registers a thread (humanoid trajopt48
// hinge 0.337 -> 0.281 ms against two blocks at 122 registers).
__global__ void __launch_bounds__(256, 3) hinge_kernel(DevRobot r, PairSchedule32 ps, HingeArgs A) {
  extern __shared__ __align__(16) float smem[];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, wpb = blockDim.x >> 5;
  const int n = r.n, S = r.S, Sg = r.Sg;
  const HingePlan pl(n, S);
  float4* radw = reinterpret_cast<float4*>(smem);  // group radii, per block
  for (int i = threadIdx.x; i < Sg; i += blockDim.x) radw[i] = __ldg(r.grp_rad + i);
  __syncthreads();
  float* ws = smem + ((4 * Sg + 31) & ~31) + (size_t)warp * pl.total;
  float* P = ws;
  float *xc = ws + pl.xc, *yc = ws + pl.yc, *zc = ws + pl.zc;
  float4* gb = reinterpret_cast<float4*>(ws + pl.gb);
  float *gx = ws + pl.gx, *gy = ws + pl.gy, *gz = ws + pl.gz;
  float* slot = ws;  // over the poses, once the spheres are placed
  uint32_t* qu = reinterpret_cast<uint32_t*>(ws + pl.q);
  const char *cxc = reinterpret_cast<const char*>(xc), *cyc = reinterpret_cast<const char*>(yc),
             *czc = reinterpret_cast<const char*>(zc), *crad = reinterpret_cast<const char*>(radw),
             *cgb = reinterpret_cast<const char*>(gb);
  const float eta = A.eta, w = A.w;
  const int rounds = ps.rounds;
  constexpr int SW = HingePlan::kSlotWords;
  for (int64_t b = (int64_t)blockIdx.x * wpb + warp; b < A.B; b += (int64_t)gridDim.x * wpb) {
    {
      const float4* src = reinterpret_cast<const float4*>(A.pose + b * (int64_t)n * 12);
      float4* dst = reinterpret_cast<float4*>(P);
      for (int i = lane; i < 3 * n; i += 32) {  // asynchronous copies into shared memory
        const unsigned a = static_cast<unsigned>(__cvta_generic_to_shared(dst + i));
        asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(a), "l"(src + i));
      }
      asm volatile("cp.async.commit_group;");
      asm volatile("cp.async.wait_group 0;" ::: "memory");
    }
    __syncwarp();
    if (r.sph_vec4) {  // every group of 4 on one link: a lane a group
      for (int g = lane; g < Sg; g += 32) {
        const float4* T4 = reinterpret_cast<const float4*>(P) + 3 * __ldg(r.grp_link + g);
        const float4 t0 = T4[0], t1 = T4[1], t2 = T4[2];
        const float T[12] = {t0.x, t0.y, t0.z, t0.w, t1.x, t1.y, t1.z, t1.w, t2.x, t2.y, t2.z, t2.w};
        float cx[4], cy[4], cz[4];
#pragma unroll
        for (int k = 0; k < 4; ++k) {
          const float4 sp = __ldg(r.sph + 4 * g + k);
          const float cl[3] = {sp.x, sp.y, sp.z};
          float c[3];
          rot(T, cl, c);
          cx[k] = c[0] + T[9];
          cy[k] = c[1] + T[10];
          cz[k] = c[2] + T[11];
        }
        reinterpret_cast<float4*>(xc)[g] = make_float4(cx[0], cx[1], cx[2], cx[3]);
        reinterpret_cast<float4*>(yc)[g] = make_float4(cy[0], cy[1], cy[2], cy[3]);
        reinterpret_cast<float4*>(zc)[g] = make_float4(cz[0], cz[1], cz[2], cz[3]);
      }
    } else {
      for (int s = lane; s < 4 * Sg; s += 32) {
        float c[3] = {0.0f, 0.0f, 0.0f};  // padding: never in a masked pair
        if (s < S) {
          const float4 sp = __ldg(r.sph + s);
          const float* T = P + 12 * __ldg(r.sph_link + s);
          const float cl[3] = {sp.x, sp.y, sp.z};
          rot(T, cl, c);
          c[0] += T[9];
          c[1] += T[10];
          c[2] += T[11];
        }
        xc[s] = c[0];
        yc[s] = c[1];
        zc[s] = c[2];
      }
    }
    __syncwarp();
    for (int g = lane; g < Sg; g += 32) {  // group bounding spheres (+ the gradient rows' zeros)
      const int gl = __ldg(r.grp_link + g);
      float4 B4;
      if (gl >= 0) {  // one link: its host-made bound, moved with the link
        const float4 L = __ldg(r.grp_loc + g);
        const float* T = P + 12 * gl;
        const float cl[3] = {L.x, L.y, L.z};
        float c[3];
        rot(T, cl, c);
        const float scale = fabsf(T[9]) + fabsf(T[10]) + fabsf(T[11]) + fabsf(L.x) +
                            fabsf(L.y) + fabsf(L.z);
        B4 = make_float4(c[0] + T[9], c[1] + T[10], c[2] + T[11],
                         fmaf(scale, 1e-6f, fmaf(L.w, 1e-6f, L.w)) + 3e-6f);
      } else {
        const int s1 = min(S, 4 * g + 4);
        float cx = 0.0f, cy = 0.0f, cz = 0.0f;
        for (int s = 4 * g; s < s1; ++s) {
          cx += xc[s];
          cy += yc[s];
          cz += zc[s];
        }
        const float inv = 1.0f / (float)max(s1 - 4 * g, 1);
        cx *= inv;
        cy *= inv;
        cz *= inv;
        const float4 rad = radw[g];
        float R = 0.0f;
        for (int s = 4 * g; s < s1; ++s)
          R = fmaxf(R, sqrtf(dist2(cx, cy, cz, xc[s], yc[s], zc[s])) + p4(rad, s - 4 * g));
        B4 = make_float4(cx, cy, cz, fmaf(R, 1e-6f, R) + 3e-6f);  // widened for rounding
      }
      gb[g] = B4;
      const float4 z = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
      reinterpret_cast<float4*>(gx)[g] = z;
      reinterpret_cast<float4*>(gy)[g] = z;
      reinterpret_cast<float4*>(gz)[g] = z;
    }
    __syncwarp();
    float cost = 0.0f;
    for (int r0 = 0; r0 < rounds; r0 += 32) {
      const int r1 = min(rounds, r0 + 32);
      // blocks whose bound (widened below the true one: 4e-6 of the distance
      // here, 2 x 2e-6 in the group radii) is under eta can hold an active pair
      uint32_t km = 0u;
      for (int rr = r0; rr < r1; ++rr) {
        const uint2 e = __ldg(ps.ent + rr * 32 + lane);
        if ((e.y >> 16) != 0u) {
          const float4 P4 = ld4(cgb, e.x & 0xFFFF), Q4 = ld4(cgb, e.x >> 16);
          const float D2 = fmaxf(dist2(P4.x, P4.y, P4.z, Q4.x, Q4.y, Q4.z), 1e-30f);
          const float dist = D2 * rsqrtf(D2);
          km |= (fmaf(dist, 0.999996f, -(P4.w + Q4.w)) < eta ? 1u : 0u) << (rr - r0);
        }
      }
      const int cnt = __popc(km);
      int off = cnt;  // inclusive scan of the counts over the lanes
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const int v = __shfl_up_sync(0xffffffffu, off, o);
        if (lane >= o) off += v;
      }
      const int tot = __shfl_sync(0xffffffffu, off, 31);
      int pos = off - cnt;
      for (int w0 = 0; w0 < tot; w0 += 32) {
        while (km && pos < w0 + 32) {
          const int rr = r0 + __ffs(km) - 1;
          km &= km - 1u;
          qu[pos - w0] = (uint32_t)(rr * 32 + lane);
          ++pos;
        }
        __syncwarp();
        const int count = min(32, tot - w0);
        // one block a lane: every masked pair exactly, in pair order
        uint32_t key = 0xFFFFFFFFu;  // no block
        float gr[12];  // the lane's block: its row spheres' gradients, then its columns'
        if (lane < count) {
          const uint2 e = __ldg(ps.ent + qu[lane]);
          const uint32_t ro = e.x & 0xFFFF, co = e.x >> 16, mask = e.y >> 16;
          key = e.x;
          const float4 XR = ld4(cxc, ro), YR = ld4(cyc, ro), ZR = ld4(czc, ro), RR = ld4(crad, ro);
          const float4 XC = ld4(cxc, co), YC = ld4(cyc, co), ZC = ld4(czc, co), RC = ld4(crad, co);
          float gc[12];
#pragma unroll
          for (int k = 0; k < 12; ++k) gr[k] = gc[k] = 0.0f;
#pragma unroll
          for (int t = 0; t < 16; ++t) {
            if (!((mask >> t) & 1u)) continue;
            const int ia = t >> 2, jc = t & 3;
            const float dx = p4(XR, ia) - p4(XC, jc), dy = p4(YR, ia) - p4(YC, jc),
                        dz = p4(ZR, ia) - p4(ZC, jc);
            const float nrm = sqrtf(fmaf(dz, dz, fmaf(dy, dy, dx * dx)));
            const float d = nrm - (p4(RR, ia) + p4(RC, jc));
            if (d < eta) {
              cost = fmaf(w, eta - d, cost);
              if (nrm > 0.0f) {
                const float k = w / nrm;
                gr[3 * ia] = fmaf(-k, dx, gr[3 * ia]);
                gr[3 * ia + 1] = fmaf(-k, dy, gr[3 * ia + 1]);
                gr[3 * ia + 2] = fmaf(-k, dz, gr[3 * ia + 2]);
                gc[3 * jc] = fmaf(k, dx, gc[3 * jc]);
                gc[3 * jc + 1] = fmaf(k, dy, gc[3 * jc + 1]);
                gc[3 * jc + 2] = fmaf(k, dz, gc[3 * jc + 2]);
              }
            }
          }
          float* sl = slot + lane * SW;
#pragma unroll
          for (int k = 0; k < 12; ++k) sl[k] = gr[k];
#pragma unroll
          for (int k = 0; k < 12; ++k) gr[k] = gc[k];  // the column side, written next
        }
        // add the slots into the spheres' gradients: the row groups, then the
        // column groups, each group's slots by their lowest lane in lane order
#pragma unroll
        for (int side = 0; side < 2; ++side) {
          if (side == 1 && lane < count) {
            float* sl = slot + lane * SW;
#pragma unroll
            for (int k = 0; k < 12; ++k) sl[k] = gr[k];
          }
          __syncwarp();
          const uint32_t grp = side == 0 ? (key & 0xFFFFu) : (key >> 16);  // byte offset
          const uint32_t same = __match_any_sync(0xffffffffu, lane < count ? grp : 0xFFFFFFFFu);
          if (lane < count && (__ffs(same) - 1) == lane) {
            float4* X4 = reinterpret_cast<float4*>(reinterpret_cast<char*>(gx) + grp);
            float4* Y4 = reinterpret_cast<float4*>(reinterpret_cast<char*>(gy) + grp);
            float4* Z4 = reinterpret_cast<float4*>(reinterpret_cast<char*>(gz) + grp);
            float4 ax = *X4, ay = *Y4, az = *Z4;
            for (uint32_t m = same; m; m &= m - 1u) {
              const float* sl = slot + (__ffs(m) - 1) * SW;
              ax.x += sl[0]; ay.x += sl[1]; az.x += sl[2];
              ax.y += sl[3]; ay.y += sl[4]; az.y += sl[5];
              ax.z += sl[6]; ay.z += sl[7]; az.z += sl[8];
              ax.w += sl[9]; ay.w += sl[10]; az.w += sl[11];
            }
            *X4 = ax;
            *Y4 = ay;
            *Z4 = az;
          }
          __syncwarp();
        }
      }
    }
    if (A.g_sph) {  // [S][3] from the SoA gradient rows
      float* o = A.g_sph + b * (int64_t)S * 3;
      for (int e = lane; e < 3 * S; e += 32) {
        const int s = e / 3, k = e - 3 * s;
        o[e] = (k == 0 ? gx : k == 1 ? gy : gz)[s];
      }
    }
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) cost += __shfl_xor_sync(0xffffffffu, cost, off);
    if (lane == 0 && A.cost) A.cost[b] = cost;
    __syncwarp();  // the shared arrays are reused by the next configuration
  }
}

cudaError_t launch_hinge(const DevRobot& r, const PairSchedule32& ps, const HingeArgs& a, int grid,
                         int warps, cudaStream_t s) {
  const size_t smem = hinge_block_smem(r, warps);
  cudaError_t e =
      cudaFuncSetAttribute(hinge_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  hinge_kernel<<<grid, warps * 32, smem, s>>>(r, ps, a);
  return cudaGetLastError();
}

cudaError_t hinge_max_blocks_per_sm(const DevRobot& r, int warps, int* out) {
  const size_t smem = hinge_block_smem(r, warps);
  cudaError_t e =
      cudaFuncSetAttribute(hinge_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  return cudaOccupancyMaxActiveBlocksPerMultiprocessor(out, hinge_kernel, warps * 32, smem);
}

}  // namespace wbe
