// k_fused.cu -- fused whole-body kernels.
//
// Layout of the work: a CTA owns a tile of `cpb` consecutive configurations;
// each configuration is owned by a group of G lanes (G = 32: one warp per
// configuration; G < 32: 32/G configurations per warp).  Per tile:
//   1. the CTA stages q, qd, qdd (joint-major [d][B] in HBM) for its tile into
//      shared memory: each joint row of the tile is a contiguous run, loaded
//      coalesced;
//   2. each group runs its configuration through the stages, level by level
//      over the tree (Sec. 6.3 "tree-level parallelism"), synchronising with
//      __syncwarp (Tab. rnea_comparison "warp" sync), with link transforms,
//      sphere centres and dynamics state in shared memory;
//   3. the CTA writes the joint-major outputs of the tile back coalesced.
// The grid is persistent: CTAs loop over tiles with a grid stride.
//
// Pair stage (Sec. 6.2).  The host groups spheres in fours and the pair list
// into 4x4 group blocks, then deals the blocks to the G lanes so that, in
// every round, the 8 lanes of a shared-memory phase read distinct bank groups
// (block column gj = lane mod 8).  A lane keeps the 4 row spheres of its
// current block in registers and tests 16 pairs per 4 vector loads with a
// sqrt-free filter d2 < (best + r_i + r_j + margin)^2; only blocks that may
// hold an improvement take the exact path (sqrtf, pair index, (d, index)
// lexicographic compare).  The G lanes then reduce (d, index) with
// shuffles.  This replaces the paper's two-kernel map-reduce: one
// configuration never spans more than one group, so the reduce stays in
// registers.
#include "spatial.cuh"

#include <climits>

namespace wbe {

__host__ __device__ constexpr int align32(int x) { return (x + 31) & ~31; }

// ---------------------------------------------------------------------------
// shared-memory plans (floats per configuration), identical on host and device
// ---------------------------------------------------------------------------
struct FwdPlan {
  int q, Rl, Rw, sx, sy, sz, v, a, F, tl, bits, total;
  __host__ __device__ FwdPlan(int n, int d, int Sg, int P, bool with_bits) {
    int o = 0;
    q = o;  o += align32(3 * d);
    Rl = o; o += align32(12 * n);
    const int u = o;
    // FK / pair phase
    Rw = u;
    sx = Rw + align32(12 * n);
    sy = sx + align32(4 * Sg);
    sz = sy + align32(4 * Sg);
    const int end1 = sz + align32(4 * Sg);
    // dynamics phase (aliases the FK / pair phase)
    v = u;
    a = v + align32(6 * n);
    F = a + align32(6 * n);
    tl = F + align32(6 * n);
    const int end2 = tl + align32(n);
    o = end1 > end2 ? end1 : end2;
    bits = o;
    if (with_bits) o += align32((P + 31) / 32);
    total = o;
  }
};

struct BwdPlan {
  int q, Rl, Rw, up, vb, lq, va, F, W, total;
  __host__ __device__ BwdPlan(int n, int d) {
    int o = 0;
    q = o;  o += align32(4 * d);   // q, qd, qdd, g_tau  -> gq, gqd, gqdd
    Rl = o; o += align32(12 * n);
    Rw = o; o += align32(12 * n);  // later: up (6n) during the force sweep,
    up = Rw;                       //        vb (6n) + lq (3n) in the adjoint
    vb = Rw;
    lq = Rw + 6 * n;
    va = o; o += align32(12 * n);  // v (6n), a (6n)
    F = o;  o += align32(6 * n);
    W = o;  o += align32(6 * n);
    total = o;
  }
};

size_t fused_fwd_smem_per_config(const DevRobot& r, int G, bool bits) {
  (void)G;
  return sizeof(float) * (size_t)FwdPlan(r.n, r.d, r.Sg, r.P, bits).total;
}
size_t fused_bwd_smem_per_config(const DevRobot& r, int G) {
  (void)G;
  return sizeof(float) * (size_t)BwdPlan(r.n, r.d).total;
}

// ---------------------------------------------------------------------------
// group helpers
// ---------------------------------------------------------------------------
template <int G>
__device__ __forceinline__ void group_min(float& best, int& idx) {
#pragma unroll
  for (int off = G / 2; off > 0; off >>= 1) {
    const float ob = __shfl_xor_sync(0xffffffffu, best, off);
    const int oi = __shfl_xor_sync(0xffffffffu, idx, off);
    if (ob < best || (ob == best && oi < idx)) {
      best = ob;
      idx = oi;
    }
  }
}

// stage joint-major rows [d][B] of a tile into per-config shared arrays
__device__ __forceinline__ void stage_rows(float* smem, int cfg_stride, int dst_off,
                                           const float* src, int d, int64_t B, int64_t b0,
                                           int cpb) {
  for (int idx = threadIdx.x; idx < d * cpb; idx += blockDim.x) {
    const int j = idx / cpb, c = idx - j * cpb;
    const int64_t b = b0 + c;
    float val = 0.0f;
    if (src && b < B) val = src[(int64_t)j * B + b];
    smem[c * cfg_stride + dst_off + j] = val;
  }
}

__device__ __forceinline__ void unstage_rows(const float* smem, int cfg_stride, int src_off,
                                             float* dst, int d, int64_t B, int64_t b0, int cpb) {
  for (int idx = threadIdx.x; idx < d * cpb; idx += blockDim.x) {
    const int j = idx / cpb, c = idx - j * cpb;
    const int64_t b = b0 + c;
    if (b < B) dst[(int64_t)j * B + b] = smem[c * cfg_stride + src_off + j];
  }
}

// FK of one configuration into Rl / Rw (shared), level by level.
template <int G>
__device__ __forceinline__ void group_fk(const DevRobot& r, int lig, const float* qs, float* Rl,
                                         float* Rw) {
  for (int k = lig; k < r.n; k += G) {
    const int j = r.jidx[k];
    const float th = j >= 0 ? joint_var(r, k, qs[j]) : 0.0f;
    local_xf(r, k, th, Rl + 12 * k, Rl + 12 * k + 9);
  }
  __syncwarp();
  for (int lev = 0; lev < r.nlev; ++lev) {
    const int s0 = r.lev_start[lev], s1 = r.lev_start[lev + 1];
    for (int i = s0 + lig; i < s1; i += G) {
      const int k = r.lev_links[i];
      const int pa = r.parent[k];
      float* W = Rw + 12 * k;
      const float* L = Rl + 12 * k;
      if (pa < 0) {
#pragma unroll
        for (int e = 0; e < 12; ++e) W[e] = L[e];
      } else {
        const float* P = Rw + 12 * pa;
        float R[9], t[3];
        matmul3(P, L, R);
        rot(P, L + 9, t);
#pragma unroll
        for (int e = 0; e < 9; ++e) W[e] = R[e];
        W[9] = P[9] + t[0];
        W[10] = P[10] + t[1];
        W[11] = P[11] + t[2];
      }
    }
    __syncwarp();
  }
}

// ---------------------------------------------------------------------------
// forward
// ---------------------------------------------------------------------------
template <int G>
__global__ void __launch_bounds__(256) fused_fwd_kernel(DevRobot r, PairSchedule ps, FwdArgs A,
                                                        int cpb) {
  extern __shared__ __align__(128) float smem[];
  const bool with_bits = A.bits != nullptr;
  const FwdPlan pl(r.n, r.d, r.Sg, r.P, with_bits);
  const int lane = threadIdx.x & 31;
  const int lig = lane & (G - 1);
  const int cfg = threadIdx.x / G;  // configuration slot in the tile
  const int64_t B = A.B;
  const int64_t ntiles = (B + cpb - 1) / cpb;
  float* cs = smem + (size_t)cfg * pl.total;
  const bool active_slot = cfg < cpb;
  const int W = (r.P + 31) >> 5;

  for (int64_t tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
    const int64_t b0 = tile * cpb;
    stage_rows(smem, pl.total, pl.q, A.q, r.d, B, b0, cpb);
    stage_rows(smem, pl.total, pl.q + r.d, A.qd, r.d, B, b0, cpb);
    stage_rows(smem, pl.total, pl.q + 2 * r.d, A.qdd, r.d, B, b0, cpb);
    __syncthreads();
    const int64_t b = b0 + cfg;
    const bool live = active_slot && b < B;
    if (active_slot) {
      float* qs = cs + pl.q;
      float* Rl = cs + pl.Rl;
      float* Rw = cs + pl.Rw;
      group_fk<G>(r, lig, qs, Rl, Rw);
      // ---- sphere centres (SoA by component, padded to whole groups) ----
      float* sx = cs + pl.sx;
      float* sy = cs + pl.sy;
      float* sz = cs + pl.sz;
      for (int s = lig; s < 4 * r.Sg; s += G) {
        float c[3] = {0.0f, 0.0f, 0.0f};
        if (s < r.S) {
          const float4 sp = __ldg(r.sph + s);
          const int l = r.sph_link[s];
          const float cl[3] = {sp.x, sp.y, sp.z};
          rot(Rw + 12 * l, cl, c);
          c[0] += Rw[12 * l + 9];
          c[1] += Rw[12 * l + 10];
          c[2] += Rw[12 * l + 11];
        }
        sx[s] = c[0];
        sy[s] = c[1];
        sz[s] = c[2];
      }
      if (with_bits)
        for (int w = lig; w < W; w += G) reinterpret_cast<uint32_t*>(cs + pl.bits)[w] = 0u;
      __syncwarp();
      // ---- outputs: poses and sphere centres (config-major, contiguous) ----
      if (live && A.pose) {
        float4* dst = reinterpret_cast<float4*>(A.pose + b * (int64_t)r.n * 12);
        const float4* srcp = reinterpret_cast<const float4*>(Rw);
        for (int e = lig; e < 3 * r.n; e += G) dst[e] = srcp[e];
      }
      if (live && A.sph) {
        float* dst = A.sph + b * (int64_t)r.S * 3;
        for (int e = lig; e < 3 * r.S; e += G) {
          const int s = e / 3, c = e - 3 * s;
          dst[e] = (c == 0 ? sx : (c == 1 ? sy : sz))[s];
        }
      }
      // ---- self-collision: map over the lane's blocks, reduce in the group ----
      if (A.dmin || with_bits) {
        const float4* sx4 = reinterpret_cast<const float4*>(sx);
        const float4* sy4 = reinterpret_cast<const float4*>(sy);
        const float4* sz4 = reinterpret_cast<const float4*>(sz);
        uint32_t* bm = reinterpret_cast<uint32_t*>(cs + pl.bits);
        float best = __int_as_float(0x7f800000);
        int bidx = INT_MAX;
        int cur = -1;
        float xi[4], yi[4], zi[4], ri[4], ti[4];
        const float margin = r.margin;
        for (int rr = 0; rr < ps.rounds; ++rr) {
          const uint2 e = __ldg(ps.ent + rr * G + lig);
          const uint32_t mask = e.x >> 16;
          if (mask == 0u) continue;
          const int gi = e.x & 0xFF, gj = (e.x >> 8) & 0xFF;
          if (gi != cur) {
            cur = gi;
            const float4 X = sx4[gi], Y = sy4[gi], Z = sz4[gi], Rr = __ldg(r.grp_rad + gi);
            xi[0] = X.x; xi[1] = X.y; xi[2] = X.z; xi[3] = X.w;
            yi[0] = Y.x; yi[1] = Y.y; yi[2] = Y.z; yi[3] = Y.w;
            zi[0] = Z.x; zi[1] = Z.y; zi[2] = Z.z; zi[3] = Z.w;
            ri[0] = Rr.x; ri[1] = Rr.y; ri[2] = Rr.z; ri[3] = Rr.w;
#pragma unroll
            for (int a = 0; a < 4; ++a) ti[a] = best + ri[a] + margin;
          }
          const float4 X = sx4[gj], Y = sy4[gj], Z = sz4[gj], Rr = __ldg(r.grp_rad + gj);
          const float xj[4] = {X.x, X.y, X.z, X.w};
          const float yj[4] = {Y.x, Y.y, Y.z, Y.w};
          const float zj[4] = {Z.x, Z.y, Z.z, Z.w};
          const float rj[4] = {Rr.x, Rr.y, Rr.z, Rr.w};
          float m = __int_as_float(0x7f800000);
          if (mask == 0xFFFFu) {
#pragma unroll
            for (int a = 0; a < 4; ++a)
#pragma unroll
              for (int c = 0; c < 4; ++c) {
                const float d2 = dist2(xi[a], yi[a], zi[a], xj[c], yj[c], zj[c]);
                const float t = ti[a] + rj[c];
                m = fminf(m, fmaf(-t, fabsf(t), d2));
              }
          } else {
#pragma unroll
            for (int a = 0; a < 4; ++a)
#pragma unroll
              for (int c = 0; c < 4; ++c) {
                const float d2 = dist2(xi[a], yi[a], zi[a], xj[c], yj[c], zj[c]);
                const float t = ti[a] + rj[c];
                const float ev = fmaf(-t, fabsf(t), d2);
                m = ((mask >> (4 * a + c)) & 1u) ? fminf(m, ev) : m;
              }
          }
          if (m < 0.0f) {
            // exact path: may improve (d, index)
#pragma unroll
            for (int a = 0; a < 4; ++a)
#pragma unroll
              for (int c = 0; c < 4; ++c) {
                if ((mask >> (4 * a + c)) & 1u) {
                  const float d2 = dist2(xi[a], yi[a], zi[a], xj[c], yj[c], zj[c]);
                  const float dd = sqrtf(d2) - (ri[a] + rj[c]);
                  if (dd <= best) {
                    const int pidx = __ldg(r.blk_pidx + 16 * e.y + 4 * a + c);
                    if (dd < best || pidx < bidx) {
                      best = dd;
                      bidx = pidx;
                    }
                  }
                }
              }
#pragma unroll
            for (int a = 0; a < 4; ++a) ti[a] = best + ri[a] + margin;
          }
          if (with_bits) {
#pragma unroll
            for (int a = 0; a < 4; ++a)
#pragma unroll
              for (int c = 0; c < 4; ++c) {
                if ((mask >> (4 * a + c)) & 1u) {
                  const float d2 = dist2(xi[a], yi[a], zi[a], xj[c], yj[c], zj[c]);
                  if (sqrtf(d2) - (ri[a] + rj[c]) < 0.0f) {
                    const int pidx = __ldg(r.blk_pidx + 16 * e.y + 4 * a + c);
                    atomicOr(bm + (pidx >> 5), 1u << (pidx & 31));
                  }
                }
              }
          }
        }
        group_min<G>(best, bidx);
        if (live && lig == 0 && A.dmin) {
          A.dmin[b] = best;
          A.worst[b] = bidx == INT_MAX ? -1 : bidx;
        }
        if (with_bits) {
          __syncwarp();
          if (live)
            for (int w = lig; w < W; w += G) A.bits[b * (int64_t)W + w] = bm[w];
        }
      }
      __syncwarp();
      // ---- RNEA (Alg. 4) ----
      if (A.tau) {
        float* v = cs + pl.v;
        float* a = cs + pl.a;
        float* F = cs + pl.F;
        float* tl = cs + pl.tl;
        const float* qd = qs + r.d;
        const float* qdd = qs + 2 * r.d;
        const float zero6[6] = {0, 0, 0, 0, 0, 0};
        const float ab6[6] = {0, 0, 0, r.abase[0], r.abase[1], r.abase[2]};
        for (int lev = 0; lev < r.nlev; ++lev) {
          const int s0 = r.lev_start[lev], s1 = r.lev_start[lev + 1];
          for (int i = s0 + lig; i < s1; i += G) {
            const int k = r.lev_links[i];
            const int pa = r.parent[k];
            const int j = r.jidx[k];
            const float4 ax4 = __ldg(reinterpret_cast<const float4*>(r.axis) + k);
            const float ax[3] = {ax4.x, ax4.y, ax4.z};
            const float mm = __ldg(reinterpret_cast<const float2*>(r.mimic) + k).x;
            const float vq = j >= 0 ? mm * qd[j] : 0.0f;
            const float aq = j >= 0 ? mm * qdd[j] : 0.0f;
            rnea_va(Rl + 12 * k, Rl + 12 * k + 9, pa < 0 ? zero6 : v + 6 * pa,
                    pa < 0 ? ab6 : a + 6 * pa, r.jtype[k], ax, vq, aq, v + 6 * k, a + 6 * k);
          }
          __syncwarp();
        }
        for (int k = lig; k < r.n; k += G) {
          float I[10], f[6];
          load_inertia(r, k, I);
          rnea_force(I, v + 6 * k, a + 6 * k, f);
#pragma unroll
          for (int e = 0; e < 6; ++e) F[6 * k + e] = f[e];
        }
        __syncwarp();
        // tips -> base: F_k = f_k + sum over children of X_c^T F_c (each child
        // leaves its X^T F in its own v slot, which is dead after pass 2)
        for (int lev = r.nlev - 1; lev >= 0; --lev) {
          const int s0 = r.lev_start[lev], s1 = r.lev_start[lev + 1];
          for (int i = s0 + lig; i < s1; i += G) {
            const int k = r.lev_links[i];
            float f[6];
#pragma unroll
            for (int e = 0; e < 6; ++e) f[e] = F[6 * k + e];
            for (int ci = r.child_start[k]; ci < r.child_start[k + 1]; ++ci) {
              const int c = r.children[ci];
#pragma unroll
              for (int e = 0; e < 6; ++e) f[e] += v[6 * c + e];
            }
            const float4 ax4 = __ldg(reinterpret_cast<const float4*>(r.axis) + k);
            const float ax[3] = {ax4.x, ax4.y, ax4.z};
            tl[k] = St_dot(r.jtype[k], ax, f);
            if (r.parent[k] >= 0) {
              float up[6];
              xf_force_T(Rl + 12 * k, Rl + 12 * k + 9, f, up);
#pragma unroll
              for (int e = 0; e < 6; ++e) v[6 * k + e] = up[e];
            }
          }
          __syncwarp();
        }
        // per joint: tau_j = sum over driven links of m_k S_k^T F_k
        for (int j = lig; j < r.d; j += G) {
          float t = 0.0f;
          for (int e = r.jl_start[j]; e < r.jl_start[j + 1]; ++e) {
            const int k = r.jl_links[e];
            t = fmaf(__ldg(reinterpret_cast<const float2*>(r.mimic) + k).x, tl[k], t);
          }
          qs[j] = t;  // q is dead after FK: stage tau in its slot
        }
      }
    }
    __syncthreads();
    if (A.tau) unstage_rows(smem, pl.total, pl.q, A.tau, r.d, B, b0, cpb);
    __syncthreads();
  }
}

// ---------------------------------------------------------------------------
// backward
// ---------------------------------------------------------------------------
__device__ __forceinline__ void motion_S6(int jt, const float* ax, float* S) {
  S[0] = S[1] = S[2] = S[3] = S[4] = S[5] = 0.0f;
  if (jt == 1) {
    S[0] = ax[0]; S[1] = ax[1]; S[2] = ax[2];
  } else if (jt == 2) {
    S[3] = ax[0]; S[4] = ax[1]; S[5] = ax[2];
  }
}

__device__ __forceinline__ float dot6f(const float* a, const float* b) {
  float s = 0.0f;
#pragma unroll
  for (int i = 0; i < 6; ++i) s = fmaf(a[i], b[i], s);
  return s;
}

// add the link-frame wrench of a world-frame point gradient g acting at the
// sphere with local centre (sp.xyz) on link l
__device__ __forceinline__ void add_point_wrench(const float* Rw_l, float4 sp, const float* g,
                                                 float* w) {
  float f[3], nn[3];
  rotT(Rw_l, g, f);
  const float c[3] = {sp.x, sp.y, sp.z};
  cross3(c, f, nn);
  w[0] += nn[0];
  w[1] += nn[1];
  w[2] += nn[2];
  w[3] += f[0];
  w[4] += f[1];
  w[5] += f[2];
}

template <int G>
__global__ void __launch_bounds__(256) fused_bwd_kernel(DevRobot r, BwdArgs A, int cpb) {
  extern __shared__ __align__(128) float smem[];
  const BwdPlan pl(r.n, r.d);
  const int lane = threadIdx.x & 31;
  const int lig = lane & (G - 1);
  const int cfg = threadIdx.x / G;
  const int64_t B = A.B;
  const int64_t ntiles = (B + cpb - 1) / cpb;
  float* cs = smem + (size_t)cfg * pl.total;
  const bool active_slot = cfg < cpb;
  const int n = r.n, d = r.d;
  const float zero6[6] = {0, 0, 0, 0, 0, 0};
  const float ab6[6] = {0, 0, 0, r.abase[0], r.abase[1], r.abase[2]};

  for (int64_t tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
    const int64_t b0 = tile * cpb;
    stage_rows(smem, pl.total, pl.q, A.q, d, B, b0, cpb);
    stage_rows(smem, pl.total, pl.q + d, A.qd, d, B, b0, cpb);
    stage_rows(smem, pl.total, pl.q + 2 * d, A.qdd, d, B, b0, cpb);
    stage_rows(smem, pl.total, pl.q + 3 * d, A.g_tau, d, B, b0, cpb);
    __syncthreads();
    const int64_t b = b0 + cfg;
    const bool live = active_slot && b < B;
    if (active_slot) {
      float* qs = cs + pl.q;
      const float* qd = qs + d;
      const float* qdd = qs + 2 * d;
      const float* gt = qs + 3 * d;
      float* Rl = cs + pl.Rl;
      float* Rw = cs + pl.Rw;
      float* v = cs + pl.va;
      float* a = cs + pl.va + 6 * n;
      float* F = cs + pl.F;
      float* Wr = cs + pl.W;
      group_fk<G>(r, lig, qs, Rl, Rw);
      // ---- gradient wrenches of the kinematic outputs, link frame ----
      for (int k = lig; k < n; k += G) {
        float w[6] = {0, 0, 0, 0, 0, 0};
        const float* R = Rw + 12 * k;
        if (live && A.g_pose) {
          const float* g = A.g_pose + (b * n + k) * 12;
          float gg[12];
#pragma unroll
          for (int e = 0; e < 12; ++e) gg[e] = g[e];
          float Gm[9];  // R^T Rbar
#pragma unroll
          for (int i = 0; i < 3; ++i)
#pragma unroll
            for (int jj = 0; jj < 3; ++jj)
              Gm[3 * i + jj] =
                  fmaf(R[6 + i], gg[6 + jj], fmaf(R[3 + i], gg[3 + jj], R[i] * gg[jj]));
          w[0] = Gm[7] - Gm[5];
          w[1] = Gm[2] - Gm[6];
          w[2] = Gm[3] - Gm[1];
          rotT(R, gg + 9, w + 3);
        }
        if (live && A.g_sph) {
          for (int e = r.ls_start[k]; e < r.ls_start[k + 1]; ++e) {
            const int s = r.ls_sph[e];
            const float* g = A.g_sph + (b * r.S + s) * 3;
            const float gg[3] = {g[0], g[1], g[2]};
            add_point_wrench(R, __ldg(r.sph + s), gg, w);
          }
        }
#pragma unroll
        for (int e = 0; e < 6; ++e) Wr[6 * k + e] = w[e];
      }
      __syncwarp();
      if (live && A.g_dmin && lig == 0) {
        const int wp = A.worst[b];
        const float gd = A.g_dmin[b];
        if (wp >= 0 && wp < r.P) {
          const int2 ij = r.pairs[wp];
          const float4 si = __ldg(r.sph + ij.x), sj = __ldg(r.sph + ij.y);
          const int l1 = r.sph_link[ij.x], l2 = r.sph_link[ij.y];
          float ci[3], cj[3];
          const float li[3] = {si.x, si.y, si.z}, lj[3] = {sj.x, sj.y, sj.z};
          rot(Rw + 12 * l1, li, ci);
          rot(Rw + 12 * l2, lj, cj);
          const float dx = (ci[0] + Rw[12 * l1 + 9]) - (cj[0] + Rw[12 * l2 + 9]);
          const float dy = (ci[1] + Rw[12 * l1 + 10]) - (cj[1] + Rw[12 * l2 + 10]);
          const float dz = (ci[2] + Rw[12 * l1 + 11]) - (cj[2] + Rw[12 * l2 + 11]);
          const float nrm = sqrtf(fmaf(dz, dz, fmaf(dy, dy, dx * dx)));
          const float sc = nrm > 0.0f ? gd / nrm : 0.0f;
          const float u[3] = {dx * sc, dy * sc, dz * sc};
          const float mu[3] = {-u[0], -u[1], -u[2]};
          add_point_wrench(Rw + 12 * l1, si, u, Wr + 6 * l1);
          add_point_wrench(Rw + 12 * l2, sj, mu, Wr + 6 * l2);
        }
      }
      __syncwarp();
      // ---- dynamics forward recompute: v, a, then accumulated F ----
      for (int lev = 0; lev < r.nlev; ++lev) {
        const int s0 = r.lev_start[lev], s1 = r.lev_start[lev + 1];
        for (int i = s0 + lig; i < s1; i += G) {
          const int k = r.lev_links[i];
          const int pa = r.parent[k];
          const int j = r.jidx[k];
          const float4 ax4 = __ldg(reinterpret_cast<const float4*>(r.axis) + k);
          const float ax[3] = {ax4.x, ax4.y, ax4.z};
          const float mm = __ldg(reinterpret_cast<const float2*>(r.mimic) + k).x;
          const float vq = j >= 0 ? mm * qd[j] : 0.0f;
          const float aq = j >= 0 ? mm * qdd[j] : 0.0f;
          rnea_va(Rl + 12 * k, Rl + 12 * k + 9, pa < 0 ? zero6 : v + 6 * pa,
                  pa < 0 ? ab6 : a + 6 * pa, r.jtype[k], ax, vq, aq, v + 6 * k, a + 6 * k);
        }
        __syncwarp();
      }
      for (int k = lig; k < n; k += G) {
        float I[10], f[6];
        load_inertia(r, k, I);
        rnea_force(I, v + 6 * k, a + 6 * k, f);
#pragma unroll
        for (int e = 0; e < 6; ++e) F[6 * k + e] = f[e];
      }
      __syncwarp();
      float* up = cs + pl.up;  // Rw is dead from here on
      for (int lev = r.nlev - 1; lev >= 0; --lev) {
        const int s0 = r.lev_start[lev], s1 = r.lev_start[lev + 1];
        for (int i = s0 + lig; i < s1; i += G) {
          const int k = r.lev_links[i];
          float f[6];
#pragma unroll
          for (int e = 0; e < 6; ++e) f[e] = F[6 * k + e];
          for (int ci = r.child_start[k]; ci < r.child_start[k + 1]; ++ci) {
            const int c = r.children[ci];
#pragma unroll
            for (int e = 0; e < 6; ++e) f[e] += up[6 * c + e];
          }
#pragma unroll
          for (int e = 0; e < 6; ++e) F[6 * k + e] = f[e];
          if (r.parent[k] >= 0) {
            float u6[6];
            xf_force_T(Rl + 12 * k, Rl + 12 * k + 9, f, u6);
#pragma unroll
            for (int e = 0; e < 6; ++e) up[6 * k + e] = u6[e];
          }
        }
        __syncwarp();
      }
      float* vb = cs + pl.vb;
      float* lq = cs + pl.lq;
      // ---- adjoint of the force sweep, base -> tips (F slot: F -> Fbar) ----
      for (int lev = 0; lev < r.nlev; ++lev) {
        const int s0 = r.lev_start[lev], s1 = r.lev_start[lev + 1];
        for (int i = s0 + lig; i < s1; i += G) {
          const int k = r.lev_links[i];
          const int pa = r.parent[k];
          const int j = r.jidx[k];
          const float4 ax4 = __ldg(reinterpret_cast<const float4*>(r.axis) + k);
          const float ax[3] = {ax4.x, ax4.y, ax4.z};
          float S[6];
          motion_S6(r.jtype[k], ax, S);
          const float mm = __ldg(reinterpret_cast<const float2*>(r.mimic) + k).x;
          const float tb = j >= 0 ? mm * gt[j] : 0.0f;
          float XF[6], cS[6], Fk[6];
          if (pa >= 0)
            xf_motion(Rl + 12 * k, Rl + 12 * k + 9, F + 6 * pa, XF);
          else
#pragma unroll
            for (int e = 0; e < 6; ++e) XF[e] = 0.0f;
#pragma unroll
          for (int e = 0; e < 6; ++e) Fk[e] = F[6 * k + e];
          crf(S, Fk, cS);
          lq[3 * k] = dot6f(XF, cS);
#pragma unroll
          for (int e = 0; e < 6; ++e) F[6 * k + e] = fmaf(S[e], tb, XF[e]);
        }
        __syncwarp();
      }
      // ---- adjoint of the per-link force (F slot: Fbar -> abar) ----
      for (int k = lig; k < n; k += G) {
        float I[10], Fb[6], Iv[6], t1[6], t2[6], t3[6], ab[6];
        load_inertia(r, k, I);
#pragma unroll
        for (int e = 0; e < 6; ++e) Fb[e] = F[6 * k + e];
        inertia_mul(I, Fb, ab);
        inertia_mul(I, v + 6 * k, Iv);
        crf(Fb, Iv, t1);
        crm(v + 6 * k, Fb, t2);
        inertia_mul(I, t2, t3);
#pragma unroll
        for (int e = 0; e < 6; ++e) {
          F[6 * k + e] = ab[e];
          vb[6 * k + e] = -t1[e] - t3[e];
        }
      }
      __syncwarp();
      // ---- adjoint of the velocity/acceleration sweep and FK, tips -> base ----
      for (int lev = r.nlev - 1; lev >= 0; --lev) {
        const int s0 = r.lev_start[lev], s1 = r.lev_start[lev + 1];
        for (int i = s0 + lig; i < s1; i += G) {
          const int k = r.lev_links[i];
          const int pa = r.parent[k];
          const int j = r.jidx[k];
          const int jt = r.jtype[k];
          const float4 ax4 = __ldg(reinterpret_cast<const float4*>(r.axis) + k);
          const float ax[3] = {ax4.x, ax4.y, ax4.z};
          float S[6];
          motion_S6(jt, ax, S);
          const float mm = __ldg(reinterpret_cast<const float2*>(r.mimic) + k).x;
          const float vq = j >= 0 ? mm * qd[j] : 0.0f;
          float ab[6], vbk[6], w[6];
#pragma unroll
          for (int e = 0; e < 6; ++e) {
            ab[e] = F[6 * k + e];
            vbk[e] = vb[6 * k + e];
            w[e] = Wr[6 * k + e];
          }
          for (int ci = r.child_start[k]; ci < r.child_start[k + 1]; ++ci) {
            const int c = r.children[ci];
#pragma unroll
            for (int e = 0; e < 6; ++e) {
              ab[e] += F[6 * c + e];
              vbk[e] += vb[6 * c + e];
              w[e] += Wr[6 * c + e];
            }
          }
          float t[6];
          crf(S, ab, t);
#pragma unroll
          for (int e = 0; e < 6; ++e) vbk[e] = fmaf(vq, t[e], vbk[e]);
          const float gqdd = dot6f(S, ab);
          crf(v + 6 * k, ab, t);
          const float gqd = dot6f(S, vbk) - dot6f(S, t);
          float Xa[6], Xv[6], c6[6];
          xf_motion(Rl + 12 * k, Rl + 12 * k + 9, pa < 0 ? ab6 : a + 6 * pa, Xa);
          xf_motion(Rl + 12 * k, Rl + 12 * k + 9, pa < 0 ? zero6 : v + 6 * pa, Xv);
          float gq = lq[3 * k];
          crm(S, Xa, c6);
          gq -= dot6f(ab, c6);
          crm(S, Xv, c6);
          gq -= dot6f(vbk, c6);
          gq += dot6f(S, w);
          lq[3 * k] = gq;
          lq[3 * k + 1] = gqd;
          lq[3 * k + 2] = gqdd;
          if (pa >= 0) {
            float u6[6];
            xf_force_T(Rl + 12 * k, Rl + 12 * k + 9, ab, u6);
#pragma unroll
            for (int e = 0; e < 6; ++e) F[6 * k + e] = u6[e];
            xf_force_T(Rl + 12 * k, Rl + 12 * k + 9, vbk, u6);
#pragma unroll
            for (int e = 0; e < 6; ++e) vb[6 * k + e] = u6[e];
            xf_force_T(Rl + 12 * k, Rl + 12 * k + 9, w, u6);
#pragma unroll
            for (int e = 0; e < 6; ++e) Wr[6 * k + e] = u6[e];
          }
        }
        __syncwarp();
      }
      // ---- per joint (mimic joints sum their links); stage in q slots ----
      for (int jj = lig; jj < d; jj += G) {
        float g0 = 0.0f, g1 = 0.0f, g2 = 0.0f;
        for (int e = r.jl_start[jj]; e < r.jl_start[jj + 1]; ++e) {
          const int k = r.jl_links[e];
          const float mm = __ldg(reinterpret_cast<const float2*>(r.mimic) + k).x;
          g0 = fmaf(mm, lq[3 * k], g0);
          g1 = fmaf(mm, lq[3 * k + 1], g1);
          g2 = fmaf(mm, lq[3 * k + 2], g2);
        }
        qs[jj] = g0;
        qs[d + jj] = g1;
        qs[2 * d + jj] = g2;
      }
    }
    __syncthreads();
    unstage_rows(smem, pl.total, pl.q, A.gq, d, B, b0, cpb);
    unstage_rows(smem, pl.total, pl.q + d, A.gqd, d, B, b0, cpb);
    unstage_rows(smem, pl.total, pl.q + 2 * d, A.gqdd, d, B, b0, cpb);
    __syncthreads();
  }
}

// ---------------------------------------------------------------------------
// launchers
// ---------------------------------------------------------------------------
template <int G>
static cudaError_t fwd_launch_t(const DevRobot& r, const PairSchedule& ps, const FwdArgs& a,
                                const FusedShape& sh, cudaStream_t s) {
  auto kern = fused_fwd_kernel<G>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)sh.smem);
  if (e != cudaSuccess) return e;
  const int threads = ((sh.cpb * G + 31) / 32) * 32;
  kern<<<sh.grid, threads, sh.smem, s>>>(r, ps, a, sh.cpb);
  return cudaGetLastError();
}

template <int G>
static cudaError_t bwd_launch_t(const DevRobot& r, const BwdArgs& a, const FusedShape& sh,
                                cudaStream_t s) {
  auto kern = fused_bwd_kernel<G>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)sh.smem);
  if (e != cudaSuccess) return e;
  const int threads = ((sh.cpb * G + 31) / 32) * 32;
  kern<<<sh.grid, threads, sh.smem, s>>>(r, a, sh.cpb);
  return cudaGetLastError();
}

cudaError_t launch_fused_fwd(const DevRobot& r, const PairSchedule& ps, const FwdArgs& a,
                             const FusedShape& sh, cudaStream_t s) {
  switch (sh.G) {
    case 4: return fwd_launch_t<4>(r, ps, a, sh, s);
    case 8: return fwd_launch_t<8>(r, ps, a, sh, s);
    case 16: return fwd_launch_t<16>(r, ps, a, sh, s);
    case 32: return fwd_launch_t<32>(r, ps, a, sh, s);
    default: return cudaErrorInvalidValue;
  }
}

cudaError_t launch_fused_bwd(const DevRobot& r, const BwdArgs& a, const FusedShape& sh,
                             cudaStream_t s) {
  switch (sh.G) {
    case 4: return bwd_launch_t<4>(r, a, sh, s);
    case 8: return bwd_launch_t<8>(r, a, sh, s);
    case 16: return bwd_launch_t<16>(r, a, sh, s);
    case 32: return bwd_launch_t<32>(r, a, sh, s);
    default: return cudaErrorInvalidValue;
  }
}

template <int G>
static cudaError_t occ_fwd_t(int cpb, size_t smem, int* out) {
  auto kern = fused_fwd_kernel<G>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)smem);
  if (e != cudaSuccess) return e;
  const int threads = ((cpb * G + 31) / 32) * 32;
  return cudaOccupancyMaxActiveBlocksPerMultiprocessor(out, kern, threads, smem);
}
template <int G>
static cudaError_t occ_bwd_t(int cpb, size_t smem, int* out) {
  auto kern = fused_bwd_kernel<G>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)smem);
  if (e != cudaSuccess) return e;
  const int threads = ((cpb * G + 31) / 32) * 32;
  return cudaOccupancyMaxActiveBlocksPerMultiprocessor(out, kern, threads, smem);
}

cudaError_t fused_fwd_max_blocks_per_sm(int G, int cpb, size_t smem, int* out) {
  switch (G) {
    case 4: return occ_fwd_t<4>(cpb, smem, out);
    case 8: return occ_fwd_t<8>(cpb, smem, out);
    case 16: return occ_fwd_t<16>(cpb, smem, out);
    case 32: return occ_fwd_t<32>(cpb, smem, out);
    default: return cudaErrorInvalidValue;
  }
}
cudaError_t fused_bwd_max_blocks_per_sm(int G, int cpb, size_t smem, int* out) {
  switch (G) {
    case 4: return occ_bwd_t<4>(cpb, smem, out);
    case 8: return occ_bwd_t<8>(cpb, smem, out);
    case 16: return occ_bwd_t<16>(cpb, smem, out);
    case 32: return occ_bwd_t<32>(cpb, smem, out);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace wbe
