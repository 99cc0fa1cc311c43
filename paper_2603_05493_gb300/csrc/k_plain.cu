// k_plain.cu -- the plain whole-body kernels: one thread per configuration,
// every stage in straight code over per-thread (local/global) memory.  They
// are the baseline the fused kernels are measured against and stay in the
// library as the reference GPU path.
//
// Forward (Sec. 6): FK in index order (parent[k] < k), sphere centres, all
// masked pairs in pair-index order (strict '<' keeps the smallest index on
// ties), RNEA (Alg. 4).
// Backward: the vector-Jacobian product of the same evaluation.  The RNEA
// adjoint is derived from Alg. 4 by reverse-mode differentiation (Alg. 5
// gives its structure); two terms that Alg. 5's listing does not show are
// included because the derivative requires them:
//   * the root link's a_k = X_k a_base depends on q_root, so the term
//     -a_bar^T crm(S) X a_pa is applied to the root too (a_pa = a_base);
//   * a_k depends on v_k through v_k x_m (S qd), so v_bar += crf(S qd) a_bar
//     before v_bar is used.
// The kinematic adjoint (Alg. 1) is computed as subtree sums of link-frame
// gradient wrenches: q_bar_j += S_j^T W_j with W accumulated tips -> base by
// the same X^T map that carries forces.
#include "spatial.cuh"

namespace wbe {

constexpr int PMAXL = 64;   // plain-kernel limits (larger robots use the fused path)
constexpr int PMAXS = 256;

__device__ __forceinline__ void motion_S(int jt, const float* ax, float* S) {
  S[0] = S[1] = S[2] = S[3] = S[4] = S[5] = 0.0f;
  if (jt == 1) {
    S[0] = ax[0]; S[1] = ax[1]; S[2] = ax[2];
  } else if (jt == 2) {
    S[3] = ax[0]; S[4] = ax[1]; S[5] = ax[2];
  }
}

__device__ __forceinline__ float dot6(const float* a, const float* b) {
  float s = 0.0f;
#pragma unroll
  for (int i = 0; i < 6; ++i) s = fmaf(a[i], b[i], s);
  return s;
}

__global__ void __launch_bounds__(128) plain_fwd_kernel(DevRobot r, FwdArgs A) {
  const int64_t b = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (b >= A.B) return;
  const int64_t B = A.B;
  const int n = r.n;
  float Rl[PMAXL][12];
  float Rw[PMAXL][12];
  // ---- forward kinematics, index order ----
  for (int k = 0; k < n; ++k) {
    const int j = r.jidx[k];
    const float th = j >= 0 ? joint_var(r, k, A.q[j * B + b]) : 0.0f;
    local_xf(r, k, th, Rl[k], Rl[k] + 9);
    const int pa = r.parent[k];
    if (pa < 0) {
      for (int i = 0; i < 12; ++i) Rw[k][i] = Rl[k][i];
    } else {
      float t[3];
      matmul3(Rw[pa], Rl[k], Rw[k]);
      rot(Rw[pa], Rl[k] + 9, t);
      for (int i = 0; i < 3; ++i) Rw[k][9 + i] = Rw[pa][9 + i] + t[i];
    }
    if (A.pose)
      for (int i = 0; i < 12; ++i) A.pose[(b * n + k) * 12 + i] = Rw[k][i];
  }
  // ---- sphere centres ----
  float cs[PMAXS][3];
  for (int s = 0; s < r.S; ++s) {
    const float4 sp = r.sph[s];
    const int l = r.sph_link[s];
    const float c[3] = {sp.x, sp.y, sp.z};
    float t[3];
    rot(Rw[l], c, t);
    for (int i = 0; i < 3; ++i) {
      cs[s][i] = t[i] + Rw[l][9 + i];
      if (A.sph) A.sph[(b * r.S + s) * 3 + i] = cs[s][i];
    }
  }
  // ---- self-collision, every masked pair ----
  if (A.dmin || A.bits) {
    float best = __int_as_float(0x7f800000);
    int bi = -1;
    const int W = (r.P + 31) >> 5;
    uint32_t word = 0;
    for (int p = 0; p < r.P; ++p) {
      const int2 ij = r.pairs[p];
      const float d2 = dist2(cs[ij.x][0], cs[ij.x][1], cs[ij.x][2], cs[ij.y][0], cs[ij.y][1],
                             cs[ij.y][2]);
      const float d = sqrtf(d2) - (r.sph[ij.x].w + r.sph[ij.y].w);
      if (d < best) {
        best = d;
        bi = p;
      }
      if (A.bits) {
        if (d < 0.0f) word |= 1u << (p & 31);
        if ((p & 31) == 31 || p == r.P - 1) {
          A.bits[b * W + (p >> 5)] = word;
          word = 0;
        }
      }
    }
    if (A.dmin) {
      A.dmin[b] = best;
      A.worst[b] = bi;
    }
  }
  // ---- RNEA (Alg. 4) ----
  if (A.tau) {
    float v[PMAXL][6], a[PMAXL][6], f[PMAXL][6];
    const float zero6[6] = {0, 0, 0, 0, 0, 0};
    const float ab6[6] = {0, 0, 0, r.abase[0], r.abase[1], r.abase[2]};
    for (int k = 0; k < n; ++k) {
      const int pa = r.parent[k];
      const int j = r.jidx[k];
      const int jt = r.jtype[k];
      const float4 ax4 = r.axis ? reinterpret_cast<const float4*>(r.axis)[k] : float4{};
      const float ax[3] = {ax4.x, ax4.y, ax4.z};
      const float mm = reinterpret_cast<const float2*>(r.mimic)[k].x;
      const float qd = j >= 0 ? mm * A.qd[j * B + b] : 0.0f;
      const float qdd = j >= 0 ? mm * A.qdd[j * B + b] : 0.0f;
      rnea_va(Rl[k], Rl[k] + 9, pa < 0 ? zero6 : v[pa], pa < 0 ? ab6 : a[pa], jt, ax, qd, qdd,
              v[k], a[k]);
    }
    for (int k = 0; k < n; ++k) {
      float I[10];
      load_inertia(r, k, I);
      rnea_force(I, v[k], a[k], f[k]);
      if (A.fext)
        for (int i = 0; i < 6; ++i) f[k][i] -= A.fext[(b * n + k) * 6 + i];
    }
    for (int j = 0; j < r.d; ++j) A.tau[j * B + b] = 0.0f;
    for (int k = n - 1; k >= 0; --k) {
      const int j = r.jidx[k];
      const int jt = r.jtype[k];
      if (j >= 0) {
        const float4 ax4 = reinterpret_cast<const float4*>(r.axis)[k];
        const float ax[3] = {ax4.x, ax4.y, ax4.z};
        const float mm = reinterpret_cast<const float2*>(r.mimic)[k].x;
        A.tau[j * B + b] += mm * St_dot(jt, ax, f[k]);
      }
      const int pa = r.parent[k];
      if (pa >= 0) {
        float up[6];
        xf_force_T(Rl[k], Rl[k] + 9, f[k], up);
        for (int i = 0; i < 6; ++i) f[pa][i] += up[i];
      }
    }
  }
}

__global__ void __launch_bounds__(128) plain_bwd_kernel(DevRobot r, BwdArgs A) {
  const int64_t b = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (b >= A.B) return;
  const int64_t B = A.B;
  const int n = r.n;
  float Rl[PMAXL][12], Rw[PMAXL][12];
  float v[PMAXL][6], a[PMAXL][6], F[PMAXL][6], Fb[PMAXL][6];
  float ab[PMAXL][6], vb[PMAXL][6], Wr[PMAXL][6];
  float qb[PMAXL], qdb[PMAXL], qddb[PMAXL];
  const float zero6[6] = {0, 0, 0, 0, 0, 0};
  const float ab6[6] = {0, 0, 0, r.abase[0], r.abase[1], r.abase[2]};
  // ---- FK recompute ----
  for (int k = 0; k < n; ++k) {
    const int j = r.jidx[k];
    const float th = j >= 0 ? joint_var(r, k, A.q[j * B + b]) : 0.0f;
    local_xf(r, k, th, Rl[k], Rl[k] + 9);
    const int pa = r.parent[k];
    if (pa < 0) {
      for (int i = 0; i < 12; ++i) Rw[k][i] = Rl[k][i];
    } else {
      float t[3];
      matmul3(Rw[pa], Rl[k], Rw[k]);
      rot(Rw[pa], Rl[k] + 9, t);
      for (int i = 0; i < 3; ++i) Rw[k][9 + i] = Rw[pa][9 + i] + t[i];
    }
  }
  // ---- link-frame gradient wrenches from pose, sphere and pair gradients ----
  for (int k = 0; k < n; ++k) {
    for (int i = 0; i < 6; ++i) Wr[k][i] = 0.0f;
    if (A.g_pose) {
      const float* g = A.g_pose + (b * n + k) * 12;
      const float* R = Rw[k];
      float G[9];  // G = R^T Rbar
      for (int i = 0; i < 3; ++i)
        for (int jj = 0; jj < 3; ++jj)
          G[3 * i + jj] = R[i] * g[jj] + R[3 + i] * g[3 + jj] + R[6 + i] * g[6 + jj];
      Wr[k][0] = G[7] - G[5];
      Wr[k][1] = G[2] - G[6];
      Wr[k][2] = G[3] - G[1];
      rotT(R, g + 9, Wr[k] + 3);
    }
  }
  if (A.g_sph) {
    for (int s = 0; s < r.S; ++s) {
      const int l = r.sph_link[s];
      const float* g = A.g_sph + (b * r.S + s) * 3;
      float f[3], nn[3];
      rotT(Rw[l], g, f);
      const float4 sp = r.sph[s];
      const float c[3] = {sp.x, sp.y, sp.z};
      cross3(c, f, nn);
      for (int i = 0; i < 3; ++i) {
        Wr[l][i] += nn[i];
        Wr[l][3 + i] += f[i];
      }
    }
  }
  if (A.g_dmin) {
    const int w = A.worst[b];
    const float gd = A.g_dmin[b];
    if (w >= 0 && w < r.P) {
      const int2 ij = r.pairs[w];
      float ci[3], cj[3];
      {
        const float4 si = r.sph[ij.x], sj = r.sph[ij.y];
        const float li[3] = {si.x, si.y, si.z}, lj[3] = {sj.x, sj.y, sj.z};
        const int a1 = r.sph_link[ij.x], a2 = r.sph_link[ij.y];
        rot(Rw[a1], li, ci);
        rot(Rw[a2], lj, cj);
        for (int i = 0; i < 3; ++i) {
          ci[i] += Rw[a1][9 + i];
          cj[i] += Rw[a2][9 + i];
        }
      }
      const float dx = ci[0] - cj[0], dy = ci[1] - cj[1], dz = ci[2] - cj[2];
      const float nrm = sqrtf(fmaf(dz, dz, fmaf(dy, dy, dx * dx)));
      const float sc = nrm > 0.0f ? gd / nrm : 0.0f;
      const float u[3] = {dx * sc, dy * sc, dz * sc};
      for (int side = 0; side < 2; ++side) {
        const int s = side == 0 ? ij.x : ij.y;
        const int l = r.sph_link[s];
        const float g[3] = {side == 0 ? u[0] : -u[0], side == 0 ? u[1] : -u[1],
                            side == 0 ? u[2] : -u[2]};
        float f[3], nn[3];
        rotT(Rw[l], g, f);
        const float4 sp = r.sph[s];
        const float c[3] = {sp.x, sp.y, sp.z};
        cross3(c, f, nn);
        for (int i = 0; i < 3; ++i) {
          Wr[l][i] += nn[i];
          Wr[l][3 + i] += f[i];
        }
      }
    }
  }
  // ---- RNEA forward recompute (v, a, accumulated F) ----
  for (int k = 0; k < n; ++k) {
    const int pa = r.parent[k];
    const int j = r.jidx[k];
    const float4 ax4 = reinterpret_cast<const float4*>(r.axis)[k];
    const float ax[3] = {ax4.x, ax4.y, ax4.z};
    const float mm = reinterpret_cast<const float2*>(r.mimic)[k].x;
    const float qd = j >= 0 ? mm * A.qd[j * B + b] : 0.0f;
    const float qdd = j >= 0 ? mm * A.qdd[j * B + b] : 0.0f;
    rnea_va(Rl[k], Rl[k] + 9, pa < 0 ? zero6 : v[pa], pa < 0 ? ab6 : a[pa], r.jtype[k], ax, qd,
            qdd, v[k], a[k]);
  }
  for (int k = 0; k < n; ++k) {
    float I[10];
    load_inertia(r, k, I);
    rnea_force(I, v[k], a[k], F[k]);
    if (A.fext)
      for (int i = 0; i < 6; ++i) F[k][i] -= A.fext[(b * n + k) * 6 + i];
  }
  for (int k = n - 1; k >= 0; --k) {
    const int pa = r.parent[k];
    if (pa >= 0) {
      float up[6];
      xf_force_T(Rl[k], Rl[k] + 9, F[k], up);
      for (int i = 0; i < 6; ++i) F[pa][i] += up[i];
    }
  }
  // ---- adjoint of the force sweep (base -> tips) ----
  for (int k = 0; k < n; ++k) {
    const int pa = r.parent[k];
    const int j = r.jidx[k];
    const float4 ax4 = reinterpret_cast<const float4*>(r.axis)[k];
    const float ax[3] = {ax4.x, ax4.y, ax4.z};
    float S[6];
    motion_S(r.jtype[k], ax, S);
    const float mm = reinterpret_cast<const float2*>(r.mimic)[k].x;
    const float tb = (j >= 0 && A.g_tau) ? mm * A.g_tau[j * B + b] : 0.0f;
    float XF[6];
    if (pa >= 0)
      xf_motion(Rl[k], Rl[k] + 9, Fb[pa], XF);
    else
      for (int i = 0; i < 6; ++i) XF[i] = 0.0f;
    float cS[6];
    crf(S, F[k], cS);
    qb[k] = dot6(XF, cS);
    for (int i = 0; i < 6; ++i) Fb[k][i] = fmaf(S[i], tb, XF[i]);
    if (A.g_fext)  // dL/df_ext,k = -Fbar_k
      for (int i = 0; i < 6; ++i) A.g_fext[(b * n + k) * 6 + i] = -Fb[k][i];
  }
  // ---- adjoint of the per-link force ----
  for (int k = 0; k < n; ++k) {
    float I[10], Iv[6], t1[6], t2[6], t3[6];
    load_inertia(r, k, I);
    inertia_mul(I, Fb[k], ab[k]);
    inertia_mul(I, v[k], Iv);
    crf(Fb[k], Iv, t1);
    crm(v[k], Fb[k], t2);
    inertia_mul(I, t2, t3);
    for (int i = 0; i < 6; ++i) vb[k][i] = -t1[i] - t3[i];
  }
  // ---- adjoint of the velocity/acceleration sweep and FK (tips -> base) ----
  for (int k = n - 1; k >= 0; --k) {
    const int pa = r.parent[k];
    const int j = r.jidx[k];
    const int jt = r.jtype[k];
    const float4 ax4 = reinterpret_cast<const float4*>(r.axis)[k];
    const float ax[3] = {ax4.x, ax4.y, ax4.z};
    float S[6];
    motion_S(jt, ax, S);
    const float mm = reinterpret_cast<const float2*>(r.mimic)[k].x;
    const float qd = j >= 0 ? mm * A.qd[j * B + b] : 0.0f;
    float t[6];
    crf(S, ab[k], t);
    for (int i = 0; i < 6; ++i) vb[k][i] = fmaf(qd, t[i], vb[k][i]);
    qddb[k] = dot6(S, ab[k]);
    crf(v[k], ab[k], t);
    qdb[k] = dot6(S, vb[k]) - dot6(S, t);
    float Xa[6], Xv[6], c[6];
    xf_motion(Rl[k], Rl[k] + 9, pa < 0 ? ab6 : a[pa], Xa);
    xf_motion(Rl[k], Rl[k] + 9, pa < 0 ? zero6 : v[pa], Xv);
    crm(S, Xa, c);
    qb[k] -= dot6(ab[k], c);
    crm(S, Xv, c);
    qb[k] -= dot6(vb[k], c);
    qb[k] += dot6(S, Wr[k]);
    if (pa >= 0) {
      float up[6];
      xf_force_T(Rl[k], Rl[k] + 9, ab[k], up);
      for (int i = 0; i < 6; ++i) ab[pa][i] += up[i];
      xf_force_T(Rl[k], Rl[k] + 9, vb[k], up);
      for (int i = 0; i < 6; ++i) vb[pa][i] += up[i];
      xf_force_T(Rl[k], Rl[k] + 9, Wr[k], up);
      for (int i = 0; i < 6; ++i) Wr[pa][i] += up[i];
    }
  }
  // ---- per-joint gather (mimic joints sum their links) ----
  for (int j = 0; j < r.d; ++j) {
    float g0 = 0.0f, g1 = 0.0f, g2 = 0.0f;
    for (int e = r.jl_start[j]; e < r.jl_start[j + 1]; ++e) {
      const int k = r.jl_links[e];
      const float mm = reinterpret_cast<const float2*>(r.mimic)[k].x;
      g0 = fmaf(mm, qb[k], g0);
      g1 = fmaf(mm, qdb[k], g1);
      g2 = fmaf(mm, qddb[k], g2);
    }
    A.gq[j * B + b] = g0;
    A.gqd[j * B + b] = g1;
    A.gqdd[j * B + b] = g2;
  }
}

cudaError_t launch_plain_fwd(const DevRobot& r, const FwdArgs& a, int threads, cudaStream_t s) {
  if (threads <= 0) threads = 128;
  const int64_t grid = (a.B + threads - 1) / threads;
  plain_fwd_kernel<<<(unsigned)grid, threads, 0, s>>>(r, a);
  return cudaGetLastError();
}

cudaError_t launch_plain_bwd(const DevRobot& r, const BwdArgs& a, int threads, cudaStream_t s) {
  if (threads <= 0) threads = 128;
  const int64_t grid = (a.B + threads - 1) / threads;
  plain_bwd_kernel<<<(unsigned)grid, threads, 0, s>>>(r, a);
  return cudaGetLastError();
}

}  // namespace wbe
