// tree_sweep.cuh -- one thread per configuration, one depth-first sweep over
// the kinematic tree (device functions shared by the single-robot and the
// batched kernels).
//
// The links are visited in depth-first pre-order (computed on the host).  A
// stack indexed by tree depth holds, for every ancestor of the current link,
// what its subtree still needs; when the sweep moves to a link of depth dep,
// every stack entry at depth >= dep belongs to a finished subtree and is
// closed ("post-order") before the new link is pushed.  All threads of a warp
// walk the same sequence, so control flow is uniform, joint-major I/O
// ([d][B]) is coalesced, and the stack (indexed by a warp-uniform depth)
// lives in coalesced, L1-cached local memory.  Every lane does useful work,
// which the level-synchronous schedule (a few links per level) cannot.
//
// Forward (Alg. 4): pre-order computes the local transform, the world pose
// (Sec. 6.1.1, written to link_pose), v_k, a_k and f_k = I a + v x* I v;
// post-order closes F_k = f_k + sum_children X_c^T F_c, emits
// tau_j += m_k S_k^T F_k and adds X_k^T F_k to the parent.
//
// Backward (the VJP of Alg. 4 and of FK; Alg. 5 and Alg. 1 give the
// structure): every pass of the adjoint fits the same sweep.
//   pre-order:  Fbar_k = S_k m_k taubar_j + X_k Fbar_pa          (base -> tips)
//               abar_k = I Fbar_k,
//               vbar_k = -crf(Fbar_k) I v_k - I crm(v_k) Fbar_k
//               W_k    = link-frame gradient wrench of the kinematic outputs
//   post-order: F_k, abar_k, vbar_k, W_k are complete (children added theirs)
//               vbar_k += crf(S qd_k) abar_k
//               qdd_bar = S^T abar_k
//               qd_bar  = S^T vbar_k - S^T crf(v_k) abar_k
//               q_bar   = (X_k Fbar_pa)^T crf(S) F_k - abar^T crm(S) X_k a_pa
//                         - vbar^T crm(S) X_k v_pa + S^T W_k
//               parent += X_k^T (F, abar, vbar, W)
// The root's a_pa is the base acceleration -g, so its q_bar terms follow the
// general formula; the v-dependence of a_k through v_k x_m (S qd) enters as
// the crf(S qd) abar term.  Both are derived from Alg. 4 by reverse-mode
// differentiation.
#pragma once

#include "spatial.cuh"

namespace wbe {

constexpr int TMAXD = 32;  // deepest tree the sweep kernels accept

__device__ __forceinline__ void motion_S6t(int jt, const float* ax, float* S) {
  S[0] = S[1] = S[2] = S[3] = S[4] = S[5] = 0.0f;
  if (jt == 1) {
    S[0] = ax[0]; S[1] = ax[1]; S[2] = ax[2];
  } else if (jt == 2) {
    S[3] = ax[0]; S[4] = ax[1]; S[5] = ax[2];
  }
}

__device__ __forceinline__ float dot6t(const float* a, const float* b) {
  float s = 0.0f;
#pragma unroll
  for (int i = 0; i < 6; ++i) s = fmaf(a[i], b[i], s);
  return s;
}

// world pose W = P o L (12 floats each)
__device__ __forceinline__ void compose(const float* P, const float* L, float* W) {
  float t[3];
  matmul3(P, L, W);
  rot(P, L + 9, t);
  W[9] = P[9] + t[0];
  W[10] = P[10] + t[1];
  W[11] = P[11] + t[2];
}

__device__ __forceinline__ void link_local(const DevRobot& r, int k, const float* q, int64_t B,
                                           int64_t b, float* L) {
  const int j = __ldg(r.jidx + k);
  const float th = j >= 0 ? joint_var(r, k, __ldg(q + (int64_t)j * B + b)) : 0.0f;
  local_xf(r, k, th, L, L + 9);
}

// ---------------------------------------------------------------------------
// forward: FK + RNEA
// ---------------------------------------------------------------------------
struct FEnt {
  float L[12];  // local transform
  float W[12];  // world pose
  float v[6], a[6], F[6];
  int k;
};

__device__ __forceinline__ void tree_fwd_one(const DevRobot& r, const FwdArgs& A, int64_t b) {
  const int64_t B = A.B;
  const int n = r.n;
  const bool dyn = A.tau != nullptr;
  FEnt stk[TMAXD];
  if (dyn && r.mimic_shared)
    for (int j = 0; j < r.d; ++j) A.tau[(int64_t)j * B + b] = 0.0f;

  auto close = [&](int e) {
    FEnt& E = stk[e];
    const int k = E.k;
    const int j = __ldg(r.jidx + k);
    if (j >= 0) {
      const float4 a4 = __ldg(reinterpret_cast<const float4*>(r.axis) + k);
      const float ax[3] = {a4.x, a4.y, a4.z};
      const float mm = __ldg(reinterpret_cast<const float2*>(r.mimic) + k).x;
      const float t = mm * St_dot(__ldg(r.jtype + k), ax, E.F);
      float* dst = A.tau + (int64_t)j * B + b;
      *dst = r.mimic_shared ? *dst + t : t;
    }
    if (e > 0) {
      float up[6];
      xf_force_T(E.L, E.L + 9, E.F, up);
#pragma unroll
      for (int i = 0; i < 6; ++i) stk[e - 1].F[i] += up[i];
    }
  };

  int sp = 0;
  for (int pos = 0; pos < n; ++pos) {
    const int2 kd = __ldg(r.dfs + pos);
    const int k = kd.x, dep = kd.y;
    if (dyn)
      while (sp > dep) close(--sp);
    sp = dep + 1;
    FEnt& E = stk[dep];
    E.k = k;
    link_local(r, k, A.q, B, b, E.L);
    if (dep > 0)
      compose(stk[dep - 1].W, E.L, E.W);
    else
#pragma unroll
      for (int i = 0; i < 12; ++i) E.W[i] = E.L[i];
    if (A.pose) {
      float4* dst = reinterpret_cast<float4*>(A.pose + (b * n + k) * 12);
      dst[0] = make_float4(E.W[0], E.W[1], E.W[2], E.W[3]);
      dst[1] = make_float4(E.W[4], E.W[5], E.W[6], E.W[7]);
      dst[2] = make_float4(E.W[8], E.W[9], E.W[10], E.W[11]);
    }
    if (dyn) {
      float vp[6], ap[6];
      if (dep > 0) {
#pragma unroll
        for (int i = 0; i < 6; ++i) {
          vp[i] = stk[dep - 1].v[i];
          ap[i] = stk[dep - 1].a[i];
        }
      } else {
        vp[0] = vp[1] = vp[2] = vp[3] = vp[4] = vp[5] = 0.0f;
        ap[0] = ap[1] = ap[2] = 0.0f;
        ap[3] = r.abase[0];
        ap[4] = r.abase[1];
        ap[5] = r.abase[2];
      }
      const int j = __ldg(r.jidx + k);
      const float4 a4 = __ldg(reinterpret_cast<const float4*>(r.axis) + k);
      const float ax[3] = {a4.x, a4.y, a4.z};
      const float mm = __ldg(reinterpret_cast<const float2*>(r.mimic) + k).x;
      const float vq = j >= 0 ? mm * __ldg(A.qd + (int64_t)j * B + b) : 0.0f;
      const float aq = j >= 0 ? mm * __ldg(A.qdd + (int64_t)j * B + b) : 0.0f;
      rnea_va(E.L, E.L + 9, vp, ap, __ldg(r.jtype + k), ax, vq, aq, E.v, E.a);
      float I[10];
      load_inertia(r, k, I);
      rnea_force(I, E.v, E.a, E.F);
    }
  }
  if (dyn)
    while (sp > 0) close(--sp);
}

// ---------------------------------------------------------------------------
// backward: the whole adjoint in one sweep
// ---------------------------------------------------------------------------
struct BEnt {
  float L[12], W[12];
  float v[6], a[6], F[6];
  float XF[6];   // X_k Fbar_pa
  float Fb[6];   // Fbar_k
  float ab[6], vb[6], Wr[6];
  int k;
};

// world pose of link l by composing its ancestor chain (topology cache)
__device__ __forceinline__ void chain_pose(const DevRobot& r, int l, const float* q, int64_t B,
                                           int64_t b, float* P) {
  const int c0 = __ldg(r.chain_start + l), c1 = __ldg(r.chain_start + l + 1);
  for (int c = c0; c < c1; ++c) {
    float L[12];
    link_local(r, __ldg(r.chain + c), q, B, b, L);
    if (c == c0) {
#pragma unroll
      for (int i = 0; i < 12; ++i) P[i] = L[i];
    } else {
      float T[12];
      compose(P, L, T);
#pragma unroll
      for (int i = 0; i < 12; ++i) P[i] = T[i];
    }
  }
}

__device__ __forceinline__ void point_wrench(const float* R, float4 sp, const float* g, float* w) {
  float f[3], nn[3];
  rotT(R, g, f);
  const float c[3] = {sp.x, sp.y, sp.z};
  cross3(c, f, nn);
  w[0] += nn[0];
  w[1] += nn[1];
  w[2] += nn[2];
  w[3] += f[0];
  w[4] += f[1];
  w[5] += f[2];
}

__device__ __forceinline__ void tree_bwd_one(const DevRobot& r, const BwdArgs& A, int64_t b) {
  const int64_t B = A.B;
  const int n = r.n;
  BEnt stk[TMAXD];
  if (r.mimic_shared)
    for (int j = 0; j < r.d; ++j) {
      A.gq[(int64_t)j * B + b] = 0.0f;
      A.gqd[(int64_t)j * B + b] = 0.0f;
      A.gqdd[(int64_t)j * B + b] = 0.0f;
    }
  // the worst pair's gradient: u = g_dmin (c_i - c_j) / |c_i - c_j|
  int pl1 = -1, pl2 = -1, ps1 = 0, ps2 = 0;
  float u[3] = {0.0f, 0.0f, 0.0f};
  if (A.g_dmin) {
    const int wp = A.worst[b];
    const float gd = A.g_dmin[b];
    if (wp >= 0 && wp < r.P && gd != 0.0f) {
      const int2 ij = __ldg(r.pairs + wp);
      ps1 = ij.x;
      ps2 = ij.y;
      pl1 = __ldg(r.sph_link + ps1);
      pl2 = __ldg(r.sph_link + ps2);
      float P1[12], P2[12], c1[3], c2[3];
      chain_pose(r, pl1, A.q, B, b, P1);
      chain_pose(r, pl2, A.q, B, b, P2);
      const float4 s1 = __ldg(r.sph + ps1), s2 = __ldg(r.sph + ps2);
      const float l1[3] = {s1.x, s1.y, s1.z}, l2[3] = {s2.x, s2.y, s2.z};
      rot(P1, l1, c1);
      rot(P2, l2, c2);
      const float dx = (c1[0] + P1[9]) - (c2[0] + P2[9]);
      const float dy = (c1[1] + P1[10]) - (c2[1] + P2[10]);
      const float dz = (c1[2] + P1[11]) - (c2[2] + P2[11]);
      const float nrm = sqrtf(fmaf(dz, dz, fmaf(dy, dy, dx * dx)));
      const float sc = nrm > 0.0f ? gd / nrm : 0.0f;
      u[0] = dx * sc;
      u[1] = dy * sc;
      u[2] = dz * sc;
    }
  }

  auto close = [&](int e) {
    BEnt& E = stk[e];
    const int k = E.k;
    const int j = __ldg(r.jidx + k);
    const int jt = __ldg(r.jtype + k);
    const float4 a4 = __ldg(reinterpret_cast<const float4*>(r.axis) + k);
    const float ax[3] = {a4.x, a4.y, a4.z};
    float S[6];
    motion_S6t(jt, ax, S);
    const float mm = __ldg(reinterpret_cast<const float2*>(r.mimic) + k).x;
    const float vq = j >= 0 ? mm * __ldg(A.qd + (int64_t)j * B + b) : 0.0f;
    float ab[6], vb[6], t[6];
#pragma unroll
    for (int i = 0; i < 6; ++i) {
      ab[i] = E.ab[i];
      vb[i] = E.vb[i];
    }
    crf(S, E.F, t);
    float gq = dot6t(E.XF, t);
    crf(S, ab, t);
#pragma unroll
    for (int i = 0; i < 6; ++i) vb[i] = fmaf(vq, t[i], vb[i]);
    const float gqdd = dot6t(S, ab);
    crf(E.v, ab, t);
    const float gqd = dot6t(S, vb) - dot6t(S, t);
    float vp[6], ap[6];
    if (e > 0) {
#pragma unroll
      for (int i = 0; i < 6; ++i) {
        vp[i] = stk[e - 1].v[i];
        ap[i] = stk[e - 1].a[i];
      }
    } else {
      vp[0] = vp[1] = vp[2] = vp[3] = vp[4] = vp[5] = 0.0f;
      ap[0] = ap[1] = ap[2] = 0.0f;
      ap[3] = r.abase[0];
      ap[4] = r.abase[1];
      ap[5] = r.abase[2];
    }
    float Xa[6], Xv[6], c6[6];
    xf_motion(E.L, E.L + 9, ap, Xa);
    xf_motion(E.L, E.L + 9, vp, Xv);
    crm(S, Xa, c6);
    gq -= dot6t(ab, c6);
    crm(S, Xv, c6);
    gq -= dot6t(vb, c6);
    gq += dot6t(S, E.Wr);
    if (j >= 0) {
      float* o0 = A.gq + (int64_t)j * B + b;
      float* o1 = A.gqd + (int64_t)j * B + b;
      float* o2 = A.gqdd + (int64_t)j * B + b;
      if (r.mimic_shared) {
        *o0 += mm * gq;
        *o1 += mm * gqd;
        *o2 += mm * gqdd;
      } else {
        *o0 = mm * gq;
        *o1 = mm * gqd;
        *o2 = mm * gqdd;
      }
    }
    if (e > 0) {
      BEnt& P = stk[e - 1];
      float up[6];
      xf_force_T(E.L, E.L + 9, E.F, up);
#pragma unroll
      for (int i = 0; i < 6; ++i) P.F[i] += up[i];
      xf_force_T(E.L, E.L + 9, ab, up);
#pragma unroll
      for (int i = 0; i < 6; ++i) P.ab[i] += up[i];
      xf_force_T(E.L, E.L + 9, vb, up);
#pragma unroll
      for (int i = 0; i < 6; ++i) P.vb[i] += up[i];
      xf_force_T(E.L, E.L + 9, E.Wr, up);
#pragma unroll
      for (int i = 0; i < 6; ++i) P.Wr[i] += up[i];
    }
  };

  int sp = 0;
  for (int pos = 0; pos < n; ++pos) {
    const int2 kd = __ldg(r.dfs + pos);
    const int k = kd.x, dep = kd.y;
    while (sp > dep) close(--sp);
    sp = dep + 1;
    BEnt& E = stk[dep];
    E.k = k;
    link_local(r, k, A.q, B, b, E.L);
    float vp[6], ap[6], Fbp[6];
    if (dep > 0) {
      const BEnt& P = stk[dep - 1];
      compose(P.W, E.L, E.W);
#pragma unroll
      for (int i = 0; i < 6; ++i) {
        vp[i] = P.v[i];
        ap[i] = P.a[i];
        Fbp[i] = P.Fb[i];
      }
    } else {
#pragma unroll
      for (int i = 0; i < 12; ++i) E.W[i] = E.L[i];
      vp[0] = vp[1] = vp[2] = vp[3] = vp[4] = vp[5] = 0.0f;
      ap[0] = ap[1] = ap[2] = 0.0f;
      ap[3] = r.abase[0];
      ap[4] = r.abase[1];
      ap[5] = r.abase[2];
      Fbp[0] = Fbp[1] = Fbp[2] = Fbp[3] = Fbp[4] = Fbp[5] = 0.0f;
    }
    const int j = __ldg(r.jidx + k);
    const int jt = __ldg(r.jtype + k);
    const float4 a4 = __ldg(reinterpret_cast<const float4*>(r.axis) + k);
    const float ax[3] = {a4.x, a4.y, a4.z};
    const float mm = __ldg(reinterpret_cast<const float2*>(r.mimic) + k).x;
    const float vq = j >= 0 ? mm * __ldg(A.qd + (int64_t)j * B + b) : 0.0f;
    const float aq = j >= 0 ? mm * __ldg(A.qdd + (int64_t)j * B + b) : 0.0f;
    // dynamics forward: v, a, f
    rnea_va(E.L, E.L + 9, vp, ap, jt, ax, vq, aq, E.v, E.a);
    float I[10];
    load_inertia(r, k, I);
    rnea_force(I, E.v, E.a, E.F);
    // adjoint of the force sweep: Fbar_k = S m taubar + X Fbar_pa
    float S[6];
    motion_S6t(jt, ax, S);
    const float tb = (j >= 0 && A.g_tau) ? mm * __ldg(A.g_tau + (int64_t)j * B + b) : 0.0f;
    xf_motion(E.L, E.L + 9, Fbp, E.XF);
#pragma unroll
    for (int i = 0; i < 6; ++i) E.Fb[i] = fmaf(S[i], tb, E.XF[i]);
    // adjoint of the per-link force: abar, vbar
    {
      float Iv[6], t1[6], t2[6], t3[6];
      inertia_mul(I, E.Fb, E.ab);
      inertia_mul(I, E.v, Iv);
      crf(E.Fb, Iv, t1);
      crm(E.v, E.Fb, t2);
      inertia_mul(I, t2, t3);
#pragma unroll
      for (int i = 0; i < 6; ++i) E.vb[i] = -t1[i] - t3[i];
    }
    // gradient wrench of the kinematic outputs, link frame
    float w[6] = {0, 0, 0, 0, 0, 0};
    if (A.g_pose) {
      const float4* g4 = reinterpret_cast<const float4*>(A.g_pose + (b * n + k) * 12);
      const float4 x0 = __ldg(g4), x1 = __ldg(g4 + 1), x2 = __ldg(g4 + 2);
      const float gg[12] = {x0.x, x0.y, x0.z, x0.w, x1.x, x1.y, x1.z, x1.w, x2.x, x2.y, x2.z, x2.w};
      const float* R = E.W;
      float Gm[9];  // R^T Rbar
#pragma unroll
      for (int ii = 0; ii < 3; ++ii)
#pragma unroll
        for (int jj = 0; jj < 3; ++jj)
          Gm[3 * ii + jj] = fmaf(R[6 + ii], gg[6 + jj], fmaf(R[3 + ii], gg[3 + jj], R[ii] * gg[jj]));
      w[0] = Gm[7] - Gm[5];
      w[1] = Gm[2] - Gm[6];
      w[2] = Gm[3] - Gm[1];
      rotT(R, gg + 9, w + 3);
    }
    if (A.g_sph) {
      const int e1 = __ldg(r.ls_start + k + 1);
      for (int e = __ldg(r.ls_start + k); e < e1; ++e) {
        const int s = __ldg(r.ls_sph + e);
        const float* g = A.g_sph + (b * r.S + s) * 3;
        const float gg[3] = {__ldg(g), __ldg(g + 1), __ldg(g + 2)};
        point_wrench(E.W, __ldg(r.sph + s), gg, w);
      }
    }
    if (k == pl1) point_wrench(E.W, __ldg(r.sph + ps1), u, w);
    if (k == pl2) {
      const float mu[3] = {-u[0], -u[1], -u[2]};
      point_wrench(E.W, __ldg(r.sph + ps2), mu, w);
    }
#pragma unroll
    for (int i = 0; i < 6; ++i) E.Wr[i] = w[i];
  }
  while (sp > 0) close(--sp);
}


}  // namespace wbe
