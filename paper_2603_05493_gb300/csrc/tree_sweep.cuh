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
//               (with the pose, v_k and a_k of the forward)
//   post-order: the link's own terms
//                 f_k    = I a_k + v_k x* I v_k
//                 abar_k = I Fbar_k,
//                 vbar_k = -crf(Fbar_k) I v_k - I crm(v_k) Fbar_k
//                 W_k    = link-frame gradient wrench of the kinematic outputs
//               plus the children's sums complete F_k, abar_k, vbar_k, W_k
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
//
// Segmented sweeps.  A tree with few links per level but many links in total
// leaves one thread per configuration with a long serial chain and, at a few
// tens of thousands of configurations, few warps per SM.  The DFS order can
// instead be cut into G contiguous segments, one warp per segment over the
// same 32 configurations.  The warp of segment g first replays the ancestors
// of its first link (pre-order data only: poses, v, a, Fbar; its own force,
// adjoint and wrench contributions are zero), then sweeps its links.  Every
// post-order quantity above is linear in the accumulated F, abar, vbar, W
// given the pre-order data, so the outputs of a link that several segments
// hold (an ancestor of a segment's first link) are the sums of the
// segments' partial outputs.  Those partials go to shared-memory slots and
// the kernel adds them in segment order (deterministic) after a barrier; all
// other outputs are written directly by the one segment that owns the link.
#pragma once

#include "spatial.cuh"
#include "spline_basis.cuh"

namespace wbe {

constexpr int TMAXD = 32;  // deepest tree the sweep kernels accept

// One segment of a segmented sweep (see above).  slot == nullptr: the whole
// DFS order, outputs written directly.
struct Seg {
  int p0, p1;          // DFS positions this segment owns
  int g, G;            // segment index, segments per configuration
  const int16_t* slot; // [n] shared output slot of a link or -1; nullptr = none
  float* part;         // partial outputs of this group: [nout][ns][G][32]
  int ns;              // shared slots
  int lane;
  // forward sweep with its force stack in shared memory: this thread's
  // entry 0, and the stride of the [depth][6][threads] layout (the block's
  // threads)
  float* fst = nullptr;
  int fstr = 0;
};

__device__ __forceinline__ Seg whole_sweep(const DevRobot& r) {
  return Seg{0, r.n, 0, 1, nullptr, nullptr, 0, 0};
}

// L2 prefetch hint for a global input of the next link, so that its DRAM
// latency overlaps the current link's arithmetic (measured on the 48-DoF
// humanoid: 11 % off the one-thread sweeps; an L1 hint gives the same).
// Only called on addresses inside the caller's buffers.
__device__ __forceinline__ void pf(const void* p) { asm volatile("prefetch.L2 [%0];" ::"l"(p)); }

// The joint states (q, qd, qdd of joint j) of the sweep's configuration b,
// from [d][B] arrays ...
struct ArrayStates {
  const float* q;
  const float* qd;
  const float* qdd;
  int64_t B, b;
  __device__ __forceinline__ float pos(int j) const { return __ldg(q + (int64_t)j * B + b); }
  __device__ __forceinline__ float vel(int j) const { return __ldg(qd + (int64_t)j * B + b); }
  __device__ __forceinline__ float acc(int j) const { return __ldg(qdd + (int64_t)j * B + b); }
  __device__ __forceinline__ void prefetch(int j, bool rates) const {
    pf(q + (int64_t)j * B + b);
    if (rates) {
      pf(qd + (int64_t)j * B + b);
      pf(qdd + (int64_t)j * B + b);
    }
  }
};

// ... or evaluated from uniform cubic B-spline control points (Sec. 4,
// Eq. bspline-cubic) where the sweep needs them: the configuration is sample
// s of trajectory tr, u points at that trajectory's first window knot of
// joint 0 (control points [d][K]) and bs at the sample's basis rows [3][4]
// (q, qd, qdd), computed once per configuration.  Same arithmetic as the
// B-spline forward kernel, so the states are the same bits.
struct SplineStates {
  const float* u;
  int K;
  const float* bs;
  __device__ __forceinline__ float row(int j, int r) const {
    const float* p = u + (int64_t)j * K;
    return bs_row(bs + 4 * r, __ldg(p), __ldg(p + 1), __ldg(p + 2), __ldg(p + 3));
  }
  __device__ __forceinline__ float pos(int j) const { return row(j, 0); }
  __device__ __forceinline__ float vel(int j) const { return row(j, 1); }
  __device__ __forceinline__ float acc(int j) const { return row(j, 2); }
  __device__ __forceinline__ void prefetch(int j, bool) const { pf(u + (int64_t)j * K); }
};

// where the partial output o of link k goes, or nullptr for a direct write
__device__ __forceinline__ float* seg_part(const Seg& sg, int k, int o) {
  if (!sg.slot) return nullptr;
  const int s = __ldg(sg.slot + k);
  if (s < 0) return nullptr;
  return sg.part + ((size_t)(o * sg.ns + s) * sg.G + sg.g) * 32 + sg.lane;
}

__device__ __forceinline__ void motion_S6t(int jt, const float* ax, float* S) {
  S[0] = S[1] = S[2] = S[3] = S[4] = S[5] = 0.0f;
  if (jt == 1) {
    S[0] = ax[0]; S[1] = ax[1]; S[2] = ax[2];
  } else if (jt == 2) {
    S[3] = ax[0]; S[4] = ax[1]; S[5] = ax[2];
  }
}

// The close's terms with the joint's motion subspace S = [a; 0] (JT = 1,
// revolute), [0; a] (JT = 2, prismatic) or 0 (JT = 0, fixed), written per
// joint type so that S's zero half costs nothing (the joint type is
// warp-uniform: every lane closes the same link).  The same operations, in
// the same order, as the dense 6-vector forms on the nonzero half.
//   parent terms: X_k v_pa = v - S qd, X_k a_pa = a - S qdd - v x_m (S qd),
//                 X_k Fbar_pa = Fbar - S taubar;
//   gradients:    gq = XF . crf(S) F - ab . crm(S) Xa - vb . crm(S) Xv + S . W,
//                 vb += qd crf(S) ab (before gq and gqd), gqdd = S . ab,
//                 gqd = S . vb - S . crf(v) ab.
template <int JT>
__device__ __forceinline__ void close_parent_terms(const float* a, float vq, float aq, float tb,
                                                   const float* cv, const float* ca,
                                                   const float* cFb, float* Xv, float* Xa,
                                                   float* XF) {
#pragma unroll
  for (int i = 0; i < 6; ++i) {
    Xv[i] = cv[i];
    Xa[i] = ca[i];
    XF[i] = cFb[i];
  }
  if (JT == 0) return;
  const float s[3] = {a[0] * vq, a[1] * vq, a[2] * vq};
  float c[3];
  if (JT == 1) {  // v x_m [s; 0] = [w x s; u x s]
    float cu[3];
    cross3(cv, s, c);
    cross3(cv + 3, s, cu);
#pragma unroll
    for (int i = 0; i < 3; ++i) {
      Xv[i] = cv[i] - s[i];
      Xa[i] = ca[i] - fmaf(a[i], aq, c[i]);
      Xa[3 + i] = ca[3 + i] - cu[i];
      XF[i] = fmaf(-a[i], tb, cFb[i]);
    }
  } else {  // v x_m [0; s] = [0; w x s]
    cross3(cv, s, c);
#pragma unroll
    for (int i = 0; i < 3; ++i) {
      Xv[3 + i] = cv[3 + i] - s[i];
      Xa[3 + i] = ca[3 + i] - fmaf(a[i], aq, c[i]);
      XF[3 + i] = fmaf(-a[i], tb, cFb[3 + i]);
    }
  }
}

template <int JT>
__device__ __forceinline__ void close_joint_grads(const float* a, float vq, const float* F,
                                                  const float* ab, float* vb, const float* Wr,
                                                  const float* cv, const float* Xv,
                                                  const float* Xa, const float* XF, float& gq,
                                                  float& gqd, float& gqdd) {
  gq = gqd = gqdd = 0.0f;
  if (JT == 0) return;
  constexpr int w = JT == 1 ? 0 : 3;  // the half of a 6-vector S lives in
  float t[3], t2[3];
  if (JT == 1) {  // crf([a; 0]) f = [a x f_n; a x f_f]
    cross3(a, F, t);
    cross3(a, F + 3, t2);
    gq = fmaf(XF[5], t2[2], fmaf(XF[4], t2[1], fmaf(XF[3], t2[0],
         fmaf(XF[2], t[2], fmaf(XF[1], t[1], XF[0] * t[0])))));
    cross3(a, ab, t);
    cross3(a, ab + 3, t2);
#pragma unroll
    for (int i = 0; i < 3; ++i) {
      vb[i] = fmaf(vq, t[i], vb[i]);
      vb[3 + i] = fmaf(vq, t2[i], vb[3 + i]);
    }
  } else {  // crf([0; a]) f = [a x f_f; 0]
    cross3(a, F + 3, t);
    gq = fmaf(XF[2], t[2], fmaf(XF[1], t[1], XF[0] * t[0]));
    cross3(a, ab + 3, t);
#pragma unroll
    for (int i = 0; i < 3; ++i) vb[i] = fmaf(vq, t[i], vb[i]);
  }
  gqdd = dot3(a, ab + w);
  // the half of crf(v) ab that S picks: [w x ab_n + u x ab_f] or [w x ab_f]
  float cr[3];
  if (JT == 1) {
    float c1[3], c2[3];
    cross3(cv, ab, c1);
    cross3(cv + 3, ab + 3, c2);
#pragma unroll
    for (int i = 0; i < 3; ++i) cr[i] = c1[i] + c2[i];
  } else {
    cross3(cv, ab + 3, cr);
  }
  gqd = dot3(a, vb + w) - dot3(a, cr);
  // crm([a; 0]) m = [a x m_w; a x m_u],  crm([0; a]) m = [0; a x m_w]
  if (JT == 1) {
    cross3(a, Xa, t);
    cross3(a, Xa + 3, t2);
    gq -= fmaf(ab[5], t2[2], fmaf(ab[4], t2[1], fmaf(ab[3], t2[0],
          fmaf(ab[2], t[2], fmaf(ab[1], t[1], ab[0] * t[0])))));
    cross3(a, Xv, t);
    cross3(a, Xv + 3, t2);
    gq -= fmaf(vb[5], t2[2], fmaf(vb[4], t2[1], fmaf(vb[3], t2[0],
          fmaf(vb[2], t[2], fmaf(vb[1], t[1], vb[0] * t[0])))));
  } else {
    cross3(a, Xa, t);
    gq -= fmaf(ab[5], t[2], fmaf(ab[4], t[1], ab[3] * t[0]));
    cross3(a, Xv, t);
    gq -= fmaf(vb[5], t[2], fmaf(vb[4], t[1], vb[3] * t[0]));
  }
  gq += dot3(a, Wr + w);
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

template <class St>
__device__ __forceinline__ void link_local_m(const DevRobot& r, int k, int meta, const St& st,
                                             float* L) {  // meta: lmeta[k]
  const int j = (meta & 0xFFFF) - 1;
  const float th = j >= 0 ? joint_var(r, k, st.pos(j)) : 0.0f;
  local_xf_m(r, k, th, (meta >> 16) & 0xFF, ((meta >> 24) & 1) != 0, L, L + 9);
}
template <class St>
__device__ __forceinline__ void link_local(const DevRobot& r, int k, const St& st, float* L) {
  const int j = __ldg(r.jidx + k);
  const float th = j >= 0 ? joint_var(r, k, st.pos(j)) : 0.0f;
  local_xf(r, k, th, L, L + 9);
}

// the dfs_kj word of link k, built from the per-link arrays (for the
// replayed ancestors of a segment, which are not at its DFS positions)
__device__ __forceinline__ int packed_link(const DevRobot& r, int k) {
  const int nch = min(__ldg(r.child_start + k + 1) - __ldg(r.child_start + k), 255);
  return (__ldg(r.lmeta + k) & 0xFFFF) | (nch << 16) | ((int)__ldg(r.jtype + k) << 24) |
         ((int)__ldg(r.rot_id + k) << 26);
}

// ---------------------------------------------------------------------------
// forward: FK + RNEA
// ---------------------------------------------------------------------------
// Per-depth stack entry.  The local transform is not kept: post-order
// recomputes it from q (cheaper than a round trip through local memory).
// W, v and a are read only by the push of a second or later child, so only
// links with two or more children store them; F (own force plus the
// children's) is stored when a child's push interrupts it.
struct FEnt {
  float W[12];  // world pose
  float v[6], a[6], F[6];
};

// FS: the accumulated forces F of the stack live in shared memory (sg.fst)
// instead of the thread's local stack
template <class St, bool FS = false>
__device__ __forceinline__ void tree_fwd_seg(const DevRobot& r, const FwdArgs& A, const St& st,
                                             int64_t b, const Seg& sg) {
  const int64_t B = A.B;
  const int n = r.n;
  const bool dyn = A.tau != nullptr;
  FEnt stk[TMAXD];
  if (dyn && r.mimic_shared)
    for (int j = 0; j < r.d; ++j) A.tau[(int64_t)j * B + b] = 0.0f;
  // Register copies that spare most stack loads: the pre-order data of the
  // last pushed entry (never changes while the entry is on the stack; a link
  // pushed right after its parent reads it from here), and the accumulated
  // force of the entry that the post-order closes next (an unwinding chain
  // passes it on in registers; it is stored when a push interrupts).
  float cW[12], cv[6], ca[6];
  int cdep = -1;
  float pF[6];
  int pdep = -1;
  int lastk = 0;  // last pushed link; the stack holds its ancestor chain
  int ck = 0;     // the link the next close takes

  auto close = [&](int e) {
    FEnt& E = stk[e];
    // the link at depth e: the last pushed one, then each closed link's
    // parent (one load off the critical path instead of two dependent ones
    // into the ancestor chains: humanoid48 forward 0.0934 -> 0.0892 ms; the
    // backward, at its register cap, spills more with it and is not faster)
    const int k = ck;
    ck = __ldg(r.parent + k);
    float F[6];
    if (pdep == e) {
#pragma unroll
      for (int i = 0; i < 6; ++i) F[i] = pF[i];
    } else {
#pragma unroll
      for (int i = 0; i < 6; ++i) F[i] = FS ? sg.fst[(6 * e + i) * sg.fstr] : E.F[i];
    }
    pdep = -1;
    const int meta = __ldg(r.lmeta + k);
    const int j = (meta & 0xFFFF) - 1;
    if (j >= 0) {
      const float4 a4 = ldp(reinterpret_cast<const float4*>(r.axis) + k);
      const float ax[3] = {a4.x, a4.y, a4.z};
      const float mm = ldp(reinterpret_cast<const float2*>(r.mimic) + k).x;
      const float t = mm * St_dot((meta >> 16) & 0xFF, ax, F);
      float* pt = seg_part(sg, k, 0);
      if (pt) {
        *pt = t;
      } else {
        float* dst = A.tau + (int64_t)j * B + b;
        *dst = r.mimic_shared ? *dst + t : t;
      }
    }
    if (e > 0) {
      float L[12], up[6];
      link_local_m(r, k, meta, st, L);
      xf_force_T(L, L + 9, F, up);
#pragma unroll
      for (int i = 0; i < 6; ++i)
        pF[i] = (FS ? sg.fst[(6 * (e - 1) + i) * sg.fstr] : stk[e - 1].F[i]) + up[i];
      pdep = e - 1;
    }
  };
  auto flush = [&]() {  // the pending force goes back to its stack entry
    if (pdep >= 0) {
#pragma unroll
      for (int i = 0; i < 6; ++i) {
        if (FS)
          sg.fst[(6 * pdep + i) * sg.fstr] = pF[i];
        else
          stk[pdep].F[i] = pF[i];
      }
      pdep = -1;
    }
  };

  // pre-order of link k at depth dep; own = false replays an ancestor of
  // the segment (pose, v, a only; no output, no force of its own); pre: the
  // joint states (pq, pqd, pqdd) were loaded ahead by the caller
  auto push = [&](int k, int dep, bool own, bool pre, float pq, float pqd, float pqdd, int ky) {
    const int jk = (ky & 0xFFFF) - 1, nch = (ky >> 16) & 0xFF, jtk = (ky >> 24) & 3;
    if (dyn) flush();  // the parent's force, when it is still pending
    FEnt& E = stk[dep];
    float L[12];
    {
      const float th = jk >= 0 ? joint_var(r, k, pre ? pq : st.pos(jk)) : 0.0f;
      local_xf_m(r, k, th, jtk, ((ky >> 26) & 1) != 0, L, L + 9);
    }
    float PW[12], vp[6], ap[6];
    if (dep > 0) {
      if (dep == cdep + 1) {
#pragma unroll
        for (int i = 0; i < 12; ++i) PW[i] = cW[i];
#pragma unroll
        for (int i = 0; i < 6; ++i) {
          vp[i] = cv[i];
          ap[i] = ca[i];
        }
      } else {
        const FEnt& P = stk[dep - 1];
#pragma unroll
        for (int i = 0; i < 12; ++i) PW[i] = P.W[i];
#pragma unroll
        for (int i = 0; i < 6; ++i) {
          vp[i] = P.v[i];
          ap[i] = P.a[i];
        }
      }
      compose(PW, L, cW);
    } else {
#pragma unroll
      for (int i = 0; i < 12; ++i) cW[i] = L[i];
      vp[0] = vp[1] = vp[2] = vp[3] = vp[4] = vp[5] = 0.0f;
      ap[0] = ap[1] = ap[2] = 0.0f;
      ap[3] = r.abase[0];
      ap[4] = r.abase[1];
      ap[5] = r.abase[2];
    }
    cdep = dep;
    lastk = k;
    ck = k;
    if (nch > 1) {
#pragma unroll
      for (int i = 0; i < 12; ++i) E.W[i] = cW[i];
    }
    if (own && A.pose) {
      float4* dst = reinterpret_cast<float4*>(A.pose + (b * n + k) * 12);
      dst[0] = make_float4(cW[0], cW[1], cW[2], cW[3]);
      dst[1] = make_float4(cW[4], cW[5], cW[6], cW[7]);
      dst[2] = make_float4(cW[8], cW[9], cW[10], cW[11]);
    }
    if (dyn) {
      const int j = jk;
      const float4 a4 = ldp(reinterpret_cast<const float4*>(r.axis) + k);
      const float ax[3] = {a4.x, a4.y, a4.z};
      const float mm = ldp(reinterpret_cast<const float2*>(r.mimic) + k).x;
      const float vq = j >= 0 ? mm * (pre ? pqd : st.vel(j)) : 0.0f;
      const float aq = j >= 0 ? mm * (pre ? pqdd : st.acc(j)) : 0.0f;
      rnea_va(L, L + 9, vp, ap, jtk, ax, vq, aq, cv, ca);
      float F[6];
      if (own) {
        float I[10];
        load_inertia(r, k, I);
        rnea_force(I, cv, ca, F);
        if (A.fext) {  // f_k = I a + v x* I v - f_ext,k
          const float* fe = A.fext + (b * n + k) * 6;
#pragma unroll
          for (int i = 0; i < 6; ++i) F[i] -= __ldg(fe + i);
        }
      } else {
#pragma unroll
        for (int i = 0; i < 6; ++i) F[i] = 0.0f;
      }
      if (nch > 1) {
#pragma unroll
        for (int i = 0; i < 6; ++i) {
          E.v[i] = cv[i];
          E.a[i] = ca[i];
        }
      }
      // the force waits in the pending registers; a child's push stores it
#pragma unroll
      for (int i = 0; i < 6; ++i) pF[i] = F[i];
      pdep = dep;
    }
  };

  int sp = 0;
  if (sg.p0 > 0) {  // replay the proper ancestors of the first link
    const int k0 = __ldg(r.dfs + sg.p0).x;
    const int c0 = __ldg(r.chain_start + k0), c1 = __ldg(r.chain_start + k0 + 1);
    for (int c = c0; c < c1 - 1; ++c) {
      const int a = __ldg(r.chain + c);
      push(a, c - c0, false, false, 0.0f, 0.0f, 0.0f, packed_link(r, a));
    }
    sp = c1 - 1 - c0;
  }
  // The joint states of the link pushed next, loaded one link ahead into
  // registers, so that their latency overlaps the current link's closes and
  // push (measured on the 48-DoF humanoid at 2 segments x 448 threads:
  // 0.0985 -> 0.0970 ms against the L2 prefetch hint it replaces).
  float nq = 0.0f, nqd = 0.0f, nqdd = 0.0f;
  int2 nkd = sg.p0 < sg.p1 ? __ldg(r.dfs_kj + sg.p0) : make_int2(0, 0);
  {
    const int j0 = sg.p0 < sg.p1 ? (nkd.y & 0xFFFF) - 1 : -1;
    if (j0 >= 0) {
      nq = st.pos(j0);
      if (dyn) {
        nqd = st.vel(j0);
        nqdd = st.acc(j0);
      }
    }
  }
  for (int pos = sg.p0; pos < sg.p1; ++pos) {
    // link | depth << 8, (joint + 1) | children << 16 of this position: one
    // load for what the DFS order, the joint index and the child table gave
    // in four (humanoid48 forward 0.0898 -> 0.0885 ms), kept from the
    // previous step's look-ahead rather than loaded again (0.0844 -> 0.0835
    // ms; the backward, at its register cap, spills more with it: 0.1664 ->
    // 0.1684 ms)
    const int2 kd = nkd;
    const int k = kd.x & 0xFF, dep = (kd.x >> 8) & 0xFF;
    const float cq = nq, cqd = nqd, cqdd = nqdd;
    if (pos + 1 < sg.p1) {  // the next link's joint inputs
      nkd = __ldg(r.dfs_kj + pos + 1);
      const int jn = (nkd.y & 0xFFFF) - 1;
      if (jn >= 0) {
        nq = st.pos(jn);
        if (dyn) {
          nqd = st.vel(jn);
          nqdd = st.acc(jn);
        }
      }
    }
    if (dyn) {
      while (sp > dep) close(--sp);
      flush();
    }
    sp = dep + 1;
    push(k, dep, true, true, cq, cqd, cqdd, kd.y);
  }
  if (dyn) {
    while (sp > 0) close(--sp);
    flush();
  }
}

__device__ __forceinline__ void tree_fwd_one(const DevRobot& r, const FwdArgs& A, int64_t b) {
  tree_fwd_seg(r, A, ArrayStates{A.q, A.qd, A.qdd, A.B, b}, b, whole_sweep(r));
}

// ---------------------------------------------------------------------------
// backward: the whole adjoint in one sweep
// ---------------------------------------------------------------------------
// The close of a link needs the link's pre-order state (world pose W, v, a,
// Fbar) and the three parent terms of its q_bar formula, X_k v_pa, X_k a_pa
// and X_k Fbar_pa.  Neither comes from a stack.  One state lives in
// registers: a push carries it down one link (W_k = W_pa L_k, v_k = X_k v_pa
// + S qd, ...) and a close carries it back up by undoing the same maps:
//   X_k v_pa    = v_k - S qd
//   X_k a_pa    = a_k - S qdd - v_k x_m (S qd)
//   X_k Fbar_pa = Fbar_k - S taubar
//   v_pa = X_k^-1 (X_k v_pa),  a_pa, Fbar_pa likewise,  W_pa = W_k L_k^-1
// (X^-1 [w; u] = [R w; R u + p x R w]).  The first three are the parent
// terms the close needs, so a close reads no parent data at all, and the
// push of a later child finds its parent's state in the registers.  The
// rounding of the repeated maps and inverses drifts by a few float ulps
// per link visited (measured on the humanoid: 5e-6 relative on the
// gradients against a sweep that stored each branching link's state and
// reloaded it, which was 4 % slower).  Per-depth stack entry, only what a
// later step reads:
//   tb  -- the link's torque adjoint m taubar (for X_k Fbar_pa), for a link
//          with children (a leaf's close follows its push and reads it from
//          a register);
//   acc -- the children's sums of F, abar, vbar, W, stored only when the
//          push of a sibling subtree interrupts them.
// The link's own F, abar and vbar are formed at its close from its state, and
// its gradient wrench of the kinematic outputs too (its world pose is in the
// registers there): nothing of the link's own travels through the stack.
struct BEnt {
  float aF[6], aab[6], avb[6], aWr[6];
  float tb;
};

// world pose of link l by composing its ancestor chain (topology cache)
template <class St>
__device__ __forceinline__ void chain_pose(const DevRobot& r, int l, const St& st, float* P) {
  const int c0 = __ldg(r.chain_start + l), c1 = __ldg(r.chain_start + l + 1);
  for (int c = c0; c < c1; ++c) {
    float L[12];
    link_local(r, __ldg(r.chain + c), st, L);
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

// parent pose from a link's world pose W and its local transform L: W L^-1
__device__ __forceinline__ void uncompose(const float* W, const float* L, float* P) {
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = 0; j < 3; ++j)
      P[3 * i + j] =
          fmaf(W[3 * i + 2], L[3 * j + 2], fmaf(W[3 * i + 1], L[3 * j + 1], W[3 * i] * L[3 * j]));
  float t[3];
  rot(P, L + 9, t);
  P[9] = W[9] - t[0];
  P[10] = W[10] - t[1];
  P[11] = W[11] - t[2];
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

// A thread's slot in shared memory for the upstream gradient rows that the
// next close reads: 6 float4 at p[q * stride], the link's pose gradient row
// (12 floats), then its first run of 4 sphere gradients.  Asynchronous copies
// (cp.async, bypassing L1) fill it while the sweep computes the link's push
// (a leaf) or its child's close, and the close waits for them: the rows' global
// latency no longer sits on the close's critical path.
struct GradSlot {
  float4* p = nullptr;
  int stride = 0;
};
constexpr int kGradSlotBytes = 6 * 16;  // a thread's slot
// the slots of a block behind `after` (any float address in dynamic shared
// memory), rounded up to 16 bytes; the block reserves kGradSlotBytes a thread
// plus 16 bytes for the rounding
__device__ __forceinline__ GradSlot grad_slot_of(float* after) {
  const uintptr_t a = reinterpret_cast<uintptr_t>(after);
  GradSlot g;
  g.p = reinterpret_cast<float4*>(after + ((16 - (a & 15)) & 15) / 4) + threadIdx.x;
  g.stride = blockDim.x;
  return g;
}
__device__ __forceinline__ void cp16(float4* dst, const void* src) {
  const unsigned a = static_cast<unsigned>(__cvta_generic_to_shared(dst));
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(a), "l"(src));
}

// With a fused cost (FC, fc) the sweep computes g_tau = [tau > hi] -
// [tau < lo] + 2 e qd^2 tau and g_dmin = -w [d_min < 0] itself, adds the
// cost's direct qd / qdd gradients (2 length qd + 2 e qd tau^2, 2 smooth qdd)
// to the outputs of the joint's link, and returns the cost terms of the joints
// of the links it owns (the caller adds the collision term and the segments'
// shares).  Needs one link per joint (no shared mimic joints).
// FC: compiled with the fused cost (a separate instantiation, so that the
// plain sweep keeps its register allocation).  gs: the thread's gradient-row
// slot, or none (the rows are then read with plain loads at each close).
template <bool FC, class St>
__device__ __forceinline__ float tree_bwd_seg(const DevRobot& r, const BwdArgs& A,
                                              const FusedCost& fc, const St& st, int64_t b,
                                              const Seg& sg, GradSlot gs = GradSlot{}) {
  const int64_t B = A.B;
  float cost_part = 0.0f;
  const int n = r.n;
  BEnt stk[TMAXD];
  if (r.mimic_shared)
    for (int j = 0; j < r.d; ++j) {
      A.gq[(int64_t)j * B + b] = 0.0f;
      A.gqd[(int64_t)j * B + b] = 0.0f;
      A.gqdd[(int64_t)j * B + b] = 0.0f;
    }
  // the worst pair's gradient: u = g_dmin (c_i - c_j) / |c_i - c_j|, needed
  // only by the segment that owns one of the pair's links
  auto owned = [&](int k) {
    if (!sg.slot) return true;
    const int p = __ldg(r.dfs_pos + k);
    return p >= sg.p0 && p < sg.p1;
  };
  int pl1 = -1, pl2 = -1, ps1 = 0, ps2 = 0;
  float u[3] = {0.0f, 0.0f, 0.0f};
  if (A.g_dmin || (FC && fc.d_min)) {
    const int wp = A.worst[b];
    const float gd = FC ? (__ldg(fc.d_min + b) < 0.0f ? -fc.w : 0.0f) : A.g_dmin[b];
    if (wp >= 0 && wp < r.P && gd != 0.0f) {
      const int2 ij = __ldg(r.pairs + wp);
      const int l1 = __ldg(r.sph_link + ij.x), l2 = __ldg(r.sph_link + ij.y);
      if (owned(l1) || owned(l2)) {
        ps1 = ij.x;
        ps2 = ij.y;
        pl1 = l1;
        pl2 = l2;
        float dx, dy, dz;
        if (A.wdiff) {  // from the pair stage: the same arithmetic on the same poses
          dx = __ldg(A.wdiff + 3 * b);
          dy = __ldg(A.wdiff + 3 * b + 1);
          dz = __ldg(A.wdiff + 3 * b + 2);
        } else {  // place the two spheres from their links' ancestor chains
          float P1[12], P2[12], c1[3], c2[3];
          chain_pose(r, pl1, st, P1);
          chain_pose(r, pl2, st, P2);
          const float4 s1 = __ldg(r.sph + ps1), s2 = __ldg(r.sph + ps2);
          const float q1[3] = {s1.x, s1.y, s1.z}, q2[3] = {s2.x, s2.y, s2.z};
          rot(P1, q1, c1);
          rot(P2, q2, c2);
          dx = (c1[0] + P1[9]) - (c2[0] + P2[9]);
          dy = (c1[1] + P1[10]) - (c2[1] + P2[10]);
          dz = (c1[2] + P1[11]) - (c2[2] + P2[11]);
        }
        const float nrm = sqrtf(fmaf(dz, dz, fmaf(dy, dy, dx * dx)));
        const float sc = nrm > 0.0f ? gd / nrm : 0.0f;
        u[0] = dx * sc;
        u[1] = dy * sc;
        u[2] = dz * sc;
      }
    }
  }

  // The state in registers: the pre-order data (W, v, a, Fbar) of the last
  // pushed link after a push, of the closed link's parent after a close; the
  // just-pushed link's torque adjoint (ctb, valid while fresh); and the
  // accumulated children's sums (F, abar, vbar, W) of the entry the
  // post-order closes next (an unwinding chain passes them on in registers;
  // they are stored when a push interrupts).
  float cW[12], cv[6], ca[6], cFb[6], ctb = 0.0f;
  bool fresh = false;
  float pF[6], pab[6], pvb[6], pWr[6];
  int pdep = -1;
  // bit e: entry e is an ancestor replayed for this segment (no own terms),
  // its acc holds children's sums
  uint32_t replayed = 0u, accv = 0u;
  int lcs = 0;  // where the last pushed link's ancestor chain starts (the stack holds it)
  const bool kin_grad = A.g_pose != nullptr || A.g_sph != nullptr;
  // sphere gradients of a link as float4 triples: the robot's spheres come
  // in runs of 4 (then b S + s is a multiple of 4) and the array (a slice of
  // a packed batch, possibly) is 16-byte aligned
  const bool sph4 = A.g_sph != nullptr && r.sph_vec4 &&
                    (reinterpret_cast<uintptr_t>(A.g_sph) & 15u) == 0;
  // the link whose gradient rows are on their way into the slot (-1: none)
  int pend = -1;
  const bool use_slot = gs.p != nullptr && kin_grad;
  auto issue = [&](int k) {
    if (A.g_pose) {
      const float4* g4 = reinterpret_cast<const float4*>(A.g_pose + (b * n + k) * 12);
      cp16(gs.p, g4);
      cp16(gs.p + gs.stride, g4 + 1);
      cp16(gs.p + 2 * gs.stride, g4 + 2);
    }
    if (sph4) {
      const int e0 = __ldg(r.ls_start + k);
      if (__ldg(r.ls_start + k + 1) > e0) {
        const float4* g4 = reinterpret_cast<const float4*>(A.g_sph + (b * r.S + __ldg(r.ls_sph + e0)) * 3);
        cp16(gs.p + 3 * gs.stride, g4);
        cp16(gs.p + 4 * gs.stride, g4 + 1);
        cp16(gs.p + 5 * gs.stride, g4 + 2);
      }
    }
    asm volatile("cp.async.commit_group;");
    pend = k;
  };

  // link-frame gradient wrench of link k's kinematic outputs (pose, spheres,
  // the worst pair's spheres), from its world pose in cW
  auto wrench = [&](int k, float* w) {
#pragma unroll
    for (int i = 0; i < 6; ++i) w[i] = 0.0f;
    const bool slot = pend == k;
    if (slot) asm volatile("cp.async.wait_group 0;" ::: "memory");
    pend = -1;
    if (A.g_pose) {
      const float4* g4 = reinterpret_cast<const float4*>(A.g_pose + (b * n + k) * 12);
      const float4 x0 = slot ? gs.p[0] : __ldg(g4), x1 = slot ? gs.p[gs.stride] : __ldg(g4 + 1),
                   x2 = slot ? gs.p[2 * gs.stride] : __ldg(g4 + 2);
      const float gg[12] = {x0.x, x0.y, x0.z, x0.w, x1.x, x1.y, x1.z, x1.w, x2.x, x2.y, x2.z, x2.w};
      const float* R = cW;
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
    if (sph4) {  // runs of 4 spheres: three float4 loads a run
      const int e1 = __ldg(r.ls_start + k + 1);
      const int ef = __ldg(r.ls_start + k);
      for (int e = ef; e < e1; e += 4) {
        const int s = __ldg(r.ls_sph + e);
        const float4* g4 = reinterpret_cast<const float4*>(A.g_sph + (b * r.S + s) * 3);
        const bool fs = slot && e == ef;
        const float4 x0 = fs ? gs.p[3 * gs.stride] : __ldg(g4),
                     x1 = fs ? gs.p[4 * gs.stride] : __ldg(g4 + 1),
                     x2 = fs ? gs.p[5 * gs.stride] : __ldg(g4 + 2);
        const float gg[12] = {x0.x, x0.y, x0.z, x0.w, x1.x, x1.y, x1.z, x1.w, x2.x, x2.y, x2.z, x2.w};
#pragma unroll
        for (int i = 0; i < 4; ++i) point_wrench(cW, __ldg(r.sph + s + i), gg + 3 * i, w);
      }
    } else if (A.g_sph) {
      const int e1 = __ldg(r.ls_start + k + 1);
      for (int e = __ldg(r.ls_start + k); e < e1; ++e) {
        const int s = __ldg(r.ls_sph + e);
        const float* g = A.g_sph + (b * r.S + s) * 3;
        const float gg[3] = {__ldg(g), __ldg(g + 1), __ldg(g + 2)};
        point_wrench(cW, __ldg(r.sph + s), gg, w);
      }
    }
    if (k == pl1) point_wrench(cW, __ldg(r.sph + ps1), u, w);
    if (k == pl2) {
      const float mu[3] = {-u[0], -u[1], -u[2]};
      point_wrench(cW, __ldg(r.sph + ps2), mu, w);
    }
  };

  // post-order of the link at depth e; the registers hold its state; tgt:
  // the closes go on down to depth tgt
  auto close = [&](int e, int tgt) {
    // the link at depth e with its joint, type and rotation flag, one load
    const int cm = __ldg(r.chain_m + lcs + e);
    const int k = cm & 0xFF;
    const bool own = !((replayed >> e) & 1u);
    // own terms: f = I a + v x* I v - f_ext, abar = I Fbar,
    // vbar = -crf(Fbar) I v - I crm(v) Fbar, and the gradient wrench
    float F[6], ab[6], vb[6], Wr[6];
    if (own) {
      float I[10];
      load_inertia(r, k, I);
      rnea_force(I, cv, ca, F);
      if (A.fext) {
        const float* fe = A.fext + (b * n + k) * 6;
#pragma unroll
        for (int i = 0; i < 6; ++i) F[i] -= __ldg(fe + i);
      }
      float Iv[6], t1[6], t2[6], t3[6];
      inertia_mul(I, cFb, ab);
      inertia_mul(I, cv, Iv);
      crf(cFb, Iv, t1);
      crm(cv, cFb, t2);
      inertia_mul(I, t2, t3);
#pragma unroll
      for (int i = 0; i < 6; ++i) vb[i] = -t1[i] - t3[i];
      if (kin_grad || k == pl1 || k == pl2) {
        wrench(k, Wr);
        // the next close's rows, while this one computes
        if (use_slot && e - 1 >= tgt && !((replayed >> (e - 1)) & 1u))
          issue(__ldg(r.chain_m + lcs + e - 1) & 0xFF);
      } else {
#pragma unroll
        for (int i = 0; i < 6; ++i) Wr[i] = 0.0f;
      }
    } else {
#pragma unroll
      for (int i = 0; i < 6; ++i) F[i] = ab[i] = vb[i] = Wr[i] = 0.0f;
    }
    // plus the children's sums
    if (pdep == e) {
#pragma unroll
      for (int i = 0; i < 6; ++i) {
        F[i] += pF[i];
        ab[i] += pab[i];
        vb[i] += pvb[i];
        Wr[i] += pWr[i];
      }
    } else if ((accv >> e) & 1u) {
      const BEnt& E = stk[e];
#pragma unroll
      for (int i = 0; i < 6; ++i) {
        F[i] += E.aF[i];
        ab[i] += E.aab[i];
        vb[i] += E.avb[i];
        Wr[i] += E.aWr[i];
      }
    }
    pdep = -1;
    const int j = ((cm >> 8) & 0x1FF) - 1;
    const int jt = (cm >> 17) & 3;
    const float4 a4 = ldp(reinterpret_cast<const float4*>(r.axis) + k);
    const float ax[3] = {a4.x, a4.y, a4.z};
    const float mm = ldp(reinterpret_cast<const float2*>(r.mimic) + k).x;
    const float vq = j >= 0 ? mm * st.vel(j) : 0.0f;
    float L[12];
    {
      const float th = j >= 0 ? joint_var(r, k, st.pos(j)) : 0.0f;
      local_xf_m(r, k, th, jt, ((cm >> 19) & 1) != 0, L, L + 9);
    }
    // the parent terms X_k v_pa, X_k a_pa, X_k Fbar_pa from the link's state
    float Xv[6], Xa[6], XF[6];
    if (e > 0) {
      const float aq = j >= 0 ? mm * st.acc(j) : 0.0f;
      const float tb = fresh ? ctb : stk[e].tb;
      if (jt == 1)
        close_parent_terms<1>(ax, vq, aq, tb, cv, ca, cFb, Xv, Xa, XF);
      else if (jt == 2)
        close_parent_terms<2>(ax, vq, aq, tb, cv, ca, cFb, Xv, Xa, XF);
      else
        close_parent_terms<0>(ax, vq, aq, tb, cv, ca, cFb, Xv, Xa, XF);
    } else {  // the root: v_pa = 0, a_pa = the base acceleration, Fbar_pa = 0
      const float ap[6] = {0.0f, 0.0f, 0.0f, r.abase[0], r.abase[1], r.abase[2]};
      xf_motion(L, L + 9, ap, Xa);
#pragma unroll
      for (int i = 0; i < 6; ++i) Xv[i] = XF[i] = 0.0f;
    }
    float gq, gqd, gqdd;
    if (jt == 1)
      close_joint_grads<1>(ax, vq, F, ab, vb, Wr, cv, Xv, Xa, XF, gq, gqd, gqdd);
    else if (jt == 2)
      close_joint_grads<2>(ax, vq, F, ab, vb, Wr, cv, Xv, Xa, XF, gq, gqd, gqdd);
    else
      close_joint_grads<0>(ax, vq, F, ab, vb, Wr, cv, Xv, Xa, XF, gq, gqd, gqdd);
    if (FC && j >= 0) {
      float dqd = 0.0f, dqdd = 0.0f;  // the cost's direct gradients, once per joint
      if (own) {
        const int64_t at = (int64_t)j * B + b;
        const float tj = __ldg(fc.tau + at), vj = st.vel(j), aj = st.acc(j);
        dqd = 2.0f * (fc.length * vj + fc.e * (vj * tj) * tj);
        dqdd = 2.0f * fc.smooth * aj;
      }
      float* p0 = seg_part(sg, k, 0);
      if (p0) {
        const size_t o = (size_t)sg.ns * sg.G * 32;
        p0[0] = mm * gq;
        p0[o] = mm * gqd + dqd;
        p0[2 * o] = mm * gqdd + dqdd;
      } else {
        A.gq[(int64_t)j * B + b] = mm * gq;
        A.gqd[(int64_t)j * B + b] = mm * gqd + dqd;
        A.gqdd[(int64_t)j * B + b] = mm * gqdd + dqdd;
      }
    } else if (j >= 0) {
      float* p0 = seg_part(sg, k, 0);
      if (p0) {
        const size_t o = (size_t)sg.ns * sg.G * 32;
        p0[0] = mm * gq;
        p0[o] = mm * gqd;
        p0[2 * o] = mm * gqdd;
      } else {
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
    }
    fresh = false;
    if (e > 0) {
      const BEnt& P = stk[e - 1];
      const bool has = (accv >> (e - 1)) & 1u;
      accv &= ~(1u << (e - 1));  // taken over by the pending registers
      float up[6];
      xf_force_T(L, L + 9, F, up);
#pragma unroll
      for (int i = 0; i < 6; ++i) pF[i] = has ? P.aF[i] + up[i] : up[i];
      xf_force_T(L, L + 9, ab, up);
#pragma unroll
      for (int i = 0; i < 6; ++i) pab[i] = has ? P.aab[i] + up[i] : up[i];
      xf_force_T(L, L + 9, vb, up);
#pragma unroll
      for (int i = 0; i < 6; ++i) pvb[i] = has ? P.avb[i] + up[i] : up[i];
      xf_force_T(L, L + 9, Wr, up);
#pragma unroll
      for (int i = 0; i < 6; ++i) pWr[i] = has ? P.aWr[i] + up[i] : up[i];
      pdep = e - 1;
      // the parent's state: this link's maps undone
      float Wp[12];
      uncompose(cW, L, Wp);
#pragma unroll
      for (int i = 0; i < 12; ++i) cW[i] = Wp[i];
      xf_motion_inv(L, L + 9, Xv, cv);
      xf_motion_inv(L, L + 9, Xa, ca);
      xf_motion_inv(L, L + 9, XF, cFb);
    }
  };
  auto flush = [&]() {  // the pending children's sums go to their entry
    if (pdep >= 0) {
      BEnt& P = stk[pdep];
#pragma unroll
      for (int i = 0; i < 6; ++i) {
        P.aF[i] = pF[i];
        P.aab[i] = pab[i];
        P.avb[i] = pvb[i];
        P.aWr[i] = pWr[i];
      }
      accv |= 1u << pdep;
      pdep = -1;
    }
  };

  // pre-order of link k at depth dep (the registers hold its parent's state);
  // own = false replays an ancestor of the segment (its own contributions
  // are zero)
  auto push = [&](int k, int dep, bool own, int ky, int cs) {
    const int j = (ky & 0xFFFF) - 1, nch = (ky >> 16) & 0xFF, jt = (ky >> 24) & 3;
    float L[12];
    {
      const float th = j >= 0 ? joint_var(r, k, st.pos(j)) : 0.0f;
      local_xf_m(r, k, th, jt, ((ky >> 26) & 1) != 0, L, L + 9);
    }
    const float4 a4 = ldp(reinterpret_cast<const float4*>(r.axis) + k);
    const float ax[3] = {a4.x, a4.y, a4.z};
    const float mm = ldp(reinterpret_cast<const float2*>(r.mimic) + k).x;
    const float vq = j >= 0 ? mm * st.vel(j) : 0.0f;
    const float aq = j >= 0 ? mm * st.acc(j) : 0.0f;
    // the adjoint of the force sweep's torque term: taubar of the joint
    float tb = 0.0f;
    if (FC && j >= 0) {  // the cost's torque gradient, as the cost kernel forms it
      const float t = __ldg(fc.tau + (int64_t)j * B + b), l = __ldg(fc.lo + j),
                  h = __ldg(fc.hi + j);
      const float v = st.vel(j), a = st.acc(j);
      const float vt = v * t;
      float gt = 2.0f * fc.e * v * vt;
      gt += (t > h ? 1.0f : 0.0f) - (t < l ? 1.0f : 0.0f);
      tb = mm * gt;
      if (own) {
        float c = fmaf(fc.smooth * a, a, 0.0f);
        c = fmaf(fc.length * v, v, c);
        c = fmaf(fc.e * vt, vt, c);
        c += fmaxf(0.0f, t - h) + fmaxf(0.0f, l - t);
        cost_part += c;
      }
    } else if (!FC && j >= 0 && A.g_tau) {
      tb = mm * __ldg(A.g_tau + (int64_t)j * B + b);
    }
    float S[6];
    motion_S6t(jt, ax, S);
    // pose, v, a (dynamics forward) and Fbar_k = S m taubar + X Fbar_pa
    float Wn[12], vn[6], an[6], XF[6];
    if (dep > 0) {
      compose(cW, L, Wn);
      rnea_va(L, L + 9, cv, ca, jt, ax, vq, aq, vn, an);
      xf_motion(L, L + 9, cFb, XF);
    } else {
#pragma unroll
      for (int i = 0; i < 12; ++i) Wn[i] = L[i];
      const float vp[6] = {0.0f, 0.0f, 0.0f, 0.0f, 0.0f, 0.0f};
      const float ap[6] = {0.0f, 0.0f, 0.0f, r.abase[0], r.abase[1], r.abase[2]};
      rnea_va(L, L + 9, vp, ap, jt, ax, vq, aq, vn, an);
#pragma unroll
      for (int i = 0; i < 6; ++i) XF[i] = 0.0f;
    }
#pragma unroll
    for (int i = 0; i < 12; ++i) cW[i] = Wn[i];
#pragma unroll
    for (int i = 0; i < 6; ++i) {
      cv[i] = vn[i];
      ca[i] = an[i];
      cFb[i] = fmaf(S[i], tb, XF[i]);
    }
    ctb = tb;
    fresh = true;
    lcs = cs;
    const uint32_t bit = 1u << dep;
    accv &= ~bit;
    replayed = own ? (replayed & ~bit) : (replayed | bit);
    if (nch > 0) stk[dep].tb = tb;
    if (own && A.g_fext) {  // dL/df_ext,k = -Fbar_k
      float* o = A.g_fext + (b * n + k) * 6;
#pragma unroll
      for (int i = 0; i < 6; ++i) o[i] = -cFb[i];
    }
  };

  int sp = 0;
  if (sg.p0 > 0) {  // replay the proper ancestors of the first link
    const int k0 = __ldg(r.dfs + sg.p0).x;
    const int c0 = __ldg(r.chain_start + k0), c1 = __ldg(r.chain_start + k0 + 1);
    for (int c = c0; c < c1 - 1; ++c) {
      const int a = __ldg(r.chain + c);
      push(a, c - c0, false, packed_link(r, a), __ldg(r.chain_start + a));
    }
    sp = c1 - 1 - c0;
  }
  for (int pos = sg.p0; pos < sg.p1; ++pos) {
    const int2 kd = __ldg(r.dfs_kj + pos);  // link | depth << 8 | chain start << 16, joint word
    const int k = kd.x & 0xFF, dep = (kd.x >> 8) & 0xFF;
    const int2 kn = pos + 1 < sg.p1 ? __ldg(r.dfs_kj + pos + 1) : make_int2(0, 0);
    // L2 prefetch of the next link's joint inputs.  The gradient rows its
    // close reads are not prefetched: measured slower (the humanoid's
    // backward 0.218 -> 0.210 ms without)
    if (pos + 1 < sg.p1) {
      const int jn = (kn.y & 0xFFFF) - 1;
      if (jn >= 0) {
        st.prefetch(jn, true);
        if (A.g_tau) pf(A.g_tau + (int64_t)jn * B + b);
        if (FC) pf(fc.tau + (int64_t)jn * B + b);
      }
    }
    while (sp > dep) close(--sp, dep);
    flush();
    sp = dep + 1;
    // a link closed right after its push (a leaf, or the segment's last
    // link): its rows start on their way now
    if (use_slot && (pos + 1 >= sg.p1 || ((kn.x >> 8) & 0xFF) <= dep)) issue(k);
    push(k, dep, true, kd.y, kd.x >> 16);
  }
  while (sp > 0) close(--sp, 0);
  flush();
  if (pend >= 0) asm volatile("cp.async.wait_group 0;" ::: "memory");
  return cost_part;
}

// the whole sweep of one configuration; with a fused cost it also writes the
// configuration's cost (joint terms, then the collision term)
__device__ __forceinline__ void tree_bwd_one(const DevRobot& r, const BwdArgs& A, int64_t b) {
  tree_bwd_seg<false>(r, A, FusedCost{}, ArrayStates{A.q, A.qd, A.qdd, A.B, b}, b,
                      whole_sweep(r));
}

template <class St>
__device__ __forceinline__ void tree_bwd_cost_one(const DevRobot& r, const BwdArgs& A,
                                                  const FusedCost& fc, const St& st, int64_t b) {
  const float c = tree_bwd_seg<true>(r, A, fc, st, b, whole_sweep(r));
  if (fc.cost) fc.cost[b] = fc.d_min ? fmaf(fc.w, fmaxf(0.0f, -__ldg(fc.d_min + b)), c) : c;
}

}  // namespace wbe
