// spatial.cuh -- compact spatial algebra on the device (Sec. 6.3, "Compact
// spatial representations", Tab. rnea_comparison).
//
// A link transform is a rotation R (row-major 3x3, child axes in parent
// coordinates) and a translation p (child origin in parent coordinates): 12
// floats instead of a 6x6 Plucker matrix.  Spatial vectors are [angular;
// linear] about the frame origin.
//   motion, parent -> child:  X m = [R^T w ; R^T (u + w x p)]
//   force,  child -> parent:  X^T f = [R n + p x (R f) ; R f]
// A spatial inertia is 10 floats (m, h = m c, Io = inertia about the link
// origin): I v = [Io w + h x u ; m u - h x w].
#pragma once

#include "wbe_internal.h"

namespace wbe {

__device__ __forceinline__ void cross3(const float* a, const float* b, float* c) {
  c[0] = fmaf(a[1], b[2], -a[2] * b[1]);
  c[1] = fmaf(a[2], b[0], -a[0] * b[2]);
  c[2] = fmaf(a[0], b[1], -a[1] * b[0]);
}

__device__ __forceinline__ float dot3(const float* a, const float* b) {
  return fmaf(a[2], b[2], fmaf(a[1], b[1], a[0] * b[0]));
}

// y = R x
__device__ __forceinline__ void rot(const float* R, const float* x, float* y) {
  y[0] = fmaf(R[2], x[2], fmaf(R[1], x[1], R[0] * x[0]));
  y[1] = fmaf(R[5], x[2], fmaf(R[4], x[1], R[3] * x[0]));
  y[2] = fmaf(R[8], x[2], fmaf(R[7], x[1], R[6] * x[0]));
}

// y = R^T x
__device__ __forceinline__ void rotT(const float* R, const float* x, float* y) {
  y[0] = fmaf(R[6], x[2], fmaf(R[3], x[1], R[0] * x[0]));
  y[1] = fmaf(R[7], x[2], fmaf(R[4], x[1], R[1] * x[0]));
  y[2] = fmaf(R[8], x[2], fmaf(R[5], x[1], R[2] * x[0]));
}

// C = A B (3x3 row-major)
__device__ __forceinline__ void matmul3(const float* A, const float* B, float* C) {
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = 0; j < 3; ++j)
      C[3 * i + j] = fmaf(A[3 * i + 2], B[6 + j], fmaf(A[3 * i + 1], B[3 + j], A[3 * i] * B[j]));
}

// Robot parameters (fixed transforms, axes, mimic factors, inertias) are read
// with plain loads, not __ldg: the segmented backward sweeps stage them in
// shared memory and hand the sweep pointers into it.
template <class T>
__device__ __forceinline__ T ldp(const T* p) {
  return *p;
}

__device__ __forceinline__ float joint_var(const DevRobot& r, int k, float qj) {
  const float2 mm = reinterpret_cast<const float2*>(r.mimic)[k];
  return fmaf(mm.x, qj, mm.y);
}

// sin and cos of a joint angle: Cody and Waite's reduction (1980) of th to
// x = th - k 2 pi, k = rint(th / 2 pi), with 2 pi split as 6.28125 (8
// significant bits, so k * 6.28125 and th - k * 6.28125 are exact for
// |k| < 2^16) plus 1.93530718e-3 (the split's residual is 1.03e-11 per
// multiple of 2 pi), then CUDA's fast intrinsic on x in [-pi, pi], where
// its absolute error is at most 2^-21.41.  Overall within about 5e-7 of the
// exact sine and cosine of the float angle for |th| <= 4e4 rad (tested
// against double precision), a few times the rounding of a float sine; the
// sweeps evaluate it at every push and close, where the library sincosf's
// longer dependency chain cost 3 % (forward) and 5 % (backward) of the
// humanoid's sweep time.
__device__ __forceinline__ void joint_sincos(float th, float* s, float* c) {
  const float k = rintf(th * 0.159154943f);
  float x = fmaf(-k, 6.28125f, th);
  x = fmaf(-k, 1.93530718e-3f, x);
  __sincosf(x, s, c);
}

// Local transform of link k (parent joint frame -> link frame) for joint
// variable th: T_fixed * J(th).  Revolute: R = R_f R_J(th) with Rodrigues'
// rotation R_J = c I + s [a]^ + (1-c) a a^T.  Prismatic: p = p_f + R_f a th.
// (jt, ident: the link's joint type and whether its fixed rotation is the
// identity, from a packed table the caller holds)
__device__ __forceinline__ void local_xf_m(const DevRobot& r, int k, float th, int jt, bool ident,
                                           float* R, float* p) {
  const float4* T4 = reinterpret_cast<const float4*>(r.Tf + 12 * k);
  const float4 t0 = ldp(T4), t1 = ldp(T4 + 1), t2 = ldp(T4 + 2);
  const float Rf[9] = {t0.x, t0.y, t0.z, t0.w, t1.x, t1.y, t1.z, t1.w, t2.x};
  p[0] = t2.y;
  p[1] = t2.z;
  p[2] = t2.w;
  if (jt == 1) {
    const float4 a = ldp(reinterpret_cast<const float4*>(r.axis) + k);
    float s, c;
    joint_sincos(th, &s, &c);
    const float t = 1.0f - c;
    const float tx = t * a.x, ty = t * a.y, tz = t * a.z;
    const float sx = s * a.x, sy = s * a.y, sz = s * a.z;
    float Rj[9];
    Rj[0] = fmaf(tx, a.x, c);
    Rj[1] = fmaf(tx, a.y, -sz);
    Rj[2] = fmaf(tx, a.z, sy);
    Rj[3] = fmaf(ty, a.x, sz);
    Rj[4] = fmaf(ty, a.y, c);
    Rj[5] = fmaf(ty, a.z, -sx);
    Rj[6] = fmaf(tz, a.x, -sy);
    Rj[7] = fmaf(tz, a.y, sx);
    Rj[8] = fmaf(tz, a.z, c);
    if (ident) {
#pragma unroll
      for (int i = 0; i < 9; ++i) R[i] = Rj[i];
    } else {
      matmul3(Rf, Rj, R);
    }
  } else {
#pragma unroll
    for (int i = 0; i < 9; ++i) R[i] = Rf[i];
    if (jt == 2) {
      const float4 a = ldp(reinterpret_cast<const float4*>(r.axis) + k);
      const float s[3] = {a.x * th, a.y * th, a.z * th};
      float Rs[3];
      rot(Rf, s, Rs);
      p[0] += Rs[0];
      p[1] += Rs[1];
      p[2] += Rs[2];
    }
  }
}

__device__ __forceinline__ void local_xf(const DevRobot& r, int k, float th, float* R, float* p) {
  local_xf_m(r, k, th, __ldg(r.jtype + k), __ldg(r.rot_id + k) != 0, R, p);
}

// motion vector m (parent coords) -> child coords
__device__ __forceinline__ void xf_motion(const float* R, const float* p, const float* m,
                                          float* out) {
  float wxp[3], t[3];
  cross3(m, p, wxp);
  t[0] = m[3] + wxp[0];
  t[1] = m[4] + wxp[1];
  t[2] = m[5] + wxp[2];
  rotT(R, m, out);
  rotT(R, t, out + 3);
}

// motion vector m (child coords) -> parent coords, the inverse of xf_motion:
// X^-1 [w; u] = [R w ; R u + p x (R w)]
__device__ __forceinline__ void xf_motion_inv(const float* R, const float* p, const float* m,
                                              float* out) {
  float pxw[3];
  rot(R, m, out);
  rot(R, m + 3, out + 3);
  cross3(p, out, pxw);
  out[3] += pxw[0];
  out[4] += pxw[1];
  out[5] += pxw[2];
}

// force vector f (child coords) -> parent coords (X^T f); the same map
// carries adjoints of motion vectors back to the parent.
__device__ __forceinline__ void xf_force_T(const float* R, const float* p, const float* f,
                                           float* out) {
  float Rn[3], pxRf[3];
  rot(R, f + 3, out + 3);
  rot(R, f, Rn);
  cross3(p, out + 3, pxRf);
  out[0] = Rn[0] + pxRf[0];
  out[1] = Rn[1] + pxRf[1];
  out[2] = Rn[2] + pxRf[2];
}

// crm(v) m = [w x mw ; u x mw + w x mu]
__device__ __forceinline__ void crm(const float* v, const float* m, float* out) {
  float a[3], b[3];
  cross3(v, m, out);
  cross3(v + 3, m, a);
  cross3(v, m + 3, b);
  out[3] = a[0] + b[0];
  out[4] = a[1] + b[1];
  out[5] = a[2] + b[2];
}

// crf(v) f = [w x fn + u x ff ; w x ff]
__device__ __forceinline__ void crf(const float* v, const float* f, float* out) {
  float a[3], b[3];
  cross3(v, f, a);
  cross3(v + 3, f + 3, b);
  out[0] = a[0] + b[0];
  out[1] = a[1] + b[1];
  out[2] = a[2] + b[2];
  cross3(v, f + 3, out + 3);
}

// I v for the compact inertia {m, h[3], Io[6] = xx yy zz xy xz yz}
__device__ __forceinline__ void inertia_mul(const float* I, const float* v, float* out) {
  const float m = I[0];
  const float h[3] = {I[1], I[2], I[3]};
  const float* w = v;
  const float* u = v + 3;
  float hxu[3], hxw[3];
  cross3(h, u, hxu);
  cross3(h, w, hxw);
  out[0] = fmaf(I[4], w[0], fmaf(I[7], w[1], fmaf(I[8], w[2], hxu[0])));
  out[1] = fmaf(I[7], w[0], fmaf(I[5], w[1], fmaf(I[9], w[2], hxu[1])));
  out[2] = fmaf(I[8], w[0], fmaf(I[9], w[1], fmaf(I[6], w[2], hxu[2])));
  out[3] = fmaf(m, u[0], -hxw[0]);
  out[4] = fmaf(m, u[1], -hxw[1]);
  out[5] = fmaf(m, u[2], -hxw[2]);
}

__device__ __forceinline__ void load_inertia(const DevRobot& r, int k, float* I) {
  const float* src = r.inert + 10 * k;
#pragma unroll
  for (int i = 0; i < 10; ++i) I[i] = ldp(src + i);
}

// Joint motion subspace S of link k as (jt, axis): revolute [a;0],
// prismatic [0;a], fixed 0.  Helpers for S^T x and S * s.
__device__ __forceinline__ float St_dot(int jt, const float* a, const float* x) {
  return jt == 1 ? dot3(a, x) : (jt == 2 ? dot3(a, x + 3) : 0.0f);
}

// RNEA forward sweep for one link (Alg. 4, pass 1): given the parent's
// velocity/acceleration (parent coords), the local transform and the joint
// rates, produce v_k and a_k in link coordinates:
//   v = X v_pa + S qd ;  a = X a_pa + S qdd + v x_m (S qd)
__device__ __forceinline__ void rnea_va(const float* R, const float* p, const float* vpa,
                                        const float* apa, int jt, const float* ax, float qd,
                                        float qdd, float* v, float* a) {
  xf_motion(R, p, vpa, v);
  xf_motion(R, p, apa, a);
  if (jt == 1) {
    const float s[3] = {ax[0] * qd, ax[1] * qd, ax[2] * qd};
    v[0] += s[0];
    v[1] += s[1];
    v[2] += s[2];
    float wxs[3], uxs[3];
    cross3(v, s, wxs);
    cross3(v + 3, s, uxs);
    a[0] += fmaf(ax[0], qdd, wxs[0]);
    a[1] += fmaf(ax[1], qdd, wxs[1]);
    a[2] += fmaf(ax[2], qdd, wxs[2]);
    a[3] += uxs[0];
    a[4] += uxs[1];
    a[5] += uxs[2];
  } else if (jt == 2) {
    const float s[3] = {ax[0] * qd, ax[1] * qd, ax[2] * qd};
    v[3] += s[0];
    v[4] += s[1];
    v[5] += s[2];
    float wxs[3];
    cross3(v, s, wxs);
    a[3] += fmaf(ax[0], qdd, wxs[0]);
    a[4] += fmaf(ax[1], qdd, wxs[1]);
    a[5] += fmaf(ax[2], qdd, wxs[2]);
  }
}

// Alg. 4, pass 2: f = I a + v x* (I v)
__device__ __forceinline__ void rnea_force(const float* I, const float* v, const float* a,
                                           float* f) {
  float Ia[6], Iv[6], c[6];
  inertia_mul(I, a, Ia);
  inertia_mul(I, v, Iv);
  crf(v, Iv, c);
#pragma unroll
  for (int i = 0; i < 6; ++i) f[i] = Ia[i] + c[i];
}

// Squared centre distance with a fixed operation order, shared by the fast
// filter and the exact path of the pair stage.
__device__ __forceinline__ float dist2(float xi, float yi, float zi, float xj, float yj,
                                       float zj) {
  const float dx = xi - xj, dy = yi - yj, dz = zi - zj;
  return fmaf(dz, dz, fmaf(dy, dy, dx * dx));
}

}  // namespace wbe
