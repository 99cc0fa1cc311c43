// spline_basis.cuh -- the sample layout and basis rows of the uniform cubic
// B-spline (Sec. 4, Eq. bspline-cubic), shared by the B-spline kernels
// (k_traj.cu) and the sweeps that evaluate the states from control points
// (tree_sweep.cuh), so that both give the same bits.
//
// Sample s of a trajectory sits at t = s (K-3) / (T-1) in segment units:
// segment k = min(floor(t), K-4), alpha = t - k, window u_k .. u_k+3.  The
// segment comes from integer division of s (K-3) by T-1 (the floor of the
// exact quotient) and alpha = remainder / (T-1).
#pragma once

#include "wbe_internal.h"

namespace wbe {

__device__ __forceinline__ void bs_sample(int s, int K, int T, int& k, float& al) {
  const int nseg = K - 3;
  const int num = s * nseg;
  int kk = num / (T - 1);
  if (kk > nseg - 1) kk = nseg - 1;
  k = kk;
  al = (float)(num - kk * (T - 1)) / (float)(T - 1);
}

// rows of B(alpha) = T P(alpha) C for theta, theta_dot, theta_ddot, with
// C = (1/6) [[-1, 3, -3, 1], [3, -6, 3, 0], [-3, 0, 3, 0], [1, 4, 1, 0]]
__device__ __forceinline__ void bs_basis(float a, float dt, float Bm[3][4]) {
  const float idt = 1.0f / dt;
  const float P[3][4] = {{a * a * a, a * a, a, 1.0f},
                         {3.0f * a * a * idt, 2.0f * a * idt, idt, 0.0f},
                         {6.0f * a * idt * idt, 2.0f * idt * idt, 0.0f, 0.0f}};
  const float c = 1.0f / 6.0f;
#pragma unroll
  for (int r = 0; r < 3; ++r) {
    const float* p = P[r];
    Bm[r][0] = c * (-p[0] + 3.0f * p[1] - 3.0f * p[2] + p[3]);
    Bm[r][1] = c * (3.0f * p[0] - 6.0f * p[1] + 4.0f * p[3]);
    Bm[r][2] = c * (-3.0f * p[0] + 3.0f * p[1] + 3.0f * p[2] + p[3]);
    Bm[r][3] = c * p[0];
  }
}

// q, qd, qdd of one sample from its window's four control points
__device__ __forceinline__ float bs_row(const float* B4, float u0, float u1, float u2, float u3) {
  return fmaf(B4[3], u3, fmaf(B4[2], u2, fmaf(B4[1], u1, B4[0] * u0)));
}

}  // namespace wbe
