// k_traj.cu -- the trajectory-optimisation ends of the whole-body evaluation:
// joint states from uniform cubic B-spline control points (Sec. 4,
// Eq. bspline-cubic), the control-point gradient (Eq. backward_grad), and the
// per-configuration cost (torque-limit hinges and the self-collision hinge on
// the worst pair) with its upstream gradients.
//
// Layouts: control points U [n_traj][d][K]; states and their gradients
// joint-major [d][B] with B = n_traj * T, configuration b = traj * T + s.
// Sample s of a trajectory sits at t = s (K-3) / (T-1) in segment units:
// segment k = min(floor(t), K-4), alpha = t - k, window u_k .. u_k+3.  The
// segment comes from integer division of s (K-3) by T-1 (the floor of the
// exact quotient, the same integer a double-precision floor gives, since an
// integer quotient is exact in double and a non-integer one is at least
// 1/(T-1) away from the next integer) and alpha = remainder / (T-1).
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

// one thread per (joint, configuration); b fastest so that stores coalesce
__global__ void __launch_bounds__(256) bspline_fwd_kernel(int64_t n_traj, int d, int K, int T,
                                                          float dt, const float* __restrict__ U,
                                                          float* q, float* qd, float* qdd) {
  const int64_t B = n_traj * T;
  const int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (idx >= B * d) return;
  const int j = (int)(idx / B);
  const int64_t b = idx - (int64_t)j * B;
  const int64_t tr = b / T;
  const int s = (int)(b - tr * T);
  int k;
  float a;
  bs_sample(s, K, T, k, a);
  float Bm[3][4];
  bs_basis(a, dt, Bm);
  const float* u = U + (tr * d + j) * K + k;
  const float u0 = __ldg(u), u1 = __ldg(u + 1), u2 = __ldg(u + 2), u3 = __ldg(u + 3);
  float out[3];
#pragma unroll
  for (int r = 0; r < 3; ++r)
    out[r] = fmaf(Bm[r][3], u3, fmaf(Bm[r][2], u2, fmaf(Bm[r][1], u1, Bm[r][0] * u0)));
  const int64_t o = (int64_t)j * B + b;
  if (q) q[o] = out[0];
  if (qd) qd[o] = out[1];
  if (qdd) qdd[o] = out[2];
}

// One thread per control point (trajectory, joint, k): it sums
// B(alpha_s)^T g_s over the samples of segments k-3 .. k in sample order (no
// atomics, deterministic).  The basis rows and segment of every sample and
// the first sample of every segment are tabled in shared memory per block.
__global__ void __launch_bounds__(256) bspline_bwd_kernel(int64_t n_traj, int d, int K, int T,
                                                          float dt, const float* __restrict__ gq,
                                                          const float* __restrict__ gqd,
                                                          const float* __restrict__ gqdd,
                                                          const float* __restrict__ gqd2,
                                                          const float* __restrict__ gqdd2,
                                                          float* gU) {
  extern __shared__ float tab[];  // [T][12] basis rows, then [K-2] first samples
  int* first = reinterpret_cast<int*>(tab + (size_t)T * 12);
  const int nseg = K - 3;
  for (int s = threadIdx.x; s < T; s += blockDim.x) {
    int k;
    float a;
    bs_sample(s, K, T, k, a);
    float Bm[3][4];
    bs_basis(a, dt, Bm);
#pragma unroll
    for (int r = 0; r < 3; ++r)
#pragma unroll
      for (int l = 0; l < 4; ++l) tab[s * 12 + r * 4 + l] = Bm[r][l];
  }
  // first[m] = first sample of segment m = ceil(m (T-1) / nseg); first[nseg] = T
  for (int m = threadIdx.x; m <= nseg; m += blockDim.x)
    first[m] = m == nseg ? T : (m * (T - 1) + nseg - 1) / nseg;
  __syncthreads();
  const int64_t B = n_traj * T;
  const int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (idx >= n_traj * d * K) return;
  const int64_t tj = idx / K;  // trajectory * d + joint
  const int k = (int)(idx - tj * K);
  const int64_t tr = tj / d;
  const int j = (int)(tj - tr * d);
  const int64_t base = (int64_t)j * B + tr * T;
  const int m0 = max(k - 3, 0), m1 = min(k, nseg - 1);
  float acc = 0.0f;
  if (m0 <= m1) {
    int m = m0;
    for (int s = first[m0]; s < first[m1 + 1]; ++s) {
      while (s >= first[m + 1]) ++m;  // segment of sample s
      const int l = k - m;            // this control point's place in the window
      const float* Bs = tab + s * 12;
      float c = 0.0f;
      if (gq) c = fmaf(Bs[l], __ldg(gq + base + s), c);
      float gv = gqd ? __ldg(gqd + base + s) : 0.0f;  // the two qd gradients add
      if (gqd2) gv += __ldg(gqd2 + base + s);
      c = fmaf(Bs[4 + l], gv, c);
      float ga = gqdd ? __ldg(gqdd + base + s) : 0.0f;
      if (gqdd2) ga += __ldg(gqdd2 + base + s);
      c = fmaf(Bs[8 + l], ga, c);
      acc += c;
    }
  }
  gU[idx] = acc;
}

// One thread per configuration.  The motion terms of the loss (smooth |qdd|^2,
// length |qd|^2, energy ||(qd . tau) dt||^2 with e = energy dt^2) and the
// hinges; g_qd / g_qdd are the cost's direct qd / qdd gradients.
__global__ void __launch_bounds__(256) trajopt_cost_kernel(int64_t B, int d,
                                                           const float* __restrict__ tau,
                                                           const float* __restrict__ d_min,
                                                           const float* __restrict__ qd,
                                                           const float* __restrict__ qdd,
                                                           const float* __restrict__ lo,
                                                           const float* __restrict__ hi,
                                                           float w, float smooth, float length,
                                                           float e, float* cost, float* g_tau,
                                                           float* g_dmin, float* g_qd,
                                                           float* g_qdd) {
  const int64_t b = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (b >= B) return;
  float c = 0.0f;
  // loads issued eight joints at a time so that their latencies overlap
  for (int j0 = 0; j0 < d; j0 += 8) {
    float t[8], v[8], a[8];
#pragma unroll
    for (int u = 0; u < 8; ++u) {
      const int64_t at = (int64_t)(j0 + u) * B + b;
      const bool in = j0 + u < d;
      t[u] = in && tau ? __ldg(tau + at) : 0.0f;
      v[u] = in && qd ? __ldg(qd + at) : 0.0f;
      a[u] = in && qdd ? __ldg(qdd + at) : 0.0f;
    }
#pragma unroll
    for (int u = 0; u < 8; ++u) {
      const int j = j0 + u;
      if (j >= d) break;
      const int64_t at = (int64_t)j * B + b;
      const float vt = v[u] * t[u];
      c = fmaf(smooth * a[u], a[u], c);
      c = fmaf(length * v[u], v[u], c);
      c = fmaf(e * vt, vt, c);
      float gt = 2.0f * e * v[u] * vt;
      if (tau) {
        const float l = __ldg(lo + j), h = __ldg(hi + j);
        c += fmaxf(0.0f, t[u] - h) + fmaxf(0.0f, l - t[u]);
        gt += (t[u] > h ? 1.0f : 0.0f) - (t[u] < l ? 1.0f : 0.0f);
      }
      if (g_tau) g_tau[at] = gt;
      if (g_qd) g_qd[at] = 2.0f * (length * v[u] + e * vt * t[u]);
      if (g_qdd) g_qdd[at] = 2.0f * smooth * a[u];
    }
  }
  if (d_min) {
    const float dm = __ldg(d_min + b);
    c = fmaf(w, fmaxf(0.0f, -dm), c);
    if (g_dmin) g_dmin[b] = dm < 0.0f ? -w : 0.0f;
  }
  if (cost) cost[b] = c;
}

// ---------------------------------------------------------------------------
// launchers
// ---------------------------------------------------------------------------
cudaError_t launch_bspline_fwd(int64_t n_traj, int d, int K, int T, float dt, const float* U,
                               float* q, float* qd, float* qdd, cudaStream_t s) {
  const int64_t n = n_traj * T * d;
  bspline_fwd_kernel<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(n_traj, d, K, T, dt, U, q, qd,
                                                                 qdd);
  return cudaGetLastError();
}

size_t bspline_bwd_smem(int K, int T) {
  return sizeof(float) * (size_t)T * 12 + sizeof(int) * (size_t)(K - 2);
}

cudaError_t launch_bspline_bwd(int64_t n_traj, int d, int K, int T, float dt, const float* gq,
                               const float* gqd, const float* gqdd, const float* gqd2,
                               const float* gqdd2, float* gU, cudaStream_t s) {
  const size_t smem = bspline_bwd_smem(K, T);
  cudaError_t e = cudaFuncSetAttribute(bspline_bwd_kernel,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  const int64_t n = n_traj * d * K;
  bspline_bwd_kernel<<<(unsigned)((n + 255) / 256), 256, smem, s>>>(n_traj, d, K, T, dt, gq, gqd,
                                                                   gqdd, gqd2, gqdd2, gU);
  return cudaGetLastError();
}

cudaError_t launch_trajopt_cost(int64_t B, int d, const float* tau, const float* d_min,
                                const float* qd, const float* qdd, const float* lo,
                                const float* hi, float w, float smooth, float length, float e,
                                float* cost, float* g_tau, float* g_dmin, float* g_qd,
                                float* g_qdd, cudaStream_t s) {
  trajopt_cost_kernel<<<(unsigned)((B + 255) / 256), 256, 0, s>>>(
      B, d, tau, d_min, qd, qdd, lo, hi, w, smooth, length, e, cost, g_tau, g_dmin, g_qd, g_qdd);
  return cudaGetLastError();
}

}  // namespace wbe
